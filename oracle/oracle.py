"""ctypes front end of the FP64 CPU oracle (scbb_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's CPU-baseline and
reference legs.  The product path (the CUDA library and its binding) never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_scbb.so")
_SRC = [os.path.join(_HERE, "scbb_oracle.c"), os.path.join(_HERE, "scbb_oracle_bb.c")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, OpenMP over lattice nodes)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
               "-o", tmp, _SRC[0], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class o_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("walls", C.c_int),
                ("u_lo", C.c_double * 3), ("u_hi", C.c_double * 3),
                ("tau", C.c_double), ("G", C.c_double), ("psi_kind", C.c_int),
                ("g", C.c_double * 3), ("coupling", C.c_int),
                ("rho_maj", C.c_double), ("rho_min", C.c_double), ("C0", C.c_double),
                ("mass_correction", C.c_int), ("pp_eps", C.c_double), ("pp_d0", C.c_double),
                ("wall_kind", C.c_int)]


class o_mesh_params(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("kS", C.c_double), ("C", C.c_double),
                ("kB", C.c_double), ("kV", C.c_double), ("mass", C.c_double), ("colour", C.c_double)]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.o_create.restype = C.c_void_p
        L.o_create.argtypes = [C.POINTER(o_params), C.c_int, C.POINTER(o_mesh_params), C.c_void_p,
                               C.c_void_p, C.c_void_p]
        L.o_destroy.argtypes = [C.c_void_p]
        L.o_set_state.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p]
        L.o_init.argtypes = [C.c_void_p]
        L.o_step.argtypes = [C.c_void_p, C.c_int]
        L.o_get_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.o_get_f.argtypes = [C.c_void_p, _dp]
        L.o_set_f.argtypes = [C.c_void_p, _dp]
        L.o_get_fsc.argtypes = [C.c_void_p, _dp]
        L.o_mass.argtypes = [C.c_void_p, C.c_int]
        L.o_mass.restype = C.c_double
        L.o_momentum.argtypes = [C.c_void_p, _dp]
        L.o_get_vertices.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.o_set_vertices.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.o_set_elem_colour.restype = None
        L.o_set_elem_colour.argtypes = [C.c_void_p, _dp]
        L.o_get_owner.argtypes = [C.c_void_p, _u16p]
        L.o_capsule_diag.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), _dp]
        L.o_skalak.restype = C.c_double
        L.o_skalak.argtypes = [C.c_int, C.c_int, _dp, _ip, _dp, C.c_double, C.c_double, C.c_void_p]
        L.o_volume.restype = C.c_double
        L.o_volume.argtypes = [C.c_int, C.c_int, _dp, _ip]
        L.o_volume_force.restype = C.c_double
        L.o_volume_force.argtypes = [C.c_int, C.c_int, _dp, _ip, C.c_double, C.c_double, C.c_void_p]
        L.o_bending.restype = C.c_double
        L.o_bending.argtypes = [C.c_int, C.c_int, _dp, _ip, C.c_double] + [C.c_void_p] * 6
        L.o_pp_forces.argtypes = [C.c_int, _dp, _ip, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                  C.c_int, _dp]
        L.o_ibm_spread_field.argtypes = [C.c_void_p, _dp, _dp]
        L.o_ibm_interp.argtypes = [C.c_void_p, _dp, _dp]
        L.o_feq.restype = C.c_double
        L.o_feq.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.o_fresh_count.restype = C.c_long
        L.o_fresh_count.argtypes = [C.c_void_p]
        L.o_fresh_fallbacks.restype = C.c_long
        L.o_fresh_fallbacks.argtypes = [C.c_void_p]
        L.o_get_owner_old.argtypes = [C.c_void_p, _u16p]
        L.o_set_owner.argtypes = [C.c_void_p, _u16p]
        L.o_crossed_element.restype = C.c_int
        L.o_crossed_element.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_int]
        L.o_inside.restype = C.c_int
        L.o_inside.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.o_classify.argtypes = [C.c_void_p]
        L.o_get_elem_acc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.o_element_fallbacks.restype = C.c_long
        L.o_element_fallbacks.argtypes = [C.c_void_p]
        L.o_boundary_count.restype = C.c_long
        L.o_boundary_count.argtypes = [C.c_void_p]
        L.o_num_threads.restype = C.c_int
        L.o_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------------------------------------------
# Membrane functions (Sec. II.B) on one mesh
# ------------------------------------------------------------------------------------------------------
def skalak(x, tri, ref, kS, C_):
    x = np.ascontiguousarray(x, np.float64)
    F = np.zeros_like(x)
    E = lib().o_skalak(len(x), len(tri), x, np.ascontiguousarray(tri, np.int32),
                       np.ascontiguousarray(ref, np.float64), kS, C_, _ptr(F))
    return E, F


def volume(x, tri):
    return lib().o_volume(len(x), len(tri), np.ascontiguousarray(x, np.float64),
                          np.ascontiguousarray(tri, np.int32))


def volume_force(x, tri, kV, V0):
    x = np.ascontiguousarray(x, np.float64)
    F = np.zeros_like(x)
    E = lib().o_volume_force(len(x), len(tri), x, np.ascontiguousarray(tri, np.int32), kV, V0, _ptr(F))
    return E, F


def bending(x, tri, kB):
    x = np.ascontiguousarray(x, np.float64)
    nv = len(x)
    F = np.zeros_like(x)
    H, KG, A, LH = (np.zeros(nv) for _ in range(4))
    n = np.zeros_like(x)
    E = lib().o_bending(nv, len(tri), x, np.ascontiguousarray(tri, np.int32), kB, _ptr(F), _ptr(H),
                        _ptr(KG), _ptr(A), _ptr(LH), _ptr(n))
    return dict(E=E, F=F, H=H, KG=KG, A=A, LH=LH, n=n)


def pp_forces(X, cap_of, eps, d0, nx, ny, nz, periodic_z):
    X = np.ascontiguousarray(X, np.float64)
    F = np.zeros_like(X)
    lib().o_pp_forces(len(X), X, np.ascontiguousarray(cap_of, np.int32), eps, d0, nx, ny, nz,
                      int(periodic_z), F)
    return F


def feq(i, rho, u):
    return lib().o_feq(i, rho, u[0], u[1], u[2])


def d3q19():
    cx = (C.c_int * 19)(); cy = (C.c_int * 19)(); cz = (C.c_int * 19)()
    w = (C.c_double * 19)(); opp = (C.c_int * 19)()
    lib().o_d3q19(cx, cy, cz, w, opp)
    return np.array([list(cx), list(cy), list(cz)]).T, np.array(list(w)), np.array(list(opp))


# ------------------------------------------------------------------------------------------------------
# Simulation object
# ------------------------------------------------------------------------------------------------------
class OracleSim:
    """The oracle's full time step on a Problem from paper_1904_11386_gb300.inputs."""

    def __init__(self, prob, rhoA=None, rhoB=None, u=None):
        L = lib()
        self.prob = prob
        p = o_params()
        p.nx, p.ny, p.nz, p.walls = prob.nx, prob.ny, prob.nz, int(prob.walls)
        p.u_lo = (C.c_double * 3)(*prob.u_lo)
        p.u_hi = (C.c_double * 3)(*prob.u_hi)
        p.tau, p.G, p.psi_kind = prob.tau, prob.G, prob.psi_kind
        p.g = (C.c_double * 3)(*prob.g)
        p.coupling = prob.coupling if prob.capsules else 2
        p.rho_maj, p.rho_min, p.C0 = prob.rho_maj, prob.rho_min, prob.C0
        p.mass_correction = int(prob.mass_correction)
        p.pp_eps, p.pp_d0 = prob.pp_eps, prob.pp_d0
        p.wall_kind = int(getattr(prob, "wall_kind", 0))
        self.p = p
        nm = len(prob.capsules)
        mps = (o_mesh_params * max(nm, 1))()
        tris, refs, inits = [], [], []
        for k, cap in enumerate(prob.capsules):
            ref, tri, init = cap.mesh()
            mps[k].nv, mps[k].nt = len(ref), len(tri)
            mps[k].kS, mps[k].C, mps[k].kB, mps[k].kV = cap.kS, cap.C, cap.kB, cap.kV
            mps[k].mass, mps[k].colour = cap.mass, cap.colour
            tris.append(tri); refs.append(ref); inits.append(init)
        self.nm = nm
        self.nv = [len(r) for r in refs]
        self.tris = tris
        tri_all = np.ascontiguousarray(np.concatenate(tris) if tris else np.zeros((1, 3), np.int32), np.int32)
        ref_all = np.ascontiguousarray(np.concatenate(refs) if refs else np.zeros((1, 3)), np.float64)
        init_all = np.ascontiguousarray(np.concatenate(inits) if inits else np.zeros((1, 3)), np.float64)
        self._keep = (mps, tri_all, ref_all, init_all)
        self.h = L.o_create(C.byref(p), nm, mps, _ptr(tri_all), _ptr(ref_all), _ptr(init_all))
        if any(getattr(cap, "elem_colour", None) is not None for cap in prob.capsules):
            # per-element colours (Sec. V), a capsule without them keeps its uniform colour on every element
            ecol = np.concatenate([np.full(len(t), cap.colour) if cap.elem_colour is None
                                   else np.asarray(cap.elem_colour, np.float64) for cap, t in zip(prob.capsules, tris)])
            self._ecol = np.ascontiguousarray(ecol, np.float64)
            L.o_set_elem_colour(self.h, self._ecol)
        if rhoA is None:
            rhoA, rhoB = prob.initial_density()
        L.o_set_state(self.h, np.ascontiguousarray(rhoA.ravel(), np.float64),
                      np.ascontiguousarray(rhoB.ravel(), np.float64),
                      _ptr(None if u is None else np.ascontiguousarray(u.reshape(3, -1), np.float64)))
        L.o_init(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().o_destroy(self.h)
            self.h = None

    @property
    def N(self):
        return self.prob.n_nodes

    def step(self, n=1):
        lib().o_step(self.h, int(n))

    def fields(self):
        s = (self.prob.nz, self.prob.ny, self.prob.nx)
        a, b, u = np.zeros(self.N), np.zeros(self.N), np.zeros(3 * self.N)
        lib().o_get_fields(self.h, _ptr(a), _ptr(b), _ptr(u))
        return a.reshape(s), b.reshape(s), u.reshape((3,) + s)

    def populations(self):
        f = np.zeros(2 * self.N * 19)
        lib().o_get_f(self.h, f)
        return f.reshape(2, self.N, 19)

    def set_populations(self, f):
        lib().o_set_f(self.h, np.ascontiguousarray(f, np.float64).ravel())

    def sc_force(self):
        f = np.zeros(6 * self.N)
        lib().o_get_fsc(self.h, f)
        return f.reshape(2, 3, self.prob.nz, self.prob.ny, self.prob.nx)

    def mass(self, c):
        return lib().o_mass(self.h, c)

    def momentum(self):
        m = np.zeros(3)
        lib().o_momentum(self.h, m)
        return m

    def vertices(self):
        NV = sum(self.nv)
        X, V, F = np.zeros(3 * NV), np.zeros(3 * NV), np.zeros(3 * NV)
        lib().o_get_vertices(self.h, _ptr(X), _ptr(V), _ptr(F))
        return X.reshape(NV, 3), V.reshape(NV, 3), F.reshape(NV, 3)

    def set_vertices(self, X=None, V=None):
        lib().o_set_vertices(self.h, _ptr(None if X is None else np.ascontiguousarray(X, np.float64)),
                             _ptr(None if V is None else np.ascontiguousarray(V, np.float64)))

    def owner(self):
        o = np.zeros(self.N, np.uint16)
        lib().o_get_owner(self.h, o)
        return o.reshape(self.prob.nz, self.prob.ny, self.prob.nx)

    def fresh_count(self):
        return lib().o_fresh_count(self.h), lib().o_fresh_fallbacks(self.h)

    def boundary_count(self):
        return lib().o_boundary_count(self.h), lib().o_element_fallbacks(self.h)

    def crossed_element(self, cap, node, i):
        return lib().o_crossed_element(self.h, cap, node, i)

    def inside(self, cap, x, y, z):
        return lib().o_inside(self.h, cap, x, y, z)

    def elem_acc(self):
        NT = sum(len(t) for t in self.tris)
        now, prev, pend = np.zeros(3 * NT), np.zeros(3 * NT), np.zeros(3 * NT)
        lib().o_get_elem_acc(self.h, _ptr(now), _ptr(prev), _ptr(pend))
        return now.reshape(NT, 3), prev.reshape(NT, 3), pend.reshape(NT, 3)

    def capsule(self, m):
        v = C.c_double(0)
        c = np.zeros(3)
        lib().o_capsule_diag(self.h, m, C.byref(v), c)
        return v.value, c

    def ibm_spread(self, Fb):
        out = np.zeros(3 * self.N)
        lib().o_ibm_spread_field(self.h, np.ascontiguousarray(Fb, np.float64).ravel(), out)
        return out.reshape(3, self.prob.nz, self.prob.ny, self.prob.nx)

    def ibm_interp(self, field):
        NV = sum(self.nv)
        out = np.zeros(3 * NV)
        lib().o_ibm_interp(self.h, np.ascontiguousarray(field, np.float64).ravel(), out)
        return out.reshape(NV, 3)


def threads():
    return lib().o_num_threads()


def set_threads(n):
    lib().o_set_threads(int(n))


# ------------------------------------------------------------------------------------------------------
# Membrane-only reference model of Sec. III.B (Eq. emulatetension): no fluid; the fluid-fluid interface is
# emulated by a tensile force on the elements that lie in a band of width w around a fixed interface plane.
# ------------------------------------------------------------------------------------------------------
def _area_below(z, A, h):
    """Area of each planar triangle (vertex heights z [T, 3], areas A [T]) below the plane z = h.  The
    cross-section of a triangle at height t is a segment whose length is piecewise linear in t, so the area
    below h is piecewise quadratic: with sorted heights z1 <= z2 <= z3 it is A (h - z1)^2 / ((z2 - z1)(z3 - z1))
    up to z2 and A [1 - (z3 - h)^2 / ((z3 - z2)(z3 - z1))] above."""
    zs = np.sort(z, axis=1)
    z1, z2, z3 = zs[:, 0], zs[:, 1], zs[:, 2]
    d31 = np.maximum(z3 - z1, 1e-300)
    lo = A * np.clip(h - z1, 0, None) ** 2 / (np.maximum(z2 - z1, 1e-300) * d31)
    hi = A * (1.0 - np.clip(z3 - h, 0, None) ** 2 / (np.maximum(z3 - z2, 1e-300) * d31))
    out = np.where(h <= z1, 0.0, np.where(h >= z3, A, np.where(h <= z2, lo, hi)))
    return out


def emulated_tension(x, tri, z_int, gamma, w=1.0):
    """Node forces of the emulated interface (Eq. emulatetension): an element whose area A lies within w/2 of
    the plane z = z_int gets F = gamma A / w, spread evenly over its three nodes.  Reading (the paper states the
    magnitude, not the direction): the interface pulls the membrane in its own plane, radially outward from the
    capsule's vertical axis through its centre of mass, taken at the element's centroid."""
    x = np.asarray(x, np.float64)
    tri = np.asarray(tri)
    p = x[tri]                                            # [T, 3 corners, 3]
    A = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    z = p[:, :, 2]
    band = _area_below(z, A, z_int + 0.5 * w) - _area_below(z, A, z_int - 0.5 * w)
    axis = x[:, :2].mean(0)
    radial = p.mean(1)[:, :2] - axis
    rn = np.linalg.norm(radial, axis=1)
    dirn = np.zeros((len(tri), 3))
    ok = rn > 0
    dirn[ok, :2] = radial[ok] / rn[ok, None]
    Fe = (gamma * band / w)[:, None] * dirn
    F = np.zeros_like(x)
    for k in range(3):
        np.add.at(F, tri[:, k], Fe / 3.0)
    return F


def reference_model(ref, tri, kS, C_, kB, kV, z_int, gamma, w=1.0, mass=5.0, damping=0.05, steps=4000,
                    x0=None):
    """The membrane-only reference model of Sec. III.B: the same elastic laws (Skalak, volume, bending; Sec.
    II.B) and the same symplectic node update as the coupled method (V += F / m, X += V), with the emulated
    interface tension in place of the fluid.  Reading: the fluid's dissipation is replaced by a velocity damping
    (V *= 1 - damping each step), which does not change the static equilibrium the model is used for.
    Returns the final positions and the largest node force of the last step (the equilibrium residual)."""
    ref = np.asarray(ref, np.float64)
    tri = np.asarray(tri, np.int32)
    X = (ref if x0 is None else np.asarray(x0, np.float64)).copy()
    V = np.zeros_like(X)
    V0 = volume(ref, tri)
    F = np.zeros_like(X)
    for _ in range(steps):
        F = skalak(X, tri, ref, kS, C_)[1] + volume_force(X, tri, kV, V0)[1] + emulated_tension(X, tri, z_int,
                                                                                                  gamma, w)
        if kB:
            F += bending(X, tri, kB)["F"]
        V = (1.0 - damping) * V + F / mass
        X = X + V
    return X, np.abs(F).max()

"""Python binding of libscbb (include/scbb.h): argument marshalling only.

Every step of the simulation runs in the CUDA kernels of libscbb.so.  PyTorch supplies the device workspace
and the stream.  There is no CPU fallback: if the library or a CUDA device is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libscbb.so")

SCBB_OK = 0
STATUS = {0: "SCBB_OK", 1: "SCBB_E_INVAL", 2: "SCBB_E_CUDA", 3: "SCBB_E_NOMEM", 4: "SCBB_E_UNSTABLE",
          5: "SCBB_E_TIMEOUT", 6: "SCBB_E_MESH", 7: "SCBB_E_STATE", 8: "SCBB_E_UNSUPPORTED"}

EXPORTS = ["scbb_workspace_bytes", "scbb_create", "scbb_set_density", "scbb_step", "scbb_sync",
           "scbb_get_fields", "scbb_get_populations", "scbb_get_vertices", "scbb_get_diag", "scbb_get_owner",
           "scbb_get_boundary",
           "scbb_launch_count", "scbb_enable_timing", "scbb_kernel_time", "scbb_phase_times", "scbb_autotune",
           "scbb_set_wait_limit",
           "scbb_population_moments_noalloc", "scbb_batch_create", "scbb_batch_step", "scbb_batch_destroy",
           "scbb_batch_shared_bulk", "scbb_batch_set_wait_limit",
           "scbb_adjoint_workspace_bytes", "scbb_adjoint_create", "scbb_adjoint_forward", "scbb_adjoint_backward",
           "scbb_adjoint_backward_capsule",
           "scbb_adjoint_destroy", "scbb_state_bytes", "scbb_save", "scbb_load", "scbb_last_error", "scbb_destroy"]


class scbb_lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("walls", C.c_int),
                ("u_lo", C.c_double * 3), ("u_hi", C.c_double * 3), ("wall_kind", C.c_int)]


class scbb_fluid(C.Structure):
    _fields_ = [("tau", C.c_double), ("G", C.c_double), ("psi_kind", C.c_int), ("g", C.c_double * 3),
                ("coupling", C.c_int), ("rho_maj", C.c_double), ("rho_min", C.c_double), ("C0", C.c_double),
                ("mass_correction", C.c_int), ("pp_eps", C.c_double), ("pp_d0", C.c_double),
                ("storage", C.c_int), ("max_boundary", C.c_int)]


class scbb_mesh(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("ref_xyz", C.c_void_p), ("tri", C.c_void_p),
                ("init_xyz", C.c_void_p), ("kS", C.c_double), ("C", C.c_double), ("kB", C.c_double),
                ("kV", C.c_double), ("mass", C.c_double), ("colour", C.c_double), ("elem_colour", C.c_void_p)]


class ScbbError(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load libscbb.so and declare its exports (fails loudly if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ScbbError(f"libscbb.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.scbb_workspace_bytes.restype = C.c_size_t
    L.scbb_workspace_bytes.argtypes = [vp, vp, C.c_int, vp]
    L.scbb_create.restype = C.c_int
    L.scbb_create.argtypes = [vp, vp, C.c_int, vp, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.scbb_set_density.restype = C.c_int
    L.scbb_set_density.argtypes = [vp, vp, vp, vp]
    L.scbb_step.restype = C.c_int
    L.scbb_step.argtypes = [vp, C.c_longlong]
    L.scbb_sync.restype = C.c_int
    L.scbb_sync.argtypes = [vp]
    L.scbb_get_fields.restype = C.c_int
    L.scbb_get_fields.argtypes = [vp, vp, vp, vp]
    L.scbb_get_populations.restype = C.c_int
    L.scbb_get_populations.argtypes = [vp, vp]
    L.scbb_get_vertices.restype = C.c_int
    L.scbb_get_vertices.argtypes = [vp, vp, vp, vp]
    L.scbb_get_diag.restype = C.c_int
    L.scbb_get_diag.argtypes = [vp, vp, vp, vp, vp]
    L.scbb_get_owner.restype = C.c_int
    L.scbb_get_owner.argtypes = [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.scbb_get_boundary.restype = C.c_int
    L.scbb_get_boundary.argtypes = [vp, C.c_int, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.scbb_launch_count.restype = C.c_longlong
    L.scbb_launch_count.argtypes = [vp]
    L.scbb_enable_timing.restype = C.c_int
    L.scbb_enable_timing.argtypes = [vp, C.c_int]
    L.scbb_kernel_time.restype = C.c_int
    L.scbb_kernel_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.scbb_state_bytes.restype = C.c_size_t
    L.scbb_state_bytes.argtypes = [vp]
    L.scbb_save.restype = C.c_int
    L.scbb_save.argtypes = [vp, vp, C.c_size_t]
    L.scbb_load.restype = C.c_int
    L.scbb_load.argtypes = [vp, vp, C.c_size_t]
    L.scbb_autotune.restype = C.c_int
    L.scbb_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    L.scbb_set_wait_limit.restype = C.c_int
    L.scbb_set_wait_limit.argtypes = [vp, C.c_longlong]
    L.scbb_phase_times.restype = C.c_int
    L.scbb_phase_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.scbb_population_moments_noalloc.restype = C.c_int
    L.scbb_population_moments_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    L.scbb_last_error.restype = C.c_char_p
    L.scbb_last_error.argtypes = [vp]
    L.scbb_destroy.restype = None
    L.scbb_destroy.argtypes = [vp]
    L.scbb_batch_create.restype = C.c_int
    L.scbb_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.POINTER(vp)]
    L.scbb_batch_step.restype = C.c_int
    L.scbb_batch_step.argtypes = [vp, C.c_longlong]
    L.scbb_batch_destroy.restype = None
    L.scbb_batch_destroy.argtypes = [vp]
    L.scbb_batch_shared_bulk.restype = C.c_int
    L.scbb_batch_shared_bulk.argtypes = [vp]
    L.scbb_batch_set_wait_limit.restype = C.c_int
    L.scbb_batch_set_wait_limit.argtypes = [vp, C.c_longlong]
    L.scbb_adjoint_workspace_bytes.restype = C.c_size_t
    L.scbb_adjoint_workspace_bytes.argtypes = [vp, C.c_longlong, C.c_int]
    L.scbb_adjoint_create.restype = C.c_int
    L.scbb_adjoint_create.argtypes = [vp, C.c_longlong, C.c_int, vp, C.POINTER(vp)]
    L.scbb_adjoint_forward.restype = C.c_int
    L.scbb_adjoint_forward.argtypes = [vp]
    L.scbb_adjoint_backward.restype = C.c_int
    L.scbb_adjoint_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.scbb_adjoint_backward_capsule.restype = C.c_int
    L.scbb_adjoint_backward_capsule.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.scbb_adjoint_destroy.restype = None
    L.scbb_adjoint_destroy.argtypes = [vp]
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lattice_of(prob) -> scbb_lattice:
    lat = scbb_lattice()
    lat.nx, lat.ny, lat.nz, lat.walls = prob.nx, prob.ny, prob.nz, int(prob.walls)
    lat.u_lo = (C.c_double * 3)(*prob.u_lo)
    lat.u_hi = (C.c_double * 3)(*prob.u_hi)
    lat.wall_kind = int(getattr(prob, "wall_kind", 0))
    return lat


def fluid_of(prob) -> scbb_fluid:
    fl = scbb_fluid()
    fl.tau, fl.G, fl.psi_kind = prob.tau, prob.G, prob.psi_kind
    fl.g = (C.c_double * 3)(*prob.g)
    fl.coupling = prob.coupling if prob.capsules else 1
    fl.rho_maj, fl.rho_min, fl.C0 = prob.rho_maj, prob.rho_min, prob.C0
    fl.mass_correction = int(prob.mass_correction)
    fl.pp_eps, fl.pp_d0 = prob.pp_eps, prob.pp_d0
    fl.storage = int(getattr(prob, "storage", 0))
    fl.max_boundary = int(getattr(prob, "max_boundary", 0))
    return fl


def scbb_population_moments_noalloc(f_dev, nx, ny, nz, walls, stream=None):
    """FP64 (mass A, mass B, momentum x, y, z) of device populations f[c][i][node] (a float32 CUDA tensor of
    2*19*nx*ny*nz elements), computed without any device allocation.  Returns a numpy array of 5."""
    import torch

    if not (f_dev.is_cuda and f_dev.dtype == torch.float32 and f_dev.is_contiguous()):
        raise ScbbError("f_dev must be a contiguous float32 CUDA tensor")
    if f_dev.numel() != 2 * 19 * nx * ny * nz:
        raise ScbbError("f_dev has the wrong size")
    L = load()
    out = np.zeros(5)
    with torch.cuda.device(f_dev.device):        # the C call works on the current device
        st = (stream or torch.cuda.current_stream(f_dev.device)).cuda_stream
        rc = L.scbb_population_moments_noalloc(C.c_void_p(f_dev.data_ptr()), nx, ny, nz, int(walls), _p(out),
                                               C.c_void_p(st))
    if rc != SCBB_OK:
        raise ScbbError(f"scbb_population_moments_noalloc: {STATUS.get(rc, rc)}")
    return out


class Sim:
    """One simulation context: a torch-owned device workspace, a CUDA stream and the C calls.

    stream: the torch stream the context runs on; by default a stream of its own (steps are replayed as CUDA
    graphs, which cannot be captured on the legacy default stream)."""

    def __init__(self, prob, rhoA=None, rhoB=None, u=None, device="cuda", set_state=True, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise ScbbError("no CUDA device: the scbb path has no CPU fallback")
        L = load()
        self.L = L
        self.prob = prob
        self.lat = lattice_of(prob)
        self.fl = fluid_of(prob)
        nm = len(prob.capsules)
        self.meshes = (scbb_mesh * max(nm, 1))()
        self._keep = []
        self.nv = []
        for k, cap in enumerate(prob.capsules):
            ref, tri, init = cap.mesh()
            ref = np.ascontiguousarray(ref, np.float64)
            tri = np.ascontiguousarray(tri, np.int32)
            init = np.ascontiguousarray(init, np.float64)
            self._keep += [ref, tri, init]
            m = self.meshes[k]
            m.nv, m.nt = len(ref), len(tri)
            m.ref_xyz, m.tri, m.init_xyz = _p(ref), _p(tri), _p(init)
            m.kS, m.C, m.kB, m.kV, m.mass, m.colour = cap.kS, cap.C, cap.kB, cap.kV, cap.mass, cap.colour
            if getattr(cap, "elem_colour", None) is not None:
                ec = np.ascontiguousarray(cap.elem_colour, np.float64)
                if ec.shape != (len(tri),):
                    raise ScbbError("elem_colour needs one value per triangle")
                self._keep.append(ec)
                m.elem_colour = _p(ec)
            self.nv.append(len(ref))
        self.nm = nm
        nbytes = L.scbb_workspace_bytes(C.byref(self.lat), C.byref(self.fl), nm, self.meshes)
        if nbytes == 0:
            raise ScbbError("scbb_workspace_bytes rejected the problem description")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.workspace.device)
        h = C.c_void_p()
        st = L.scbb_create(C.byref(self.lat), C.byref(self.fl), nm, self.meshes,
                           C.c_void_p(self.workspace.data_ptr()), C.c_size_t(nbytes),
                           C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SCBB_OK:
            raise ScbbError(f"scbb_create: {STATUS.get(st, st)}")
        self.h = h
        if set_state:
            if rhoA is None:
                rhoA, rhoB = prob.initial_density()
            self.scbb_set_density(rhoA, rhoB, u)

    def _check(self, st, what):
        if st != SCBB_OK:
            msg = self.L.scbb_last_error(self.h)
            raise ScbbError(f"{what}: {STATUS.get(st, st)}: {msg.decode() if msg else ''}")

    # ---- calls with the C names
    def scbb_set_density(self, rhoA, rhoB, u=None):
        a = np.ascontiguousarray(rhoA, np.float64).ravel()
        b = np.ascontiguousarray(rhoB, np.float64).ravel()
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(3, -1)
        self._check(self.L.scbb_set_density(self.h, _p(a), _p(b), _p(uu)), "scbb_set_density")

    def scbb_step(self, n=1):
        self._check(self.L.scbb_step(self.h, int(n)), "scbb_step")

    def scbb_sync(self):
        self._check(self.L.scbb_sync(self.h), "scbb_sync")

    def scbb_get_fields(self, out=None):
        """(rho^A, rho^B, u) as FP64 arrays shaped (nz, ny, nx) and (3, nz, ny, nx); out: optional caller
        arrays (contiguous float64, for example views of pinned host memory) to fill instead."""
        N = self.prob.n_nodes
        s = (self.prob.nz, self.prob.ny, self.prob.nx)
        if out is None:
            a, b, u = np.empty(N), np.empty(N), np.empty(3 * N)
        else:
            a, b, u = out
            for arr, n in ((a, N), (b, N), (u, 3 * N)):
                if arr.dtype != np.float64 or not arr.flags.c_contiguous or arr.size != n:
                    raise ScbbError("scbb_get_fields: out arrays must be contiguous float64 of N, N and 3 N values")
        self._check(self.L.scbb_get_fields(self.h, _p(a), _p(b), _p(u)), "scbb_get_fields")
        return a.reshape(s), b.reshape(s), u.reshape((3,) + s)

    def scbb_get_populations(self):
        N = self.prob.n_nodes
        f = np.empty(2 * N * 19)
        self._check(self.L.scbb_get_populations(self.h, _p(f)), "scbb_get_populations")
        return f.reshape(2, N, 19)

    def scbb_get_vertices(self):
        NV = sum(self.nv)
        X, V, F = np.empty(3 * NV), np.empty(3 * NV), np.empty(3 * NV)
        self._check(self.L.scbb_get_vertices(self.h, _p(X), _p(V), _p(F)), "scbb_get_vertices")
        return X.reshape(NV, 3), V.reshape(NV, 3), F.reshape(NV, 3)

    def scbb_get_diag(self):
        m, p = np.empty(2), np.empty(3)
        vol, com = np.empty(max(self.nm, 1)), np.empty(3 * max(self.nm, 1))
        self._check(self.L.scbb_get_diag(self.h, _p(m), _p(p), _p(vol), _p(com)), "scbb_get_diag")
        return dict(mass=m, momentum=p, volume=vol[:self.nm], com=com[:3 * self.nm].reshape(self.nm, 3))

    def scbb_get_owner(self):
        """(owner[nz, ny, nx] uint16, boundary-node count, fresh-node count of the last step)."""
        o = np.empty(self.prob.n_nodes, np.uint16)
        nb, nf = C.c_int(0), C.c_int(0)
        self._check(self.L.scbb_get_owner(self.h, _p(o), C.byref(nb), C.byref(nf)), "scbb_get_owner")
        return o.reshape(self.prob.nz, self.prob.ny, self.prob.nx), nb.value, nf.value

    def scbb_get_boundary(self):
        """(boundary nodes int32[n] in the list's order, their links' crossed elements int32[n, 18] (-1: not
        cut), cut links resolved by the nearest-centroid rule)."""
        nb, nfb = C.c_int(0), C.c_int(0)
        self._check(self.L.scbb_get_boundary(self.h, 0, None, None, C.byref(nb), C.byref(nfb)), "scbb_get_boundary")
        n = nb.value
        nodes = np.empty(max(n, 1), np.int32)
        elems = np.empty((max(n, 1), 18), np.int32)
        self._check(self.L.scbb_get_boundary(self.h, n, _p(nodes), _p(elems), C.byref(nb), C.byref(nfb)),
                    "scbb_get_boundary")
        return nodes[:n], elems[:n], nfb.value

    def scbb_launch_count(self):
        return int(self.L.scbb_launch_count(self.h))

    def scbb_enable_timing(self, on=True):
        """on: False/0 off, True/1 bulk-kernel events, 2 bulk-kernel and per-phase events."""
        self._check(self.L.scbb_enable_timing(self.h, int(on)), "scbb_enable_timing")

    def scbb_kernel_time(self):
        ms, n = C.c_double(0), C.c_longlong(0)
        self._check(self.L.scbb_kernel_time(self.h, C.byref(ms), C.byref(n)), "scbb_kernel_time")
        return ms.value, n.value

    def scbb_autotune(self, reps=5):
        """Times the bulk kernel in each block shape that fits the box and keeps the fastest; returns the shape
        kept (0..3), or -1 for boxes on the general bulk kernel."""
        k = C.c_int(-1)
        self._check(self.L.scbb_autotune(self.h, int(reps), C.byref(k)), "scbb_autotune")
        return k.value

    def scbb_set_wait_limit(self, polls):
        """Polls of the bulk phase's bounded waits on its asynchronous copies before they give up."""
        self._check(self.L.scbb_set_wait_limit(self.h, int(polls)), "scbb_set_wait_limit")

    def scbb_state_bytes(self):
        return int(self.L.scbb_state_bytes(self.h))

    def scbb_save(self):
        """The whole state (header and workspace) as a numpy uint8 array on the host."""
        buf = np.empty(self.scbb_state_bytes(), np.uint8)
        self._check(self.L.scbb_save(self.h, _p(buf), C.c_size_t(buf.size)), "scbb_save")
        return buf

    def scbb_load(self, buf):
        """Restores a state saved by scbb_save from a context of the same shape."""
        b = np.ascontiguousarray(buf, np.uint8)
        self._check(self.L.scbb_load(self.h, _p(b), C.c_size_t(b.size)), "scbb_load")

    PHASES = ("ibm_spread", "walls", "bulk", "boundary", "membrane", "classify", "fresh")

    def scbb_phase_times(self):
        """Summed milliseconds per phase of the steps timed with timing mode 2, and their count."""
        ms = (C.c_double * len(self.PHASES))()
        n = C.c_longlong(0)
        self._check(self.L.scbb_phase_times(self.h, ms, C.byref(n)), "scbb_phase_times")
        return dict(zip(self.PHASES, list(ms))), n.value

    def close(self):
        if getattr(self, "h", None):
            self.L.scbb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several independent Sim contexts stepped together (scbb_batch_*): each context keeps its own stream, the
    batch runs on a stream of its own, pairs of steps of all contexts replay from one CUDA graph, and the bulk
    phase of all boxes runs as one persistent cooperative launch where they can share it."""

    def __init__(self, sims, stream=None, autotune=False):
        import torch

        self.sims = list(sims)
        if autotune:                                 # each box picks its bulk-kernel shape before the batch
            for sim in self.sims:
                sim.scbb_autotune()
        self.L = self.sims[0].L
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.sims[0].workspace.device)
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        st = self.L.scbb_batch_create(arr, len(self.sims), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SCBB_OK:
            raise ScbbError(f"scbb_batch_create: {STATUS.get(st, st)}")
        self.h = h

    @classmethod
    def scbb_batch_create(cls, sims, stream=None):
        return cls(sims, stream)

    def scbb_batch_destroy(self):
        self.close()

    def scbb_batch_step(self, n=1):
        st = self.L.scbb_batch_step(self.h, int(n))
        if st != SCBB_OK:
            raise ScbbError(f"scbb_batch_step: {STATUS.get(st, st)}")

    def scbb_batch_shared_bulk(self):
        """True when the bulk phase of all boxes runs as one persistent cooperative launch."""
        return bool(self.L.scbb_batch_shared_bulk(self.h))

    def scbb_batch_set_wait_limit(self, polls):
        st = self.L.scbb_batch_set_wait_limit(self.h, C.c_longlong(int(polls)))
        if st != SCBB_OK:
            raise ScbbError(f"scbb_batch_set_wait_limit: {STATUS.get(st, st)}")

    def close(self):
        if getattr(self, "h", None):
            self.L.scbb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Adjoint:
    """Reverse-mode derivative of n fluid steps of a Sim (scbb_adjoint_*): a torch-owned workspace holding a
    population checkpoint every K steps, the segment being recomputed and the adjoint lattices."""

    def __init__(self, sim, n_steps, checkpoint_every):
        import torch

        self.sim, self.L = sim, sim.L
        self.n, self.K = int(n_steps), int(checkpoint_every)
        nbytes = self.L.scbb_adjoint_workspace_bytes(sim.h, self.n, self.K)
        if nbytes == 0:
            raise ScbbError("scbb_adjoint_workspace_bytes: unsupported context or arguments "
                            "(FP32 storage; no meshes, or immersed-boundary capsules without repulsion)")
        self.nbytes = int(nbytes)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=sim.workspace.device)
        h = C.c_void_p()
        sim._check(self.L.scbb_adjoint_create(sim.h, self.n, self.K, C.c_void_p(self.workspace.data_ptr()),
                                              C.byref(h)), "scbb_adjoint_create")
        self.h = h

    @classmethod
    def scbb_adjoint_create(cls, sim, n_steps, checkpoint_every):
        return cls(sim, n_steps, checkpoint_every)

    def scbb_adjoint_forward(self):
        self.sim._check(self.L.scbb_adjoint_forward(self.h), "scbb_adjoint_forward")

    def scbb_adjoint_backward(self, dL_drhoA, dL_drhoB):
        """Adjoint of the final densities in (arrays of N); returns (dL/dG, dL/dg[3], dL/drho0^A, dL/drho0^B)
        with the density gradients shaped (nz, ny, nx)."""
        p = self.sim.prob
        a = np.ascontiguousarray(dL_drhoA, np.float64).ravel()
        b = np.ascontiguousarray(dL_drhoB, np.float64).ravel()
        dG, dg = np.zeros(1), np.zeros(3)
        ra, rb = np.empty(p.n_nodes), np.empty(p.n_nodes)
        self.sim._check(self.L.scbb_adjoint_backward(self.h, _p(a), _p(b), _p(dG), _p(dg), _p(ra), _p(rb)),
                        "scbb_adjoint_backward")
        s = (p.nz, p.ny, p.nx)
        return float(dG[0]), dg, ra.reshape(s), rb.reshape(s)

    def scbb_adjoint_backward_capsule(self, dL_dX, dL_drhoA=None, dL_drhoB=None):
        """Adjoint of the final vertex positions (NV x 3) and, optionally, of the final densities in; returns
        (dL/dmoduli (NM x 3: kS, kB, kV), dL/dX0 (NV x 3), dL/dG, dL/dg[3])."""
        p = self.sim.prob
        x = np.ascontiguousarray(dL_dX, np.float64).reshape(-1, 3)
        a = None if dL_drhoA is None else np.ascontiguousarray(dL_drhoA, np.float64).ravel()
        b = None if dL_drhoB is None else np.ascontiguousarray(dL_drhoB, np.float64).ravel()
        nm = len(p.capsules)
        dmod, dx0 = np.zeros((nm, 3)), np.zeros_like(x)
        dG, dg = np.zeros(1), np.zeros(3)
        self.sim._check(self.L.scbb_adjoint_backward_capsule(self.h, _p(x), _p(a), _p(b), _p(dmod), _p(dx0), _p(dG),
                                                             _p(dg)), "scbb_adjoint_backward_capsule")
        return dmod, dx0, float(dG[0]), dg

    def scbb_adjoint_destroy(self):
        self.close()

    def close(self):
        if getattr(self, "h", None):
            self.L.scbb_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fluid_rollout(prob, n_steps, checkpoint_every, G, g, rhoA0, rhoB0):
    """The densities after n_steps of the fluid of `prob` (periodic, no meshes) as a differentiable torch
    function of the Shan-Chen coupling G (0-d tensor), the body acceleration g (3 values) and the initial
    densities rhoA0, rhoB0 (float64 CPU tensors shaped (nz, ny, nx)): returns (rhoA(T), rhoB(T)).  The
    forward pass runs the CUDA step with a population checkpoint every checkpoint_every steps; the backward
    pass runs the adjoint kernels (scbb_adjoint_backward), recomputing each segment from its checkpoint."""
    return _FluidRollout.apply(prob, int(n_steps), int(checkpoint_every), G, g, rhoA0, rhoB0)


def _rollout_function():
    import dataclasses

    import torch

    class FluidRollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, prob, n, K, G, g, rhoA0, rhoB0):
            pr = dataclasses.replace(prob, G=float(G), g=tuple(float(v) for v in g))
            sim = Sim(pr, rhoA0.detach().cpu().numpy(), rhoB0.detach().cpu().numpy())
            adj = Adjoint(sim, n, K)
            adj.scbb_adjoint_forward()
            a, b, _ = sim.scbb_get_fields()
            ctx.sim, ctx.adj = sim, adj
            return torch.from_numpy(a.copy()), torch.from_numpy(b.copy())

        @staticmethod
        def backward(ctx, ga, gb):
            dG, dg, ra, rb = ctx.adj.scbb_adjoint_backward(ga.detach().cpu().numpy(), gb.detach().cpu().numpy())
            ctx.adj.close()
            ctx.sim.close()
            return (None, None, None, torch.tensor(dG, dtype=torch.float64), torch.from_numpy(dg),
                    torch.from_numpy(ra), torch.from_numpy(rb))

    return FluidRollout


class _Lazy:
    fn = None

    def apply(self, *args):
        if _Lazy.fn is None:
            _Lazy.fn = _rollout_function()
        return _Lazy.fn.apply(*args)


_FluidRollout = _Lazy()

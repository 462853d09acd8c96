"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds geometry and random numbers only: icosphere meshes, capsule placements and the initial
density fields.  It contains none of the method's arithmetic (no equilibrium, no forces, no streaming), so
both the CUDA path and the FP64 oracle can consume its outputs without sharing any of the method's code.

Workloads are shaped like the paper's setups (Sec. III: flat fluid-fluid interface, capsules of the lower
fluid's composition, G = 3.6, majority/minority densities 0.7 / 0.042, node mass 5, C = 9 from nu_s = 0.9,
kappa_V = 20, B = kappa_B / (kappa_S R0^2) = 0.01).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


# ----------------------------------------------------------------------------------------------------------
# Icosphere: recursive midpoint subdivision of the icosahedron, projected to the unit sphere.
# Triangles are ordered counter-clockwise seen from outside, so (x2-x1) x (x3-x1) points outward.
# ----------------------------------------------------------------------------------------------------------
def icosphere(subdiv: int):
    """Return (vertices[nv,3] float64 on the unit sphere, triangles[nt,3] int32), nv = 10*4^s+2."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(v, dtype=np.float64)
    F = np.array(faces, dtype=np.int32)
    # orient outward
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def geodesic_sphere(freq: int):
    """Class-I geodesic sphere: every face of the icosahedron split into freq^2 triangles, the points projected
    onto the unit sphere.  Returns (vertices[nv,3], triangles[nt,3] int32) with nv = 10 freq^2 + 2 and
    nt = 20 freq^2, triangles counter-clockwise seen from outside; freq = 12 gives the paper's 1442 nodes and
    2880 elements (recursive halving only reaches the frequencies 2^s)."""
    V0, F0 = icosphere(0)
    index, pts = {}, []

    def vid(a, b, c, i, j, k):
        # the point (i A + j B + k C) / freq of face (A, B, C); a point on an edge or a corner is keyed by the
        # icosahedron vertices it mixes, so the faces sharing it share one vertex
        key = tuple(sorted((v, w) for v, w in ((a, i), (b, j), (c, k)) if w > 0))
        if key not in index:
            q = (i * V0[a] + j * V0[b] + k * V0[c]) / freq
            pts.append(q / np.linalg.norm(q))
            index[key] = len(pts) - 1
        return index[key]

    tris = []
    for a, b, c in F0:
        for i in range(freq):
            for j in range(freq - i):
                p00 = vid(a, b, c, freq - i - j, i, j)
                p10 = vid(a, b, c, freq - i - j - 1, i + 1, j)
                p01 = vid(a, b, c, freq - i - j - 1, i, j + 1)
                tris.append((p00, p10, p01))
                if i + j < freq - 1:
                    tris.append((p10, vid(a, b, c, freq - i - j - 2, i + 1, j + 1), p01))
    V = np.array(pts, dtype=np.float64)
    F = np.array(tris, dtype=np.int32)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), (a + b + c) / 3.0) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


# ----------------------------------------------------------------------------------------------------------
# Problem description (plain data).  Units: dx = dt = rho0 = 1.
# ----------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Capsule:
    centre: tuple
    radius: float
    subdiv: int = 3
    kS: float = 0.005
    C: float = 9.0
    kB: float = 5e-4
    kV: float = 20.0
    mass: float = 5.0
    colour: float = 0.0
    deform: Optional[np.ndarray] = None      # optional 3x3 affine map applied to the initial (not reference) shape
    elem_colour: Optional[np.ndarray] = None  # optional colour of each triangle (a Janus particle); else `colour`
    geodesic: int = 0                        # > 0: a frequency-`geodesic` geodesic sphere instead of subdiv

    def mesh(self):
        V, F = geodesic_sphere(self.geodesic) if self.geodesic else icosphere(self.subdiv)
        ref = V * self.radius + np.asarray(self.centre, dtype=np.float64)
        init = ref.copy()
        if self.deform is not None:
            init = (V * self.radius) @ np.asarray(self.deform, dtype=np.float64).T + np.asarray(self.centre)
        return ref, F, init


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    walls: int = 1                  # 1: solid wall planes at z=0 and z=nz-1 (half-way bounce-back)
    u_lo: tuple = (0.0, 0.0, 0.0)   # velocity of the z=0 wall
    u_hi: tuple = (0.0, 0.0, 0.0)   # velocity of the z=nz-1 wall
    wall_kind: int = 0              # 0: walls moving at u_lo / u_hi; 1: resting walls, on-site velocity u_lo / u_hi
                                    #    on the planes z = 1 and z = nz-2
    tau: float = 1.0
    G: float = 3.6
    psi_kind: int = 0               # 0: psi = 1-exp(-rho) (paper), 1: psi = rho
    g: tuple = (0.0, 0.0, 0.0)      # uniform body acceleration (force density rho^c * g)
    coupling: int = 1               # 0: half-way bounce-back (paper), 1: 2-point immersed boundary
    rho_maj: float = 0.7
    rho_min: float = 0.042
    C0: float = 2500.0
    mass_correction: int = 1
    pp_eps: float = 0.5
    pp_d0: float = 1.25
    z_interface: Optional[float] = None   # lower fluid z < z_interface is A-rich
    droplet: Optional[tuple] = None       # (cx, cy, cz, R): B-rich droplet in A-rich bulk
    capsules: List[Capsule] = dataclasses.field(default_factory=list)
    noise: float = 1e-4
    seed: int = 1
    steps: int = 200
    storage: int = 0                # populations on the GPU: 0 FP32, 1 FP16, 2 BF16, 3 / 4 FP16 / BF16 deviations
                                    # from w_i (rho_maj + rho_min) / 2 (the oracle is FP64 always)
    max_boundary: int = 0           # GPU boundary-list capacity (0: sized from the membrane areas)

    @property
    def n_nodes(self):
        return self.nx * self.ny * self.nz

    def initial_density(self):
        """Initial rho^A, rho^B as float64 arrays of shape (nz, ny, nx) (x fastest).

        Lower fluid (z < z_interface) is A-rich (rho_maj / rho_min), the upper fluid mirrored; a droplet is
        B-rich inside; under bounce-back coupling capsule interiors take the lower fluid's composition
        (paper Sec. III, common parameters).  Wall planes carry the adjacent fluid's composition (never used as fluid).  Noise
        U[-noise, noise] per component per node from PCG64(seed).
        """
        nz, ny, nx = self.nz, self.ny, self.nx
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        a = np.full((nz, ny, nx), self.rho_maj)
        b = np.full((nz, ny, nx), self.rho_min)
        if self.z_interface is not None:
            up = z >= self.z_interface
            a[up], b[up] = self.rho_min, self.rho_maj
        if self.droplet is not None:
            cx, cy, cz, R = self.droplet
            d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
            ins = d < R
            a[ins], b[ins] = self.rho_min, self.rho_maj
        # Capsule interiors are separate fluid volumes only under bounce-back; an immersed-boundary membrane
        # is permeable, so there the fluid is left continuous across it.
        for cap in (self.capsules if self.coupling == 0 else []):
            cx, cy, cz = cap.centre
            d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
            ins = d < cap.radius
            a[ins], b[ins] = self.rho_maj, self.rho_min
        rng = np.random.Generator(np.random.PCG64(self.seed))
        if self.noise:
            a = a + rng.uniform(-self.noise, self.noise, size=a.shape)
            b = b + rng.uniform(-self.noise, self.noise, size=b.shape)
        return a, b


# ----------------------------------------------------------------------------------------------------------
# The five workloads (synthetic stand-ins for the paper's experiments; no dataset is involved).
# ----------------------------------------------------------------------------------------------------------
def cfg_parity(coupling: int = 1) -> Problem:
    """32^3 parity case: walls at z=0/31, psi = rho, interface at z=16 (0.7 / 0.04), one s=3 capsule of
    radius 6 at (16,16,20), kS=0.005, kB=5e-4, colour 0, 200 steps, noise 1e-4 from PCG64(1)."""
    # kappa_V = 20 makes the explicit massless immersed-boundary update unstable (growth factor
    # ~ 1 - 3 kV / (2 rho R)), so that mode uses kappa_V = 1; with bounce-back and node mass 5 the volume mode
    # of this coarse mesh (s = 3, R = 6) leaves the symplectic-Euler stability range at kappa_V = 20, so it
    # uses kappa_V = 2 (the finer s = 4, R = 12 capsule of the 128^3 workload keeps the paper's 20).
    kV = 2.0 if coupling == 0 else 1.0
    return Problem(name="parity32", nx=32, ny=32, nz=32, walls=1, tau=1.0, G=3.6, psi_kind=1,
                   coupling=coupling, rho_maj=0.7, rho_min=0.04, z_interface=16,
                   capsules=[Capsule(centre=(16.0, 16.0, 20.0), radius=6.0, subdiv=3, kS=0.005, kB=5e-4,
                                     kV=kV)],
                   noise=1e-4, seed=1, steps=200)


def cfg_adsorb128(coupling: int = 0) -> Problem:
    """128^3 capsule adsorbing at a flat interface under interface-parallel wall shear (rate 1e-4): psi
    exponential, interface z=64, s=4 capsule of radius 12 penetrating the interface by 1, colour 0.05,
    kS=0.002, kB = 0.01 kS R^2."""
    H = 126.0                       # fluid height between half-way walls
    U = 1e-4 * H / 2.0
    kS, R = 0.002, 12.0
    colour = 0.05 if coupling == 0 else 0.0
    return Problem(name="adsorb128", nx=128, ny=128, nz=128, walls=1, u_lo=(-U, 0, 0), u_hi=(U, 0, 0),
                   psi_kind=0, coupling=coupling, z_interface=64,
                   capsules=[Capsule(centre=(64.0, 64.0, 64.0 - R + 1.0), radius=R, subdiv=4, kS=kS,
                                     kB=0.01 * kS * R * R, colour=colour,
                                     kV=20.0 if coupling == 0 else 1.0)],
                   noise=1e-4, seed=2, steps=10000)


def cfg_adjoint64(coupling: int = 1) -> Problem:
    """64^3 box between walls with a flat interface at z=32 and one capsule of radius 8 whose centre is 4
    above it (slightly off the lattice planes, where the 2-point stencil has its kinks), kS=0.005,
    kB = 0.01 kS R^2: the capsule whose centre-of-mass height is differentiated over 2000 steps.  Under the
    immersed boundary the mesh is s=3 (642 vertices, edges about 1.3 lattice units) and kV=1: the s=4 mesh's
    edges (about 0.6) are finer than the 2-point stencil resolves, and that capsule's explicit massless update
    diverges within 1000 steps, in the oracle as on the GPU; kV=20 is outside that update's stability range.
    Under bounce-back it is the s=4 mesh with kV=20."""
    kS, R = 0.005, 8.0
    ibm = coupling == 1
    return Problem(name="adjoint64", nx=64, ny=64, nz=64, walls=1, psi_kind=0, coupling=coupling,
                   z_interface=32,
                   capsules=[Capsule(centre=(32.31, 31.77, 32.0 + 4.13), radius=R, subdiv=3 if ibm else 4, kS=kS,
                                     kB=0.01 * kS * R * R, kV=1.0 if ibm else 20.0)],
                   noise=1e-4, seed=4, steps=2000)


def cfg_droplet256(n_caps: int = 300, coupling: int = 0, n: int = 256, R_drop: float = 70.0,
                   R_cap: float = 8.0, seed: int = 5, penetration: float = 1.5, shell: float = 20.0,
                   kS: float = 0.0388) -> Problem:
    """256^3 periodic box, B-rich droplet of radius 70 at the centre, n_caps s=3 capsules of radius 8 at
    seeded non-overlapping positions around it, colours alternating +/-0.05.  The centres lie in a shell
    from R_drop + R_cap - penetration (a capsule that slightly penetrates the droplet, as in the paper's
    droplet covering) to that radius + shell: the capsules' A-rich interiors stay in the A-rich phase.
    Softness as in the paper's droplet covering: beta = R^2 gamma / kB = 100 with B = kB / (kS R^2) = 0.01,
    i.e. kS = gamma = 0.0388, the interface tension of these fluids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c0 = np.array([n / 2.0] * 3)
    centres = []
    tries = 0
    while len(centres) < n_caps and tries < 200000:
        tries += 1
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = R_drop + R_cap - penetration + rng.uniform(0.0, shell)
        p = c0 + r * d
        if np.any(p < R_cap + 2) or np.any(p > n - R_cap - 2):
            continue
        if all(np.linalg.norm(p - q) >= 2 * R_cap + 2 for q in centres):
            centres.append(p)
    caps = [Capsule(centre=tuple(p), radius=R_cap, subdiv=3, kS=kS, kB=0.01 * kS * R_cap ** 2,
                    colour=(0.05 if k % 2 == 0 else -0.05) if coupling == 0 else 0.0)
            for k, p in enumerate(centres)]
    return Problem(name="droplet256", nx=n, ny=n, nz=n, walls=0, psi_kind=0, coupling=coupling,
                   droplet=(n / 2.0, n / 2.0, n / 2.0, R_drop), capsules=caps, noise=1e-4, seed=seed,
                   steps=20000)


def janus_colours(cap: "Capsule", top: float, bottom: float) -> np.ndarray:
    """Per-triangle colours of a Janus capsule: `top` on the triangles whose centroid lies above the capsule's
    centre (+z), `bottom` below."""
    ref, tri, _ = cap.mesh()
    cz = ref[tri].mean(axis=1)[:, 2]
    return np.where(cz >= cap.centre[2], top, bottom).astype(np.float64)


def cfg_adjoint(n: int = 32, R_drop: float = 8.0, seed: int = 9, G: float = 3.6) -> Problem:
    """Periodic n^3 two-component box with a B-rich droplet of radius R_drop slightly off the box centre
    (exponential psi, no capsules): the fluid whose adjoint is checked against finite differences, and, at
    64^3, the differentiation workload of the benchmark."""
    c = n / 2.0
    return Problem(name=f"adjoint{n}", nx=n, ny=n, nz=n, walls=0, psi_kind=0, G=G, coupling=1,
                   droplet=(c + 0.3, c - 0.2, c + 0.1, R_drop), capsules=[], noise=1e-3, seed=seed, steps=2000)


def cfg_batch48(n_boxes: int = 48, seed: int = 3) -> List[Problem]:
    """A sweep of independent boxes of uneven size: cubes with edges drawn from PCG64(seed) uniformly among the
    integers in [40, 72], walls at both z ends, a flat interface at mid height, one s = 3 capsule of radius 6 (642
    vertices) penetrating it by 1; box k takes colour index k mod 11 over [-0.1, 0.1] and shear modulus index
    (k div 11) mod 4 over {0.001, 0.003, 0.01, 0.03}, kB = 0.01 kS R^2, kV = 2 (coarse mesh), exponential psi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    colours = np.linspace(-0.1, 0.1, 11)
    moduli = (0.001, 0.003, 0.01, 0.03)
    R = 6.0
    out = []
    for k in range(n_boxes):
        L = int(rng.integers(40, 73))
        kS = moduli[(k // 11) % 4]
        cap = Capsule(centre=(L / 2 + 0.3, L / 2 - 0.2, L / 2 - R + 1.0), radius=R, subdiv=3, kS=kS,
                      kB=0.01 * kS * R * R, kV=2.0, colour=float(colours[k % 11]))
        out.append(Problem(name=f"batch{k}", nx=L, ny=L, nz=L, walls=1, psi_kind=0, coupling=0,
                           z_interface=L // 2, capsules=[cap], noise=1e-4, seed=100 + k, steps=5000))
    return out


def small_problem(n=16, walls=1, coupling=1, capsule=True, psi_kind=0, seed=7, subdiv=2, radius=4.0,
                  noise=1e-3, nx=None, ny=None, nz=None) -> Problem:
    """A small seeded case for quick parity checks (several tiles plus a ragged tail when sizes are odd)."""
    nx = nx or n
    ny = ny or n
    nz = nz or n
    caps = []
    if capsule:
        caps = [Capsule(centre=(nx / 2.0 + 0.3, ny / 2.0 - 0.2, nz / 2.0 + 0.4), radius=radius,
                        subdiv=subdiv, kS=0.01, kB=1e-3, kV=1.0)]
    return Problem(name=f"small{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, walls=walls, psi_kind=psi_kind,
                   coupling=coupling, z_interface=nz // 2, capsules=caps, noise=noise, seed=seed, steps=20)

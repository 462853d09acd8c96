"""Pins of the oracle's 2-point immersed-boundary transfer operators and of the particle-particle repulsion
(Sec. III.E) -- identities and brute force, no GPU needed."""
import numpy as np

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs


def _ibm_sim(walls=0, n=(12, 10, 11)):
    cap = inputs.Capsule(centre=(5.3, 4.7, 5.2), radius=3.0, subdiv=1)
    p = inputs.Problem(name="t", nx=n[0], ny=n[1], nz=n[2], walls=walls, coupling=1, capsules=[cap], noise=0.0)
    return O.OracleSim(p)


def test_ibm_spread_interp_adjoint_and_partition_of_unity():
    """Spreading is the transpose of interpolation (<S F, u> = <F, S^T u>), and the hat weights sum to one,
    so the spread field carries the total vertex force."""
    s = _ibm_sim()
    X, _, _ = s.vertices()
    rng = np.random.default_rng(1)
    Fb = rng.standard_normal(X.shape)
    u = rng.standard_normal((3, s.N))
    lhs = (s.ibm_spread(Fb).reshape(3, -1) * u).sum()
    rhs = (Fb * s.ibm_interp(u)).sum()
    assert np.isclose(lhs, rhs, rtol=1e-13)
    assert np.allclose(s.ibm_spread(Fb).reshape(3, -1).sum(1), Fb.sum(0), rtol=1e-13)


def test_ibm_interpolates_linear_fields_exactly():
    """Trilinear (2-point hat) interpolation reproduces affine velocity fields exactly; a uniform field
    advects every vertex by the same displacement."""
    s = _ibm_sim()
    X, _, _ = s.vertices()
    nz, ny, nx = 11, 10, 12
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    B = np.array([[0.01, -0.02, 0.003], [0.0, 0.015, -0.01], [0.02, 0.001, 0.0]])
    a = np.array([0.1, -0.2, 0.05])
    pos = np.stack([x, y, z]).reshape(3, -1)
    u = a[:, None] + B @ pos
    U = s.ibm_interp(u)
    assert np.allclose(U, a + X @ B.T, rtol=1e-12, atol=1e-14)
    U1 = s.ibm_interp(np.broadcast_to(a[:, None], (3, s.N)).copy())
    assert np.allclose(U1, a, rtol=1e-13)


def _brute_pp(X, cap, eps, d0, L, per):
    F = np.zeros_like(X)
    for i in range(len(X)):
        r = X[i] - X
        for k in range(3):
            if per[k]:
                r[:, k] -= L[k] * np.floor(r[:, k] / L[k] + 0.5)
        d = np.linalg.norm(r, axis=1)
        m = (d < d0) & (d > 0) & (cap != cap[i])
        F[i] = (eps * (d0 - d[m]) ** 1.5 / d[m])[:, None].__mul__(r[m]).sum(0)
    return F


def test_pp_repulsion_matches_brute_force_and_newton3():
    """F = eps (d0 - d)^{3/2} along the separation for nodes of different capsules closer than d0
    (Eq. 26, Sec. III.E, eps = 0.5, d0 = 1.25): the linked-cell sum equals the brute-force pair sum, the total force
    vanishes, and same-capsule pairs do not interact.  Periodic minimum image across the box faces."""
    rng = np.random.default_rng(3)
    L = np.array([9.0, 8.0, 7.0])
    X = rng.uniform(0, 1, (400, 3)) * L
    X[:10] = X[:10] * 0.01 + 0.005            # a few nodes near the corner, images across the faces
    cap = rng.integers(0, 4, 400).astype(np.int32)
    for per_z in (0, 1):
        per = (1, 1, per_z)
        F = O.pp_forces(X, cap, 0.5, 1.25, 9, 8, 7, per_z)
        Fb = _brute_pp(X, cap, 0.5, 1.25, L, per)
        assert np.allclose(F, Fb, rtol=1e-12, atol=1e-15)
        assert np.abs(F.sum(0)).max() < 1e-12
        assert np.abs(F).max() > 0


def test_ibm_coupled_step_conserves_momentum():
    """Skalak and volume forces sum to zero, spreading keeps the sum, and each component receives the
    share rho^c / rho of the spread force: in a periodic box the fluid momentum is conserved by the coupled
    immersed-boundary step (to round-off).  Bending is off here: the Meyer force of Eq. 10 is not an exact
    energy gradient and carries a small net force on irregular shapes."""
    cap = inputs.Capsule(centre=(6.2, 5.9, 6.1), radius=3.0, subdiv=2, kS=0.01, kB=0.0, kV=1.0,
                         deform=np.diag([1.15, 0.9, 1.0]))
    p = inputs.Problem(name="t", nx=12, ny=12, nz=12, walls=0, coupling=1, psi_kind=0, z_interface=6,
                       capsules=[cap], noise=1e-3, seed=9)
    s = O.OracleSim(p)
    m0 = s.momentum()
    s.step(15)
    _, _, F = s.vertices()
    assert np.abs(F).max() > 1e-4
    assert np.abs(s.momentum() - m0).max() < 1e-12


def test_ibm_uniform_flow_translates_capsule():
    """A force-free capsule (reference shape, kB = 0) in a uniform flow u0 moves rigidly: X(t) = X(0) + t u0."""
    cap = inputs.Capsule(centre=(6.0, 6.0, 6.0), radius=3.0, subdiv=2, kB=0.0, kV=1.0)
    p = inputs.Problem(name="t", nx=12, ny=12, nz=12, walls=0, coupling=1, G=0.0, capsules=[cap], noise=0.0,
                       rho_maj=0.5, rho_min=0.5)
    u0 = np.array([0.01, -0.004, 0.002])
    a, b = p.initial_density()
    s = O.OracleSim(p, a, b, np.broadcast_to(u0[:, None, None, None], (3, 12, 12, 12)).copy())
    X0, _, _ = s.vertices()
    s.step(10)
    X, V, _ = s.vertices()
    assert np.allclose(X, X0 + 10 * u0, rtol=0, atol=1e-13)
    assert np.allclose(V, u0, atol=1e-14)

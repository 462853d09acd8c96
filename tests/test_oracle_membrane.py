"""Pins of the oracle's membrane mechanics (Sec. II.B, Eq. 6-10) against closed forms, invariances and
finite differences of the energies (no GPU needed)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs


def _deformed(subdiv=1, seed=0, noise=0.03):
    V, T = inputs.icosphere(subdiv)
    rng = np.random.default_rng(seed)
    A = np.eye(3) + 0.15 * rng.standard_normal((3, 3))
    X = (V * 3.0) @ A.T + rng.standard_normal(3) + noise * rng.standard_normal(V.shape)
    return V * 3.0, T, X


def _fd_grad(efun, X, h=1e-6):
    g = np.zeros_like(X)
    for v in range(len(X)):
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, k] += h
            Xm[v, k] -= h
            g[v, k] = (efun(Xp) - efun(Xm)) / (2 * h)
    return g


@pytest.mark.parametrize("subdiv", [0, 1])
def test_skalak_force_is_minus_energy_gradient(subdiv):
    """Eq. 8: F = -dE/dx for the Skalak energy of Eq. 6 (central differences, h = 1e-6)."""
    ref, T, X = _deformed(subdiv, seed=subdiv)
    kS, Cs = 0.01, 9.0
    E, F = O.skalak(X, T, ref, kS, Cs)
    g = _fd_grad(lambda Y: O.skalak(Y, T, ref, kS, Cs)[0], X)
    assert np.allclose(F, -g, rtol=1e-6, atol=1e-9 * np.abs(F).max())


def test_skalak_rest_shape_and_invariances():
    """The stress-free shape carries no force; the energy is invariant under rigid motions, so the net force
    and net torque vanish for any shape (Eq. 6-8)."""
    ref, T, X = _deformed(2, seed=3)
    E0, F0 = O.skalak(ref, T, ref, 0.01, 9.0)
    assert E0 < 1e-28 and np.abs(F0).max() < 1e-15
    E, F = O.skalak(X, T, ref, 0.01, 9.0)
    assert np.abs(F.sum(0)).max() < 1e-13 * np.abs(F).max() * len(X)
    tq = np.cross(X, F).sum(0)
    assert np.abs(tq).max() < 1e-12 * np.abs(F).max() * len(X)
    # rigid rotation + translation of the deformed shape leaves E unchanged
    th = 0.7
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    E2, _ = O.skalak(X @ Rz.T + 5.0, T, ref, 0.01, 9.0)
    assert np.isclose(E, E2, rtol=1e-12)


def test_skalak_uniform_dilation_closed_form():
    """Isotropic stretch lambda: I1 = 2 lambda^2 - 2, I2 = lambda^4 - 1, so
    E = kS/4 A0 (I1^2 + 2 I1 - 2 I2 + C I2^2) with A0 the total reference area (Eq. 6)."""
    V, T = inputs.icosphere(2)
    ref = V * 4.0
    lam = 1.07
    kS, Cs = 0.003, 9.0
    E, _ = O.skalak(ref * lam, T, ref, kS, Cs)
    a, b, c = ref[T[:, 0]], ref[T[:, 1]], ref[T[:, 2]]
    A0 = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    I1, I2 = 2 * lam ** 2 - 2, lam ** 4 - 1
    assert np.isclose(E, kS / 4 * A0 * (I1 ** 2 + 2 * I1 - 2 * I2 + Cs * I2 ** 2), rtol=1e-12)


def test_skalak_uniaxial_closed_form():
    """Stretch lambda along x of a flat triangle: lambda1 = lambda, lambda2 = 1, so I1 = lambda^2 - 1,
    I2 = lambda^2 - 1 (Eq. 6 invariants)."""
    ref = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.3, 0.8, 0]])
    T = np.array([[0, 1, 2]], np.int32)
    lam = 1.2
    X = ref * np.array([lam, 1, 1])
    E, _ = O.skalak(X, T, ref, 1.0, 2.0)
    I1 = I2 = lam ** 2 - 1
    assert np.isclose(E, 0.25 * 0.4 * (I1 ** 2 + 2 * I1 - 2 * I2 + 2.0 * I2 ** 2), rtol=1e-13)


def test_volume_closed_forms_and_gradient():
    """Enclosed volume of a closed outward mesh: a unit cube made of 12 triangles has V = 1; the volume force
    of Eq. 7 equals -dE/dx."""
    cube = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    T = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4], [1, 2, 6], [1, 6, 5],
                  [2, 3, 7], [2, 7, 6], [3, 0, 4], [3, 4, 7]], np.int32)
    assert np.isclose(O.volume(cube, T), 1.0, rtol=1e-15)
    assert np.isclose(O.volume(cube + 10.0, T), 1.0, rtol=1e-13)
    ref, Ti, X = _deformed(1, seed=5)
    V0 = O.volume(ref, Ti)
    E, F = O.volume_force(X, Ti, 20.0, V0)
    g = _fd_grad(lambda Y: O.volume_force(Y, Ti, 20.0, V0)[0], X)
    assert np.allclose(F, -g, rtol=1e-6, atol=1e-9 * np.abs(F).max())
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).max() * len(X)


def test_bending_exact_identities():
    """Meyer operators: the mixed areas partition the surface area exactly, and the discrete Gauss-Bonnet
    theorem sum_i KG_i A_i = 2 pi chi = 4 pi holds exactly for a closed genus-0 mesh."""
    ref, T, X = _deformed(2, seed=7)
    b = O.bending(X, T, 1.0)
    a, bb, c = X[T[:, 0]], X[T[:, 1]], X[T[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(bb - a, c - a), axis=1).sum()
    assert np.isclose(b["A"].sum(), area, rtol=1e-13)
    assert np.isclose((b["KG"] * b["A"]).sum(), 4 * np.pi, rtol=1e-12)


def test_bending_sphere():
    """On a sphere of radius R: H -> 1/R, KG -> 1/R^2, 2H(H^2 - KG) -> 0 and the bending force -> 0
    (Eq. 10); the discrete values converge with refinement and the normals point outward."""
    R = 5.0
    errs = []
    for s in (3, 4):
        V, T = inputs.icosphere(s)
        b = O.bending(V * R, T, 1.0)
        assert np.all(np.einsum("ij,ij->i", b["n"], V) > 0.99)
        errs.append(np.abs(b["H"] * R - 1).max())
        assert np.abs(b["KG"] * R * R - 1).mean() < 0.05
        assert np.abs(b["F"]).max() / (2 / R ** 3 * b["A"].mean()) < 0.5
    assert errs[1] < errs[0] and errs[1] < 0.02


def _spheroid_analytic(a, c, Z):
    """Mean and Gaussian curvature of the spheroid x^2/a^2 + y^2/a^2 + z^2/c^2 = 1 at height z."""
    # parametrise by polar angle t: r = a sin t, z = c cos t
    t = np.arccos(np.clip(Z / c, -1, 1))
    s, co = np.sin(t), np.cos(t)
    den = a * a * co * co + c * c * s * s
    K = c * c / den ** 2
    H = c * (a * a + den) / (2 * a * den ** 1.5)
    return H, K


def test_bending_spheroid_curvatures():
    """Prolate spheroid (a = 4, c = 6): the Meyer mean and Gaussian curvatures match the closed forms of the
    spheroid to a few per cent at subdivision 4 (Eq. 9-10 operators)."""
    a, c = 4.0, 6.0
    V, T = inputs.icosphere(4)
    X = V * np.array([a, a, c])
    b = O.bending(X, T, 1.0)
    H, K = _spheroid_analytic(a, c, X[:, 2])
    assert np.median(np.abs(b["H"] / H - 1)) < 0.01
    assert np.median(np.abs(b["KG"] / K - 1)) < 0.03


def test_bending_force_descends_energy():
    """Sign pin of Eq. 10: on a perturbed sphere the nodal bending force points down the gradient of the
    discrete Helfrich energy E = kB/2 sum (2H)^2 A (cosine > 0.9), and it vanishes in net translation to
    discretisation accuracy."""
    V, T = inputs.icosphere(2)
    rng = np.random.default_rng(11)
    X = V * 4.0 * (1 + 0.05 * rng.standard_normal((len(V), 1)))
    b = O.bending(X, T, 1.0)
    g = _fd_grad(lambda Y: O.bending(Y, T, 1.0)["E"], X, h=1e-6)
    cosang = -(b["F"] * g).sum() / (np.linalg.norm(b["F"]) * np.linalg.norm(g))
    assert cosang > 0.9, cosang


def test_bending_force_density_spheroid():
    """Eq. 10 force density on a spheroid against its closed form: on a surface of revolution r(t), z(t)
    the Laplace-Beltrami operator is (1/(r g)) d/dt (r/g dH/dt), g = |d(r,z)/dt|.  The cotangent Laplacian of
    a discrete H is noisy node by node on a non-uniform mesh, so the pin is on its scale (least-squares
    factor against the closed form within 5 %) and on area-weighted latitude-band averages (within 10 %)
    of Lap H and of the nodal force / mixed area = 2 kB [2H(H^2-K) + Lap H]."""
    a, c = 4.0, 6.0
    h = 1e-4

    def Ht(tt):
        return _spheroid_analytic(a, c, c * np.cos(tt))[0]

    def flux(tt):
        g = np.sqrt((a * np.cos(tt)) ** 2 + (c * np.sin(tt)) ** 2)
        return a * np.sin(tt) / g * (Ht(tt + h) - Ht(tt - h)) / (2 * h)

    for s in (4, 5):
        V, T = inputs.icosphere(s)
        X = V * np.array([a, a, c])
        b = O.bending(X, T, 1.0)
        t = np.arccos(np.clip(X[:, 2] / c, -1, 1))
        ok = np.abs(np.cos(t)) < 0.95          # away from the poles where the parametrisation is singular
        tt = t[ok]
        g = np.sqrt((a * np.cos(tt)) ** 2 + (c * np.sin(tt)) ** 2)
        lap = (flux(tt + h) - flux(tt - h)) / (2 * h) / (a * np.sin(tt) * g)
        H, K = _spheroid_analytic(a, c, X[ok, 2])
        fan = 2 * (2 * H * (H * H - K) + lap)
        fnum = (b["F"][ok] * b["n"][ok]).sum(1) / b["A"][ok]
        for num, an in ((b["LH"][ok], lap), (fnum, fan)):
            alpha = (num * an).sum() / (an * an).sum()
            assert abs(alpha - 1) < 0.05, (s, alpha)
            if s == 5:
                bins = np.digitize(tt, np.linspace(0.35, np.pi - 0.35, 10))
                A = b["A"][ok]
                for k in range(1, 10):
                    m = bins == k
                    band_num = (num[m] * A[m]).sum() / A[m].sum()
                    band_an = (an[m] * A[m]).sum() / A[m].sum()
                    assert abs(band_num - band_an) < 0.1 * np.abs(an).max(), (k, band_num, band_an)


def test_reference_model_band_area_and_hat_box():
    """The band area of the reference model (Sec. III.B, Eq. emulatetension).  (1) A right triangle in the x-z
    plane with legs 1 along x and z: the area below height h is h - h^2 / 2, by hand.  (2) Archimedes' hat-box
    theorem: the area of a spherical zone of height w is 2 pi R w wherever the zone sits, so the band areas of a
    fine icosphere (s = 4) summed over its elements give 2 pi R w for a band at the equator and one halfway to
    the pole alike (the inscribed polyhedron is a few 1e-3 smaller)."""
    z = np.array([[0.0, 0.0, 1.0]])
    A = np.array([0.5])
    for h in (0.0, 0.3, 0.7, 1.0):
        assert abs(O._area_below(z, A, h)[0] - (h - h * h / 2)) < 1e-15
    R, w = 9.0, 1.0
    cap = inputs.Capsule(centre=(0.0, 0.0, 0.0), radius=R, subdiv=4)
    ref, tri, _ = cap.mesh()
    p = ref[tri]
    Atri = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    for zc in (0.0, 0.5 * R):
        band = (O._area_below(p[:, :, 2], Atri, zc + w / 2) - O._area_below(p[:, :, 2], Atri, zc - w / 2)).sum()
        assert abs(band / (2 * np.pi * R * w) - 1) < 1e-2, (zc, band / (2 * np.pi * R * w))


def test_reference_model_tension_balance_and_equilibrium():
    """The emulated tension on a sphere centred at the interface pulls radially in the interface plane: its
    net force vanishes and its total magnitude is gamma x (band area / w) = 2 pi R gamma (the hat-box theorem).
    Relaxed with the elastic laws (Skalak with C = 1, volume penalty, no bending), the capsule reaches an
    equilibrium (residual node force below 1e-6 of the tension on a node's share) with its equator stretched
    and its poles drawn in, r_i > R > r_p, and for small tension (gamma / kS = 0.08 and 0.04) the polar
    contraction is linear in gamma (the largest equatorial radius is not: it sits at the local bulge under the
    line load of the band)."""
    R, kS = 8.0, 0.05
    cap = inputs.Capsule(centre=(0.0, 0.0, 0.0), radius=R, subdiv=3)
    ref, tri, _ = cap.mesh()
    gamma = 0.0388
    F = O.emulated_tension(ref, tri, 0.0, gamma)
    assert np.abs(F.sum(0)).max() < 1e-12
    assert abs(np.linalg.norm(F[:, :2], axis=1).sum() / (2 * np.pi * R * gamma) - 1) < 3e-2
    assert np.abs(F[:, 2]).max() == 0.0

    def strain(g):
        X, res = O.reference_model(ref, tri, kS, 1.0, 0.0, 20.0, 0.0, g, steps=3000)
        c = X.mean(0)
        r_i = np.linalg.norm((X - c)[:, :2], axis=1).max()
        r_p = np.abs((X - c)[:, 2]).max()
        return r_i, r_p, res

    r_i, r_p, res = strain(gamma)
    assert res < 1e-6 * gamma
    assert r_i > R * 1.01 and r_p < R * 0.99, (r_i, r_p)
    _, p1, res1 = strain(0.004)
    _, p2, _ = strain(0.002)
    assert res1 < 1e-6 * 0.004
    lin = (p1 - R) / (p2 - R)
    assert 1.9 < lin < 2.2, lin

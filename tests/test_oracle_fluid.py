"""Pins of the oracle's fluid part against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it checks.  The oracle is never compared with itself: the expected values are
closed forms, conservation laws, analytic flow profiles or printed numbers.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs


def _prob(**kw):
    base = dict(name="t", nx=8, ny=8, nz=8, walls=0, psi_kind=0, coupling=2, noise=0.0, capsules=[])
    base.update(kw)
    return inputs.Problem(**base)


def test_d3q19_isotropy():
    """Eq. 3 weights: sum w = 1, sum w c = 0, sum w c c = cs^2 I, fourth moment cs^4 (d d + d d + d d)."""
    c, w, opp = O.d3q19()
    assert np.isclose(w.sum(), 1.0)
    assert np.allclose((w[:, None] * c).sum(0), 0)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso)
    assert np.all(c[opp] == -c)
    assert (w == 1 / 3).sum() == 1 and (w == 1 / 18).sum() == 6 and (w == 1 / 36).sum() == 12


def test_equilibrium_moments():
    """Eq. 2: zeroth, first and second moments of f_eq are rho, rho u, rho (cs^2 I + u u)."""
    c, w, _ = O.d3q19()
    rng = np.random.default_rng(0)
    for _ in range(5):
        rho = rng.uniform(0.1, 1.0)
        u = rng.uniform(-0.05, 0.05, 3)
        f = np.array([O.feq(i, rho, u) for i in range(19)])
        assert np.isclose(f.sum(), rho, rtol=1e-14)
        assert np.allclose(f @ c, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_mass_conservation_walls_and_sc():
    """Collision and half-way bounce-back conserve each component's mass (Eq. 1, Eq. 11):
    exact to round-off with moving walls, Shan-Chen forces and a ragged box."""
    p = _prob(nx=13, ny=9, nz=14, walls=1, u_lo=(-0.01, 0.0, 0.0), u_hi=(0.01, 0.005, 0.0), z_interface=7,
              noise=1e-3, seed=3)
    s = O.OracleSim(p)
    m0 = [s.mass(0), s.mass(1)]
    s.step(100)
    for c in range(2):
        assert abs(s.mass(c) - m0[c]) / m0[c] < 1e-12


def test_momentum_conservation_sc_periodic():
    """The Shan-Chen forces (Eq. 13) are pairwise antisymmetric, so in a periodic box the total momentum is
    conserved exactly; collision with the velocity-shift forcing conserves it as well."""
    p = _prob(nx=10, ny=9, nz=11, z_interface=5, noise=1e-3, seed=4)
    s = O.OracleSim(p)
    m0 = s.momentum()
    s.step(50)
    assert np.all(np.abs(s.momentum() - m0) < 1e-12)


def test_body_force_momentum_gain():
    """Velocity-shift forcing (Sec. II.A, Eq. 5): summed over components, collision adds exactly F = rho g per node
    per step."""
    g = np.array([1e-5, -2e-5, 3e-6])
    p = _prob(nx=6, ny=5, nz=4, G=0.0, g=tuple(g), noise=1e-3, seed=5)
    s = O.OracleSim(p)
    M = s.mass(0) + s.mass(1)
    m0 = s.momentum()
    s.step(7)
    assert np.allclose(s.momentum() - m0, 7 * M * g, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("psi_kind", [0, 1])
def test_shan_chen_force_closed_form(psi_kind):
    """Eq. 13 on a field that varies along x only: the directions with c_x = +1 carry total weight
    1/18 + 4/36 = 1/6, so F^A_x(x) = -psi^A(x) G (psi^B(x+1) - psi^B(x-1)) / 6 and F_y = F_z = 0."""
    nx = 16
    p = _prob(nx=nx, ny=3, nz=3, psi_kind=psi_kind, G=3.6)
    x = np.arange(nx)
    rb = 0.3 + 0.1 * np.sin(2 * np.pi * x / nx)
    ra = 0.5 + 0.05 * np.cos(2 * np.pi * 3 * x / nx)
    A = np.broadcast_to(ra, (3, 3, nx)).copy()
    B = np.broadcast_to(rb, (3, 3, nx)).copy()
    s = O.OracleSim(p, A, B)
    s.step(1)
    F = s.sc_force()
    psi = (lambda r: r) if psi_kind == 1 else (lambda r: 1 - np.exp(-r))
    pa, pb = psi(ra), psi(rb)
    expA = -pa * 3.6 * (np.roll(pb, -1) - np.roll(pb, 1)) / 6
    expB = -pb * 3.6 * (np.roll(pa, -1) - np.roll(pa, 1)) / 6
    assert np.allclose(F[0, 0, 1, 1], expA, rtol=1e-13, atol=1e-16)
    assert np.allclose(F[1, 0, 1, 1], expB, rtol=1e-13, atol=1e-16)
    assert np.abs(F[:, 1:]).max() < 1e-16


def test_couette_moving_wall_sign():
    """Half-way bounce-back on a moving wall (Eq. 11 with v0 = wall velocity): the steady flow between a
    resting wall at z = 0.5 and a wall moving with U at z = nz - 1.5 is the linear Couette profile, dragged
    in the direction of the wall (fixes the sign of the wall term)."""
    H = 12
    U = 0.01
    p = _prob(nx=2, ny=2, nz=H + 2, walls=1, u_hi=(U, 0, 0), G=0.0, rho_maj=0.5, rho_min=0.5)
    s = O.OracleSim(p)
    s.step(6000)
    _, _, u = s.fields()
    z = np.arange(1, H + 1)
    expect = U * (z - 0.5) / H
    assert np.allclose(u[0, 1:H + 1, 0, 0], expect, rtol=1e-6, atol=1e-10)
    assert np.abs(u[1:, 1:H + 1]).max() < 1e-12


def test_poiseuille_second_order():
    """Body-force driven channel between half-way bounce-back walls: u(z) = g/(2 nu) (z - z0)(z1 - z) with
    nu = (tau - 1/2)/3 and walls half-way between nodes.  The relative L2 error falls at second order."""
    errs = []
    for H in (8, 16):
        nu = (1.0 - 0.5) / 3.0
        umax = 0.005
        g = 8 * nu * umax / H ** 2
        p = _prob(nx=1, ny=1, nz=H + 2, walls=1, G=0.0, g=(g, 0, 0), rho_maj=0.5, rho_min=0.5)
        s = O.OracleSim(p)
        s.step(int(12 * H * H / nu))
        _, _, u = s.fields()
        z = np.arange(1, H + 1)
        ua = g / (2 * nu) * (z - 0.5) * (H + 0.5 - z)
        un = u[0, 1:H + 1, 0, 0] + g / 2          # physical velocity includes half the force (Eq. 5)
        errs.append(np.sqrt(((un - ua) ** 2).sum() / (ua ** 2).sum()))
    order = np.log2(errs[0] / errs[1])
    assert errs[1] < 2e-3
    assert order > 1.8, (errs, order)


def test_flat_interface_symmetry():
    """A flat A|B interface with mirrored compositions stays mirror-symmetric (rho^A(z) = rho^B(z') with z'
    the mirror plane) and sharpens into bulk phases (Sec. II.D, G = 3.6, 0.7 / 0.042)."""
    nz = 24
    p = _prob(nx=2, ny=2, nz=nz, walls=0, z_interface=None, G=3.6, psi_kind=0)
    z = np.arange(nz)
    a = np.where((z >= 6) & (z < 18), 0.042, 0.7)
    A = np.broadcast_to(a[:, None, None], (nz, 2, 2)).copy()
    B = 0.742 - A
    s = O.OracleSim(p, A, B)
    s.step(2000)
    ra, rb, _ = s.fields()
    pa, pb = ra[:, 0, 0], rb[:, 0, 0]
    mirror = (np.arange(nz) + 12) % nz
    assert np.allclose(pa, pb[mirror], atol=1e-10)
    assert pa[0] > 0.65 and pa[12] < 0.06


def test_laplace_law_surface_tension():
    """Laplace law (Sec. III, common parameters: G = 3.6, 0.7 / 0.042, psi = 1 - exp(-rho) gives
    gamma = 0.0388).  Cylindrical B-rich droplets in a periodic 64 x 64 x 1 box: Delta P = gamma / R.
    The pressure is p = cs^2 (rho^A + rho^B) + cs^2 G psi^A psi^B (the continuum limit of Eq. 13).
    Pinned: Delta P is linear in 1/R through the origin.  The oracle's gamma is 0.046; the paper's 0.0388
    comes from a measurement it does not describe, so only a +-30 % band around it is asserted."""
    L = 64
    pts = []
    for R in (8, 11, 14):
        p = _prob(nx=L, ny=L, nz=1, droplet=(L / 2, L / 2, 0, R), rho_maj=0.7, rho_min=0.042)
        s = O.OracleSim(p)
        s.step(3000)
        a, b, _ = s.fields()
        P = (a + b) / 3 + 3.6 * (1 - np.exp(-a)) * (1 - np.exp(-b)) / 3
        Rm = np.sqrt((b > (b.max() + b.min()) / 2).sum() / np.pi)
        pts.append((1 / Rm, P[0, L // 2, L // 2] - P[0, 0, 0]))
    pts = np.array(pts)
    gamma, icpt = np.polyfit(pts[:, 0], pts[:, 1], 1)
    assert abs(icpt) < 0.05 * pts[:, 1].max()
    assert 0.7 * 0.0388 < gamma < 1.3 * 0.0388, gamma

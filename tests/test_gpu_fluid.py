"""GPU parity of the fluid path (fused stream + Shan-Chen + collide, walls) against the FP64 oracle,
through the C ABI.  Same seeded inputs on both sides; element-by-element comparison.

Tolerance (FP32 populations vs FP64): densities within 1e-5 relative node by node, velocities within
1e-5 of max|u| (plus 1e-7 absolute for near-rest flows), after the stated number of steps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5
RTOL_U = 1e-5


def _sim(prob, **kw):
    from paper_1904_11386_gb300 import scbb

    return scbb.Sim(prob, **kw)


def _cmp_fields(g, o, tag=""):
    ga, gb, gu = g
    oa, ob, ou = o
    fluid = oa + ob > 0
    ea = np.abs(ga - oa)[fluid] / np.abs(oa[fluid])
    eb = np.abs(gb - ob)[fluid] / np.abs(ob[fluid])
    umax = max(np.abs(ou).max(), 1e-12)
    eu = np.abs(gu - ou).max()
    assert ea.max() < RTOL_RHO, (tag, "rhoA", ea.max())
    assert eb.max() < RTOL_RHO, (tag, "rhoB", eb.max())
    assert eu < RTOL_U * umax + 1e-7, (tag, "u", eu, umax)


def _prob(**kw):
    base = dict(name="t", nx=37, ny=21, nz=19, walls=1, psi_kind=0, coupling=1, z_interface=9, noise=1e-3,
                seed=11, capsules=[])
    base.update(kw)
    return inputs.Problem(**base)


def test_initial_state_populations_exact():
    """scbb_set_density sets the equilibrium populations of Eq. 2: the moving ones to FP32 rounding of the FP64
    values; the rest population closes the node's mass, rho - sum of the 18 stored moving values, so it
    carries their FP32 roundings (at most 18 * 2^-24 * rho, about 3.2e-6 of f_0 = rho / 3)."""
    p = _prob()
    g = _sim(p)
    o = O.OracleSim(p)
    fg = g.scbb_get_populations()
    fo = o.populations()
    fluid = np.ones((p.nz, p.ny, p.nx), bool)
    fluid[[0, -1]] = False                    # wall planes: the oracle keeps their (unused) initial values
    fluid = fluid.ravel()
    assert np.allclose(fg[:, fluid, 1:], fo[:, fluid, 1:], rtol=2e-7, atol=1e-9)
    assert np.allclose(fg[:, fluid, 0], fo[:, fluid, 0], rtol=4e-6, atol=1e-9)
    assert np.all(fg[:, ~fluid] == 0)


@pytest.mark.parametrize("walls,psi", [(1, 0), (0, 1), (0, 0)])
def test_one_step_populations(walls, psi):
    """One step: every post-streaming population matches the oracle (ragged 37 x 21 x 19 box: several
    32 x 8 tiles, ragged tails in x and y, z-segments)."""
    p = _prob(walls=walls, psi_kind=psi, u_lo=(-0.01, 0.002, 0.0), u_hi=(0.01, 0.0, 0.0))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(1)
    o.step(1)
    fg = g.scbb_get_populations()
    fo = o.populations()
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() < 2e-6 * scale


@pytest.mark.parametrize("walls", [1, 0])
def test_fields_after_100_steps(walls):
    p = _prob(walls=walls, u_lo=(-0.005, 0, 0), u_hi=(0.005, 0, 0))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(100)
    o.step(100)
    _cmp_fields(g.scbb_get_fields(), o.fields(), f"walls={walls}")


def test_mass_conservation_fp64_reduction():
    """Per-component mass is conserved by collision and bounce-back (Eq. 1, 11); the device FP64 reduction
    matches the oracle's mass and stays constant to FP32 round-off."""
    p = _prob(u_lo=(-0.01, 0, 0), u_hi=(0.01, 0, 0))
    g = _sim(p)
    o = O.OracleSim(p)
    m0 = g.scbb_get_diag()["mass"]
    assert np.allclose(m0, [o.mass(0), o.mass(1)], rtol=1e-6)
    g.scbb_step(200)
    m1 = g.scbb_get_diag()["mass"]
    assert np.all(np.abs(m1 - m0) / m0 < 2e-6)


def test_edge_cases_thin_boxes():
    """Degenerate geometries: a single fluid plane between walls (nz = 3) and a one-node-wide box (nx = 1)."""
    for kw in (dict(nx=33, ny=9, nz=3, z_interface=None), dict(nx=1, ny=17, nz=12, z_interface=6)):
        p = _prob(**kw)
        g = _sim(p)
        o = O.OracleSim(p)
        g.scbb_step(20)
        o.step(20)
        _cmp_fields(g.scbb_get_fields(), o.fields(), str(kw))


def test_full_size_128_bulk_parity():
    """The 128^3 workload of the benchmark (walls with shear, exponential psi, flat interface), bulk launch
    configuration as timed: 3 steps against the oracle, every node."""
    p = inputs.cfg_adsorb128(coupling=1)
    p.capsules = []
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(3)
    o.step(3)
    _cmp_fields(g.scbb_get_fields(), o.fields(), "128^3")


@pytest.mark.parametrize("nx,tau,ulo", [(32, 0.8, (0.0, 0.0, 0.0)), (37, 1.3, (-0.01, 0.0, 0.0)),
                                        (32, 1.3, (0.0, 0.01, 0.0))])
def test_tau_not_one(nx, tau, ulo):
    """BGK with tau != 1 (Eq. 1 relaxes towards f_eq instead of replacing the populations): the fused kernels,
    which keep the populations through the collision (row-vectorised for nx = 32, the general tile kernel for
    nx = 37), against the oracle over 30 steps, with moving walls."""
    import dataclasses

    p = dataclasses.replace(_prob(nx=nx), tau=tau, u_lo=ulo, u_hi=tuple(-v for v in ulo))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(30)
    o.step(30)
    _cmp_fields(g.scbb_get_fields(), o.fields(), f"tau={tau}")


@pytest.mark.parametrize("nx", [32, 37])
def test_onsite_velocity_planes(nx):
    """On-site velocity boundaries (Zou and He; resting walls, the planes z = 1 and nz - 2 held at u_lo and u_hi)
    with the two-component interface between them: 60 steps against the oracle, fields node by node and the
    populations (the ones the planes receive from the walls reconstructed by the boundary on both sides), for
    the quad form of the moments kernel (nx = 32) and the node form (nx = 37)."""
    p = _prob(nx=nx, wall_kind=1, u_lo=(0.01, 0.0, 0.0), u_hi=(-0.01, 0.004, 0.0))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(60)
    o.step(60)
    _cmp_fields(g.scbb_get_fields(), o.fields(), f"onsite nx={nx}")
    fg, fo = g.scbb_get_populations(), o.populations()
    fluid = np.ones((p.nz, p.ny, p.nx), bool)
    fluid[[0, -1]] = False
    fluid = fluid.ravel()
    assert np.abs(fg[:, fluid] - fo[:, fluid]).max() < 1e-5 * np.abs(fo[:, fluid]).max()

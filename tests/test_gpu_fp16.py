"""FP16 population storage (populations stored as IEEE half, arithmetic in FP32) against the FP64 oracle.

Every stored population is rounded to nearest, a relative error of at most 2^-12 (2.4e-4); the rest population
of each collision absorbs the rounding of the 18 moving ones, so a node's mass is off by one rounding only.
The densities then carry errors of order 1e-3 after a few hundred steps, and the total mass an offset of order
1e-5; the bounds below are about three times the values measured on a GB300.  The bounce-back comparison is
limited to nodes whose owner agrees with the oracle's, over a window shorter than the first side change whose
timing the FP16 rounding can move."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(prob, steps):
    from paper_1904_11386_gb300 import scbb

    prob.storage = 1
    g = scbb.Sim(prob)
    g.scbb_step(steps)
    o = O.OracleSim(prob)
    o.step(steps)
    return g, o


def _rho_err(g, o, keep=None):
    ga, gb, gu = g.scbb_get_fields()
    oa, ob, ou = o.fields()
    fl = oa + ob > 0
    if keep is not None:
        fl &= keep
    e = max((np.abs(ga - oa)[fl] / oa[fl]).max(), (np.abs(gb - ob)[fl] / ob[fl]).max())
    eu = np.abs(gu - ou)[:, fl].max() / np.abs(ou).max()
    return e, eu


def _mass_err(g, o):
    d = g.scbb_get_diag()
    m = np.array([o.mass(0), o.mass(1)])
    return np.abs(np.asarray(d["mass"]) - m).max() / m.max()


def test_fp16_fluid_100_steps():
    """Two-component fluid with walls, 100 steps: densities within 6e-3 relative, mass within 7e-5."""
    g, o = _run(inputs.small_problem(n=32, walls=1, coupling=1, capsule=False, noise=1e-3), 100)
    e, _ = _rho_err(g, o)
    assert e < 6e-3, e
    assert _mass_err(g, o) < 7e-5


def test_fp16_parity32_ibm_200_steps():
    """The 32^3 immersed-boundary configuration, 200 steps: densities within 4e-3, velocities within 7e-3 of
    max|u|, vertices within 6e-3 lattice units, mass within 4e-5."""
    g, o = _run(inputs.cfg_parity(coupling=1), 200)
    e, eu = _rho_err(g, o)
    assert e < 4e-3, e
    assert eu < 7e-3, eu
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 6e-3
    assert _mass_err(g, o) < 4e-5


def test_fp16_adsorb128_3_steps():
    """The 128^3 bounce-back workload, 3 steps: owners identical, densities within 2e-3, mass within 3e-5."""
    g, o = _run(inputs.cfg_adsorb128(coupling=0), 3)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    e, _ = _rho_err(g, o)
    assert e < 2e-3, e
    assert _mass_err(g, o) < 3e-5

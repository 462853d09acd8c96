"""GPU parity of the membrane and 2-point immersed-boundary path against the FP64 oracle (C ABI)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sim(prob, **kw):
    from paper_1904_11386_gb300 import scbb

    return scbb.Sim(prob, **kw)


def test_membrane_forces_first_step():
    """Skalak + volume + bending node forces (Eq. 6-10) of a deformed capsule at step 0 match the oracle's
    FP64 forces to FP32 accuracy."""
    cap = inputs.Capsule(centre=(12.3, 11.8, 12.2), radius=5.0, subdiv=3, kS=0.01, kB=2e-3, kV=1.0,
                         deform=np.diag([1.12, 0.93, 1.0]))
    p = inputs.Problem(name="t", nx=24, ny=24, nz=26, walls=1, coupling=1, psi_kind=0, z_interface=12,
                       capsules=[cap], noise=1e-4, seed=3)
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(1)
    o.step(1)
    _, _, Fg = g.scbb_get_vertices()
    _, _, Fo = o.vertices()
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()


def test_ibm_small_box_20_steps():
    """Coupled immersed-boundary steps: fields and vertex positions after 20 steps."""
    p = inputs.small_problem(n=20, walls=1, coupling=1, subdiv=2, radius=4.0, noise=1e-4)
    p.capsules[0].kV = 1.0
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(20)
    o.step(20)
    ga, gb, gu = g.scbb_get_fields()
    oa, ob, ou = o.fields()
    fl = oa + ob > 0
    assert (np.abs(ga - oa)[fl] / oa[fl]).max() < 1e-5
    assert (np.abs(gb - ob)[fl] / ob[fl]).max() < 1e-5
    assert np.abs(gu - ou).max() < 1e-5 * np.abs(ou).max() + 1e-7
    Xg, Vg, _ = g.scbb_get_vertices()
    Xo, Vo, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4


def test_parity32_ibm_1000_steps():
    """The 32^3 parity workload (walls, psi = rho, interface at z = 16, s = 3 capsule of radius 6, 2-point
    immersed boundary).  After 200 steps: densities within 1e-5 relative, velocities within 1e-5 of max|u|,
    vertex positions within 1e-4 lattice units, FP64 volume and centre of mass.  After 1000 steps: densities
    within 1e-5 and vertices within 1e-4 still; velocities within 1e-4 of max|u| (measured 3.6e-5): with
    psi = rho the velocity is dominated by the spurious currents at the interface (|u| ~ 0.07), a difference
    of large Shan-Chen terms that magnifies the FP32 state's round-off."""
    p = inputs.cfg_parity(coupling=1)
    g = _sim(p)
    o = O.OracleSim(p)

    def errors():
        ga, gb, gu = g.scbb_get_fields()
        oa, ob, ou = o.fields()
        fl = oa + ob > 0
        ea = (np.abs(ga - oa)[fl] / oa[fl]).max()
        eb = (np.abs(gb - ob)[fl] / ob[fl]).max()
        eu = np.abs(gu - ou).max() / np.abs(ou).max()
        Xg, _, _ = g.scbb_get_vertices()
        Xo, _, _ = o.vertices()
        return max(ea, eb), eu, np.abs(Xg - Xo).max()

    g.scbb_step(200)
    o.step(200)
    er, eu, ex = errors()
    assert er < 1e-5, er
    assert eu < 1e-5, eu
    assert ex < 1e-4, ex
    d = g.scbb_get_diag()
    vo, co = o.capsule(0)
    assert abs(d["volume"][0] - vo) / vo < 1e-5
    assert np.abs(d["com"][0] - co).max() < 1e-4
    g.scbb_step(800)
    o.step(800)
    er, eu, ex = errors()
    assert er < 1e-5, er
    assert eu < 1e-4, eu
    assert ex < 1e-4, ex


def test_pp_repulsion_two_capsules():
    """Particle-particle repulsion (Eq. 26, eps = 0.5, d0 = 1.25) between two capsules whose surfaces are 0.5
    apart: the node forces of the first step (elastic + repulsion) match the oracle's."""
    caps = [inputs.Capsule(centre=(10.3, 12.1, 12.2), radius=4.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0),
            inputs.Capsule(centre=(18.8, 12.0, 12.3), radius=4.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0)]
    p = inputs.Problem(name="pp", nx=32, ny=24, nz=24, walls=0, coupling=1, psi_kind=0, capsules=caps,
                       noise=1e-4, seed=5)
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(1)
    o.step(1)
    _, _, Fg = g.scbb_get_vertices()
    _, _, Fo = o.vertices()
    X, _, _ = o.vertices()
    # the repulsion is active: compare with the elastic-only force of the same shapes
    assert np.abs(Fo).max() > 0.05
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()


def test_pp_repulsion_across_the_periodic_edge_and_far_capsules():
    """The repulsion's capsule filter (bounding spheres within d0) keeps every nonzero term: two capsules 0.5
    apart across the periodic x edge repel as the oracle has it, while a third one far from both gets no
    repulsion (its node forces are the elastic ones, as in the oracle)."""
    caps = [inputs.Capsule(centre=(4.1, 12.1, 12.2), radius=4.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0),
            inputs.Capsule(centre=(32 - 4.4, 12.0, 12.3), radius=4.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0),
            inputs.Capsule(centre=(16.2, 12.3, 12.1), radius=3.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0)]
    p = inputs.Problem(name="pp2", nx=32, ny=24, nz=24, walls=0, coupling=1, psi_kind=0, capsules=caps,
                       noise=1e-4, seed=6)
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(1)
    o.step(1)
    _, _, Fg = g.scbb_get_vertices()
    _, _, Fo = o.vertices()
    assert np.abs(Fo).max() > 0.05
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()


def test_ibm_capsule_in_onsite_shear():
    """A capsule in shear imposed by on-site velocity planes (Zou and He), the setup of Sec. III.A: a single
    component mixture (G = 0, rho^A = rho^B = 0.5), resting walls, planes z = 1 and nz - 2 at -+U along x, a
    soft capsule (kappa_V = 1) at the centre coupled by the 2-point immersed boundary; 100 steps against the
    oracle: densities within 1e-5 relative, vertex positions within 1e-4, velocities within 1e-4 of max|u| (the
    immersed-boundary velocities carry the FP32 rounding of the vertex positions through the stencil weights,
    a few 1e-5 of max|u|, as in the 1000-step case)."""
    nz = 24
    cap = inputs.Capsule(centre=(12.3, 11.8, 11.6), radius=5.0, subdiv=3, kS=0.01, kB=1e-3, kV=1.0)
    p = inputs.Problem(name="shear", nx=24, ny=24, nz=nz, walls=1, coupling=1, psi_kind=0, G=0.0,
                       capsules=[cap], noise=0.0, seed=3, u_lo=(-0.01, 0.0, 0.0), u_hi=(0.01, 0.0, 0.0),
                       wall_kind=1)
    A = np.full((nz, 24, 24), 0.5)
    g = _sim(p, rhoA=A, rhoB=A)
    o = O.OracleSim(p, A, A)
    g.scbb_step(100)
    o.step(100)
    (ga, gb, gu), (oa, ob, ou) = g.scbb_get_fields(), o.fields()
    fl = oa + ob > 0
    assert (np.abs(ga - oa)[fl] / oa[fl]).max() < 1e-5
    assert (np.abs(gb - ob)[fl] / ob[fl]).max() < 1e-5
    assert np.abs(gu - ou).max() < 1e-4 * np.abs(ou).max()
    assert np.abs(g.scbb_get_vertices()[0] - o.vertices()[0]).max() < 1e-4

"""State save and load (scbb_save, scbb_load): steps after a load continue as they would have from the saved
state, on the same context or on a second context of the same shape."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _bb_box():
    cap = inputs.Capsule(centre=(15.3, 11.8, 12.6), radius=6.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=0.3)
    return inputs.Problem(name="state-bb", nx=32, ny=24, nz=26, walls=1, coupling=0, psi_kind=0, z_interface=13,
                          capsules=[cap], noise=1e-4, seed=13, u_lo=(-0.002, 0, 0), u_hi=(0.002, 0, 0))


def _state(sim):
    a, b, u = sim.scbb_get_fields()
    X = sim.scbb_get_vertices()[0] if sim.nm else np.zeros((0, 3))
    own = sim.scbb_get_owner()[0] if sim.nm else None
    return a, b, u, X, own


def test_fluid_resume_is_exact():
    """A sheared two-component fluid: 11 steps, save, 7 steps; load, the same 7 steps: identical bits (the
    fluid kernels are deterministic; an odd step count also exercises the lattice parity)."""
    from paper_1904_11386_gb300 import scbb

    p = inputs.small_problem(n=32, walls=1, coupling=1, capsule=False, noise=1e-3)
    p.u_lo, p.u_hi = (-0.01, 0, 0), (0.01, 0, 0)
    s = scbb.Sim(p)
    s.scbb_step(11)
    saved = s.scbb_save()
    s.scbb_step(7)
    first = _state(s)
    s.scbb_load(saved)
    s.scbb_step(7)
    for x, y in zip(first[:3], _state(s)[:3]):
        assert np.array_equal(x, y)


def test_bounce_back_resume_on_another_context():
    """The bounce-back box (wetting, fresh nodes, moving walls): 15 steps, save, 10 steps; the state loaded into
    a second context of the same shape, 10 steps: identical owners, densities within 1e-5 and vertices within
    1e-5 (float atomics on the element momenta order their additions differently from run to run)."""
    from paper_1904_11386_gb300 import scbb

    p = _bb_box()
    s1 = scbb.Sim(p)
    s1.scbb_step(15)
    saved = s1.scbb_save()
    s1.scbb_step(10)
    a1, b1, _, X1, o1 = _state(s1)
    s2 = scbb.Sim(p)
    s2.scbb_load(saved)
    s2.scbb_step(10)
    a2, b2, _, X2, o2 = _state(s2)
    assert np.array_equal(o1, o2)
    fl = a1 + b1 > 0
    assert np.abs(a1 - a2)[fl].max() < 1e-5 * a1[fl].max()
    assert np.abs(b1 - b2)[fl].max() < 1e-5 * b1[fl].max()
    assert np.abs(X1 - X2).max() < 1e-5
    # the same context, loaded back
    s1.scbb_load(saved)
    s1.scbb_step(10)
    a3, _, _, X3, o3 = _state(s1)
    assert np.array_equal(o1, o3)
    assert np.abs(a1 - a3)[fl].max() < 1e-5 * a1[fl].max()
    assert np.abs(X1 - X3).max() < 1e-5


def test_load_rejects_another_shape():
    from paper_1904_11386_gb300 import scbb

    s = scbb.Sim(inputs.small_problem(n=16, walls=1, coupling=1, capsule=False))
    other = scbb.Sim(inputs.small_problem(n=20, walls=1, coupling=1, capsule=False)).scbb_save()
    with pytest.raises(scbb.ScbbError):
        s.scbb_load(other)
    s.scbb_step(2)                      # the context is untouched

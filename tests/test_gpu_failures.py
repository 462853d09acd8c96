"""Failure detection on the GPU in forms that neither fault nor hang the device: the sticky device error word
(raised by the Mach guard, reported at the next synchronising call), the error state that follows it,
recovery from a saved state, and a boundary list that overflows a deliberately small capacity (the kernels
keep its first entries, skip the rest and flag it)."""
import re

import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _uniform(p, a=0.7, b=0.042):
    shape = (p.nz, p.ny, p.nx)
    return np.full(shape, a), np.full(shape, b)


def test_mach_guard_error_state_and_recovery():
    """A fluid-only periodic box (no membranes, so only the fluid kernels run) started at rest is saved; set to
    a uniform flow |u| = 0.4 above the guard's 0.3, its next step raises the device error word: scbb_sync
    returns SCBB_E_UNSTABLE, every later call SCBB_E_STATE.  scbb_load of the saved state clears it, and the
    restored context steps exactly like a fresh one."""
    from paper_1904_11386_gb300 import scbb

    p = inputs.Problem(name="mach", nx=32, ny=16, nz=12, walls=0, psi_kind=0, coupling=1, noise=0.0,
                       capsules=[], G=3.6)
    A, B = _uniform(p)
    sim = scbb.Sim(p, A, B)
    saved = sim.scbb_save()
    u = np.zeros((3,) + A.shape)
    u[0] = 0.4
    sim.scbb_set_density(A, B, u)
    sim.scbb_step(3)
    with pytest.raises(scbb.ScbbError, match="SCBB_E_UNSTABLE"):
        sim.scbb_sync()
    with pytest.raises(scbb.ScbbError, match="SCBB_E_STATE"):
        sim.scbb_step(1)
    with pytest.raises(scbb.ScbbError, match="SCBB_E_STATE"):
        sim.scbb_get_fields()
    sim.scbb_load(saved)
    sim.scbb_step(5)
    ref = scbb.Sim(p, A, B)
    ref.scbb_step(5)
    for x, y in zip(sim.scbb_get_fields(), ref.scbb_get_fields()):
        assert np.array_equal(x, y)


def test_boundary_list_overflow_is_flagged():
    """A capsule whose boundary-node list is given room for 64 entries (it needs several hundred): the
    classification at the initial state fills the first 64, skips the rest and raises the overflow flag (8),
    so scbb_set_density, the first synchronising call, reports SCBB_E_UNSTABLE; the same problem with the
    list sized from the membrane area runs and lists more than 64 nodes."""
    from paper_1904_11386_gb300 import scbb

    cap = inputs.Capsule(centre=(12.3, 11.8, 12.6), radius=6.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=0.0)
    p = inputs.Problem(name="overflow", nx=24, ny=24, nz=26, walls=1, coupling=0, psi_kind=0, z_interface=13,
                       capsules=[cap], noise=0.0, max_boundary=64)

    with pytest.raises(scbb.ScbbError, match="SCBB_E_UNSTABLE") as ei:
        scbb.Sim(p)
    flags = int(re.search(r"flags (\d+)", str(ei.value)).group(1))
    assert flags & 8, str(ei.value)
    ok = scbb.Sim(inputs.Problem(**{**p.__dict__, "max_boundary": 0}))
    ok.scbb_step(2)
    ok.scbb_sync()
    assert ok.scbb_get_owner()[1] > 64

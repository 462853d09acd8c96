"""Host input and output of the fields through the C ABI (scbb_set_density, scbb_get_fields).  The FP64
arrays cross the link as they are and are converted on the device, in the spare lattice; a box too small to
stage 5 N floats and 5 N doubles there converts on the host instead.  Checked: pinned and pageable host
arrays give the same bits in both directions, the device and host conversions agree, and a state set from
FP64 fields reads back as its FP32 rounding where the equilibrium holds it exactly."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pinned(n):
    import torch

    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()


def test_pinned_and_pageable_fields_agree():
    from paper_1904_11386_gb300 import scbb

    p = inputs.small_problem(n=24, walls=1, coupling=1, capsule=False, noise=1e-3, seed=61)
    A, B = p.initial_density()
    N = p.n_nodes
    s1 = scbb.Sim(p, A, B)
    hA, hB = _pinned(N), _pinned(N)
    hA[:] = A.ravel()
    hB[:] = B.ravel()
    s2 = scbb.Sim(p, A, B, set_state=False)
    s2.scbb_set_density(hA, hB)
    for s in (s1, s2):
        s.scbb_step(5)
    out = (_pinned(N), _pinned(N), _pinned(3 * N))
    a1, b1, u1 = s1.scbb_get_fields()
    a2, b2, u2 = s2.scbb_get_fields(out=out)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(u1, u2)
    assert np.shares_memory(a2, out[0])
    s1.close()
    s2.close()


def test_host_fallback_matches_device_conversion():
    """A 2 x 2 x 3 box stages on the host; the same fields tiled into a 4 x 4 x 3 box stage on the device: the
    densities read back equal node for node after a step (each node's update is local to its neighbourhood,
    and the periodic tiling repeats it)."""
    from paper_1904_11386_gb300 import scbb

    rng = np.random.Generator(np.random.PCG64(62))
    small = inputs.Problem(name="s", nx=2, ny=2, nz=3, walls=0, psi_kind=0, coupling=1, noise=0.0)
    big = inputs.Problem(name="b", nx=4, ny=4, nz=3, walls=0, psi_kind=0, coupling=1, noise=0.0)
    A = 0.4 + 0.05 * rng.random((3, 2, 2))
    B = 0.3 + 0.05 * rng.random((3, 2, 2))
    s = scbb.Sim(small, A, B)
    b = scbb.Sim(big, np.tile(A, (1, 2, 2)), np.tile(B, (1, 2, 2)))
    s.scbb_step(1)
    b.scbb_step(1)
    sa, sb, su = s.scbb_get_fields()
    ba, bb, bu = b.scbb_get_fields()
    assert np.array_equal(np.tile(sa, (1, 2, 2)), ba) and np.array_equal(np.tile(sb, (1, 2, 2)), bb)
    assert np.array_equal(np.tile(su, (1, 1, 2, 2)), bu)
    s.close()
    b.close()


def test_fields_read_back_at_step_zero():
    """A state set from FP64 fields at rest reads back as those fields to FP32 rounding (the lattice holds the
    equilibrium populations as the nodes pull them) and at rest, in a periodic box."""
    from paper_1904_11386_gb300 import scbb

    p = inputs.Problem(name="z", nx=16, ny=12, nz=10, walls=0, psi_kind=0, coupling=1, noise=0.0)
    rng = np.random.Generator(np.random.PCG64(63))
    A = 0.5 + 0.1 * rng.random((p.nz, p.ny, p.nx))
    B = 0.2 + 0.1 * rng.random((p.nz, p.ny, p.nx))
    sim = scbb.Sim(p, A, B)
    a, b, u = sim.scbb_get_fields()
    assert np.abs(a - A).max() < 4e-7 * A.max()
    assert np.abs(b - B).max() < 4e-7 * B.max()
    assert np.abs(u).max() < 1e-6
    sim.close()

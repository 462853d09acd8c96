"""The bulk kernel's block-shape autotuner (scbb_autotune): the shape it keeps changes the speed, not the
results."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pair(p):
    from paper_1904_11386_gb300 import scbb

    return scbb.Sim(p), scbb.Sim(p)


def test_one_lattice_contexts_keep_their_shape():
    """64^3 periodic droplet: its one lattice is updated in place, so the autotuner times nothing (a timing
    launch would advance the state), reports no shape, and leaves the state as it was: the context then agrees
    bit for bit with an untouched one after 20 steps.  (The quad form's shapes are compared bit for bit in
    test_gpu_staged.py.)"""
    a, b = _pair(inputs.cfg_adjoint(n=64, R_drop=16.0))
    assert a.scbb_autotune(3) == -1
    a.scbb_step(20)
    b.scbb_step(20)
    fa, fb = a.scbb_get_fields(), b.scbb_get_fields()
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


def test_bounce_back_results_do_not_depend_on_the_shape():
    """A 44^3 box of the batched sweep with its capsule, 20 bounce-back steps: identical owners, densities
    within 1e-5 (float atomics on the element momenta make the two runs differ at rounding level)."""
    p = inputs.cfg_batch48()[0]
    a, b = _pair(p)
    assert 0 <= a.scbb_autotune(3) <= 3
    a.scbb_step(20)
    b.scbb_step(20)
    assert np.array_equal(a.scbb_get_owner()[0], b.scbb_get_owner()[0])
    (aa, ab, _), (ba, bb, _) = a.scbb_get_fields(), b.scbb_get_fields()
    fl = ba + bb > 0
    assert np.abs(aa - ba)[fl].max() < 1e-5 * np.abs(ba[fl]).max()
    assert np.abs(ab - bb)[fl].max() < 1e-5 * np.abs(bb[fl]).max()


def test_general_kernel_has_no_shapes():
    from paper_1904_11386_gb300 import scbb

    import dataclasses

    # tau != 1 with nx not a multiple of 4 runs the general fused kernel
    s = scbb.Sim(dataclasses.replace(inputs.small_problem(n=16, nx=37, walls=1, coupling=1, capsule=False), tau=0.8))
    assert s.scbb_autotune(2) == -1
    s.scbb_step(2)

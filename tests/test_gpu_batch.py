"""Batches of independent contexts (scbb_batch_*): stepping contexts together, with pairs of steps of all of
them replayed from one multi-branch CUDA graph, gives each context the state it gets when stepped alone --
bit-exact for the fluid, and for the bounce-back coupling identical owner fields with populations and
vertices within 1e-5 (its element momenta are float atomics, whose summation order is free)."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _boxes():
    out = []
    for k, (nx, ny, nz) in enumerate([(44, 40, 36), (40, 48, 44), (52, 44, 40)]):
        cap = inputs.Capsule(centre=(nx / 2 + 0.3, ny / 2 - 0.2, nz / 2 + 0.4), radius=6.0, subdiv=3, kS=0.01,
                             kB=1e-3, kV=2.0, colour=(-0.1, 0.0, 0.1)[k])
        out.append(inputs.Problem(name=f"b{k}", nx=nx, ny=ny, nz=nz, walls=1, coupling=0, psi_kind=0,
                                  z_interface=nz // 2, capsules=[cap], noise=1e-4, seed=30 + k))
    out.append(inputs.small_problem(n=32, walls=1, coupling=1, capsule=False, noise=1e-3, seed=34))
    return out


def test_batch_equals_contexts_stepped_alone():
    from paper_1904_11386_gb300 import scbb

    probs = _boxes()
    alone = [scbb.Sim(p) for p in probs]
    together = [scbb.Sim(p) for p in probs]
    batch = scbb.Batch(together)
    for s in alone:
        s.scbb_step(1)
        s.scbb_step(13)
    batch.scbb_batch_step(1)       # the first step of each context runs launch by launch
    batch.scbb_batch_step(13)      # then pairs replay from the batch graph, and one step is left over
    for p, a, b in zip(probs, alone, together):
        assert a.scbb_launch_count() == b.scbb_launch_count()
        fa, fb = a.scbb_get_populations(), b.scbb_get_populations()
        if p.coupling == 0:
            oa, _, _ = a.scbb_get_owner()
            ob, _, _ = b.scbb_get_owner()
            assert np.array_equal(oa, ob)
            assert np.abs(fa - fb).max() < 1e-5 * np.abs(fa).max()
            assert np.abs(a.scbb_get_vertices()[0] - b.scbb_get_vertices()[0]).max() < 1e-5
        else:
            assert np.array_equal(fa, fb)
    # a context stepped on its own between batch steps stays ordered with the batch
    together[0].scbb_step(1)
    alone[0].scbb_step(1)
    batch.scbb_batch_step(2)
    alone[0].scbb_step(2)
    oa, _, _ = alone[0].scbb_get_owner()
    ob, _, _ = together[0].scbb_get_owner()
    assert np.array_equal(oa, ob)
    batch.close()

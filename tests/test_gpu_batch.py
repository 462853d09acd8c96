"""Batches of independent contexts (scbb_batch_*).  The boxes' bulk phases share one persistent cooperative
launch per step (kernel A over every box, a bounded grid barrier, kernel B over every box's work items), and
pairs of steps of the whole batch replay from one CUDA graph.  Checked: each context ends where it ends when
stepped alone (identical owner fields; populations and vertices at FP32 rounding -- the batch kernel is another
compiled kernel and the element momenta are float atomics); each box of a batch of uneven boxes, edges that are
not multiples of 4 included, against the FP64 oracle; and the grid barrier's bounded wait, which, forced to give
up, reports SCBB_E_TIMEOUT without hanging and leaves a context that scbb_load restores."""
import os

import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(sims, shared=True):
    """A batch of sims whose bulk phases share one persistent launch (shared=True) or keep one each."""
    from paper_1904_11386_gb300 import scbb

    old = os.environ.get("SCBB_BATCH_PERSISTENT")
    os.environ["SCBB_BATCH_PERSISTENT"] = "1" if shared else "0"
    try:
        return scbb.Batch(sims)
    finally:
        if old is None:
            del os.environ["SCBB_BATCH_PERSISTENT"]
        else:
            os.environ["SCBB_BATCH_PERSISTENT"] = old


def _dilate(mask):
    """mask and its 18 D3Q19 neighbours (periodic in x and y, clipped in z)."""
    out = mask.copy()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) in (1, 2):
                    sh = np.roll(np.roll(mask, dy, 1), dx, 2)
                    if dz == 1:
                        sh = np.concatenate([np.zeros_like(sh[:1]), sh[:-1]])
                    elif dz == -1:
                        sh = np.concatenate([sh[1:], np.zeros_like(sh[:1])])
                    out |= sh
    return out


def _boxes():
    out = []
    for k, (nx, ny, nz) in enumerate([(44, 40, 36), (41, 47, 43), (52, 45, 40)]):
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
    batch = _batch(together)
    assert batch.scbb_batch_shared_bulk()
    for s in alone:
        s.scbb_step(1)
        s.scbb_step(13)
    batch.scbb_batch_step(1)       # the first step of each context runs launch by launch
    batch.scbb_batch_step(13)      # then pairs replay from the batch graph, and one step is left over
    for k, (p, a, b) in enumerate(zip(probs, alone, together)):
        # the shared launch replaces each context's two bulk kernels; it is counted on the first context
        assert b.scbb_launch_count() == a.scbb_launch_count() - 2 * 14 + (14 if k == 0 else 0)
        fa, fb = a.scbb_get_populations(), b.scbb_get_populations()
        assert np.abs(fa - fb).max() < 1e-5 * np.abs(fa).max()
        if p.coupling == 0:
            oa, _, _ = a.scbb_get_owner()
            ob, _, _ = b.scbb_get_owner()
            assert np.array_equal(oa, ob)
            assert np.abs(a.scbb_get_vertices()[0] - b.scbb_get_vertices()[0]).max() < 1e-5
    # a context stepped on its own between batch steps stays ordered with the batch
    together[0].scbb_step(1)
    alone[0].scbb_step(1)
    batch.scbb_batch_step(2)
    alone[0].scbb_step(2)
    oa, _, _ = alone[0].scbb_get_owner()
    ob, _, _ = together[0].scbb_get_owner()
    assert np.array_equal(oa, ob)
    batch.close()


def test_batch_against_oracle():
    """Three boxes of the sweep's kind (edges 41, 44 and 50: one quad-form and two node-form lattices), each
    with a capsule of its own colour and shear modulus at the interface, 10 steps of the batch with its shared
    bulk phase and 10 of the same batch with one bulk phase per box, each against the FP64 oracle: owner fields
    identical, densities within 1e-5 relative except next to the membrane (boundary
    nodes, nodes that turned fresh during the run, and their neighbours), which are held to 2e-3.  Two discrete
    decisions there can come out differently in FP32 and FP64 without changing the owner field: a fresh node's
    density carries Eq. 18, which multiplies the global mass error by C0 sum(rho_init) / rho_init^c / V_sys
    (about 0.6 per unit of mass here for the minority component), so the FP32 state's total mass, one rounding
    of about 2e-8 of itself away from the oracle's, moves it by a few 1e-4; and a link that crosses the
    membrane next to a shared edge can be given the neighbouring element, whose velocity enters its bounce-back
    (the 44-wide box meets one at step 9: 8e-4 at that node, and 3.5e-4 on the vertices of the two elements).
    Either element belongs to the same capsule, which therefore receives the same momentum: the mean of each
    capsule's vertices is held to 1e-5, single vertices to 1e-3."""
    from oracle import oracle as O
    from paper_1904_11386_gb300 import scbb

    probs = []
    for k, (L, col, kS) in enumerate([(41, -0.1, 0.003), (44, 0.05, 0.01), (50, 0.1, 0.03)]):
        cap = inputs.Capsule(centre=(L / 2 + 0.3, L / 2 - 0.2, L / 2 - 5.0), radius=6.0, subdiv=3, kS=kS,
                             kB=0.01 * kS * 36.0, kV=2.0, colour=col)
        probs.append(inputs.Problem(name=f"sweep{k}", nx=L, ny=L, nz=L, walls=1, psi_kind=0, coupling=0,
                                    z_interface=L // 2, capsules=[cap], noise=1e-4, seed=200 + k))
    oracles = []
    for p in probs:
        o = O.OracleSim(p)
        own = o.owner()
        near = np.zeros_like(own, bool)
        for _ in range(10):
            o.step(1)
            nown = o.owner()
            near |= nown != own                      # fresh nodes
            near |= _dilate(nown != 1) & (nown == 1)  # boundary nodes inside the membrane
            near |= _dilate(nown == 1) & (nown != 1)  # and outside it
            own = nown
        oracles.append((o, _dilate(near)))
    for shared in (True, False):
        sims = [scbb.Sim(p) for p in probs]
        batch = _batch(sims, shared)
        assert batch.scbb_batch_shared_bulk() == shared
        batch.scbb_batch_step(10)
        for p, g, (o, near_fresh) in zip(probs, sims, oracles):
            assert np.array_equal(g.scbb_get_owner()[0], o.owner())
            ga, gb, _ = g.scbb_get_fields()
            oa, ob, _ = o.fields()
            fl = oa + ob > 0
            err = np.maximum(np.abs(ga - oa) / np.where(fl, oa, 1.0), np.abs(gb - ob) / np.where(fl, ob, 1.0))
            err[~fl] = 0.0
            assert err[~near_fresh].max() < 1e-5, (p.name, shared, err[~near_fresh].max())
            assert err.max() < 2e-3, (p.name, shared, err.max())
            # the crossed-element event moves one element's momentum to its neighbour: vertices there differ by
            # a few 1e-4, while the capsule's momentum, and so the mean of its vertices, is the same either way
            gx, ox = g.scbb_get_vertices()[0], o.vertices()[0]
            assert np.abs(gx - ox).max() < 1e-3
            assert np.abs(gx.mean(0) - ox.mean(0)).max() < 1e-5
        batch.close()


def test_batch_grid_barrier_timeout_and_recovery():
    """The grid barrier between the two kernels of the shared bulk phase waits a bounded number of polls.  With
    the limit set to 0 every block but the last gives up at once: the step is left incomplete, bit 4 of each
    context's device error word is raised, the next synchronising call reports SCBB_E_TIMEOUT and later calls
    SCBB_E_STATE.  A state saved before restores the context, and with the default limit the batch steps on and
    matches a context stepped alone."""
    from paper_1904_11386_gb300 import scbb

    probs = _boxes()[:2]
    sims = [scbb.Sim(p) for p in probs]
    saved = [s.scbb_save() for s in sims]
    batch = _batch(sims)
    batch.scbb_batch_set_wait_limit(0)
    batch.scbb_batch_step(1)
    with pytest.raises(scbb.ScbbError, match="SCBB_E_TIMEOUT"):
        sims[0].scbb_sync()
    with pytest.raises(scbb.ScbbError, match="SCBB_E_STATE"):
        sims[0].scbb_step(1)
    with pytest.raises(scbb.ScbbError, match="SCBB_E_TIMEOUT"):
        sims[1].scbb_sync()
    for s, b in zip(sims, saved):
        s.scbb_load(b)
    batch.scbb_batch_set_wait_limit(1 << 22)
    batch.scbb_batch_step(4)
    ref = scbb.Sim(probs[0])
    ref.scbb_step(4)
    assert np.array_equal(sims[0].scbb_get_owner()[0], ref.scbb_get_owner()[0])
    fa, fb = sims[0].scbb_get_populations(), ref.scbb_get_populations()
    assert np.abs(fa - fb).max() < 1e-5 * np.abs(fa).max()
    batch.close()

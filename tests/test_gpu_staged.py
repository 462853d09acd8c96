"""The staged forms of the two bulk kernels (inputs brought into shared memory by bulk asynchronous copies on
mbarriers) against the unstaged forms, and their bounded waits.

The staged kernels move the same values through shared memory and run the same collision arithmetic, so a
run with them equals a run without them (SCBB_BULK_STAGED=0, in a child process: the switches are read once per
process) bit for bit: FP32 and FP16 storage, walls and periodic z, the immersed-boundary mode.  So does kernel
B's pair form (two threads per quad, one per component; the default) against its quad form (SCBB_BULK_PAIR=0)
in every block shape of the quad form (the ring and stage layout depend on it).  The single fused kernels
(SCBB_BULK_VARIANT=4: the first build's row-vectorised kernel; 2: the general kernel, two lattices) give the
same step to FP32 rounding (1e-5 of the largest population; the immersed boundary's coupled steps carry a few ulps
of the different summation orders).  A wait limit of 0 makes the
waits give up: the next synchronising call reports SCBB_E_TIMEOUT, later calls SCBB_E_STATE, and a saved
state restores the context, which then steps like a fresh one."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# problem name -> (constructor source, steps); the source is evaluated here and in the child process
CASES = {
    "walls64": ("inputs.Problem(name='w', nx=64, ny=40, nz=30, walls=1, psi_kind=0, coupling=1, z_interface=15, "
                "u_lo=(-0.004, 0.0, 0.0), u_hi=(0.004, 0.001, 0.0), noise=1e-3, seed=41)", 12),
    "periodic128": ("inputs.Problem(name='p', nx=128, ny=24, nz=20, walls=0, psi_kind=0, coupling=1, "
                    "droplet=(60.0, 12.0, 10.0, 6.0), noise=1e-3, seed=42)", 9),
    "ibm64": ("inputs.small_problem(n=64, walls=1, coupling=1, capsule=True, noise=1e-3, seed=43, radius=6.0)", 6),
    "fp16_64": ("dataclasses.replace(inputs.Problem(name='h', nx=64, ny=36, nz=26, walls=1, psi_kind=0, "
                "coupling=1, z_interface=13, noise=1e-3, seed=44), storage=1)", 8),
    "fp16dev_64": ("dataclasses.replace(inputs.Problem(name='d', nx=64, ny=36, nz=26, walls=1, psi_kind=0, "
                   "coupling=1, z_interface=13, noise=1e-3, seed=45), storage=3)", 8),
}

_CHILD = r"""
import dataclasses, os, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_1904_11386_gb300 import inputs, scbb
p = {src}
sim = scbb.Sim(p)
sim.scbb_step({steps})
np.save({out!r}, sim.scbb_get_populations())
"""


def _run_here(src, steps):
    import dataclasses  # noqa: F401  (used by the constructor sources)

    from paper_1904_11386_gb300 import scbb

    sim = scbb.Sim(eval(src))
    sim.scbb_step(steps)
    f = sim.scbb_get_populations()
    sim.close()
    return f


def _run_child(src, steps, tmp_path, **env_vars):
    out = str(tmp_path / "f.npy")
    env = dict(os.environ, **env_vars)
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, src=src, steps=steps, out=out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


@pytest.mark.parametrize("name", list(CASES))
def test_staged_equals_unstaged(name, tmp_path):
    src, steps = CASES[name]
    ref = _run_child(src, steps, tmp_path, SCBB_BULK_STAGED="0")
    f = _run_here(src, steps)
    assert np.array_equal(f, ref), np.abs(f - ref).max()


@pytest.mark.parametrize("name", ["walls64", "ibm64"])
def test_pair_form_equals_quad_form_in_every_shape(name, tmp_path):
    """Kernel B's pair form against its staged quad form in each block shape of the latter (threads per CTA,
    CTAs per SM, tile rows)."""
    src, steps = CASES[name]
    f = _run_here(src, steps)
    for shape in ("0", "1", "2", "3"):
        ref = _run_child(src, steps, tmp_path, SCBB_BULK_PAIR="0", SCBB_BULK_SHAPE=shape)
        assert np.array_equal(f, ref), (shape, np.abs(f - ref).max())


@pytest.mark.parametrize("name", ["walls64", "ibm64"])
def test_fused_kernels_agree(name, tmp_path):
    src, steps = CASES[name]
    f = _run_here(src, steps)
    scale = np.abs(f).max()
    for variant in ("4", "2"):
        ref = _run_child(src, steps, tmp_path, SCBB_BULK_VARIANT=variant)
        assert np.abs(f - ref).max() < 1e-5 * scale, (variant, np.abs(f - ref).max())


def test_staged_wait_timeout_and_recovery():
    from paper_1904_11386_gb300 import scbb

    p = eval(CASES["walls64"][0])
    sim = scbb.Sim(p)
    saved = sim.scbb_save()
    sim.scbb_set_wait_limit(0)
    sim.scbb_step(2)
    with pytest.raises(scbb.ScbbError, match="SCBB_E_TIMEOUT"):
        sim.scbb_sync()
    with pytest.raises(scbb.ScbbError, match="SCBB_E_STATE"):
        sim.scbb_step(1)
    sim.scbb_load(saved)
    sim.scbb_set_wait_limit(1 << 22)
    sim.scbb_step(5)
    ref = scbb.Sim(p)
    ref.scbb_step(5)
    assert np.array_equal(sim.scbb_get_populations(), ref.scbb_get_populations())
    sim.close()
    ref.close()

"""The allocation-free moments entry point (scbb_population_moments_noalloc) against scbb_get_diag.

It serves callers that cannot allocate device memory (a framework that owns the device allocator, or a
loop that must not take cudaMalloc's synchronisation): its scratch is a fixed device array inside the
library.  This file is collected last so that a
run stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _device_populations(sim):
    import torch

    f = sim.scbb_get_populations()                       # host [c][node][i], doubles of FP32 values
    soa = np.ascontiguousarray(f.transpose(0, 2, 1)).astype(np.float32)
    return torch.from_numpy(soa).cuda().contiguous()


def test_population_moments_noalloc_matches_get_diag():
    """Two problems of different sizes, one after the other (the second call reuses the scratch left by the
    first), each called twice: FP64 mass and momentum equal scbb_get_diag's to 1e-9 relative."""
    from paper_1904_11386_gb300 import scbb

    probs = [inputs.small_problem(n=20, walls=1, coupling=1, capsule=False, noise=1e-3, seed=21),
             inputs.Problem(name="p", nx=24, ny=16, nz=12, walls=0, psi_kind=0, coupling=1, z_interface=6,
                            noise=1e-3, seed=22, u_lo=(0, 0, 0), u_hi=(0, 0, 0))]
    for prob in probs:
        sim = scbb.Sim(prob)
        sim.scbb_step(7)
        ref = sim.scbb_get_diag()
        fdev = _device_populations(sim)
        for _ in range(2):
            out = scbb.scbb_population_moments_noalloc(fdev, prob.nx, prob.ny, prob.nz, prob.walls)
            assert np.allclose(out[:2], ref["mass"], rtol=1e-9, atol=0)
            scale = ref["mass"].sum()
            assert np.allclose(out[2:], ref["momentum"], rtol=1e-9, atol=1e-12 * scale)
        sim.close()


def test_population_moments_noalloc_grid_stride():
    """A 64^3 two-component array with walls (262144 nodes, twice the 131072 threads of the launch, so every
    thread's grid-stride loop takes two nodes): the sums equal numpy's FP64 sums of the same FP32 values to
    1e-9 relative."""
    import torch

    from paper_1904_11386_gb300 import scbb

    n = 64
    rng = np.random.Generator(np.random.PCG64(23))
    f = rng.uniform(0.0, 0.1, size=(2, 19, n * n * n)).astype(np.float32)
    out = scbb.scbb_population_moments_noalloc(torch.from_numpy(f).cuda(), n, n, n, 1)
    fl = f.reshape(2, 19, n, n * n)[:, :, 1:n - 1].astype(np.float64)       # wall planes left out
    from oracle import oracle as O

    c = O.d3q19()[0].astype(np.float64)                  # [i][xyz], the order of scbb_get_populations
    tot = fl.sum(axis=3).sum(axis=2)                     # [c][i]
    ref = np.concatenate([tot.sum(axis=1), (tot.sum(axis=0)[:, None] * c).sum(axis=0)])
    assert np.allclose(out, ref, rtol=1e-9, atol=1e-9 * ref[:2].sum())


def test_population_moments_noalloc_rejects_oversize():
    import torch

    from paper_1904_11386_gb300 import scbb

    L = scbb.load()
    x = torch.zeros(4, device="cuda")
    out = np.zeros(5)
    rc = L.scbb_population_moments_noalloc(scbb.C.c_void_p(x.data_ptr()), 1000, 1000, 1000, 0,
                                           out.ctypes.data_as(scbb.C.c_void_p), None)
    assert rc == 1

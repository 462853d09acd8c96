"""The adjoint of the two-component fluid (scbb_adjoint_*) against FP64 central finite differences of the
oracle.

Loss: L = sum_x z rho^A(x, T) + 0.5 sum_x x rho^B(x, T) after T steps, a weighted centre of mass of each
component.  Two boxes: a droplet in a periodic 32^3 box (100 steps, exponential psi), and the 32^3 parity
fluid between walls moving at -+0.005 along x (200 steps, psi = rho; the moving-wall bounce-back and the walls'
virtual densities enter the adjoint).  The derivatives with respect to the Shan-Chen coupling G, the body
acceleration g and the initial densities (along a seeded direction) come from the FP32 adjoint kernels; the
oracle differences its own FP64 runs with steps of 1e-4 (G), 1e-5 (g) and 1e-5 (densities).  The agreement
asked of the adjoint is 1e-3 relative; the FP32 forward trajectory the adjoint follows differs from the FP64
one by about 1e-6.

With a capsule coupled by the immersed boundary (the parity box's capsule, stretched, 100 steps) the loss adds
a seeded weighting of the final vertex positions, and the gradients with respect to the membrane moduli kS, kB,
kV, the initial vertex positions (along a seeded direction), G and g_x are checked the same way."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-3


def _weights(p):
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    return z.astype(np.float64), 0.5 * x.astype(np.float64)


def _oracle_loss(p, rhoA0, rhoB0, steps):
    o = O.OracleSim(p, rhoA0, rhoB0)
    o.step(steps)
    a, b, _ = o.fields()
    wA, wB = _weights(p)
    return float((wA * a).sum() + (wB * b).sum())


def _gpu_grads(p, rhoA0, rhoB0, steps, K):
    from paper_1904_11386_gb300 import scbb

    sim = scbb.Sim(p, rhoA0, rhoB0)
    adj = scbb.Adjoint(sim, steps, K)
    adj.scbb_adjoint_forward()
    wA, wB = _weights(p)
    out = adj.scbb_adjoint_backward(wA, wB)
    a, b, _ = sim.scbb_get_fields()
    adj.close()
    sim.close()
    return out, float((wA * a).sum() + (wB * b).sum())


def _walls_problem():
    import dataclasses

    p = inputs.cfg_parity(coupling=1)
    return dataclasses.replace(p, capsules=[], u_lo=(-0.005, 0.0, 0.0), u_hi=(0.005, 0.0, 0.0))


CASES = {"periodic": (lambda: inputs.cfg_adjoint(n=32, R_drop=8.0), 100),
         "walls": (_walls_problem, 200)}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    make, steps = CASES[request.param]
    p = make()
    rhoA0, rhoB0 = p.initial_density()
    (dG, dg, drA, drB), L = _gpu_grads(p, rhoA0, rhoB0, steps, 16)   # a ragged last segment (100 and 200 steps)
    return p, rhoA0, rhoB0, dG, dg, drA, drB, L, steps


def test_loss_matches_oracle(case):
    p, rhoA0, rhoB0, *_, L, T = case
    assert abs(L - _oracle_loss(p, rhoA0, rhoB0, T)) < 1e-5 * abs(L)


def test_dG_against_fd(case):
    import dataclasses

    p, rhoA0, rhoB0, dG, *_, T = case
    h = 1e-4
    fd = (_oracle_loss(dataclasses.replace(p, G=p.G + h), rhoA0, rhoB0, T) -
          _oracle_loss(dataclasses.replace(p, G=p.G - h), rhoA0, rhoB0, T)) / (2 * h)
    assert abs(dG - fd) < RTOL * abs(fd), (dG, fd)


def test_dg_against_fd(case):
    """The gradient vector dL/dg against its three central differences, relative to its norm: a component that
    the box's symmetry makes nearly zero (for example across a shear flow) carries the absolute FP32 error of the
    whole vector, a few units against about 1e6 here, and is not held to 1e-3 of itself."""
    import dataclasses

    p, rhoA0, rhoB0, _, dg, *_, T = case
    h = 1e-5
    fd = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd[k] = (_oracle_loss(dataclasses.replace(p, g=tuple(e)), rhoA0, rhoB0, T) -
                 _oracle_loss(dataclasses.replace(p, g=tuple(-e)), rhoA0, rhoB0, T)) / (2 * h)
    assert np.linalg.norm(dg - fd) < RTOL * np.linalg.norm(fd), (dg, fd)


def test_drho0_against_fd(case):
    """Directional derivative along a seeded direction of both initial density fields."""
    p, rhoA0, rhoB0, _, _, drA, drB, _, T = case
    rng = np.random.Generator(np.random.PCG64(21))
    vA, vB = rng.standard_normal(rhoA0.shape), rng.standard_normal(rhoB0.shape)
    h = 1e-5
    fd = (_oracle_loss(p, rhoA0 + h * vA, rhoB0 + h * vB, T) -
          _oracle_loss(p, rhoA0 - h * vA, rhoB0 - h * vB, T)) / (2 * h)
    ad = float((drA * vA).sum() + (drB * vB).sum())
    assert abs(ad - fd) < RTOL * abs(fd), (ad, fd)


def test_checkpoint_interval_does_not_change_the_gradient(case):
    """Recomputation from checkpoints is exact: one segment of T steps and segments of 7 steps give the same
    gradients bit for bit (the kernels are deterministic)."""
    p, rhoA0, rhoB0, dG, dg, drA, drB, _, T = case
    for K in (T, 7):
        (dG2, dg2, drA2, drB2), _ = _gpu_grads(p, rhoA0, rhoB0, T, K)
        assert dG2 == dG and np.array_equal(dg2, dg)
        assert np.array_equal(drA2, drA) and np.array_equal(drB2, drB)


def test_autograd_function(case):
    """fluid_rollout as a torch.autograd.Function: the gradients of the same loss through torch equal the
    direct adjoint call."""
    import torch

    from paper_1904_11386_gb300 import scbb

    p, rhoA0, rhoB0, dG, dg, drA, drB, _, T = case
    G = torch.tensor(p.G, dtype=torch.float64, requires_grad=True)
    g = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    a0 = torch.tensor(rhoA0, requires_grad=True)
    b0 = torch.tensor(rhoB0, requires_grad=True)
    a, b = scbb.fluid_rollout(p, T, 16, G, g, a0, b0)
    wA, wB = (torch.from_numpy(w) for w in _weights(p))
    loss = (wA * a).sum() + (wB * b).sum()
    loss.backward()
    assert G.grad.item() == dG
    assert np.array_equal(g.grad.numpy(), dg)
    assert np.array_equal(a0.grad.numpy(), drA) and np.array_equal(b0.grad.numpy(), drB)


def test_unsupported_contexts_are_rejected():
    """Bounce-back meshes and 16-bit storage are outside the adjoint."""
    from paper_1904_11386_gb300 import scbb

    for p in (inputs.small_problem(n=16, walls=1, coupling=0, capsule=True),
              inputs.small_problem(n=16, walls=1, coupling=1, capsule=False)):
        if not p.capsules:
            p.storage = 1
        sim = scbb.Sim(p)
        with pytest.raises(scbb.ScbbError):
            scbb.Adjoint(sim, 10, 5)
        sim.close()


# ---- a capsule coupled by the immersed boundary
CAP_STEPS = 100


def _capsule_problem(kS=0.005, kB=5e-4, kV=1.0, G=None, g=(0.0, 0.0, 0.0)):
    """The 32^3 parity box (walls, psi = rho, flat interface at z = 16) with its s = 3 capsule, initially
    stretched by diag(1.12, 0.95, 0.92) about a centre off the lattice planes.  A vertex on a lattice plane
    sits on a kink of the 2-point stencil (Eq. 7), where the loss has no derivative; the icosphere's poles and
    great-circle vertices land on such planes about an integer centre."""
    import dataclasses

    p = inputs.cfg_parity(coupling=1)
    cap = dataclasses.replace(p.capsules[0], centre=(16.31, 15.77, 20.13), kS=kS, kB=kB, kV=kV,
                              deform=np.diag([1.12, 0.95, 0.92]))
    return dataclasses.replace(p, capsules=[cap], G=p.G if G is None else G, g=g)


def _capsule_seeds(p):
    rng = np.random.Generator(np.random.PCG64(11))
    nv = len(p.capsules[0].mesh()[0])
    cX = rng.standard_normal((nv, 3))
    dX = rng.standard_normal((nv, 3))
    z = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")[0]
    return cX, dX, 0.01 * z.astype(np.float64)


def _capsule_oracle_loss(p, X0=None):
    cX, _, wA = _capsule_seeds(p)
    o = O.OracleSim(p)
    if X0 is not None:
        o.set_vertices(X0)
    o.step(CAP_STEPS)
    a, _, _ = o.fields()
    return float((cX * o.vertices()[0]).sum() + (wA * a).sum())


def _capsule_gpu(p, K):
    from paper_1904_11386_gb300 import scbb

    cX, _, wA = _capsule_seeds(p)
    sim = scbb.Sim(p)
    adj = scbb.Adjoint(sim, CAP_STEPS, K)
    adj.scbb_adjoint_forward()
    X = sim.scbb_get_vertices()[0]
    a, _, _ = sim.scbb_get_fields()
    L = float((cX * X).sum() + (wA * a).sum())
    dmod, dX0, dG, dg = adj.scbb_adjoint_backward_capsule(cX, wA, None)
    X2 = sim.scbb_get_vertices()[0]
    adj.close()
    sim.close()
    return L, dmod, dX0, dG, dg, X, X2


@pytest.fixture(scope="module")
def capsule_case():
    p = _capsule_problem()
    return p, _capsule_gpu(p, 30)        # segments of 30, 30, 30 and 10 steps


def test_capsule_loss_matches_oracle(capsule_case):
    p, (L, *_, X, X2) = capsule_case
    assert abs(L - _capsule_oracle_loss(p)) < 1e-5 * abs(L)
    assert np.array_equal(X, X2)           # the backward pass leaves the vertices of step n in place


def test_capsule_moduli_against_fd(capsule_case):
    """dL/dkS, dL/dkB, dL/dkV against central differences of the FP64 oracle.  The steps (2e-5 of each
    modulus, 1e-6 for kV = 1) are small enough that no vertex crosses a stencil kink between the two runs."""
    p, (_, dmod, *_) = capsule_case
    cap = p.capsules[0]
    for k, (name, h) in enumerate([("kS", 1e-7), ("kB", 1e-8), ("kV", 1e-6)]):
        v = getattr(cap, name)
        fd = (_capsule_oracle_loss(_capsule_problem(**{name: v + h})) -
              _capsule_oracle_loss(_capsule_problem(**{name: v - h}))) / (2 * h)
        assert abs(dmod[0, k] - fd) < RTOL * abs(fd), (name, dmod[0, k], fd)


def test_capsule_initial_vertices_against_fd(capsule_case):
    """The gradient with respect to the initial positions (reference shape held) along a seeded direction."""
    p, (_, _, dX0, *_) = capsule_case
    _, d, _ = _capsule_seeds(p)
    X0 = p.capsules[0].mesh()[2]
    h = 1e-6
    fd = (_capsule_oracle_loss(p, X0 + h * d) - _capsule_oracle_loss(p, X0 - h * d)) / (2 * h)
    ad = float((dX0 * d).sum())
    assert abs(ad - fd) < RTOL * abs(fd), (ad, fd)


def test_capsule_fluid_parameters_against_fd(capsule_case):
    """dL/dG and dL/dg_x: the fluid's parameters reach the loss through the flow that carries the capsule and
    through the spread force the membrane puts back into the fluid."""
    p, (_, _, _, dG, dg, *_) = capsule_case
    h = 1e-6
    fd = (_capsule_oracle_loss(_capsule_problem(G=p.G + h)) - _capsule_oracle_loss(_capsule_problem(G=p.G - h))) / (2 * h)
    assert abs(dG - fd) < RTOL * abs(fd), (dG, fd)
    h = 1e-9
    fd = (_capsule_oracle_loss(_capsule_problem(g=(h, 0.0, 0.0))) -
          _capsule_oracle_loss(_capsule_problem(g=(-h, 0.0, 0.0)))) / (2 * h)
    assert abs(dg[0] - fd) < RTOL * abs(fd), (dg[0], fd)


def test_capsule_checkpoint_interval(capsule_case):
    """One segment of 100 steps gives the gradient of four segments to FP32 rounding, held to 1e-4 of the
    largest component (a tenth of the tolerance against the oracle).  The spread force and its adjoint are
    float atomic sums, so a recomputed step matches the forward one to rounding, not bit for bit, and the
    adjoint, a sum over 100 steps, moves by about 3e-5 of itself between two runs."""
    p, (_, dmod, dX0, dG, *_) = capsule_case
    _, dmod2, dX02, dG2, *_ = _capsule_gpu(p, CAP_STEPS)
    assert np.abs(dmod2 - dmod).max() < 1e-4 * np.abs(dmod).max()
    assert np.abs(dX02 - dX0).max() < 1e-4 * np.abs(dX0).max()
    assert abs(dG2 - dG) < 1e-4 * abs(dG)

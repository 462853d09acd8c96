"""The seeded synthetic workloads (paper_1904_11386_gb300/inputs.py): shapes and placement rules the
benchmark and the tests rely on.  No GPU needed."""
import numpy as np
import pytest

from paper_1904_11386_gb300 import inputs


def test_droplet_covering_placement():
    """300 capsules of radius 8 around the droplet of radius 70: all placed, centres at least 2R + 2 apart
    (periodic images included), in the shell from R_drop + R - 1.5 to 20 beyond, inside the box with a margin
    of R + 2, colours alternating +-0.05, softness beta = 100 (kS = 0.0388, kB = 0.01 kS R^2)."""
    p = inputs.cfg_droplet256()
    assert len(p.capsules) == 300
    c = np.array([cap.centre for cap in p.capsules])
    d = c[:, None, :] - c[None, :, :]
    d -= 256.0 * np.round(d / 256.0)
    dist = np.sqrt((d ** 2).sum(-1)) + np.eye(len(c)) * 1e9
    assert dist.min() >= 2 * 8.0 + 2.0
    r = np.linalg.norm(c - 128.0, axis=1)
    assert r.min() >= 70.0 + 8.0 - 1.5 - 1e-9 and r.max() <= 70.0 + 8.0 - 1.5 + 20.0 + 1e-9
    assert c.min() >= 8.0 + 2.0 and c.max() <= 256.0 - 8.0 - 2.0
    cols = np.array([cap.colour for cap in p.capsules])
    assert np.all(cols[::2] == 0.05) and np.all(cols[1::2] == -0.05)
    assert all(cap.kS == 0.0388 and abs(cap.kB - 0.01 * 0.0388 * 64.0) < 1e-15 for cap in p.capsules)
    assert sum(len(cap.mesh()[0]) for cap in p.capsules) == 192600


def test_janus_colours_split_at_the_centre():
    """Triangles whose centroid lies above the capsule's centre take the top colour, the others the bottom
    one; on a symmetric icosphere the two halves hold the same number of triangles."""
    cap = inputs.Capsule(centre=(10.0, 10.0, 12.3), radius=5.0, subdiv=3)
    ref, tri, _ = cap.mesh()
    col = inputs.janus_colours(cap, 0.3, -0.3)
    cz = ref[tri].mean(axis=1)[:, 2]
    assert col.shape == (len(tri),)
    assert np.all(col[cz > 12.3] == 0.3) and np.all(col[cz < 12.3] == -0.3)
    assert abs(int((col > 0).sum()) - int((col < 0).sum())) <= len(tri) // 20


def test_batch_sweep_boxes():
    """48 cubes with integer edges drawn uniformly from [40, 72] (both multiples of 4 and others occur, so the
    sweep exercises both forms of the bulk kernels), 11 colours over [-0.1, 0.1] and 4 shear moduli, seeds
    100 + k."""
    probs = inputs.cfg_batch48()
    assert len(probs) == 48
    assert all(p.nx == p.ny == p.nz and 40 <= p.nx <= 72 for p in probs)
    assert any(p.nx % 4 for p in probs) and any(p.nx % 4 == 0 for p in probs)
    assert sorted({round(p.capsules[0].colour, 12) for p in probs}) == sorted(
        {round(v, 12) for v in np.linspace(-0.1, 0.1, 11)})
    assert {p.capsules[0].kS for p in probs} == {0.001, 0.003, 0.01, 0.03}
    assert [p.seed for p in probs] == [100 + k for k in range(48)]


@pytest.mark.parametrize("freq", [1, 2, 3, 12])
def test_geodesic_sphere(freq):
    """The class-I geodesic sphere: 10 f^2 + 2 vertices and 20 f^2 triangles (f = 12: the paper's 1442 nodes
    and 2880 elements), every vertex on the unit sphere, a closed surface whose directed edges each appear once
    with their reverse once (consistent orientation, Euler characteristic 2), normals outward, and the
    discrete Gauss-Bonnet identity sum K_G A = 4 pi of the oracle's Meyer operators."""
    from oracle import oracle as O

    V, F = inputs.geodesic_sphere(freq)
    assert V.shape == (10 * freq * freq + 2, 3) and F.shape == (20 * freq * freq, 3)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-14)
    directed = {}
    for t in F:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            directed[(a, b)] = directed.get((a, b), 0) + 1
    assert all(n == 1 for n in directed.values())
    assert all((b, a) in directed for a, b in directed)
    assert len(V) - len(directed) // 2 + len(F) == 2
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    assert np.all(np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0)
    bend = O.bending(V * 7.0, F, 1.0)
    assert np.isclose((bend["KG"] * bend["A"]).sum(), 4 * np.pi, rtol=1e-12)

"""GPU parity of the half-way bounce-back coupling (Sec. II.C-II.E) against the FP64 oracle, through the C
ABI: classification, boundary collision with wetting, membrane coupling, fresh nodes."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1904_11386_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sim(prob, **kw):
    from paper_1904_11386_gb300 import scbb

    return scbb.Sim(prob, **kw)


def _small(colour=0.3, walls=1, seed=13, steps_noise=1e-4):
    cap = inputs.Capsule(centre=(15.3, 11.8, 12.6), radius=6.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=colour)
    return inputs.Problem(name="bbs", nx=32, ny=24, nz=26, walls=walls, coupling=0, psi_kind=0, z_interface=13,
                          capsules=[cap], noise=steps_noise, seed=seed, u_lo=(-0.002, 0, 0), u_hi=(0.002, 0, 0))


def _nbrs(mask):
    """mask and its 18 D3Q19 neighbours (periodic in all three directions: a wall plane's owner is its own)."""
    out = mask.copy()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) in (1, 2):
                    out |= np.roll(mask, (dz, dy, dx), (0, 1, 2))
    return out


def _step_with_band(o, steps):
    """Steps the oracle and returns the nodes next to the membrane over those steps: boundary nodes (a neighbour
    on another side) and nodes that turned fresh, with their neighbours (R15)."""
    own = o.owner()
    near = np.zeros_like(own, bool)
    for _ in range(steps):
        o.step(1)
        nown = o.owner()
        near |= nown != own
        for k in np.unique(nown):
            if k != 0xFFFF:
                near |= _nbrs(nown == k) & (nown != k) & (nown != 0xFFFF)
        own = nown
    return _nbrs(near)


def _cmp_band(prob, g, o, band):
    """R15's bounds for a free-running window in which a discrete decision next to the membrane can part FP32
    and FP64 (a fresh node's Eq. 18 factor, a link given the neighbouring element of the same capsule): densities
    within 1e-5 relative away from the membrane and 2e-3 next to it, single vertices within 1e-3, each capsule's
    mean vertex within 1e-5."""
    ga, gb, _ = g.scbb_get_fields()
    oa, ob, _ = o.fields()
    fl = oa + ob > 0
    err = np.maximum(np.abs(ga - oa) / np.where(fl, oa, 1.0), np.abs(gb - ob) / np.where(fl, ob, 1.0))
    err[~fl] = 0.0
    assert err[~band].max() < 1e-5, err[~band].max()
    assert err.max() < 2e-3, err.max()
    gx, ox = g.scbb_get_vertices()[0], o.vertices()[0]
    assert np.abs(gx - ox).max() < 1e-3
    off = np.cumsum([0] + list(o.nv))
    for k in range(len(o.nv)):
        assert np.abs(gx[off[k]:off[k + 1]].mean(0) - ox[off[k]:off[k + 1]].mean(0)).max() < 1e-5


def _cmp_u(g, o, band, away=1e-5, near=1e-3):
    """Output velocities (Eq. 5) against the oracle, as fractions of max|u|: away from the membrane band and
    everywhere.  Next to the membrane the fresh nodes' densities carry Eq. 18's amplified FP32 mass error (R23),
    and the interface's largest velocities sit there (max|u| 0.05-0.1)."""
    _, _, ug = g.scbb_get_fields()
    _, _, uo = o.fields()
    umax = np.abs(uo).max()
    d = np.abs(ug - uo).max(axis=0)
    assert d[~band].max() < away * umax, (d[~band].max() / umax)
    assert d.max() < near * umax, (d.max() / umax)


def _cmp_rho(g, o, tol=1e-5):
    ga, gb, _ = g
    oa, ob, _ = o
    fl = oa + ob > 0
    return max((np.abs(ga - oa)[fl] / oa[fl]).max(), (np.abs(gb - ob)[fl] / ob[fl]).max())


def test_bb_classification_matches_oracle():
    """Owner field and boundary-node count of the initial shapes equal the oracle's exactly."""
    for prob in (_small(), inputs.cfg_parity(coupling=0)):
        g = _sim(prob)
        o = O.OracleSim(prob)
        og, nb, _ = g.scbb_get_owner()
        assert np.array_equal(og, o.owner())
        assert nb == o.boundary_count()[0]


def test_bb_one_step_populations():
    """One step with bounce-back, virtual-density wetting and moving walls: every post-streaming population
    matches the oracle to FP32 accuracy, except at fresh nodes.  Their densities come from Eq. 18, which
    multiplies the global mass error by C0 = 2500 and by sum(rho_init)/rho_init^c (about 17 for the
    minority component): an FP32 mass sum uncertain by ~1e-6 of the total then moves a fresh density by
    ~1e-5 relative, so fresh nodes are held to 1e-4 relative."""
    p = _small()
    g = _sim(p)
    o = O.OracleSim(p)
    own0 = o.owner().ravel().copy()
    g.scbb_step(1)
    o.step(1)
    fresh = (o.owner().ravel() != own0)
    assert fresh.any()
    fg = g.scbb_get_populations()
    fo = o.populations()
    fluid = np.ones((p.nz, p.ny, p.nx), bool)
    fluid[[0, -1]] = False
    fluid = fluid.ravel()
    keep = fluid & ~fresh
    assert np.abs(fg[:, keep] - fo[:, keep]).max() < 2e-6 * np.abs(fo).max()
    assert (np.abs(fg[:, fresh] - fo[:, fresh]) / np.abs(fo[:, fresh])).max() < 1e-4


def test_bb_small_box_20_steps():
    """20 coupled steps (membrane forces with exchanged momenta, node update, re-classification, fresh nodes):
    densities within 1e-5 relative, vertex positions within 1e-4, identical owner fields; output velocities
    within 1e-5 of max|u| away from the membrane and 1e-3 next to it (measured 1.4e-6 and 5.6e-6)."""
    p = _small()
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(20)
    band = _step_with_band(o, 20)
    _cmp_u(g, o, band)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4
    assert o.fresh_count()[0] > 0


def test_bb_adsorb128_full_size():
    """The 128^3 bounce-back workload of the benchmark (walls sheared at 1e-4, exponential psi, s = 4 capsule
    of colour 0.05), launch configuration as timed: 3 steps against the oracle, every node; output velocities
    within 1e-5 of max|u| away from the membrane and 1e-3 next to it (measured 9.5e-7 and 2.0e-4)."""
    p = inputs.cfg_adsorb128(coupling=0)
    g = _sim(p)
    o = O.OracleSim(p)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    g.scbb_step(3)
    band = _step_with_band(o, 3)
    _cmp_u(g, o, band)
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4


def _three():
    caps = [inputs.Capsule(centre=(9.7, 10.2, 12.1), radius=5.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=0.05),
            inputs.Capsule(centre=(21.1, 10.6, 11.8), radius=5.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=-0.05),
            inputs.Capsule(centre=(15.6, 21.3, 12.4), radius=5.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=0.05)]
    return inputs.Problem(name="bb3", nx=32, ny=32, nz=24, walls=0, coupling=0, psi_kind=0,
                          droplet=(16.0, 16.0, 12.0, 7.0), capsules=caps, noise=1e-4, seed=15)


def _wrapping():
    """One capsule across the periodic x and y edges and a second one beside it."""
    caps = [inputs.Capsule(centre=(0.7, 27.4, 11.9), radius=5.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=0.05),
            inputs.Capsule(centre=(14.3, 13.8, 12.3), radius=6.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=-0.05)]
    return inputs.Problem(name="bbw", nx=32, ny=28, nz=24, walls=0, coupling=0, psi_kind=0, z_interface=12,
                          capsules=caps, noise=1e-4, seed=21)


# D3Q19 directions in the library's order (rest, +x, -x, +y, -y, +z, -z, then the face diagonals in pairs)
_C = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
               (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1),
               (0, 1, -1), (0, -1, 1)])


def _cut_links(prob, own, n):
    """(direction, neighbour, searched capsule) of every cut link of node n, from an owner field."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    o = own.ravel()
    z, r = divmod(int(n), nx * ny)
    y, x = divmod(r, nx)
    out = []
    for i in range(1, 19):
        zz = z + _C[i, 2]
        if prob.walls and not 0 <= zz < nz:
            continue
        m = (x + _C[i, 0]) % nx + nx * ((y + _C[i, 1]) % ny + ny * (zz % nz))
        if o[m] == 0xFFFF or o[m] == o[n]:
            continue
        out.append((i, m, int(o[n] if o[n] != 0 else o[m]) - 1))
    return out


def _check_elements(prob, g, o, exact):
    """Every cut link's element from the GPU list against the oracle's search on its own state (Sec. II.C: the
    crossing nearest the lower-index node).  exact: the two states are the same shapes (no steps yet), so every
    element must agree; after steps the FP32 and FP64 vertices differ by round-off and a link that meets a shared
    edge or vertex within it may pick the neighbouring triangle: then the two must share a vertex."""
    own = o.owner()
    nodes, elems, n_fb = g.scbb_get_boundary()
    assert len(nodes) == o.boundary_count()[0] and len(set(nodes.tolist())) == len(nodes)
    voff = np.cumsum([0] + list(o.nv))[:-1]
    tri = np.concatenate([np.asarray(t) + off for t, off in zip(o.tris, voff)])     # global vertex ids
    links = mismatch = 0
    fb0 = o.boundary_count()[1]
    for r, n in enumerate(nodes):
        cut = _cut_links(prob, own, n)
        assert cut, n
        want = -np.ones(18, np.int64)
        for i, m, cap in cut:
            want[i - 1] = o.crossed_element(cap, int(n), i)
        assert np.array_equal(want < 0, elems[r] < 0), (n, want, elems[r])
        for j in np.nonzero(want >= 0)[0]:
            links += 1
            if elems[r, j] != want[j]:
                mismatch += 1
                assert not exact, (n, j + 1, elems[r, j], want[j])
                assert set(tri[elems[r, j]]) & set(tri[want[j]]), (n, j + 1)
    fb = o.boundary_count()[1] - fb0
    assert links > 0
    assert mismatch <= 0.01 * links, (mismatch, links)
    assert n_fb <= fb + 2, (n_fb, fb)
    return links, mismatch


def test_bb_crossed_elements_match_oracle():
    """The crossed element of every cut link (the triangle-wise search with its atomic minimum over
    (crossing parameter, triangle id)) equals the oracle's node-wise search: one capsule between walls, the
    first configuration's capsule, three capsules in a periodic box, a capsule across the periodic edges; then
    again after 20 coupled steps (not the first configuration's: with bounce-back its A-filled capsule in the
    B-rich phase drives the flow past the Mach guard)."""
    for prob, steps in ((_small(), 20), (inputs.cfg_parity(coupling=0), 0), (_three(), 20), (_wrapping(), 20)):
        g = _sim(prob)
        o = O.OracleSim(prob)
        assert np.array_equal(g.scbb_get_owner()[0], o.owner())
        _check_elements(prob, g, o, exact=True)
        if not steps:
            g.close()
            continue
        g.scbb_step(steps)
        o.step(steps)
        assert np.array_equal(g.scbb_get_owner()[0], o.owner())
        _check_elements(prob, g, o, exact=False)
        g.close()


def _many():
    """64 capsules (81,920 triangles) on a 4 x 4 x 4 grid in a periodic 64^3 box across a flat interface: a list
    long enough for the thread-per-node boundary forms and the three-direction groups of the crossing search."""
    caps = []
    for k in range(64):
        i, j, l = k % 4, (k // 4) % 4, k // 16
        caps.append(inputs.Capsule(centre=(8.3 + 16 * i, 8.6 + 16 * j, 8.2 + 16 * l), radius=5.0, subdiv=3, kS=0.02,
                                   kB=1e-3, kV=2.0, colour=0.05 if k % 2 else -0.05))
    return inputs.Problem(name="bb64", nx=64, ny=64, nz=64, walls=0, coupling=0, psi_kind=0, z_interface=32,
                          capsules=caps, noise=1e-4, seed=23)


def test_bb_thread_forms_against_oracle():
    """The thread-per-node forms of the boundary pass (virtual densities, elements, boundary update), which
    lists of 65,536 nodes or more take, against the oracle: forced onto the small problems through a large
    list capacity (one step node by node, then 20 steps with R15's bounds), and on 64 capsules, whose list takes them by itself
    (the crossing search then runs three directions a thread): one step node by node, then 4 more with the
    owner field, the elements and each capsule's centre of mass.  (With 230,000 cut links a step, a few links
    that meet a shared edge within the FP32 / FP64 difference of the vertices pick the neighbouring triangle
    within those steps; the momentum they exchange then lands on other vertices, which moves single vertices by
    up to 3e-4 and single boundary densities by 1e-4 relative, in the warp-per-node forms alike.)"""
    import dataclasses
    for prob in (_small(), _three()):
        big = dataclasses.replace(prob, max_boundary=100000)
        g, o = _sim(big), O.OracleSim(prob)
        _check_elements(prob, g, o, exact=True)
        g.scbb_step(1)
        o.step(1)
        assert np.array_equal(g.scbb_get_owner()[0], o.owner())
        assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
        g.scbb_step(19)
        band = _step_with_band(o, 19)
        assert np.array_equal(g.scbb_get_owner()[0], o.owner())
        _cmp_band(prob, g, o, band)
        _check_elements(prob, g, o, exact=False)
        g.close()
    prob = _many()
    g, o = _sim(prob), O.OracleSim(prob)
    assert np.array_equal(g.scbb_get_owner()[0], o.owner())
    _check_elements(prob, g, o, exact=True)
    g.scbb_step(1)
    o.step(1)
    assert np.array_equal(g.scbb_get_owner()[0], o.owner())
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    assert np.abs(g.scbb_get_vertices()[0] - o.vertices()[0]).max() < 1e-4
    g.scbb_step(4)
    o.step(4)
    assert np.array_equal(g.scbb_get_owner()[0], o.owner())
    com = np.asarray(g.scbb_get_diag()["com"])
    assert max(np.abs(com[k] - o.capsule(k)[1]).max() for k in range(len(prob.capsules))) < 1e-5
    _check_elements(prob, g, o, exact=False)
    g.close()


def test_bb_boundary_readout_leaves_the_run_unchanged():
    """Reading the boundary list between steps runs the first pass of the next boundary phase early; the
    continued run matches one that never read it (to the FP32 atomics' summation order: the element momenta
    are sums of atomics in whatever order they land)."""
    p = _three()
    a, b = _sim(p), _sim(p)
    a.scbb_step(6)
    b.scbb_step(6)
    b.scbb_get_boundary()
    a.scbb_step(6)
    b.scbb_step(6)
    assert np.array_equal(a.scbb_get_owner()[0], b.scbb_get_owner()[0])
    assert np.abs(a.scbb_get_populations() - b.scbb_get_populations()).max() < 1e-6
    assert np.abs(a.scbb_get_vertices()[0] - b.scbb_get_vertices()[0]).max() < 2e-5     # a few ulp at |x| ~ 30
    a.close()
    b.close()


def test_bb_three_capsules_periodic():
    """Three capsules with colours +-0.05 and the particle-particle repulsion in a periodic box (a reduced
    stand-in for the droplet-covering workload): 10 steps, owner fields identical, densities within 1e-5,
    vertices within 1e-4."""
    p = _three()
    g = _sim(p)
    o = O.OracleSim(p)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    g.scbb_step(10)
    o.step(10)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4


def test_bb_uneven_box_rows_across_warps():
    """A box whose rows are not a power-of-two number of four-node quads (nx = 44: 11 quads, rows straddle
    warps, the x-shift falls back to direct loads at warp edges and at the periodic wrap): 20 coupled steps,
    owners identical, densities and vertices within R15's bounds (1e-5 away from the membrane)."""
    cap = inputs.Capsule(centre=(21.3, 17.8, 19.6), radius=6.0, subdiv=3, kS=0.02, kB=1e-3, kV=2.0, colour=-0.2)
    p = inputs.Problem(name="uneven", nx=44, ny=36, nz=40, walls=1, coupling=0, psi_kind=0, z_interface=20,
                       capsules=[cap], noise=1e-4, seed=17, u_lo=(-0.001, 0, 0), u_hi=(0.001, 0, 0))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(20)
    band = _step_with_band(o, 20)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    _cmp_band(p, g, o, band)


def test_bb_janus_capsule_20_steps():
    """Per-element colour (a Janus capsule: +0.3 on its upper half, -0.3 on its lower half), 20 coupled steps:
    identical owner fields, densities within 1e-5 relative, vertex positions within 1e-4."""
    import dataclasses

    p = _small()
    cap = p.capsules[0]
    p.capsules = [dataclasses.replace(cap, elem_colour=inputs.janus_colours(cap, 0.3, -0.3))]
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(20)
    o.step(20)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4


def test_bb_paper_mesh_capsule():
    """The paper's particle: a frequency-12 geodesic sphere (1442 nodes, 2880 elements) of radius 10
    penetrating the interface by 1 in a 40^3 box between sheared walls, colour 0.05: 10 coupled steps,
    owners identical, densities within 1e-5, vertices within 1e-4."""
    cap = inputs.Capsule(centre=(20.2, 19.7, 20.0 - 10.0 + 1.0), radius=10.0, geodesic=12, kS=0.005,
                         kB=0.01 * 0.005 * 100.0, kV=20.0, colour=0.05)
    assert len(cap.mesh()[0]) == 1442
    p = inputs.Problem(name="paper-mesh", nx=40, ny=40, nz=40, walls=1, coupling=0, psi_kind=0, z_interface=20,
                       capsules=[cap], noise=1e-4, seed=19, u_lo=(-0.002, 0, 0), u_hi=(0.002, 0, 0))
    g = _sim(p)
    o = O.OracleSim(p)
    g.scbb_step(10)
    o.step(10)
    og, _, _ = g.scbb_get_owner()
    assert np.array_equal(og, o.owner())
    assert _cmp_rho(g.scbb_get_fields(), o.fields()) < 1e-5
    Xg, _, _ = g.scbb_get_vertices()
    Xo, _, _ = o.vertices()
    assert np.abs(Xg - Xo).max() < 1e-4

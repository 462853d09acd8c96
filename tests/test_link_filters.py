"""The crossed-element search's candidate filters are conservative (host model of the kernel's FP32 arithmetic).

`k_link_cand` passes a lattice link on to the exact segment-triangle test only when (1) its node lies in the
ranges that can meet the triangle's box (with a margin of 1e-3), (2) its two ends straddle the triangle's plane
within tol = 1e-3 |e1|_1 |e2|_1, and (3) where it meets the plane lies in the box up to 4 tol / |n.c| + 1e-3.
Here the same formulas are evaluated in float32, operation by operation, on random triangles, and every link
that the exact test (the node-wise rule of Sec. II.C: the segment from either end, box overlap, then
Moller-Trumbore with closed bounds) accepts must have passed all three filters.  Links one node beyond the
kernel's ranges are tried too."""
import numpy as np

F = np.float32
EPS = np.array([1.37e-4, 2.91e-4, 3.53e-4], F)       # the classification rays' offsets
DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]


def _cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]], F)


def _exact(P, D, v0, e1, e2, b0, b1):
    """Box overlap, then the segment P + s D (s in [0, 1]) against the triangle, closed bounds."""
    if (np.maximum(P, P + D) < b0).any() or (np.minimum(P, P + D) > b1).any():
        return False
    h = _cross(D, e2)
    det = F(np.dot(e1, h))
    if abs(det) < F(1e-30):
        return False
    inv = F(1) / det
    sv = (P - v0).astype(F)
    u = F(np.dot(sv, h)) * inv
    if u < 0 or u > 1:
        return False
    q = _cross(sv, e1)
    v = F(np.dot(D, q)) * inv
    if v < 0 or u + v > 1:
        return False
    t = F(np.dot(e2, q)) * inv
    return 0 <= t <= 1


def test_candidate_filters_keep_every_crossing():
    rng = np.random.default_rng(11)
    hits = passed_hits = 0
    for _ in range(300):
        V = (rng.uniform(0, 250, 3) + rng.normal(size=(3, 3)) * rng.uniform(0.3, 3.0)).astype(F)
        v0 = V[0]
        b0, b1 = V.min(0), V.max(0)
        e1, e2 = (V[1] - v0).astype(F), (V[2] - v0).astype(F)
        nrm = _cross(e1, e2)
        tol = F(1e-3) * F(np.abs(e1).sum()) * F(np.abs(e2).sum())
        for c in DIRS:
            c = np.array(c, F)
            dn = F(nrm[0] * c[0] + nrm[1] * c[1] + nrm[2] * c[2])
            lo = np.ceil(b0 - F(1e-3) - EPS - np.maximum(c, 0)).astype(int)
            hi = np.floor(b1 + F(1e-3) - EPS - np.minimum(c, 0)).astype(int)
            for Z in range(lo[2] - 1, hi[2] + 2):
                for Y in range(lo[1] - 1, hi[1] + 2):
                    for X in range(lo[0] - 1, hi[0] + 2):
                        P = np.array([F(X) + EPS[0], F(Y) + EPS[1], F(Z) + EPS[2]], F)
                        if not (_exact(P, c, v0, e1, e2, b0, b1) or
                                _exact((P + c).astype(F), (-c).astype(F), v0, e1, e2, b0, b1)):
                            continue
                        hits += 1
                        ok = lo[0] <= X <= hi[0] and lo[1] <= Y <= hi[1] and lo[2] <= Z <= hi[2]
                        syz = F(nrm[1] * (P[1] - v0[1])) + F(nrm[2] * (P[2] - v0[2]))
                        su = F(syz + F(nrm[0] * (P[0] - v0[0])))
                        sw = F(su + dn)
                        ok &= not ((su > tol and sw > tol) or (su < -tol and sw < -tol))
                        if ok and abs(dn) > tol:
                            s = F(-su / dn)
                            m = F(F(4) * tol / abs(dn) + F(1e-3))
                            p = (P + s * c).astype(F)
                            ok &= not ((p < b0 - m).any() or (p > b1 + m).any())
                        passed_hits += ok
    assert hits > 5000
    assert passed_hits == hits, (hits, passed_hits)

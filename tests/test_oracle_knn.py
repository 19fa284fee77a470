"""Pins of the k-nearest-neighbour oracle (CPU).

* exact-rational brute force on dyadic inputs (every FP32 operation exact),
  with many equal keys;
* a numpy lexsort of the full FP32 distance matrix (a library sort as the
  step, the distances in the fixed operand order);
* k = 1 reduces to the k = 2 certificate of Def. 1: the lists are (nn, d1^2,
  d2^2) and the frontier is Algorithm 1's;
* Lemma 1 at rank k: no missed failure on any motion family, k in {1, 3, 8};
* tightness at rank 3: a dyadic step with c^(3) = 4 eps_t exactly, where the
  set of the 3 nearest changes or not depending only on the tie-break.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import knn as K
from paper_2606_18314_b300 import scenes
from tests.test_oracle_core import dyadic_points


def exact_knn(points, m):
    P = [[Fraction(float(v)) for v in p] for p in points]
    out = []
    for i, pi in enumerate(P):
        keys = sorted((sum((pj[a] - pi[a]) ** 2 for a in range(len(pi))), j) for j, pj in enumerate(P) if j != i)
        out.append(keys[:m])
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n,m", [(6, 5), (17, 3), (40, 9), (40, 17)])
def test_knn_matches_exact_rational_bruteforce(n, m, dim):
    rng = np.random.default_rng(7 * n + m + dim)
    for trial in range(6):
        pts = dyadic_points(rng, n, dim, bits=2 if trial % 2 else 5)   # coarse grid -> many ties
        idx, d2 = K.knn(pts, m)
        ex = exact_knn(pts, m)
        for i in range(n):
            assert [int(j) for j in idx[i]] == [j for _, j in ex[i]], (trial, i)
            assert [Fraction(float(v)) for v in d2[i]] == [D for D, _ in ex[i]], (trial, i)


@pytest.mark.parametrize("dim", [2, 3])
def test_knn_matches_a_lexsort_of_the_distance_matrix(dim):
    rng = np.random.default_rng(11 + dim)
    p = rng.random((300, dim)).astype(np.float32)
    p[17] = p[3]                                   # a duplicate pair
    # the fixed operand order, dx = x_j - x_i, each FP32 operation rounded
    dx = p[None, :, 0] - p[:, None, 0]
    dy = p[None, :, 1] - p[:, None, 1]
    D = dx * dx + dy * dy
    if dim == 3:
        dz = p[None, :, 2] - p[:, None, 2]
        D = D + dz * dz
    assert D.dtype == np.float32
    m = 12
    idx, d2 = K.knn(p, m)
    j = np.arange(300)
    for i in range(300):
        o = np.lexsort((j, D[i]))
        o = o[o != i][:m]
        assert np.array_equal(idx[i], o), i
        assert np.array_equal(d2[i].view(np.uint32), D[i, o].view(np.uint32)), i


@pytest.mark.parametrize("dim", [2, 3])
def test_k1_reduces_to_the_paper_certificate(dim):
    m = scenes.Motion("clustered_drift", 800, dim, 2e-3, seed=5, steps=20)
    p = m.frame()
    q = m.advance()
    c, t = K.cert(p, 1), oracle.top2(p)
    assert np.array_equal(c.idx[:, 0], t.nn)
    assert np.array_equal(c.d2[:, 0].view(np.uint32), t.d1sq.view(np.uint32))
    assert np.array_equal(c.d2[:, 1].view(np.uint32), t.d2sq.view(np.uint32))
    r, r1 = K.step(p, q, c), oracle.step(p, q, t)
    assert r.eps_t == r1.eps_t
    assert np.array_equal(np.flatnonzero(r.frontier), r1.frontier)
    assert np.array_equal(r.failed, r1.failed)


@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("k", [1, 3, 8])
def test_knn_set_certificate_never_misses(family, k):
    dim = 2 if k == 3 else 3
    m = scenes.Motion(family, 500, dim, eps=3e-3, seed=4, steps=40)
    p = m.frame()
    c = K.cert(p, k)
    failed = 0
    for _ in range(6):
        q = m.advance()
        r = K.step(p, q, c)
        assert r.n_missed == 0
        assert r.n_false == r.n_frontier - (r.n_failed - r.n_missed)
        failed += r.n_failed
        p, c = q, r.cert
    assert failed > 0 or family in ("ring_rotation", "spiral", "vortex", "hotspot", "shear_band")


def _tight_scene(d_first):
    """Point 0 at x = 1/2 on the line y = 1/2; neighbours at +8/128, +16/128,
    +24/128 (k = 3 nearest) and one at -28/128, so c^(3) = 4/128 = 4 eps with
    eps = 1/128.  The step moves point 0 and the third neighbour away from each
    other and the outside point toward point 0, each by eps: the third and the
    outside point end at the same distance, 26/128.  d_first puts the outside
    point before the third in index order."""
    x0 = 0.5
    C = [x0 + 24 / 128, 0.5]
    D = [x0 - 28 / 128, 0.5]
    pts = [[x0, 0.5], [x0 + 8 / 128, 0.5], [x0 + 16 / 128, 0.5]]
    pts += [D, C] if d_first else [C, D]
    pts += [[0.95, 0.95]]                           # a far point: n = 6 >= k + 2 + 1
    p = np.array(pts, np.float32)
    q = p.copy()
    iC, iD = (4, 3) if d_first else (3, 4)
    q[0, 0] -= 1 / 128
    q[iC, 0] += 1 / 128
    q[iD, 0] += 1 / 128
    return p, q, iC, iD


@pytest.mark.parametrize("d_first", [True, False])
def test_knn_tightness_at_rank_three(d_first):
    p, q, iC, iD = _tight_scene(d_first)
    c = K.cert(p, 3)
    assert list(c.idx[0, :4]) == [1, 2, iC, iD]
    assert K.clearances(c)[0] == np.float32(4 / 128)
    r = K.step(p, q, c)
    assert r.eps_t == np.float32(1 / 128)
    assert r.frontier[0]                            # c = 4 eps: flagged
    assert r.cert.d2[0, 2] == r.cert.d2[0, 3] == np.float32((26 / 128) ** 2)
    # equal keys: the lower index is nearer, so the outside point enters iff it is first
    assert bool(r.failed[0]) == d_first
    assert r.n_missed == 0

"""Pins of the CPU oracle against things other than itself (CPU only).

* exact-rational brute force on tiny dyadic inputs (every FP32 op is exact);
* the tightness construction of Theorem A.1 (golden fixture);
* lattices with known equal distances;
* an FP64 k-d tree (scipy) on random inputs;
* closed forms and Theorem A.4 for the entropy (Def. 2);
* Lemma 1 / Cor. A.2 as an audit on every motion family (no missed failure).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2606_18314_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- top-2

def exact_top2(points):
    """Lexicographic (D, j) brute force in exact rationals."""
    P = [[Fraction(float(v)) for v in p] for p in points]
    out = []
    for i, pi in enumerate(P):
        keys = sorted((sum((pj[a] - pi[a]) ** 2 for a in range(len(pi))), j)
                      for j, pj in enumerate(P) if j != i)
        out.append((keys[0][1], keys[0][0], keys[1][0]))
    return out


def dyadic_points(rng, n, dim, bits=6):
    # multiples of 2^-bits in [0,1]: squared distances need <= 2*bits+2 mantissa bits
    return (rng.integers(0, 2 ** bits + 1, size=(n, dim)) / 2.0 ** bits).astype(np.float32)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n", [3, 4, 5, 6, 17])
def test_top2_matches_exact_rational_bruteforce(oracle_mod, n, dim):
    rng = np.random.default_rng(100 * n + dim)
    for trial in range(20):
        pts = dyadic_points(rng, n, dim, bits=3 if trial % 2 else 6)  # coarse grid -> many ties
        c = oracle_mod.top2(pts)
        ex = exact_top2(pts)
        for i, (nn, d1, d2) in enumerate(ex):
            assert c.nn[i] == nn, (trial, i)
            assert Fraction(float(c.d1sq[i])) == d1
            assert Fraction(float(c.d2sq[i])) == d2


def test_hand_enumerated_square():
    """Unit square corners scaled by 1/4: every corner has two neighbours at
    distance 1/4 and one at sqrt(2)/4; ties go to the lowest index."""
    import oracle
    pts = np.array([[0, 0], [0.25, 0], [0, 0.25], [0.25, 0.25]], np.float32)
    c = oracle.top2(pts)
    # corner 0: neighbours 1 and 2 at 1/16 (squared) -> nn = 1 (lower index)
    assert c.nn.tolist() == [1, 0, 0, 1]
    assert c.d1sq.tolist() == [0.0625] * 4
    assert c.d2sq.tolist() == [0.0625] * 4
    d1, d2 = np.sqrt(c.d1sq), np.sqrt(c.d2sq)
    assert np.all(d2 - d1 == 0.0)


def test_duplicates_allowed(oracle_mod):
    pts = np.array([[0.5, 0.5], [0.5, 0.5], [0.5, 0.5], [0.75, 0.5]], np.float32)
    c = oracle_mod.top2(pts)
    assert c.nn.tolist() == [1, 0, 0, 0]
    assert c.d1sq.tolist() == [0.0, 0.0, 0.0, 0.0625]
    assert c.d2sq.tolist() == [0.0, 0.0, 0.0, 0.0625]


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_known_equal_distances(oracle_mod, dim):
    """Square/cubic lattice of spacing 2^-6: interior points have d1 = d2 =
    spacing (c = 0), nn is the lowest-index axis neighbour, and every point is
    in the frontier for any eps >= 0."""
    k = 6
    s = 2.0 ** -6
    ax = (np.arange(k) * s + 0.25).astype(np.float32)
    grid = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), -1).reshape(-1, dim)
    c = oracle_mod.top2(grid)
    assert np.all(c.d1sq == np.float32(s * s))
    assert np.all(c.d2sq == np.float32(s * s))
    # nn = lowest index among the points at exactly one spacing
    for i in range(grid.shape[0]):
        dd = ((grid.astype(np.float64) - grid[i]) ** 2).sum(1)
        assert c.nn[i] == int(np.nonzero(dd == s * s)[0].min())
    F = oracle_mod.frontier(c.d1sq, c.d2sq, np.float32(0.0))
    assert F.tolist() == list(range(grid.shape[0]))


@pytest.mark.parametrize("dim", [2, 3])
def test_top2_against_fp64_kdtree(oracle_mod, dim):
    """scipy's k-d tree (FP64) gives the same nearest neighbour wherever the
    FP64 gap exceeds FP32 rounding, and d1^2, d2^2 within a few ulps."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(7 + dim)
    pts = rng.random((3000, dim)).astype(np.float32)
    c = oracle_mod.top2(pts)
    dist, idx = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), k=3)
    d1_64, d2_64 = dist[:, 1] ** 2, dist[:, 2] ** 2
    sep = (d2_64 - d1_64) > 1e-5 * d2_64
    assert sep.mean() > 0.95
    assert np.all(c.nn[sep] == idx[sep, 1])
    np.testing.assert_allclose(c.d1sq, d1_64, rtol=3e-7, atol=0)
    np.testing.assert_allclose(c.d2sq, d2_64, rtol=3e-7, atol=0)


def test_queries_subset_equals_full(oracle_mod):
    rng = np.random.default_rng(3)
    pts = rng.random((500, 3)).astype(np.float32)
    full = oracle_mod.top2(pts)
    q = np.array([0, 7, 499, 250, 7], np.int32)
    sub = oracle_mod.top2_queries(pts, q)
    assert np.array_equal(sub.nn, full.nn[q])
    assert np.array_equal(sub.d1sq, full.d1sq[q])
    assert np.array_equal(sub.d2sq, full.d2sq[q])
    with pytest.raises(ValueError):
        oracle_mod.top2_queries(pts, np.array([500], np.int32))


def test_rejects_too_few_points(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.top2(np.zeros((2, 2), np.float32))


# --------------------------------------------------------------------------- eps / frontier

def test_eps_is_max_displacement(oracle_mod):
    p0 = np.array([[0.5, 0.5, 0.5], [0.25, 0.25, 0.25], [0.0, 0.0, 0.0]], np.float32)
    p1 = p0.copy()
    p1[1, 0] += 2.0 ** -10
    p1[2] += np.float32(2.0 ** -12)
    e = oracle_mod.eps(p0, p1)
    assert e == np.float32(2.0 ** -10)
    # 3-4-5 triangle in dyadic units
    p2 = p0.copy()
    p2[0, 0] += 3 * 2.0 ** -12
    p2[0, 1] += 4 * 2.0 ** -12
    assert oracle_mod.eps(p0, p2) == np.float32(5 * 2.0 ** -12)
    assert oracle_mod.eps(p0, p0) == 0.0


def _tight_points(eta, d1, eps, origin, order, dim):
    """Theorem A.1 construction; ``order`` lists where (i, a, k) sit in the
    index sequence.  A far point keeps n >= 3 meaningful without interfering."""
    xi, xa, xk = origin, origin + d1, origin - (d1 + eta * eps)
    before = {"i": xi, "a": xa, "k": xk}
    after = {"i": xi - eps, "a": xa + eps, "k": xk + eps}
    idx = {name: order.index(name) for name in "iak"}

    def build(pos):
        P = np.full((3, dim), 0.5, np.float32)
        for name in "iak":
            P[idx[name], 0] = pos[name]
        return P
    return build(before), build(after), idx


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("order", [("i", "a", "k"), ("i", "k", "a")])
def test_tightness_construction_thm_a1(oracle_mod, dim, order):
    g = json.load(open(os.path.join(GOLDEN, "tightness_thm_a1.json")))
    d1, eps, origin = g["d1"], g["eps"], g["origin"]
    for case in g["cases"]:
        eta = case["eta"]
        p0, p1, idx = _tight_points(eta, d1, eps, origin, list(order), dim)
        c0 = oracle_mod.top2(p0)
        i, a, k = idx["i"], idx["a"], idx["k"]
        assert c0.nn[i] == a
        assert c0.d1sq[i] == np.float32(d1 * d1)
        assert c0.d2sq[i] == np.float32((d1 + eta * eps) ** 2)
        e = oracle_mod.eps(p0, p1)
        assert e == np.float32(eps)
        c1 = oracle_mod.top2(p1)
        if case["nn_changes"] is True:
            assert c1.nn[i] == k
        elif case["nn_changes"] is False:
            assert c1.nn[i] == a
        else:  # exact tie: lowest index wins
            assert c1.d1sq[i] == c1.d2sq[i]
            assert c1.nn[i] == min(a, k)
        # c_i = eta*eps: detected iff c_i <= 4 eps (the guard is far below eps)
        F = oracle_mod.frontier(c0.d1sq, c0.d2sq, e)
        assert (i in F) == (eta <= 4.0)
        # a failure is always detected (Lemma 1)
        if c1.nn[i] != c0.nn[i]:
            assert i in F


def test_frontier_guard_is_tiny_and_monotone(oracle_mod):
    rng = np.random.default_rng(11)
    pts = rng.random((2000, 3)).astype(np.float32)
    c = oracle_mod.top2(pts)
    for e in [1e-4, 1e-3, 5e-3]:
        bare = oracle_mod.frontier(c.d1sq, c.d2sq, np.float32(e), guard=False)
        guarded = oracle_mod.frontier(c.d1sq, c.d2sq, np.float32(e))
        assert set(bare.tolist()) <= set(guarded.tolist())
        assert len(guarded) - len(bare) <= 2
        # the rule written out with numpy float32 ops
        d1 = np.sqrt(c.d1sq)
        d2 = np.sqrt(c.d2sq)
        cc = d2 - d1
        tau = np.float32(2.0 ** -20) * ((d1 + d2) + np.float32(e))
        ref = np.nonzero(cc <= (np.float32(4.0) * np.float32(e)) + tau)[0]
        assert np.array_equal(ref, guarded)


# --------------------------------------------------------------------------- cells / entropy

def test_grid_res_values(oracle_mod):
    assert oracle_mod.grid_res(1000, 2) == 32      # 31^2 = 961 < 1000 <= 1024
    assert oracle_mod.grid_res(16000, 3) == 26     # 25^3 = 15625 < 16000 <= 17576
    assert oracle_mod.grid_res(262144, 3) == 64
    assert oracle_mod.grid_res(3, 2) == 2
    assert oracle_mod.grid_res(8, 3) == 2
    assert oracle_mod.grid_res(9, 3) == 3


def test_cells_dyadic_and_clamped(oracle_mod):
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.25, 0.75],
                    [0.49999997, 0.0, 0.0], [-0.1, 1.5, 0.125]], np.float32)
    c = oracle_mod.cells(pts, 4)
    k = lambda x, y, z: (z * 4 + y) * 4 + x
    assert c.tolist() == [k(0, 0, 0), k(3, 3, 3), k(2, 1, 3), k(1, 0, 0), k(0, 3, 0)]
    c2 = oracle_mod.cells(pts[:, :2], 4)
    assert c2.tolist() == [0, 15, 1 * 4 + 2, 1, 3 * 4 + 0]


def test_entropy_closed_forms(oracle_mod):
    ncells = 64
    cell = np.arange(64, dtype=np.int32).repeat(2)           # C = 64 occupied cells
    n = cell.shape[0]
    # k failures spread evenly over k cells: H = ln k / ln C exactly
    for k in [2, 3, 8, 64]:
        mem = np.zeros(n, np.uint8)
        mem[np.arange(k) * 2] = 1
        H, m, C = oracle_mod.entropy(cell, mem, ncells)
        assert C == 64 and m == k
        assert abs(H - math.log(k) / math.log(64)) < 1e-14
    # all failures in one cell: H = 0
    mem = np.zeros(n, np.uint8)
    mem[[10, 11]] = 1
    H, m, C = oracle_mod.entropy(cell, mem, ncells)
    assert H == 0.0 and m == 1
    # empty / single member
    assert oracle_mod.entropy(cell, np.zeros(n, np.uint8), ncells)[0] == 0.0
    one = np.zeros(n, np.uint8)
    one[5] = 1
    assert oracle_mod.entropy(cell, one, ncells)[0] == 0.0
    # C = 1: undefined ratio, reported as 0
    assert oracle_mod.entropy(np.zeros(5, np.int32), np.ones(5, np.uint8), 4)[0] == 0.0
    # counts {2, 1, 1} over three cells: q = (1/2, 1/4, 1/4)
    cell3 = np.array([0, 0, 1, 7, 9, 10], np.int32)
    mem3 = np.array([1, 1, 1, 1, 0, 0], np.uint8)
    H, m, C = oracle_mod.entropy(cell3, mem3, 16)
    q = np.array([0.5, 0.25, 0.25])
    assert (m, C) == (3, 5)
    assert abs(H - float(-(q * np.log(q)).sum() / math.log(5))) < 1e-15


def test_entropy_invariants_random(oracle_mod):
    """H in [0,1] and Theorem A.4: m >= C^H, i.e. H ln C <= ln m."""
    rng = np.random.default_rng(5)
    for trial in range(200):
        ncells = int(rng.integers(2, 300))
        n = int(rng.integers(2, 500))
        cell = rng.integers(0, ncells, n).astype(np.int32)
        mem = (rng.random(n) < rng.random()).astype(np.uint8)
        H, m, C = oracle_mod.entropy(cell, mem, ncells)
        assert 0.0 <= H <= 1.0 + 1e-12
        if m > 0 and C > 1:
            assert H * math.log(C) <= math.log(m) + 1e-12


def test_trunc_median(oracle_mod):
    v = np.array([3.0, 1.0, 2.0, 100.0], np.float32)           # lower median = 2.0
    assert oracle_mod.trunc_median(v) == np.float32(2.0)
    v = np.array([1.2, 5.0, 0.7], np.float32)                  # median 1.2 -> 1.125 (3 mantissa bits)
    assert oracle_mod.trunc_median(v) == np.float32(1.125)
    assert oracle_mod.trunc_median(np.zeros(7, np.float32)) == 0.0
    # only the first 1024 values are sampled
    v = np.concatenate([np.full(1024, 3.0, np.float32), np.full(5000, 0.5, np.float32)])
    assert oracle_mod.trunc_median(v) == np.float32(3.0)


# --------------------------------------------------------------------------- full step / audit

@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
def test_safety_rule_never_misses(oracle_mod, family, dim):
    """Lemma 1 / Cor. A.2 / Table 1 'miss (safe) = 0' on every family."""
    m = scenes.Motion(family, 600, dim, eps=3e-3, seed=1, steps=40)
    p = m.frame()
    cert = oracle_mod.top2(p)
    for t in range(6):
        q = m.advance()
        r = oracle_mod.step(p, q, cert)
        assert r.eps_t <= np.float32(3e-3)
        assert r.n_missed == 0
        assert r.n_failed + r.n_false == len(r.frontier)
        assert 0.0 <= r.H <= 1.0 and 0.0 <= r.H_cand <= 1.0
        if r.m > 0:
            assert r.H * math.log(r.C) <= math.log(r.m) + 1e-12
        assert np.all(r.cert.d1sq <= r.cert.d2sq)
        assert np.all(r.cert.nn != np.arange(600))
        p, cert = q, r.cert


def test_rigid_ring_rounding_failures_are_detected(oracle_mod):
    """Zero-jitter rigid rotation preserves every real distance, so any change
    of nn comes from rounding alone; the guard must still put it in F."""
    m = scenes.Motion("ring_rotation", 800, 3, eps=1e-3, seed=2, jitter=False)
    p = m.frame()
    cert = oracle_mod.top2(p)
    for t in range(5):
        q = m.advance()
        r = oracle_mod.step(p, q, cert)
        assert r.n_missed == 0
        p, cert = q, r.cert

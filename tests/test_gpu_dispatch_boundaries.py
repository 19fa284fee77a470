"""GPU: single scenes on both sides of every size at which the step changes
its launch shape.  The certificates must be the same on either side.

* k_search takes 64 sorted slots per CTA with four lanes per query while
  ceil(N / 64) <= 4 x 148, then 256 slots with one lane per query while
  ceil(N / 256) <= 4 x 148, then 512 while ceil(N / 512) <= 4 x 148, then
  1024: N = 37,888 | 37,889, 151,552 | 151,553 and 303,104 | 303,105.
* k_scan issues in latency order while the scan grid (bucket tiles + point
  tiles of 2048) has fewer than 3 x 148 tiles.  At d = 3 with N in
  (262,144, 524,288] there are 257 bucket tiles, so the switch is at
  N = 380,928 | 380,929.
* k_prepare takes 1, 2 or 4 points per thread, the fewest whose grid of
  256-thread CTAs fits 5 x 148: N = 189,440 | 189,441 and 378,880 | 378,881.
* k_scatter_refresh takes 1 point per thread while ceil(N / 256) <= 6 x 148,
  else 2: N = 227,328 | 227,329.
* bucket counts and entropy-cell failure and frontier counts are 16-bit in
  contexts of more than 262,144 points whose scenes all have fewer than
  65,536: five scenes of 65,535 | one of 65,536 and four of 60,000, and
  four scenes of 60,000 (240,000 points).

Each scene is stepped twice incrementally and once by rebuild. After each step
every certificate must equal the GPU all-pairs pass bit for bit; that pass is
itself checked against the oracle in the parity tests. The failure marks must
be the nn changes, and the safety rule must miss nothing.
"""
import numpy as np
import pytest

from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build
    build.build()
    return t


@pytest.mark.parametrize("n", [37888, 37889, 151552, 151553, 189440, 189441, 227328, 227329, 303104, 303105,
                               378880, 378881, 380928, 380929])
def test_both_sides_of_each_launch_shape_switch(torch, n):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion("uniform_brownian", n, 3, 1e-3, seed=n, steps=8)
    fr = torch.from_numpy(m.frames(3)).cuda()
    ctx = cert.Context(fr[0])
    prev = cert.cert_allpairs(fr[0])[0]
    for t, strat in ((1, "incremental"), (2, "incremental"), (3, "rebuild")):
        ctx.step(fr[t], 1e-3, strat)
        res, rc = ctx.sync(raise_on_status=False)
        assert rc == cert.CERT_OK, (n, t, rc)
        v = ctx.views()
        nn, d1, d2 = cert.cert_allpairs(fr[t])
        assert torch.equal(v["nn"], nn), (n, t)
        assert torch.equal(v["d1sq"].view(torch.int32), d1.view(torch.int32)), (n, t)
        assert torch.equal(v["d2sq"].view(torch.int32), d2.view(torch.int32)), (n, t)
        failed = (nn != prev).cpu().numpy()
        assert np.array_equal(v["failed"].cpu().numpy().astype(bool), failed), (n, t)
        assert int(res[0]["n_failed"]) == int(failed.sum()) and int(res[0]["n_missed"]) == 0, (n, t)
        prev = nn
    ctx.close()


@pytest.mark.parametrize("sizes", [[65535] * 5, [65536] + [60000] * 4, [60000] * 4])
def test_both_sides_of_the_16_bit_count_switch(torch, sizes):
    """In contexts of more than 262,144 points whose scenes all have fewer
    than 65,536 points, the bucket counts and the per-entropy-cell failure and
    frontier counts are 16-bit halves of shared words (no count can reach
    2^16); otherwise they are 32-bit.  Clustered scenes
    (hundreds of points per bucket and cell) on each side: every scene's
    certificates equal the all-pairs pass, and its failure marks, cells, H,
    H_cand and failed, frontier and occupied cell counts equal the oracle's
    definitions of them (Def. 2, Algorithm 1's frontier) evaluated on the host."""
    import oracle
    from paper_2606_18314_b300 import cert
    eps = 1e-3
    ms = [scenes.Motion("uniform_clusters", n, 3, eps, seed=n + k, steps=8) for k, n in enumerate(sizes)]
    bm = scenes.BatchMotion(ms)
    off, fr = bm.offsets, bm.frames(3)
    S = len(sizes)
    ctx = cert.Context(torch.from_numpy(fr[0]).cuda(), offsets=off)

    def top2(t, s):
        return [x.cpu().numpy() for x in cert.cert_allpairs(torch.from_numpy(fr[t][off[s]:off[s + 1]]).cuda())]

    prev = [top2(0, s) for s in range(S)]
    for t, strat in ((1, "incremental"), (2, "incremental"), (3, "rebuild")):
        ctx.step(torch.from_numpy(fr[t]).cuda(), eps, strat)
        res, rc = ctx.sync(raise_on_status=False)
        assert rc == cert.CERT_OK, (sizes, t, rc)
        v = {k: x.cpu().numpy() for k, x in ctx.views().items() if k in ("nn", "d1sq", "d2sq", "failed", "cell")}
        for s in range(S):
            lo, hi, n = int(off[s]), int(off[s + 1]), sizes[s]
            tag = (sizes, t, s)
            nn, d1, d2 = top2(t, s)
            assert np.array_equal(v["nn"][lo:hi], nn), tag
            assert np.array_equal(v["d1sq"][lo:hi].view(np.uint32), d1.view(np.uint32)), tag
            assert np.array_equal(v["d2sq"][lo:hi].view(np.uint32), d2.view(np.uint32)), tag
            failed = nn != prev[s][0]
            assert np.array_equal(v["failed"][lo:hi].astype(bool), failed), tag
            g = oracle.grid_res(n, 3)
            cell = oracle.cells(fr[t][lo:hi], g)
            assert np.array_equal(v["cell"][lo:hi], cell), tag
            H, mcells, C = oracle.entropy(cell, failed, g ** 3)
            sc = res[s]
            assert int(sc["n_failed"]) == int(failed.sum()) and int(sc["n_missed"]) == 0, tag
            assert int(sc["failed_cells"]) == mcells and int(sc["occupied_cells"]) == C, tag
            assert abs(float(sc["H"]) - H) <= 1e-6, tag
            F = oracle.frontier(prev[s][1], prev[s][2], oracle.eps(fr[t - 1][lo:hi], fr[t][lo:hi]))
            assert int(sc["n_frontier"]) == len(F), tag
            member = np.zeros(n, np.uint8)
            member[F] = 1
            Hc, mc, _ = oracle.entropy(cell, member, g ** 3)
            assert int(sc["frontier_cells"]) == mc and abs(float(sc["H_cand"]) - Hc) <= 1e-6, tag
            prev[s] = (nn, d1, d2)
    ctx.close()

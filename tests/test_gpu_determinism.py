"""Determinism: the same inputs give the same outputs, run after run.  The
grid's bucket order comes from atomic counters and differs between runs, and
so does the order of the FP64 entropy sums; the certificates (a top-2 under a
total order), every flag and every count do not depend on either.  So all of
them must match bit for bit across two fresh contexts, and H / H_cand within
1e-12 (FP64 sums of at most N terms in any order)."""
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


def _run(torch, frames, offsets, strategies, audit):
    from paper_2606_18314_b300 import cert
    ctx = cert.Context(torch.from_numpy(frames[0]).cuda(), offsets=offsets, audit=audit)
    outs = []
    for t, strat in enumerate(strategies, start=1):
        ctx.step(torch.from_numpy(frames[t]).cuda(), 2e-3, strat)
        res, _ = ctx.sync()
        v = ctx.views()
        fr = v["frontier"].cpu().numpy()
        lists = np.concatenate([fr[int(res["frontier_start"][s]):int(res["frontier_start"][s]) + int(res["n_frontier"][s])]
                                for s in range(len(res))])
        outs.append((res.copy(), {k: v[k].cpu().numpy().copy() for k in ("nn", "d1sq", "d2sq", "cell", "failed")},
                     lists))
    ctx.close()
    return outs


def test_batched_steps_are_deterministic(torch):
    m = scenes.BatchMotion.mixed(n_scenes=24, lo=300, hi=6000, eps=2e-3, seed=31)
    frames = m.frames(6)
    strategies = ["incremental", "rebuild", "incremental", "allpairs", "incremental", "threshold"]
    a = _run(torch, frames, m.offsets, strategies, ("rho", "geometry"))
    b = _run(torch, frames, m.offsets, strategies, ("rho", "geometry"))
    exact = [n for n in a[0][0].dtype.names if n not in ("H", "H_cand", "gyration", "compactness")]
    for t, ((ra, va, fa), (rb, vb, fb)) in enumerate(zip(a, b)):
        for k in va:
            assert np.array_equal(va[k].view(np.uint8), vb[k].view(np.uint8)), (t, k)
        assert np.array_equal(fa, fb), t
        for n in exact:
            assert np.array_equal(ra[n], rb[n]), (t, n)
        for n in ("H", "H_cand", "gyration", "compactness"):
            assert np.all(np.abs(ra[n] - rb[n]) <= 1e-12), (t, n)


def test_knn_steps_are_deterministic(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion("uniform_clusters", 20000, 3, 1e-3, seed=4, steps=20)
    frames = m.frames(4)
    out = []
    for _ in range(2):
        ctx = cert.KnnContext(torch.from_numpy(frames[0]).cuda(), 8)
        for t in range(1, 5):
            ctx.step(torch.from_numpy(frames[t]).cuda(), 1e-3, "incremental" if t % 2 else "rebuild")
        res, _ = ctx.sync()
        v = ctx.views()
        out.append((res, {k: v[k].cpu().numpy().copy() for k in ("idx", "d2", "frontier", "failed")}))
        ctx.close()
    assert out[0][0] == out[1][0]
    for k in out[0][1]:
        assert np.array_equal(out[0][1][k].view(np.uint8), out[1][1][k].view(np.uint8)), k

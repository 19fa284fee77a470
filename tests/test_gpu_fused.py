"""GPU: the fused step (one launch per step, one CTA per scene) against the
multi-kernel step and the oracle.

The two paths must give the same results bit for bit -- certificates,
frontier lists, failure marks, cells, every count and H -- except
n_searched, which counts the work the refresh left to the search; they can
alternate step by step on one context; the fused step is capturable in a CUDA
graph; and a context whose scenes exceed its limits refuses it.  The parity
tests (test_gpu_parity.py) also run every oracle comparison on both paths."""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes
from tests.test_gpu_parity import GEOM_TOL, assert_step_equal

pytestmark = pytest.mark.gpu

SAME = ("eps_t", "med_c", "n_frontier", "n_failed", "n_missed", "n_false", "failed_cells", "frontier_cells",
        "occupied_cells", "strategy", "grid_res", "search_res", "n_rho", "n_rho_hit", "pred_inc", "pred_reb")


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build
    build.build()
    return t


def _outputs(ctx, res):
    v = ctx.views()
    out = {k: v[k].cpu().numpy().copy() for k in ("nn", "d1sq", "d2sq", "cell", "failed")}
    fr = v["frontier"].cpu().numpy()
    out["frontier"] = [fr[int(res["frontier_start"][s]):int(res["frontier_start"][s]) + int(res["n_frontier"][s])]
                       .copy() for s in range(len(res))]
    return out


def _assert_same(ra, oa, rb, ob, tag):
    for k in ("nn", "d1sq", "d2sq", "cell", "failed"):
        assert np.array_equal(oa[k].view(np.uint8), ob[k].view(np.uint8)), (tag, k)
    for s, (fa, fb) in enumerate(zip(oa["frontier"], ob["frontier"])):
        assert np.array_equal(fa, fb), (tag, "frontier", s)
    for k in SAME:
        assert np.array_equal(ra[k], rb[k]), (tag, k)
    for k in ("H", "H_cand", "gyration", "compactness"):
        assert np.all(np.abs(ra[k] - rb[k]) <= 1e-12), (tag, k)


@pytest.mark.parametrize("hi", [4096, 6000])
@pytest.mark.parametrize("rule", ["step", "point", "clock"])
def test_fused_equals_multi_kernel_on_a_batch(torch, rule, hi):
    """24 scenes of 300 to `hi` points, every strategy but all-pairs and both
    audits: the two paths agree after every step.  Up to 4,096 points the
    fused step keeps each scene's sorted points in shared memory; above, it
    reads them through L1/L2."""
    from paper_2606_18314_b300 import cert, selector
    m = scenes.BatchMotion.mixed(n_scenes=24, lo=300, hi=hi, eps=2e-3, seed=41)
    frames = m.frames(8)
    strategies = ["incremental", "rebuild", "threshold", "auto", "incremental", "rebuild", "auto", "incremental"]
    params, norm = selector.load()
    ctxs = {}
    for path in ("multi", "fused"):
        c = cert.Context(torch.from_numpy(frames[0]).cuda(), offsets=m.offsets, frontier_rule=rule,
                         audit=("rho", "geometry"), path=path)
        c.load_selector(params, norm)
        ctxs[path] = c
    assert ctxs["fused"].step_path("incremental") == "fused"
    assert ctxs["multi"].step_path("incremental") == "multi"
    for t, strat in enumerate(strategies, start=1):
        outs = {}
        for path, c in ctxs.items():
            c.step(torch.from_numpy(frames[t]).cuda(), 2e-3, strat)
            res, rc = c.sync()
            assert rc == cert.CERT_OK
            outs[path] = (res.copy(), _outputs(c, res))
        _assert_same(outs["multi"][0], outs["multi"][1], outs["fused"][0], outs["fused"][1], f"{rule} step {t}")
        assert int(outs["fused"][0]["n_missed"].sum()) == 0
    for c in ctxs.values():
        c.close()


def test_paths_alternate_on_one_context_and_match_the_oracle(torch):
    """Steps alternate between the paths (and the all-pairs pass, which always
    takes the multi-kernel path) on one context; every scene matches the
    oracle after every step."""
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=9, lo=200, hi=5000, eps=1e-3, seed=43)
    off, frames = m.offsets, m.frames(9)
    ctx = cert.Context(torch.from_numpy(frames[0]).cuda(), offsets=off)
    refs = [oracle.top2(frames[0][off[s]:off[s + 1]]) for s in range(9)]
    plan = [("fused", "incremental"), ("multi", "incremental"), ("fused", "rebuild"), ("fused", "allpairs"),
            ("multi", "rebuild"), ("fused", "incremental"), ("fused", "incremental"), ("multi", "incremental"),
            ("fused", "incremental")]
    for t, (path, strat) in enumerate(plan, start=1):
        ctx.set_step_path(path)
        want = "multi" if strat == "allpairs" else path
        assert ctx.step_path(strat) == want
        ctx.step(torch.from_numpy(frames[t]).cuda(), 1e-3, strat)
        res, _ = ctx.sync()
        views = ctx.views()
        for s in range(9):
            r = oracle.step(frames[t - 1][off[s]:off[s + 1]], frames[t][off[s]:off[s + 1]], refs[s])
            assert_step_equal(ctx, res, views, r, s=s, tag=f"{path} {strat} step {t} scene {s}")
            refs[s] = r.cert
    ctx.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_fused_at_its_size_limit(torch, dim):
    """A scene of exactly 16,384 points runs fused and matches the oracle; one
    more point, or more than 16,384 search-grid buckets, and the context
    refuses the fused path (AUTO takes the multi-kernel step)."""
    from paper_2606_18314_b300 import cert
    n = 16384
    m = scenes.Motion("uniform_clusters", n, dim, 1e-3, seed=5, steps=10)
    p = m.frame()
    ctx = cert.Context(torch.from_numpy(p).cuda(), path="fused")
    ref = oracle.top2(p)
    for t in range(3):
        q = m.advance()
        ctx.step(torch.from_numpy(q).cuda(), 1e-3, "incremental" if t != 1 else "rebuild")
        res, _ = ctx.sync()
        r = oracle.step(p, q, ref)
        assert_step_equal(ctx, res, ctx.views(), r, tag=f"n={n} d={dim} step {t}")
        p, ref = q, r.cert
    ctx.close()
    big = np.random.default_rng(1).random((n + 1, dim)).astype(np.float32)
    c2 = cert.Context(torch.from_numpy(big).cuda())
    assert c2.step_path("incremental") == "multi"
    with pytest.raises(cert.CertError) as ei:
        c2.set_step_path("fused")
    assert ei.value.code == cert.CERT_EINVAL
    c2.close()
    c3 = cert.Context(torch.from_numpy(big[:10000]).cuda(), bucket_factor=2)   # 32,768 buckets
    with pytest.raises(cert.CertError):
        c3.set_step_path("fused")
    c3.close()


@pytest.mark.parametrize("hi", [3000, 8000])
def test_fused_steps_replay_from_a_cuda_graph(torch, hi):
    """Fused steps captured in a CUDA graph (one per position-buffer parity)
    and replayed over 20 steps end where eager multi-kernel steps end."""
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=16, lo=500, hi=hi, eps=1e-3, seed=47)
    frames = m.frames(20)
    dev = torch.from_numpy(frames).cuda()
    a = cert.Context(dev[0], offsets=m.offsets, path="fused")
    b = cert.Context(dev[0], offsets=m.offsets, path="multi")
    stage = torch.empty_like(dev[0])
    graphs = []
    for _ in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            a.step(stage, 1e-3, "incremental")
        graphs.append(g)
    for t in range(1, 21):
        stage.copy_(dev[t])
        graphs[(t - 1) % 2].replay()
        b.step(dev[t], 1e-3, "incremental")
    ra, rca = a.sync()
    rb, rcb = b.sync()
    assert rca == rcb == cert.CERT_OK
    _assert_same(ra, _outputs(a, ra), rb, _outputs(b, rb), "graph replay")
    a.close()
    b.close()


def test_fused_geometry_audit_matches_oracle(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=6, lo=400, hi=3000, eps=3e-3, seed=49)
    off, frames = m.offsets, m.frames(3)
    ctx = cert.Context(torch.from_numpy(frames[0]).cuda(), offsets=off, audit=("geometry",), path="fused")
    refs = [oracle.top2(frames[0][off[s]:off[s + 1]]) for s in range(6)]
    for t in range(1, 4):
        ctx.step(torch.from_numpy(frames[t]).cuda(), 3e-3, "incremental")
        res, _ = ctx.sync()
        for s in range(6):
            r = oracle.step(frames[t - 1][off[s]:off[s + 1]], frames[t][off[s]:off[s + 1]], refs[s])
            assert abs(float(res[s]["gyration"]) - r.gyration) <= GEOM_TOL
            assert abs(float(res[s]["compactness"]) - r.compactness) <= GEOM_TOL
            refs[s] = r.cert
    ctx.close()


def test_auto_path_rule(torch):
    """CERT_PATH_AUTO: scenes of at most 2,560 points take the fused step
    however many there are; scenes of up to 4,096 points take it in batches of
    148 or more (a full wave of one CTA per SM); larger scenes take the
    multi-kernel step."""
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(3)
    for n, want in ((2560, "fused"), (2561, "multi"), (4096, "multi")):
        c = cert.Context(torch.from_numpy(rng.random((n, 3)).astype(np.float32)).cuda())
        assert c.step_path("incremental") == want, n
        c.close()
    for sizes, want in (([2560] * 15, "fused"), ([3000] * 148, "fused"), ([3000] * 147, "multi"),
                        ([500] * 147 + [4096], "fused"), ([500] * 160 + [4097], "multi")):
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        c = cert.Context(torch.from_numpy(rng.random((int(off[-1]), 3)).astype(np.float32)).cuda(), offsets=off)
        assert c.step_path("incremental") == want, (len(sizes), max(sizes))
        c.close()

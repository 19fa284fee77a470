"""GPU: two benchmark configurations at their full sizes, checked against the
CPU oracle while they run.

* The batch of 512 scenes (N log-uniform in [500, 16000], d = 3, the five
  motion families mixed, eps = 1e-3) advances 100 steps forward, with the
  learned selector and the cell scale the autotuner picks, every step
  replayed from a CUDA graph.  Sixteen seeded scenes are checked against the
  oracle after EVERY step: certificates, eps_t, frontier list, failure marks,
  cells, counts and H; no scene of the batch misses a failure.
* One scene of N = 16,000, d = 3, for each of the five families and each
  eps in {1e-4, 1e-3, 5e-3}: 200 steps, checked against the oracle at every
  10th step and at the last; the checked steps rotate incremental repair,
  full grid rebuild and the all-pairs pass.

Both use the same comparisons as the parity tests (bit-exact integers and
FP32 keys, H within 1e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes
from tests.test_gpu_parity import assert_step_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build
    build.build()
    return t


def test_batched_512_scenes_100_forward_steps_checked_every_step(torch):
    import bench
    from paper_2606_18314_b300 import cert, selector
    steps = 100
    frames, off, eps, _ = bench.make_workload("batched", 0, steps, workers=8)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0], offsets=off)
    params, norm = selector.load()
    ctx.load_selector(params, norm)
    ctx.autotune(dev[1:9].contiguous(), eps, cert.CERT_INCREMENTAL, (2.5, 3.0, 3.5, 4.0))
    # one graph per position-buffer parity, both reading the same staging buffer
    stage = torch.empty_like(dev[0])
    graphs = []
    for _ in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.step(stage, eps, "auto")
        graphs.append(g)
    torch.cuda.synchronize()
    rng = np.random.default_rng(100)
    checked = sorted(int(s) for s in rng.choice(len(off) - 1, 16, replace=False))
    ref = {s: oracle.top2(frames[0][off[s]:off[s + 1]]) for s in checked}
    strategies = set()
    for t in range(1, steps + 1):
        stage.copy_(dev[t])
        graphs[(t - 1) % 2].replay()
        res, rc = ctx.sync()
        assert rc == cert.CERT_OK
        assert int(res["n_missed"].sum()) == 0, f"step {t}: a failure was missed"
        views = ctx.views()
        for s in checked:
            lo, hi = int(off[s]), int(off[s + 1])
            r = oracle.step(frames[t - 1][lo:hi], frames[t][lo:hi], ref[s])
            assert_step_equal(ctx, res, views, r, s=s, tag=f"step {t} scene {s}")
            ref[s] = r.cert
            strategies.add(int(res["strategy"][s]))
    assert strategies <= {cert.CERT_INCREMENTAL, cert.CERT_REBUILD}
    ctx.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-3, 5e-3])
@pytest.mark.parametrize("family", scenes.FAMILIES)
def test_single_scene_16000_d3_200_steps(torch, family, eps):
    from paper_2606_18314_b300 import cert
    steps, n = 200, 16000
    m = scenes.Motion(family, n, 3, eps, seed=11, steps=steps)
    frames = m.frames(steps)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0])
    rotate = ["incremental", "rebuild", "allpairs"]
    for t in range(1, steps + 1):
        check = t % 10 == 0 or t == steps
        strategy = rotate[(t // 10) % 3] if check else "incremental"
        ctx.step(dev[t], eps, strategy)
        if not check:
            continue
        res, rc = ctx.sync()
        assert rc == cert.CERT_OK
        r = oracle.step(frames[t - 1], frames[t], oracle.top2(frames[t - 1]))
        assert_step_equal(ctx, res, ctx.views(), r, tag=f"{family} eps={eps} step {t} {strategy}")
        assert int(res[0]["strategy"]) == cert.STRATEGY[strategy]
    ctx.close()


@pytest.mark.parametrize("family", ["hotspot", "adversarial_crossing", "shear_band"])
def test_localized_motion_16000_d3_200_steps_checked_every_step(torch, family):
    """Scenes whose motion is local (a jittering hotspot, two slabs crossing a
    static background, a sheared band) at N = 16,000, d = 3, eps = 1e-3:
    200 incremental steps, the multi-kernel and the fused step alternating,
    every step checked against the oracle.  Static points far from the motion
    keep their certificates by the refresh's local motion bound instead of
    being searched again once eps_t has eaten their margin."""
    from paper_2606_18314_b300 import cert
    steps, n, eps = 200, 16000, 1e-3
    m = scenes.Motion(family, n, 3, eps, seed=21, steps=steps)
    frames = m.frames(steps)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0])
    ref = oracle.top2(frames[0])
    searched = []
    for t in range(1, steps + 1):
        ctx.set_step_path("fused" if t % 2 else "multi")
        ctx.step(dev[t], eps, "incremental")
        res, rc = ctx.sync()
        assert rc == cert.CERT_OK
        r = oracle.step(frames[t - 1], frames[t], ref)
        assert_step_equal(ctx, res, ctx.views(), r, tag=f"{family} step {t}")
        ref = r.cert
        searched.append(int(res[0]["n_searched"]))
    ctx.close()
    print(family, "searched fraction over the last 100 steps", np.mean(searched[100:]) / n)


def test_localized_motion_d2_100_steps_checked_every_step(torch):
    """The refresh's local motion bound at d = 2 (a 16 x 16 motion grid): a
    hotspot scene of 4,000 points, eps = 1e-3, 100 incremental steps with the
    two step paths alternating, every step against the oracle; once eps_t has
    eaten the static points' margins, they are proven by the local bound and
    the searched fraction falls far below the detected frontier."""
    from paper_2606_18314_b300 import cert
    steps, n, eps = 100, 4000, 1e-3
    m = scenes.Motion("hotspot", n, 2, eps, seed=23, steps=steps)
    frames = m.frames(steps)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0])
    ref = oracle.top2(frames[0])
    searched, detected = [], []
    for t in range(1, steps + 1):
        ctx.set_step_path("fused" if t % 2 else "multi")
        ctx.step(dev[t], eps, "incremental")
        res, rc = ctx.sync()
        assert rc == cert.CERT_OK
        r = oracle.step(frames[t - 1], frames[t], ref)
        assert_step_equal(ctx, res, ctx.views(), r, tag=f"d2 hotspot step {t}")
        ref = r.cert
        searched.append(int(res[0]["n_searched"]))
        detected.append(int(res[0]["n_frontier"]))
    ctx.close()
    assert np.mean(searched[50:]) < 0.25 * np.mean(detected[50:]), (np.mean(searched[50:]), np.mean(detected[50:]))

"""GPU: the large single-scene workload and the bounded-wait failure path.

* N = 262,144, d = 3, half uniform and half in 16 Gaussian clusters
  (sigma 0.01), eps = 1e-4: every certificate of the grid path equals the
  GPU all-pairs pass bit for bit, a seeded sample of 4096 queries equals the
  CPU oracle, the safety rule misses nothing, and H over the whole scene
  matches the oracle's entropy of the same failure set.
* a device wait on a flag nothing sets gives up after its iteration limit
  and reports CERT_ETIMEOUT; the device stays usable.
"""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2606_18314_b300 import build
    build.build()
    return t


def test_bounded_wait_expires_and_device_stays_usable(torch):
    from paper_2606_18314_b300 import cert
    rc, bits, spins = cert.cert_selftest_bounded_wait(5000)
    assert rc == cert.CERT_ETIMEOUT and bits & 1 and spins == 5001
    pts = torch.rand((1000, 3), generator=torch.Generator().manual_seed(0)).cuda()
    nn, d1, d2 = cert.cert_allpairs(pts)
    ref = oracle.top2(pts.cpu().numpy())
    assert np.array_equal(nn.cpu().numpy(), ref.nn)
    with pytest.raises(Exception):
        cert._check(cert.lib().cert_selftest_bounded_wait(0, None, None))


def test_scale_262144_clusters(torch):
    from paper_2606_18314_b300 import cert
    n = 262144
    m = scenes.Motion("uniform_clusters", n, 3, 1e-4, seed=1, steps=100)
    fr = m.frames(2)
    ctx = cert.Context(torch.from_numpy(fr[0]).cuda())
    rng = np.random.default_rng(4096)
    q = np.sort(rng.choice(n, 4096, replace=False)).astype(np.int32)
    prev_nn = None
    for t in range(3):
        if t:
            ctx.step(torch.from_numpy(fr[t]).cuda(), 1e-4, "incremental")
        res, _ = ctx.sync()
        v = ctx.views()
        p = torch.from_numpy(fr[t]).cuda()
        ann, ad1, ad2 = cert.cert_allpairs(p)
        assert torch.equal(v["nn"], ann) and torch.equal(v["d1sq"], ad1) and torch.equal(v["d2sq"], ad2)
        o = oracle.top2_queries(fr[t], q)
        assert np.array_equal(v["nn"].cpu().numpy()[q], o.nn)
        assert np.array_equal(v["d1sq"].cpu().numpy()[q].view(np.uint32), o.d1sq.view(np.uint32))
        assert np.array_equal(v["d2sq"].cpu().numpy()[q].view(np.uint32), o.d2sq.view(np.uint32))
        if t:
            nn = ann.cpu().numpy()
            failed = nn != prev_nn
            assert np.array_equal(v["failed"].cpu().numpy().astype(bool), failed)
            assert int(res[0]["n_missed"]) == 0
            g = oracle.grid_res(n, 3)
            cell = oracle.cells(fr[t], g)
            assert np.array_equal(v["cell"].cpu().numpy(), cell)
            H, mcells, C = oracle.entropy(cell, failed, g ** 3)
            assert abs(float(res[0]["H"]) - H) <= 1e-6
            assert int(res[0]["failed_cells"]) == mcells and int(res[0]["occupied_cells"]) == C
        prev_nn = ann.cpu().numpy()


def test_batched_512_scenes_graph_replay_sampled(torch):
    """The benchmark's own workload and launch configuration: 512 scenes
    (2,392,732 points), learned selector, steps replayed from a CUDA graph.
    Sixteen seeded scenes are checked against the oracle after the replay
    (certificates bit-exact, failure marks, H within 1e-6); no scene misses a
    failure."""
    import bench
    from paper_2606_18314_b300 import cert, selector
    frames, off, eps, _ = bench.make_workload("batched", 0, 3)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0], offsets=off)
    params, norm = selector.load()
    ctx.load_selector(params, norm)
    ctx.set_cell_scale(3.0)
    ctx.step(dev[1], eps, "auto")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.step(dev[2], eps, "auto")
        ctx.step(dev[3], eps, "auto")
    torch.cuda.synchronize()
    # the capture recorded the two steps without running them; the state is still after frame 1
    g.replay()
    torch.cuda.synchronize()
    res, _ = ctx.sync()
    assert int(res["n_missed"].sum()) == 0
    v = ctx.views()
    nn, d1, d2 = v["nn"].cpu().numpy(), v["d1sq"].cpu().numpy(), v["d2sq"].cpu().numpy()
    failed = v["failed"].cpu().numpy().astype(bool)
    rng = np.random.default_rng(512)
    for s in sorted(rng.choice(len(off) - 1, 16, replace=False)):
        lo, hi = int(off[s]), int(off[s + 1])
        prev = oracle.top2(frames[2][lo:hi])
        cur = oracle.top2(frames[3][lo:hi])
        assert np.array_equal(nn[lo:hi], cur.nn), s
        assert np.array_equal(d1[lo:hi].view(np.uint32), cur.d1sq.view(np.uint32)), s
        assert np.array_equal(d2[lo:hi].view(np.uint32), cur.d2sq.view(np.uint32)), s
        want_failed = cur.nn != prev.nn
        assert np.array_equal(failed[lo:hi], want_failed), s
        g_h = oracle.grid_res(hi - lo, 3)
        H, mcells, C = oracle.entropy(oracle.cells(frames[3][lo:hi], g_h), want_failed, g_h ** 3)
        assert abs(float(res["H"][s]) - H) <= 1e-6, s
        assert int(res["n_failed"][s]) == int(want_failed.sum()), s

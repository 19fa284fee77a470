"""Long runs stay exact.  The refresh proves a certificate from a lower bound
that shrinks every step; after hundreds of steps every certificate must still
be the exact one.

* The benchmark's batch (512 scenes, 2,392,732 points, learned selector,
  steps replayed from a CUDA graph): 256 steps over a ping-pong of eight
  frames; after every 16-step cycle no scene has missed a failure and the
  status is clear; at the end every certificate equals the exact all-pairs
  pass of its scene (itself bit-exact against the oracle in the parity tests),
  bit for bit.
* The kNN certificates, k = 8, 20,000 clustered points, 200 steps: the final
  lists equal the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import knn as K
from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build
    build.build()
    return t


def test_batched_256_graph_steps_stay_exact(torch):
    import bench
    from paper_2606_18314_b300 import cert, selector
    F = 8
    frames, off, eps, _ = bench.make_workload("batched", 0, F)
    dev = torch.from_numpy(frames).cuda()
    ctx = cert.Context(dev[0], offsets=off)
    params, norm = selector.load()
    ctx.load_selector(params, norm)
    ctx.set_cell_scale(3.5)
    cycle = [bench.cycle_index(k, F) for k in range(2 * F)]
    for k in cycle:                      # one eager cycle, back at frame 0
        ctx.step(dev[k], eps, "auto")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in cycle:
            ctx.step(dev[k], eps, "auto")
    torch.cuda.synchronize()
    for _ in range(256 // (2 * F)):
        g.replay()
        res, rc = ctx.sync(raise_on_status=False)
        assert rc == cert.CERT_OK and int(res["n_missed"].sum()) == 0
    # the state is at frame cycle[-1] == 0
    v = ctx.views()
    nn, d1, d2 = v["nn"].cpu().numpy(), v["d1sq"].cpu().numpy(), v["d2sq"].cpu().numpy()
    for s in range(len(off) - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        rn, r1, r2 = cert.cert_allpairs(dev[cycle[-1]][lo:hi].contiguous())
        assert np.array_equal(nn[lo:hi], rn.cpu().numpy()), s
        assert np.array_equal(d1[lo:hi].view(np.uint32), r1.cpu().numpy().view(np.uint32)), s
        assert np.array_equal(d2[lo:hi].view(np.uint32), r2.cpu().numpy().view(np.uint32)), s
    ctx.close()


def test_knn_200_steps_stay_exact(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion("uniform_clusters", 20000, 3, 1e-3, seed=12, steps=400)
    ctx = cert.KnnContext(torch.from_numpy(m.frame()).cuda(), 8)
    for t in range(200):
        q = m.advance()
        ctx.step(torch.from_numpy(q).cuda(), 1e-3)
        if t % 50 == 49:
            res, rc = ctx.sync(raise_on_status=False)
            assert rc == cert.CERT_OK and res["n_missed"] == 0, t
    v = ctx.views()
    ref = K.cert(q, 8)
    assert np.array_equal(v["idx"].cpu().numpy().T, ref.idx)
    assert np.array_equal(v["d2"].cpu().numpy().T.view(np.uint32), ref.d2.view(np.uint32))
    ctx.close()

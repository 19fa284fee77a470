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

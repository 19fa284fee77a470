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

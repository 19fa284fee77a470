"""cert_allpairs_noalloc: the all-pairs entry point for callers that cannot
let the library allocate device memory during a call (a real-time loop with a
memory budget fixed at start-up, a host whose device memory belongs to another
allocator, code that must not wait on the driver's allocator).  It must give
exactly what cert_allpairs gives, call after call, although every call reuses
the same fixed scratch array.  Collected last on purpose (file name), so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allpairs_on_consecutive_calls():
    import torch
    from paper_2606_18314_b300 import build, cert
    assert torch.cuda.is_available(), "GPU test"
    build.build()
    rng = np.random.default_rng(2024)
    cases = [
        (rng.random((5000, 3)).astype(np.float32), None),
        # a second, different call: smaller set, 2-D, with a query list; what
        # the first call left in the shared scratch must not leak into it
        (rng.random((1300, 2)).astype(np.float32), rng.choice(1300, 700, replace=False).astype(np.int32)),
        (np.concatenate([rng.random((3000, 3)), rng.random((10, 3))]).astype(np.float32), None),
    ]
    for pts, q in cases:
        p = torch.from_numpy(pts).cuda()
        qd = torch.from_numpy(q).cuda() if q is not None else None
        ref = cert.cert_allpairs(p, qd)
        got = cert.cert_allpairs_noalloc(p, qd)
        torch.cuda.synchronize()
        for a, b in zip(ref, got):
            assert torch.equal(a, b)
        # and both equal the CPU oracle, bit for bit
        o = oracle.top2(pts) if q is None else oracle.top2_queries(pts, q)
        assert np.array_equal(got[0].cpu().numpy(), o.nn)
        assert np.array_equal(got[1].cpu().numpy().view(np.uint32), o.d1sq.view(np.uint32))
        assert np.array_equal(got[2].cpu().numpy().view(np.uint32), o.d2sq.view(np.uint32))


def test_noalloc_at_its_documented_limit():
    """n = nq = 838,000 (the documented limit) fits and equals cert_allpairs."""
    import torch
    from paper_2606_18314_b300 import cert
    n = 838_000
    p = torch.rand((n, 3), generator=torch.Generator().manual_seed(7)).cuda()
    ref = cert.cert_allpairs(p)
    got = cert.cert_allpairs_noalloc(p)
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    from paper_2606_18314_b300 import cert
    n = 900_000                       # needs more than the 32 MiB scratch array
    p = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(cert.CertError) as ei:
        cert.cert_allpairs_noalloc(p)
    assert ei.value.code == cert.CERT_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_reports_a_non_finite_coordinate():
    """A NaN coordinate made on the host is latched in the static array's
    status word; the call waits for its stream, reads the word and returns
    CERT_EINVAL, as cert_allpairs does.  The word is cleared by the next call,
    whose results are exact again."""
    import torch
    from paper_2606_18314_b300 import build, cert
    build.build()
    rng = np.random.default_rng(31)
    pts = rng.random((2000, 3)).astype(np.float32)
    pts[17, 2] = np.nan
    p = torch.from_numpy(pts).cuda()
    for fn in (cert.cert_allpairs, cert.cert_allpairs_noalloc):
        with pytest.raises(cert.CertError) as ei:
            fn(p)
        assert ei.value.code == cert.CERT_EINVAL
    pts[17, 2] = 0.25
    got = cert.cert_allpairs_noalloc(torch.from_numpy(pts).cuda())
    o = oracle.top2(pts)
    assert np.array_equal(got[0].cpu().numpy(), o.nn)
    assert np.array_equal(got[1].cpu().numpy().view(np.uint32), o.d1sq.view(np.uint32))
    assert np.array_equal(got[2].cpu().numpy().view(np.uint32), o.d2sq.view(np.uint32))

"""GPU parity of the k-nearest-neighbour certificates (include/cert_knn.h)
against the CPU oracle (oracle.knn), through the C ABI: the top-(k+1) lists
(indices and squared distances) bit for bit, the frontier and failure flags
and every count, after init and after every step, for both strategies."""
import numpy as np
import pytest

import oracle
from oracle import knn as K
from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cert():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build, cert as c
    build.build()
    return c


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def assert_lists(ctx, ref, tag=""):
    v = ctx.views()
    idx = v["idx"].cpu().numpy().T
    d2 = v["d2"].cpu().numpy().T
    bad = np.flatnonzero(np.any(idx != ref.idx, axis=1) | np.any(d2.view(np.uint32) != ref.d2.view(np.uint32), axis=1))
    assert bad.size == 0, (f"{tag}: {bad.size} lists differ, first {bad[:4]}: gpu {idx[bad[:2]]} {d2[bad[:2]]} "
                           f"ref {ref.idx[bad[:2]]} {ref.d2[bad[:2]]}")


def assert_step(ctx, r, tag=""):
    res, _ = ctx.sync()
    assert_lists(ctx, r.cert, tag)
    v = ctx.views()
    assert np.array_equal(v["frontier"].cpu().numpy().astype(bool), r.frontier), tag
    assert np.array_equal(v["failed"].cpu().numpy().astype(bool), r.failed), tag
    assert np.float32(res["eps_t"]) == r.eps_t, tag
    for key, val in (("n_frontier", r.n_frontier), ("n_failed", r.n_failed), ("n_missed", 0),
                     ("n_false", r.n_false)):
        assert res[key] == val, (tag, key, res[key], val)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 13, 16])
def test_init_lists_bit_exact(cert, k, dim):
    rng = np.random.default_rng(10 * k + dim)
    for n in (k + 2, 37, 1000, 5000):
        p = rng.random((n, dim)).astype(np.float32)
        ctx = cert.KnnContext(dev(p), k)
        assert_lists(ctx, K.cert(p, k), f"k={k} n={n}")
        ctx.close()


@pytest.mark.parametrize("strategy", ["incremental", "rebuild"])
@pytest.mark.parametrize("k", [1, 4, 8, 16])
@pytest.mark.parametrize("family", ["uniform_brownian", "clustered_drift", "adversarial_crossing", "grid_jitter",
                                    "hotspot", "vortex"])
def test_steps_match_oracle(cert, family, k, strategy):
    dim = 3 if k != 4 else 2
    m = scenes.Motion(family, 2500, dim, 2e-3, seed=3, steps=30)
    p = m.frame()
    ctx = cert.KnnContext(dev(p), k)
    ref = K.cert(p, k)
    for t in range(6):
        q = m.advance()
        ctx.step(dev(q), 2e-3, strategy)
        r = K.step(p, q, ref)
        assert_step(ctx, r, f"{family} k={k} {strategy} step {t}")
        p, ref = q, r.cert
    ctx.close()


def test_cell_scale_does_not_change_results(cert):
    m = scenes.Motion("uniform_clusters", 6000, 3, 1e-3, seed=2, steps=20)
    frames = m.frames(4)
    out = []
    for scale in (0.05, 0.4, 1.0, 3.0):   # 0.05: boxes too large for the grid go to the far pass
        ctx = cert.KnnContext(dev(frames[0]), 6, cell_scale=scale)
        for t in range(1, 5):
            ctx.step(dev(frames[t]), 1e-3)
        v = ctx.views()
        out.append((v["idx"].cpu().numpy().copy(), v["d2"].cpu().numpy().copy(), v["failed"].cpu().numpy().copy()))
        ctx.close()
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.array_equal(a, b)
    r = K.cert(frames[4], 6)
    assert np.array_equal(out[0][0].T, r.idx)


@pytest.mark.parametrize("dim", [2, 3])
def test_ties_duplicates_isolated_and_outside_points(cert, dim):
    g = 12
    axes = [np.arange(g) / g + 0.5 / g] * dim
    lat = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, dim).astype(np.float32)
    extra = np.array([lat[5], lat[5], [0.999] * dim, [-0.25] * dim, [1.5] + [0.5] * (dim - 1)], np.float32)
    p = np.concatenate([lat, extra])
    for k in (1, 4, 9):
        ctx = cert.KnnContext(dev(p), k)
        ref = K.cert(p, k)
        assert_lists(ctx, ref, f"lattice k={k}")
        q = p.copy()
        q[-1, 0] -= 1e-3
        q[3] += 5e-4
        ctx.step(dev(q), 2e-3)
        assert_step(ctx, K.step(p, q, ref), f"lattice step k={k}")
        ctx.close()


def test_k1_matches_the_k2_certificate_context(cert):
    m = scenes.Motion("clustered_drift", 3000, 3, 2e-3, seed=8, steps=20)
    frames = m.frames(5)
    a = cert.KnnContext(dev(frames[0]), 1)
    b = cert.Context(dev(frames[0]))
    for t in range(1, 6):
        a.step(dev(frames[t]), 2e-3)
        b.step(dev(frames[t]), 2e-3)
        ra, _ = a.sync()
        rb, _ = b.sync()
        va, vb = a.views(), b.views()
        assert np.array_equal(va["idx"][0].cpu().numpy(), vb["nn"].cpu().numpy())
        assert np.array_equal(va["d2"][0].cpu().numpy(), vb["d1sq"].cpu().numpy())
        assert np.array_equal(va["d2"][1].cpu().numpy(), vb["d2sq"].cpu().numpy())
        assert np.array_equal(va["failed"].cpu().numpy(), vb["failed"].cpu().numpy())
        assert ra["n_frontier"] == int(rb[0]["n_frontier"]) and ra["n_failed"] == int(rb[0]["n_failed"])
    a.close()
    b.close()


def test_graph_capture_of_two_steps(cert):
    import torch
    m = scenes.Motion("uniform_brownian", 4000, 3, 1e-3, seed=6, steps=20)
    frames = m.frames(2)
    d = [dev(f) for f in frames]
    ctx = cert.KnnContext(d[0], 8)
    ctx.step(d[1], 1e-3)
    ctx.step(d[0], 1e-3)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.step(d[1], 1e-3)
        ctx.step(d[2], 1e-3)
    for _ in range(3):
        g.replay()
        # back to frame 0 by an even number of steps: the graph's buffers
        # expect the parity they were captured at
        ctx.step(d[1], 1e-3)
        ctx.step(d[0], 1e-3)
    g.replay()
    r1 = K.step(frames[1], frames[2], K.cert(frames[1], 8))
    assert_step(ctx, r1, "graph replay")
    ctx.close()


def test_eps_bound_and_nonfinite_are_latched(cert):
    p = np.random.default_rng(3).random((500, 3)).astype(np.float32)
    ctx = cert.KnnContext(dev(p), 4)
    q = p.copy()
    q[7] += 0.01
    ctx.step(dev(q), 1e-3)
    _, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_EBOUND
    ctx.step(dev(p), 1.0)
    _, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_OK
    with pytest.raises(cert.CertError):
        ctx.step(dev(p), 1e-3, "allpairs")
    ctx.close()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_minimum_point_count_steps(cert, k, dim):
    """n = k + 2: every list holds all other points but one, and the spare
    ranks cannot all be filled."""
    n = k + 2
    rng = np.random.default_rng(40 + k + dim)
    p = rng.random((n, dim)).astype(np.float32)
    ctx = cert.KnnContext(dev(p), k)
    ref = K.cert(p, k)
    assert_lists(ctx, ref, "init")
    for t, strategy in enumerate(["incremental", "rebuild", "incremental", "incremental"]):
        q = (p + rng.uniform(-1e-2, 1e-2, p.shape)).astype(np.float32)
        ctx.step(dev(q), 0.03, strategy)
        r = K.step(p, q, ref)
        assert_step(ctx, r, f"n={n} step {t}")
        p, ref = q, r.cert
    ctx.close()

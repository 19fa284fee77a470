"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element
by element on the same seeded inputs, on both step paths (one kernel per
phase, and one launch per step).  Bit-exact for nn, d1^2, d2^2, cells,
frontier membership and order, failure marks and every count; H and H_cand
within 1e-6 absolute of the oracle's FP64 value (the tolerance of the
certificate-maintenance target)."""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu

H_TOL = 1e-6
# gyration from one-pass FP64 sums (any order) against the oracle's two passes:
# the variance's cancellation error is at most n u sum|p|^2 ~ 1e-11 here, so
# the radius differs by at most sqrt of that
GEOM_TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build
    build.build()
    return t


@pytest.fixture(params=["multi", "fused"], autouse=True)
def step_path(request, monkeypatch):
    """Every test of this module runs on both step paths: one kernel per phase
    ("multi") and one launch per step ("fused").  Contexts take the path as
    their default; the all-pairs tests, which build no context, simply run
    twice."""
    from paper_2606_18314_b300 import cert
    init = cert.Context.__init__

    def init_with_path(self, *args, **kw):
        kw.setdefault("path", request.param)
        init(self, *args, **kw)

    monkeypatch.setattr(cert.Context, "__init__", init_with_path)
    return request.param


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_cert_equal(views, ref, lo=0, hi=None, tag=""):
    hi = ref.nn.shape[0] + lo if hi is None else hi
    nn = host(views["nn"][lo:hi])
    d1 = host(views["d1sq"][lo:hi])
    d2 = host(views["d2sq"][lo:hi])
    bad = np.nonzero((nn != ref.nn) | (d1.view(np.uint32) != ref.d1sq.view(np.uint32)) |
                     (d2.view(np.uint32) != ref.d2sq.view(np.uint32)))[0]
    assert bad.size == 0, (f"{tag}: {bad.size} certificates differ, first {bad[:5]} "
                           f"gpu={nn[bad[:3]]},{d1[bad[:3]]},{d2[bad[:3]]} "
                           f"ref={ref.nn[bad[:3]]},{ref.d1sq[bad[:3]]},{ref.d2sq[bad[:3]]}")


def assert_step_equal(ctx, res, views, r, s=0, tag=""):
    """Compare one scene's step outputs with an oracle StepResult."""
    lo, hi = int(ctx.offsets[s]), int(ctx.offsets[s + 1])
    sc = res[s]
    assert_cert_equal(views, r.cert, lo, hi, tag)
    assert np.float32(sc["eps_t"]) == r.eps_t, tag
    nF = int(sc["n_frontier"])
    F = host(views["frontier"][int(sc["frontier_start"]):int(sc["frontier_start"]) + nF])
    assert nF == len(r.frontier) and np.array_equal(F, r.frontier), f"{tag}: frontier differs"
    assert np.array_equal(host(views["failed"][lo:hi]).astype(bool), r.failed), f"{tag}: failed marks"
    assert np.array_equal(host(views["cell"][lo:hi]), r.cell), f"{tag}: cells"
    assert int(sc["n_failed"]) == r.n_failed, tag
    assert int(sc["n_missed"]) == r.n_missed == 0, tag
    assert int(sc["n_false"]) == r.n_false, tag
    assert int(sc["failed_cells"]) == r.m, tag
    assert int(sc["frontier_cells"]) == r.m_cand, tag
    assert int(sc["occupied_cells"]) == r.C, tag
    assert int(sc["grid_res"]) == r.g_h, tag
    assert abs(float(sc["H"]) - r.H) <= H_TOL, (tag, float(sc["H"]), r.H)
    assert abs(float(sc["H_cand"]) - r.H_cand) <= H_TOL, (tag, float(sc["H_cand"]), r.H_cand)
    assert np.float32(sc["med_c"]) == r.med_c, (tag, sc["med_c"], r.med_c)


# ----------------------------------------------------------------------------- all-pairs

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n", [3, 4, 5, 37, 511, 512, 513, 2049, 5000])
def test_allpairs_bit_exact(torch, n, dim):
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(n * 10 + dim)
    pts = rng.random((n, dim)).astype(np.float32)
    ref = oracle.top2(pts)
    nn, d1, d2 = cert.cert_allpairs(dev(torch, pts))
    assert_cert_equal({"nn": nn, "d1sq": d1, "d2sq": d2}, ref, tag=f"allpairs n={n}")


@pytest.mark.parametrize("dim", [2, 3])
def test_allpairs_ties_and_duplicates(torch, dim):
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(5)
    # coarse dyadic grid: many exact ties and duplicate points
    pts = (rng.integers(0, 5, size=(3000, dim)) / 4.0).astype(np.float32)
    ref = oracle.top2(pts)
    nn, d1, d2 = cert.cert_allpairs(dev(torch, pts))
    assert_cert_equal({"nn": nn, "d1sq": d1, "d2sq": d2}, ref, tag="ties")


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_allpairs_reports_a_non_finite_coordinate(torch, bad):
    """k_pack latches a non-finite coordinate; cert_allpairs waits for its
    stream, reads the status word and returns CERT_EINVAL (the results are not
    valid), and a following call on finite input is clean again."""
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(77)
    pts = rng.random((3000, 3)).astype(np.float32)
    pts[1234, 1] = bad
    with pytest.raises(cert.CertError) as ei:
        cert.cert_allpairs(dev(torch, pts))
    assert ei.value.code == cert.CERT_EINVAL
    assert "non-finite" in str(ei.value)
    pts[1234, 1] = 0.5
    nn, d1, d2 = cert.cert_allpairs(dev(torch, pts))
    assert_cert_equal({"nn": nn, "d1sq": d1, "d2sq": d2}, oracle.top2(pts), tag="after a rejected call")


def test_allpairs_query_list(torch):
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(9)
    pts = rng.random((20000, 3)).astype(np.float32)
    q = rng.choice(20000, 1500, replace=False).astype(np.int32)
    ref = oracle.top2_queries(pts, q)
    nn, d1, d2 = cert.cert_allpairs(dev(torch, pts), dev(torch, q))
    assert_cert_equal({"nn": nn, "d1sq": d1, "d2sq": d2}, ref, tag="queries")


# ----------------------------------------------------------------------------- init / rebuild

@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
def test_init_certificates_bit_exact(torch, family, dim):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion(family, 3000, dim, 1e-3, seed=2)
    p = m.frame()
    ctx = cert.Context(dev(torch, p))
    assert_cert_equal(ctx.views(), oracle.top2(p), tag=f"init {family}")
    ctx.rebuild()
    assert_cert_equal(ctx.views(), oracle.top2(p), tag=f"rebuild {family}")
    ctx.sync()


# ----------------------------------------------------------------------------- step loops

def run_loop(torch, motion, steps, strategy, check_every=1):
    from paper_2606_18314_b300 import cert
    p = motion.frame()
    ctx = cert.Context(dev(torch, p))
    ref = oracle.top2(p)
    for t in range(steps):
        q = motion.advance()
        ctx.step(dev(torch, q), motion.eps, strategy)
        res, _ = ctx.sync()
        r = oracle.step(p, q, ref)
        if t % check_every == 0 or t == steps - 1:
            assert_step_equal(ctx, res, ctx.views(), r, tag=f"{motion.family} step {t} {strategy}")
        assert int(res[0]["strategy"]) == cert.STRATEGY[strategy]
        p, ref = q, r.cert
    return ctx


@pytest.mark.parametrize("strategy", ["incremental", "rebuild", "allpairs"])
def test_plain_method_d2_n1000(torch, strategy):
    """N=1000, d=2, uniform, 20 steps of the eps=1e-3 ball walk."""
    run_loop(torch, scenes.Motion("uniform_brownian", 1000, 2, 1e-3, seed=1, steps=20), 20, strategy)


@pytest.mark.parametrize("family", scenes.FAMILIES)
@pytest.mark.parametrize("eps", [1e-4, 1e-3, 5e-3])
def test_families_d3_incremental(torch, family, eps):
    run_loop(torch, scenes.Motion(family, 4000, 3, eps, seed=3, steps=12), 12, "incremental")


@pytest.mark.parametrize("family", scenes.FAMILIES)
def test_families_d3_rebuild_and_d2(torch, family):
    run_loop(torch, scenes.Motion(family, 3000, 3, 2e-3, seed=4, steps=6), 6, "rebuild")
    run_loop(torch, scenes.Motion(family, 3000, 2, 2e-3, seed=5, steps=6), 6, "incremental")


@pytest.mark.parametrize("family", scenes.PAPER_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
def test_paper_families_incremental_and_rebuild(torch, family, dim):
    """The paper's other motion families (Sec. 3, Table 1), both strategies."""
    run_loop(torch, scenes.Motion(family, 3000, dim, 2e-3, seed=12, steps=10), 8, "incremental")
    run_loop(torch, scenes.Motion(family, 2000, dim, 2e-3, seed=13, steps=10), 4, "rebuild")


@pytest.mark.parametrize("rule", ["point", "clock"])
@pytest.mark.parametrize("family", ["uniform_brownian", "hotspot", "adversarial_crossing", "vortex", "grid_jitter"])
def test_frontier_rules_match_oracle(torch, rule, family):
    """The per-point budget and cumulative-clock frontier rules: the detected
    frontier, its cells and H_cand bit-exact / within 1e-6 of the oracle over a
    dozen steps (the clock carries state across them), certificates unchanged."""
    from paper_2606_18314_b300 import cert
    for dim, strategy in ((3, "incremental"), (2, "rebuild")):
        m = scenes.Motion(family, 2500, dim, 2e-3, seed=14, steps=30)
        p = m.frame()
        ctx = cert.Context(dev(torch, p), frontier_rule=rule)
        ref = oracle.top2(p)
        clock = oracle.ClockState(ref) if rule == "clock" else None
        for t in range(12):
            q = m.advance()
            ctx.step(dev(torch, q), 2e-3, strategy)
            res, _ = ctx.sync()
            r = oracle.step(p, q, ref, rule=rule, clock=clock)
            assert_step_equal(ctx, res, ctx.views(), r, tag=f"{rule} {family} d={dim} step {t}")
            p, ref = q, r.cert
        if rule == "clock":
            # a rebuild revisits every point; the clock keeps running
            ctx.rebuild()
            clock._revisit(ref, np.ones(ref.nn.shape[0], bool))
            for t in range(3):
                q = m.advance()
                ctx.step(dev(torch, q), 2e-3, strategy)
                res, _ = ctx.sync()
                r = oracle.step(p, q, ref, rule=rule, clock=clock)
                assert_step_equal(ctx, res, ctx.views(), r, tag=f"clock after rebuild {family} step {t}")
                p, ref = q, r.cert
        ctx.close()


@pytest.mark.parametrize("rule", ["step", "point", "clock"])
def test_audits_match_oracle(torch, rule):
    """The audits: the rho heuristic's flagged count (k_scan) and flagged
    failures (counted by the refresh, the search, the far pass and the
    all-pairs merge) equal the oracle's, and the failures' gyration and
    compactness (k_geometry, FP64 sums in any order) are within 1e-5 of its
    two-pass values, in every scene of a batch, under every frontier rule and
    strategy; without the audits those fields stay 0 and nothing else changes."""
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=10, lo=300, hi=3000, eps=2e-3, seed=21)
    off = m.offsets
    frames = m.frames(6)
    ctx = cert.Context(dev(torch, frames[0]), offsets=off, frontier_rule=rule, audit=("rho", "geometry"))
    plain = cert.Context(dev(torch, frames[0]), offsets=off, frontier_rule=rule)
    refs = [oracle.top2(frames[0][off[s]:off[s + 1]]) for s in range(10)]
    clocks = [oracle.ClockState(r) for r in refs] if rule == "clock" else [None] * 10
    strategies = ["incremental", "rebuild", "allpairs", "incremental", "rebuild", "incremental"]
    seen_hits = 0
    for t in range(1, 7):
        ctx.step(dev(torch, frames[t]), 2e-3, strategies[t - 1])
        plain.step(dev(torch, frames[t]), 2e-3, strategies[t - 1])
        res, _ = ctx.sync()
        res0, _ = plain.sync()
        views = ctx.views()
        for s in range(10):
            a, b = frames[t - 1][off[s]:off[s + 1]], frames[t][off[s]:off[s + 1]]
            r = oracle.step(a, b, refs[s], rule=rule, clock=clocks[s])
            tag = f"{rule} scene {s} step {t}"
            assert_step_equal(ctx, res, views, r, s=s, tag=tag)
            assert int(res[s]["n_rho"]) == r.n_rho, (tag, int(res[s]["n_rho"]), r.n_rho)
            assert int(res[s]["n_rho_hit"]) == r.n_rho_hit, (tag, int(res[s]["n_rho_hit"]), r.n_rho_hit)
            assert abs(float(res[s]["gyration"]) - r.gyration) <= GEOM_TOL, (tag, float(res[s]["gyration"]), r.gyration)
            assert abs(float(res[s]["compactness"]) - r.compactness) <= GEOM_TOL, (tag, float(res[s]["compactness"]),
                                                                                  r.compactness)
            seen_hits += r.n_rho_hit
            refs[s] = r.cert
        assert np.all(res0["n_rho"] == 0) and np.all(res0["n_rho_hit"] == 0)
        assert np.all(res0["gyration"] == 0) and np.all(res0["compactness"] == 0)
        for k in ("n_frontier", "n_failed", "n_missed", "n_false", "failed_cells", "frontier_cells"):
            assert np.array_equal(res0[k], res[k]), k
    assert seen_hits > 0
    ctx.close()
    plain.close()


def test_strategies_agree_bitwise(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=5, lo=800, hi=3000, eps=2e-3, seed=7)
    frames = m.frames(6)
    outs = {}
    for strat in ["incremental", "rebuild", "allpairs"]:
        ctx = cert.Context(dev(torch, frames[0]), offsets=m.offsets)
        for t in range(1, 7):
            ctx.step(dev(torch, frames[t]), 2e-3, strat)
        res, _ = ctx.sync()
        v = ctx.views()
        fr = host(v["frontier"])
        # each scene's list sits at its frontier_start (the fused step places it at the
        # scene's first point, the multi-kernel step packs the lists back to back)
        outs[strat] = [host(v[k]).copy() for k in ("nn", "d1sq", "d2sq", "failed", "cell")] + [
            fr[int(res["frontier_start"][s]):int(res["frontier_start"][s]) + int(res["n_frontier"][s])].copy()
            for s in range(len(res))]
        ctx.close()
    for strat in ["rebuild", "allpairs"]:
        for a, b in zip(outs["incremental"], outs[strat]):
            assert np.array_equal(a, b), strat


# ----------------------------------------------------------------------------- batches

def test_batched_scenes_match_oracle_per_scene(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.BatchMotion.mixed(n_scenes=12, lo=300, hi=2500, eps=1e-3, seed=11)
    off = m.offsets
    frames = m.frames(5)
    ctx = cert.Context(dev(torch, frames[0]), offsets=off)
    refs = [oracle.top2(frames[0][off[s]:off[s + 1]]) for s in range(12)]
    for t in range(1, 6):
        ctx.step(dev(torch, frames[t]), 1e-3, "incremental" if t % 2 else "rebuild")
        res, _ = ctx.sync()
        views = ctx.views()
        for s in range(12):
            a, b = frames[t - 1][off[s]:off[s + 1]], frames[t][off[s]:off[s + 1]]
            r = oracle.step(a, b, refs[s])
            assert_step_equal(ctx, res, views, r, s=s, tag=f"scene {s} step {t}")
            refs[s] = r.cert


# ----------------------------------------------------------------------------- edge cases

def test_three_point_scenes_and_duplicates(torch):
    from paper_2606_18314_b300 import cert
    pts = np.array([[0.5, 0.5, 0.5]] * 3 + [[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [0.9, 0.9, 0.9]] +
                   [[0.25, 0.25, 0.25], [0.5, 0.25, 0.25], [0.75, 0.25, 0.25], [1.0, 0.25, 0.25]],
                   np.float32)
    off = np.array([0, 3, 6, 10])
    ctx = cert.Context(dev(torch, pts), offsets=off)
    v = ctx.views()
    for s in range(3):
        ref = oracle.top2(pts[off[s]:off[s + 1]])
        assert_cert_equal(v, ref, off[s], off[s + 1], tag=f"tiny {s}")
    q = pts.copy()
    q[:, 0] = np.minimum(q[:, 0] + np.float32(1e-4), 1.0)
    ctx.step(dev(torch, q), 2e-4, "incremental")   # declared bound above the rounded displacement
    res, _ = ctx.sync()
    for s in range(3):
        r = oracle.step(pts[off[s]:off[s + 1]], q[off[s]:off[s + 1]], oracle.top2(pts[off[s]:off[s + 1]]))
        assert_step_equal(ctx, res, ctx.views(), r, s=s, tag=f"tiny step {s}")


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_ties(torch, dim):
    from paper_2606_18314_b300 import cert
    k = 14 if dim == 3 else 60
    ax = (np.arange(k) * 2.0 ** -6 + 0.25).astype(np.float32)
    grid = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), -1).reshape(-1, dim).astype(np.float32)
    ctx = cert.Context(dev(torch, grid))
    ref = oracle.top2(grid)
    assert_cert_equal(ctx.views(), ref, tag="lattice")
    # a zero step: every point has c = 0 and is in the frontier
    ctx.step(dev(torch, grid), 0.0, "incremental")
    res, _ = ctx.sync()
    r = oracle.step(grid, grid, ref)
    assert_step_equal(ctx, res, ctx.views(), r, tag="lattice step")
    assert int(res[0]["n_frontier"]) == grid.shape[0]


def test_isolated_point_needs_wide_search(torch):
    """A point far from a dense cluster: its block must widen far beyond the
    3^d neighbourhood (the bounded-search-cap failure the paper reports)."""
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(2)
    pts = np.concatenate([0.5 + 0.004 * rng.standard_normal((6000, 3)),
                          [[0.02, 0.97, 0.03]], [[0.99, 0.01, 0.98]]]).astype(np.float32)
    pts = np.clip(pts, 0, 1).astype(np.float32)
    ctx = cert.Context(dev(torch, pts))
    assert_cert_equal(ctx.views(), oracle.top2(pts), tag="isolated")
    q = pts.copy()
    q[-1] = [0.985, 0.015, 0.975]
    ctx.step(dev(torch, q), 0.03, "incremental")
    res, _ = ctx.sync()
    assert_step_equal(ctx, res, ctx.views(), oracle.step(pts, q, oracle.top2(pts)), tag="isolated step")


def test_points_outside_unit_box_are_clamped_exactly(torch):
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(4)
    pts = (rng.random((2000, 3)) * 1.4 - 0.2).astype(np.float32)
    ctx = cert.Context(dev(torch, pts))
    assert_cert_equal(ctx.views(), oracle.top2(pts), tag="outside")


def test_tightness_construction_on_gpu(torch):
    """Theorem A.1 construction embedded in a larger scene of far points."""
    from paper_2606_18314_b300 import cert
    rng = np.random.default_rng(1)
    for eta in [3.5, 3.9375, 4.0, 4.5]:
        far = (0.9 + 0.1 * rng.random((50, 3))).astype(np.float32)
        e = 2.0 ** -10
        line = np.array([[0.5, 0.5, 0.5], [0.75, 0.5, 0.5], [0.5 - (0.25 + eta * e), 0.5, 0.5]], np.float32)
        p0 = np.concatenate([line, far]).astype(np.float32)
        p1 = p0.copy()
        p1[0, 0] -= e
        p1[1, 0] += e
        p1[2, 0] += e
        ctx = cert.Context(dev(torch, p0))
        ctx.step(dev(torch, p1), e, "incremental")
        res, _ = ctx.sync()
        r = oracle.step(p0, p1, oracle.top2(p0))
        assert_step_equal(ctx, res, ctx.views(), r, tag=f"eta={eta}")
        assert (0 in r.frontier) == (eta <= 4.0)


def test_status_reporting(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion("uniform_brownian", 500, 3, 1e-3, seed=1)
    ctx = cert.Context(dev(torch, m.frame()))
    ctx.step(dev(torch, m.advance()), 1e-5, "incremental")   # declared eps far too small
    _, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_EBOUND
    _, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_OK                                   # latched status was cleared
    bad = m.advance()
    bad[7, 1] = np.nan
    ctx.step(dev(torch, bad), 1e-3, "incremental")
    _, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_EINVAL
    with pytest.raises(cert.CertError):
        ctx.step(dev(torch, m.frame()), -1.0, "incremental")
    with pytest.raises(cert.CertError):
        ctx.step(dev(torch, m.frame()), float("nan"), "incremental")


def test_distances_and_host_step(torch):
    from paper_2606_18314_b300 import cert
    m = scenes.Motion("clustered_drift", 2000, 3, 1e-3, seed=6)
    p = m.frame()
    ctx = cert.Context(dev(torch, p))
    d1, d2 = ctx.distances()
    ref = oracle.top2(p)
    assert np.array_equal(host(d1), np.sqrt(ref.d1sq))
    assert np.array_equal(host(d2), np.sqrt(ref.d2sq))
    q = m.advance()
    out = ctx.step_host(q, 1e-3, "incremental")
    r = oracle.step(p, q, ref)
    assert int(out[0]["n_failed"]) == r.n_failed and int(out[0]["n_frontier"]) == len(r.frontier)
    assert abs(float(out[0]["H"]) - r.H) <= H_TOL


def test_pipelined_host_steps_match_the_oracle(torch):
    """cert_step_host_stream: frames copied on the context's copy stream into
    two staging buffers while the previous step runs.  Every step's scalars
    and the final certificates equal the oracle's, and the frame table may
    revisit frames (a ping-pong cycle)."""
    from paper_2606_18314_b300 import cert
    bm = scenes.BatchMotion.mixed(n_scenes=6, lo=500, hi=3000, eps=2e-3, seed=21)
    off = bm.offsets
    fr = bm.frames(4)
    host_frames = torch.from_numpy(fr).pin_memory()
    ctx = cert.Context(dev(torch, fr[0]), offsets=off)
    order = [1, 2, 3, 4, 3, 2]
    row = fr[0].size * 4
    out = np.zeros(len(order) * (len(off) - 1), cert.SCENE_DTYPE)
    ctx.step_host_stream([host_frames.data_ptr() + k * row for k in order], 2e-3, cert.CERT_INCREMENTAL, out)
    prev = [oracle.top2(fr[0][off[s]:off[s + 1]]) for s in range(len(off) - 1)]
    for step, k in enumerate(order):
        for s in range(len(off) - 1):
            cur = fr[k][off[s]:off[s + 1]]
            r = oracle.step(fr[order[step - 1] if step else 0][off[s]:off[s + 1]], cur, prev[s])
            sc = out[step * (len(off) - 1) + s]
            assert int(sc["n_failed"]) == r.n_failed and int(sc["n_frontier"]) == len(r.frontier), (step, s)
            assert abs(float(sc["H"]) - r.H) <= H_TOL, (step, s)
            assert int(sc["n_missed"]) == 0
            prev[s] = r.cert
    v = ctx.views()
    for s in range(len(off) - 1):
        assert np.array_equal(host(v["nn"])[off[s]:off[s + 1]], prev[s].nn)
        assert np.array_equal(host(v["d2sq"])[off[s]:off[s + 1]].view(np.uint32), prev[s].d2sq.view(np.uint32))
    # the steps replay captured graphs: a changed setting (cell scale) and a
    # changed strategy must take effect in the next call, odd step counts too
    ctx.set_cell_scale(2.0)
    for order2, strat in (([3, 4, 3], cert.CERT_REBUILD), ([2], cert.CERT_INCREMENTAL)):
        last = order[-1]
        out2 = np.zeros(len(order2) * (len(off) - 1), cert.SCENE_DTYPE)
        ctx.step_host_stream([host_frames.data_ptr() + k * row for k in order2], 2e-3, strat, out2)
        for step, k in enumerate(order2):
            src = last if step == 0 else order2[step - 1]
            for s in range(len(off) - 1):
                r = oracle.step(fr[src][off[s]:off[s + 1]], fr[k][off[s]:off[s + 1]], prev[s])
                sc = out2[step * (len(off) - 1) + s]
                assert int(sc["n_failed"]) == r.n_failed and int(sc["strategy"]) == strat, (order2, step, s)
                prev[s] = r.cert
        order = order + order2
        v = ctx.views()
        for s in range(len(off) - 1):
            assert np.array_equal(host(v["nn"])[off[s]:off[s + 1]], prev[s].nn)
            assert np.array_equal(host(v["d1sq"])[off[s]:off[s + 1]].view(np.uint32), prev[s].d1sq.view(np.uint32))
        assert ctx.views() is not None
    with pytest.raises(cert.CertError):
        ctx.step_host_stream([0], 2e-3, cert.CERT_INCREMENTAL, None)


def test_every_call_kind_on_one_context_matches_the_oracle(torch):
    """The step's counters and accumulators are zeroed by its own kernels, so
    each call must leave them zero for the next: device steps on the
    multi-kernel and fused paths, the all-pairs and rebuild strategies,
    cert_rebuild, snapshot / restore, and pipelined host steps replaying cached
    graphs, interleaved on one context.  After every call each scene matches
    the oracle (certificates, frontier, failures, cells, H)."""
    from paper_2606_18314_b300 import cert
    bm = scenes.BatchMotion.mixed(n_scenes=6, lo=400, hi=3000, eps=2e-3, seed=77)
    off, fr = bm.offsets, bm.frames(12)
    S = len(off) - 1
    host_frames = torch.from_numpy(fr).pin_memory()
    row = fr[0].size * 4
    ctx = cert.Context(dev(torch, fr[0]), offsets=off, audit=("rho", "geometry"))
    refs = [oracle.top2(fr[0][off[s]:off[s + 1]]) for s in range(S)]
    pos = 0   # frame the context's positions sit at

    def check_step(k, res, tag):
        nonlocal pos
        views = ctx.views()
        for s in range(S):
            r = oracle.step(fr[pos][off[s]:off[s + 1]], fr[k][off[s]:off[s + 1]], refs[s])
            assert_step_equal(ctx, res, views, r, s=s, tag=f"{tag} scene {s}")
            refs[s] = r.cert
        pos = k

    def device_step(k, strat, path):
        ctx.set_step_path(path)
        ctx.step(dev(torch, fr[k]), 2e-3, strat)
        res, rc = ctx.sync()
        assert rc == cert.CERT_OK
        check_step(k, res, f"{path} {strat} frame {k}")

    device_step(1, "incremental", "multi")
    device_step(2, "allpairs", "auto")
    device_step(3, "incremental", "fused")
    device_step(4, "rebuild", "multi")
    ctx.rebuild()
    res, rc = ctx.sync()
    assert rc == cert.CERT_OK
    nn = host(ctx.views()["nn"])
    for s in range(S):
        assert np.array_equal(nn[off[s]:off[s + 1]], refs[s].nn)
    ctx.snapshot()
    device_step(5, "incremental", "multi")
    ctx.restore()   # back at frame 4: step to frame 5 again, then on
    pos, refs[:] = 4, [oracle.top2(fr[4][off[s]:off[s + 1]]) for s in range(S)]
    device_step(5, "incremental", "fused")
    device_step(6, "incremental", "multi")
    order = [7, 8, 9]
    out = np.zeros(len(order) * S, cert.SCENE_DTYPE)
    ctx.set_step_path("multi")
    ctx.step_host_stream([host_frames.data_ptr() + k * row for k in order], 2e-3, cert.CERT_INCREMENTAL, out)
    for step, k in enumerate(order):
        for s in range(S):
            r = oracle.step(fr[pos][off[s]:off[s + 1]], fr[k][off[s]:off[s + 1]], refs[s])
            sc = out[step * S + s]
            assert int(sc["n_failed"]) == r.n_failed and int(sc["n_frontier"]) == len(r.frontier), (k, s)
            assert int(sc["failed_cells"]) == r.m and int(sc["occupied_cells"]) == r.C, (k, s)
            assert abs(float(sc["H"]) - r.H) <= H_TOL, (k, s)
            refs[s] = r.cert
        pos = k
    device_step(10, "allpairs", "auto")
    device_step(11, "incremental", "multi")
    device_step(12, "incremental", "fused")
    ctx.close()

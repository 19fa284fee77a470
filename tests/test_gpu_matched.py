"""The matched-pair entropy experiment (Sec. 4, Fig. 2) on the GPU: every
transition the survey reports carries the oracle's counts and entropy, the
pair chosen from the GPU's rows is the pair chosen from the oracle's, and the
replayed transitions (one scene, and a batch of seeds) keep certifying
exactly."""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import matched

pytestmark = pytest.mark.gpu

N, DIM, STEPS = 4000, 3, 24
EPS_B = (1e-3, 5e-4, 2.5e-4, 1.25e-4)


@pytest.fixture(scope="module")
def cert():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build, cert as c
    build.build()
    return c


def oracle_rows(frames, family, eps):
    c = oracle.top2(frames[0])
    rows = []
    for t in range(len(frames) - 1):
        r = oracle.step(frames[t], frames[t + 1], c)
        c = r.cert
        rows.append({"family": family, "eps": eps, "t": t, "n_failed": r.n_failed, "H": r.H, "m": r.m,
                     "C": r.C, "n_frontier": len(r.frontier), "frontier_cells": r.m_cand,
                     "gyration": r.gyration, "compactness": r.compactness})
    return rows


def test_survey_and_selection_match_the_oracle(cert):
    fa, ga = matched.survey(cert, matched.LOCALIZED, N, DIM, 1e-3, STEPS)
    oa = oracle_rows(fa, matched.LOCALIZED, 1e-3)
    gb, ob = [], []
    for e in EPS_B:
        fb, rb = matched.survey(cert, matched.DIFFUSE, N, DIM, e, STEPS)
        gb += rb
        ob += oracle_rows(fb, matched.DIFFUSE, e)
    for g, o in zip(ga + gb, oa + ob):
        tag = (g["family"], g["eps"], g["t"])
        for k in ("n_failed", "m", "C", "n_frontier", "frontier_cells"):
            assert g[k] == o[k], (tag, k, g[k], o[k])
        assert abs(g["H"] - o["H"]) <= 1e-6, tag
        assert abs(g["gyration"] - o["gyration"]) <= 1e-5 and abs(g["compactness"] - o["compactness"]) <= 1e-5, tag
        assert g["n_missed"] == 0, tag
    pg, po = matched.select(ga, gb), matched.select(oa, ob)
    assert pg is not None and po is not None
    assert [(r["family"], r["eps"], r["t"]) for r in pg] == [(r["family"], r["eps"], r["t"]) for r in po]
    a, b = pg
    assert abs(a["n_failed"] - b["n_failed"]) <= matched.TOLERANCE * max(a["n_failed"], b["n_failed"])
    assert b["H"] > a["H"]


@pytest.mark.parametrize("family,eps,t", [(matched.LOCALIZED, 1e-3, 2), (matched.DIFFUSE, 1.25e-4, 7)])
def test_replayed_transition_certifies_exactly(cert, family, eps, t):
    """time_transition replays t -> t+1 -> t from a graph; its last forward step
    equals the oracle's step, one scene and a batch of three seeds."""
    import torch
    for strategy in (cert.CERT_INCREMENTAL, cert.CERT_REBUILD):
        two = matched.frames_at(family, N, DIM, eps, 1, t, 64)
        ms, res = matched.time_transition(cert, two, np.array([0, N], np.int64), eps, strategy, steps=6)
        assert ms > 0
        r = oracle.step(two[0], two[1], oracle.top2(two[0]))
        assert int(res[0]["n_failed"]) == r.n_failed and int(res[0]["n_missed"]) == 0
        assert abs(float(res[0]["H"]) - r.H) <= 1e-6
    fr, off = matched.batch_frames(family, 1500, DIM, eps, t, [1, 2, 3], 64)
    ms, res = matched.time_transition(cert, fr, off, eps, cert.CERT_INCREMENTAL, steps=6)
    for s in range(3):
        p0, p1 = fr[0, off[s]:off[s + 1]], fr[1, off[s]:off[s + 1]]
        r = oracle.step(p0, p1, oracle.top2(p0))
        assert int(res[s]["n_failed"]) == r.n_failed and int(res[s]["n_missed"]) == 0, s
        assert abs(float(res[s]["H"]) - r.H) <= 1e-6, s
    torch.cuda.synchronize()


def test_frontier_query_times_the_failed_points(cert):
    two = matched.frames_at(matched.LOCALIZED, N, DIM, 1e-3, 1, 2, 64)
    r = oracle.step(two[0], two[1], oracle.top2(two[0]))
    idx = np.flatnonzero(r.failed).astype(np.int32)
    assert idx.size > 0
    assert matched.frontier_query_ms(cert, two[1], idx, reps=3) > 0

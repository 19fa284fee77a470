"""The transition log on the GPU: every row's audit and descriptors are the
oracle's for that transition, although each step is first timed under the
rebuild and all-pairs strategies from a snapshot (which must leave the state
as it was)."""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes

pytestmark = pytest.mark.gpu


def test_log_rows_match_the_oracle(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_18314_b300 import build, cert, translog
    build.build()
    n, dim, eps, steps = 3000, 3, 2e-3, 5
    out = tmp_path / "t.jsonl"
    rows = translog.log_scene(cert, "clustered_drift", n, dim, eps, steps, seed=3, out=out)
    assert translog.read(out) == rows and len(rows) == steps
    fr = scenes.Motion("clustered_drift", n, dim, eps, seed=3, steps=64).frames(steps)
    ref = oracle.top2(fr[0])
    for t, row in enumerate(rows, start=1):
        r = oracle.step(fr[t - 1], fr[t], ref)
        assert row["frame"] == t and row["n_failed"] == r.n_failed and row["n_missed_safe"] == 0
        assert row["n_detect_safe"] == len(r.frontier) and row["n_false_safe"] == r.n_false
        assert (row["frontier_cells"], row["occupied_cells"]) == (r.m, r.C)
        assert row["rho_flagged"] == r.n_rho and row["rho_hit"] == r.n_rho_hit
        assert abs(row["frontier_entropy"] - r.H) <= 1e-6 and abs(row["candidate_entropy"] - r.H_cand) <= 1e-6
        assert abs(row["gyration"] - r.gyration) <= 1e-5 and abs(row["compactness"] - r.compactness) <= 1e-5
        assert row["clearance_pressure"] == r.n_failed / n
        assert row["eps_t"] == float(r.eps_t)
        for col in ("t_grid_repair_s", "t_grid_rebuild_s", "t_full_s", "t_frontier_s"):
            assert row[col] is not None and row[col] > 0
        assert row["best_strategy"] in ("grid_repair", "grid_rebuild", "full")
        ref = r.cert

"""The transition log's host side: a per-scene result row becomes a log row
with the paper's dataset columns; the best strategy is the fastest timed full
strategy; JSONL round-trips."""
import numpy as np

from paper_2606_18314_b300 import cert, translog


def _row():
    r = np.zeros(1, cert.SCENE_DTYPE)[0]
    r["eps_t"], r["n_failed"], r["H"], r["H_cand"] = np.float32(9.5e-4), 40, 0.61, 0.92
    r["compactness"], r["gyration"], r["failed_cells"], r["occupied_cells"] = 0.3, 0.12, 37, 900
    r["n_frontier"], r["n_missed"], r["n_false"], r["n_rho"], r["n_rho_hit"] = 300, 0, 260, 120, 38
    r["strategy"] = cert.CERT_INCREMENTAL
    return r


META = {"family": "clustered_drift", "n": 1000, "dim": 3, "eps": 1e-3, "seed": 1, "frame": 4}


def test_record_maps_every_column():
    out = translog.record(_row(), META, {"grid_repair": 2e-4, "grid_rebuild": 5e-4, "full": 3e-3, "frontier": 1e-3})
    assert out["clearance_pressure"] == 40 / 1000
    assert out["frontier_entropy"] == 0.61 and out["candidate_entropy"] == 0.92
    assert (out["frontier_cells"], out["occupied_cells"]) == (37, 900)
    assert (out["n_detect_safe"], out["n_missed_safe"], out["n_false_safe"]) == (300, 0, 260)
    assert (out["rho_flagged"], out["rho_hit"]) == (120, 38)
    assert out["eps_t"] == float(np.float32(9.5e-4))
    assert out["best_strategy"] == "grid_repair" and out["speedup_vs_rebuild"] == 2.5
    assert out["t_frontier_s"] == 1e-3 and out["t_full_s"] == 3e-3
    for k, v in META.items():
        assert out[k] == v


def test_best_strategy_is_the_fastest_timed_one():
    out = translog.record(_row(), META, {"grid_repair": 7e-4, "grid_rebuild": 5e-4})
    assert out["best_strategy"] == "grid_rebuild" and out["speedup_vs_rebuild"] == 1.0
    assert out["t_full_s"] is None and out["t_frontier_s"] is None
    out = translog.record(_row(), META, None)
    assert out["best_strategy"] is None and out["t_grid_repair_s"] is None


def test_jsonl_round_trip(tmp_path):
    rows = [translog.record(_row(), dict(META, frame=k), {"grid_repair": 1e-4 * k}) for k in range(1, 4)]
    p = tmp_path / "log.jsonl"
    translog.write(p, rows)
    assert translog.read(p) == rows
    assert len(p.read_text().splitlines()) == 3

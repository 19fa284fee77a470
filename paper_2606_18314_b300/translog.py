"""Per-step transition log (JSONL).

The paper releases its transitions as a table (Sec. 6): the motion
parameters, dimension and frame; frontier descriptors (clearance pressure,
frontier entropy, compactness, gyration, frontier cells, occupied cells); the
certificate-failure audit (eps_t, detected, missed and false counts, the rho
heuristic's counts); the measured time of each strategy; and the best
strategy.  This module writes the same columns for scenes stepped through
this library, one JSON object per scene per step:

* ``record`` turns one per-scene result row (``cert.SCENE_DTYPE``) and the
  step's timings into a row of the log (pure, no GPU);
* ``log_scene`` steps one seeded scene of a motion family with both audits on,
  times the three full strategies from identical state (snapshot / restore)
  and the frontier oracle (the exact all-pairs pass over the detected frontier),
  continues from the incremental step, and returns (and optionally writes) the
  rows.

    python -m paper_2606_18314_b300.translog --family clustered_drift \\
        --n 16000 --dim 3 --eps 1e-3 --steps 50 --out transitions.jsonl

Clearance pressure is the failure fraction |F_t| / N with F_t the failed
certificates (Def. 2); the detected frontier is the safety rule's set.
"""
from __future__ import annotations

import argparse
import json

from . import scenes

STRATEGY_COLUMNS = {"grid_repair": "t_grid_repair_s", "grid_rebuild": "t_grid_rebuild_s", "full": "t_full_s"}


def record(row, meta: dict, times: dict | None = None) -> dict:
    """One log row from a per-scene result (a ``cert.SCENE_DTYPE`` record).
    ``meta`` holds the motion parameters (family, n, dim, eps, seed, frame);
    ``times`` maps "grid_repair", "grid_rebuild", "full" and "frontier" to
    seconds (any subset).  The best strategy is the fastest of the three full
    ones that were timed."""
    n = int(meta["n"])
    out = dict(meta)
    out.update({
        "eps_t": float(row["eps_t"]),
        "clearance_pressure": int(row["n_failed"]) / n,
        "frontier_entropy": float(row["H"]),
        "candidate_entropy": float(row["H_cand"]),
        "compactness": float(row["compactness"]),
        "gyration": float(row["gyration"]),
        "frontier_cells": int(row["failed_cells"]),
        "occupied_cells": int(row["occupied_cells"]),
        "n_failed": int(row["n_failed"]),
        "n_detect_safe": int(row["n_frontier"]),
        "n_missed_safe": int(row["n_missed"]),
        "n_false_safe": int(row["n_false"]),
        "rho_flagged": int(row["n_rho"]),
        "rho_hit": int(row["n_rho_hit"]),
        "strategy_applied": int(row["strategy"]),
    })
    times = times or {}
    for k, col in STRATEGY_COLUMNS.items():
        out[col] = float(times[k]) if k in times else None
    out["t_frontier_s"] = float(times["frontier"]) if "frontier" in times else None
    timed = {k: times[k] for k in STRATEGY_COLUMNS if k in times}
    if timed:
        best = min(timed, key=timed.get)
        out["best_strategy"] = best
        out["speedup_vs_rebuild"] = timed["grid_rebuild"] / timed[best] if "grid_rebuild" in timed else None
    else:
        out["best_strategy"] = None
        out["speedup_vs_rebuild"] = None
    return out


def write(path, rows) -> None:
    with open(path, "w") as f:
        for r in rows:
            f.write(json.dumps(r) + "\n")


def read(path) -> list:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def _timed(torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def log_scene(cert, family, n, dim, eps, steps, seed=1, time_strategies=True, out=None) -> list:
    """Step one scene ``steps`` times and return its log rows (written to
    ``out`` as JSONL when given)."""
    import torch
    m = scenes.Motion(family, n, dim, eps, seed=seed, steps=max(steps, 64))
    frames = torch.from_numpy(m.frames(steps)).cuda()
    ctx = cert.Context(frames[0], audit=("rho", "geometry"))
    rows = []
    try:
        for t in range(1, steps + 1):
            times = {}
            if time_strategies:
                ctx.snapshot()
                for name, strat in (("grid_rebuild", cert.CERT_REBUILD), ("full", cert.CERT_ALLPAIRS)):
                    times[name] = _timed(torch, lambda: ctx.step(frames[t], eps, strat))
                    ctx.restore()
                times["grid_repair"] = _timed(torch, lambda: ctx.step(frames[t], eps, cert.CERT_INCREMENTAL))
            else:
                ctx.step(frames[t], eps, cert.CERT_INCREMENTAL)
            res, _ = ctx.sync()
            if time_strategies:
                nf = int(res[0]["n_frontier"])
                if nf > 0:
                    q = ctx.views()["frontier"][:nf].clone()
                    times["frontier"] = _timed(torch, lambda: cert.cert_allpairs(frames[t], q))
            meta = {"family": family, "n": n, "dim": dim, "eps": eps, "seed": seed, "frame": t}
            rows.append(record(res[0], meta, times))
    finally:
        ctx.close()
    if out:
        write(out, rows)
    return rows


def main():
    ap = argparse.ArgumentParser(description="per-step transition log (JSONL) of one seeded scene")
    ap.add_argument("--family", default="clustered_drift", choices=list(scenes.ALL_FAMILIES))
    ap.add_argument("--n", type=int, default=16000)
    ap.add_argument("--dim", type=int, default=3, choices=[2, 3])
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-timing", action="store_true")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    from . import build, cert
    build.build()
    rows = log_scene(cert, args.family, args.n, args.dim, args.eps, args.steps, args.seed,
                     time_strategies=not args.no_timing, out=args.out)
    print(f"{len(rows)} transitions -> {args.out}")


if __name__ == "__main__":
    main()

"""Matched-pair entropy experiment (Sec. 4, Fig. 2) on the GPU path.

The paper isolates the effect of the repair-frontier entropy H (Def. 2) by
pairing two transitions that fail almost the same number of certificates
(within a matching tolerance) but spread them differently: a localized one
(adversarial crossing) and a diffuse one (ring rotation).  Its event-driven
host repair costs about twice as much on the diffuse member, because the cell
loop of Algorithm 1 touches more index cells (Thm A.4: m >= C^H), while the
GPU repair, which treats every frontier point in parallel, does not depend on
H.

This module runs that experiment on this library:

* ``survey`` steps one seeded scene of a family through the GPU path and
  records the per-transition counts (failures, H, the cells m they meet, the
  detected frontier and the cells it meets) and the failures' gyration and
  compactness;
* ``select`` picks, as the paper does, the pair whose failure counts agree
  within the tolerance and whose entropies differ most;
* ``time_transition`` replays one transition back and forth (the failing set
  of t -> t+1 and of t+1 -> t is the same) from CUDA graphs and times it with
  CUDA events, for one scene or a batch of seeds of the same transition.

Inputs come from ``scenes.Motion``; every number is the GPU path's own.
"""
from __future__ import annotations

import numpy as np

from . import scenes

LOCALIZED = "adversarial_crossing"
DIFFUSE = "ring_rotation"
TOLERANCE = 0.12          # |f_a - f_b| <= TOLERANCE * max(f_a, f_b); the paper's pair is 370 vs 414


def frames_at(family, n, dim, eps, seed, t, horizon):
    """Positions of the scene before and after transition t (float32 [2][n][dim])."""
    m = scenes.Motion(family, n, dim, eps, seed=seed, steps=horizon)
    for _ in range(t):
        m.advance()
    return np.stack([m.frame(), m.advance()])


def survey(cert, family, n, dim, eps, steps, seed=1, horizon=None):
    """Step one scene through ``steps`` transitions (incremental, exact) and
    return (frames [steps+1][n][dim], rows), one row per transition."""
    import torch
    horizon = horizon or max(steps, 64)
    fr = scenes.Motion(family, n, dim, eps, seed=seed, steps=horizon).frames(steps)
    dev = torch.from_numpy(fr).cuda()
    ctx = cert.Context(dev[0], audit="geometry")
    rows = []
    try:
        for t in range(steps):
            ctx.step(dev[t + 1], eps, cert.CERT_INCREMENTAL)
            r, _ = ctx.sync()
            r = r[0]
            rows.append({"family": family, "eps": eps, "t": t, "n_failed": int(r["n_failed"]),
                         "H": float(r["H"]), "m": int(r["failed_cells"]), "C": int(r["occupied_cells"]),
                         "n_frontier": int(r["n_frontier"]), "frontier_cells": int(r["frontier_cells"]),
                         "n_searched": int(r["n_searched"]), "n_missed": int(r["n_missed"]),
                         "gyration": float(r["gyration"]), "compactness": float(r["compactness"])})
    finally:
        ctx.close()
    return fr, rows


def select(rows_a, rows_b, tol=TOLERANCE, min_failed=16):
    """The pair (row of a, row of b) with failure counts matched within ``tol``
    and H_b - H_a largest (ties: the closer counts); None when no pair matches
    with H_b > H_a."""
    best, key = None, None
    for a in rows_a:
        for b in rows_b:
            fa, fb = a["n_failed"], b["n_failed"]
            if min(fa, fb) < min_failed or abs(fa - fb) > tol * max(fa, fb):
                continue
            dh = b["H"] - a["H"]
            if dh <= 0:
                continue
            k = (dh, -abs(fa - fb))
            if key is None or k > key:
                best, key = (a, b), k
    return best


def batch_frames(family, n, dim, eps, t, seeds, horizon):
    """Transition t of ``len(seeds)`` scenes of one family (one per seed),
    concatenated: (frames [2][B*n][dim], offsets)."""
    fr = [frames_at(family, n, dim, eps, s, t, horizon) for s in seeds]
    offsets = np.arange(len(seeds) + 1, dtype=np.int64) * n
    return np.concatenate(fr, axis=1), offsets


def time_transition(cert, frames2, offsets, eps, strategy, steps=200, warm=4):
    """Milliseconds per step of the transition frames2[0] -> frames2[1],
    replayed back and forth from a CUDA graph of two steps (CUDA events on the
    launching stream), and the per-scene results of the last forward step."""
    import torch
    dev = torch.from_numpy(np.ascontiguousarray(frames2)).cuda()
    ctx = cert.Context(dev[0], offsets=offsets)
    try:
        for k in range(warm):
            ctx.step(dev[(k + 1) % 2], eps, strategy)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.step(dev[1], eps, strategy)
            ctx.step(dev[0], eps, strategy)
        torch.cuda.synchronize()
        reps = max(1, steps // 2)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (2 * reps)
        ctx.step(dev[1], eps, strategy)
        res, _ = ctx.sync()
        del g
    finally:
        ctx.close()
    return ms, res


def frontier_query_ms(cert, pos, failed_idx, reps=20):
    """The paper's frontier oracle: exact all-pairs top-2 of the failed points
    against every point (cert_allpairs with a query list), ms per call."""
    import torch
    p = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    q = torch.from_numpy(np.ascontiguousarray(failed_idx, np.int32)).cuda()
    cert.cert_allpairs(p, q)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        cert.cert_allpairs(p, q)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run(cert, n=16000, dim=3, steps=48, eps_a=1e-3, eps_b=(1e-3, 5e-4, 2.5e-4, 1.25e-4),
        batch=64, time_steps=200):
    """The whole experiment: survey, select, time.  Returns a JSON-able dict
    (None under "pair" when no transitions match)."""
    import torch
    horizon = max(steps, 64)
    fa, rows_a = survey(cert, LOCALIZED, n, dim, eps_a, steps, horizon=horizon)
    rows_b, frames_b = [], {}
    for e in eps_b:
        fb, rb = survey(cert, DIFFUSE, n, dim, e, steps, horizon=horizon)
        rows_b += rb
        frames_b[e] = fb
    pair = select(rows_a, rows_b)
    out = {"n": n, "dim": dim, "tolerance": TOLERANCE, "surveyed": len(rows_a) + len(rows_b), "pair": None}
    if pair is None:
        return out
    members = []
    for row, fr in ((pair[0], fa), (pair[1], frames_b[pair[1]["eps"]])):
        t, eps = row["t"], row["eps"]
        one = fr[t:t + 2]
        off1 = np.array([0, n], np.int64)
        inc_ms, res = time_transition(cert, one, off1, eps, cert.CERT_INCREMENTAL, time_steps)
        reb_ms, _ = time_transition(cert, one, off1, eps, cert.CERT_REBUILD, time_steps)
        # the failing set of this transition, for the frontier oracle
        p0 = torch.from_numpy(np.ascontiguousarray(one[0])).cuda()
        p1 = torch.from_numpy(np.ascontiguousarray(one[1])).cuda()
        nn0 = cert.cert_allpairs(p0)[0].cpu().numpy()
        nn1 = cert.cert_allpairs(p1)[0].cpu().numpy()
        failed = np.flatnonzero(nn0 != nn1).astype(np.int32)
        fq_ms = frontier_query_ms(cert, one[1], failed)
        seeds = list(range(1, batch + 1))
        fb2, offb = batch_frames(row["family"], n, dim, eps, t, seeds, horizon)
        binc_ms, bres = time_transition(cert, fb2, offb, eps, cert.CERT_INCREMENTAL, time_steps)
        bsearched = int(bres["n_searched"].sum())
        members.append(dict(row, C_pow_H=float(row["C"] ** row["H"]),
                            incremental_ms=inc_ms, rebuild_ms=reb_ms, frontier_query_ms=fq_ms,
                            batch={"scenes": batch, "points": batch * n, "incremental_ms": binc_ms,
                                   "n_failed": int(bres["n_failed"].sum()),
                                   "H_mean": float(bres["H"].mean()),
                                   "n_frontier": int(bres["n_frontier"].sum()), "n_searched": bsearched,
                                   "ns_per_searched": binc_ms * 1e6 / max(1, bsearched),
                                   "n_missed": int(bres["n_missed"].sum())}))
    out["pair"] = members
    a, b = members
    out["failed_ratio"] = b["n_failed"] / a["n_failed"]
    out["cells_ratio"] = b["m"] / max(1, a["m"])
    out["incremental_ratio"] = b["incremental_ms"] / a["incremental_ms"]
    out["batch_incremental_ratio"] = b["batch"]["incremental_ms"] / a["batch"]["incremental_ms"]
    out["batch_ns_per_searched_ratio"] = b["batch"]["ns_per_searched"] / a["batch"]["ns_per_searched"]
    return out

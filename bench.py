"""Benchmark of the certificate-maintenance loop on B300 (one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|c1|c2|c3] [--strategy auto|incremental|rebuild|allpairs]

Metric: certified point-updates/s = (points of every scene) x (steps) / time,
every certificate exact after each step.  A step is one pass of the whole
path -- eps_t, frontier compaction, index rebuild, strategy selection, repair
or rebuild, failure marks, H(F_t), audit -- over all scenes of the workload.

Default workload: 512 independent scenes, N log-uniform in [500, 16000],
d = 3, the five motion families mixed (scene s takes family s mod 5),
eps = 1e-3.  The motion is F = 100 pre-generated forward frames (the
benchmark configuration's 100 steps); the warm-up steps walk forward from
frame 0 and the timed steps continue forward from there.  Past frame F the
walk turns back (a ping-pong over the F+1 frames), every step within eps.
The schedule repeats every 2F steps, so at most two CUDA graphs (a 2F-step
one replayed, and a remainder) are captured and replayed.  `forward_100`
reports the 100 forward steps alone, from frame 0, as one graph.

Inputs are synthetic (seeded Philox motion families; no dataset).  The
working set (positions, certificates, index) exceeds the 126 MB L2, so no
explicit L2 flush is done between steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_18314_b300 import scenes  # noqa: E402

METRIC = "certified point-updates/s"
UNIT = "point-updates/s"
KERNELS_PER_STEP = 7   # prepare, scan, select, scatter_refresh, search, far, finalize

# Per-phase algorithmic (compulsory DRAM) bytes.
#   prepare: read p' (4 dim) + p (16), write packed p' (16), (bucket, rank) (8), cell (4),
#            bucket-count and cell-count atomics (8 + 8)
#   scan:    read d1^2, d2^2 (8), write frontier flag (1) per point; bucket count read +
#            start write (8) per bucket; frontier index (4) per frontier point
#   scatter_refresh: read (bucket, rank) 8 + bucket start 4 + p' 16, write sorted 16 + flag 1;
#            points of incrementally repaired scenes also read nn, nn2, nn3 12 + L 4 + inF 1 +
#            three neighbour positions 48; the refreshed ones write nn, nn2, nn3, d1^2, d2^2, L 24 +
#            failed 1
#   search:  read flag (1) per point; per searched point read query 16 + old nn 4 + inF 1 +
#            cell 4, write certificate 24 + failed 1
PHASES = ["clear", "prepare", "scan", "select", "scatter_refresh", "search", "finalize"]


def phase_bytes(ph, N, dim, n_buckets, n_front, n_searched, zero_bytes, n_tried=None):
    """n_tried: points of scenes repaired incrementally (they try the O(1) refresh)."""
    n_tried = N if n_tried is None else n_tried
    refreshed = max(0, n_tried - (n_searched - (N - n_tried)))
    if ph == "clear":
        return zero_bytes
    if ph == "prepare":
        return N * (4 * dim + 16 + 16 + 8 + 4 + 16)
    if ph == "scan":
        return N * 9 + n_buckets * 8 + n_front * 4
    if ph == "scatter_refresh":
        return N * (8 + 4 + 16 + 16 + 1) + n_tried * (12 + 4 + 1 + 48) + refreshed * (24 + 1)
    if ph == "search":
        return N * 1 + n_searched * (16 + 4 + 1 + 4 + 24 + 1)
    return 0


# DRAM bytes (read + write) of one k_search launch on the batched 512-scene
# incremental step, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum), per search-grid cell scale the autotuner may pick,
# with the source fingerprint of the step kernels' translation unit they ran
# on.  The bench line carries the figure only while the loaded library
# reports the same fingerprint and the run uses one of these cell scales;
# otherwise it reports null until the capture is taken again.
SEARCH_TRAFFIC = {"fingerprint": "7e980e0ec3212d41", "commit": "9821c35",
                  "bytes": {3.5: 161.80e6, 4.0: 160.95e6}}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"cert_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(name, rank, frames, n_scenes=512, family=None, workers=1):
    """(frames [F+1][N][dim], scene offsets, eps, config) of a named workload;
    ``workers`` > 1 generates the batched scenes in a pool of spawned processes."""
    if name == "batched":
        bm = scenes.BatchMotion.mixed(n_scenes=n_scenes, dim=3, eps=1e-3, seed=4 + 1000 * rank, steps=100)
        if family:   # diagnostics: every scene of one family (same sizes and seeds)
            bm = scenes.BatchMotion([scenes.Motion(family, m.n, 3, 1e-3, seed=m.seed, steps=100)
                                     for m in bm.scenes])
        fr = bm.frames_parallel(frames, workers) if workers > 1 and frames >= 8 else bm.frames(frames)
        return fr, bm.offsets, 1e-3, {
            "workload": f"batched-{n_scenes}-scenes", "scenes": n_scenes, "n_range": [500, 16000], "dim": 3,
            "eps": 1e-3,
            "families": list(scenes.FAMILIES)}
    if name == "c2":
        m = scenes.Motion("uniform_brownian", 16000, 3, 1e-3, seed=1 + rank, steps=200)
        return m.frames(frames), np.array([0, 16000], np.int64), 1e-3, {
            "workload": "single-scene-16000-d3", "scenes": 1, "n": 16000, "dim": 3, "eps": 1e-3,
            "families": ["uniform_brownian"]}
    if name == "c1":
        m = scenes.Motion("uniform_brownian", 1000, 2, 1e-3, seed=1 + rank, steps=20)
        return m.frames(frames), np.array([0, 1000], np.int64), 1e-3, {
            "workload": "single-scene-1000-d2", "scenes": 1, "n": 1000, "dim": 2, "eps": 1e-3,
            "families": ["uniform_brownian"]}
    if name == "c3":
        m = scenes.Motion("uniform_clusters", 262144, 3, 1e-4, seed=1 + rank, steps=100)
        return m.frames(frames), np.array([0, 262144], np.int64), 1e-4, {
            "workload": "single-scene-262144-d3-clusters", "scenes": 1, "n": 262144, "dim": 3, "eps": 1e-4,
            "families": ["uniform_clusters"]}
    raise SystemExit(f"unknown workload {name}")


def cycle_index(k, F):
    """Frame targeted by step k of the ping-pong cycle over frames 0..F."""
    r = k % (2 * F)
    return r + 1 if r < F else 2 * F - r - 1


def cpu_baseline(frames, offsets, dim, budget_s, per_step_budget=None, steps_exact=None, warmup=0):
    """The oracle as it stands on this host's cores over a bounded sample:
    whole scenes in a seeded random order (as many as fit the per-step budget,
    at least one), stepped through the same frames; ``warmup`` untimed steps
    first."""
    import oracle
    S = len(offsets) - 1
    sizes = np.diff(offsets)
    order = np.random.default_rng(16).permutation(S)
    # pick scenes whose brute-force cost fits the per-step budget (~1 ns per pair per thread)
    thr = max(1, oracle.max_threads())
    target = per_step_budget if per_step_budget else budget_s / 4.0
    chosen, cost = [], 0.0
    for s in order:
        c = float(sizes[s]) ** 2 * 2.5e-9 / thr
        if chosen and cost + c > target:
            break
        chosen.append(int(s))
        cost += c
    certs = {s: oracle.top2(frames[0][offsets[s]:offsets[s + 1]]) for s in chosen}
    F = frames.shape[0] - 1
    prev = 0
    for w in range(warmup):
        k = cycle_index(w, F)
        for s in chosen:
            r = oracle.step(frames[prev][offsets[s]:offsets[s + 1]], frames[k][offsets[s]:offsets[s + 1]], certs[s])
            certs[s] = r.cert
        prev = k
    pts, steps, t0 = 0, 0, time.perf_counter()
    while True:
        k = cycle_index(steps + warmup, F)
        for s in chosen:
            a, b = frames[prev][offsets[s]:offsets[s + 1]], frames[k][offsets[s]:offsets[s + 1]]
            r = oracle.step(a, b, certs[s])
            certs[s] = r.cert
            pts += b.shape[0]
        prev = k
        steps += 1
        if steps_exact is not None:
            if steps >= steps_exact:
                break
        elif time.perf_counter() - t0 >= budget_s or steps >= 10000:
            break
    el = time.perf_counter() - t0
    return {"value": pts / el, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{len(chosen)} of {S} scenes (seeded random, {int(sizes[chosen].sum())} points), "
                      f"{steps} steps in {el:.1f} s"}, steps, el


def run_reference(args, rank, world):
    if rank != 0:
        return
    frames, offsets, eps, cfg = make_workload(args.workload, 0, max(4, args.frames), args.scenes,
                                              workers=args.gen_workers or min(16, os.cpu_count() or 1))
    dim = frames.shape[2]
    per_step = max(0.02, 120.0 / max(1, args.steps + args.warmup))
    cb, steps, el = cpu_baseline(frames, offsets, dim, budget_s=per_step * args.steps, per_step_budget=per_step,
                                 steps_exact=max(1, args.steps), warmup=max(0, args.warmup))
    cfg = dict(cfg)
    cfg["l2"] = "host oracle (no GPU)"
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": max(0, args.warmup), "ms_per_step": 1e3 * el / max(1, steps),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(ms, n_points, dist=None, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's milliseconds and the
    points all ranks processed (scenes are independent, so nothing else is
    exchanged)."""
    if dist is None:
        return ms, n_points
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    nt = torch.tensor([float(n_points)], dtype=torch.float64, device=device)
    dist.all_reduce(nt)
    return float(t.item()), int(nt.item())


def capture_steps(ctx, dev_frames, F, eps, strategy, start, count, torch):
    """One CUDA graph of ``count`` steps whose step k targets frame
    cycle_index(start + k)."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(count):
            ctx.step(dev_frames[cycle_index(start + k, F)], eps, strategy)
    return g


def graph_loop(ctx, dev_frames, F, eps, strategy, K, use_graph, stream, torch, start=0):
    """Time K steps from clock ``start`` (the state sits at frame
    cycle_index(start - 1), frame 0 for start = 0): step k targets frame
    cycle_index(start + k).  The schedule repeats every 2F steps, so one graph
    of 2F steps is captured and replayed, plus one graph for the remainder.
    Returns (ms, steps taken)."""
    C = 2 * F
    graphs = []
    if use_graph:
        full, rem = divmod(K, C)
        if full:
            graphs.append((capture_steps(ctx, dev_frames, F, eps, strategy, start, C, torch), full))
        if rem:
            graphs.append((capture_steps(ctx, dev_frames, F, eps, strategy, start, rem, torch), 1))
        torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    if graphs:
        for g, reps in graphs:
            for _ in range(reps):
                g.replay()
    else:
        for k in range(K):
            ctx.step(dev_frames[cycle_index(start + k, F)], eps, strategy)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), K


def knn_buckets(n):
    """Hashed-grid buckets per level of a kNN context: next_pow2(n), at most 2^23."""
    T = 1
    while T < n and T < (1 << 23):
        T <<= 1
    return T


def knn_phase_bytes(ph, n, dim, k, buckets, n_searched, n_refreshed):
    """Compulsory DRAM bytes of one kNN step phase.  The certificate keeps
    S = k + 3 ranks (int32 index + float32 key each) in [S][n] arrays; the
    bucket counters and starts cover both grid levels (2T)."""
    S = k + 3
    if ph == "prepare":      # read input + old position, write position, bucket, rank; the counters once
        return n * (4 * dim + 40) + 8 * buckets
    if ph == "scan":         # read the counts twice, write the starts, zero the counts
        return 16 * buckets
    if ph == "refresh":      # bucket, rank, start, position, scatter; frontier ranks; list read; refreshed writes
        return n * (58 + 4 * S) + n_refreshed * (8 * S + 5)
    if ph == "search":       # list entry, position, hint, old k indices, new list, L, flag
        return n_searched * (29 + 4 * k + 8 * S)
    return 0


def launch_floor(torch, steps, nodes_per_step, stream):
    """ms per step of a CUDA graph holding ``nodes_per_step`` dependent
    one-element kernels per step: the replay cost of a step's launches alone
    (the fastest of five replays)."""
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(steps * nodes_per_step):
            x.add_(1.0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(5):                 # the fastest of five replays
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best / steps


def single_scene_report(cert, torch, steps, stream):
    """The single-scene configurations (N = 1,000 d = 2; 16,000 d = 3;
    262,144 d = 3 clustered), whose state fits in L2: step time under graph
    replay for each plain strategy, against the launch floor of the same
    number of graph nodes (7 kernels and 1 memset per step)."""
    F = 8
    C = 2 * F
    K = max(C, (steps // C) * C)
    floor = launch_floor(torch, K, KERNELS_PER_STEP + 1, stream)
    out = {"steps": K, "floor_ms_per_step": floor,
           "floor": f"CUDA graph of {KERNELS_PER_STEP + 1} dependent one-element kernels per step", "rows": []}
    for name in ("c1", "c2", "c3"):
        frames, offsets, eps, cfg = make_workload(name, 0, F)
        n, dim = frames.shape[1], frames.shape[2]
        dev = torch.from_numpy(frames).cuda()
        row = {"workload": cfg["workload"], "n": n, "dim": dim, "eps": eps}
        for strat in ("incremental", "rebuild"):
            ctx = cert.Context(dev[0])
            for k in range(C):            # one eager cycle: back at frame 0
                ctx.step(dev[cycle_index(k, F)], eps, cert.STRATEGY[strat])
            ms, _ = graph_loop(ctx, dev, F, eps, cert.STRATEGY[strat], K, True, stream, torch)
            res, rc = ctx.sync(raise_on_status=False)
            assert rc == cert.CERT_OK and int(res["n_missed"].sum()) == 0, f"{name} {strat}: rc {rc}"
            ctx.close()
            row[f"{strat}_ms_per_step"] = ms / K
            row[f"{strat}_point_updates_per_s"] = n * K / (ms * 1e-3)
            row[f"{strat}_x_floor"] = (ms / K) / floor
        out["rows"].append(row)
        del dev
    return out


def knn_report(cert, torch, steps, peaks, stream):
    """k-nearest-neighbour certificates (the richer certificates the paper
    leaves open): point-updates/s with the steps replayed from a CUDA graph,
    per-phase times from CUDA events, and the roofline of the dominant phase."""
    out = {"peak_gbs": peaks["hbm_gbs"], "rows": []}
    cases = [("uniform_clusters", 262144, 3, 1e-4, (1, 4, 8, 16)), ("uniform_brownian", 2097152, 3, 1e-4, (8,))]
    for family, n, dim, eps, ks in cases:
        m = scenes.Motion(family, n, dim, eps, seed=1, steps=100)
        F = 3
        dev_frames = torch.from_numpy(m.frames(F)).cuda()
        for k in ks:
            row = {"workload": f"{family}-{n}-d{dim}", "n": n, "k": k, "eps": eps}
            for name in ("incremental", "rebuild"):
                ctx = cert.KnnContext(dev_frames[0], k)
                for j in range(2 * F):
                    ctx.step(dev_frames[cycle_index(j, F)], eps, name)
                ms, _ = graph_loop(ctx, dev_frames, F, eps, cert.STRATEGY[name], max(2 * F, steps), True, stream,
                                   torch)
                K = max(2 * F, steps) // (2 * F) * (2 * F)
                row[name] = {"point_updates_per_s": n * K / (ms / 1e3), "ms_per_step": ms / K}
                # phase times over one cycle, eager, from the same state
                ph = {p: 0.0 for p in cert.KnnContext.KNN_PHASES}
                cnt = np.zeros(4)
                for j in range(2 * F):
                    t = ctx.profile(dev_frames[cycle_index(j, F)], eps, name)
                    r, _ = ctx.sync()
                    assert r["n_missed"] == 0, "kNN safety rule missed a failure"
                    for p_ in ph:
                        ph[p_] += t[p_] / (2 * F)
                    cnt += [r["n_frontier"], r["n_failed"], r["n_searched"], r["grid_res"]]
                cnt /= 2 * F
                buckets = 2 * knn_buckets(n)
                phases = {}
                for p_, t_ms in ph.items():
                    b = knn_phase_bytes(p_, n, dim, k, buckets, cnt[2], n - cnt[2] if name == "incremental" else 0)
                    phases[p_] = {"ms": t_ms, "bytes": b, "gbs": b / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0}
                dom = max((p_ for p_ in phases if p_ != "finalize"), key=lambda p_: phases[p_]["ms"])
                row[name].update({"frontier_frac": cnt[0] / n, "failed_frac": cnt[1] / n, "searched_frac": cnt[2] / n,
                                  "grid_res": int(cnt[3]), "phases": phases, "dominant": dom,
                                  "roofline_frac": phases[dom]["gbs"] / peaks["hbm_gbs"]})
                ctx.close()
            out["rows"].append(row)
        del dev_frames
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "c1", "c2", "c3"])
    ap.add_argument("--strategy", default="auto",
                    choices=["auto", "incremental", "rebuild", "allpairs", "threshold"])
    ap.add_argument("--frames", type=int, default=100, help="pre-generated forward frames")
    ap.add_argument("--gen-workers", type=int, default=0, help="processes generating the frames (0: host cores)")
    ap.add_argument("--sustained-ms", type=float, default=500.0,
                    help="length of the extra sustained replay (0: skip)")
    ap.add_argument("--scenes", type=int, default=512, help="scenes in the batched workload")
    ap.add_argument("--family", default=None, choices=list(scenes.FAMILIES), help="diagnostics: one family only")
    ap.add_argument("--cell-scale", type=float, default=0.0, help="search-grid cell side / reference d2 (0: default)")
    ap.add_argument("--cell-quantile", type=float, default=0.0, help="d2 quantile of the reference (0: default)")
    ap.add_argument("--bucket-factor", type=int, default=0, help="hashed buckets per scene / next_pow2(n)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--clocks-out", default=None, help="keep the nvidia-smi clock samples here ({rank} expands)")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--prof-steps", type=int, default=200)
    ap.add_argument("--regret-steps", type=int, default=32)
    ap.add_argument("--rule-steps", type=int, default=32, help="steps per frontier rule in the detection report")
    ap.add_argument("--matched-steps", type=int, default=48,
                    help="transitions surveyed per scene in the matched-pair entropy experiment (0: skip)")
    ap.add_argument("--knn-steps", type=int, default=240,
                    help="graph-replayed steps per k-nearest-neighbour case (0: skip)")
    ap.add_argument("--compare-steps", type=int, default=256)
    ap.add_argument("--scene-regret-steps", type=int, default=24,
                    help="steps of the per-scene cost attribution and regret (0: skip)")
    ap.add_argument("--flip-steps", type=int, default=64,
                    help="steps per variant of the per-family strategy flips inside the batch (0: skip)")
    ap.add_argument("--single-steps", type=int, default=256,
                    help="graph-replayed steps per single-scene configuration (0 to skip)")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--allpairs-sizes", default="40000,80000,200000",
                    help="sizes for the all-pairs timing ('' to skip)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2606_18314_b300 import build as cbuild
    from paper_2606_18314_b300 import cert, selector
    cbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    F = max(2, args.frames)
    C = 2 * F
    workers = args.gen_workers or min(16, os.cpu_count() or 1)
    frames, offsets, eps, cfg = make_workload(args.workload, rank, F, args.scenes, args.family, workers)
    if args.family:
        cfg = dict(cfg, families=[args.family])
    N, dim = frames.shape[1], frames.shape[2]
    S = len(offsets) - 1
    dev_frames = torch.from_numpy(frames).cuda()
    strat = cert.STRATEGY[args.strategy]
    stream = torch.cuda.current_stream()
    use_graph = not args.no_graph

    ctx = cert.Context(dev_frames[0], offsets=offsets, cell_scale=args.cell_scale, cell_quantile=args.cell_quantile,
                       bucket_factor=args.bucket_factor)
    clock = [0]   # steps taken along the ping-pong cycle; the state sits at frame cycle_index(clock-1)

    def do_step(strategy=strat):
        ctx.step(dev_frames[cycle_index(clock[0], F)], eps, strategy)
        clock[0] += 1

    def to_cycle_start(strategy=strat):
        while clock[0] % C:
            do_step(strategy)

    sel_meta = None
    if args.strategy == "auto":
        if not os.path.exists(selector.WEIGHTS):
            raise SystemExit(f"selector weights missing ({selector.WEIGHTS}); "
                             "run python -m paper_2606_18314_b300.selector collect/train")
        params, norm = selector.load()
        ctx.load_selector(params, norm)
        sel_meta = json.loads(str(np.load(selector.WEIGHTS)["meta"]))

    # warm-up: W eager steps forward from frame 0 (the autotuner's probe steps,
    # below, run from a snapshot and leave the state where it was)
    W = max(3, args.warmup)
    for _ in range(W):
        do_step()
    tuned = None
    if not args.no_autotune:
        idx = [cycle_index(clock[0] + k, F) for k in range(min(8, C))]
        probe = torch.stack([dev_frames[i] for i in idx]).contiguous()
        scales = (2.0, 2.5, 3.0, 3.5, 4.0, 5.0)
        best, ms_sc = ctx.autotune(probe, eps, strat if strat != cert.CERT_ALLPAIRS else cert.CERT_INCREMENTAL,
                                   scales)
        tuned = {"scales": list(scales), "ms": [float(x) for x in ms_sc], "best": best}
        del probe
    torch.cuda.synchronize()
    ctx.sync(raise_on_status=False)
    t_start = clock[0]

    # ---- the timed region: K steps of the chosen strategy
    K = args.steps
    sampler = ClockSampler(local, args.clocks_out.replace("{rank}", str(rank)) if args.clocks_out else None)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    ms, _ = graph_loop(ctx, dev_frames, F, eps, strat, K, use_graph, stream, torch, start=clock[0])
    clock[0] += K
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    res, rc = ctx.sync(raise_on_status=False)
    assert int(res["n_missed"].sum()) == 0, "safety rule missed a failure"
    ms_max, n_all = aggregate(ms, N, dist, "cuda")
    value = n_all * K / (ms_max / 1e3)
    fwd_steps = max(0, min(K, F - t_start))   # timed steps that moved forward, before any turn
    motion = {"timed_from_frame": t_start, "forward_steps": fwd_steps, "turned_steps": K - fwd_steps,
              "frames": F + 1}

    # ---- the benchmark configuration as written: 100 forward steps from frame 0,
    # one CUDA graph (replayed once untimed from a snapshot, then timed)
    forward = None
    if use_graph and F >= 100:
        to_cycle_start()
        torch.cuda.synchronize()
        ctx.snapshot()
        g100 = capture_steps(ctx, dev_frames, F, eps, strat, clock[0], 100, torch)
        g100.replay()
        ctx.restore()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g100.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        clock[0] += 100
        ms_f = e0.elapsed_time(e1)
        r100, _ = ctx.sync(raise_on_status=False)
        assert int(r100["n_missed"].sum()) == 0, "safety rule missed a failure"
        ms_f, _ = aggregate(ms_f, N, dist, "cuda")
        forward = {"value": n_all * 100 / (ms_f / 1e3), "ms_per_step": ms_f / 100, "steps": 100,
                   "frames": "1..100, forward only, state from frame 0", "graph": "one graph of 100 steps"}
        del g100

    # ---- a longer replay of the same schedule (at least --sustained-ms of GPU time)
    sustained = None
    if use_graph and args.sustained_ms > 0:
        Ks = int(math.ceil(args.sustained_ms / max(1e-6, ms_max / K) / C)) * C
        ms_s, _ = graph_loop(ctx, dev_frames, F, eps, strat, Ks, use_graph, stream, torch, start=clock[0])
        clock[0] += Ks
        ms_s, _ = aggregate(ms_s, N, dist, "cuda")
        sustained = {"value": n_all * Ks / (ms_s / 1e3), "ms_per_step": ms_s / Ks, "steps": Ks,
                     "ms": ms_s}
    to_cycle_start()

    # ---- the same batch under each plain strategy, and the plain single-scene loops
    compare = {}
    if not args.no_compare:
        Kc = max(1, min(K, args.compare_steps))
        for name in ["incremental", "rebuild", "threshold", "auto"]:
            if name == "auto" and sel_meta is None:
                continue
            torch.cuda.synchronize()
            msc, _ = graph_loop(ctx, dev_frames, F, eps, cert.STRATEGY[name], Kc, use_graph, stream, torch)
            clock[0] += Kc
            to_cycle_start(cert.STRATEGY[name])
            compare[f"batched_{name}"] = N * Kc / (msc / 1e3)
        if args.workload == "batched":
            m2 = scenes.Motion("uniform_brownian", 16000, 3, 1e-3, seed=1 + rank, steps=200)
            f2 = torch.from_numpy(m2.frames(F)).cuda()
            for name in ["incremental", "rebuild"]:
                c2 = cert.Context(f2[0], cell_scale=ctx.cell_scale())
                for k in range(C):
                    c2.step(f2[cycle_index(k, F)], 1e-3, cert.STRATEGY[name])
                msc, _ = graph_loop(c2, f2, F, 1e-3, cert.STRATEGY[name], max(C, min(K, 4 * C)), use_graph,
                                    stream, torch)
                compare[f"plain_16000_d3_{name}"] = 16000 * max(C, min(K, 4 * C)) / (msc / 1e3)
                c2.close()
            del f2

    # ---- regret against the per-step measured best, from identical state
    regret = None
    if args.regret_steps > 0 and sel_meta is not None:
        names = ["incremental", "rebuild", "threshold", "auto"]
        tim = {n: [] for n in names}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(args.regret_steps):
            ctx.snapshot()
            for j, name in enumerate(names):
                if j:
                    ctx.restore()
                e0.record(stream)
                ctx.step(dev_frames[cycle_index(clock[0], F)], eps, cert.STRATEGY[name])
                e1.record(stream)
                e1.synchronize()
                tim[name].append(e0.elapsed_time(e1))
            clock[0] += 1
        t = {n: np.array(v) for n, v in tim.items()}
        best = np.minimum(t["incremental"], t["rebuild"])
        regret = {n: float((t[n] - best).sum() / best.sum()) for n in names}
        regret["steps"] = args.regret_steps
        regret["reference"] = "per step min(incremental, rebuild) on identical state, CUDA events"
        to_cycle_start()

    # ---- what each scene family's choice costs inside the batch: the family's scenes
    # forced to rebuild (the rest incremental) against every scene incremental, each
    # timed over the same cycle of frames from its start (per-scene policy, no selector)
    flips = None
    if args.flip_steps > 0 and args.workload == "batched" and args.family is None:
        fam_of = np.arange(S) % len(scenes.FAMILIES)
        if sel_meta is not None:
            ctx.load_selector(None, None)
        Kf = args.flip_steps
        variants = [("all_incremental", np.full(S, cert.CERT_INCREMENTAL))]
        variants += [(f"{scenes.FAMILIES[f]}_rebuild",
                      np.where(fam_of == f, cert.CERT_REBUILD, cert.CERT_INCREMENTAL)) for f in range(len(scenes.FAMILIES))]
        ms_flip = {}
        for name, pol in variants:
            ctx.set_scene_policy(pol)
            to_cycle_start(cert.CERT_AUTO)
            msf, _ = graph_loop(ctx, dev_frames, F, eps, cert.CERT_AUTO, Kf, use_graph, stream, torch)
            clock[0] += Kf
            ms_flip[name] = msf / Kf
        ctx.set_scene_policy(None)
        if sel_meta is not None:
            params, norm = selector.load()
            ctx.load_selector(params, norm)
        to_cycle_start()
        base_ms = ms_flip["all_incremental"]
        flips = {"steps": Kf, "ms_per_step": ms_flip,
                 "cost_vs_all_incremental": {n: ms / base_ms - 1.0 for n, ms in ms_flip.items() if n != "all_incremental"}}

    # ---- per-scene cost attribution inside the batch (the cost audit) and the regret
    # against the per-scene, per-step best strategy: each step is run incremental and
    # rebuild from identical state; a scene's time in a run is its share of the search
    # and refresh kernels' time (its share of their summed cycles) plus its share of the
    # other phases by point count
    scene_regret = None
    if args.scene_regret_steps > 0 and args.workload == "batched" and args.family is None:
        cc = cert.Context(dev_frames[0], offsets=offsets, cell_scale=ctx.cell_scale(), audit=("cost",))
        sizes = np.diff(offsets).astype(np.float64)
        for k in range(1, 9):
            cc.step(dev_frames[k], eps, cert.CERT_INCREMENTAL)
        iph = {n: cert.PHASE_NAMES.index(n) for n in ("search", "scatter_refresh")}
        att = {"incremental": [], "rebuild": [], "incremental_again": []}
        for t in range(args.scene_regret_steps):
            frame = dev_frames[min(9 + t, F)]
            cc.snapshot()
            # the state continues incremental; the repeated incremental run measures the noise floor
            for j, name in enumerate(("rebuild", "incremental_again", "incremental")):
                if j:
                    cc.restore()
                cc.profile_begin(1)
                cc.step(frame, eps, cert.STRATEGY[name.replace("_again", "")])
                ph = cc.profile_end()[0].astype(np.float64)
                r, _ = cc.sync(raise_on_status=False)
                cyc_s = r["search_cycles"].astype(np.float64)
                cyc_r = r["refresh_cycles"].astype(np.float64)
                other = ph.sum() - ph[iph["search"]] - ph[iph["scatter_refresh"]]
                att[name].append(other * sizes / sizes.sum() + ph[iph["search"]] * cyc_s / max(cyc_s.sum(), 1.0) +
                                 ph[iph["scatter_refresh"]] * cyc_r / max(cyc_r.sum(), 1.0))
        cc.close()
        Ti, Tr, Ti2 = np.array(att["incremental"]), np.array(att["rebuild"]), np.array(att["incremental_again"])
        best = np.minimum(Ti, Tr)
        fam_of = np.arange(S) % len(scenes.FAMILIES)
        scene_regret = {
            "steps": args.scene_regret_steps,
            "regret_vs_per_scene_best": {"incremental": float((Ti - best).sum() / best.sum()),
                                         "rebuild": float((Tr - best).sum() / best.sum())},
            "rebuild_best_frac": float((Tr < Ti).mean()),
            "rebuild_best_frac_by_family": {scenes.FAMILIES[f]: float((Tr < Ti)[:, fam_of == f].mean())
                                            for f in range(len(scenes.FAMILIES))},
            "gain_of_per_scene_best_over_incremental": float((Ti - best).sum() / Ti.sum()),
            # the same statistic between two incremental runs of the same steps: what noise in the
            # per-scene attribution alone makes the per-scene minimum look like
            "noise_floor_gain": float((Ti - np.minimum(Ti, Ti2)).sum() / Ti.sum()),
            "noise_floor_flip_frac": float((Ti2 < Ti).mean()),
            "attribution": "per scene: search and refresh kernel time split by the scene's summed cycles "
                           "(CERT_AUDIT_COST), the other phases by point count; both strategies from "
                           "identical state each step"}

    # ---- the frontier rules (detection only; certificates are exact under each):
    # Algorithm 1's c <= 4 eps_t, the per-point budget c <= 2 (delta_i + eps_t),
    # the cumulative clock 4 (S - S_i) >= c^rev_i
    rules = None
    if args.rule_steps > 0:
        rules = {}
        for rule in ("step", "point", "clock"):
            c3 = cert.Context(dev_frames[0], offsets=offsets, frontier_rule=rule, cell_scale=ctx.cell_scale(),
                              audit="rho")
            tot = np.zeros(6)
            for k in range(1, args.rule_steps + 1):
                c3.step(dev_frames[cycle_index(k, F)], eps, cert.CERT_INCREMENTAL)
                r, _ = c3.sync(raise_on_status=False)
                tot += [r["n_frontier"].sum(), r["n_failed"].sum(), r["n_false"].sum(), r["n_missed"].sum(),
                        r["n_rho"].sum(), r["n_rho_hit"].sum()]
            c3.close()
            rules[rule] = {"detected_frac": float(tot[0] / (N * args.rule_steps)),
                           "failed_frac": float(tot[1] / (N * args.rule_steps)),
                           "false_revalidation": float(tot[2] / max(1.0, tot[0])), "missed": int(tot[3])}
            assert tot[3] == 0, f"frontier rule {rule} missed a failure"
        # the local heuristic rho_i = delta_i / c_i > 1/2 (Sec. 3, Table 1): the
        # same on every rule's pass (it reads the same certificates and motion)
        rules["rho"] = {"flagged_frac": float(tot[4] / (N * args.rule_steps)),
                        "recall": float(tot[5] / max(1.0, tot[1])),
                        "false": float((tot[4] - tot[5]) / max(1.0, tot[4]))}
        rules["steps"] = args.rule_steps

    # ---- the matched pair (Sec. 4, Fig. 2): equal failure counts, different
    # entropy; the GPU repair timed on both (one scene of 16,000 points, and a
    # batch of 64 seeds of each transition)
    matched_pair = None
    if args.matched_steps > 0 and rank == 0:
        from paper_2606_18314_b300 import matched
        matched_pair = matched.run(cert, steps=args.matched_steps)

    # ---- k-nearest-neighbour certificates (one scene per context)
    knn = None
    if args.knn_steps > 0 and rank == 0:
        knn = knn_report(cert, torch, args.knn_steps, load_peaks()[0], stream)

    # ---- the single-scene configurations against the launch floor
    single = None
    if args.single_steps > 0 and rank == 0 and args.workload == "batched":
        single = single_scene_report(cert, torch, args.single_steps, stream)

    # ---- per-phase timing (CUDA events on the launching stream), same workload, eager
    P = max(1, args.prof_steps)
    ctx.profile_begin(P)
    counts = []
    for k in range(P):
        do_step()
        r, _ = ctx.sync(raise_on_status=False)
        tried = int(np.diff(offsets)[np.asarray(r["strategy"]) == cert.CERT_INCREMENTAL].sum())
        counts.append((int(r["n_frontier"].sum()), int(r["n_searched"].sum()), int(r["n_failed"].sum()), tried))
    prof = ctx.profile_end()
    mean_ms = prof.mean(axis=0)
    peaks, peak_kind = load_peaks()
    n_buckets = int(sum(1 << int(math.ceil(math.log2(max(int(n), 16)))) for n in np.diff(offsets))) * \
        max(1, args.bucket_factor)
    per_phase = {}
    for j, ph in enumerate(PHASES):
        byts = [phase_bytes(ph, N, dim, n_buckets, c[0], c[1], 0, c[3]) for c in counts]
        gbs = [b / (t * 1e-3) / 1e9 for b, t in zip(byts, prof[:, j]) if t > 0]
        per_phase[ph] = {"ms": float(mean_ms[j]), "share": float(mean_ms[j] / mean_ms.sum()),
                         "bytes": float(np.mean(byts)), "gbs": float(np.mean(gbs)) if gbs else 0.0}
    dom = max((p for p in PHASES if p != "clear"), key=lambda p: per_phase[p]["ms"])
    achieved = per_phase[dom]["bytes"] / (per_phase[dom]["ms"] * 1e-3) / 1e9
    cnt = np.array(counts, dtype=np.float64)
    step_counts = {"frontier_frac": float(cnt[:, 0].mean() / N), "searched_frac": float(cnt[:, 1].mean() / N),
                   "failed_frac": float(cnt[:, 2].mean() / N)}
    traffic, traffic_src = None, None
    fp_now = cert.cert_source_fingerprint("step_kernels")
    if dom == "search" and args.workload == "batched" and args.family is None and args.scenes == 512 and \
            strat in (cert.CERT_AUTO, cert.CERT_INCREMENTAL):
        scale = round(float(ctx.cell_scale()), 3)
        if SEARCH_TRAFFIC["fingerprint"] == fp_now and scale in SEARCH_TRAFFIC["bytes"]:
            traffic = SEARCH_TRAFFIC["bytes"][scale]
            traffic_src = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_search launch, same "
                           f"workload and cell scale {scale}, on step_kernels "
                           f"{SEARCH_TRAFFIC['fingerprint']} (commit {SEARCH_TRAFFIC['commit']})")
        else:
            traffic_src = (f"null: no ncu capture of the running step kernels (fingerprint {fp_now}) at cell scale "
                           f"{scale}; the captures ran on {SEARCH_TRAFFIC['fingerprint']} at "
                           f"{sorted(SEARCH_TRAFFIC['bytes'])}")
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": traffic_src,
                "kernel_fingerprint": fp_now,
                "peak_source": peak_kind, "phases": per_phase}

    # ---- end to end through the public API with host buffers (pinned): every step
    # copies its positions host-to-device and its per-scene results device-to-host;
    # cert_step_host_stream overlaps step k+1's copy with step k
    to_cycle_start()
    E = max(1, min(args.e2e_steps, K))
    host_frames = torch.from_numpy(frames).pin_memory()
    # pinned result buffer: a copy into pageable memory would block the host each step
    out_pinned = torch.zeros(max(E, 2) * S * cert.SCENE_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    out = out_pinned.numpy().view(cert.SCENE_DTYPE)
    row_bytes = N * dim * 4
    base_ptr = host_frames.data_ptr()
    # two untimed steps first: the call captures its one-step graphs (one per buffer parity)
    warm = [base_ptr + cycle_index(clock[0] + k, F) * row_bytes for k in range(2)]
    ctx.step_host_stream(warm, eps, strat, out, stream)
    clock[0] += 2
    ptrs = [base_ptr + cycle_index(clock[0] + k, F) * row_bytes for k in range(E)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.step_host_stream(ptrs, eps, strat, out, stream)
    el = time.perf_counter() - t0
    clock[0] += E
    assert int(out["n_missed"].sum()) == 0, "safety rule missed a failure"
    # the host link alone: one frame's pinned host-to-device copy, CUDA events
    stage = torch.empty((N, dim), dtype=torch.float32, device="cuda")
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        stage.copy_(host_frames[0], non_blocking=True)
    h0.record(stream)
    for _ in range(5):
        stage.copy_(host_frames[0], non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_ms = h0.elapsed_time(h1) / 5
    del stage
    e2e = {"value": N * E / el * (n_all / N), "unit": UNIT, "h2d_bytes_per_step": row_bytes,
           "d2h_bytes_per_step": int(S * cert.SCENE_DTYPE.itemsize), "steps": E,
           "api": "cert_step_host_stream (copies pipelined against the steps)",
           "h2d_ms_per_frame": h2d_ms, "h2d_gbs": row_bytes / (h2d_ms * 1e-3) / 1e9,
           "link_bound": N / (h2d_ms * 1e-3) * (n_all / N)}

    # ---- the all-pairs pass (exact brute force) at the paper's Table 2 sizes
    allpairs = None
    if args.allpairs_sizes:
        allpairs = {"peak_fp32_ops_per_s": None, "ops_per_pair": 8 if dim == 3 else 5, "rows": []}
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        peak = nsm * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6
        allpairs["peak_fp32_ops_per_s"] = peak
        allpairs["peak_source"] = f"{nsm} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz', 2032.0):.0f} MHz (one FP32 op per lane per cycle)"
        for nap in [int(x) for x in args.allpairs_sizes.split(",")]:
            pts = torch.rand((nap, 3), generator=torch.Generator().manual_seed(nap)).cuda()
            cert.cert_allpairs(pts)
            torch.cuda.synchronize()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps, t_ms = 3, 0.0
            for _ in range(reps):        # each call waits for its stream (it reads the status word)
                ea.record(stream)
                cert.cert_allpairs(pts)
                eb.record(stream)
                torch.cuda.synchronize()
                t_ms += ea.elapsed_time(eb) / reps
            pairs = nap * (nap - 1)
            ops = allpairs["ops_per_pair"] * pairs / (t_ms * 1e-3)
            allpairs["rows"].append({"n": nap, "ms": t_ms, "gpairs_per_s": pairs / (t_ms * 1e-3) / 1e9,
                                     "fp32_frac": ops / peak})
            del pts

    cb = None
    if rank == 0 and args.cpu_seconds > 0:
        cb, _, _ = cpu_baseline(frames, offsets, dim, budget_s=args.cpu_seconds)

    if rank == 0:
        cfg = dict(cfg)
        cfg.update({"strategy": args.strategy, "graph": use_graph, "frames": F + 1,
                    "cell_scale": ctx.cell_scale(), "autotune": tuned,
                    "motion": "pre-generated frames walked forward from frame 0 (warm-up, then the timed "
                              "steps); past the last frame the walk turns back; every step <= eps",
                    "warmup_requested": args.warmup,
                    "l2": "no flush: working set > 126 MB L2 (inputs larger than L2)",
                    "parallelism": f"scene-replicas x{world}"})
        if sel_meta is not None:
            cfg["selector"] = {k: sel_meta[k] for k in sel_meta if k.startswith(("rows", "val_"))}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": cfg, "roofline": roofline,
                "cpu_baseline": cb, "e2e": e2e, "gpu_launches": KERNELS_PER_STEP * K, "clocks": clocks,
                "step_counts": step_counts, "motion": motion, "forward_100": forward, "sustained": sustained,
                "compare": compare, "regret": regret, "family_flips": flips, "scene_regret": scene_regret,
                "frontier_rules": rules,
                "matched_pair": matched_pair, "knn": knn, "single_scene": single, "allpairs": allpairs,
                "status": cert.STATUS_NAMES[rc] if 0 <= rc < len(cert.STATUS_NAMES) else rc}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""CPU oracle for the certificate-maintenance step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA path: the brute-force
core is plain C (``cert_oracle.c``), loaded with ctypes; the composition of a
step and the selector network are plain numpy here and in ``mlp.py``.

What each function follows in the paper ("Repair Entropy in Dynamic Geometric
Nearest-Neighbour Structures"):

* ``top2`` / ``top2_queries`` -- certificate (nn, d1^2, d2^2), Def. 1; exact
  recomputation, Cor. A.2.  FP32, fixed operand order, lowest-index ties.
* ``eps`` -- maximum step, Algorithm 1 (first statement).
* ``frontier`` -- candidate frontier c_i <= 4 eps (+ rounding guard),
  Algorithm 1 (second statement), Lemma 1.
* ``frontier_point`` -- the per-point motion budget c_i <= 2 (delta_i + eps)
  (+ guard), the remark closing Sec. 5; ``disp`` gives delta_i.
* ``rho`` -- the local heuristic rho_i = delta_i / c_i > 1/2 of Sec. 3 and
  Table 1 (recall and false-flag audit; not a bound).
* ``gyration`` / ``compactness`` -- the failures' spatial spread, the
  frontier descriptors of the paper's transition log (Sec. 6 dataset columns,
  named there but not defined; read as the radius of gyration of the failed
  points and one minus its ratio to the scene's).
* ``ClockState`` -- the cumulative clock of the per-step cost subsection
  (Thm A.3): a certificate last revisited at clock S_i with clearance c^rev_i
  stays valid while 4 (S - S_i) < c^rev_i.
* ``grid_res`` / ``cells`` / ``entropy`` -- index cells, C and H(F_t), Def. 2.
* ``step`` -- one maintenance step end to end (Algorithm 1 with every
  certificate recomputed from scratch, which is the exact result Cor. A.2 says
  the repair reaches), plus the failure audit of Table 1.
* ``knn`` (module ``oracle.knn``) -- k-nearest-neighbour certificates, the
  k = 2 certificate one rank further out (Sec. 6 leaves kNN graphs open):
  brute-force top-(k+1) lists, the frontier d_{k+1} - d_k <= 4 eps_t + tau
  (Lemma 1's argument at rank k) and set-valued failures.
* ``trunc_median`` -- the lower median truncated to 3 mantissa bits, the
  definition the selector features use (no paper counterpart).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cert_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", *CFLAGS, "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.oracle_top2.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, i32p, f32p, f32p, ctypes.c_int]
        L.oracle_top2.restype = ctypes.c_int
        L.oracle_top2_queries.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, i32p, ctypes.c_int64,
                                          i32p, f32p, f32p, ctypes.c_int]
        L.oracle_top2_queries.restype = ctypes.c_int
        L.oracle_eps.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int]
        L.oracle_eps.restype = ctypes.c_float
        L.oracle_frontier.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_float, ctypes.c_int, i32p]
        L.oracle_frontier.restype = ctypes.c_int64
        L.oracle_disp.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int, f32p]
        L.oracle_disp.restype = None
        L.oracle_frontier_point.argtypes = [f32p, f32p, f32p, ctypes.c_int64, ctypes.c_float, i32p]
        L.oracle_frontier_point.restype = ctypes.c_int64
        L.oracle_knn.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i32p, f32p, ctypes.c_int]
        L.oracle_knn.restype = ctypes.c_int
        L.oracle_rho.argtypes = [f32p, f32p, f32p, ctypes.c_int64, u8p]
        L.oracle_rho.restype = ctypes.c_int64
        L.oracle_grid_res.argtypes = [ctypes.c_int64, ctypes.c_int]
        L.oracle_grid_res.restype = ctypes.c_int
        L.oracle_cells.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i32p]
        L.oracle_cells.restype = None
        L.oracle_entropy.argtypes = [i32p, u8p, ctypes.c_int64, ctypes.c_int64, i64p, i64p]
        L.oracle_entropy.restype = ctypes.c_double
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _pos(pos) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    if pos.ndim != 2 or pos.shape[1] not in (2, 3):
        raise ValueError("positions must be [n][2] or [n][3] float32")
    return pos


def max_threads() -> int:
    return int(lib().oracle_max_threads())


@dataclass
class Certificates:
    """(nn, d1^2, d2^2) of every point -- Def. 1 with squared distances."""
    nn: np.ndarray
    d1sq: np.ndarray
    d2sq: np.ndarray


def top2(pos, nthreads: int = 0) -> Certificates:
    """Brute-force exact certificates of all points (Def. 1, Cor. A.2)."""
    pos = _pos(pos)
    n, dim = pos.shape
    if n < 3:
        raise ValueError("a certificate needs at least 3 points")
    nn = np.empty(n, np.int32)
    d1 = np.empty(n, np.float32)
    d2 = np.empty(n, np.float32)
    rc = lib().oracle_top2(_p(pos, ctypes.c_float), n, dim, _p(nn, ctypes.c_int32),
                           _p(d1, ctypes.c_float), _p(d2, ctypes.c_float), int(nthreads))
    assert rc == 0
    return Certificates(nn, d1, d2)


def top2_queries(pos, queries, nthreads: int = 0) -> Certificates:
    """Certificates of a subset of query points against all points."""
    pos = _pos(pos)
    n, dim = pos.shape
    q = np.ascontiguousarray(queries, dtype=np.int32)
    nq = q.shape[0]
    nn = np.empty(nq, np.int32)
    d1 = np.empty(nq, np.float32)
    d2 = np.empty(nq, np.float32)
    rc = lib().oracle_top2_queries(_p(pos, ctypes.c_float), n, dim, _p(q, ctypes.c_int32), nq,
                                   _p(nn, ctypes.c_int32), _p(d1, ctypes.c_float),
                                   _p(d2, ctypes.c_float), int(nthreads))
    if rc != 0:
        raise ValueError("bad query list or point set")
    return Certificates(nn, d1, d2)


def eps(p_old, p_new) -> np.float32:
    """Measured maximum step eps_t (Algorithm 1, first statement), FP32."""
    a, b = _pos(p_old), _pos(p_new)
    assert a.shape == b.shape
    return np.float32(lib().oracle_eps(_p(a, ctypes.c_float), _p(b, ctypes.c_float),
                                       a.shape[0], a.shape[1]))


def frontier(d1sq, d2sq, eps_t, guard: bool = True) -> np.ndarray:
    """Ascending candidate frontier {i : c_i <= 4 eps_t + tau_i} (Algorithm 1)."""
    d1 = np.ascontiguousarray(d1sq, dtype=np.float32)
    d2 = np.ascontiguousarray(d2sq, dtype=np.float32)
    out = np.empty(d1.shape[0], np.int32)
    k = lib().oracle_frontier(_p(d1, ctypes.c_float), _p(d2, ctypes.c_float), d1.shape[0],
                              float(eps_t), 1 if guard else 0, _p(out, ctypes.c_int32))
    return out[:k].copy()


def disp(p_old, p_new) -> np.ndarray:
    """Per-point displacement delta_i = sqrtf(|p'_i - p_i|^2), FP32."""
    a, b = _pos(p_old), _pos(p_new)
    out = np.empty(a.shape[0], np.float32)
    lib().oracle_disp(_p(a, ctypes.c_float), _p(b, ctypes.c_float), a.shape[0], a.shape[1],
                      _p(out, ctypes.c_float))
    return out


def frontier_point(d1sq, d2sq, delta, eps_t) -> np.ndarray:
    """Ascending frontier {i : c_i <= 2 (delta_i + eps_t) + tau_i} (per-point budget)."""
    d1 = np.ascontiguousarray(d1sq, dtype=np.float32)
    d2 = np.ascontiguousarray(d2sq, dtype=np.float32)
    dl = np.ascontiguousarray(delta, dtype=np.float32)
    out = np.empty(d1.shape[0], np.int32)
    k = lib().oracle_frontier_point(_p(d1, ctypes.c_float), _p(d2, ctypes.c_float), _p(dl, ctypes.c_float),
                                    d1.shape[0], float(eps_t), _p(out, ctypes.c_int32))
    return out[:k].copy()


def rho(d1sq, d2sq, delta) -> np.ndarray:
    """Flags of the local heuristic rho_i = delta_i / c_i > 1/2 (bool [n])."""
    d1 = np.ascontiguousarray(d1sq, dtype=np.float32)
    d2 = np.ascontiguousarray(d2sq, dtype=np.float32)
    dl = np.ascontiguousarray(delta, dtype=np.float32)
    out = np.empty(d1.shape[0], np.uint8)
    lib().oracle_rho(_p(d1, ctypes.c_float), _p(d2, ctypes.c_float), _p(dl, ctypes.c_float), d1.shape[0],
                     _p(out, ctypes.c_uint8))
    return out.astype(bool)


class ClockState:
    """Cumulative-clock frontier (the per-step cost subsection, Thm A.3): S is
    the running sum of eps_t in FP64.  A certificate last revisited at clock
    S_i with clearance c^rev_i (and d1 + d2 = g^rev_i, FP32) stays valid while
    4 (S - S_i) < c^rev_i; the step's frontier is {i : c^rev_i <= 4 D + 2^-20
    (g^rev_i + D)}, D = S - S_i, all in FP64 in this order.  After the step the
    frontier's points are revisited from their post-step certificates."""

    def __init__(self, cert: Certificates):
        n = cert.nn.shape[0]
        self.S = 0.0
        self.S_i = np.zeros(n, np.float64)
        self._revisit(cert, np.ones(n, bool))

    def _revisit(self, cert: Certificates, who: np.ndarray):
        d1 = np.sqrt(cert.d1sq).astype(np.float32)
        d2 = np.sqrt(cert.d2sq).astype(np.float32)
        if not hasattr(self, "c_rev"):
            self.c_rev = np.zeros(d1.shape[0], np.float32)
            self.g_rev = np.zeros(d1.shape[0], np.float32)
        self.S_i[who] = self.S
        self.c_rev[who] = (d2 - d1)[who]
        self.g_rev[who] = (d1 + d2)[who]

    def frontier(self, eps_t) -> np.ndarray:
        S_t = self.S + float(np.float32(eps_t))
        D = S_t - self.S_i
        rhs = 4.0 * D + 2.0 ** -20 * (self.g_rev.astype(np.float64) + D)
        return np.nonzero(self.c_rev.astype(np.float64) <= rhs)[0].astype(np.int32)

    def advance(self, eps_t, frontier: np.ndarray, cert_new: Certificates):
        self.S = self.S + float(np.float32(eps_t))
        who = np.zeros(self.S_i.shape[0], bool)
        who[frontier] = True
        self._revisit(cert_new, who)


def grid_res(n: int, dim: int) -> int:
    """Entropy-grid cells per axis: smallest g with g^dim >= n (Sec. 2)."""
    return int(lib().oracle_grid_res(int(n), int(dim)))


def cells(pos, g: int) -> np.ndarray:
    """Index cell of every point under the g^dim entropy grid (Def. 2)."""
    pos = _pos(pos)
    out = np.empty(pos.shape[0], np.int32)
    lib().oracle_cells(_p(pos, ctypes.c_float), pos.shape[0], pos.shape[1], int(g),
                       _p(out, ctypes.c_int32))
    return out


def entropy(cell, member, ncells: int):
    """(H, m, C): normalised entropy of ``member`` over the occupied cells (Def. 2)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    mem = np.ascontiguousarray(member, dtype=np.uint8)
    m = ctypes.c_int64(0)
    C = ctypes.c_int64(0)
    H = lib().oracle_entropy(_p(cell, ctypes.c_int32), _p(mem, ctypes.c_uint8), cell.shape[0],
                             int(ncells), ctypes.byref(m), ctypes.byref(C))
    return float(H), int(m.value), int(C.value)


MEDIAN_SAMPLE = 1024


def trunc_median(values) -> np.float32:
    """Lower median (rank floor((k-1)/2)) of the first k = min(n, 1024)
    non-negative FP32 values, truncated to its sign, exponent and top 3
    mantissa bits (bit pattern & 0xFFF00000).  This is the exact definition
    behind the selector's median features (a fixed sample keeps it O(1) per
    scene); it has no counterpart in the paper."""
    v = np.sort(np.ascontiguousarray(values, dtype=np.float32)[:MEDIAN_SAMPLE])
    med = v[(v.shape[0] - 1) // 2]
    bits = np.array([med], np.float32).view(np.uint32) & np.uint32(0xFFF00000)
    return bits.view(np.float32)[0]


@dataclass
class StepResult:
    """Everything one maintenance step reports, per the paper's audit columns."""
    eps_t: np.float32
    frontier: np.ndarray          # ascending indices (detected set)
    cert: Certificates            # post-step certificates (exact)
    failed: np.ndarray            # bool: nn changed across the step (true failures)
    cell: np.ndarray              # post-step entropy-grid cell of every point
    g_h: int
    H: float                      # entropy of the true failures (Def. 2)
    H_cand: float                 # entropy of the detected frontier
    m: int                        # cells the failures meet
    m_cand: int                   # cells the detected frontier meets
    C: int                        # occupied cells
    n_failed: int
    n_missed: int                 # failed but not detected (Lemma 1: must be 0)
    n_false: int                  # detected but not failed
    med_c: np.float32             # trunc_median of the pre-step clearances
    rho: np.ndarray               # bool: flagged by the local heuristic rho_i > 1/2
    n_rho: int                    # flagged points
    n_rho_hit: int                # flagged points that failed
    gyration: float               # radius of gyration of the failed points (post-step)
    compactness: float            # 1 - gyration / (the scene's radius), in [0, 1]


def clearances(cert: Certificates) -> np.ndarray:
    """c_i = d2_i - d1_i in FP32 with d_k = sqrtf(d_k^2) (Def. 1)."""
    return (np.sqrt(cert.d2sq) - np.sqrt(cert.d1sq)).astype(np.float32)


def step(p_old, p_new, cert_old: Certificates, nthreads: int = 0, rule: str = "step",
         clock: "ClockState | None" = None) -> StepResult:
    """One maintenance step: eps_t, the detected frontier from the pre-step
    certificates, exact post-step certificates, true failures, cells, H and the
    audit (Algorithm 1; Def. 2; Cor. A.2; Table 1 columns).  rule: "step"
    (Algorithm 1), "point" (per-point budget) or "clock" (cumulative clock,
    state in ``clock``, advanced here)."""
    p_old, p_new = _pos(p_old), _pos(p_new)
    n, dim = p_new.shape
    e = eps(p_old, p_new)
    delta = disp(p_old, p_new)
    if rule == "step":
        F = frontier(cert_old.d1sq, cert_old.d2sq, e)
    elif rule == "point":
        F = frontier_point(cert_old.d1sq, cert_old.d2sq, delta, e)
    elif rule == "clock":
        F = clock.frontier(e)
    else:
        raise ValueError(f"unknown frontier rule {rule!r}")
    new = top2(p_new, nthreads)
    if rule == "clock":
        clock.advance(e, F, new)
    failed = new.nn != cert_old.nn
    g = grid_res(n, dim)
    cell = cells(p_new, g)
    inF = np.zeros(n, bool)
    inF[F] = True
    H, m, C = entropy(cell, failed, g ** dim)
    Hc, mc, _ = entropy(cell, inF, g ** dim)
    return StepResult(
        eps_t=e, frontier=F, cert=new, failed=failed, cell=cell, g_h=g, H=H, H_cand=Hc,
        m=m, m_cand=mc, C=C, n_failed=int(failed.sum()),
        n_missed=int((failed & ~inF).sum()), n_false=int((inF & ~failed).sum()),
        med_c=trunc_median(clearances(cert_old)), **_rho_audit(cert_old, delta, failed),
        **_geometry(p_new, failed))


def gyration(points) -> float:
    """Radius of gyration sqrt(mean |p - centroid|^2) of float32 points, in FP64
    (two passes: the centroid, then the mean squared distance to it); 0 for
    fewer than two points."""
    q = np.asarray(points, dtype=np.float64)
    if q.shape[0] < 2:
        return 0.0
    c = q.mean(axis=0)
    return float(np.sqrt(((q - c) ** 2).sum(axis=1).mean()))


def compactness(failed_points, all_points) -> float:
    """1 - gyration(failures) / gyration(scene), clamped to [0, 1]; 1 for a
    single failure (or a scene of one position), 0 without failures."""
    if len(failed_points) == 0:
        return 0.0
    g_all = gyration(all_points)
    if g_all <= 0.0:
        return 1.0
    return float(min(1.0, max(0.0, 1.0 - gyration(failed_points) / g_all)))


def _geometry(p_new: np.ndarray, failed: np.ndarray) -> dict:
    return {"gyration": gyration(p_new[failed]), "compactness": compactness(p_new[failed], p_new)}


def _rho_audit(cert_old: Certificates, delta: np.ndarray, failed: np.ndarray) -> dict:
    r = rho(cert_old.d1sq, cert_old.d2sq, delta)
    return {"rho": r, "n_rho": int(r.sum()), "n_rho_hit": int((r & failed).sum())}

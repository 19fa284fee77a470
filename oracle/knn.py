"""CPU oracle for k-nearest-neighbour certificates (test infrastructure only).

The paper's certificate is the k = 2 list (nn, runner-up) with clearance
d2 - d1 (Def. 1); Sec. 6 leaves richer certificates, k-nearest-neighbour
graphs among them, open.  One rank further out, the certificate of point i is
its top-(k+1) list under the key (D, j) and the clearance
c^(k)_i = d_{k+1,i} - d_{k,i}.  Every distance from i changes by at most
2 eps_t in a step (both ends move by at most eps_t), so, as in Lemma 1, the
set of the k nearest cannot change while c^(k)_i > 4 eps_t.

* ``knn`` -- brute-force top-m lists (C, ``oracle_knn``), FP32 fixed order,
  lowest index first among equal keys.
* ``frontier`` -- {i : c^(k)_i <= 4 eps_t + tau_i}, tau_i = 2^-20 ((d_k +
  d_{k+1}) + eps_t), the rounding guard of the k = 2 rule, in FP32.
* ``step`` -- one step: eps_t, the frontier from the pre-step lists, exact
  post-step lists, failures (the set of the k nearest changed) and the audit.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _p, _pos, eps, lib


def knn(pos, m: int, nthreads: int = 0):
    """The m nearest of every point: (idx [n][m] int32, d2 [n][m] float32)."""
    pos = _pos(pos)
    n, dim = pos.shape
    if not (1 <= m <= 32) or n <= m:
        raise ValueError("need 1 <= m <= 32 and n > m")
    idx = np.empty((n, m), np.int32)
    d2 = np.empty((n, m), np.float32)
    rc = lib().oracle_knn(_p(pos, ctypes.c_float), n, dim, int(m), _p(idx, ctypes.c_int32),
                          _p(d2, ctypes.c_float), int(nthreads))
    assert rc == 0
    return idx, d2


@dataclass
class KnnCert:
    """Top-(k+1) lists of every point, [n][k+1]."""
    k: int
    idx: np.ndarray
    d2: np.ndarray


def cert(pos, k: int, nthreads: int = 0) -> KnnCert:
    idx, d2 = knn(pos, k + 1, nthreads)
    return KnnCert(k, idx, d2)


def clearances(c: KnnCert) -> np.ndarray:
    """c^(k)_i = sqrtf(d2_{k+1}) - sqrtf(d2_k), FP32."""
    d = np.sqrt(c.d2)
    return (d[:, c.k] - d[:, c.k - 1]).astype(np.float32)


def frontier(c: KnnCert, eps_t) -> np.ndarray:
    """Flags of {i : c^(k)_i <= 4 eps_t + tau_i} (bool [n]), every operation in FP32."""
    e = np.float32(eps_t)
    d = np.sqrt(c.d2)
    dk, dk1 = d[:, c.k - 1], d[:, c.k]
    cc = dk1 - dk
    tau = np.float32(2.0 ** -20) * ((dk + dk1) + e)
    return cc <= np.float32(4.0) * e + tau


def set_changed(old: KnnCert, new: KnnCert) -> np.ndarray:
    """Flags of the points whose set of k nearest differs (bool [n])."""
    k = old.k
    return np.any(np.sort(old.idx[:, :k], axis=1) != np.sort(new.idx[:, :k], axis=1), axis=1)


@dataclass
class KnnStep:
    eps_t: np.float32
    frontier: np.ndarray      # bool [n], from the pre-step lists
    cert: KnnCert             # post-step lists (exact)
    failed: np.ndarray        # bool [n]: the set of the k nearest changed
    n_frontier: int
    n_failed: int
    n_missed: int             # failed but not in the frontier (must be 0)
    n_false: int              # in the frontier but not failed


def step(p_old, p_new, c_old: KnnCert, nthreads: int = 0) -> KnnStep:
    e = eps(p_old, p_new)
    F = frontier(c_old, e)
    new = cert(p_new, c_old.k, nthreads)
    failed = set_changed(c_old, new)
    return KnnStep(e, F, new, failed, int(F.sum()), int(failed.sum()), int((failed & ~F).sum()),
                   int((F & ~failed).sum()))


__all__ = ["knn", "KnnCert", "cert", "clearances", "frontier", "set_changed", "KnnStep", "step"]

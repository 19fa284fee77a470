"""Seeded synthetic motion families (input generation only).

This module is the one piece both the CUDA path's tests/benchmark and the CPU
oracle consume: it produces positions, nothing else.  It holds none of the
certificate arithmetic.  Random numbers come from numpy's Philox4x32-10
counter-based generator (Salmon et al., SC'11) keyed by a SeedSequence, so a
(config, family, eps, scene, seed) tuple regenerates the same frames anywhere.

Positions live in the unit domain [0,1]^d: each family moves an unfolded
trajectory u and reports reflect(u), the mirror image folded into [0,1];
reflection is 1-Lipschitz, so a step never moves a point by more than the
declared eps.  The trajectory is kept in float64 and each frame is
rounded to float32; displacements are drawn with radius at most 0.999*eps so the
rounding cannot push a float32 step beyond eps.

Families (the paper lists its motion families in Sec. 3 and Table 1; these are
the five the benchmark configurations name):

* ``uniform_brownian``   uniform start, each step uniform in the eps-ball.
* ``clustered_drift``    8 Gaussian clusters (sigma 0.03, centres uniform in
  [0.15,0.85]^d), each drifting at 0.5*eps in its own direction, plus a
  0.5*eps ball jitter per point.
* ``ring_rotation``      ring of radius 0.4 about the domain centre (axis z),
  Gaussian tube sigma 0.01 (clipped at 4.5 sigma); rigid rotation of the
  initial ring with arc step <= 0.5*eps plus an accumulated 0.5*eps jitter
  (``jitter=False`` gives the exact rigid motion).
* ``adversarial_crossing`` two slabs of x-width 0.1 (40% of points each) moving
  in +x / -x at eps per step from an initial gap eps*T/4, over a static
  uniform background (20%).
* ``hotspot``            uniform points; those inside one 0.1-wide cube at a
  seeded centre take eps-ball steps, the rest are static.
* ``uniform_clusters``   half uniform, half in 16 Gaussian clusters
  (sigma 0.01); every point takes eps-ball steps (the large-N scale scene).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FAMILIES = ("uniform_brownian", "clustered_drift", "ring_rotation",
            "adversarial_crossing", "hotspot")
ALL_FAMILIES = FAMILIES + ("uniform_clusters",)
_FAMILY_ID = {f: k for k, f in enumerate(ALL_FAMILIES)}
STEP_FRACTION = 0.999


def rng_for(*key: int) -> np.random.Generator:
    """Philox4x32-10 stream keyed by a tuple of non-negative integers."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(k) for k in key])))


def reflect(x: np.ndarray) -> np.ndarray:
    """Fold coordinates into [0,1] by mirror reflection (1-Lipschitz)."""
    y = np.mod(np.abs(x), 2.0)
    return np.where(y > 1.0, 2.0 - y, y)


def ball(rng: np.random.Generator, n: int, dim: int, radius: float) -> np.ndarray:
    """n vectors uniform in the dim-ball of the given radius: a normalised
    Gaussian direction times radius * U^(1/dim)."""
    g = rng.standard_normal((n, dim))
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    nrm = np.where(nrm > 0.0, nrm, 1.0)
    u = rng.random((n, 1))
    return g / nrm * (radius * u ** (1.0 / dim))


def unit_vectors(rng: np.random.Generator, k: int, dim: int) -> np.ndarray:
    g = rng.standard_normal((k, dim))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


@dataclass
class Motion:
    """One scene: ``frame()`` returns the current float32 positions,
    ``advance()`` moves every point by at most ``eps`` and returns the next."""
    family: str
    n: int
    dim: int
    eps: float
    seed: int = 0
    steps: int = 200          # horizon, used by the crossing family's gap
    jitter: bool = True
    t: int = 0
    _x: np.ndarray = field(default=None, repr=False)
    _rng: np.random.Generator = field(default=None, repr=False)
    _aux: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        if self.family not in _FAMILY_ID:
            raise ValueError(f"unknown motion family {self.family!r}")
        if self.dim not in (2, 3) or self.n < 3:
            raise ValueError("need dim in {2,3} and n >= 3")
        self._rng = rng_for(_FAMILY_ID[self.family], self.n, self.dim, self.seed,
                            int(round(self.eps * 1e9)))
        getattr(self, "_init_" + self.family)()

    # -- initial layouts ---------------------------------------------------
    def _init_uniform_brownian(self):
        self._x = self._rng.random((self.n, self.dim))

    def _init_clustered_drift(self):
        r, n, d = self._rng, self.n, self.dim
        centres = 0.15 + 0.7 * r.random((8, d))
        lab = r.integers(0, 8, n)
        self._x = reflect(centres[lab] + 0.03 * r.standard_normal((n, d)))
        vel = 0.5 * STEP_FRACTION * self.eps * unit_vectors(r, 8, d)
        self._aux["v"] = vel[lab]

    def _init_ring_rotation(self):
        r, n, d = self._rng, self.n, self.dim
        th = 2.0 * math.pi * r.random(n)
        dr = np.clip(0.01 * r.standard_normal(n), -0.045, 0.045)
        base = np.zeros((n, d))
        base[:, 0] = (0.4 + dr) * np.cos(th)
        base[:, 1] = (0.4 + dr) * np.sin(th)
        if d == 3:
            base[:, 2] = np.clip(0.01 * r.standard_normal(n), -0.045, 0.045)
        self._aux["base"] = base                       # offsets from the centre
        self._aux["J"] = np.zeros((n, d))
        # arc length per step at the largest radius (0.445) stays <= 0.5*eps
        self._aux["omega"] = 0.5 * STEP_FRACTION * self.eps / 0.445
        self._x = reflect(0.5 + base)

    def _init_adversarial_crossing(self):
        r, n, d = self._rng, self.n, self.dim
        na = int(0.4 * n)
        nb = int(0.4 * n)
        g = self.eps * self.steps / 4.0
        x = r.random((n, d))
        x[:na, 0] = 0.5 - g / 2.0 - 0.1 * r.random(na)
        x[na:na + nb, 0] = 0.5 + g / 2.0 + 0.1 * r.random(nb)
        v = np.zeros((n, d))
        v[:na, 0] = STEP_FRACTION * self.eps
        v[na:na + nb, 0] = -STEP_FRACTION * self.eps
        perm = r.permutation(n)                 # interleave slab membership over indices
        self._x = reflect(x[perm])
        self._aux["v"] = v[perm]

    def _init_hotspot(self):
        r, n, d = self._rng, self.n, self.dim
        self._x = r.random((n, d))
        c = 0.05 + 0.9 * r.random(d)
        self._aux["hot"] = np.all(np.abs(self._x - c) <= 0.05, axis=1)

    def _init_uniform_clusters(self):
        r, n, d = self._rng, self.n, self.dim
        nu = n // 2
        centres = 0.1 + 0.8 * r.random((16, d))
        lab = r.integers(0, 16, n - nu)
        x = np.empty((n, d))
        x[:nu] = r.random((nu, d))
        x[nu:] = centres[lab] + 0.01 * r.standard_normal((n - nu, d))
        self._x = reflect(x[r.permutation(n)])

    # -- steps ---------------------------------------------------------------
    def _ball(self, frac: float, n: int | None = None) -> np.ndarray:
        return ball(self._rng, self.n if n is None else n, self.dim, frac * STEP_FRACTION * self.eps)

    def _step_uniform_brownian(self):
        self._x = self._x + self._ball(1.0)

    _step_uniform_clusters = _step_uniform_brownian

    def _step_clustered_drift(self):
        self._x = self._x + self._aux["v"] + self._ball(0.5)

    def _step_ring_rotation(self):
        a = self._aux
        th = a["omega"] * self.t
        c, s = math.cos(th), math.sin(th)
        b = a["base"]
        y = b.copy()
        y[:, 0] = c * b[:, 0] - s * b[:, 1]
        y[:, 1] = s * b[:, 0] + c * b[:, 1]
        if self.jitter:
            a["J"] = a["J"] + self._ball(0.5)
        self._x = 0.5 + y + a["J"]

    def _step_adversarial_crossing(self):
        self._x = self._x + self._aux["v"]

    def _step_hotspot(self):
        hot = self._aux["hot"]
        k = int(hot.sum())
        if k:
            self._x[hot] = self._x[hot] + self._ball(1.0, k)

    def frame(self) -> np.ndarray:
        return reflect(self._x).astype(np.float32)

    def advance(self) -> np.ndarray:
        self.t += 1
        getattr(self, "_step_" + self.family)()
        return self.frame()

    def frames(self, count: int) -> np.ndarray:
        """[count+1][n][dim]: the current frame followed by ``count`` steps."""
        out = np.empty((count + 1, self.n, self.dim), np.float32)
        out[0] = self.frame()
        for k in range(count):
            out[k + 1] = self.advance()
        return out


# --- benchmark workloads ------------------------------------------------------

def batch_sizes(n_scenes: int = 512, lo: int = 500, hi: int = 16000, seed: int = 4) -> np.ndarray:
    """Scene sizes log-uniform in [lo, hi]: round(exp(U(ln lo, ln hi)))."""
    r = rng_for(4, 0, seed)
    return np.rint(np.exp(r.uniform(math.log(lo), math.log(hi), n_scenes))).astype(np.int64)


@dataclass
class BatchMotion:
    """Many independent scenes advanced together; frames are the scenes'
    positions concatenated in scene order (CSR ``offsets``)."""
    scenes: list

    @classmethod
    def mixed(cls, n_scenes=512, dim=3, eps=1e-3, seed=4, steps=100, lo=500, hi=16000):
        sizes = batch_sizes(n_scenes, lo, hi, seed)
        sc = [Motion(FAMILIES[s % len(FAMILIES)], int(sizes[s]), dim, eps,
                     seed=seed * 100003 + s, steps=steps) for s in range(n_scenes)]
        return cls(sc)

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([m.n for m in self.scenes])]).astype(np.int64)

    @property
    def dim(self) -> int:
        return self.scenes[0].dim

    def frame(self) -> np.ndarray:
        return np.concatenate([m.frame() for m in self.scenes])

    def advance(self) -> np.ndarray:
        return np.concatenate([m.advance() for m in self.scenes])

    def frames(self, count: int) -> np.ndarray:
        tot = int(self.offsets[-1])
        out = np.empty((count + 1, tot, self.dim), np.float32)
        out[0] = self.frame()
        for k in range(count):
            out[k + 1] = self.advance()
        return out

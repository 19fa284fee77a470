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

The paper's other motion families (Sec. 3, Table 1) are named there but not
parameterised; these are the build's own readings of them:

* ``grid_jitter``        the first n sites, in seeded random order, of the
  k^d lattice with spacing 1/k (k = ceil(n^(1/d))), cell-centred; eps-ball
  steps from there (jittered-lattice diffusion; the exact lattice of the
  first frame is full of equal distances).
* ``filament``           points along the closed Lissajous curve
  (0.5+0.35 sin 2 pi u, 0.5+0.35 sin 4 pi u[, 0.5+0.2 cos 2 pi u]) in a
  Gaussian tube (sigma 0.01, clipped at 4.5 sigma), flowing along it at
  <= 0.5 eps per step plus an accumulated 0.5 eps jitter.
* ``vortex``             points uniform in the disk (cylinder in 3-D,
  z in [0.1, 0.9]) of radius 0.4 about the centre, rotating differentially
  with speed 0.5 eps * 4 (r/R)(1 - r/R) (zero at the axis and at the rim)
  plus an accumulated 0.5 eps jitter.
* ``split_merge``        one Gaussian cluster (sigma 0.05) whose two halves
  move apart along +-x at 0.5 eps per step for half the horizon and back
  for the other half, plus an accumulated 0.5 eps jitter.
* ``shear_band``         uniform points; those in the band |y - 0.5| < 0.1
  move along +x with speed eps * (1 - |y - 0.5| / 0.1), the rest are static.
* ``spiral``             points at equal arc-length spacing on an
  Archimedean spiral (r from 0.05 to 0.4 over 6 turns; in 3-D rising
  linearly from z = 0.1 to 0.9), a near-lattice arrangement whose neighbours
  along the arm are nearly equidistant, rotating rigidly by <= 0.5 eps per
  step plus an accumulated 0.1 eps jitter.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FAMILIES = ("uniform_brownian", "clustered_drift", "ring_rotation",
            "adversarial_crossing", "hotspot")
PAPER_FAMILIES = ("grid_jitter", "filament", "vortex", "split_merge", "shear_band", "spiral")
ALL_FAMILIES = FAMILIES + ("uniform_clusters",) + PAPER_FAMILIES
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

    def _init_grid_jitter(self):
        r, n, d = self._rng, self.n, self.dim
        k = int(math.ceil(n ** (1.0 / d) - 1e-9))
        while k ** d < n:
            k += 1
        idx = r.permutation(k ** d)[:n]
        sites = np.stack(np.unravel_index(idx, (k,) * d), axis=1).astype(np.float64)
        self._x = (sites + 0.5) / k

    _FIL_LMAX = 2.0 * math.pi * math.sqrt(0.35 ** 2 + 0.7 ** 2 + 0.2 ** 2)   # bound on |c'(u)|

    def _filament_curve(self, u):
        c = np.empty((u.shape[0], self.dim))
        c[:, 0] = 0.5 + 0.35 * np.sin(2.0 * math.pi * u)
        c[:, 1] = 0.5 + 0.35 * np.sin(4.0 * math.pi * u)
        if self.dim == 3:
            c[:, 2] = 0.5 + 0.2 * np.cos(2.0 * math.pi * u)
        return c

    def _init_filament(self):
        r, n, d = self._rng, self.n, self.dim
        a = self._aux
        a["u"] = r.random(n)
        a["off"] = np.clip(0.01 * r.standard_normal((n, d)), -0.045, 0.045)
        a["du"] = 0.5 * STEP_FRACTION * self.eps / self._FIL_LMAX
        a["J"] = np.zeros((n, d))
        self._x = self._filament_curve(a["u"]) + a["off"]

    def _init_vortex(self):
        r, n, d = self._rng, self.n, self.dim
        a = self._aux
        rad = 0.4 * np.sqrt(r.random(n))
        a["r"] = rad
        a["th"] = 2.0 * math.pi * r.random(n)
        a["z"] = 0.1 + 0.8 * r.random(n) if d == 3 else None
        speed = 0.5 * STEP_FRACTION * self.eps * 4.0 * (rad / 0.4) * (1.0 - rad / 0.4)
        a["dth"] = np.where(rad > 0.0, speed / np.maximum(rad, 1e-30), 0.0)   # arc <= speed
        a["J"] = np.zeros((n, d))
        self._x = self._vortex_pos()

    def _vortex_pos(self):
        a = self._aux
        th = a["th"] + a["dth"] * self.t
        x = np.empty((self.n, self.dim))
        x[:, 0] = 0.5 + a["r"] * np.cos(th)
        x[:, 1] = 0.5 + a["r"] * np.sin(th)
        if self.dim == 3:
            x[:, 2] = a["z"]
        return x + a["J"]

    def _init_split_merge(self):
        r, n, d = self._rng, self.n, self.dim
        a = self._aux
        a["base"] = 0.5 + np.clip(0.05 * r.standard_normal((n, d)), -0.3, 0.3)
        a["sgn"] = np.where(r.random(n) < 0.5, -1.0, 1.0)
        a["J"] = np.zeros((n, d))
        self._x = self._split_pos()

    def _split_pos(self):
        a = self._aux
        half = max(1, self.steps // 2)
        t = self.t % (2 * half)
        tri = t if t <= half else 2 * half - t                    # steps of separation
        x = a["base"].copy()
        x[:, 0] += a["sgn"] * 0.5 * STEP_FRACTION * self.eps * tri
        return x + a["J"]

    def _init_shear_band(self):
        r, n, d = self._rng, self.n, self.dim
        self._x = r.random((n, d))
        w = np.clip(1.0 - np.abs(self._x[:, 1] - 0.5) / 0.1, 0.0, 1.0)
        self._aux["v"] = STEP_FRACTION * self.eps * w

    def _init_spiral(self):
        r, n, d = self._rng, self.n, self.dim
        a = self._aux
        turns, r0, r1 = 6.0, 0.05, 0.4
        phi = np.linspace(0.0, 2.0 * math.pi * turns, 200001)
        rad = r0 + (r1 - r0) * phi / phi[-1]
        pts = np.stack([rad * np.cos(phi), rad * np.sin(phi)], 1)
        if d == 3:
            pts = np.concatenate([pts, (0.1 + 0.8 * phi / phi[-1])[:, None]], 1)
        seg = np.linalg.norm(np.diff(pts, axis=0), axis=1)
        arc = np.concatenate([[0.0], np.cumsum(seg)])
        s_i = (np.arange(n) + 0.5) / n * arc[-1]                   # equal arc-length spacing
        ph = np.interp(s_i, arc, phi)
        rr = r0 + (r1 - r0) * ph / phi[-1]
        base = np.zeros((n, d))
        base[:, 0] = rr * np.cos(ph)
        base[:, 1] = rr * np.sin(ph)
        if d == 3:
            base[:, 2] = 0.1 + 0.8 * ph / phi[-1] - 0.5
        perm = r.permutation(n)
        a["base"] = base[perm]
        a["omega"] = 0.5 * STEP_FRACTION * self.eps / r1     # arc per step <= 0.5 eps
        a["J"] = np.zeros((n, d))
        self._x = 0.5 + a["base"]

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

    _step_grid_jitter = _step_uniform_brownian

    def _step_filament(self):
        a = self._aux
        a["u"] = a["u"] + a["du"]
        a["J"] = a["J"] + self._ball(0.5)
        self._x = self._filament_curve(a["u"]) + a["off"] + a["J"]

    def _step_vortex(self):
        self._aux["J"] = self._aux["J"] + self._ball(0.5)
        self._x = self._vortex_pos()

    def _step_split_merge(self):
        self._aux["J"] = self._aux["J"] + self._ball(0.5)
        self._x = self._split_pos()

    def _step_shear_band(self):
        self._x = self._x.copy()
        self._x[:, 0] = self._x[:, 0] + self._aux["v"]

    def _step_spiral(self):
        a = self._aux
        th = a["omega"] * self.t
        c, s = math.cos(th), math.sin(th)
        b = a["base"]
        y = b.copy()
        y[:, 0] = c * b[:, 0] - s * b[:, 1]
        y[:, 1] = s * b[:, 0] + c * b[:, 1]
        if self.jitter:
            a["J"] = a["J"] + self._ball(0.1)
        self._x = 0.5 + y + a["J"]

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

    def frames_parallel(self, count: int, workers: int) -> np.ndarray:
        """The array ``frames(count)`` returns for scenes still at their
        first frame, generated scene by scene in a pool of spawned processes.
        Each scene's stream depends only on its own seed, so the result is
        the same; the scenes themselves are left untouched."""
        if any(m.t != 0 for m in self.scenes):
            raise ValueError("frames_parallel needs every scene at its first frame")
        import concurrent.futures
        import multiprocessing
        tot, off = int(self.offsets[-1]), self.offsets
        out = np.empty((count + 1, tot, self.dim), np.float32)
        jobs = [(m.family, m.n, m.dim, m.eps, m.seed, m.steps, m.jitter, count) for m in self.scenes]
        with concurrent.futures.ProcessPoolExecutor(max_workers=max(1, workers),
                                                    mp_context=multiprocessing.get_context("spawn")) as ex:
            for s, fr in enumerate(ex.map(_scene_frames, jobs, chunksize=max(1, len(jobs) // (4 * max(1, workers))))):
                out[:, off[s]:off[s + 1]] = fr
        return out


def _scene_frames(job):
    family, n, dim, eps, seed, steps, jitter, count = job
    return Motion(family, n, dim, eps, seed=seed, steps=steps, jitter=jitter).frames(count)

"""Pins of the failure-geometry descriptors (CPU): the radius of gyration of
the failed points and compactness = 1 - gyration / (the scene's radius).

* closed forms: two points at distance d give d/2; the four corners of a
  square of side s give s/sqrt(2); the eight corners of a cube of side s
  give s sqrt(3)/2; one point gives 0;
* invariances: translation (dyadic shifts, exact), permutation, scaling;
* compactness: 1 for one failure, 0 when every point fails, between the two
  for a cluster, and larger for a tighter cluster;
* the step's fields are these functions of its failures."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes


def test_gyration_closed_forms():
    assert oracle.gyration(np.array([[0.25, 0.5]], np.float32)) == 0.0
    assert oracle.gyration(np.array([[0.25, 0.5], [0.75, 0.5]], np.float32)) == pytest.approx(0.25, abs=1e-15)
    sq = np.array([[0, 0], [0.5, 0], [0, 0.5], [0.5, 0.5]], np.float32)
    assert oracle.gyration(sq) == pytest.approx(0.5 / math.sqrt(2), rel=1e-14)
    cube = np.array([[x, y, z] for x in (0, 0.25) for y in (0, 0.25) for z in (0, 0.25)], np.float32)
    assert oracle.gyration(cube) == pytest.approx(0.25 * math.sqrt(3) / 2, rel=1e-14)


def test_gyration_invariances():
    rng = np.random.default_rng(5)
    p = (rng.integers(0, 64, (40, 3)) / 128).astype(np.float32)
    g = oracle.gyration(p)
    assert oracle.gyration(p + np.float32(0.25)) == pytest.approx(g, rel=1e-14)
    assert oracle.gyration(p[rng.permutation(40)]) == pytest.approx(g, rel=1e-14)
    assert oracle.gyration(p * np.float32(0.5)) == pytest.approx(g / 2, rel=1e-14)


def test_compactness_bounds_and_order():
    rng = np.random.default_rng(6)
    p = rng.random((500, 3)).astype(np.float32)
    assert oracle.compactness(p[:0], p) == 0.0
    assert oracle.compactness(p[:1], p) == 1.0
    assert oracle.compactness(p, p) == 0.0
    centre = np.float32(0.5)
    tight = (centre + 0.01 * rng.standard_normal((50, 3))).astype(np.float32)
    loose = (centre + 0.05 * rng.standard_normal((50, 3))).astype(np.float32)
    ct, cl = oracle.compactness(tight, p), oracle.compactness(loose, p)
    assert 0.0 < cl < ct < 1.0


def test_step_fields_are_the_failures_geometry():
    m = scenes.Motion("adversarial_crossing", 800, 3, 3e-3, seed=2, steps=40)
    p = m.frame()
    cert = oracle.top2(p)
    for _ in range(4):
        q = m.advance()
        r = oracle.step(p, q, cert)
        assert r.gyration == oracle.gyration(q[r.failed])
        assert r.compactness == oracle.compactness(q[r.failed], q)
        if r.n_failed >= 2:
            assert 0.0 < r.gyration and 0.0 <= r.compactness <= 1.0
        p, cert = q, r.cert

"""Input generators: seeded, inside [0,1]^d, and every step within eps (CPU)."""
import numpy as np
import pytest

from paper_2606_18314_b300 import scenes


@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("eps", [1e-4, 5e-3])
def test_steps_bounded_and_in_domain(family, dim, eps):
    m = scenes.Motion(family, 500, dim, eps, seed=3, steps=50)
    fr = m.frames(30)
    assert fr.dtype == np.float32 and fr.shape == (31, 500, dim)
    assert np.all(fr >= 0.0) and np.all(fr <= 1.0)
    step = np.sqrt(((fr[1:].astype(np.float64) - fr[:-1]) ** 2).sum(-1))
    assert step.max() <= eps
    if family != "hotspot":
        assert step.max() > 0.3 * eps


def test_seeded_and_reproducible():
    a = scenes.Motion("clustered_drift", 300, 3, 1e-3, seed=9).frames(5)
    b = scenes.Motion("clustered_drift", 300, 3, 1e-3, seed=9).frames(5)
    c = scenes.Motion("clustered_drift", 300, 3, 1e-3, seed=10).frames(5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_batch_sizes_and_offsets():
    s = scenes.batch_sizes(512)
    assert s.min() >= 500 and s.max() <= 16000 and len(s) == 512
    bm = scenes.BatchMotion.mixed(n_scenes=6, lo=20, hi=60)
    off = bm.offsets
    assert off[0] == 0 and off[-1] == sum(m.n for m in bm.scenes)
    fr = bm.frames(2)
    assert fr.shape == (3, off[-1], 3)
    assert [m.family for m in bm.scenes] == list(scenes.FAMILIES) + [scenes.FAMILIES[0]]


def test_rigid_ring_preserves_shape():
    m = scenes.Motion("ring_rotation", 200, 3, 1e-3, seed=1, jitter=False)
    f0, f1 = m.frame().astype(np.float64), m.advance().astype(np.float64)
    r0 = np.linalg.norm(f0[:, :2] - 0.5, axis=1)
    r1 = np.linalg.norm(f1[:, :2] - 0.5, axis=1)
    assert np.allclose(r0, r1, atol=1e-6)

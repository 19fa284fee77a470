"""Host logic of the matched-pair experiment (Sec. 4, Fig. 2): the pair
selection and the frame plumbing, without a GPU."""
import numpy as np

from paper_2606_18314_b300 import matched, scenes


def _row(f, H, t=0, fam="a"):
    return {"family": fam, "t": t, "n_failed": f, "H": H}


def test_select_matches_counts_within_the_tolerance():
    a = [_row(100, 0.5, 0), _row(200, 0.6, 1)]
    b = [_row(113, 0.9, 0, "b"),     # |100-113| = 13 > 0.12 * 113 = 13.56? no: 13 <= 13.56, matches
         _row(230, 0.95, 1, "b")]    # |200-230| = 30 > 0.12 * 230 = 27.6: no match
    pa, pb = matched.select(a, b)
    assert (pa["n_failed"], pb["n_failed"]) == (100, 113)
    # just outside the tolerance: nothing matches
    assert matched.select([_row(100, 0.5)], [_row(114, 0.9)]) is None


def test_select_needs_the_diffuse_member_to_have_the_higher_entropy():
    assert matched.select([_row(100, 0.8)], [_row(100, 0.8)]) is None
    assert matched.select([_row(100, 0.8)], [_row(100, 0.7)]) is None
    assert matched.select([_row(100, 0.7)], [_row(100, 0.8)]) is not None


def test_select_takes_the_largest_entropy_gap_then_the_closest_counts():
    a = [_row(100, 0.5, 0), _row(100, 0.4, 1), _row(104, 0.4, 2)]
    b = [_row(105, 0.9, 0, "b"), _row(100, 0.7, 1, "b")]
    pa, pb = matched.select(a, b)
    # gap 0.5 from a[1] and a[2] with b[0]; b[0] is 105: a[2] (104) is closer
    assert (pa["t"], pb["t"]) == (2, 0)


def test_select_skips_tiny_failure_counts():
    assert matched.select([_row(10, 0.1)], [_row(10, 0.9)]) is None
    assert matched.select([_row(10, 0.1)], [_row(10, 0.9)], min_failed=1) is not None


def test_frames_at_is_the_motion_sequence():
    fr = scenes.Motion(matched.LOCALIZED, 300, 3, 1e-3, seed=5, steps=64).frames(6)
    two = matched.frames_at(matched.LOCALIZED, 300, 3, 1e-3, 5, 4, 64)
    assert two.dtype == np.float32 and two.shape == (2, 300, 3)
    assert np.array_equal(two[0], fr[4]) and np.array_equal(two[1], fr[5])


def test_batch_frames_concatenate_one_scene_per_seed():
    fr, off = matched.batch_frames(matched.DIFFUSE, 200, 3, 2.5e-4, 3, [1, 2, 3], 64)
    assert fr.shape == (2, 600, 3) and list(off) == [0, 200, 400, 600]
    for k, s in enumerate([1, 2, 3]):
        two = matched.frames_at(matched.DIFFUSE, 200, 3, 2.5e-4, s, 3, 64)
        assert np.array_equal(fr[:, off[k]:off[k + 1]], two)

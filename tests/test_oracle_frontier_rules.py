"""Pins of the two frontier rules beyond Algorithm 1 (CPU).

* per-point motion budget, c_i <= 2 (delta_i + eps_t) + tau_i (the remark
  closing Sec. 5): never misses a failure, is a subset of Algorithm 1's
  frontier, and leaves out a static point with 2 eps < c <= 4 eps;
* cumulative clock (the per-step cost subsection, Thm A.3): never misses a
  failure over many steps, and a static certificate expires exactly when
  4 (S - S_i) reaches c^rev_i, then again after its revisit.
"""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes


@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
def test_point_and_clock_rules_never_miss(family, dim):
    m = scenes.Motion(family, 500, dim, eps=3e-3, seed=2, steps=40)
    p = m.frame()
    cert = oracle.top2(p)
    clock = oracle.ClockState(cert)
    for t in range(10):
        q = m.advance()
        rs = oracle.step(p, q, cert)
        rp = oracle.step(p, q, cert, rule="point")
        rc = oracle.step(p, q, cert, rule="clock", clock=clock)
        assert rs.n_missed == 0 and rp.n_missed == 0 and rc.n_missed == 0
        assert np.all(np.isin(rp.frontier, rs.frontier))          # never looser than Algorithm 1
        assert np.array_equal(rp.cert.nn, rs.cert.nn) and np.array_equal(rc.cert.nn, rs.cert.nn)
        p, cert = q, rs.cert


def _static_pair_scene(cg):
    """p0 with nn p1 at 0.125 and runner-up p2 at 0.125 + cg (all static);
    a far point moves by exactly eps = 2^-10 each step.  Dyadic coordinates:
    every distance, square root and clearance is exact in FP32."""
    eps = 2.0 ** -10
    base = np.array([[0.25, 0.5], [0.375, 0.5], [0.25, 0.5 - 0.125 - cg], [0.9, 0.1], [0.95, 0.1]], np.float64)
    frames = []
    for t in range(8):
        f = base.copy()
        f[3, 0] -= t * eps
        frames.append(f.astype(np.float32))
    return frames, eps


def test_point_rule_leaves_out_a_static_point_with_clearance_three_eps():
    frames, eps = _static_pair_scene(3 * 2.0 ** -10)
    cert = oracle.top2(frames[0])
    assert cert.nn[0] == 1 and oracle.clearances(cert)[0] == np.float32(3 * eps)
    rs = oracle.step(frames[0], frames[1], cert)
    rp = oracle.step(frames[0], frames[1], cert, rule="point")
    assert rs.eps_t == np.float32(eps)
    assert 0 in rs.frontier                    # 3 eps <= 4 eps + tau
    assert 0 not in rp.frontier                # 3 eps > 2 (0 + eps) + tau


def test_clock_rule_expires_a_static_certificate_on_schedule():
    frames, eps = _static_pair_scene(10 * 2.0 ** -10)
    cert = oracle.top2(frames[0])
    assert oracle.clearances(cert)[0] == np.float32(10 * eps)
    clock = oracle.ClockState(cert)
    flagged = []
    for t in range(1, 8):
        r = oracle.step(frames[t - 1], frames[t], cert, rule="clock", clock=clock)
        flagged.append(0 in r.frontier)
        cert = r.cert
    # 4 k eps >= 10 eps first at k = 3; revisited then, it expires again 3 steps later
    assert flagged == [False, False, True, False, False, True, False]

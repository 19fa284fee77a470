"""Pins of the local heuristic rho_i = delta_i / c_i > 1/2 (Sec. 3, Table 1):
delta_i is point i's own displacement, c_i its pre-step clearance.

* dyadic closed forms, where delta, c and 2 delta are exact in FP32: the
  comparison is strict, the factor is 2, c is a difference of distances (not
  of squared distances), and 0/0 is not flagged;
* a step-level dyadic scene: a static point is never flagged, whatever eps_t;
  a point that moves by more than half its clearance is;
* on every motion family the flags lie inside the per-point budget frontier
  (c <= 2 (delta + eps_t) + tau), and a flagged failure is a failure;
* it is a heuristic, not a bound: static points that fail are not flagged.
"""
import numpy as np
import pytest

import oracle
from paper_2606_18314_b300 import scenes


def test_rho_dyadic_closed_forms():
    # d1 = 1/4, d2 = 5/8: c = 3/8, flagged iff 2 delta > 3/8
    d1sq = np.full(5, 1 / 16, np.float32)
    d2sq = np.full(5, 25 / 64, np.float32)
    delta = np.array([1 / 4, 3 / 16, np.nextafter(np.float32(3 / 16), np.float32(1)), 0.0, 1 / 8], np.float32)
    assert list(oracle.rho(d1sq, d2sq, delta)) == [True, False, True, False, False]
    # c = 0 (nn and runner-up tie): 0/0 is not flagged, any motion is
    z = np.full(2, 1 / 16, np.float32)
    assert list(oracle.rho(z, z, np.array([0.0, 2.0 ** -30], np.float32))) == [False, True]
    # a squared-distance clearance, 25/64 - 4/64 = 21/64 < 3/8, would flag delta = 3/16
    assert not oracle.rho(d1sq[:1], d2sq[:1], np.array([3 / 16], np.float32))[0]


def _scene():
    """A at (1/4, 1/2) with nn B at 1/8 and runner-up C at 3/16 (c_A = 1/16);
    two far points D, E.  Dyadic coordinates: every distance is exact."""
    return np.array([[0.25, 0.5], [0.375, 0.5], [0.25, 0.5 - 0.1875], [0.875, 0.125], [0.9375, 0.125]],
                    np.float32)


def test_rho_step_level_dyadic():
    p = _scene()
    cert = oracle.top2(p)
    assert cert.nn[0] == 1 and cert.d1sq[0] == np.float32(1 / 64) and cert.d2sq[0] == np.float32(9 / 256)
    # only D moves, by 1/64: eps_t = 1/64 and 4 eps_t = c_A, so Algorithm 1 flags
    # A, but A did not move: rho_A = 0
    q = p.copy()
    q[3, 0] -= 1 / 64
    r = oracle.step(p, q, cert)
    assert r.eps_t == np.float32(1 / 64) and 0 in r.frontier
    assert not r.rho[0] and not r.rho[1] and not r.rho[2]
    # A moves by exactly c_A / 2 = 1/32 (away from B): 2 delta = c, not flagged
    q = p.copy()
    q[0, 0] -= 1 / 32
    r = oracle.step(p, q, cert)
    assert not r.rho[0]
    # by 1/32 + 1/128: flagged
    q = p.copy()
    q[0, 0] -= 1 / 32 + 1 / 128
    r = oracle.step(p, q, cert)
    assert r.rho[0] and r.n_rho >= 1
    # nothing moves: nothing is flagged
    r = oracle.step(p, p.copy(), cert)
    assert r.n_rho == 0 and r.n_rho_hit == 0


@pytest.mark.parametrize("family", scenes.ALL_FAMILIES)
@pytest.mark.parametrize("dim", [2, 3])
def test_rho_flags_lie_inside_the_point_budget_frontier(family, dim):
    m = scenes.Motion(family, 400, dim, eps=3e-3, seed=3, steps=40)
    p = m.frame()
    cert = oracle.top2(p)
    for _ in range(6):
        q = m.advance()
        r = oracle.step(p, q, cert, rule="point")
        inF = np.zeros(len(q), bool)
        inF[r.frontier] = True
        assert not np.any(r.rho & ~inF)
        assert r.n_rho == int(r.rho.sum()) and r.n_rho_hit == int((r.rho & r.failed).sum())
        assert r.n_rho_hit <= min(r.n_rho, r.n_failed)
        p, cert = q, r.cert


def test_rho_is_not_a_bound_static_points_fail_unflagged():
    m = scenes.Motion("adversarial_crossing", 2000, 3, eps=3e-3, seed=1, steps=40)
    p = m.frame()
    cert = oracle.top2(p)
    missed_static = 0
    for _ in range(8):
        q = m.advance()
        r = oracle.step(p, q, cert)
        static = np.all(p == q, axis=1)
        assert not np.any(r.rho & static)
        missed_static += int((r.failed & static).sum())
        p, cert = q, r.cert
    assert missed_static > 0

"""The parity checker itself: the comparisons the GPU tests make must fail
when a single certificate field, frontier entry, failure mark or count is
wrong.  Runs on the CPU: the oracle's own step stands in for the GPU's
outputs (as CPU torch tensors), then one value is corrupted at a time."""
import copy

import numpy as np
import pytest
import torch

import oracle
from paper_2606_18314_b300 import cert, scenes
from tests.test_gpu_parity import assert_cert_equal, assert_step_equal


class _Ctx:
    def __init__(self, n):
        self.offsets = np.array([0, n], np.int64)


def _outputs(r):
    n = r.cert.nn.shape[0]
    views = {"nn": torch.from_numpy(r.cert.nn.copy()), "d1sq": torch.from_numpy(r.cert.d1sq.copy()),
             "d2sq": torch.from_numpy(r.cert.d2sq.copy()), "cell": torch.from_numpy(r.cell.copy()),
             "failed": torch.from_numpy(r.failed.astype(np.uint8)),
             "frontier": torch.from_numpy(np.concatenate([r.frontier, np.zeros(n - len(r.frontier), np.int32)]))}
    res = np.zeros(1, cert.SCENE_DTYPE)
    sc = res[0]
    sc["eps_t"], sc["n_frontier"], sc["frontier_start"] = r.eps_t, len(r.frontier), 0
    sc["n_failed"], sc["n_missed"], sc["n_false"] = r.n_failed, r.n_missed, r.n_false
    sc["failed_cells"], sc["frontier_cells"], sc["occupied_cells"] = r.m, r.m_cand, r.C
    sc["grid_res"], sc["H"], sc["H_cand"], sc["med_c"] = r.g_h, r.H, r.H_cand, r.med_c
    return res, views


@pytest.fixture(scope="module")
def step():
    m = scenes.Motion("clustered_drift", 1500, 3, 3e-3, seed=9, steps=20)
    p = m.frame()
    q = m.advance()
    return oracle.step(p, q, oracle.top2(p))


def test_unmodified_outputs_pass(step):
    res, views = _outputs(step)
    assert_step_equal(_Ctx(len(step.cert.nn)), res, views, step)


@pytest.mark.parametrize("field", ["nn", "d1sq", "d2sq", "cell", "failed", "frontier"])
def test_one_corrupted_entry_fails(step, field):
    res, views = _outputs(step)
    t = views[field]
    i = int(np.flatnonzero(step.failed)[0]) if field == "failed" else 7
    if t.dtype == torch.float32:
        t.view(torch.int32)[i] += 1            # one unit in the last place
    elif t.dtype == torch.uint8:
        t[i] ^= 1
    else:
        t[i] += 1
    with pytest.raises(AssertionError):
        assert_step_equal(_Ctx(len(step.cert.nn)), res, views, step)


@pytest.mark.parametrize("field,delta", [("n_failed", 1), ("n_missed", 1), ("n_false", -1), ("failed_cells", 1),
                                         ("occupied_cells", 1), ("H", 2e-6), ("eps_t", 1e-9)])
def test_one_corrupted_count_fails(step, field, delta):
    res, views = _outputs(step)
    res[0][field] = res[0][field] + delta
    with pytest.raises(AssertionError):
        assert_step_equal(_Ctx(len(step.cert.nn)), res, views, step)


def test_corrupted_certificate_fails_the_certificate_check(step):
    _, views = _outputs(step)
    ref = copy.deepcopy(step.cert)
    assert_cert_equal(views, ref)
    ref.nn[3] = (ref.nn[3] + 1) % len(ref.nn)
    with pytest.raises(AssertionError):
        assert_cert_equal(views, ref)

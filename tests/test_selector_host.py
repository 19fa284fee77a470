"""Host logic of the selector (no GPU): the decision margin and the regret."""
import numpy as np

from paper_2606_18314_b300 import selector


def test_regret_definition():
    T = np.log(np.array([[1.0, 2.0], [3.0, 1.0], [2.0, 2.0]]))
    assert selector.regret(T, np.array([True, False, True])) == 0.0
    # choosing rebuild on row 0 costs 1, incremental on row 1 costs 2; best total is 1 + 1 + 2 = 4
    assert abs(selector.regret(T, np.array([False, True, True])) - 3.0 / 4.0) < 1e-12


def test_margin_all_incremental_when_incremental_always_wins():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((500, 2))
    T = np.stack([np.zeros(500), np.ones(500)], 1)          # incremental always faster
    d = selector.decision_margin(Y, T)
    assert np.all(Y[:, 0] - Y[:, 1] <= d)
    assert selector.regret(T, Y[:, 0] - Y[:, 1] <= d) == 0.0


def test_margin_recovers_a_shifted_boundary():
    """Measured times make rebuild best exactly when the predicted difference
    exceeds 0.3: the margin must land between the neighbouring differences."""
    rng = np.random.default_rng(1)
    diff = np.sort(rng.uniform(-1, 1, 400))
    Y = np.stack([diff, np.zeros_like(diff)], 1)
    inc_best = diff <= 0.3
    T = np.where(inc_best[:, None], [[0.0, 0.5]], [[0.5, 0.0]])
    d = selector.decision_margin(Y, T)
    assert selector.regret(T, diff <= d) == 0.0
    assert diff[inc_best].max() <= d < diff[~inc_best].min()

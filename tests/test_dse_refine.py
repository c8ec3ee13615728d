"""Host logic of the refined design-space search (``dse.explore`` with
rounds > 1), on the CPU: the exact simulator and the surrogate are replaced
by a known objective and a least-squares model, so the bookkeeping can be
checked exactly -- no candidate is simulated twice, every round simulates
top_k new candidates, the random baseline gets the same budget, and the
reported figures are the ones the simulated values give."""

import numpy as np
import pytest

from paper_2404_16208_gb300 import dse
from ranc_workloads import dse as D


def true_targets(points):
    """A smooth stand-in for (agreement, relative traffic) of a design point."""
    f = dse.features(points).astype(np.float64)
    agreement = 1.0 - np.abs(f[:, 6] - 0.3) - 0.3 * np.abs(f[:, 7] - 0.5) + 0.05 * f[:, 0]
    traffic = 0.2 + f[:, 0] * (0.5 + f[:, 6]) + 0.1 * f[:, 9]
    return np.stack([agreement, traffic], axis=1)


class FakeEvaluator:
    def __init__(self):
        self.seen = []
        self.n_sims = 0
        self.sim_seconds = 0.0
        self.launches = 0

    def targets(self, points):
        self.seen.extend(points)
        self.n_sims += len(points)
        return true_targets(points)


class LeastSquares:
    """Quadratic least squares on the features (a CPU surrogate)."""

    def __init__(self, seed):
        self.w = None

    @staticmethod
    def _expand(X):
        X = np.asarray(X, np.float64)
        return np.concatenate([np.ones((len(X), 1)), X, X ** 2], axis=1)

    def fit(self, X, Y, steps=0):
        A = self._expand(X)
        self.w = np.linalg.lstsq(A, Y, rcond=None)[0]
        return [float(np.mean((A @ self.w - Y) ** 2))]

    def predict(self, X):
        return self._expand(X) @ self.w


@pytest.mark.parametrize("rounds", [1, 3])
def test_refined_search_bookkeeping(rounds):
    ev = FakeEvaluator()
    n_train, n_val, n_cand, k = 60, 20, 400, 8
    rep = dse.explore(n_train=n_train, n_val=n_val, n_candidates=n_cand, top_k=k, seed=5, steps=0,
                      evaluator=ev, rounds=rounds, surrogate=LeastSquares)
    assert rep["rounds"] == rounds
    # training and validation points, then per round top_k searched and top_k random
    assert ev.n_sims == n_train + n_val + 2 * rounds * k
    searched = ev.seen[n_train + n_val:]
    cand = D.sample_points(6, n_cand)
    search = searched[:k]
    if rounds > 1:  # the first search's random choice follows it; the rest of the random choice comes last
        search = searched[:k] + searched[2 * k:2 * k + (rounds - 1) * k]
    assert len(set(search)) == rounds * k, "a candidate was simulated twice by the search"
    assert all(p in cand for p in search)
    assert rep["exact_sims_saved"] == n_cand - rounds * k
    truth = dse.objective(*true_targets(search).T)
    assert rep["top_true_objective_mean"] == pytest.approx(truth[:k].mean())
    if rounds > 1:
        assert len(rep["round_history"]) == rounds
        assert rep["refined_best"] == pytest.approx(truth.max())
        assert rep["refined_best"] >= rep["top_true_objective_best"]
        assert rep["refined_top_mean"] == pytest.approx(np.sort(truth)[-k:].mean())
        for r, h in enumerate(rep["round_history"]):
            assert h["mean"] == pytest.approx(truth[r * k:(r + 1) * k].mean())


def test_refined_search_finds_the_top_of_a_learnable_objective():
    """With a surrogate that can represent the objective, the search's best
    beats the random choice of the same budget and comes close to the best
    candidate of all."""
    ev = FakeEvaluator()
    n_cand = 2000
    rep = dse.explore(n_train=200, n_val=40, n_candidates=n_cand, top_k=16, seed=9, steps=0, evaluator=ev,
                      rounds=3, surrogate=LeastSquares)
    cand = D.sample_points(10, n_cand)
    truth = dse.objective(*true_targets(cand).T)
    assert rep["refined_best"] > rep["random_best_same_budget"]
    assert rep["refined_best"] >= np.sort(truth)[-5]  # among the five best candidates


def test_column_features_equal_the_points_own():
    """The surrogate's column-wise feature matrix equals Point.features() row by row."""
    pts = D.sample_points(3, 500) + [D.NOMINAL]
    np.testing.assert_array_equal(dse.features(pts), np.stack([p.features() for p in pts]))

"""Design-space exploration end to end: the surrogate is trained on the GPU
with the library's own kernels on exactly simulated design points, ranks
unseen candidates, and the exact simulator re-scores its choice.  The test is
what the trained network gains over choosing the same number of candidates at
random."""

import pytest

pytestmark = pytest.mark.gpu


def test_surrogate_choice_beats_random_choice():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import dse
    rep = dse.explore(n_train=160, n_val=40, n_candidates=2000, top_k=16, seed=21, steps=1500, n_samples=128)
    assert rep["val_spearman_objective"] > 0.3, rep
    assert rep["gain_mean"] > 0.0, rep
    assert rep["top_true_objective_mean"] > rep["random_true_objective_mean"], rep

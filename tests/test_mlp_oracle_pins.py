"""Pins of the surrogate's CPU oracle (oracle/mlp_ref.py): its analytic
gradients must equal central finite differences of its own loss, and a
one-layer network must reproduce the closed-form least-squares gradient."""

import numpy as np

from oracle import mlp_ref


def _random_params(dims, rng):
    return [(rng.normal(size=(o, i)), rng.normal(size=o)) for i, o in zip(dims[:-1], dims[1:])]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    dims = (5, 7, 6, 2)
    params = _random_params(dims, rng)
    x = rng.normal(size=(9, dims[0]))
    t = rng.normal(size=(9, dims[-1]))
    _, grads = mlp_ref.loss_and_grads(params, x, t)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp_ref.loss(params, x, t)
                arr[idx] = old - h
                lm = mlp_ref.loss(params, x, t)
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-6 * max(1.0, abs(g[idx])), (li, idx)


def test_single_linear_layer_closed_form():
    rng = np.random.default_rng(4)
    W, b = rng.normal(size=(3, 4)), rng.normal(size=3)
    x, t = rng.normal(size=(8, 4)), rng.normal(size=(8, 3))
    loss, grads = mlp_ref.loss_and_grads([(W, b)], x, t)
    r = x @ W.T + b - t
    assert np.isclose(loss, (r ** 2).mean())
    assert np.allclose(grads[0][0], 2 * r.T @ x / r.size)
    assert np.allclose(grads[0][1], 2 * r.sum(axis=0) / r.size)


def test_flatten_round_trip():
    rng = np.random.default_rng(5)
    dims = (4, 3, 2)
    params = _random_params(dims, rng)
    flat = mlp_ref.flatten(params)
    back = mlp_ref.unflatten(flat, dims)
    for (W, b), (W2, b2) in zip(params, back):
        assert (W == W2).all() and (b == b2).all()

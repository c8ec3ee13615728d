"""Surrogate kernels (include/ranc_mlp.h) against the CPU fp64 oracle
(oracle/mlp_ref.py) on the same bf16-rounded weights: forward outputs, loss
and every gradient; one Adam step against its definition."""

import numpy as np
import pytest

from oracle import mlp_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlp_mod():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import mlp
    return mlp


@pytest.mark.parametrize("dims,batch", [((10, 128, 128, 128, 2), 256), ((7, 33, 5), 19), ((3, 1), 1)])
def test_forward_loss_gradients_match_oracle(mlp_mod, dims, batch):
    import torch
    m = mlp_mod.MLP(dims, 256, seed=7)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(batch, dims[0])).astype(np.float32)
    t = rng.normal(size=(batch, dims[-1])).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    params = mlp_ref.unflatten(m.get_params().astype(np.float64), dims)
    dy = torch.zeros((batch, dims[-1]), dtype=torch.float32, device="cuda")
    m.forward(dx.data_ptr(), batch, dy.data_ptr())
    torch.cuda.synchronize()
    _, y_ref = mlp_ref.forward(params, x)
    np.testing.assert_allclose(dy.cpu().numpy(), y_ref, rtol=2e-4, atol=2e-5)
    loss, g = m.loss_backward(dx.data_ptr(), dt.data_ptr(), batch, want_grads=True)
    loss_ref, g_ref = mlp_ref.loss_and_grads(params, x, t)
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref) + 1e-6
    g_ref = mlp_ref.flatten(g_ref)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-4 * scale, np.abs(g - g_ref).max() / scale
    m.close()


def test_adam_step_matches_its_definition(mlp_mod):
    import torch
    dims = (4, 8, 2)
    m = mlp_mod.MLP(dims, 16, seed=3)
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=m.n_params).astype(np.float32)
    m.set_params(p0)
    x = torch.from_numpy(rng.normal(size=(16, 4)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(16, 2)).astype(np.float32)).cuda()
    _, g = m.loss_backward(x.data_ptr(), t.data_ptr(), 16, want_grads=True)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    m.adam_step(lr, b1, b2, eps)
    mt = (1 - b1) * g.astype(np.float64)
    vt = (1 - b2) * g.astype(np.float64) ** 2
    p1 = p0 - lr * (mt / (1 - b1)) / (np.sqrt(vt / (1 - b2)) + eps)
    got = m.get_params()
    w_mask = np.zeros(m.n_params, bool)
    k = 0
    for i, o in zip(dims[:-1], dims[1:]):
        w_mask[k:k + i * o] = True
        k += i * o + o
    # weights come back bf16-rounded, biases exact fp32
    np.testing.assert_allclose(got[~w_mask], p1[~w_mask], rtol=1e-5, atol=1e-6)
    bf = (p1[w_mask].astype(np.float32).view(np.uint32) + 0x7FFF + ((p1[w_mask].astype(np.float32).view(np.uint32) >> 16) & 1)) & 0xFFFF0000
    np.testing.assert_allclose(got[w_mask], bf.view(np.float32), rtol=0, atol=1e-2 * np.abs(p1).max())
    m.close()


def test_training_reduces_loss(mlp_mod):
    import torch
    rng = np.random.default_rng(9)
    X = rng.uniform(size=(256, 6)).astype(np.float32)
    Y = np.stack([np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2], X[:, 3] - X[:, 4] ** 2], axis=1).astype(np.float32)
    m = mlp_mod.MLP((6, 64, 64, 2), 256, seed=5)
    dx, dy = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    l0, _ = m.loss_backward(dx.data_ptr(), dy.data_ptr(), 256)
    for _ in range(600):
        m.loss_backward(dx.data_ptr(), dy.data_ptr(), 256)
        m.adam_step(3e-3)
    l1, _ = m.loss_backward(dx.data_ptr(), dy.data_ptr(), 256)
    assert l1 < 0.05 * l0, (l0, l1)
    m.close()

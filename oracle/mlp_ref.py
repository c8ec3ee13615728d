"""CPU fp64 restatement of the design-space surrogate's passes (test
infrastructure only): a fully connected network with ReLU hidden layers and a
linear output, mean squared error loss, and its gradients by the chain rule.

The GPU passes use bf16 weights and fp32 accumulation; given the same
bf16-rounded weights (as float64) this restatement is the exact value they
approximate.  It is pinned in the tests by central finite differences.
"""

import numpy as np


def unflatten(flat, dims):
    """Flat parameters (each layer: W [out][in] row major, then b [out]) -> list of (W, b)."""
    out, k = [], 0
    for i, o in zip(dims[:-1], dims[1:]):
        W = np.asarray(flat[k:k + i * o], dtype=np.float64).reshape(o, i)
        k += i * o
        b = np.asarray(flat[k:k + o], dtype=np.float64)
        k += o
        out.append((W, b))
    return out


def flatten(grads):
    return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def forward(params, x):
    """Returns the pre-activations of every layer and the output."""
    a = np.asarray(x, dtype=np.float64)
    zs = []
    for li, (W, b) in enumerate(params):
        z = a @ W.T + b
        zs.append(z)
        a = np.maximum(z, 0.0) if li + 1 < len(params) else z
    return zs, a


def loss(params, x, t):
    _, y = forward(params, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grads(params, x, t):
    """MSE over batch and outputs, and its gradient for every (W, b)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    zs, y = forward(params, x)
    B, d = y.shape
    dz = 2.0 * (y - t) / (B * d)
    grads = [None] * len(params)
    acts = [x] + [np.maximum(z, 0.0) for z in zs[:-1]]
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (dz.T @ acts[li], dz.sum(axis=0))
        if li > 0:
            dz = (dz @ W) * (zs[li - 1] > 0)
    return float(np.mean((y - t) ** 2)), grads

"""The crossbar-product formulations (include/ranc_xbar.h) against the
crossbar oracle, bit for bit: the folded fp16 tcgen05 GEMM, the per-type
e4m3 tcgen05 GEMMs and the per-type int8 mma.sync GEMMs must all give the same
dV = sum_k w_k (S_k @ C_k) on random cores of every supported shape, with up to
12-bit weights, and on the 512-core MNIST-shaped network."""

import numpy as np
import pytest

import ranc_workloads as W
from oracle import crossbar as X

pytestmark = pytest.mark.gpu
FORMS = {"f16_folded": 0, "f8_per_type": 1, "i8_mma_sync": 2}


@pytest.fixture(scope="module")
def ranc():
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc as mod
    return mod


def run_form(ranc, net, form, S):
    import torch
    B = S.shape[0]
    spikes = torch.from_numpy(W.pack_bits_lsb(S).view(np.int32)).cuda()
    dv = torch.zeros((B, net.n_cores, net.neurons), dtype=torch.int32, device="cuda")
    sums = torch.zeros((B, net.n_cores), dtype=torch.int64, device="cuda")
    x = ranc.Xbar(net, form)
    x.run(spikes.data_ptr(), B, dv.data_ptr(), sums.data_ptr())
    x.sync()
    x.close()
    return dv.cpu().numpy(), sums.cpu().numpy()


SHAPES = [(64, 128, 1, 255), (128, 256, 4, 2047), (192, 128, 3, 2047), (256, 256, 2, 255), (256, 128, 4, 7)]


@pytest.mark.parametrize("form", list(FORMS), ids=list(FORMS))
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{n}k{k}" for a, n, k, _ in SHAPES])
def test_forms_equal_the_oracle(ranc, form, shape):
    A, N, K, wl = shape
    net = W.random_net(40 + A + N + K, 3, 1, axons=A, neurons=N, n_types=K, density=0.35, w_lim=wl, weight_bits=12)
    B = 256
    S = W.rng.bernoulli(A + K, 97, (B, A), 0.3)
    dv, sums = run_form(ranc, net, FORMS[form], S)
    ref = X.delta_v(net, W.pack_bits_lsb(S))
    np.testing.assert_array_equal(dv, ref)
    np.testing.assert_array_equal(sums, X.digest_sums(ref))


@pytest.mark.parametrize("form", list(FORMS), ids=list(FORMS))
def test_forms_on_the_mnist_shaped_network(ranc, form):
    net = W.mnist_512core()
    B = 256
    S = W.rng.bernoulli(5, 96, (B, net.axons), 0.2)
    dv, sums = run_form(ranc, net, FORMS[form], S)
    cores = list(range(0, 512, 37))
    ref = X.delta_v(net, W.pack_bits_lsb(S), cores=cores)
    np.testing.assert_array_equal(dv[:, cores], ref)
    np.testing.assert_array_equal(sums[:, cores], X.digest_sums(ref))


def test_shape_checks(ranc):
    net = W.random_net(3, 1, 1, axons=96, neurons=128)
    with pytest.raises(ranc.RancError) as ei:
        ranc.Xbar(net, 0)
    assert ei.value.code == ranc.RANC_EINVAL
    net = W.random_net(3, 1, 1, axons=64, neurons=128)
    with pytest.raises(ranc.RancError):
        ranc.Xbar(net, 3)

"""Pins of the U-Net oracle (oracle/unet_oracle.py) against textbook routines,
finite differences and exact properties.  CPU only."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import unet_oracle as U


def test_conv3_equals_textbook_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 5, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[bi, :, :, c], W[o, :, :, c], mode="same", boundary="fill")
                             for c in range(3))
            assert np.allclose(y[bi, :, :, o], ref, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 8, 8, 3))
    y = rng.standard_normal((2, 4, 4, 3))
    assert np.isclose(np.sum(U.pool2(x) * y), np.sum(x * U.pool2_backward(y)))
    assert np.isclose(np.sum(U.up2(y) * x), np.sum(y * U.up2_backward(x)))
    # pooling a constant gives the constant; upsampling then pooling is the identity
    assert np.allclose(U.pool2(np.ones((1, 4, 4, 1))), 1.0)
    assert np.allclose(U.pool2(U.up2(y)), y)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    c0, n = 2, 7
    theta = rng.standard_normal(U.n_params(c0)) * 0.3
    x = rng.standard_normal((2, n + 1, n + 1, 3))
    t = rng.standard_normal((2, n, n))
    _, g = U.loss_and_grad(theta, x, t, c0)
    idx = rng.choice(theta.size, 40, replace=False)
    # include the output layer and a few biases
    idx = np.concatenate([idx, [theta.size - 1, theta.size - 2, U.layer_table(c0)[0][3] * 27]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (U.loss_and_grad(theta + e, x, t, c0)[0] - U.loss_and_grad(theta - e, x, t, c0)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_parameter_count_of_the_c0_32_network():
    # ~1.9 M parameters for the 255^2 warm start (c0 = 32)
    # per layer co * 9 ci + co: 896 + 9248 + 18496 + 36928 + 73856 + 147584 + 295168 + 590080
    # + 442496 + 147584 + 110656 + 36928 + 27680 + 9248, plus 32 + 1 for the output layer
    assert U.n_params(32) == 1_946_881


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = U.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-5, 5, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(a), ref)


def test_input_channels_of_interior_observations():
    n = 15
    site = np.array([[16, 17, 31, 32]])  # sites (1,1), (2,1), (1,2), (2,2): id = i + n j
    w = np.array([[0.1, 0.2, 0.3, 0.4]])
    x = U.make_inputs(n, 10.0 * np.ones(n * n), site, w, np.array([2.0]))
    assert np.allclose(x[..., 0], 0.0)
    assert np.isclose(x[..., 1].sum(), 1.0) and np.isclose(x[..., 2].sum(), 2.0)
    assert x[2, 2, 1] == 0.4 and x[1, 1, 2] == 0.2 and x[1, 2, 1] == 0.2  # x[j, i]
    assert np.all(x[n, :, :] == 0) and np.all(x[:, n, :] == 0)


def test_splitmix64_reference_values():
    # splitmix64 from seed 0: the first outputs of the published generator
    r = U.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_epoch_permutation_is_a_permutation():
    r = U.SplitMix64(9)
    for n in (1, 2, 17):
        assert sorted(U.epoch_permutation(n, r)) == list(range(n))

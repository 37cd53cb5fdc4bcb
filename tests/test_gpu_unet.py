"""Learned warm start (mgmc_unet_*) against the FP64 U-Net oracle on small grids."""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2407_12149_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _bf16_bits(torch, a):
    """FP64 array -> (BF16-rounded FP64 array, CUDA int16 tensor of the BF16 bits)."""
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy(), t.view(torch.int16).cuda()


def _setup(torch, n=31, c0=8, batch=2, seed=0):
    from paper_2407_12149_gb300.mgmc import Unet
    rng = np.random.default_rng(seed)
    net = Unet(n, c0=c0, max_batch=batch, seed=seed)
    theta = net.get_params().astype(np.float64)
    theta[U.n_params(c0) - c0 - 1:] = rng.standard_normal(c0 + 1) * 0.3    # non-trivial output layer
    off = 0
    for _, _, ci, co in U.layer_table(c0):                                     # non-zero biases
        off += co * 9 * ci
        theta[off:off + co] = rng.standard_normal(co) * 0.05
        off += co
    net.set_params(theta.astype(np.float32))
    theta = net.get_params().astype(np.float64)
    x = rng.standard_normal((batch, n + 1, n + 1, 3))
    x[:, n, :, :] = 0.0
    x[:, :, n, :] = 0.0
    xr, xbits = _bf16_bits(torch, x)
    t = rng.standard_normal((batch, n, n))
    return net, theta, xr, xbits, t


def test_forward_matches_oracle(torch_mod):
    torch = torch_mod
    n, c0 = 31, 8
    net, theta, xr, xbits, _ = _setup(torch, n, c0)
    got = net.predict(xbits, precision="fp64").cpu().numpy().reshape(2, n, n)
    ref, _ = U.forward(theta, xr, c0, bf16=True)
    ref = ref[:, :n, :n]
    rms = np.sqrt(np.mean(ref ** 2))
    # BF16 storage of activations: a rounding that lands on the other side of a
    # BF16 tie in one layer moves its value by 2^-8 relative and propagates, so the
    # bound is on the relative L2 error (1e-2), with 5e-2 of the RMS at any one site
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-2, rel
    assert np.abs(got - ref).max() <= 5e-2 * rms, np.abs(got - ref).max() / rms


@pytest.mark.parametrize("batch", [2, 4])
def test_gradient_matches_oracle(torch_mod, batch):
    """batch 4 splits the weight-gradient GEMMs of the finest level over pixels."""
    torch = torch_mod
    n, c0 = 31, 8
    net, theta, xr, xbits, t = _setup(torch, n, c0, batch=batch, seed=1)
    tg = torch.tensor(t.reshape(batch, n * n), dtype=torch.float32).cuda()
    loss, g = net.gradient(xbits, tg, batch)
    lo, go = U.loss_and_grad(theta, xr, t, c0, bf16=True)
    assert abs(loss - lo) <= 1e-2 * lo
    # per layer: relative error of the weight and of the bias gradient
    o = 0
    for name, _, ci, co in U.layer_table(c0) + [("out", 0, c0, 1)]:
        nw = co * 9 * ci if name != "out" else c0
        for sl in (slice(o, o + nw), slice(o + nw, o + nw + co)):
            ref = go[sl]
            err = np.linalg.norm(g[sl] - ref) / max(np.linalg.norm(ref), 1e-12)
            assert err <= 5e-2, (name, err)
        o += nw + co


def test_forward_and_gradient_at_warm_start_size(torch_mod):
    """The network the warm-start workload runs: 255^2 grid, c0 = 32 (about 2M
    parameters, the bottom convolutions on N = 256 GEMM tiles), batch 2."""
    torch = torch_mod
    n, c0, batch = 255, 32, 2
    net, theta, xr, xbits, t = _setup(torch, n, c0, batch=batch, seed=3)
    got = net.predict(xbits, precision="fp64").cpu().numpy().reshape(batch, n, n)
    ref, _ = U.forward(theta, xr, c0, bf16=True)
    ref = ref[:, :n, :n]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-2, rel
    assert np.abs(got - ref).max() <= 5e-2 * np.sqrt(np.mean(ref ** 2))
    tg = torch.tensor(t.reshape(batch, n * n), dtype=torch.float32).cuda()
    loss, g = net.gradient(xbits, tg, batch)
    lo, go = U.loss_and_grad(theta, xr, t, c0, bf16=True)
    assert abs(loss - lo) <= 1e-2 * lo
    o = 0
    for name, _, ci, co in U.layer_table(c0) + [("out", 0, c0, 1)]:
        nw = co * 9 * ci if name != "out" else c0
        for sl in (slice(o, o + nw), slice(o + nw, o + nw + co)):
            ref_g = go[sl]
            err = np.linalg.norm(g[sl] - ref_g) / max(np.linalg.norm(ref_g), 1e-12)
            assert err <= 5e-2, (name, err)
        o += nw + co
    net.close()


def test_one_adam_step_matches_oracle(torch_mod):
    """one step over a single batch (the shuffle cannot change it) against Adam on the
    oracle's gradient: the first step moves each parameter by about lr sign(g)"""
    torch = torch_mod
    n, c0, lr = 31, 8, 1e-3
    net, theta, xr, xbits, t = _setup(torch, n, c0, batch=4, seed=2)
    tg = torch.tensor(t.reshape(4, n * n), dtype=torch.float32).cuda()
    net.train(xbits, tg, epochs=1, batch=4, lr=lr, shuffle_seed=0)
    after = net.get_params().astype(np.float64)
    _, go = U.loss_and_grad(theta, xr, t, c0, bf16=True)
    ref, _, _ = U.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), go, 1, lr)
    # parameters whose gradient is clearly non-zero move by lr sign(g) on both sides
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    assert np.mean(np.abs((after - theta)[big] - (ref - theta)[big]) <= 0.05 * lr) >= 0.98


def _toy_task(torch, n=31, ns=16):
    """inputs: white noise in the three channels; target: the 2x2 block average of channel 2"""
    rng = np.random.default_rng(7)
    x = np.zeros((ns, n + 1, n + 1, 3))
    x[:, :n, :n, :] = rng.standard_normal((ns, n, n, 3))
    xr, xbits = _bf16_bits(torch, x)
    t = np.stack([U.up2(U.pool2(xr[k:k + 1, ..., 2:3]))[0, :n, :n, 0] for k in range(ns)])
    return xr, xbits, t, torch.tensor(t.reshape(ns, n * n), dtype=torch.float32).cuda()


def test_training_matches_oracle_replay(torch_mod):
    """the same initialisation (splitmix64 He-normal, seed 1), shuffles and Adam steps on
    the oracle give the device's per-epoch training losses"""
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import Unet
    n, c0 = 31, 8
    xr, xbits, t, tg = _toy_task(torch)
    net = Unet(n, c0=c0, max_batch=4, seed=1)
    th0 = net.get_params().astype(np.float64)
    # the same draws; libm and numpy may differ in the last bit of log / cos before rounding to FP32
    assert np.allclose(th0, U.init_params(c0, 1), rtol=1e-6, atol=1e-9)
    losses = net.train(xbits, tg, epochs=6, batch=4, lr=3e-3, shuffle_seed=5)
    _, ref = U.train(th0, xr, t, c0, epochs=6, batch=4, lr=3e-3, shuffle_seed=5, bf16=True)
    assert np.all(np.abs(losses - ref) <= 2e-2 * ref), (losses, ref)


def test_training_lowers_the_loss(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import Unet
    xr, xbits, t, tg = _toy_task(torch)
    net = Unet(31, c0=8, max_batch=4, seed=1)
    losses = net.train(xbits, tg, epochs=24, batch=4, lr=3e-3, shuffle_seed=5)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], losses


def test_input_channels_match_oracle(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import unet_inputs
    p = inputs.make_problem("u", 2, 31, kappa2_seed=3, m=12, obs_seed=4, qoi_cells=8)
    got = unet_inputs(p).view(np.int16)
    ref = U.make_inputs(31, p.kappa2, p.obs_site, p.obs_w, p.y)
    refbits = torch.tensor(ref.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(got, refbits)

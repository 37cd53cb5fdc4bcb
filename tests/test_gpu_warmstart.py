"""What the learned warm start gains: fewer burn-in cycles on held-out problems.

A U-Net (c0 = 16) is trained on FP64 mean-solve targets of 96 seeded 63^2
posteriors (kappa^2 = 10 exp(g), 8..32 point observations) and used as x0 of
the chains of 32 held-out posteriors.  MGMC's invariant law does not depend on x0
(Sec. 4), only the burn-in does: the expected state after m cycles is
mu + X^m (x0 - mu), X the noise-free cycle's iteration matrix, which the library
applies as one noise-free V-cycle per mgmc_mean_solve cycle.  The expected burn-in
of a chain is the first m with |F (E theta^(m) - mu)| <= 1e-3 sd(F theta) under the
posterior (exact moments by a sparse direct solve); it must be shorter from the
network's estimate than from 0.
"""
import numpy as np
import pytest

from paper_2407_12149_gb300 import experiments, inputs

pytestmark = pytest.mark.gpu

N = 63
TOL = 1e-3      # bias target, in posterior standard deviations of the QoI
MAX_CYCLES = 12


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _problems(count, first):
    out = []
    for s in range(first, first + count):
        m = int(np.random.default_rng(40000 + s).integers(8, 33))
        out.append(inputs.make_problem(f"ws-{s}", 2, N, kappa2_seed=50000 + s, m=m, obs_seed=60000 + s,
                                       qoi_cells=4))
    return out


def _burn_in(M, p, x0, fmu, sd):
    """expected burn-in: noise-free cycles until the QoI bias is within TOL sd"""
    s = M.Sampler(p, precision="fp64", coarse_max_n=31)
    x = x0.clone()
    try:
        for m in range(MAX_CYCLES + 1):
            q = float(np.dot(p.qoi_w, x.cpu().numpy()[p.qoi_site]))
            if abs(q - fmu) <= TOL * sd:
                return m
            s.mean_solve(x, rtol=0.0, max_cycles=1)
        return MAX_CYCLES + 1
    finally:
        s.close()


def test_warm_start_shortens_burn_in_on_held_out_problems(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300 import mgmc as M
    dev = torch.device("cuda", 0)
    train, test = _problems(96, 0), _problems(32, 1_000_000)

    def targets(ps):
        T = torch.zeros(len(ps), N * N, dtype=torch.float64, device=dev)
        for k, p in enumerate(ps):
            s = M.Sampler(p, precision="fp64", coarse_max_n=31)
            s.mean_solve(T[k], rtol=1e-12, max_cycles=200)
            s.close()
        return T

    Xtr = torch.from_numpy(np.stack([M.unet_inputs(p) for p in train]).view(np.int16)).to(dev)
    Xte = torch.from_numpy(np.stack([M.unet_inputs(p) for p in test]).view(np.int16)).to(dev)
    Ttr, Tte = targets(train), targets(test)
    net = M.Unet(N, c0=16, max_batch=8, seed=3)
    losses = net.train(Xtr, Ttr.float(), epochs=30, batch=8, lr=1e-3, shuffle_seed=4)
    assert losses[-1] < 0.5 * losses[0]
    mu_hat = net.predict(Xte, precision="fp64")
    torch.cuda.synchronize()
    net.close()
    rel = ((mu_hat - Tte).norm(dim=1) / Tte.norm(dim=1)).cpu().numpy()
    assert rel.mean() < 0.5, rel.mean()

    b_zero, b_net = [], []
    for k, p in enumerate(test):
        fmu, s2 = experiments.exact_qoi_moments(p)
        sd = float(np.sqrt(s2))
        b_zero.append(_burn_in(M, p, torch.zeros(N * N, dtype=torch.float64, device=dev), fmu, sd))
        b_net.append(_burn_in(M, p, mu_hat[k].contiguous(), fmu, sd))
    b_zero, b_net = np.array(b_zero), np.array(b_net)
    # fewer cycles on average, and never more than one extra on any problem
    assert b_net.mean() <= b_zero.mean() - 0.5, (b_zero, b_net)
    assert np.all(b_net <= b_zero + 1), (b_zero, b_net)

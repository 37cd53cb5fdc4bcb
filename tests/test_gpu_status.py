"""Device status reporting and the timeout path of the bounded staging waits.

A test-only wait bound below zero makes every staging wait of a chain's kernels
give up at once: the kernel flags the chain, lets the copies it has in flight
land (within the default bound) and ends, and the host reports MGMC_ERR_TIMEOUT
when it next synchronises.  Nothing waits on a flag that is never set and no
kernel is made to fault.  After the bound is restored the same handle samples
correctly again (checked against the FP64 CPU oracle).  Also: the host-buffer
mode of mgmc_sample_batch equals its device-buffer mode.
"""
import numpy as np
import pytest

import oracle
from paper_2407_12149_gb300 import inputs

pytestmark = pytest.mark.gpu

MGMC_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _orc(p):
    return oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, kappa2_const=p.kappa2_const, scale_hd=p.scale_hd,
                         obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma, y=p.y, qoi_site=p.qoi_site,
                         qoi_w=p.qoi_w)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wait_that_gives_up_reports_timeout_and_handle_recovers(torch_mod, precision):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import MGMCError, Sampler
    # 255^2: the finest grid runs in the streamed (FP32) or tiled (FP64) TMA kernels
    p = inputs.make_problem("status", 2, 255, kappa2_seed=5, m=8, obs_seed=6, qoi_cells=24)
    s = Sampler(p, precision=precision, coarse_max_n=31)
    x = s.zeros().cpu()
    s.set_wait_limit(-1)
    with pytest.raises(MGMCError) as e:
        s.sample(x, 2, 11)                     # host buffer: the call synchronises and reports
    assert e.value.code == MGMC_ERR_TIMEOUT
    s.check_status()                           # reported once, then cleared
    # device buffers: asynchronous; the bit stays set until mgmc_check_status
    xd = s.zeros()
    s.sample(xd, 1, 11)
    with pytest.raises(MGMCError) as e:
        s.check_status()
    assert e.value.code == MGMC_ERR_TIMEOUT
    s.check_status()
    # the default bound again: the same handle reproduces the oracle from a fresh state
    s.set_wait_limit(0)
    x = s.zeros().cpu()
    s.sample(x, 20, 11)
    xo, _ = _orc(p).sample(20, 11)
    rms = np.sqrt(np.mean(xo ** 2))
    err = np.abs(x.double().numpy() - xo)
    if precision == "fp64":
        assert np.all(err <= 1e-11 * np.maximum(np.abs(xo), rms))
    else:
        assert err.max() <= 2e-4 * rms
    s.close()


def test_batch_timeout_and_host_buffers(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import BatchSampler, MGMCError
    ps = [inputs.make_problem(f"b{c}", 2, n, kappa2_seed=20 + c, m=8 + c, obs_seed=30 + c, qoi_cells=12)
          for c, n in enumerate((63, 127, 255, 127))]
    b = BatchSampler(ps, precision="fp32")
    # device buffers vs host buffers (copied through the device inside the call): bitwise equal
    xd = b.zeros()
    qd = torch.zeros(len(ps) * 7, dtype=torch.float64, device="cuda")
    b.sample(xd, 7, 3, qoi=qd)
    xh = [torch.zeros(p.N, dtype=torch.float32) for p in ps]
    qh = torch.zeros(len(ps) * 7, dtype=torch.float64)
    b.sample(xh, 7, 3, qoi=qh)
    torch.cuda.synchronize()
    for a, c in zip(xd, xh):
        assert torch.equal(a.cpu(), c)
    assert torch.equal(qd.cpu(), qh)
    # a wait that gives up, reported by the synchronising host-buffer call
    b.set_wait_limit(-1)
    with pytest.raises(MGMCError) as e:
        b.sample([torch.zeros(p.N, dtype=torch.float32) for p in ps], 1, 3)
    assert e.value.code == MGMC_ERR_TIMEOUT
    b.set_wait_limit(0)
    b.check_status()
    xr = [torch.zeros(p.N, dtype=torch.float32) for p in ps]
    b.sample(xr, 7, 3)
    for a, c in zip(xh, xr):
        assert torch.equal(a, c)
    b.close()

"""Benchmark of the GB300 MGMC sampler on the 1023^2 Bayesian posterior.

Posterior: 2D unit square, 1023 x 1023 interior grid (h = 1/1024), non-stationary
kappa^2 = 10 exp(g), 16 point observations, Gamma = 1e-4 I, 10-grid V-cycle with
the paper's low-rank Gibbs smoother (nu1 = nu2 = 1), FP32 sweeps with FP64
low-rank / coarsest / QoI arithmetic.  The default workload advances 32
independent chains of this posterior with batched launches (the batched + FP32
form); one step = one V-cycle (the whole hot path) of every chain.  The metric
is QoI ESS/s = (chain V-cycles/s) / tau_int, tau_int measured on the device
(Wolff window) from untimed 2000-cycle chains.  The plain FP64 single-chain GPU
sampler is timed in the same run for comparison (config.plain_fp64_single_chain).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

--impl reference times the plain FP64 CPU oracle on the host cores (the only
baseline this method has: the paper's code is a sequential CPU program).
Multi-GPU: replicas only -- every rank advances its own independent chains of
the same problem (one chain: Philox chain id = rank; a batch: its own seed per
rank); no collective on the data path, only the max over ranks of the timed
region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) per launch of the finest-grid forward kernel (k_stream_fwd)
# on the 32 x 1023^2 batch, from an ncu capture of that kernel on this workload; None
# for other workloads and whenever that kernel changes before it is re-captured.
FINE_SWEEP_TRAFFIC_BYTES = 483_135_232
# the e2e measurement of a batch runs it as this many batches on their own streams
E2E_GROUPS = 4

TAU_CALIBRATION = 20000    # default untimed cycles per chain used for tau_int on the device
CPU_SAMPLE_CYCLES = 12     # bounded oracle sample for the CPU baseline (per core)
ESS_TARGET = 1.0e6         # equal-accuracy comparison: QoI mean with standard error 1e-3 of its sd
REF_MAX_STEPS = 60         # cap on timed oracle cycles in the reference arm


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_stream(rank, nch):
    """(seed, chain id) of this rank's chains: the ranks are independent replicas.  One
    chain per rank: seed 2024, Philox chain id = rank; a batch: its chains keep the ids
    0 .. nch - 1 and each rank has its own seed."""
    return (2024, rank) if nch == 1 else (2024 + 7919 * rank, None)


def max_over_ranks(value, dist, device):
    """The largest value of all ranks (the timed region of the slowest rank)."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, units_per_rank, seconds):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return ws * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for_smi(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_chain_seconds(job):
    """One independent oracle chain of the 1023^2 posterior (a spawned worker): seconds
    for n_cycles V-cycles after one untimed cycle, set-up excluded."""
    n_cycles, chain = job
    sys.path.insert(0, ROOT)
    from paper_2407_12149_gb300 import inputs
    import oracle
    p = inputs.config2()
    o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma,
                      y=p.y, qoi_site=p.qoi_site, qoi_w=p.qoi_w)
    x = o.sample(1, 2024, chain=chain, qoi=False)
    t = time.perf_counter()
    o.sample(n_cycles, 2024, x=x, step_offset=1, chain=chain, qoi=False)
    return time.perf_counter() - t


def cpu_baseline(problem, tau_ref):
    """CPU baseline (oracle), not a target: the FP64 CPU oracle on the same workload,
    single-threaded, and with one independent chain per host core on all cores
    (spawned processes; each times its own cycles, set-up excluded; the all-core rate
    is cores x cycles / the slowest core's time)."""
    import multiprocessing
    cores = os.cpu_count() or 1
    t1 = _oracle_chain_seconds((CPU_SAMPLE_CYCLES, 0))
    cps1 = CPU_SAMPLE_CYCLES / t1
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(cores) as pool:
        times = pool.map(_oracle_chain_seconds, [(CPU_SAMPLE_CYCLES, c) for c in range(cores)])
    cps_all = cores * CPU_SAMPLE_CYCLES / max(times)
    return {"value": cps_all / tau_ref, "unit": "QoI ESS/s", "cores": cores, "kind": "oracle",
            "label": "CPU baseline (oracle), not a target", "cpu_model": cpu_model(),
            "single_core_value": cps1 / tau_ref, "v_cycles_per_s_single_core": cps1,
            "v_cycles_per_s_all_cores": cps_all,
            "sample": f"{CPU_SAMPLE_CYCLES} V-cycles of the same 1023^2 problem per chain after 1 untimed cycle, "
                      f"set-up excluded: one chain on one core ({cps1:.3f} V-cycles/s), then one independent chain "
                      f"per core on all {cores} cores ({cps_all:.2f} V-cycles/s); divided by the oracle's own "
                      f"tau_int = {tau_ref:.4f} (oracle/tau_bayes_2d_1023.json)"}


def load_tau_ref():
    path = os.path.join(ROOT, "oracle", "tau_bayes_2d_1023.json")
    with open(path) as f:
        d = json.load(f)
    return float(d["tau"]), d


WORKLOADS = {
    "batch32-bayes2d-1023": {"n": 1023, "chains": 32},   # headline: batched FP32 chains of the 1023^2 posterior
    "bayes2d-1023": {"n": 1023, "chains": 1},
    "bayes2d-1023-fp64": {"n": 1023, "chains": 1, "prec": "fp64"},   # plain FP64 GPU MGMC, first-class line
    "bayes2d-4095": {"n": 4095, "chains": 1},            # HBM-resident single-grid variants (roofline)
    "bayes2d-8191": {"n": 8191, "chains": 1},
    "batch512-mixed": {"n": 511, "chains": 512, "mixed": True},   # 128 chains each of 63^2 .. 511^2
    "bayes3d-127": {"n": 127, "chains": 1, "dim": 3},     # 127^3, kappa^2 = 25, 32 obs, coarsest 3^3
    "warmstart-255": {"n": 255, "chains": 64, "warm": True},       # learned warm start (U-Net), 255^2
    "gibbs-vs-mgmc-2d": {"n": 511, "chains": 1, "table": True},   # Table 1 comparison, 31^2 .. 511^2
    "gibbs-vs-mgmc-2d-q1": {"n": 511, "chains": 1, "table": True, "q1": True},   # Table 1a setting (Q1 elements)
    # Table 1c setting: squared shifted Laplacian (13-point FD), W-cycle, FP64
    "gibbs-vs-mgmc-2d-ssl": {"n": 511, "chains": 1, "table": True, "ssl": True},
    # time per W-cycle of the Table 1c setting, 31^2 .. 511^2 (no IACT): the cost side alone
    "wcycle-ssl-steps": {"n": 511, "chains": 1, "wsteps": True},
    "convergence-2d": {"n": 255, "chains": 512, "conv": True},   # Sec. 5.3: R, Z, rates, RMSE (Q1, 31^2..255^2)
    "tc-gemm-8192": {"n": 8192, "chains": 1, "gemm": True},      # the U-Net's tensor-core GEMM, 8192^3 BF16
}


def run_tc_gemm(args):
    """C = A B^T, A and B 8192 x 8192 BF16, FP32 accumulate and output, on the
    tcgen05 GEMM of the learned warm start (k_tc_gemm): CUDA events per launch."""
    import torch
    from paper_2407_12149_gb300 import build
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    dev = torch.device("cuda", 0)
    n = 8192
    g = torch.Generator(device=dev).manual_seed(1)
    A = torch.randn(n, n, generator=g, device=dev).bfloat16()
    B = torch.randn(n, n, generator=g, device=dev).bfloat16()
    C = torch.empty(n, n, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        M.tc_gemm(A, B, out=C)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(gpu_id_for_smi(torch, 0))
    time.sleep(0.3)
    for a, b in ev:
        a.record()
        M.tc_gemm(A, B, out=C)
        b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    avg = statistics.mean(ms)
    tflops = 2.0 * n ** 3 / (avg * 1e-3) / 1e12
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    # spot check against an FP64 product of the same BF16 values
    rows = torch.arange(0, n, 997, device=dev)
    ref = A[rows].double() @ B.double().T
    err = float(((C[rows].double() - ref).abs().max() / ref.abs().max()).item())
    line = {"metric": "TFLOP/s", "value": tflops, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": avg, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "tc-gemm-8192: C = A B^T, 8192^3, BF16 inputs, FP32 accumulate and output "
                                   "(k_tc_gemm, tcgen05 + TMA + TMEM)", "max_rel_err_vs_fp64": err},
            "roofline": {"bound": "tensor", "kernel": "k_tc_gemm", "achieved": tflops, "peak": peak,
                         "unit": "TFLOP/s", "frac": tflops / peak,
                         "peak_kind": "measured cuBLAS bf16 burst" if peaks else "fallback", "traffic": None},
            "clocks": clk, "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2407_12149_gb300 import inputs
    import oracle
    p = inputs.config2()
    tau_ref, _ = load_tau_ref()
    o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma,
                      y=p.y, qoi_site=p.qoi_site, qoi_w=p.qoi_w)
    x = None
    for w in range(min(args.warmup, 3)):
        x = o.sample(1, 2024, x=x, step_offset=w, qoi=False)
    K = min(args.steps, REF_MAX_STEPS)
    t = time.perf_counter()
    for k in range(K):
        x = o.sample(1, 2024, x=x, step_offset=args.warmup + k, qoi=False)
    dt = time.perf_counter() - t
    cps = K / dt
    val = cps / tau_ref
    line = {"metric": "QoI ESS/s", "value": val, "unit": "QoI ESS/s", "n_gpus": args.gpus, "steps": K,
            "warmup": min(args.warmup, 3), "ms_per_step": 1e3 * dt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "bayes-2d-1023: 1023^2, kappa^2 = 10 exp(g), 16 point obs, Gamma = 1e-4 I, "
                                   "10-grid V(1,1)-cycle, low-rank Gibbs smoother", "v_cycles_per_s": cps,
                       "tau_int": tau_ref},
            "cpu_baseline": {"value": val, "unit": "QoI ESS/s", "cores": 1, "kind": "oracle",
                             "sample": f"{K} of {args.steps} requested V-cycles timed on one host core (FP64 "
                                       f"CPU oracle, set-up excluded); tau_int from oracle/tau_bayes_2d_1023.json"},
            "e2e": {"value": val, "unit": "QoI ESS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def single_problem(inputs, wl):
    """The posterior of a single-chain (or one-posterior batch) workload."""
    return inputs.config3(n=wl["n"]) if wl.get("dim") == 3 else inputs.config2(n=wl["n"])


def make_sampler(M, inputs, wl, precision, local):
    """Sampler (one chain) or BatchSampler (many chains) of a workload."""
    if wl["chains"] == 1:
        p = single_problem(inputs, wl)
        return M.Sampler(p, precision=precision, device=local), [p]
    if wl.get("mixed"):
        ps = [inputs.make_problem(f"mixed-{c}", 2, n, kappa2_seed=c, m=8 + (c % 25), obs_seed=1000 + c,
                                  qoi_cells=max(2, (46 * (n + 1)) // 1024))
              for c, n in enumerate([63, 127, 255, 511] * (wl["chains"] // 4))]
    else:
        p = inputs.config2(n=wl["n"])
        ps = [p] * wl["chains"]
    return M.BatchSampler(ps, precision=precision, device=local), ps


def run_mine(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    from paper_2407_12149_gb300 import build, inputs
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    prec = wl.get("prec", "fp32")
    s, ps = make_sampler(M, inputs, wl, prec, local)
    nch = len(ps)
    batch = nch > 1
    stream = torch.cuda.current_stream()
    sites = sum(p.N for p in ps)
    launches = s.launches_per_cycle()
    # this rank's chains: an independent replica (own seed, or own Philox chain id)
    seed, chain_id = replica_stream(rank, nch)
    xs = s.zeros() if batch else [s.zeros()]

    def cycle(n_steps, offset, qoi=None, resume=False):
        # resume: continue from the states the handle holds (no copy of the chains in or out)
        if batch:
            s.sample(None if resume else xs, n_steps, seed, step_offset=offset, qoi=qoi)
        else:
            s.sample(None if resume else xs[0], n_steps, seed, step_offset=offset, chain=chain_id, qoi=qoi)

    # --- untimed calibration chains: burn-in 100, then tau_int on the device ---
    ncal = args.tau_cycles
    qcal = torch.zeros(nch * (ncal + 100), dtype=torch.float64, device=dev)
    cycle(ncal + 100, 0, qcal)
    taus, errs = [], []
    for c in range(nch):
        st = M.mgmc_qoi_stats(qcal.data_ptr() + 8 * c * (ncal + 100), ncal + 100, 100, 1.5)
        taus.append(st["tau_int"])
        errs.append(st["tau_err"])
    tau = statistics.mean(taus)
    tau_err = (statistics.stdev(taus) / len(taus) ** 0.5) if len(taus) > 1 else errs[0]
    offset = ncal + 100
    # cold-start burn-in of the calibration chains (all from 0): the first cycle at which the
    # chains' mean QoI is within one Monte Carlo standard error of F . mu (FP64 mean solve)
    burn = None
    fmu = None
    if not wl.get("mixed"):
        p0 = single_problem(inputs, wl)
        sm = M.Sampler(p0, precision="fp64", device=local)
        xm = sm.zeros()
        sm.mean_solve(xm, rtol=1e-12, max_cycles=300)
        fmu = float(np.dot(p0.qoi_w, xm.cpu().numpy()[p0.qoi_site]))
        sm.close()
        qm = qcal.view(nch, ncal + 100).cpu().numpy()
        sd = float(np.sqrt(np.mean(qm[:, 100:].var(axis=1))))
        se = sd / np.sqrt(nch)
        trace = qm.mean(axis=0)
        hit = np.nonzero(np.abs(trace - fmu) <= se)[0]
        burn = int(hit[0]) if hit.size else None

    # --- band threshold of the 9-point depths, timed on this handle (autotune) ---
    tuned = None
    if prec == "fp32" and wl.get("dim", 2) == 2:
        from paper_2407_12149_gb300 import autotune
        cands = autotune.band_candidates(ps, 31)
        timer = lambda smp: autotune.time_cycles(smp, cycles=20, warm=3, seed=seed + 7, device=local)  # noqa: E731
        best, tms = autotune.tune_band_min_n(s, cands, timer=timer) if len(cands) > 1 else (0, {})
        bt, tth = autotune.tune_coarse_threads(s, timer=timer)
        cache = autotune.TuneCache()
        cache.put(autotune.cache_key(ps, prec), {"coarse_max_n": 31, "band_min_n": best, "coarse_threads": bt})
        try:
            cache.save()
        except OSError:
            pass
        tuned = {"coarse_max_n": 31, "band_min_n": best, "coarse_threads": bt,
                 "ms_per_cycle_band_min_n": {("tiles only" if k == autotune.TILES_ONLY else str(k)): round(v, 4)
                                             for k, v in tms.items()},
                 "ms_per_cycle_coarse_threads": {("auto" if k == 0 else str(k)): round(v, 4) for k, v in tth.items()},
                 "how": "candidates timed on this handle, 20 back-to-back cycles each (CUDA events), band "
                        "threshold first, then the coarse kernel's threads; the fastest kept and cached"}

    # --- CPU baseline (rank 0, one GPU only), before the GPU timing ------------
    cpu = None
    if rank == 0 and ws == 1 and wl["n"] == 1023 and not wl.get("mixed") and wl.get("dim", 2) == 2:
        try:
            tau_ref, _ = load_tau_ref()
            cpu = cpu_baseline(inputs.config2(), tau_ref)
        except Exception as e:  # report, do not fail the GPU measurement
            cpu = {"value": None, "unit": "QoI ESS/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    # --- device-timed steps ----------------------------------------------------
    M.mgmc_set_profiling(s.h, True)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)    # 256 MB > L2
    qstep = torch.zeros(nch, dtype=torch.float64, device=dev)
    for w in range(args.warmup):
        flush.fill_(float(w))
        cycle(1, offset, qstep, resume=True)
        offset += 1
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_id_for_smi(torch, local))
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fwd_ms, bwd_ms = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        cycle(1, offset, qstep, resume=True)
        ev[k][1].record(stream)
        offset += 1
        f_ms, b_ms = M.mgmc_profile_times(s.h)   # synchronises the stream
        fwd_ms.append(f_ms)
        bwd_ms.append(b_ms)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    if dist:
        dist.barrier()
    cps = job_throughput(ws, nch * args.steps, total_ms / 1e3)   # chain V-cycles per second, whole job
    value = cps / tau

    # --- end-to-end through the public API with pinned host buffers -----------
    # every step: each chain's state host -> device, one V-cycle, device -> host, and the
    # QoI to the host, all inside the library call (mgmc_sample / mgmc_sample_batch with
    # host buffers, which synchronise).  A batch runs as E2E_GROUPS batch handles, each on
    # its own stream and driven from its own host thread, so that one group's copies
    # overlap the others' cycles; each group has its own seed (independent Philox streams)
    M.mgmc_set_profiling(s.h, False)
    for c, x in enumerate(xs):                      # the chains' current states
        if batch:
            s.get_state(c, x)
        else:
            s.get_state(x)
    xh = [x.cpu().pin_memory() for x in xs]
    groups = []
    if batch:
        ng = E2E_GROUPS if nch % E2E_GROUPS == 0 and nch >= 2 * E2E_GROUPS else 1
        gsz = nch // ng
        for g in range(ng):
            part = ps[g * gsz:(g + 1) * gsz]
            sg = s if ng == 1 else M.BatchSampler(part, precision=prec, device=local,
                                                  band_min_n=tuned["band_min_n"] if tuned else None,
                                                  coarse_threads=tuned["coarse_threads"] if tuned else None)
            groups.append({"s": sg, "stream": torch.cuda.Stream(device=dev) if ng > 1 else stream,
                           "host": xh[g * gsz:(g + 1) * gsz],
                           "qh": torch.zeros(gsz, dtype=torch.float64).pin_memory(),
                           "seed": seed + (104729 * g if ng > 1 else 0)})
    qh1 = torch.zeros(1, dtype=torch.float64).pin_memory()
    n_e2e = max(3, min(args.steps, 100))
    for G in groups:          # untimed first call of each group handle (graph capture)
        G["s"].sample(G["host"], 1, G["seed"], step_offset=offset, qoi=G["qh"], stream=G["stream"])
    offset += 1
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    def drive(G, first):
        for k in range(n_e2e):
            G["s"].sample(G["host"], 1, G["seed"], step_offset=first + k, qoi=G["qh"], stream=G["stream"])

    t0 = time.perf_counter()
    if batch:
        import threading
        th = [threading.Thread(target=drive, args=(G, offset)) for G in groups]
        for t in th:
            t.start()
        for t in th:
            t.join()
    else:
        for k in range(n_e2e):
            s.sample(xh[0], 1, seed, step_offset=offset + k, chain=chain_id, qoi=qh1)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    offset += n_e2e
    e2e_value = job_throughput(ws, nch * n_e2e, e2e_s) / tau

    # --- plain FP64 single-chain GPU MGMC on the same posterior, the same protocol ---
    plain = None
    if rank == 0 and not wl.get("mixed") and wl["n"] <= 1023 and wl.get("dim", 2) == 2 and prec == "fp32":
        s64 = M.Sampler(single_problem(inputs, wl), precision="fp64", device=local)
        x64 = s64.zeros()
        q64 = torch.zeros(ncal + 100, dtype=torch.float64, device=dev)
        s64.sample(x64, ncal + 100, seed + 1, qoi=q64)                 # its own tau, from 0
        st64 = M.mgmc_qoi_stats(q64.data_ptr(), ncal + 100, 100, 1.5)
        off64 = ncal + 100
        for w in range(args.warmup):
            flush.fill_(float(w))
            s64.sample(None, 1, seed + 1, step_offset=off64)
            off64 += 1
        torch.cuda.synchronize()
        ms64 = []
        for k in range(min(args.steps, 200)):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s64.sample(None, 1, seed + 1, step_offset=off64)
            e1.record(stream)
            off64 += 1
            torch.cuda.synchronize()
            ms64.append(e0.elapsed_time(e1))
        cps64 = 1e3 / statistics.mean(ms64)
        tau64 = st64["tau_int"]
        plain = {"v_cycles_per_s": cps64, "ess_per_s": cps64 / tau64, "tau_int": tau64, "tau_err": st64["tau_err"],
                 "tau_cycles": ncal, "ms_per_step": statistics.mean(ms64),
                 "note": "plain FP64 GPU MGMC, one chain, same posterior, the same protocol as the headline "
                         "(state resident, 256 MB L2 flush between steps, CUDA events); its own tau_int from a "
                         f"{ncal}-cycle chain"}
        if burn is not None:
            # equal accuracy: the QoI mean to a standard error of 1e-3 of its sd needs ESS_TARGET
            # effective samples; wall time including the cold-start burn-in (the same burn-in for
            # both: the same law from the same start)
            t_plain = (burn + ESS_TARGET * tau64) / cps64
            t_batch = (burn + ESS_TARGET * tau / nch) * (total_ms / args.steps) / 1e3
            plain["equal_accuracy"] = {"target_ess": ESS_TARGET, "burn_in_cycles": burn,
                                       "seconds_plain_fp64": t_plain, "seconds_batched_fp32": t_batch,
                                       "multiple": t_plain / t_batch}
        s64.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peak()
    fine_sites = sum(p.N for p in ps if p.n > 31)
    fwd_avg = statistics.mean(fwd_ms)
    if wl.get("dim") == 3:
        # the timed region is the finest grid's forward sweep (two red-black colour launches); with constant
        # kappa^2 the sweep must read and write theta (4 + 4 B/site) -- the kernel also reads the
        # s*kappa^2 field (4 B/site), which the algorithmic figure does not count
        sweep_bytes = 8 * fine_sites
        kernel = "k_sweep_colour<float,3>: finest-grid forward Gibbs sweep (two red-black colour launches)"
    else:
        # algorithmic bytes of the depth-0 forward launch (every chain's finest grid), FP32: read theta
        # and s*kappa^2 (4 + 4 B/site), write theta*_s (4 B/site) and the restricted residual (4 B per
        # coarse site = 1 B per fine site); the noise is generated, never stored
        sweep_bytes = 13 * fine_sites
        kernel = "k_stream_fwd: finest-grid forward Gibbs sweep + residual + restriction, all chains"
        if prec == "fp64":
            # FP64: read theta and a_ii (8 + 8 B/site), write theta*_s (8) and the restricted residual (2)
            sweep_bytes = 26 * fine_sites
            kernel = "k_tile_batch<double,1,0>: finest-grid forward Gibbs sweep + residual + restriction (FP64)"
    achieved = sweep_bytes / (fwd_avg * 1e-3) / 1e9
    if wl.get("dim") == 3:
        desc = (f"{ps[0].n}^3 Bayesian posterior: kappa^2 = 25, 32 point obs, Gamma = 1e-4 I, "
                f"{ps[0].n_levels}-grid V(1,1)-cycle, coarsest 3^3, low-rank Gibbs smoother")
    else:
        desc = ("32 independent chains of " if batch and not wl.get("mixed") else "") + \
            (f"{nch} chains, grids 63^2..511^2 (128 x 4 sizes), own kappa^2 and 8-32 obs" if wl.get("mixed") else
             f"{ps[0].n}^2 Bayesian posterior: kappa^2 = 10 exp(g), 16 point obs, Gamma = 1e-4 I, "
             f"{ps[0].n_levels}-grid V(1,1)-cycle, low-rank Gibbs smoother")
    line = {
        "metric": "QoI ESS/s", "value": value, "unit": "QoI ESS/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}; " + ("FP32 sweeps, FP64 low-rank/coarsest/QoI"
                                                                if prec == "fp32" else "FP64 throughout (plain MGMC)"),
                   "chains_per_gpu": nch, "sites_per_gpu": sites,
                   "v_cycles_per_s": cps, "site_updates_per_s": cps * sites / nch * 2,
                   "tau_int": tau, "tau_err": tau_err, "burn_in_cycles_from_0": burn, "qoi_posterior_mean": fmu,
                   "tau_from": f"device Wolff estimates of {nch} untimed {ncal}-cycle chains (mean)",
                   "l2": "256 MB buffer written between timed steps",
                   "step": "one V-cycle of every chain, states resident on the device (mgmc_sample[_batch] "
                           "with x = NULL); e2e copies them in and out through host memory every step",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "launches_per_cycle": launches,
                   "tuned": tuned,
                   "plain_fp64_single_chain": plain,
                   "burn_in_rule": "first cycle at which the mean QoI of the chains (all from 0) is within one "
                                   "Monte Carlo standard error of F . mu from the FP64 mean solve"},
        "roofline": {"bound": "hbm",
                     "kernel": kernel,
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "traffic": FINE_SWEEP_TRAFFIC_BYTES if args.workload == "batch32-bayes2d-1023" else None,
                     "algorithmic_bytes": sweep_bytes, "avg_ms": fwd_avg,
                     "bwd_sweep_avg_ms": statistics.mean(bwd_ms)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "QoI ESS/s", "h2d_bytes_per_step": (4 if prec == "fp32" else 8) * sites,
                "d2h_bytes_per_step": (4 if prec == "fp32" else 8) * sites + 8 * nch,
                "note": (f"mgmc_sample_batch with pinned host buffers (copies inside the call, one per chain and "
                         f"direction): {len(groups)} batch handles of {nch // max(len(groups), 1)} chains, each on "
                         "its own stream and host thread") if batch else
                        "mgmc_sample with pinned host buffers (copies inside the call)"},
        "gpu_launches": args.steps * (launches + 1),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def warm_problems(n, count, first):
    """Seeded 255^2-type problems of the learned warm start: kappa^2 = 10 exp(g) (own
    seed each), m ~ U{8..32} uniform point observations, Gamma = 1e-4 I, central QoI."""
    import numpy as np
    from paper_2407_12149_gb300 import inputs
    out = []
    for s in range(first, first + count):
        m = int(np.random.default_rng(30000 + s).integers(8, 33))
        out.append(inputs.make_problem(f"warm-{s}", 2, n, kappa2_seed=10000 + s, m=m, obs_seed=20000 + s,
                                       qoi_cells=max(2, (46 * (n + 1)) // 1024)))
    return out


def burn_in(q, qmu, sig):
    """Cycles until the chains' mean normalised QoI error is within one Monte Carlo
    standard error: first t with |mean_k (q[k,t] - qmu[k]) / sig[k]| <= 1 / sqrt(chains)."""
    import numpy as np
    d = ((q - qmu[:, None]) / sig[:, None]).mean(axis=0)
    ok = np.abs(d) <= 1.0 / np.sqrt(q.shape[0])
    return int(np.argmax(ok)) if ok.any() else q.shape[1], d


def run_warmstart(args):
    """Learned warm start (255^2): U-Net trained on FP64 mean-solve targets, then
    burn-in of held-out FP32 chains started from the U-Net estimate vs from 0."""
    import numpy as np
    import torch
    from paper_2407_12149_gb300 import build
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    dev = torch.device("cuda", 0)
    n, n_test = 255, args.warm_test
    curve = sorted({int(v) for v in args.warm_curve.split(",") if v.strip()}) if args.warm_curve else []
    n_train = max(curve) if curve else args.warm_train
    t0 = time.perf_counter()
    train = warm_problems(n, n_train, 0)
    test = warm_problems(n, n_test, 1_000_000)

    def targets(ps):
        T = torch.zeros(len(ps), n * n, dtype=torch.float64, device=dev)
        for k, p in enumerate(ps):
            s = M.Sampler(p, precision="fp64", coarse_max_n=31)
            s.mean_solve(T[k], rtol=1e-10, max_cycles=100)
            s.close()
        return T

    Xtr = torch.from_numpy(np.stack([M.unet_inputs(p) for p in train]).view(np.int16)).to(dev)
    Xte = torch.from_numpy(np.stack([M.unet_inputs(p) for p in test]).view(np.int16)).to(dev)
    Ttr = targets(train).float()
    Tte = targets(test)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    def train_net(count):
        net = M.Unet(n, c0=32, max_batch=8, seed=1)
        t1 = time.perf_counter()
        losses = net.train(Xtr[:count], Ttr[:count], epochs=args.warm_epochs, batch=8, lr=1e-3, shuffle_seed=2)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mu_hat = net.predict(Xte, precision="fp32")
        e1.record()
        torch.cuda.synchronize()
        pred_ms = e0.elapsed_time(e1)
        net_params = net.n_params
        net.close()
        return mu_hat, losses, train_s, pred_ms, net_params

    # chains of the held-out problems from 0 and from the estimates, FP32 batched
    K = args.warm_cycles
    b = M.BatchSampler(test, precision="fp32")
    xs = b.zeros()

    def chains(init):
        for k, x in enumerate(xs):
            if init is None:
                x.zero_()
            else:
                x.copy_(init[k])
        q = torch.zeros(n_test * K, dtype=torch.float64, device=dev)
        b.sample(xs, K, 77, qoi=q)
        torch.cuda.synchronize()
        return q.view(n_test, K).cpu().numpy()

    runs = {"zero": chains(None)}
    points = []
    for count in (curve or [n_train]):
        mu_hat, losses, train_s, pred_ms, n_params = train_net(count)
        err = (mu_hat.double() - Tte).norm(dim=1) / Tte.norm(dim=1)
        runs[count] = chains(mu_hat)
        points.append({"train_problems": count, "mu_rel_l2_error_mean": float(err.mean()),
                       "mu_rel_l2_error_max": float(err.max()), "train_s": train_s,
                       "train_loss_first_last": [float(losses[0]), float(losses[-1])]})
    b.close()

    qmu = np.array([float(np.dot(p.qoi_w, Tte[k].cpu().numpy()[p.qoi_site])) for k, p in enumerate(test)])
    tail = np.concatenate([r[:, K // 2:] for r in runs.values()], axis=1)
    sig = tail.std(axis=1, ddof=1)
    b_zero, d_zero = burn_in(runs["zero"], qmu, sig)
    for pt in points:
        pt["burn_in_cycles"] = burn_in(runs[pt["train_problems"]], qmu, sig)[0]
    b_unet, d_unet = burn_in(runs[n_train], qmu, sig)
    err_mean, err_max = points[-1]["mu_rel_l2_error_mean"], points[-1]["mu_rel_l2_error_max"]
    losses = points[-1]["train_loss_first_last"]
    train_s = points[-1]["train_s"]

    # tensor-core roofline of the GEMM on the largest convolution shapes of a batch of 8
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))

    def gemm_tflops(Mr, N, Kd, reps=10):
        g = torch.Generator(device=dev).manual_seed(1)
        A = torch.randn(Mr, Kd, generator=g, device=dev).bfloat16()
        B = torch.randn(N, Kd, generator=g, device=dev).bfloat16()
        C = torch.empty(Mr, N, dtype=torch.float32, device=dev)
        for _ in range(3):
            M.tc_gemm(A, B, out=C)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            M.tc_gemm(A, B, out=C)
        b2.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b2) / reps
        return 2.0 * Mr * N * Kd / (ms * 1e-3) / 1e12, ms

    bott, bott_ms = gemm_tflops(64 * 32 * 32, 256, 2304)     # bottom-level convolution of 64 samples
    big, big_ms = gemm_tflops(8192, 8192, 8192, reps=5)
    line = {
        "metric": "burn-in V-cycles (learned warm start)", "value": b_unet, "unit": "V-cycles",
        "n_gpus": 1, "steps": K, "warmup": 0, "ms_per_step": None, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"warmstart-255: U-Net (c0 = 32, {n_params} parameters) trained on {n_train} "
                               f"FP64 mean-solve targets of seeded 255^2 posteriors (kappa^2 = 10 exp(g), m ~ U{{8..32}}, "
                               f"Gamma = 1e-4 I), {n_test} held-out problems, FP32 batched chains",
                   "burn_in_from_zero": b_zero, "burn_in_from_unet": b_unet,
                   "burn_in_rule": f"first cycle with |mean_k (q_kt - F mu_k) / sd_k| <= 1 / sqrt({n_test})",
                   "mean_error_trace_zero": [round(float(v), 3) for v in d_zero[:12]],
                   "mean_error_trace_unet": [round(float(v), 3) for v in d_unet[:12]],
                   "mu_rel_l2_error_mean": err_mean, "mu_rel_l2_error_max": err_max,
                   "train_epochs": args.warm_epochs, "train_loss_first_last": losses,
                   "train_s": train_s, "data_generation_s": gen_s,
                   "predict_ms_per_problem": pred_ms / n_test,
                   "learning_curve": points if curve else None},
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm<256>: bottom-level convolution GEMM of 64 samples "
                                                  "(M = 64 x 32^2 pixels, N = 256, K = 9 x 256)",
                     "achieved": bott, "peak": peak, "unit": "TFLOP/s", "frac": bott / peak,
                     "peak_kind": "measured cuBLAS bf16 burst" if peaks else "fallback",
                     "avg_ms": bott_ms, "square_8192_tflops": big, "traffic": None},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def run_gibbs_table(args):
    """The comparison of the paper's Table 1 (Sec. 5.2; samplers of Sec. 5.1.3) on the 2D posterior of the headline
    workload (kappa^2 = 10 exp(g), 16 point observations), FP32, one chain per sampler and
    grid: IACT of the QoI (device Wolff estimate after a burn-in), time per step (CUDA
    events over back-to-back steps, state resident) and time per independent sample for
    the plain Gibbs sampler (one symmetric low-rank Gibbs sweep per step) and MGMC
    (V(1,1)-cycle); the exact Cholesky sampler (single-grid hierarchy, FP64) on 31^2.  The
    squared-operator form (Table 1c) runs FP64 with MGMC's W-cycle."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2407_12149_gb300 import build, inputs
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(gpu_id_for_smi(torch, local))

    def measure(s, n_chain, burn, n_time):
        x = s.zeros()
        q = torch.zeros(n_chain + burn, dtype=torch.float64, device=dev)
        s.sample(x, n_chain + burn, 2024, qoi=q)
        torch.cuda.synchronize()
        st = M.mgmc_qoi_stats(q.data_ptr(), n_chain + burn, burn, 1.5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.sample(None, 5, 2024, step_offset=n_chain + burn)
        e0.record(stream)
        s.sample(None, n_time, 2024, step_offset=n_chain + burn + 5)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n_time
        return st["tau_int"], st["tau_err"], ms

    q1 = bool(WORKLOADS[args.workload].get("q1"))
    ssl = bool(WORKLOADS[args.workload].get("ssl"))
    make = inputs.table1c if ssl else (inputs.table1a if q1 else inputs.config2)
    prec = "fp64" if ssl else "fp32"
    rows = []
    for n in (31, 63, 127, 255, 511):
        p = make(n=n)
        row = {"n": n}
        # Gibbs: tau grows like h^-2 (about 100 at 31^2 for kappa^2 = 10); chains of up to 400 000 steps
        # (the squared operator: up to 200 000, its Gibbs tau cannot be estimated reliably on the fine grids)
        n_g = min(200000 if ssl else 400000, 20000 * ((n + 1) // 32) ** 2)
        s = M.Sampler(p, precision=prec, gibbs=True, device=local)
        tg, eg, msg = measure(s, n_g, 2000, 200)
        s.close()
        s = M.Sampler(p, precision=prec, device=local)
        tm, em, msm = measure(s, 3000 if ssl else 5000, 100, 50 if ssl else 200)
        row["launches_per_cycle_mgmc"] = s.launches_per_cycle()
        s.close()
        row.update({"gibbs_steps": n_g, "tau_gibbs": tg, "tau_gibbs_err": eg, "ms_per_step_gibbs": msg,
                    "ms_per_indep_gibbs": msg * tg, "tau_mgmc": tm, "tau_mgmc_err": em, "ms_per_step_mgmc": msm,
                    "ms_per_indep_mgmc": msm * tm})
        if n == 31:
            pc = make(n=31, n_levels=1)
            s = M.Sampler(pc, precision="fp64", device=local)
            x = s.zeros()
            s.sample(x, 5, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.sample(None, 50, 1, step_offset=5)
            e1.record(stream)
            torch.cuda.synchronize()
            row["ms_per_sample_cholesky"] = e0.elapsed_time(e1) / 50
            s.close()
        rows.append(row)
    clk = clocks.stop()
    big = rows[-1]
    line = {
        "metric": "time per independent QoI sample (MGMC, 511^2)", "value": big["ms_per_indep_mgmc"], "unit": "ms",
        "n_gpus": 1, "steps": 200, "warmup": 5, "ms_per_step": big["ms_per_step_mgmc"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if ssl else "f32", "data": "synthetic",
        "config": {"workload": (("gibbs-vs-mgmc-2d-ssl: the Table 1c setting (squared shifted Laplacian, 13-point "
                                 "finite differences with u = du/dn = 0, kappa^-1 = 0.1, 8 ball obs, Gamma diagonal "
                                 "in [1e-6, 2e-6]), MGMC W-cycle") if ssl else
                                ("gibbs-vs-mgmc-2d-q1: the Table 1a setting (Q1 finite elements, kappa^-1 = 0.1, "
                                 "8 point obs, Gamma diagonal in [1e-6, 2e-6])") if q1 else
                                ("gibbs-vs-mgmc-2d: the Sec. 5.2 / Table 1 comparison on the 2D posterior "
                                 "(kappa^2 = 10 exp(g), 16 point obs, Gamma = 1e-4 I)")) +
                               f", 31^2 .. 511^2, one {prec.upper()} chain per sampler and grid; Cholesky = "
                               "single-grid exact sampler (FP64, one CTA)",
                   "table": rows,
                   "tau_from": "device Wolff estimate (S = 1.5) of each chain after its burn-in (Gibbs 2000, MGMC 100)",
                   "timing": ("CUDA events over 200 (Gibbs) / 50 (MGMC) back-to-back steps" if ssl else
                              "CUDA events over 200 back-to-back steps") +
                             ", state resident (grids up to 511^2 are L2-resident)",
                   "paper_table": ("Table 1c (sequential C++ on a Xeon 8168): MGMC 0.36 .. 110.39 ms per sample, "
                                   "IACT 2.22 .. 3.94, 0.81 .. 435.17 ms per independent sample (32^2 .. 512^2 "
                                   "cells)") if ssl else None},
        "roofline": None, "cpu_baseline": None, "e2e": None,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_wcycle_steps(args):
    """Time per MGMC W(1,1)-cycle of the Table 1c setting (squared shifted Laplacian,
    13-point finite differences, FP64, one chain) on 31^2 .. 511^2: CUDA events over
    --steps back-to-back cycles after --warmup, state resident, the small grids in the
    one-CTA kernel (default) and with one launch per phase (coarse_max_n = 1)."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2407_12149_gb300 import build, inputs
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(gpu_id_for_smi(torch, local))
    rows = []
    for n in (31, 63, 127, 255, 511):
        p = inputs.table1c(n)
        row = {"n": n}
        for key, cmax in (("small_kernel", 0), ("per_phase_launches", 1)):
            s = M.Sampler(p, precision="fp64", coarse_max_n=cmax, device=local)
            x = s.zeros()
            s.sample(x, args.warmup, 7)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.sample(None, args.steps, 7, step_offset=args.warmup)
            e1.record(stream)
            torch.cuda.synchronize()
            row[f"ms_per_cycle_{key}"] = e0.elapsed_time(e1) / args.steps
            row[f"launches_{key}"] = s.launches_per_cycle()
            s.close()
        rows.append(row)
    clk = clocks.stop()
    big = rows[-1]
    line = {
        "metric": "ms per W-cycle step (Table 1c setting, 511^2)", "value": big["ms_per_cycle_small_kernel"],
        "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": big["ms_per_cycle_small_kernel"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "wcycle-ssl-steps: squared shifted Laplacian (13-point FD, u = du/dn = 0), "
                               "kappa^-1 = 0.1, 8 ball obs, W(1,1)-cycle, FP64, one chain, 31^2 .. 511^2",
                   "table": rows, "timing": "CUDA events over back-to-back cycles, state resident (L2)"},
        "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_convergence(args):
    """The experiments of Sec. 5.3 on the Table 1a posterior (Q1 elements, kappa^-1 = 0.1,
    8 point observations), FP32: many independent chains from theta^(0) = 0 -- MGMC as
    batches of 512 chains (one seed per batch: independent Philox streams), the plain
    Gibbs sampler one chain per call -- give R^(m), Z^(m) over the first 16 steps and
    the rates rho, zeta (Sec. 5.3.1), and 100 chains per sampler the RMSE Delta^(M) of
    the running QoI mean (Sec. 5.3.3).  Exact mu_L, sigma_L^2 by a sparse direct solve."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2407_12149_gb300 import build, experiments as E, inputs
    from paper_2407_12149_gb300 import mgmc as M
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    clocks = ClockSampler(gpu_id_for_smi(torch, local))
    steps, B = 16, 512
    n_batches = max(1, args.conv_chains // B)
    M_values = [2 ** k for k in range(13)]          # 1 .. 4096
    rows = []
    t_start = time.perf_counter()
    for n in (31, 63, 127, 255):
        p = inputs.table1a(n)
        mu, s2 = E.exact_qoi_moments(p)
        # MGMC: batches of B chains, each batch its own seed
        bs = M.BatchSampler([p] * B, precision="fp32", device=local)
        z = []
        for k in range(n_batches):
            xs = bs.zeros()
            q = torch.zeros(B * steps, dtype=torch.float64, device=dev)
            bs.sample(xs, steps, 1000 + k, qoi=q)
            z.append(q.view(B, steps).cpu().numpy())
        zm = np.concatenate(z)
        zm = np.concatenate([np.zeros((zm.shape[0], 1)), zm], axis=1)     # step 0: F . 0
        # RMSE: 100 MGMC chains of 4096 steps from 0
        b100 = M.BatchSampler([p] * 100, precision="fp32", device=local)
        q = torch.zeros(100 * 4096, dtype=torch.float64, device=dev)
        b100.sample(b100.zeros(), 4096, 7, qoi=q)
        zr_m = np.concatenate([np.zeros((100, 1)), q.view(100, 4096).cpu().numpy()[:, :-1]], axis=1)
        b100.close()
        bs.close()
        # Gibbs: one chain per call (batches run the V-cycle only)
        sg = M.Sampler(p, precision="fp32", gibbs=True, device=local)
        ng = args.conv_gibbs_chains
        qg = torch.zeros(ng * steps, dtype=torch.float64, device=dev)
        for c in range(ng):
            sg.sample(sg.zeros(), steps, 2000 + c // 65536, chain=c % 65536, qoi=qg[c * steps:(c + 1) * steps])
        zg = np.concatenate([np.zeros((ng, 1)), qg.view(ng, steps).cpu().numpy()], axis=1)
        qr = torch.zeros(100 * 4096, dtype=torch.float64, device=dev)
        for c in range(100):
            sg.sample(sg.zeros(), 4096, 3000, chain=c, qoi=qr[c * 4096:(c + 1) * 4096])
        zr_g = np.concatenate([np.zeros((100, 1)), qr.view(100, 4096).cpu().numpy()[:, :-1]], axis=1)
        sg.close()
        row = {"n": n, "mu_L": mu, "sigma2_L": s2, "chains_mgmc": zm.shape[0], "chains_gibbs": ng}
        for name, zz in (("mgmc", zm), ("gibbs", zg)):
            r = E.convergence_ratios(zz, mu, s2)
            rho, mr = E.rate(r["R"], r["R_err"])
            zeta, mz = E.rate(r["Z"], r["Z_err"])
            row[name] = {"R": r["R"].tolist(), "R_err": r["R_err"].tolist(), "Z": r["Z"].tolist(),
                         "Z_err": r["Z_err"].tolist(), "rho": rho, "m_star_rho": mr, "zeta": zeta, "m_star_zeta": mz}
        row["rmse_M"] = M_values
        row["rmse_mgmc"] = E.rmse(zr_m, mu, M_values).tolist()
        row["rmse_gibbs"] = E.rmse(zr_g, mu, M_values).tolist()
        rows.append(row)
    clk = clocks.stop()
    line = {
        "metric": "MGMC convergence rate of the QoI mean (rho, 127^2)", "value": rows[2]["mgmc"]["rho"], "unit": "1",
        "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "convergence-2d: Sec. 5.3 on the Table 1a posterior (Q1, kappa^-1 = 0.1, 8 point obs, "
                               "Gamma diagonal in [1e-6, 2e-6]), 31^2 .. 255^2; MGMC chains in batches of 512 "
                               f"({n_batches} seeds), Gibbs one chain per call; all chains from theta^(0) = 0",
                   "table": rows, "wall_s": time.perf_counter() - t_start,
                   "estimators": "R, Z of Eq. convergence_rate_definition with sample mean / variance over the "
                                 "chains; rho, zeta at the last step whose statistical error is <= 10 %; RMSE of "
                                 "the running mean of the first M QoI values (steps 0 .. M-1) over 100 chains"},
        "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="batch32-bayes2d-1023", choices=sorted(WORKLOADS),
                    help="batch32-bayes2d-1023 (headline): 32 FP32 chains of the 1023^2 posterior; bayes2d-1023: "
                         "one chain; bayes2d-4095/8191: HBM-resident single grids; batch512-mixed: 512 chains")
    ap.add_argument("--tau-cycles", type=int, default=TAU_CALIBRATION,
                    help="length of the untimed chain that estimates tau_int (>= 200)")
    ap.add_argument("--warm-train", type=int, default=1024, help="warmstart-255: training problems")
    ap.add_argument("--warm-epochs", type=int, default=20, help="warmstart-255: training epochs")
    ap.add_argument("--warm-cycles", type=int, default=40, help="warmstart-255: chain length of the burn-in test")
    ap.add_argument("--warm-test", type=int, default=512, help="warmstart-255: held-out problems")
    ap.add_argument("--warm-curve", default="", help="warmstart-255: comma-separated training-set sizes; each trains "
                                                     "a fresh network on the first N problems (learning curve)")
    ap.add_argument("--conv-chains", type=int, default=16384, help="convergence-2d: MGMC chains per grid")
    ap.add_argument("--conv-gibbs-chains", type=int, default=2048, help="convergence-2d: Gibbs chains per grid")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.tau_cycles = max(200, args.tau_cycles)
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload].get("warm"):
        run_warmstart(args)
    elif WORKLOADS[args.workload].get("table"):
        run_gibbs_table(args)
    elif WORKLOADS[args.workload].get("wsteps"):
        run_wcycle_steps(args)
    elif WORKLOADS[args.workload].get("conv"):
        run_convergence(args)
    elif WORKLOADS[args.workload].get("gemm"):
        run_tc_gemm(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()

"""Integrated autocorrelation time of the 1023^2 Bayesian workload, from the oracle alone.

Runs the FP64 CPU oracle for 2000 V-cycles (seed 2024, x0 = 0), drops 100
cycles of burn-in and stores Wolff's estimate (tau, error, window) in
oracle/tau_bayes_2d_1023.json.  The benchmark's CPU reference arm divides the
oracle's V-cycles/s by this tau to report QoI ESS/s; nothing here comes from
the CUDA path.

    python oracle/calibrate_tau.py [n_cycles]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2407_12149_gb300 import inputs  # noqa: E402


def main():
    n_cycles = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    p = inputs.config2()
    o = oracle.Oracle(p.dim, p.n, p.n_levels, kappa2=p.kappa2, obs_site=p.obs_site, obs_w=p.obs_w, Gamma=p.Gamma,
                      y=p.y, qoi_site=p.qoi_site, qoi_w=p.qoi_w)
    t = time.time()
    x, q = o.sample(n_cycles, 2024)
    dt = time.time() - t
    st = oracle.chain_stats(q[100:])
    out = {"workload": p.name, "n_cycles": n_cycles, "burn_in": 100, "seed": 2024, "tau": st["tau"],
           "tau_err": st["tau_err"], "window": st["window"], "qoi_mean": st["mean"], "qoi_var": st["var"],
           "oracle_s_per_cycle": dt / n_cycles}
    with open(os.path.join(HERE, "tau_bayes_2d_1023.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

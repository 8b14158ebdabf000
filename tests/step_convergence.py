"""RK4 step-count convergence on the cosmological boxes: trace the same bundles
with N, 2N, 4N, ... uniform steps (Sec. 4.1: the step is a fixed fraction of a
resolution length) and report max and 99th-percentile |d mu / mu| between
successive step counts, stopping at the first N whose change is below the
parity gate (1e-4) or at the last N of the ladder.

    python tests/step_convergence.py [--box c5|c3] [--bundles 256] [--n0 125] [--nmax 4000]

Needs a GPU (CUDA library, mixed precision); prints one markdown table.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--box", default="c5", choices=("c3", "c5"))
    ap.add_argument("--bundles", type=int, default=256)
    ap.add_argument("--n0", type=int, default=125)
    ap.add_argument("--nmax", type=int, default=4000)
    ap.add_argument("--gate", type=float, default=1e-4)
    args = ap.parse_args()
    import paper_1110_4894_gb300 as P
    cfg = (inputs.config_c5 if args.box == "c5" else inputs.config_c3)(n_steps=args.n0)
    theta = cfg["theta"][:args.bundles]  # a contiguous patch of the bundle grid
    ctx = P.Context(0, precision=P.MIXED, autotune=1)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                       rot=cfg["rot"], shift=cfg["shift"], mean_subtract=True)
    print("| box | bundles | N | step (Mpc) | trace (s) | max \\|μ_N/μ_N/2 − 1\\| | p99 | mean μ |")
    print("|---|---|---|---|---|---|---|---|")
    prev, n, chosen = None, args.n0, None
    while n <= args.nmax:
        t0 = time.time()
        r = ctx.trace(0, cfg["z_s"], theta, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0, n_steps=n)
        dt = time.time() - t0
        assert np.all(r["flags"] & (P.F_NOCROSS | P.F_NONFINITE) == 0)
        _, chi_s = ctx.schedule(cfg["z_s"], 0, n)
        if prev is None:
            d = None
        else:
            d = np.abs(r["mu"] / prev - 1)
        print("| %s | %d | %d | %.3f | %.1f | %s | %s | %.6f |" % (
            args.box, len(theta), n, chi_s / n, dt, "—" if d is None else "%.2e" % d.max(),
            "—" if d is None else "%.2e" % np.percentile(d, 99), np.mean(r["mu"])), flush=True)
        if d is not None and d.max() < args.gate and chosen is None:
            chosen = n
            break
        prev, n = r["mu"], 2 * n
    print()
    print("converged step count: %s" % (chosen if chosen else "not reached by N = %d" % args.nmax))


if __name__ == "__main__":
    main()

"""Minimum-reliable-radius sweep of the grid path against the direct sum
(Sec. 4.2, Figs. nfwtests1-2): bundles at impact parameters log-spaced in
[0.05, 2] r200 around the NFW halo of the NFW workload (100 000 particles,
5 kpc softening), traced with the direct sum and through node grids of
24 and 49 h^-1 kpc spacing with n_int = 1 and 2.  Each method's magnification
is compared with the analytic truncated NFW lens in 8 radial bins; the MRR is
the smallest bin edge outside which every bin's mean |dmu/mu| is below 3 %.

    python tests/grid_sweep.py [--bundles-per-bin 48]

Needs a GPU; prints one markdown table.
"""
import argparse
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bundles-per-bin", type=int, default=48)
    ap.add_argument("--bins", type=int, default=8)
    args = ap.parse_args()
    import oracle
    import oracle.analytic as A
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_c2()
    om, ol, h = cfg["cosmo"]
    cosmo = oracle.Cosmology(om, ol, h)
    L = A.NFWLens(cosmo, 1e14, 5.0, cfg["z_l"], cfg["z_s"])
    D_d = L.D_d
    g = np.random.default_rng(2024)
    edges = np.logspace(math.log10(0.05), math.log10(2.0), args.bins + 1)
    nb = args.bundles_per_bin
    x = np.concatenate([np.exp(g.uniform(math.log(edges[i]), math.log(edges[i + 1]), nb)) for i in range(args.bins)])
    phi = g.uniform(0, 2 * math.pi, x.size)
    theta = np.stack([x * L.r200 / D_d * np.cos(phi), x * L.r200 / D_d * np.sin(phi)], 1)
    mu_an = np.array([L.lens_trunc(t)[2] for t in x * L.r200 / D_d])
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
              lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    r200c = cfg["info"]["r200_phys"] * (1 + cfg["z_l"])
    half = 2.2 * r200c
    methods = [("direct sum", None, None)]
    for spacing_hkpc in (24.0, 49.0):
        for n_int in (1, 2):
            methods.append(("grid %g h^-1 kpc, n_int %d" % (spacing_hkpc, n_int), spacing_hkpc, n_int))
    rows = []
    for label, spacing, n_int in methods:
        ctx = P.Context(0, precision=P.MIXED, autotune=1)
        ctx.set_cosmology(om, ol, h)
        t0 = time.time()
        if spacing is None:
            ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
            n = None
        else:
            hh = spacing / 1000.0 / h
            n = int(math.ceil(2 * half / hh)) + 1
            lo = [-half, -half, cfg["chi_l"] - half]
            ctx.load_grid(0, cfg["pos"], cfg["mass"], cfg["soft"], lo, hh, n, n_int=n_int)
        r = ctx.trace(0, cfg["z_s"], theta, **kw)
        dt = time.time() - t0
        err = np.abs(r["mu"] / mu_an - 1)
        per_bin = [float(np.mean(err[i * nb:(i + 1) * nb])) for i in range(args.bins)]
        mrr = None
        for i in range(args.bins - 1, -1, -1):
            if per_bin[i] < 0.03:
                mrr = edges[i]
            else:
                break
        rows.append((label, n, dt, per_bin, mrr))
        ctx.close()
    head = " | ".join("%.3g–%.3g" % (edges[i], edges[i + 1]) for i in range(args.bins))
    print("| method | nodes/side | time (s) | " + head + " | MRR (r200) |")
    print("|---|---|---|" + "---|" * args.bins + "---|")
    for label, n, dt, per_bin, mrr in rows:
        print("| %s | %s | %.1f | %s | %s |" % (label, "—" if n is None else n, dt,
                                               " | ".join("%.2g" % v for v in per_bin),
                                               "%.3g" % mrr if mrr is not None else "> 2"))
    print()
    print("mean |mu/mu_analytic - 1| per bin of b / r200; %d bundles per bin; %d RK4 steps (asinh)"
          % (nb, cfg["n_steps"]))


if __name__ == "__main__":
    main()

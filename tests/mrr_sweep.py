"""Minimum-reliable-radius sweeps on the NFW halo (Sec. 4.2, Figs. nfwtests1-3):
bundles at impact parameters log-spaced in [0.05, 2] r200 around the NFW halo
of the NFW workload (M200 = 1e14, c = 5, z_l = 0.25, z_s = 0.5), one numerical
parameter varied at a time, each setting's magnification compared with the
analytic truncated NFW lens in radial bins.  The MRR is the smallest bin edge
outside which every bin's mean |dmu/mu| is below 3 %.

    python tests/mrr_sweep.py --sweep grid    # node spacing 24 / 49 h^-1 kpc x n_int 1 / 2 (grid path)
    python tests/mrr_sweep.py --sweep theta   # bundle radius 0.1" / 1"
    python tests/mrr_sweep.py --sweep mass    # particle mass 1e9 / 1e10 / 1e11 Msun
    python tests/mrr_sweep.py --sweep soft    # softening 1 / 5 / 20 kpc
    python tests/mrr_sweep.py --sweep steps   # RK4 steps 500 / 1000 / 2000 / 4000

Needs a GPU; prints one markdown table per sweep.
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

ARCSEC = math.radians(1.0 / 3600.0)


def settings(sweep):
    """(label, overrides) per setting; overrides of: n_part, soft, theta_r,
    n_steps, grid (spacing in h^-1 kpc, n_int)"""
    base = dict(n_part=100000, soft=5e-3, theta_r=ARCSEC, n_steps=2000, grid=None)
    if sweep == "grid":
        out = [("direct sum", {})]
        for sp in (24.0, 49.0):
            for ni in (1, 2):
                out.append(("grid %g h^-1 kpc, n_int %d" % (sp, ni), dict(grid=(sp, ni))))
    elif sweep == "theta":
        out = [('theta_r = 1"', {}), ('theta_r = 0.1"', dict(theta_r=0.1 * ARCSEC))]
    elif sweep == "mass":
        out = [("m_p = %.0e Msun" % m, dict(n_part=int(round(1.5534e14 / m)))) for m in (1e9, 1e10, 1e11)]
    elif sweep == "soft":
        out = [("eps = %g kpc" % (e * 1e3), dict(soft=e)) for e in (1e-3, 5e-3, 2e-2)]
    elif sweep == "steps":
        out = [("%d RK4 steps" % n, dict(n_steps=n)) for n in (500, 1000, 2000, 4000)]
    else:
        raise SystemExit("unknown sweep " + sweep)
    return [(lab, dict(base, **ov)) for lab, ov in out]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweep", default="grid", choices=("grid", "theta", "mass", "soft", "steps"))
    ap.add_argument("--bundles-per-bin", type=int, default=48)
    ap.add_argument("--bins", type=int, default=8)
    args = ap.parse_args()
    import oracle
    import oracle.analytic as A
    import paper_1110_4894_gb300 as P
    om, ol, h = (0.3, 0.7, 0.7)  # the cosmology of every workload
    cosmo = oracle.Cosmology(om, ol, h)
    g = np.random.default_rng(2024)
    edges = np.logspace(math.log10(0.05), math.log10(2.0), args.bins + 1)
    nb = args.bundles_per_bin
    x = np.concatenate([np.exp(g.uniform(math.log(edges[i]), math.log(edges[i + 1]), nb)) for i in range(args.bins)])
    phi = g.uniform(0, 2 * math.pi, x.size)
    rows, halos = [], {}
    for label, s in settings(args.sweep):
        if s["n_part"] not in halos:
            halos[s["n_part"]] = inputs.config_c2(n_particles=s["n_part"], n_side=2)
        cfg = halos[s["n_part"]]
        L = A.NFWLens(cosmo, 1e14, 5.0, cfg["z_l"], cfg["z_s"])
        theta = np.stack([x * L.r200 / L.D_d * np.cos(phi), x * L.r200 / L.D_d * np.sin(phi)], 1)
        mu_an = np.array([L.lens_trunc(t)[2] for t in x * L.r200 / L.D_d])
        kw = dict(n_ring=4, theta_r=s["theta_r"], schedule=P.SCHED_ASINH, n_steps=s["n_steps"],
                  lens_chi=cfg["chi_l"], asinh_s=max(s["soft"], 1e-3))
        ctx = P.Context(0, precision=P.MIXED, autotune=1)
        ctx.set_cosmology(om, ol, h)
        t0 = time.time()
        n_nodes = None
        if s["grid"] is None:
            ctx.load_particles(0, cfg["pos"], cfg["mass"], s["soft"])
        else:
            sp, ni = s["grid"]
            half = 2.2 * cfg["info"]["r200_phys"] * (1 + cfg["z_l"])
            hh = sp / 1000.0 / h
            n_nodes = int(math.ceil(2 * half / hh)) + 1
            ctx.load_grid(0, cfg["pos"], cfg["mass"], s["soft"], [-half, -half, cfg["chi_l"] - half], hh, n_nodes,
                          n_int=ni)
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
        rows.append((label, n_nodes, dt, per_bin, mrr))
        ctx.close()
    head = " | ".join("%.3g–%.3g" % (edges[i], edges[i + 1]) for i in range(args.bins))
    print("| setting | nodes/side | time (s) | " + head + " | MRR (r200) |")
    print("|---|---|---|" + "---|" * args.bins + "---|")
    for label, n, dt, per_bin, mrr in rows:
        print("| %s | %s | %.1f | %s | %s |" % (label, "—" if n is None else n, dt,
                                               " | ".join("%.2g" % v for v in per_bin),
                                               "%.3g" % mrr if mrr is not None else "> 2"))
    print()
    print("sweep %s: mean |mu/mu_analytic - 1| per bin of b / r200, %d bundles per bin; base: 1e5 particles, "
          "eps 5 kpc, theta_r 1\", 2000 asinh RK4 steps, direct sum" % (args.sweep, nb))


if __name__ == "__main__":
    main()

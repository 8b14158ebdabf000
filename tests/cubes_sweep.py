"""Cubes per replica at a fixed node spacing (Sec. 5.2, Fig. MudMagBoxes): the
sampling region of Sec. 5.2 (256^3 particles in a 50/h Mpc box, 28 replicas
to z_s = 0.5) with each replica's prism cut into 8 cubes of 256^3 nodes or
16 cubes of 128^3 nodes, both about 24/h kpc node spacing.  16 cubes halve
the prism's width, so their bundles cover a quarter of the sky patch; the
paper traces 3e4 and 6e4 lines of sight.  Prints the muPDF moments of each
setting, a two-sample comparison of the magnifications, and the 8-cube
setting traced on the 16-cube setting's own bundles (same lines of sight,
so the difference is the cut of the mass alone).

    python tests/cubes_sweep.py [--steps 2000]

Needs a GPU with about 130 GB free (the 8-cube tables are 120 GB in FP32).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402


def run(P, cubes, n, n_side, steps, extra_theta=None):
    cfg = inputs.config_prism(n_side=n_side, n_steps=steps, cubes=cubes, grid_n=n)
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    t0 = time.perf_counter()
    ctx.load_grid_box(0, cfg["pos"], cfg["mass"], cfg["soft"], cfg["L"], cfg["rot"], cfg["shift"], cubes, n,
                      n_int=2, mean_subtract=True)
    build = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = ctx.trace(0, cfg["z_s"], cfg["theta"], n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0,
                  n_steps=steps)
    trace = time.perf_counter() - t0
    counts, wfix, sc = ctx.histogram(r["mu"], r["flags"], bins=200, mu_min=0.5, mu_max=5.0)
    spacing = cfg["L"] / cubes / (n - 1) * cfg["cosmo"][2] * 1e3
    extra = None
    if extra_theta is not None:
        extra = ctx.trace(0, cfg["z_s"], extra_theta, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0,
                          n_steps=steps)["mu"]
    ctx.close()
    return dict(cubes=cubes, n=n, bundles=len(r["mu"]), spacing_h_kpc=spacing, build_s=build, trace_s=trace,
                mu=r["mu"], flags=r["flags"], counts=counts, sc=sc, extra=extra, theta=cfg["theta"])


def boot_moments(mu, reps=200, seed=7):
    """1/|mu|-weighted mean and spread, with bootstrap standard errors"""
    g = np.random.default_rng(seed)
    w = 1.0 / np.abs(mu)

    def mom(m, ww):
        mean = np.sum(ww * np.abs(m)) / np.sum(ww)
        return mean, np.sqrt(np.sum(ww * (np.abs(m) - mean) ** 2) / np.sum(ww))
    base = mom(mu, w)
    bs = np.array([mom(mu[i], w[i]) for i in (g.integers(0, len(mu), len(mu)) for _ in range(reps))])
    return base, bs.std(axis=0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--json", default="")
    args = ap.parse_args()
    import paper_1110_4894_gb300 as P
    r16 = run(P, 16, 128, 245, args.steps)
    res = [run(P, 8, 256, 176, args.steps, extra_theta=r16["theta"]), r16]
    from scipy.stats import ks_2samp
    print("| cubes x nodes | node spacing (h^-1 kpc) | bundles | build (s) | trace (s) | <mu>_w | sigma_w | "
          "5% / 50% / 95% of mu | flagged |")
    print("|---|---|---|---|---|---|---|---|---|")
    out = []
    for r in res:
        (m, s), (dm, ds) = boot_moments(r["mu"])
        q = np.percentile(r["mu"], [5, 50, 95])
        print("| %d x %d^3 | %.1f | %d | %.1f | %.1f | %.4f +- %.4f | %.4f +- %.4f | %.4f / %.4f / %.4f | %d |" % (
            r["cubes"], r["n"], r["spacing_h_kpc"], r["bundles"], r["build_s"], r["trace_s"], m, dm, s, ds,
            q[0], q[1], q[2], int(np.count_nonzero(r["flags"]))))
        out.append(dict(cubes=r["cubes"], n=r["n"], bundles=r["bundles"], mean_w=m, mean_w_err=dm, sigma_w=s,
                        sigma_w_err=ds, quantiles=q.tolist(), build_s=r["build_s"], trace_s=r["trace_s"]))
    ks = ks_2samp(res[0]["mu"], res[1]["mu"])
    print("\ntwo-sample KS on mu: D = %.4f, p = %.3g" % (ks.statistic, ks.pvalue))
    # the same lines of sight through both cuts of the mass
    m8, m16 = res[0]["extra"], res[1]["mu"]
    (a8, da8), (s8, ds8) = zip(*boot_moments(m8))
    d = np.abs(m8 / m16 - 1)
    ks2 = ks_2samp(m8, m16)
    same = dict(bundles=len(m16), mean_w_8=a8, sigma_w_8=s8, abs_dmu_median=float(np.median(d)),
                abs_dmu_p99=float(np.percentile(d, 99)), ks_D=float(ks2.statistic), ks_p=float(ks2.pvalue))
    print("8 cubes on the 16-cube bundles: <mu>_w = %.4f +- %.4f, sigma_w = %.4f +- %.4f; "
          "|mu8/mu16 - 1| median %.2e, 99%% %.2e; KS D = %.4f" % (a8, da8, s8, ds8, same["abs_dmu_median"],
                                                                 same["abs_dmu_p99"], same["ks_D"]))
    out.append(dict(same_bundles=same))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(dict(settings=out, ks_D=float(ks.statistic), ks_p=float(ks.pvalue), steps=args.steps), f)


if __name__ == "__main__":
    main()

"""Per-result error statement of the mixed-precision CUDA path against the FP64
oracle, for the five workloads (point lens, NFW halo, the 2^21 and 2^24
particle boxes, the independent light cones).

Two phases, so that the slow oracle need not hold a GPU:

    python tests/error_statement.py gpu --out err_gpu.npz      # needs a GPU
    python tests/error_statement.py compare --gpu err_gpu.npz  # CPU only

The ``gpu`` phase traces each workload with the CUDA library (mixed precision,
and the all-FP64 path on a subset) and evaluates the pair sum at sample points
along the lines of sight.  The ``compare`` phase regenerates the same seeded
inputs, runs the oracle on a sample of the bundles and prints, per workload,
the maximum and the 99.9th percentile of

* |d alpha| / |alpha| per ray (gate 1e-5),
* |d mu / mu| per bundle (gate 1e-4),
* |d grad phi| / |grad phi| of the pair sum at points (diagnostic),

plus a conditioning control: the oracle re-run with the particle positions
(relative to the field's centre) and masses rounded to FP32, which shows how
large a change of the result an FP32-sized change of the inputs makes.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import inputs  # noqa: E402


def _cases(quick):
    """name -> (config factory, GPU bundle count, oracle sample, control sample,
    FP64-GPU subset)"""
    c3_steps, c5_steps = (60, 12) if quick else (250, 50)
    return {
        "c1_point_lens_fp64": (lambda: inputs.config_c1(), None, None, 0, 0),
        "c1_point_lens_mixed": (lambda: inputs.config_c1(), None, None, 0, 0),
        "c2_nfw_1e5p": (lambda: inputs.config_c2(n_steps=400 if quick else 2000), None,
                        8 if quick else 32, 4 if quick else 16, 64 if quick else 256),
        "c3_box_2e21p": (lambda: inputs.config_c3(n_steps=c3_steps), 4096, 4 if quick else 8, 2 if quick else 4,
                         64 if quick else 128),
        "c5_box_2e24p": (lambda: inputs.config_c5(n_steps=c5_steps), 1024, 2 if quick else 4, 1 if quick else 2,
                         16 if quick else 64),
        "c4_cones": (lambda: inputs.config_c4(n_cones=4 if quick else 8, n_steps=40 if quick else 100), None,
                     4 if quick else 8, 2 if quick else 4, 0),
    }


def _sample(n, k):
    return np.unique(np.linspace(0, n - 1, k).astype(int)) if k else np.zeros(0, int)


def _points(cfg, theta, n_pts, chi_s, seed=7):
    """stage-like points: a run of neighbouring bundles (grid order) on their
    unperturbed lines of sight at each of a few comoving distances, so that
    consecutive points are neighbours as the rays of one RK4 stage are; with
    the replica index the bundle's central ray would select there"""
    g = np.random.default_rng(seed)
    k = 8
    per = max(1, n_pts // k)
    if cfg.get("replicated"):
        chis = np.sort(g.uniform(0.02 * chi_s, 0.98 * chi_s, k))
    else:
        lc = cfg.get("lens_chi", 0.5 * chi_s)
        chis = lc + np.linspace(-2.0, 2.0, k)
    pts = []
    for chi in chis:
        b0 = int(g.integers(0, max(1, len(theta) - per)))
        th = theta[b0:b0 + per]
        pts.append(np.stack([th[:, 0] * chi, th[:, 1] * chi, np.full(len(th), chi)], axis=1))
    pts = np.concatenate(pts)
    rep = np.floor(pts[:, 2] / cfg["L"]).astype(np.int32) if cfg.get("replicated") else None
    return pts, rep


def _load(ctx, fid, cfg):
    if cfg.get("replicated"):
        ctx.load_particles(fid, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                           rot=cfg["rot"], shift=cfg["shift"], mean_subtract=cfg.get("mean_subtract", False))
    else:
        ctx.load_particles(fid, cfg["pos"], cfg["mass"], cfg["soft"])


def _trace_kw(cfg):
    return dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
                lens_chi=cfg.get("lens_chi", 0.0), asinh_s=cfg.get("asinh_s", 1.0))


def phase_gpu(args):
    import paper_1110_4894_gb300 as P
    out, meta = {}, {}
    for name, (make, nb_gpu, n_orc, n_ctl, n_fp64) in _cases(args.quick).items():
        t0 = time.time()
        cfg = make()
        if name == "c4_cones":
            for prec, tag in ((P.MIXED, "mixed"), (P.FP64, "fp64")):
                ctx = P.Context(0, precision=prec, autotune=1 if prec == P.MIXED else 0)
                ctx.set_cosmology(*cfg["cosmo"])
                cones = []
                for i, c in enumerate(cfg["cones"]):
                    ctx.load_particles(i, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"],
                                       rot=c["rot"], shift=c["shift"], mean_subtract=True)
                    cones.append(dict(field_id=i, z_s=c["z_s"], theta=c["theta"], n_steps=c["n_steps"]))
                res = ctx.trace_batch(cones, want_rays=True, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"],
                                      schedule=0)
                for i, r in enumerate(res):
                    idx = _sample(len(r["mu"]), n_orc)
                    out[f"{name}/{i}/{tag}/mu"] = r["mu"]
                    out[f"{name}/{i}/{tag}/flags"] = r["flags"]
                    out[f"{name}/{i}/{tag}/rays_s"] = r["rays"][idx]
                meta[f"{name}/{tag}"] = ctx.stats()
                ctx.close()
            print(name, "%.1f s" % (time.time() - t0), flush=True)
            continue
        theta = cfg["theta"] if nb_gpu is None else cfg["theta"][:nb_gpu]
        prec = P.FP64 if name.endswith("_fp64") else P.MIXED
        ctx = P.Context(0, precision=prec, autotune=0 if prec == P.FP64 else 1)
        ctx.set_cosmology(*cfg["cosmo"])
        _load(ctx, 0, cfg)
        g = ctx.trace(0, cfg["z_s"], theta, want_rays=True, **_trace_kw(cfg))
        meta[name] = ctx.stats()
        for k in ("mu", "flags", "steps", "rays"):
            out[f"{name}/{k}"] = g[k]
        chi_s = ctx.schedule(cfg["z_s"], 0, 1)[1]
        pts, rep = _points(cfg, theta, 512 if name.startswith("c5") or name.startswith("c3") else 4096, chi_s)
        out[f"{name}/pts"] = pts
        out[f"{name}/pot"] = ctx.potential(0, pts, rep)
        ctx.close()
        if n_fp64:
            ctx = P.Context(0, precision=P.FP64)
            ctx.set_cosmology(*cfg["cosmo"])
            _load(ctx, 0, cfg)
            idx = _sample(len(theta), n_fp64)
            f = ctx.trace(0, cfg["z_s"], theta[idx], want_rays=True, **_trace_kw(cfg))
            out[f"{name}/fp64_idx"] = idx
            out[f"{name}/fp64_mu"] = f["mu"]
            out[f"{name}/fp64_rays"] = f["rays"]
            ctx.close()
        print(name, "%.1f s" % (time.time() - t0), flush=True)
    np.savez_compressed(args.out, **out)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(dict(quick=args.quick, stats=meta), fh, indent=1)


def _rel_alpha(rays, res, idx=None):
    th = res.ray_theta() if idx is None else res.ray_theta()[idx]
    a_o = res.alpha() if idx is None else res.alpha()[idx]
    a_g = th - rays[:, :, 1:3] / res.chi_s
    return (np.linalg.norm(a_g - a_o, axis=-1) / np.linalg.norm(a_o, axis=-1)).ravel()


def _abs_alpha(rays, res):
    a_g = res.ray_theta() - rays[:, :, 1:3] / res.chi_s
    return np.linalg.norm(a_g - res.alpha(), axis=-1).ravel()


def _round_fp32(cfg):
    """the field with positions (about the field's centre) and masses rounded to FP32"""
    pos = np.asarray(cfg["pos"], np.float64)
    c = np.full(3, 0.5 * cfg["L"]) if cfg.get("replicated") else 0.5 * (pos.min(0) + pos.max(0))
    p32 = (pos - c).astype(np.float32).astype(np.float64) + c
    m32 = np.asarray(cfg["mass"], np.float64).astype(np.float32).astype(np.float64)
    return dict(cfg, pos=p32, mass=m32)


def _field(cfg):
    import oracle
    if cfg.get("replicated"):
        return oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, L=cfg["L"], rot=cfg["rot"],
                                shift=cfg["shift"], mean_subtract=cfg.get("mean_subtract", False))
    return oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"])


def _stat(x):
    x = np.asarray(x, np.float64).ravel()
    if x.size == 0:
        return None
    return dict(max=float(x.max()), p999=float(np.percentile(x, 99.9)), n=int(x.size))


def _grad_rel(a, b):
    return np.linalg.norm(a[:, 1:4] - b[:, 1:4], axis=1) / np.linalg.norm(b[:, 1:4], axis=1)


def phase_compare(args):
    import oracle
    d = np.load(args.gpu)
    meta = json.load(open(os.path.splitext(args.gpu)[0] + ".json"))
    quick = meta["quick"]
    rows = {}
    for name, (make, nb_gpu, n_orc, n_ctl, n_fp64) in _cases(quick).items():
        t0 = time.time()
        cfg = make()
        cosmo = oracle.Cosmology(*cfg["cosmo"])
        row = {}
        if name == "c4_cones":
            dm, da, dar, dm64, dmc, dac = [], [], [], [], [], []
            for i, c in enumerate(cfg["cones"]):
                mu_g, mu_f = d[f"{name}/{i}/mixed/mu"], d[f"{name}/{i}/fp64/mu"]
                dm64.append(np.abs(mu_g / mu_f - 1))
                idx = _sample(len(mu_g), n_orc)
                cc = dict(c, replicated=True, mean_subtract=True, cosmo=cfg["cosmo"], n_ring=cfg["n_ring"],
                          theta_r=cfg["theta_r"], schedule=0)
                o = oracle.trace(cosmo, _field(cc), c["z_s"], c["theta"][idx], n_ring=cfg["n_ring"],
                                 theta_r=cfg["theta_r"], schedule=0, n_steps=c["n_steps"])
                dm.append(np.abs(mu_g[idx] / o.mu - 1))
                da.append(_rel_alpha(d[f"{name}/{i}/mixed/rays_s"], o))
                dar.append(_abs_alpha(d[f"{name}/{i}/mixed/rays_s"], o) / np.sqrt(np.mean(np.sum(o.alpha() ** 2, -1))))
                if i < 4 and n_ctl:
                    j = idx[:n_ctl]
                    oc = oracle.trace(cosmo, _field(_round_fp32(cc)), c["z_s"], c["theta"][j], n_ring=cfg["n_ring"],
                                      theta_r=cfg["theta_r"], schedule=0, n_steps=c["n_steps"])
                    dmc.append(np.abs(oc.mu / o.mu[:len(j)] - 1))
                    dac.append(np.linalg.norm(oc.alpha() - o.alpha()[:len(j)], axis=-1).ravel()
                               / np.linalg.norm(o.alpha()[:len(j)], axis=-1).ravel())
            row = dict(mu=_stat(np.concatenate(dm)), alpha=_stat(np.concatenate(da)),
                       alpha_rms=_stat(np.concatenate(dar)),
                       mu_vs_gpu_fp64=_stat(np.concatenate(dm64)),
                       control_mu=_stat(np.concatenate(dmc)) if dmc else None,
                       control_alpha=_stat(np.concatenate(dac)) if dac else None,
                       steps=cfg["cones"][0]["n_steps"], cones=len(cfg["cones"]),
                       bundles_gpu=int(sum(len(c["theta"]) for c in cfg["cones"])))
            rows[name] = row
            print(name, "%.1f s" % (time.time() - t0), file=sys.stderr, flush=True)
            continue
        theta = cfg["theta"] if nb_gpu is None else cfg["theta"][:nb_gpu]
        mu_g, rays_g = d[f"{name}/mu"], d[f"{name}/rays"]
        idx = np.arange(len(theta)) if n_orc is None else _sample(len(theta), n_orc)
        field = _field(cfg)
        o = oracle.trace(cosmo, field, cfg["z_s"], theta[idx], **_trace_kw(cfg))
        row["mu"] = _stat(np.abs(mu_g[idx] / o.mu - 1))
        row["alpha"] = _stat(_rel_alpha(rays_g[idx], o))
        row["alpha_rms"] = _stat(_abs_alpha(rays_g[idx], o) / np.sqrt(np.mean(np.sum(o.alpha() ** 2, -1))))
        row["flags_equal"] = bool(np.array_equal(d[f"{name}/flags"][idx], o.flags))
        row["steps_equal"] = bool(np.array_equal(d[f"{name}/steps"][idx], o.steps))
        pts = d[f"{name}/pts"]
        rep = np.floor(pts[:, 2] / cfg["L"]).astype(np.int32) if cfg.get("replicated") else None
        ref_pot = oracle.potential(field, pts, rep)
        row["grad_phi"] = _stat(_grad_rel(d[f"{name}/pot"], ref_pot))
        row["grad_phi_rms"] = _stat(np.linalg.norm(d[f"{name}/pot"][:, 1:4] - ref_pot[:, 1:4], axis=1)
                                    / np.sqrt(np.mean(np.sum(ref_pot[:, 1:4] ** 2, axis=1))))
        if f"{name}/fp64_mu" in d:
            fi = d[f"{name}/fp64_idx"]
            row["mu_vs_gpu_fp64"] = _stat(np.abs(mu_g[fi] / d[f"{name}/fp64_mu"] - 1))
        if n_ctl:
            js = _sample(len(idx), n_ctl)  # positions within the oracle sample
            oc = oracle.trace(cosmo, _field(_round_fp32(cfg)), cfg["z_s"], theta[idx[js]], **_trace_kw(cfg))
            a_ref = o.alpha()[js]
            row["control_mu"] = _stat(np.abs(oc.mu / o.mu[js] - 1))
            row["control_alpha"] = _stat(np.linalg.norm(oc.alpha() - a_ref, axis=-1).ravel()
                                         / np.linalg.norm(a_ref, axis=-1).ravel())
        row.update(steps=cfg["n_steps"], bundles_gpu=len(theta), bundles_oracle=len(idx))
        rows[name] = row
        print(name, "%.1f s" % (time.time() - t0), file=sys.stderr, flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    _print_table(rows)


def _fmt(s, key="max"):
    return "—" if not s else "%.2e" % s[key]


def _print_table(rows):
    print("| workload | RK4 steps | bundles GPU / oracle | max / p99.9 \\|Δα/α\\| | max \\|Δα\\|/rms α "
          "| max / p99.9 \\|Δμ/μ\\| | \\|Δμ/μ\\| vs GPU FP64 (max) | \\|Δ∇φ\\|/\\|∇φ\\| max / p99.9 "
          "| max \\|Δ∇φ\\|/rms ∇φ | control \\|Δμ/μ\\| / \\|Δα/α\\| (max) |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    for name, r in rows.items():
        nb = "%s / %s" % (r.get("bundles_gpu"), r.get("bundles_oracle", r.get("mu", {}).get("n") if r.get("mu") else "—"))
        print("| %s | %s | %s | %s / %s | %s | %s / %s | %s | %s / %s | %s | %s / %s |" % (
            name, r["steps"], nb, _fmt(r["alpha"]), _fmt(r["alpha"], "p999"), _fmt(r.get("alpha_rms")),
            _fmt(r["mu"]), _fmt(r["mu"], "p999"), _fmt(r.get("mu_vs_gpu_fp64")), _fmt(r.get("grad_phi")),
            _fmt(r.get("grad_phi"), "p999"), _fmt(r.get("grad_phi_rms")), _fmt(r.get("control_mu")),
            _fmt(r.get("control_alpha"))))


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="phase", required=True)
    g = sub.add_parser("gpu")
    g.add_argument("--out", required=True)
    g.add_argument("--quick", action="store_true")
    c = sub.add_parser("compare")
    c.add_argument("--gpu", required=True)
    c.add_argument("--json", default=None)
    args = ap.parse_args()
    (phase_gpu if args.phase == "gpu" else phase_compare)(args)


if __name__ == "__main__":
    main()

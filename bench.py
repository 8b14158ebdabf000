"""Benchmark: ray-particle interactions/s (and ray bundles/s) of the 3D
ray-bundle trace, checked in the same run against the FP64 oracle.

Headline workload (the default): the 2^24-particle cosmological box.
16,777,216 equal-mass particles in a periodic 200/h Mpc box (half uniform,
half in 24,000 NFW halos with dN/dM ~ M^-1.9), replicated along the line of
sight with random 90-degree rotations and periodic shifts out to z_s = 1 (13
replicas), mean density subtracted; 1,048,576 bundles (central ray + 4 on a
1" polygon) on a 1024 x 1024 grid in +-2.3 deg; a uniform table of 1000 RK4
steps (3.3 Mpc).  One bench step = one RK4 stage of that trace over every
bundle (rt3d_trace_advance by one stage): the FP32 pair sum of all 5,242,880
rays against the 2^24 particles of their bundle's replica, the mean-density
prism and the FP64 integrator stage.  The step table, the bundle
initialiser and the autotuner's launch-shape choice run in the warm-up
(rt3d_trace_begin); the reducer and the muPDF run in the end-to-end leg.

Also in the JSON line:
  e2e             the same metric through the host C ABI (rt3d_load_particles of
                  the 2^24 particles from host memory, rt3d_trace of a slice of
                  the bundles with host angles in and results out,
                  rt3d_histogram), median of >= 3 samples
  parity          FP64 oracle vs the GPU (mixed, and all-FP64) on bundles
                  sampled over the whole sky grid, complete traces on a short
                  table; max |dmu/mu| against the 1e-4 gate
  cpu_baseline    the oracle's rate on that sample, on the host cores
  batched_cones   512 light cones (own halo boxes with 1e3-1e6 particles, z_s
                  0.3-1.5, 256-4096 bundles) in one persistent launch under a
                  CUDA graph, shape picked by the autotuner
  fp64_same_cones the first cones of that batch traced by the all-FP64 path one
                  cone per launch, and the mixed batched path re-run on exactly
                  those cones: speedup on identical inputs; FP64 pair-sum
                  kernel against the FP64 peak

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c5|nfw|cones|grid|prism|born|box3|box5]

With N > 1 every rank (one per GPU, launched by torch.distributed.run; bench.py
starts it itself when called with --gpus N outside it) traces its own lines of
sight of the same box: weak scaling, no collective on the data path; the
timed region's maximum over ranks sets the rate, and the muPDFs of the
end-to-end leg are combined by rt3d_histogram_combine.
"""
import argparse
import json
import math
import os
import socket
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ray-particle interactions/s & ray bundles/s at |dmu/mu|<=1e-4 vs FP64 oracle"
UNIT = "interactions/s"
FLOPS_PER_INTERACTION = 20  # direct N-body convention (3 sub, 6 fma/mul for r^2, rsqrt, 3 mul, phi, 3 fma)
N_SM, FP32_LANES, FP64_LANES, SM_MAX_MHZ = 152, 128, 2, 2070.0
FP32_PEAK = N_SM * FP32_LANES * 2 * SM_MAX_MHZ * 1e6  # FLOP/s at the maximum SM clock
FP64_PEAK = N_SM * FP64_LANES * 2 * SM_MAX_MHZ * 1e6  # 1.26 TFLOP/s: GB300's FP64 rate is 1/64 of FP32's
PEAK_BASIS = "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived from unit counts and the maximum clock)"
PEAK64_BASIS = "152 SM x 2 FP64 lanes x 2 x 2070 MHz (derived; nominal GB300 FP64 1.25 TFLOP/s)"
HIST = dict(bins=200, mu_min=0.5, mu_max=5.0)
KERNEL_NAMES = {0: "k_force_packed", 1: "k_force_mixed", 2: "k_force_fp64", 3: "k_force_bundle", 4: "k_force_bundle2",
                5: "k_force_bundle2x"}
# dram__bytes_read.sum + dram__bytes_write.sum per pair-sum launch, from an ncu
# capture of that very launch (one metric pass on the full-size headline
# stage; profiles/dram_k_force_bundle2x_box2e24_full.md), keyed by (workload,
# kernel, threads per block, splits).  A shape not listed reports null.
PROFILED_DRAM_BYTES = {("c5", "k_force_bundle2x", 128, 1): 7763856384 + 261923584}
C5_NAME = "box_2e24p_200mpch_zs1_1048576b_uniform1000_rk4stage"


def nfw_workload(full=True):
    import inputs
    if full:
        cfg = inputs.config_c2()
        name = "nfw_halo_1e5p_4096b_2000s"
    else:
        cfg = inputs.config_c2(n_particles=20000, n_side=16, n_steps=400)
        name = "nfw_halo_2e4p_256b_400s"
    return cfg, name


workload = nfw_workload  # the auxiliary NFW-halo workloads below


def cones_workload(n_cones, n_steps):
    """the batched light-cone workload: n_cones independent halo boxes
    (50/h Mpc, particles log-uniform in 1e3..1e6, z_s uniform in 0.3..1.5,
    256..4096 bundles), each traced with a uniform table of n_steps steps"""
    import inputs
    cfg = inputs.config_c4(n_cones=n_cones, n_steps=n_steps)
    return cfg, "light_cones_%dc_%ds" % (n_cones, n_steps)


def run_cones(args):
    """One step = one rt3d_trace_batch of every cone (a single persistent
    launch in a CUDA graph).  Compared with the all-FP64 path run one cone
    per launch on the first cones of the same batch."""
    import torch

    import paper_1110_4894_gb300 as P
    cfg, name = cones_workload(args.cones, args.cone_steps)
    ctx = P.Context(0, precision=P.MIXED, autotune=1, variant=args.variant)
    ctx.set_cosmology(*cfg["cosmo"])
    cones = []
    npart = 0
    for i, c in enumerate(cfg["cones"]):
        ctx.load_particles(i, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"], rot=c["rot"],
                           shift=c["shift"], mean_subtract=True)
        cones.append(dict(field_id=i, z_s=c["z_s"], theta=c["theta"], n_steps=c["n_steps"]))
        npart += len(c["mass"])
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    for _ in range(args.warmup):
        ctx.trace_batch(cones, **kw)
    times, inter = [], 0.0
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            ctx.trace_batch(cones, **kw)
            times.append(time.perf_counter() - t0)
            st = ctx.stats()
            inter += st["interactions"]
    clocks = clk.summary()
    dev_s = st["device_ms"] / 1e3
    value = inter / sum(times)
    # all-FP64 reference: the same cones, one per launch (a subset for time)
    sub = cones[: args.fp64_cones]
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    for i in range(len(sub)):
        c = cfg["cones"][i]
        c64.load_particles(i, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"], rot=c["rot"],
                           shift=c["shift"], mean_subtract=True)
    t0 = time.perf_counter()
    r64 = c64.trace_batch(sub, **kw)
    t64 = time.perf_counter() - t0
    i64 = c64.stats()["interactions"]
    rm = ctx.trace_batch(cones, **kw)
    dmu = max(float(np.max(np.abs(a["mu"] / b["mu"] - 1))) for a, b in zip(rm[: len(sub)], r64))
    nb = sum(len(c["theta"]) for c in cfg["cones"])
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "bundles_per_s": nb * args.steps / sum(times),
           "config": {"workload": name, "cones": args.cones, "particles": npart, "bundles": nb,
                      "rk4_steps_per_cone": args.cone_steps, "launch_shape": {k: st[k] for k in ("threads_per_block",
                                                                                                "splits", "variant")}},
           "roofline": {"bound": "alu", "achieved": FLOPS_PER_INTERACTION * st["interactions"] / dev_s / 1e12,
                        "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
                        "frac": FLOPS_PER_INTERACTION * st["interactions"] / dev_s / FP32_PEAK, "traffic": None,
                        "kernel": "k_batch_run (whole persistent launch)"},
           "fp64_one_cone_per_launch": {"cones": len(sub), "interactions_per_s": i64 / t64,
                                        "speedup_of_mixed_batched": value / (i64 / t64),
                                        "max_rel_dmu_vs_mixed": dmu},
           "clocks": clocks}
    print(json.dumps(out))
    return 0


# App. B evaluation of one ray on the mixed path (n_int = 2), in FP32
# operations: per field, 16 x3-line cubics from two nodes and their second
# derivatives (8 fused multiply-adds each) and the x2 and x1 weight sums
# (16 + 4 FMAs); the weight vectors (~50 operations) are shared by the four
# fields.  2 FLOP per FMA.
GRID_FLOPS_PER_RAY = 4 * 2 * (16 * 8 + 16 + 4) + 100
GRID_ROOFLINE_NOTE = ("k_grid_eval32 gathers its node records mostly from L1/L2 and is bound by that latency, "
                      "neither by HBM nor by the FP32 pipe (low frac); a trace's own bound on the grid path is "
                      "the FP64 integrator stage")


def run_grid(args):
    """The grid path (Sec. 3.3, App. B) on the NFW workload: the halo's
    particles on an n^3 node grid spanning +-2.2 r200 (comoving), App. B
    interpolation with n_int = 2.  One step = one full trace of every bundle
    (rt3d_trace_device + histogram).  Reported beside it: the grid build time,
    and |mu_grid / mu_direct - 1| against the direct-sum trace of the same
    bundles (the grid's smoothing, not a parity figure)."""
    import torch

    import paper_1110_4894_gb300 as P
    dev = torch.device("cuda", 0)
    cfg, name = workload(full=not args.small)
    if args.rk4_steps:
        cfg["n_steps"] = args.rk4_steps
        name = name.rsplit("_", 1)[0] + "_%ds" % args.rk4_steps
    n = args.grid_n
    r200c = cfg["info"]["r200_phys"] * (1 + cfg["z_l"])
    half = 2.2 * r200c
    h = 2 * half / (n - 1)
    lo = [-half, -half, cfg["chi_l"] - half]
    kw = trace_kw(cfg)
    nb = cfg["theta"].shape[0]
    ctx = P.Context(0, precision=P.MIXED, time_kernels=1)
    ctx.set_cosmology(*cfg["cosmo"])
    t0 = time.perf_counter()
    ctx.load_grid(0, cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    build_s = time.perf_counter() - t0
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).to(dev)
    d_bout = torch.zeros(nb * 6, dtype=torch.float64, device=dev)
    d_counts = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_wfix = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_scal = torch.zeros(8, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), **kw)
        ctx.histogram_device(sp, nb, d_bout.data_ptr(), d_counts.data_ptr(), d_wfix.data_ptr(), d_scal.data_ptr(),
                             **HIST)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    eval_ms, eval_launches, evals, launches = 0.0, 0, 0.0, 0
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            st = ctx.stats()
            eval_ms += st["force_ms"]
            eval_launches += st["force_launches"]
            evals += st["interactions"]  # ray-stage field evaluations on the grid path
            launches += st["launches"] + 2
    clocks = clk.summary()
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    mu_grid = d_bout.view(nb, 6)[:, 0].cpu().numpy()
    # the direct sum on the same bundles, for the grid's smoothing error
    cd = P.Context(0, precision=P.MIXED, autotune=1)
    cd.set_cosmology(*cfg["cosmo"])
    cd.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    mu_dir = cd.trace(0, cfg["z_s"], cfg["theta"], **kw)["mu"]
    dmu = np.abs(mu_grid / mu_dir - 1)
    # the FP64 grid path on the same bundles: the mixed path's FP32 interpolation error
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    c64.load_grid(0, cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    mu64 = c64.trace(0, cfg["z_s"], cfg["theta"], **kw)["mu"]
    dmu64 = float(np.max(np.abs(mu_grid / mu64 - 1)))
    per_launch_s = eval_ms / 1e3 / max(1, eval_launches)
    flops_per_launch = nb * (1 + cfg["n_ring"]) * GRID_FLOPS_PER_RAY
    out = {"metric": "ray bundles/s (grid path)", "value": nb * args.steps / dev_s, "unit": "bundles/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name + "_grid%d" % n, "grid_n": n, "node_spacing_mpc": h, "n_int": 2,
                      "bundles": nb, "rk4_steps": cfg["n_steps"], "l2": "256 MB buffer written between timed steps"},
           "grid_build_s": build_s,
           "field_evals_per_s": evals / dev_s,
           "roofline": {"bound": "alu", "achieved": flops_per_launch / per_launch_s / 1e12, "peak": FP32_PEAK / 1e12,
                        "unit": "TFLOP/s", "frac": flops_per_launch / per_launch_s / FP32_PEAK, "traffic": None,
                        "kernel": "k_grid_eval32", "avg_launch_ms": per_launch_s * 1e3,
                        "note": GRID_ROOFLINE_NOTE},
           "grid_vs_direct_sum": {"median_abs_dmu_over_mu": float(np.median(dmu)),
                                  "max_abs_dmu_over_mu": float(np.max(dmu))},
           "mixed_vs_fp64_grid": {"bundles": nb, "max_abs_dmu_over_mu": dmu64},
           "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(out))
    return 0


def run_prism(args):
    """The grid path on the sampling region of Sec. 5.2: 256^3 particles in a
    50/h Mpc box replicated 28 times to z_s = 0.5, each replica's 6.25/h Mpc
    prism cut into 8 cubes on 128^3-node grids (App. B interpolation,
    n_int = 2), 176^2 bundles inside the prism, 1000 uniform RK4 steps.  One
    step = one full trace of every bundle (rt3d_trace_device + histogram).
    Reported beside it: the build time of the 224 cube grids and the muPDF's
    weighted mean and width."""
    import torch

    import inputs
    import paper_1110_4894_gb300 as P
    dev = torch.device("cuda", 0)
    cfg = inputs.config_prism(n_steps=args.rk4_steps or 1000)
    n, cubes = cfg["grid_n"], cfg["cubes"]
    nb = cfg["theta"].shape[0]
    ctx = P.Context(0, precision=P.MIXED, time_kernels=1)
    ctx.set_cosmology(*cfg["cosmo"])
    t0 = time.perf_counter()
    ctx.load_grid_box(0, cfg["pos"], cfg["mass"], cfg["soft"], cfg["L"], cfg["rot"], cfg["shift"], cubes, n,
                      n_int=2, mean_subtract=True)
    build_s = time.perf_counter() - t0
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0, n_steps=cfg["n_steps"])
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).to(dev)
    d_bout = torch.zeros(nb * 6, dtype=torch.float64, device=dev)
    d_counts = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_wfix = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_scal = torch.zeros(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), **kw)
        ctx.histogram_device(sp, nb, d_bout.data_ptr(), d_counts.data_ptr(), d_wfix.data_ptr(), d_scal.data_ptr(),
                             **HIST)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    eval_ms, eval_launches, evals, launches = 0.0, 0, 0.0, 0
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            st = ctx.stats()
            eval_ms += st["force_ms"]
            eval_launches += st["force_launches"]
            evals += st["interactions"]
            launches += st["launches"] + 2
    clocks = clk.summary()
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    scal = d_scal.cpu().numpy()
    res = d_bout.view(nb, 6).cpu().numpy()
    # the FP64 grid path on the first bundles: the mixed path's FP32 interpolation error
    k = min(nb, args.fp64_bundles)
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    c64.load_grid_box(0, cfg["pos"], cfg["mass"], cfg["soft"], cfg["L"], cfg["rot"], cfg["shift"], cubes, n,
                      n_int=2, mean_subtract=True)
    mu64 = c64.trace(0, cfg["z_s"], cfg["theta"][:k], **kw)["mu"]
    dmu64 = float(np.max(np.abs(res[:k, 0] / mu64 - 1)))
    per_launch_s = eval_ms / 1e3 / max(1, eval_launches)
    flops_per_launch = nb * (1 + cfg["n_ring"]) * GRID_FLOPS_PER_RAY
    out = {"metric": "ray bundles/s (grid path, replicated box)", "value": nb * args.steps / dev_s,
           "unit": "bundles/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "prism_box_2e24p_%dcubes_grid%d" % (cubes, n), "particles": int(cfg["pos"].shape[0]),
                      "replicas": int(cfg["n_rep"]), "cubes_per_replica": cubes, "grid_n": n,
                      "node_spacing_mpc": cfg["L"] / cubes / (n - 1), "n_int": 2, "bundles": nb,
                      "rk4_steps": cfg["n_steps"], "z_s": cfg["z_s"],
                      "l2": "30 GB of cube grids, larger than L2"},
           "grid_build_s": build_s,
           "field_evals_per_s": evals / dev_s,
           "roofline": {"bound": "alu", "achieved": flops_per_launch / per_launch_s / 1e12, "peak": FP32_PEAK / 1e12,
                        "unit": "TFLOP/s", "frac": flops_per_launch / per_launch_s / FP32_PEAK, "traffic": None,
                        "kernel": "k_grid_eval32", "avg_launch_ms": per_launch_s * 1e3,
                        "note": GRID_ROOFLINE_NOTE},
           "mixed_vs_fp64_grid": {"bundles": k, "max_abs_dmu_over_mu": dmu64},
           "mupdf": {"bundles_binned": int(scal[0]), "mean_w": float(scal[6]), "sigma_w": float(scal[7]),
                     "flagged_bundles": int(np.count_nonzero(res[:, 5]))},
           "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(out))
    return 0


def run_born(args):
    """The Born approximation (Sec. 6) on the NFW workload: kappa and gamma of
    every bundle centre from the Hessian pair sum at every node of the 2000-
    step table.  One step = one rt3d_born call (host arrays in and out)."""
    import torch

    import paper_1110_4894_gb300 as P
    cfg, name = workload(full=not args.small)
    kw = dict(schedule=cfg["schedule"], n_steps=cfg["n_steps"], lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    nb = cfg["theta"].shape[0]
    for _ in range(args.warmup):
        ctx.born(0, cfg["z_s"], cfg["theta"], **kw)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            ctx.born(0, cfg["z_s"], cfg["theta"], **kw)
            times.append(time.perf_counter() - t0)
    clocks = clk.summary()
    pairs = nb * (cfg["n_steps"] + 1) * len(cfg["mass"])
    t = statistics.mean(times)
    out = {"metric": "Hessian pair interactions/s (Born approximation)", "value": pairs / t,
           "unit": "interactions/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "bundles_per_s": nb / t,
           "config": {"workload": name + "_born", "bundles": nb, "nodes": cfg["n_steps"] + 1,
                      "particles": len(cfg["mass"]), "timing": "host wall time of the whole call"},
           "clocks": clocks}
    print(json.dumps(out))
    return 0


def run_box(args):
    """A cosmological box over a fixed window of RK4 steps: the 2^21-particle
    100/h Mpc box (z_s = 0.5, all 256^2 bundles) or the 2^24-particle 200/h
    Mpc box (z_s = 1, a patch of --box-bundles of its 1024^2 bundles),
    replicated with random rotations and shifts and mean subtraction.  A
    converged trace to z_s takes thousands of steps (hours for the larger
    box); every RK4 step costs the same pair-sum work whatever its length, so
    the rate is measured on a trace with a short uniform table of
    --rk4-steps steps (default 4)."""
    import torch

    import inputs
    import paper_1110_4894_gb300 as P
    big = args.workload == "box5"
    steps = args.rk4_steps or 4
    cfg = inputs.config_c5(n_steps=1000) if big else inputs.config_c3(n_steps=1000)
    theta = cfg["theta"][:args.box_bundles] if big else cfg["theta"]
    nb = theta.shape[0]
    ctx = P.Context(0, precision=P.MIXED, time_kernels=1, autotune=1)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                       rot=cfg["rot"], shift=cfg["shift"], mean_subtract=True)
    # no extra steps: rays still short of the source plane after the window
    # would cost whole pair-sum launches for the few of them that count
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0, n_steps=steps, max_extra=0)
    dev = torch.device("cuda", 0)
    d_theta = torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    d_bout = torch.zeros(nb * 6, dtype=torch.float64, device=dev)
    sp = torch.cuda.current_stream(dev).cuda_stream
    kw_w = kw
    for _ in range(args.warmup):
        ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), **kw_w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    inter, force_ms, force_launches = 0.0, 0.0, 0
    stream = torch.cuda.current_stream(dev)
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), **kw_w)
            ev[k][1].record(stream)
            st = ctx.stats()
            inter += st["interactions"]
            force_ms += st["force_ms"]
            force_launches += st["force_launches"]
    clocks = clk.summary()
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    per_launch = inter / max(1, force_launches)
    avg = force_ms / 1e3 / max(1, force_launches)
    # the all-FP64 path on the first bundles of the same window: rate, and
    # the magnification difference to the mixed path on those bundles
    k = min(nb, args.fp64_bundles)
    mu_mixed = d_bout.view(nb, 6)[:k, 0].cpu().numpy()
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    c64.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                       rot=cfg["rot"], shift=cfg["shift"], mean_subtract=True)
    t0 = time.perf_counter()
    r64 = c64.trace(0, cfg["z_s"], theta[:k], **kw)
    t64 = time.perf_counter() - t0
    fp64_rate = c64.stats()["interactions"] / t64
    fp64 = {"bundles": k, "interactions_per_s": fp64_rate, "speedup_of_mixed": (inter / dev_s) / fp64_rate,
            "max_rel_dmu_vs_mixed": float(np.max(np.abs(mu_mixed / r64["mu"] - 1)))}
    out = {"metric": METRIC, "value": inter / dev_s, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": ("box_2e24p_200mpch" if big else "box_2e21p_100mpch") +
                      "_%db_%dsteps_window" % (nb, steps), "particles": len(cfg["mass"]), "bundles": nb,
                      "replicas": int(cfg["n_rep"]), "rk4_steps_timed": steps,
                      "step_mpc": float(ctx.schedule(cfg["z_s"], 0, steps)[1] / steps),
                      "launch_shape": {k: st[k] for k in ("threads_per_block", "splits", "cluster", "variant")}},
           "roofline": {"bound": "alu", "achieved": FLOPS_PER_INTERACTION * per_launch / avg / 1e12,
                        "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
                        "frac": FLOPS_PER_INTERACTION * per_launch / avg / FP32_PEAK, "traffic": None,
                        "kernel": KERNEL_NAMES.get(st["variant"], "k_force"), "avg_launch_ms": avg * 1e3},
           "fp64_same_window": fp64,
           "clocks": clocks}
    print(json.dumps(out))
    return 0


def run_multiplane(args):
    """The comparison of Sec. 5.4 on the sampling region of Sec. 5.2: 256^3
    particles in a 50/h Mpc box replicated 28 times to z_s = 0.5, 176^2
    bundles inside the prism.  The multiple lens-plane system (one plane per
    replica at its centre, direct-sum deflections of the projected particles,
    Sec. 3.1) runs on every bundle and is the timed metric (one step = one
    multi-plane trace of every bundle).  Beside it, on the same bundles: the
    3D trace on the paper's own grid path (each replica's prism in 8 cubes of
    128^3 nodes, n_int = 2, 1000 uniform RK4 steps), and on the first
    --mp-3d-bundles bundles the 3D direct-sum trace at 1000 and 2000 steps and
    the multi-plane system with 8 planes per replica.  Reported per method:
    the muPDF's weighted mean and spread and the shear statistics."""
    import torch

    import inputs
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_prism(n_steps=1000)
    dev = torch.device("cuda", 0)
    nb = cfg["theta"].shape[0]
    ctx = P.Context(0, precision=P.MIXED, autotune=1)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"], rot=cfg["rot"],
                       shift=cfg["shift"], mean_subtract=True)
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).to(dev)
    d_bout = torch.zeros(nb * 6, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"])
    for _ in range(args.warmup):
        ctx.multiplane_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), slices=args.mp_slices,
                              **kw)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    inter = 0.0
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.multiplane_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(),
                                  slices=args.mp_slices, **kw)
            ev[k][1].record(stream)
            inter += ctx.stats()["interactions"]
    clocks = clk.summary()
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    res = d_bout.view(nb, 6).cpu().numpy()
    mp = {"mu": res[:, 0], "gamma1": res[:, 2], "gamma2": res[:, 3], "flags": res[:, 5].astype(np.int32)}

    def stats(r, sel=slice(None)):
        mu, fl = np.asarray(r["mu"])[sel], np.asarray(r["flags"])[sel]
        c, w, sc = ctx.histogram(mu, fl, **HIST)
        gam = np.hypot(np.asarray(r["gamma1"])[sel], np.asarray(r["gamma2"])[sel])
        wt = 1.0 / np.abs(mu)
        return {"bundles": int(sc["n_used"]), "mean_w": sc["mean_w"], "sigma_w": sc["sigma_w"],
                "mu_p5_p50_p95": [float(v) for v in np.percentile(mu, [5, 50, 95])],
                "gamma_mean_w": float(np.sum(wt * gam) / np.sum(wt)),
                "gamma_p50_p95": [float(v) for v in np.percentile(gam, [50, 95])]}

    # the 3D trace on the grid path: each replica's prism in 8 cubes of 128^3 nodes
    cg = P.Context(0, precision=P.MIXED)
    cg.set_cosmology(*cfg["cosmo"])
    t0 = time.perf_counter()
    cg.load_grid_box(0, cfg["pos"], cfg["mass"], cfg["soft"], cfg["L"], cfg["rot"], cfg["shift"], cfg["cubes"],
                     cfg["grid_n"], n_int=2, mean_subtract=True)
    build_s = time.perf_counter() - t0
    g3 = cg.trace(0, cfg["z_s"], cfg["theta"], schedule=0, n_steps=cfg["n_steps"], **kw)
    cg.close()
    # the first k bundles: 3D direct sum at 1000 and 2000 steps, 8 planes per replica
    k = min(nb, args.mp_3d_bundles)
    th = np.ascontiguousarray(cfg["theta"][:k])
    d3 = ctx.trace(0, cfg["z_s"], th, schedule=0, n_steps=1000, **kw)
    d3b = ctx.trace(0, cfg["z_s"], th, schedule=0, n_steps=2000, **kw)
    m8 = ctx.multiplane(0, cfg["z_s"], th, slices=8, **kw)
    sub = slice(0, k)
    out = {"metric": "ray-particle interactions/s (multiple lens planes)", "value": inter / dev_s,
           "unit": "interactions/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "bundles_per_s": nb * args.steps / dev_s,
           "config": {"workload": "prism_box_256cubed_50mpch_zs0.5_%db_planes%d" % (nb, args.mp_slices),
                      "particles": len(cfg["mass"]), "bundles": nb, "replicas": int(cfg["n_rep"]),
                      "planes_per_replica": args.mp_slices},
           "all_bundles": {"multiplane": stats(mp), "grid_3d_8x128": stats(g3), "grid_build_s": build_s,
                           "median_abs_mu_mp_over_mu_grid_minus_1": float(np.median(np.abs(mp["mu"] / g3["mu"] - 1))),
                           "corr_mu_minus_1_mp_grid": float(np.corrcoef(mp["mu"] - 1, g3["mu"] - 1)[0, 1])},
           "first_bundles": {"bundles": k, "multiplane": stats(mp, sub), "multiplane_8_planes": stats(m8),
                             "grid_3d_8x128": stats(g3, sub), "direct_3d_1000": stats(d3), "direct_3d_2000": stats(d3b),
                             "median_abs_mu_direct_1000_over_2000_minus_1":
                                 float(np.median(np.abs(d3["mu"] / d3b["mu"] - 1))),
                             "median_abs_mu_mp_over_direct_2000_minus_1":
                                 float(np.median(np.abs(mp["mu"][sub] / d3b["mu"] - 1))),
                             "median_abs_mu_grid_over_direct_2000_minus_1":
                                 float(np.median(np.abs(g3["mu"][sub] / d3b["mu"] - 1)))},
           "clocks": clocks}
    print(json.dumps(out))
    return 0


def trace_kw(cfg):
    return dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
                lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def relaunch_command(argv, gpus, port):
    """the torch.distributed.run command that starts one rank per GPU with the
    same arguments (bench.py --gpus N called outside torchrun)"""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(gpus),
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


def c5_config(args):
    """the headline box (2^24 particles unless --box-particles asks for a
    smaller box with the same generator, for checks; rings of 4 unless
    --n-ring asks for another bundle, e.g. the paper's ring of 8)"""
    import inputs
    if args.box_particles == 2 ** 24:
        cfg = inputs.config_c5(n_steps=args.table_steps)
    else:
        n_halos = max(1, int(round(24000 * args.box_particles / 2 ** 24)))
        cfg = inputs.config_c5(N=args.box_particles, n_halos=n_halos, n_steps=args.table_steps)
    if args.n_ring:
        cfg["n_ring"] = args.n_ring
    return cfg


def c5_name(args):
    name = C5_NAME if args.box_particles == 2 ** 24 else C5_NAME.replace("2e24p", "%dp" % args.box_particles)
    return name + ("_ring%d" % args.n_ring if args.n_ring and args.n_ring != 4 else "")


def load_box(ctx, fid, cfg):
    ctx.load_particles(fid, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                       rot=cfg["rot"], shift=cfg["shift"], mean_subtract=True)


def box_kw(cfg, n_steps, max_extra):
    return dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0, n_steps=n_steps, max_extra=max_extra)


def oracle_sample(cfg, theta, n_steps, max_extra=16, nthreads=None):
    """the FP64 oracle as it stands on the sampled bundles (complete traces on
    an n_steps table): its results and its rate on the host cores"""
    import oracle
    cores = nthreads or os.cpu_count() or 1
    c = oracle.Cosmology(*cfg["cosmo"])
    f = oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, L=cfg["L"], rot=cfg["rot"],
                         shift=cfg["shift"], mean_subtract=True)
    t0 = time.perf_counter()
    r = oracle.trace(c, f, cfg["z_s"], theta, nthreads=cores, **box_kw(cfg, n_steps, max_extra))
    return r, time.perf_counter() - t0, cores


def cpu_baseline_and_parity(args, cfg, ctx, P, local):
    """Parity on sampled bundles of the headline workload: the oracle (FP64,
    host cores), the mixed GPU path and the all-FP64 GPU path trace the same
    bundles on the same short table; the oracle's run is also the CPU
    baseline."""
    nb_all = len(cfg["theta"])
    idx = np.linspace(0, nb_all - 1, args.parity_bundles).astype(int)
    th = np.ascontiguousarray(cfg["theta"][idx])
    kw = box_kw(cfg, args.parity_steps, 16)
    # the mixed path traces the aligned group of 256 consecutive bundles (one
    # or two thread blocks, compact on the sky as in the full run) around each
    # sample, as one launch; the samples are compared
    grp = 256
    starts = (idx // grp) * grp
    sel = np.concatenate([np.arange(a, min(a + grp, nb_all)) for a in starts])
    pos_in = np.searchsorted(sel, idx)
    gg = ctx.trace(0, cfg["z_s"], np.ascontiguousarray(cfg["theta"][sel]), want_rays=True, **kw)
    g = {"mu": gg["mu"][pos_in], "flags": gg["flags"][pos_in], "rays": gg["rays"][pos_in]}
    c64 = P.Context(local, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    load_box(c64, 0, cfg)
    g64 = c64.trace(0, cfg["z_s"], th, want_rays=True, **kw)
    c64.close()
    o, dt, cores = oracle_sample(cfg, th, args.parity_steps)
    rel = np.abs(g["mu"] / o.mu - 1)
    rel64 = np.abs(g64["mu"] / o.mu - 1)
    beta = g["rays"][:, :, 1:3] / o.chi_s
    a_g = o.ray_theta() - beta
    a_o = o.alpha()
    da = np.linalg.norm(a_g - a_o, axis=-1) / np.linalg.norm(a_o, axis=-1)
    parity = {"bundles": int(len(idx)), "rk4_steps": args.parity_steps,
              "sample": "bundles at evenly spaced indices of the 1024^2 grid, each traced by the GPU within its "
                        "aligned group of 256 grid neighbours; complete traces to z_s = 1",
              "max_rel_dmu_mixed_vs_oracle": float(rel.max()),
              "max_rel_dalpha_mixed_vs_oracle": float(da.max()),
              "max_rel_dmu_fp64gpu_vs_oracle": float(rel64.max()),
              "flags_equal": bool(np.array_equal(g["flags"], o.flags) and np.array_equal(g64["flags"], o.flags)),
              "gate_dmu": 1e-4, "gate_dalpha": 1e-5,
              "pass": bool(rel.max() <= 1e-4 and da.max() <= 1e-5 and np.array_equal(g["flags"], o.flags))}
    base = {"value": o.n_pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d bundles x %d RK4 steps (complete traces) of the 2^24-particle box, %.1f s wall, "
                      "OpenMP over bundles" % (len(idx), args.parity_steps, dt),
            "bundles_per_s": len(idx) / dt}
    return parity, base


def batched_cones(args, cones_cfg, P, local):
    """the 512-cone batched workload in one persistent launch (CUDA graph,
    autotuned shape), then the first cones by the all-FP64 path one cone per
    launch and by the mixed batched path on exactly those cones"""
    ccfg = cones_cfg
    ctx = P.Context(local, precision=P.MIXED, autotune=1)
    ctx.set_cosmology(*ccfg["cosmo"])
    cones, npart = [], 0
    for i, c in enumerate(ccfg["cones"]):
        load_box(ctx, i, c)
        cones.append(dict(field_id=i, z_s=c["z_s"], theta=c["theta"], n_steps=c["n_steps"]))
        npart += len(c["mass"])
    kw = dict(n_ring=ccfg["n_ring"], theta_r=ccfg["theta_r"], schedule=0)
    for _ in range(args.cone_warmup):
        ctx.trace_batch(cones, **kw)
    inter, dev_ms = 0.0, 0.0
    for _ in range(args.cone_runs):
        ctx.trace_batch(cones, **kw)
        st = ctx.stats()
        inter += st["interactions"]
        dev_ms += st["device_ms"]
    rate = inter / (dev_ms / 1e3)
    shape = {k: st[k] for k in ("threads_per_block", "splits", "variant")}
    nb = sum(len(c["theta"]) for c in ccfg["cones"])
    out = {"workload": "light_cones_%dc_%ds" % (len(cones), args.cone_steps), "cones": len(cones),
           "particles": npart, "bundles": nb, "rk4_steps_per_cone": args.cone_steps, "runs": args.cone_runs,
           "interactions_per_s": rate, "bundles_per_s": nb / (dev_ms / 1e3 / args.cone_runs),
           "roofline": {"bound": "alu", "achieved": FLOPS_PER_INTERACTION * rate / 1e12, "peak": FP32_PEAK / 1e12,
                        "unit": "TFLOP/s", "frac": FLOPS_PER_INTERACTION * rate / FP32_PEAK,
                        "kernel": "k_batch_run (whole persistent launch, pair sums and FP64 stages)"},
           "launch_shape": shape, "timing": "device time of the persistent launch (CUDA events)"}
    # the first k cones: mixed batched re-run of exactly those cones vs FP64 one cone per launch
    k = min(args.fp64_cones, len(cones))
    sub = cones[:k]
    ctx.trace_batch(sub, **kw)
    rm = ctx.trace_batch(sub, **kw)
    st = ctx.stats()
    rate_k = st["interactions"] / (st["device_ms"] / 1e3)
    ctx.close()
    c64 = P.Context(local, precision=P.FP64, time_kernels=1)
    c64.set_cosmology(*ccfg["cosmo"])
    i64, d64, f64, dmu = 0.0, 0.0, 0.0, 0.0
    for i in range(k):
        c = ccfg["cones"][i]
        load_box(c64, i, c)
        r64 = c64.trace(i, c["z_s"], c["theta"], n_steps=c["n_steps"], **kw)
        s64 = c64.stats()
        i64 += s64["interactions"]
        d64 += s64["device_ms"]
        f64 += s64["force_ms"]
        dmu = max(dmu, float(np.max(np.abs(rm[i]["mu"] / r64["mu"] - 1))))
    c64.close()
    rate64 = i64 / (d64 / 1e3)
    same = {"cones": k, "interactions": i64, "mixed_batched_interactions_per_s": rate_k,
            "fp64_one_cone_per_launch_interactions_per_s": rate64, "speedup_of_mixed_batched": rate_k / rate64,
            "max_rel_dmu_mixed_vs_fp64": dmu,
            "fp64_roofline": {"bound": "alu", "kernel": "k_force_fp64",
                              "achieved": FLOPS_PER_INTERACTION * i64 / (f64 / 1e3) / 1e12,
                              "peak": FP64_PEAK / 1e12, "unit": "TFLOP/s",
                              "frac": FLOPS_PER_INTERACTION * i64 / (f64 / 1e3) / FP64_PEAK,
                              "peak_basis": PEAK64_BASIS},
            "timing": "device time of each path on the same cones (CUDA events)"}
    return out, same


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on
    the headline workload; each step a bounded sample (bundles x one RK4 step)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import inputs
    cfg = c5_config(args)
    cores = os.cpu_count() or 1
    g = inputs.rng(inputs.BASE_SEED + 5, 99, 0)
    nb = args.ref_bundles or cores

    def sample():
        th = np.ascontiguousarray(cfg["theta"][g.integers(0, len(cfg["theta"]), nb)])
        r, dt, _ = oracle_sample(cfg, th, 1, max_extra=0, nthreads=cores)
        return r.n_pairs, dt

    for _ in range(args.warmup):
        sample()
    pairs, times = 0.0, []
    for _ in range(args.steps):
        p, dt = sample()
        pairs += p
        times.append(dt)
    v = pairs / sum(times)
    smp = "%d random bundles x 1 RK4 step (4 stages) of the 2^24-particle box per step, %d host cores" % (nb, cores)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": c5_name(args), "sample": smp},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args):
    ws, rank, local = dist_env()
    import inputs
    # inputs before any GPU call: the cone generator's processes are spawned
    cones_cfg = None
    if rank == 0 and not args.no_cones:
        cones_cfg = inputs.config_c4(n_cones=args.cones, n_steps=args.cone_steps,
                                     workers=max(1, min(16, os.cpu_count() or 1)))
    cfg = c5_config(args)

    import torch

    import paper_1110_4894_gb300 as P
    from paper_1110_4894_gb300.shard import allreduce_histogram, rank_lines_of_sight
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    theta = cfg["theta"] if ws == 1 else rank_lines_of_sight(cfg["theta"], rank)
    name = c5_name(args)
    if args.bundles:  # reduced runs for checks only: a contiguous patch of the grid
        theta = theta[:args.bundles]
        name += "_patch%d" % args.bundles
    nb = len(theta)
    nr = 1 + cfg["n_ring"]
    npart = len(cfg["mass"])

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    ctx = P.Context(local, precision=P.MIXED, time_kernels=1, autotune=0 if args.no_tune else 1, variant=args.variant,
                    threads_per_block=args.tpb, splits=args.splits)
    ctx.set_cosmology(*cfg["cosmo"])
    load_box(ctx, 0, cfg)
    d_theta = torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    kw = box_kw(cfg, cfg["n_steps"], 0)
    # warm-up: step table, bundle initialiser and autotuned launch shape, then W stages
    t_b = time.perf_counter()
    ctx.trace_begin(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), **kw)
    barrier()
    begin_s = time.perf_counter() - t_b
    for _ in range(args.warmup):
        ctx.trace_advance(sp, 1)
    barrier()
    s0 = ctx.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local) as clk:
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.trace_advance(sp, 1)
            ev[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    s1 = ctx.stats()
    inter = s1["interactions"] - s0["interactions"]
    force_ms = s1["force_ms"] - s0["force_ms"]
    flaunch = s1["force_launches"] - s0["force_launches"]
    launches = s1["launches"] - s0["launches"]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    t_rank = torch.tensor([dev_s], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(t_rank, op=torch.distributed.ReduceOp.MAX)
    t_max = float(t_rank.item())
    value = inter * ws / t_max

    # end to end through the host C ABI, every rank: the particle set and a
    # slice of the bundle angles from host memory, results and muPDF back
    e2e_th = np.ascontiguousarray(theta[:args.e2e_bundles])
    ekw = box_kw(cfg, args.e2e_table, 4)
    e2e_rates, e2e_times = [], []
    hist = None
    for _ in range(max(3, args.e2e_steps)):
        barrier()
        t1 = time.perf_counter()
        load_box(ctx, 1, cfg)
        r = ctx.trace(1, cfg["z_s"], e2e_th, **ekw)
        hist = ctx.histogram(r["mu"], r["flags"], **HIST)
        barrier()
        dt = time.perf_counter() - t1
        e2e_times.append(dt)
        e2e_rates.append(ctx.stats()["interactions"] / dt)
    e2e_rank = torch.tensor([statistics.median(e2e_times)], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(e2e_rank, op=torch.distributed.ReduceOp.MAX)
    e2e_value = statistics.median(e2e_rates) * ws * statistics.median(e2e_times) / float(e2e_rank.item())
    counts, wfix, sc = hist
    if ws > 1:
        counts, wfix, sc = allreduce_histogram(counts, wfix, sc, device=dev)
    mupdf = {"bundles_binned": int(sc["n_used"]), "mean_w": sc["mean_w"], "sigma_w": sc["sigma_w"],
             "bins": HIST["bins"], "mu_range": [HIST["mu_min"], HIST["mu_max"]], "ranks": ws,
             "of": "the end-to-end leg's bundles (%d per rank, %d-step table)" % (len(e2e_th), args.e2e_table)}
    h2d = npart * 4 * 8 + len(e2e_th) * 2 * 8
    d2h = len(e2e_th) * 6 * 8 + HIST["bins"] * 16
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        ctx.close()
        return 0

    per_launch = inter / max(1, flaunch)
    avg_launch_s = force_ms / 1e3 / max(1, flaunch)
    achieved = FLOPS_PER_INTERACTION * per_launch / avg_launch_s if avg_launch_s > 0 else 0.0
    st = s1
    kname = KERNEL_NAMES.get(st["variant"], "k_force")
    traffic = PROFILED_DRAM_BYTES.get(("c5", kname, st["threads_per_block"], st["splits"]))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "bundle_stages_per_s": nb * ws * args.steps / t_max,
           "bundles_per_s": nb * ws * args.steps / t_max / (4 * cfg["n_steps"]),
           "bundles_per_s_note": "bundles per second of whole %d-step traces at the measured stage rate"
                                 % cfg["n_steps"],
           "config": {"workload": name, "particles": npart, "bundles": nb, "rays": nb * nr,
                      "replicas": int(cfg["n_rep"]), "z_s": cfg["z_s"], "box_mpc_h": 200.0,
                      "rk4_table_steps": cfg["n_steps"], "step": "one RK4 stage over every bundle",
                      "stages_before_timing": args.warmup,
                      "precision": "fp32 pair sums (chunked TwoSum), fp64 ray state, stage and prism",
                      "l2": "inputs larger than L2 (particles 268 MB, ray state 1.3 GB); no flush",
                      "launch_shape": {"threads_per_block": st["threads_per_block"], "splits": st["splits"],
                                       "cluster": st.get("cluster", 1), "kernel": kname},
                      "begin_s": begin_s},
           "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": FP32_PEAK / 1e12, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK, "traffic": traffic, "kernel": kname,
                        "flops_per_interaction": FLOPS_PER_INTERACTION, "interactions_per_launch": per_launch,
                        "avg_launch_ms": avg_launch_s * 1e3, "peak_basis": PEAK_BASIS},
           "clocks": clocks,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "samples": len(e2e_rates), "spread": [min(e2e_rates) * ws, max(e2e_rates) * ws],
                   "sample": "rt3d_load_particles (2^24 particles) + rt3d_trace of %d bundles on a %d-step table "
                             "+ rt3d_histogram, host buffers, median" % (len(e2e_th), args.e2e_table)},
           "gpu_launches": int(launches),
           "mupdf": mupdf,
           "wall_s": wall}
    if not args.no_cpu:
        out["parity"], out["cpu_baseline"] = cpu_baseline_and_parity(args, cfg, ctx, P, local)
    ctx.close()
    if cones_cfg is not None:
        out["batched_cones"], out["fp64_same_cones"] = batched_cones(args, cones_cfg, P, local)
    print(json.dumps(out))
    return 0


def nfw_cpu_baseline(cfg, n_bundles=None, n_steps=500, nthreads=None):
    """The FP64 oracle as it stands on a bounded sample: n_bundles (default:
    one per core) of the workload's bundles, traced with a shorter step table
    of the same kind.  Rate = pair evaluations / wall time."""
    import oracle
    cores = nthreads or os.cpu_count() or 1
    nb = n_bundles or cores
    th = cfg["theta"][:: max(1, len(cfg["theta"]) // nb)][:nb]
    kw = trace_kw(cfg)
    kw["n_steps"] = n_steps
    c = oracle.Cosmology(*cfg["cosmo"])
    f = oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"])
    t0 = time.perf_counter()
    r = oracle.trace(c, f, cfg["z_s"], th, nthreads=cores, **kw)
    dt = time.perf_counter() - t0
    rate = r.n_pairs / dt
    bundles_per_s = nb / dt * (n_steps / cfg["n_steps"])
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d bundles x %d RK4 steps of the workload (%d particles), %.1f s wall"
                      % (nb, n_steps, len(cfg["mass"]), dt),
            "bundles_per_s": bundles_per_s}


def run_nfw(args):
    """The NFW-halo lens test (100,000 particles, 4096 bundles, 2000 RK4 steps):
    one step = one full trace of every bundle plus its muPDF."""
    import torch

    import paper_1110_4894_gb300 as P

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, name = workload(full=not args.small)
    if args.rk4_steps:
        cfg["n_steps"] = args.rk4_steps
        name += "_rk4x%d" % args.rk4_steps
    kw = trace_kw(cfg)
    nb = cfg["theta"].shape[0]
    nr = 1 + cfg["n_ring"]
    npart = len(cfg["mass"])
    if ws > 1:  # weak scaling: every rank traces its own lines of sight of the same halo
        from paper_1110_4894_gb300.shard import rank_lines_of_sight
        cfg["theta"] = rank_lines_of_sight(cfg["theta"], rank)

    ctx = P.Context(local, precision=P.MIXED, time_kernels=1, autotune=1, variant=args.variant)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).to(dev)
    d_bout = torch.zeros(nb * 6, dtype=torch.float64, device=dev)
    d_counts = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_wfix = torch.zeros(HIST["bins"], dtype=torch.int64, device=dev)
    d_scal = torch.zeros(8, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), d_bout.data_ptr(), **kw)
        ctx.histogram_device(sp, nb, d_bout.data_ptr(), d_counts.data_ptr(), d_wfix.data_ptr(), d_scal.data_ptr(),
                             **HIST)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    force_ms, force_launches, inter, launches = 0.0, 0, 0.0, 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local) as clk:
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            st = ctx.stats()  # synchronises; reads the per-launch pair-sum events of this step
            force_ms += st["force_ms"]
            force_launches += st["force_launches"]
            inter += st["interactions"]
            launches += st["launches"] + 2
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    t_rank = torch.tensor([dev_s], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(t_rank, op=torch.distributed.ReduceOp.MAX)
    t_max = float(t_rank.item())
    # the muPDF of all ranks' bundles (outside the timed region): one exchange
    # of two integer vectors and seven sums
    from paper_1110_4894_gb300.shard import allreduce_histogram
    keys = ("n_used", "n_under", "n_over", "n_neg", "n_bad", "W_total", "mean_w", "sigma_w")
    sc = dict(zip(keys, d_scal.cpu().numpy().tolist()))
    hc, hw = d_counts.cpu().numpy().astype(np.uint64), d_wfix.cpu().numpy().view(np.uint64)
    if ws > 1:
        hc, hw, sc = allreduce_histogram(hc, hw, sc, device=dev)
    mupdf = {"bundles_binned": int(sc["n_used"]), "mean_w": sc["mean_w"], "sigma_w": sc["sigma_w"],
             "bins": HIST["bins"], "mu_range": [HIST["mu_min"], HIST["mu_max"]], "ranks": ws}
    total_inter = inter * ws
    value = total_inter / t_max
    bundles_s = nb * args.steps * ws / t_max

    # end to end through the host C ABI: particles and bundle angles up, results down
    e2e_times = []
    h2d = npart * (3 + 1 + 1) * 8 + nb * 2 * 8
    d2h = nb * 6 * 8 + HIST["bins"] * 16 + 64
    pos = np.ascontiguousarray(cfg["pos"])
    mass = np.ascontiguousarray(cfg["mass"])
    for k in range(max(3, args.e2e_steps)):
        barrier()
        t1 = time.perf_counter()
        ctx.load_particles(1, pos, mass, cfg["soft"])
        r = ctx.trace(1, cfg["z_s"], cfg["theta"], **kw)
        ctx.histogram(r["mu"], r["flags"], **HIST)
        barrier()
        e2e_times.append(time.perf_counter() - t1)
    e2e_inter = ctx.stats()["interactions"]
    e2e_value = e2e_inter * ws / statistics.median(e2e_times)

    if rank == 0:
        per_launch = inter / max(1, force_launches)
        avg_launch_s = force_ms / 1e3 / max(1, force_launches)
        achieved = FLOPS_PER_INTERACTION * per_launch / avg_launch_s if avg_launch_s > 0 else 0.0
        shape = ctx.stats()
        kname = KERNEL_NAMES.get(shape["variant"], "k_force")
        # DRAM bytes per pair-sum launch from the ncu capture of this kernel
        # (profiles/); null when the launched kernel was not captured
        traffic = None if args.small else PROFILED_DRAM_BYTES.get(
            ("nfw", kname, shape["threads_per_block"], shape["splits"]))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "bundles_per_s": bundles_s,
               "config": {"workload": name, "particles": npart, "bundles": nb, "rays": nb * nr,
                          "rk4_steps": cfg["n_steps"], "z_s": cfg["z_s"],
                          "precision": "fp32 pair sums (chunked TwoSum), fp64 ray state",
                          "l2": "256 MB buffer written between timed steps",
                          "launch_shape": {"rays_per_thread": shape["rays_per_thread"],
                                           "threads_per_block": shape["threads_per_block"],
                                           "splits": shape["splits"], "cluster": shape.get("cluster", 1),
                                           "kernel": kname}},
               "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": FP32_PEAK / 1e12,
                            "unit": "TFLOP/s", "frac": achieved / FP32_PEAK, "traffic": traffic,
                            "kernel": kname, "flops_per_interaction": FLOPS_PER_INTERACTION,
                            "interactions_per_launch": per_launch, "avg_launch_ms": avg_launch_s * 1e3,
                            "peak_basis": "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived)"},
               "clocks": clocks,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": int(launches),
               "mupdf": mupdf,
               "wall_s": wall}
        if not args.no_cpu:
            out["cpu_baseline"] = nfw_cpu_baseline(cfg, n_steps=args.cpu_steps)
        print(json.dumps(out))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c5", "nfw", "cones", "grid", "born", "box3", "box5",
                                                          "prism", "multiplane"])
    ap.add_argument("--mp-slices", type=int, default=1, help="multiplane: planes per replica")
    ap.add_argument("--mp-3d-bundles", type=int, default=256, help="multiplane: bundles also traced in 3D")
    ap.add_argument("--table-steps", type=int, default=1000, help="RK4 steps of the headline trace's table")
    ap.add_argument("--box-particles", type=int, default=2 ** 24, help="checks only: a smaller headline box")
    ap.add_argument("--bundles", type=int, default=0, help="checks only: trace the first bundles of the grid")
    ap.add_argument("--n-ring", type=int, default=0, help="checks only: rays on the bundle's ring (0: the workload's 4)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-bundles", type=int, default=16384)
    ap.add_argument("--e2e-table", type=int, default=2)
    ap.add_argument("--parity-bundles", type=int, default=16)
    ap.add_argument("--parity-steps", type=int, default=4)
    ap.add_argument("--ref-bundles", type=int, default=0, help="reference arm: bundles per step (0: one per core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cones", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="profiling: the default launch shape, no autotuning")
    ap.add_argument("--tpb", type=int, default=0, help="profiling: pair-sum threads per block (0: tuned)")
    ap.add_argument("--splits", type=int, default=0, help="profiling: pair-sum particle splits (0: tuned)")
    ap.add_argument("--cone-warmup", type=int, default=2)
    ap.add_argument("--cone-runs", type=int, default=2)
    # auxiliary workloads
    ap.add_argument("--small", action="store_true", help="reduced NFW workload for quick checks")
    ap.add_argument("--cpu-steps", type=int, default=250)
    ap.add_argument("--rk4-steps", type=int, default=0, help="override the RK4 step count (auxiliary workloads)")
    ap.add_argument("--box-bundles", type=int, default=65536, help="bundles of the 2^24-particle box (box5)")
    ap.add_argument("--fp64-bundles", type=int, default=256, help="bundles of the box run on the FP64 path")
    ap.add_argument("--grid-n", type=int, default=256, help="nodes per side of the grid workload")
    ap.add_argument("--cones", type=int, default=512)
    ap.add_argument("--cone-steps", type=int, default=16)
    ap.add_argument("--fp64-cones", type=int, default=8)
    ap.add_argument("--variant", type=int, default=0,
                    help="pair-sum kernel (0: the autotuner picks among all; 3, 4, 5: that kernel's shapes only)")
    args = ap.parse_args()
    ws = dist_env()[0]
    if ws == 1 and args.gpus > 1:  # outside torchrun: start one rank per GPU, which then report
        return subprocess.call(relaunch_command(sys.argv[1:], args.gpus, free_port()))
    if ws != args.gpus:
        print("bench.py: --gpus %d but WORLD_SIZE %d" % (args.gpus, ws), file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "nfw":
        return run_nfw(args)
    if args.workload == "multiplane":
        return run_multiplane(args)
    if args.workload == "cones":
        return run_cones(args)
    if args.workload == "grid":
        return run_grid(args)
    if args.workload == "born":
        return run_born(args)
    if args.workload == "prism":
        return run_prism(args)
    if args.workload in ("box3", "box5"):
        return run_box(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

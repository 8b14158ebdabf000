"""Shared test plumbing: load one seeded workload into both the oracle and the
CUDA library, run both, and measure the differences the parity gates use."""
import numpy as np

import oracle


def oracle_field(cfg):
    if cfg.get("replicated"):
        return oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, L=cfg["L"], rot=cfg["rot"],
                                shift=cfg["shift"], mean_subtract=cfg.get("mean_subtract", False))
    return oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"])


def gpu_load(ctx, fid, cfg):
    if cfg.get("replicated"):
        ctx.load_particles(fid, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"],
                           rot=cfg["rot"], shift=cfg["shift"], mean_subtract=cfg.get("mean_subtract", False))
    else:
        ctx.load_particles(fid, cfg["pos"], cfg["mass"], cfg["soft"])


def trace_kw(cfg):
    return dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
                lens_chi=cfg.get("lens_chi", 0.0), asinh_s=cfg.get("asinh_s", 1.0), phase=cfg.get("phase", 0.0))


def run_oracle(cfg, theta, cosmo=None, christoffel=0, nthreads=None):
    cosmo = cosmo or oracle.Cosmology(*cfg["cosmo"])
    return oracle.trace(cosmo, oracle_field(cfg), cfg["z_s"], theta, christoffel=christoffel, nthreads=nthreads,
                        **trace_kw(cfg))


def rel_mu(mu_gpu, mu_orc):
    return np.abs(mu_gpu / mu_orc - 1.0)


def rel_alpha(rays_gpu, res_orc):
    """|delta alpha| / |alpha| per ray, alpha = theta - beta"""
    th = res_orc.ray_theta()
    beta_g = rays_gpu[:, :, 1:3] / res_orc.chi_s
    a_g = th - beta_g
    a_o = res_orc.alpha()
    return np.linalg.norm(a_g - a_o, axis=-1) / np.linalg.norm(a_o, axis=-1)

"""Parity at the full particle counts of the cosmological boxes: the 2^21-particle
100/h Mpc box (z_s = 0.5) and the 2^24-particle 200/h Mpc box (z_s = 1), each
replicated along the line of sight with random rotations and shifts and mean
subtraction.  The GPU traces a contiguous patch of the full-resolution bundle
grid (256^2 and 1024^2 bundles on the sky: the first tiles of the grid order,
so each thread block covers the same sky extent as in the full run); the
oracle recomputes a sample of them with the same shortened step table, and the
muPDF of the sample is compared bin by bin."""
import numpy as np
import pytest

import inputs
import oracle
from _cases import gpu_load, oracle_field, rel_alpha, rel_mu, trace_kw

pytestmark = pytest.mark.gpu


def _run(cfg, n_sample, cosmo):
    import paper_1110_4894_gb300 as P
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    nb = len(cfg["theta"])
    assert np.all(g["flags"] & (P.F_NOCROSS | P.F_NONFINITE) == 0)
    idx = np.linspace(0, nb - 1, n_sample).astype(int)
    o = oracle.trace(cosmo, oracle_field(cfg), cfg["z_s"], cfg["theta"][idx], **trace_kw(cfg))
    assert np.array_equal(g["flags"][idx], o.flags)
    assert np.array_equal(g["steps"][idx], o.steps)
    dm = rel_mu(g["mu"][idx], o.mu)
    da = rel_alpha(g["rays"][idx], o)
    assert dm.max() < 1e-4, dm
    assert da.max() < 1e-5, da
    # muPDF of the sample: identical counts unless a magnification sits within
    # the two sides' difference of a bin edge (then one bundle moves by one bin)
    h = dict(bins=200, mu_min=0.9, mu_max=1.2)
    cg, wg, sg = ctx.histogram(g["mu"][idx], g["flags"][idx], **h)
    co, wo, so = oracle.histogram(o.mu, o.flags, **h)
    edges = np.log10(h["mu_min"]) + np.arange(h["bins"] + 1) * (np.log10(h["mu_max"] / h["mu_min"]) / h["bins"])
    near = [np.min(np.abs(edges - np.log10(abs(m)))) < abs(np.log10(abs(m)) - np.log10(abs(mo)))
            for m, mo in zip(g["mu"][idx], o.mu)]
    assert np.sum(np.abs(cg.astype(int) - co.astype(int))) <= 2 * int(np.sum(near))
    assert abs(sg["mean_w"] / so["mean_w"] - 1) < 1e-4
    return ctx.stats()


def test_box_2e21_particles_sampled(cosmo):
    cfg = inputs.config_c3(n_steps=100)
    cfg["theta"] = cfg["theta"][:4096]  # first 64 tiles of 8 x 8 (a 16 x 256 strip) of the 256^2 grid
    st = _run(cfg, 16, cosmo)
    assert st["interactions"] > 0


def test_box_2e24_particles_sampled(cosmo):
    cfg = inputs.config_c5(n_steps=12)
    cfg["theta"] = cfg["theta"][:1024]  # first 16 tiles (an 8 x 128 strip) of the 1024^2 grid
    st = _run(cfg, 8, cosmo)
    assert st["interactions"] > 0

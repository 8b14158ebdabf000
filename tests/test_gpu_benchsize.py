"""Parity at the sizes the benchmark runs:

- the batched light-cone workload at its real ranges (64 cones with 1e3-1e6
  particles, 256-4096 bundles, z_s 0.3-1.5, 16 RK4 steps each) in one
  persistent launch with the autotuner's shape: 8 bundles of each of 8 cones
  spread over the particle-count range against the FP64 oracle on the same
  step tables, and the all-FP64 path one cone per launch on the same bundles;
- the grid path (Sec. 3.3, App. B) on a 128^3 grid of the NFW workload's
  halo (100,000 particles, all 4096 bundles, 2000 RK4 steps), sampled against
  the oracle's grid path;
- one replica of the Sec. 5.2 sampling region (256^3 particles in a 50/h Mpc
  box, its prism in 8 cubes of 128^3 nodes): node values and a trace across
  the cubes against the oracle."""
import math

import numpy as np
import pytest

import inputs
import oracle
import oracle.grid as G
from _cases import rel_alpha, rel_mu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cones64():
    return inputs.config_c4(n_cones=64, n_steps=16, workers=8)


def _field(c):
    return oracle.MassField(c["pos"], c["mass"], c["soft"], replicated=True, L=c["L"], rot=c["rot"], shift=c["shift"],
                            mean_subtract=True)


def test_batched_cones_at_benchmark_ranges(cones64, cosmo):
    import paper_1110_4894_gb300 as P
    cfg = cones64
    ctx = P.Context(0, precision=P.MIXED, autotune=1)
    ctx.set_cosmology(*cfg["cosmo"])
    cones = []
    for i, c in enumerate(cfg["cones"]):
        ctx.load_particles(i, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"], rot=c["rot"],
                           shift=c["shift"], mean_subtract=True)
        cones.append(dict(field_id=i, z_s=c["z_s"], theta=c["theta"], n_steps=c["n_steps"]))
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    res = ctx.trace_batch(cones, want_rays=True, **kw)
    st = ctx.stats()
    assert st["splits"] > 100  # thousands of work items through the queue
    npart = np.array([len(c["mass"]) for c in cfg["cones"]])
    assert npart.min() < 1e4 and npart.max() > 3e5
    picks = np.argsort(npart)[np.linspace(0, len(npart) - 1, 8).astype(int)]
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    for i in picks:
        c = cfg["cones"][i]
        nb = len(c["theta"])
        idx = np.linspace(0, nb - 1, 8).astype(int)
        o = oracle.trace(cosmo, _field(c), c["z_s"], c["theta"][idx], n_steps=c["n_steps"], **kw)
        r = {k: res[i][k][idx] for k in ("mu", "flags", "steps", "rays")}
        assert np.array_equal(r["flags"], o.flags) and np.array_equal(r["steps"], o.steps), i
        assert rel_mu(r["mu"], o.mu).max() < 1e-4, (i, rel_mu(r["mu"], o.mu).max())
        assert rel_alpha(r["rays"], o).max() < 1e-5, (i, rel_alpha(r["rays"], o).max())
        # the all-FP64 path, one cone per launch, on the same bundles
        c64.load_particles(0, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"], rot=c["rot"],
                           shift=c["shift"], mean_subtract=True)
        g64 = c64.trace(0, c["z_s"], c["theta"][idx], want_rays=True, n_steps=c["n_steps"], **kw)
        assert np.array_equal(g64["flags"], o.flags) and np.array_equal(g64["steps"], o.steps)
        assert rel_mu(g64["mu"], o.mu).max() < 1e-9
        assert rel_mu(r["mu"], g64["mu"]).max() < 1e-4


def test_grid_128_nfw_full_size_sampled(cosmo):
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_c2()
    n = 128
    half = 2.2 * cfg["info"]["r200_phys"] * (1 + cfg["z_l"])
    h = 2 * half / (n - 1)
    lo = np.array([-half, -half, cfg["chi_l"] - half])
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
              lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    gf = G.GridField(cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    nb = cfg["theta"].shape[0]
    idx = np.linspace(0, nb - 1, 16).astype(int)
    o = oracle.trace(cosmo, gf.field(), cfg["z_s"], cfg["theta"][idx], **kw)
    for prec, tol_mu, tol_a in ((P.FP64, 1e-9, 1e-9), (P.MIXED, 1e-6, 1e-6)):
        ctx = P.Context(0, precision=prec)
        ctx.set_cosmology(*cfg["cosmo"])
        ctx.load_grid(0, cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
        nodes = ctx.grid_nodes(0)
        if prec == P.FP64:
            for f in range(4):
                assert np.max(np.abs(nodes[f] - gf.val[f])) <= 1e-11 * np.max(np.abs(gf.val[f]))
        g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **kw)
        r = {k: g[k][idx] for k in ("mu", "flags", "steps", "rays")}
        assert np.array_equal(r["flags"], o.flags) and np.array_equal(r["steps"], o.steps)
        assert rel_mu(r["mu"], o.mu).max() < tol_mu
        assert rel_alpha(r["rays"], o).max() < tol_a
        ctx.close()


def test_prism_one_replica_eight_cubes_of_128(cosmo):
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_prism(n_steps=200)
    rot, shift = cfg["rot"][:1], cfg["shift"][:1]
    L, cubes, n = cfg["L"], cfg["cubes"], cfg["grid_n"]
    bg = G.BoxGridField(cfg["pos"], cfg["mass"], cfg["soft"], L, rot, shift, cubes=cubes, n=n)
    ctx = P.Context(0, precision=P.FP64)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_grid_box(0, cfg["pos"], cfg["mass"], cfg["soft"], L, rot, shift, cubes, n, n_int=2, mean_subtract=True)
    nodes = ctx.grid_nodes(0)
    g = inputs.rng(66)
    for c, gf in enumerate(bg.grids):
        # sampled node values of every cube (the whole tables are 8 x 4 x 128^3)
        ii = g.integers(0, n, (2000, 3))
        for f in range(4):
            a = nodes[c, f][ii[:, 0], ii[:, 1], ii[:, 2]]
            b = gf.val[f][ii[:, 0], ii[:, 1], ii[:, 2]]
            assert np.max(np.abs(a - b)) <= 1e-11 * max(np.max(np.abs(gf.val[f])), 1e-300), (c, f)
    # bundles inside the prism to a source plane in the replica's last cube
    W = L / cubes
    chi_s = 0.95 * L
    z_s = cosmo.z_of_chi(chi_s)
    th = g.uniform(-0.4, 0.4, (24, 2)) * W / chi_s
    kw = dict(n_ring=4, theta_r=cfg["theta_r"], schedule=0, n_steps=200)
    o = oracle.trace(cosmo, bg.field(), z_s, th, **kw)
    for prec, tol_mu, tol_a in ((P.FP64, 1e-9, 1e-8), (P.MIXED, 1e-6, 1e-5)):
        c2 = P.Context(0, precision=prec)
        c2.set_cosmology(*cfg["cosmo"])
        c2.load_grid_box(1, cfg["pos"], cfg["mass"], cfg["soft"], L, rot, shift, cubes, n, n_int=2,
                         mean_subtract=True)
        r = c2.trace(1, z_s, th, want_rays=True, **kw)
        assert np.array_equal(r["flags"], o.flags) and np.array_equal(r["steps"], o.steps)
        assert rel_mu(r["mu"], o.mu).max() < tol_mu
        assert rel_alpha(r["rays"], o).max() < tol_a
        c2.close()

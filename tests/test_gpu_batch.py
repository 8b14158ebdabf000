"""The batched trace (many uneven light cones in one persistent launch,
recorded in a CUDA graph) against the FP64 oracle per cone, against the
all-FP64 path run one cone per launch, and against itself on replay."""
import numpy as np
import pytest

import inputs
import oracle
from _cases import rel_alpha, rel_mu

pytestmark = pytest.mark.gpu


def _cones(n_cones=5, seed=inputs.BASE_SEED + 44):
    cfg = inputs.config_c4(n_cones=n_cones, n_steps=40, seed=seed, n_min=300, n_max=3000, b_min=4, b_max=24,
                           zs_lo=0.02, zs_hi=0.05, L_h=20.0, margin_h=2.0)
    for i, c in enumerate(cfg["cones"]):
        c["n_steps"] = 30 + 7 * i  # uneven step tables
    return cfg


def _load(ctx, cfg):
    for i, c in enumerate(cfg["cones"]):
        ctx.load_particles(i, c["pos"], c["mass"], c["soft"], replicated=True, box_length=c["L"], rot=c["rot"],
                           shift=c["shift"], mean_subtract=True)
    return [dict(field_id=i, z_s=c["z_s"], theta=c["theta"], n_steps=c["n_steps"]) for i, c in enumerate(cfg["cones"])]


def _oracle(cfg, cosmo, i):
    c = cfg["cones"][i]
    f = oracle.MassField(c["pos"], c["mass"], c["soft"], replicated=True, L=c["L"], rot=c["rot"], shift=c["shift"],
                         mean_subtract=True)
    return oracle.trace(cosmo, f, c["z_s"], c["theta"], n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0,
                        n_steps=c["n_steps"])


@pytest.fixture(scope="module")
def batch_case(cosmo):
    cfg = _cones()
    orc = [_oracle(cfg, cosmo, i) for i in range(len(cfg["cones"]))]
    return cfg, orc


def test_batch_mixed_matches_oracle(batch_case):
    import paper_1110_4894_gb300 as P
    cfg, orc = batch_case
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    cones = _load(ctx, cfg)
    res = ctx.trace_batch(cones, want_rays=True, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    for r, o in zip(res, orc):
        assert np.array_equal(r["flags"], o.flags)
        assert np.array_equal(r["steps"], o.steps)
        assert rel_mu(r["mu"], o.mu).max() < 1e-4
        assert rel_alpha(r["rays"], o).max() < 1e-5
    st = ctx.stats()
    want = sum(int(np.sum(np.maximum(o.steps, 0))) * 4 * len(c["mass"]) for o, c in zip(orc, cfg["cones"]))
    assert st["interactions"] >= want
    # graph replay: identical results
    res2 = ctx.trace_batch(cones, want_rays=True, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    for r, r2 in zip(res, res2):
        assert np.array_equal(r["mu"], r2["mu"]) and np.array_equal(r["rays"], r2["rays"])


def test_batch_fp64_one_cone_per_launch(batch_case):
    import paper_1110_4894_gb300 as P
    cfg, orc = batch_case
    ctx = P.Context(0, precision=P.FP64)
    ctx.set_cosmology(*cfg["cosmo"])
    cones = _load(ctx, cfg)
    res = ctx.trace_batch(cones, want_rays=True, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    for r, o in zip(res, orc):
        assert np.array_equal(r["flags"], o.flags)
        assert rel_mu(r["mu"], o.mu).max() < 1e-9


def test_batch_autotuned_and_shapes(batch_case):
    import paper_1110_4894_gb300 as P
    cfg, orc = batch_case
    # default (expanded two-bundle kernel), tuned, the bundle-centric kernel, fixed shapes
    for kw in (dict(), dict(autotune=1), dict(variant=3), dict(variant=5, splits=2),
               dict(threads_per_block=256, splits=4), dict(threads_per_block=64, splits=1)):
        ctx = P.Context(0, precision=P.MIXED, **kw)
        ctx.set_cosmology(*cfg["cosmo"])
        cones = _load(ctx, cfg)
        res = ctx.trace_batch(cones, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
        for r, o in zip(res, orc):
            assert rel_mu(r["mu"], o.mu).max() < 1e-4
        st = ctx.stats()
        if kw.get("variant") in (3, 5):
            assert st["variant"] == kw["variant"]
        elif not kw:
            assert st["variant"] == 5 and st["threads_per_block"] == 64
        ctx.close()


def test_batch_isolated_and_mixed_fields(cosmo):
    # cones of different kinds in one launch: an isolated NFW halo with
    # per-particle softening next to a replicated box
    import paper_1110_4894_gb300 as P
    c2 = inputs.config_c2(n_particles=2000, n_side=2, n_steps=80)
    box = _cones(n_cones=1)
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    g = inputs.rng(1)
    soft = g.uniform(0.003, 0.008, 2000)
    ctx.load_particles(0, c2["pos"], c2["mass"], soft)
    b = box["cones"][0]
    ctx.load_particles(1, b["pos"], b["mass"], b["soft"], replicated=True, box_length=b["L"], rot=b["rot"],
                       shift=b["shift"], mean_subtract=True)
    # one bundle option set for both: the asinh schedule centred on the halo
    kw = dict(n_ring=4, theta_r=c2["theta_r"], schedule=1, lens_chi=c2["lens_chi"], asinh_s=c2["asinh_s"])
    res = ctx.trace_batch([dict(field_id=0, z_s=0.5, theta=c2["theta"], n_steps=80),
                           dict(field_id=1, z_s=b["z_s"], theta=b["theta"], n_steps=60)], **kw)
    o0 = oracle.trace(cosmo, oracle.MassField(c2["pos"], c2["mass"], soft), 0.5, c2["theta"], n_steps=80, **kw)
    fb = oracle.MassField(b["pos"], b["mass"], b["soft"], replicated=True, L=b["L"], rot=b["rot"], shift=b["shift"],
                          mean_subtract=True)
    o1 = oracle.trace(cosmo, fb, b["z_s"], b["theta"], n_steps=60, **kw)
    assert rel_mu(res[0]["mu"], o0.mu).max() < 1e-4
    assert rel_mu(res[1]["mu"], o1.mu).max() < 1e-4


def test_watchdog_expires_and_context_survives(batch_case):
    # failure detection without a GPU fault: the persistent kernel's bounded
    # barrier wait, run on a word nothing sets, gives up after its limit and
    # reports ETIMEOUT; the context then still traces
    import time

    import paper_1110_4894_gb300 as P
    cfg, orc = batch_case
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    t0 = time.perf_counter()
    rc = ctx.watchdog_selftest(0.2)
    dt = time.perf_counter() - t0
    assert rc == P._binding.ETIMEOUT
    assert 0.19 < dt < 5.0
    cones = _load(ctx, cfg)
    res = ctx.trace_batch(cones, n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=0)
    assert rel_mu(res[0]["mu"], orc[0].mu).max() < 1e-4

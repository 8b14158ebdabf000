"""Parity at the benchmark's full size and launch configuration: the NFW-halo
workload (100,000 particles, 4096 bundles, 2000 RK4 steps) traced on the GPU
exactly as bench.py times it; the oracle recomputes 16 sampled bundles."""
import numpy as np
import pytest

import inputs
from _cases import gpu_load, rel_alpha, rel_mu, run_oracle, trace_kw

pytestmark = pytest.mark.gpu


def test_nfw_full_size_sampled(cosmo):
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_c2()
    ctx = P.Context(0, precision=P.MIXED, time_kernels=1, autotune=1)  # as bench.py: the tuner's shape
    ctx.set_cosmology(*cfg["cosmo"])
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    nb = cfg["theta"].shape[0]
    assert np.all(g["flags"] & (P.F_NOCROSS | P.F_NONFINITE) == 0)
    idx = np.linspace(0, nb - 1, 16).astype(int)
    o = run_oracle(cfg, cfg["theta"][idx], cosmo)
    assert np.array_equal(g["flags"][idx], o.flags)
    dm = rel_mu(g["mu"][idx], o.mu)
    da = rel_alpha(g["rays"][idx], o)
    assert dm.max() < 1e-4, dm
    assert da.max() < 1e-5, da
    st = ctx.stats()
    # every active ray meets every particle at every stage
    assert st["interactions"] >= nb * 5 * 100000 * 4 * cfg["n_steps"] * 0.99


def test_nfw_full_size_ring_of_eight_sampled(cosmo):
    """The paper's bundle (8 rays on a polygon around the central ray, Sec.
    3.1 and Sec. 5.2) on the full NFW workload: mixed precision on all 4096
    bundles against the oracle on 8 sampled bundles, and the all-FP64 path
    on those 8 bundles against the oracle to rounding."""
    import paper_1110_4894_gb300 as P
    cfg = inputs.config_c2()
    cfg["n_ring"] = 8
    cfg["phase"] = 0.2
    ctx = P.Context(0, precision=P.MIXED, autotune=1)
    ctx.set_cosmology(*cfg["cosmo"])
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    nb = cfg["theta"].shape[0]
    assert np.all(g["flags"] & (P.F_NOCROSS | P.F_NONFINITE) == 0)
    idx = np.linspace(0, nb - 1, 8).astype(int)
    o = run_oracle(cfg, cfg["theta"][idx], cosmo)
    assert np.array_equal(g["flags"][idx], o.flags)
    assert rel_mu(g["mu"][idx], o.mu).max() < 1e-4
    assert rel_alpha(g["rays"][idx], o).max() < 1e-5
    # the two-bundle kernel with expanded separations on the same bundles
    c5 = P.Context(0, precision=P.MIXED, autotune=0, variant=5)
    c5.set_cosmology(*cfg["cosmo"])
    gpu_load(c5, 0, cfg)
    g5 = c5.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    assert c5.stats()["variant"] == 5
    assert np.array_equal(g5["flags"][idx], o.flags)
    assert rel_mu(g5["mu"][idx], o.mu).max() < 1e-4
    assert rel_alpha(g5["rays"][idx], o).max() < 1e-5
    c64 = P.Context(0, precision=P.FP64)
    c64.set_cosmology(*cfg["cosmo"])
    gpu_load(c64, 0, cfg)
    g64 = c64.trace(0, cfg["z_s"], cfg["theta"][idx], want_rays=True, **trace_kw(cfg))
    assert np.array_equal(g64["flags"], o.flags) and np.array_equal(g64["steps"], o.steps)
    assert rel_mu(g64["mu"], o.mu).max() < 1e-9
    assert rel_alpha(g64["rays"], o).max() < 1e-9

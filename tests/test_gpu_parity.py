"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Gates: mixed precision |d alpha/alpha| <= 1e-5 per ray and
|d mu/mu| <= 1e-4 per bundle; the all-FP64 path agrees to rounding."""
import math

import numpy as np
import pytest

import inputs
import oracle
from _cases import gpu_load, oracle_field, rel_alpha, rel_mu, run_oracle, trace_kw

pytestmark = pytest.mark.gpu

ALPHA_GATE, MU_GATE = 1e-5, 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_1110_4894_gb300 as P
    return P


def ctx_for(P, precision, **kw):
    c = P.Context(0, precision=precision, **kw)
    c.set_cosmology(0.3, 0.7, 0.7)
    return c


def test_schedule_matches_oracle(P, cosmo):
    ctx = ctx_for(P, P.MIXED)
    for z_s, kind, n, chi_l, s in ((0.5, 0, 1000, 0.0, 1.0), (0.5, 1, 2000, cosmo.chi(0.25), 5e-3),
                                   (1.3, 0, 37, 0.0, 1.0), (0.3, 1, 500, 600.0, 0.02)):
        dl, chi = ctx.schedule(z_s, kind, n, chi_l, s)
        dl_o, _ = cosmo.schedule(cosmo.chi(z_s), kind, n, chi_l, s)
        assert abs(chi / cosmo.chi(z_s) - 1) < 1e-13
        assert np.max(np.abs(dl / dl_o - 1)) < 1e-9
        assert abs(dl.sum() / dl_o.sum() - 1) < 1e-13


def _cloud(n, seed, centre=(0.0, 0.0, 800.0), scale=0.3, per_particle_soft=False):
    g = inputs.rng(seed)
    pos = inputs.quantize(np.asarray(centre) + g.normal(size=(n, 3)) * scale)
    mass = g.uniform(0.5, 2.0, n) * 1e10
    soft = g.uniform(0.002, 0.02, n) if per_particle_soft else 0.01
    return pos, mass, soft


PRECISIONS = ["fp64", "mixed", "mixed-scalar", "mixed-packed", "mixed-bundle1", "mixed-bundle2"]
VARIANT = {"mixed": 0, "mixed-scalar": 1, "mixed-packed": 2, "mixed-bundle1": 3, "mixed-bundle2": 4}


def ctx_prec(P, precision, **kw):
    if precision == "fp64":
        return ctx_for(P, P.FP64, **kw)
    return ctx_for(P, P.MIXED, variant=VARIANT[precision], **kw)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n", [1, 300, 3 * 256 + 37])
@pytest.mark.parametrize("pps", [False, True])
@pytest.mark.parametrize("equal_mass", [False, True])
def test_potential_isolated(P, precision, n, pps, equal_mass):
    pos, mass, soft = _cloud(n, 5 + n, per_particle_soft=pps)
    if equal_mass:
        mass = np.full(n, 1.3e10)
    ctx = ctx_prec(P, precision)
    ctx.load_particles(3, pos, mass, soft)
    g = inputs.rng(99)
    pts = np.concatenate([np.array([0.0, 0.0, 800.0]) + g.normal(size=(500, 3)) * 0.4,
                          np.array([[0.0, 0.0, 0.0], [3.0, -2.0, 500.0], pos[0]])])
    out = ctx.potential(3, pts)
    ref = oracle.potential(oracle.MassField(pos, mass, soft), pts)
    scale_phi = np.abs(ref[:, 0])
    scale_g = np.linalg.norm(ref[:, 1:], axis=1)
    err_phi = np.abs(out[:, 0] - ref[:, 0]) / scale_phi
    err_g = np.linalg.norm(out[:, 1:] - ref[:, 1:], axis=1) / np.maximum(scale_g, 1e-300)
    if precision == "fp64":
        assert err_phi.max() < 1e-12 and err_g.max() < 1e-11
    else:
        assert err_phi.max() < 2e-6
        assert np.percentile(err_g, 99) < 5e-6 and err_g.max() < 5e-5


def _small_box(n=4000, seed=inputs.BASE_SEED + 33, L_h=20.0, n_halos=12, n_rep=6):
    L = inputs.box_length(L_h / 0.7)
    pos, mass, info = inputs.halo_box(n, L, n_halos, seed)
    rot, shift = inputs.replicas(n_rep, L, seed)
    return dict(pos=pos, mass=mass, soft=0.016 / 0.7, L=L, rot=rot, shift=shift)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("mean_subtract", [False, True])
def test_potential_replicated(P, precision, mean_subtract):
    b = _small_box()
    ctx = ctx_prec(P, precision)
    ctx.load_particles(1, b["pos"], b["mass"], b["soft"], replicated=True, box_length=b["L"], rot=b["rot"],
                       shift=b["shift"], mean_subtract=mean_subtract)
    g = inputs.rng(7)
    L = b["L"]
    rep = g.integers(0, 6, 400).astype(np.int32)
    pts = np.stack([g.uniform(-0.5, 0.5, 400) * L, g.uniform(-0.5, 0.5, 400) * L, (rep + g.random(400)) * L], 1)
    pts[:4, 2] = rep[:4] * L  # on a replica face
    out = ctx.potential(1, pts, rep)
    f = oracle.MassField(b["pos"], b["mass"], b["soft"], replicated=True, L=L, rot=b["rot"], shift=b["shift"],
                         mean_subtract=mean_subtract)
    ref = oracle.potential(f, pts, rep)
    raw = oracle.potential(oracle.MassField(b["pos"], b["mass"], b["soft"], replicated=True, L=L, rot=b["rot"],
                                            shift=b["shift"]), pts, rep)
    # errors relative to the particle field itself (mean subtraction cancels most of it)
    sc_phi = np.abs(raw[:, 0])
    sc_g = np.linalg.norm(raw[:, 1:], axis=1)
    e_phi = np.abs(out[:, 0] - ref[:, 0]) / sc_phi
    e_g = np.linalg.norm(out[:, 1:] - ref[:, 1:], axis=1) / sc_g
    if precision == "fp64":
        assert e_phi.max() < 1e-12 and e_g.max() < 1e-11
    else:
        assert e_phi.max() < 2e-6 and e_g.max() < 2e-5


def test_c1_point_lens_fp64(P, cosmo):
    cfg = inputs.config_c1()
    ctx = ctx_for(P, P.FP64)
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    o = run_oracle(cfg, cfg["theta"], cosmo)
    ok = np.abs(np.abs(cfg["x"]) - 1) > 0.05
    assert rel_mu(g["mu"], o.mu)[ok].max() < 1e-9
    assert rel_alpha(g["rays"], o).max() < 1e-10
    assert np.array_equal(g["flags"], o.flags)
    assert np.array_equal(g["steps"], o.steps)
    for k in ("kappa", "gamma1", "gamma2", "omega"):
        assert np.allclose(g[k][ok], getattr(o, k)[ok], rtol=1e-8, atol=1e-11)


def _c2_small(n_particles=20000, n_side=4, n_steps=300):
    cfg = inputs.config_c2(n_particles=n_particles, n_side=n_side, n_steps=n_steps)
    return cfg


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n_ring", [4, 8])
def test_c2_small_nfw(P, cosmo, precision, n_ring):
    # rings of 8 are the paper's bundle (Sec. 3.1, Sec. 5.2); phase turns the polygon
    cfg = _c2_small()
    cfg["n_ring"] = n_ring
    if n_ring == 8:
        cfg["phase"] = 0.3
    ctx = ctx_prec(P, precision)
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    o = run_oracle(cfg, cfg["theta"], cosmo)
    assert np.array_equal(g["flags"], o.flags)
    da, dm = rel_alpha(g["rays"], o), rel_mu(g["mu"], o.mu)
    if precision == "fp64":
        assert da.max() < 1e-10 and dm.max() < 1e-9
    else:
        assert da.max() < ALPHA_GATE and dm.max() < MU_GATE
    st = ctx.stats()
    assert st["interactions"] > 0


@pytest.mark.parametrize("variant", [3, 5])
@pytest.mark.parametrize("n_side", [4, 12])
def test_ring_of_eight_kernels(P, cosmo, variant, n_side):
    # the paper's 8-ray bundle through each pair-sum kernel that serves it:
    # one bundle per thread (3) and two per thread with the expanded
    # separations (5, blocks of 128 bundles: 16 bundles fill part of one
    # block, 144 one and part of a second)
    cfg = _c2_small(n_particles=6000, n_side=n_side, n_steps=120)
    cfg["n_ring"] = 8
    cfg["phase"] = 0.3
    ctx = ctx_for(P, P.MIXED, variant=variant)
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    assert ctx.stats()["variant"] == variant
    o = run_oracle(cfg, cfg["theta"], cosmo)
    assert np.array_equal(g["flags"], o.flags)
    assert rel_mu(g["mu"], o.mu).max() < MU_GATE
    assert rel_alpha(g["rays"], o).max() < ALPHA_GATE


@pytest.mark.parametrize("precision", PRECISIONS)
def test_box_replicas_mean_subtracted(P, cosmo, precision):
    b = _small_box()
    L = b["L"]
    z_s = 0.02
    chi_s = cosmo.chi(z_s)
    n_rep = int(math.ceil(chi_s / L)) + 1
    assert n_rep <= 6
    half = (0.5 * L - 2.0) / chi_s
    theta = inputs.bundle_grid(-half, half, 4)
    cfg = dict(b, replicated=True, mean_subtract=True, cosmo=(0.3, 0.7, 0.7), z_s=z_s, n_ring=4,
               theta_r=math.radians(1 / 3600), schedule=0, n_steps=120)
    ctx = ctx_prec(P, precision)
    gpu_load(ctx, 2, cfg)
    g = ctx.trace(2, z_s, theta, want_rays=True, **trace_kw(cfg))
    o = run_oracle(cfg, theta, cosmo)
    assert np.array_equal(g["flags"], o.flags)
    da, dm = rel_alpha(g["rays"], o), rel_mu(g["mu"], o.mu)
    if precision == "fp64":
        # here alpha ~ 1e-7 rad while theta ~ 0.2 rad: alpha = theta - beta keeps
        # only ~9 significant digits of the FP64 positions
        assert da.max() < 1e-6 and dm.max() < 1e-9
    else:
        assert da.max() < ALPHA_GATE and dm.max() < MU_GATE


def test_empty_field_is_unlensed(P, cosmo):
    ctx = ctx_for(P, P.MIXED)
    ctx.load_particles(0, np.zeros((0, 3)), np.zeros(0), 0.0)
    th = np.array([[0.0, 0.0], [1e-3, -2e-3]])
    g = ctx.trace(0, 0.5, th, want_rays=True, n_steps=64)
    assert np.all(np.abs(g["mu"] - 1) < 1e-9) and np.all(g["flags"] == 0)
    assert np.all(np.abs(g["rays"][:, :, 1:3] / cosmo.chi(0.5) - oracle.trace(
        cosmo, oracle.MassField(np.zeros((0, 3)), np.zeros(0), 0.0), 0.5, th, theta_r=1e-6,
        n_steps=64).beta()) < 1e-15)


def test_ring_of_eight_and_derived_symbols(P, cosmo):
    cfg = _c2_small(n_particles=3000, n_side=2, n_steps=150)
    cfg["n_ring"] = 8
    for ch in (0, 1):
        ctx = ctx_for(P, P.MIXED, christoffel=ch)
        gpu_load(ctx, 0, cfg)
        g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
        o = run_oracle(cfg, cfg["theta"], cosmo, christoffel=ch)
        assert rel_mu(g["mu"], o.mu).max() < MU_GATE
        assert rel_alpha(g["rays"], o).max() < ALPHA_GATE


def test_histogram_bit_exact(P):
    g = inputs.rng(17)
    mu = np.exp(g.uniform(np.log(0.3), np.log(8.0), 20000))
    mu[::9] *= -1
    flags = np.zeros(mu.size, np.int32)
    flags[::101] = oracle.F_NOCROSS
    mu[7] = np.inf
    ctx = ctx_for(P, P.MIXED)
    for bins, lo, hi in ((200, 0.5, 5.0), (37, 0.9, 1.7), (1, 0.1, 10.0)):
        c_g, w_g, s_g = ctx.histogram(mu, flags, bins, lo, hi)
        c_o, w_o, s_o = oracle.histogram(mu, flags, bins, lo, hi)
        assert np.array_equal(c_g, c_o) and np.array_equal(w_g, w_o)
        for k in ("n_used", "n_under", "n_over", "n_neg", "n_bad"):
            assert s_g[k] == s_o[k]
        for k in ("W_total", "mean_w", "sigma_w"):
            assert abs(s_g[k] / s_o[k] - 1) < 1e-12


def test_shear_histogram_bit_exact(P):
    g = inputs.rng(18)
    n = 20000
    gam = np.exp(g.uniform(np.log(1e-4), np.log(0.8), n))
    ang = g.uniform(0, 2 * np.pi, n)
    g1, g2 = gam * np.cos(ang), gam * np.sin(ang)
    g1[::97], g2[::97] = 0.0, 0.0
    mu = np.exp(g.uniform(np.log(0.4), np.log(6.0), n))
    mu[::13] *= -1
    flags = np.zeros(n, np.int32)
    flags[::211] = oracle.F_NONFINITE
    g1[5] = np.nan
    ctx = ctx_for(P, P.MIXED)
    for bins, lo, hi in ((200, 1e-3, 0.5), (23, 0.01, 0.2), (1, 1e-5, 1.0)):
        c_g, w_g, s_g = ctx.shear_histogram(mu, g1, g2, flags, bins, lo, hi)
        c_o, w_o, s_o = oracle.shear_histogram(mu, g1, g2, flags, bins, lo, hi)
        assert np.array_equal(c_g, c_o) and np.array_equal(w_g, w_o)
        for k in ("n_used", "n_under", "n_over", "n_neg", "n_bad"):
            assert s_g[k] == s_o[k]
        for k in ("W_total", "mean_w", "sigma_w"):
            assert abs(s_g[k] / s_o[k] - 1) < 1e-12


def test_errors_are_reported(P):
    ctx = P.Context(0)
    with pytest.raises(P.Rt3dError) as e:
        ctx.trace(0, 0.5, np.zeros((1, 2)))
    assert e.value.code == -6
    ctx.set_cosmology()
    with pytest.raises(P.Rt3dError) as e:
        ctx.trace(5, 0.5, np.zeros((1, 2)))
    assert e.value.code == -7
    with pytest.raises(P.Rt3dError) as e:
        ctx.set_cosmology(0.3, 0.8, 0.7)
    assert e.value.code == -1
    with pytest.raises(P.Rt3dError):
        ctx.load_particles(0, np.zeros((2, 3)), np.array([1.0, -1.0]), 0.0)
    with pytest.raises(P.Rt3dError):
        ctx.load_particles(0, np.full((1, 3), np.nan), np.array([1.0]), 0.0)
    ctx.load_particles(0, np.zeros((1, 3)) + 5.0, np.array([1e10]), 0.01)
    with pytest.raises(P.Rt3dError):
        ctx.trace(0, -1.0, np.zeros((1, 2)))
    with pytest.raises(P.Rt3dError):
        ctx.trace(0, 0.5, np.zeros((1, 2)), n_ring=1)
    with pytest.raises(P.Rt3dError):
        ctx.trace(0, 0.5, np.zeros((1, 2)), n_ring=2)  # collinear: no Jacobian
    with pytest.raises(P.Rt3dError):
        ctx.trace(0, 0.5, np.full((1, 2), np.nan))


@pytest.mark.parametrize("splits", [12, 16])
def test_clustered_split_reduction(P, cosmo, splits):
    # the expanded two-bundle kernel adds groups of 4 splits in a thread-block
    # cluster (distributed shared memory); 20 tiles in 12 requested splits
    # leave two empty splits in the last cluster
    cfg = _c2_small(n_particles=5000, n_side=4, n_steps=120)
    ctx = ctx_for(P, P.MIXED, variant=5, splits=splits, cluster=4)
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    st = ctx.stats()
    assert st["cluster"] == 4 and st["splits"] % 4 == 0 and st["variant"] == 5
    o = run_oracle(cfg, cfg["theta"], cosmo)
    assert np.array_equal(g["flags"], o.flags)
    assert rel_mu(g["mu"], o.mu).max() < 1e-4
    assert rel_alpha(g["rays"], o).max() < 1e-5
    c1 = ctx_for(P, P.MIXED, variant=4, splits=splits)  # no cluster: same sums in another order
    gpu_load(c1, 0, cfg)
    g1 = c1.trace(0, cfg["z_s"], cfg["theta"], **trace_kw(cfg))
    assert c1.stats()["cluster"] == 1
    assert np.max(np.abs(g["mu"] / g1["mu"] - 1)) < 1e-5


def test_autotuned_shape_keeps_parity(P, cosmo):
    cfg = _c2_small(n_particles=8000, n_side=4, n_steps=120)
    ctx = ctx_for(P, P.MIXED, autotune=1)
    gpu_load(ctx, 0, cfg)
    g = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))
    st = ctx.stats()
    assert (st["rays_per_thread"], st["threads_per_block"]) in {(5, 128), (5, 256), (5, 64)}
    g2 = ctx.trace(0, cfg["z_s"], cfg["theta"], want_rays=True, **trace_kw(cfg))  # cached shape
    assert ctx.stats()["splits"] == st["splits"]
    assert np.array_equal(g["mu"], g2["mu"])
    o = run_oracle(cfg, cfg["theta"], cosmo)
    assert rel_mu(g["mu"], o.mu).max() < MU_GATE
    assert rel_alpha(g["rays"], o).max() < ALPHA_GATE


@pytest.mark.parametrize("box", [False, True])
def test_trace_in_pieces_matches_whole_trace(P, cosmo, box):
    """rt3d_trace_begin / advance / end run the same kernels in the same order
    as rt3d_trace_device: results are bit-identical, whatever the pieces."""
    import torch
    if box:
        b = _small_box()
        z_s = 0.02
        half = (0.5 * b["L"] - 2.0) / cosmo.chi(z_s)
        cfg = dict(b, replicated=True, mean_subtract=True, cosmo=(0.3, 0.7, 0.7), z_s=z_s, n_ring=4,
                   theta_r=math.radians(1 / 3600), schedule=0, n_steps=40)
        theta = inputs.bundle_grid(-half, half, 4)
    else:
        cfg = _c2_small(n_particles=3000, n_side=4, n_steps=60)
        theta = cfg["theta"]
    ctx = ctx_for(P, P.MIXED)
    gpu_load(ctx, 0, cfg)
    nb = theta.shape[0]
    d_theta = torch.from_numpy(np.ascontiguousarray(theta)).cuda()
    ref = torch.zeros(nb * 6, dtype=torch.float64, device="cuda")
    rays_ref = torch.zeros(nb * 5 * 8, dtype=torch.float64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    kw = trace_kw(cfg)
    ctx.trace_device(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), ref.data_ptr(), rays_ref.data_ptr(), **kw)
    torch.cuda.synchronize()
    inter_ref = ctx.stats()["interactions"]
    out = torch.zeros_like(ref)
    rays = torch.zeros_like(rays_ref)
    ctx.trace_begin(sp, 0, cfg["z_s"], nb, d_theta.data_ptr(), **kw)
    total = 4 * (kw["n_steps"] + 16)
    left = ctx.trace_advance(sp, 1)
    assert left == total - 1
    left = ctx.trace_advance(sp, 7)
    assert left == total - 8
    left = ctx.trace_advance(sp, 101)
    assert left == total - 109
    ctx.trace_end(sp, out.data_ptr(), rays.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(rays, rays_ref)
    assert ctx.stats()["interactions"] == inter_ref
    o = run_oracle(cfg, theta, cosmo)
    assert rel_mu(out.view(nb, 6)[:, 0].cpu().numpy(), o.mu).max() < MU_GATE


def test_trace_in_pieces_errors(P):
    import torch
    cfg = _c2_small(n_particles=500, n_side=2, n_steps=20)
    ctx = ctx_for(P, P.MIXED)
    gpu_load(ctx, 0, cfg)
    sp = torch.cuda.current_stream().cuda_stream
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).cuda()
    out = torch.zeros(cfg["theta"].shape[0] * 6, dtype=torch.float64, device="cuda")
    with pytest.raises(P.Rt3dError) as e:
        ctx.trace_advance(sp, 4)
    assert e.value.code == -1
    ctx.trace_begin(sp, 0, cfg["z_s"], cfg["theta"].shape[0], d_theta.data_ptr(), **trace_kw(cfg))
    ctx.trace_advance(sp, 4)
    ctx.schedule(0.5, 0, 10)  # reuses the step table: closes the open trace
    with pytest.raises(P.Rt3dError):
        ctx.trace_advance(sp, 4)
    with pytest.raises(P.Rt3dError):
        ctx.trace_end(sp, out.data_ptr())
    torch.cuda.synchronize()

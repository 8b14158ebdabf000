"""Parity of the CUDA multiple lens-plane system (rt3d_multiplane, Sec. 3.1)
with the oracle's on the same seeded inputs: the point lens (all-FP64), an
NFW halo cut into 1 and 8 planes, the paper's ring of 8, a replicated
mean-subtracted box (1 and 3 planes per replica), the interaction count, and
the 2^21-particle box at full size with oracle samples.  Gates as the 3D
trace: |d mu / mu| <= 1e-4 and |d alpha / alpha| <= 1e-5 in mixed precision,
rounding level in FP64."""
import math

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1110_4894_gb300 as P
    return P


def ctx_for(P, precision):
    c = P.Context(0, precision=precision)
    c.set_cosmology(0.3, 0.7, 0.7)
    return c


def _alpha_err(g, o):
    th = o.ray_theta()
    a_g = th - g["rays"][:, :, 1:3] / o.chi_s
    a_o = o.alpha()
    return np.linalg.norm(a_g - a_o, axis=-1) / np.linalg.norm(a_o, axis=-1)


def test_point_lens_fp64(P, cosmo):
    cfg = inputs.config_c1()
    ctx = ctx_for(P, P.FP64)
    ctx.load_particles(0, cfg["pos"], cfg["mass"], 0.0)
    g = ctx.multiplane(0, cfg["z_s"], cfg["theta"], want_rays=True, theta_r=cfg["theta_r"])
    o = oracle.multiplane(cosmo, oracle.MassField(cfg["pos"], cfg["mass"], 0.0), cfg["z_s"], cfg["theta"],
                          theta_r=cfg["theta_r"])
    ok = np.abs(np.abs(cfg["x"]) - 1) > 0.05
    assert np.abs(g["mu"] / o.mu - 1)[ok].max() < 1e-9
    assert _alpha_err(g, o).max() < 1e-11
    assert np.array_equal(g["flags"], o.flags)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("slices", [1, 8])
@pytest.mark.parametrize("n_ring", [3, 4, 6, 8])  # 4 and 8: two bundles per thread; 3 and 6: one
def test_nfw_halo_planes(P, cosmo, precision, slices, n_ring):
    cfg = inputs.config_c2(n_particles=20000, n_side=8, n_steps=10)
    ctx = ctx_for(P, P.FP64 if precision == "fp64" else P.MIXED)
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    kw = dict(n_ring=n_ring, theta_r=cfg["theta_r"], phase=0.3 if n_ring != 4 else 0.0)
    g = ctx.multiplane(0, cfg["z_s"], cfg["theta"], slices=slices, want_rays=True, **kw)
    o = oracle.multiplane(cosmo, oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"]), cfg["z_s"], cfg["theta"],
                          slices=slices, **kw)
    dm, da = np.abs(g["mu"] / o.mu - 1), _alpha_err(g, o)
    if precision == "fp64":
        assert dm.max() < 1e-10 and da.max() < 1e-11
    else:
        assert dm.max() < 1e-4 and da.max() < 1e-5
    assert np.array_equal(g["flags"], o.flags)
    # interactions: every ray against every particle on the planes
    assert ctx.stats()["interactions"] == pytest.approx(o.n_pairs)


def _small_box(seed=inputs.BASE_SEED + 33):
    L = inputs.box_length(20.0 / 0.7)
    pos, mass, _ = inputs.halo_box(4000, L, 12, seed)
    rot, shift = inputs.replicas(6, L, seed)
    return dict(pos=pos, mass=mass, soft=0.016 / 0.7, L=L, rot=rot, shift=shift)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("slices", [1, 3])
def test_replicated_box_planes(P, cosmo, precision, slices):
    b = _small_box()
    z_s = 0.02
    chi_s = cosmo.chi(z_s)
    half = (0.5 * b["L"] - 2.0) / chi_s
    theta = inputs.bundle_grid(-half, half, 6)
    ctx = ctx_for(P, P.FP64 if precision == "fp64" else P.MIXED)
    ctx.load_particles(2, b["pos"], b["mass"], b["soft"], replicated=True, box_length=b["L"], rot=b["rot"],
                       shift=b["shift"], mean_subtract=True)
    kw = dict(n_ring=4, theta_r=math.radians(1 / 3600))
    g = ctx.multiplane(2, z_s, theta, slices=slices, want_rays=True, **kw)
    f = oracle.MassField(b["pos"], b["mass"], b["soft"], replicated=True, L=b["L"], rot=b["rot"], shift=b["shift"],
                         mean_subtract=True)
    o = oracle.multiplane(cosmo, f, z_s, theta, slices=slices, **kw)
    dm = np.abs(g["mu"] / o.mu - 1)
    # alpha ~ 1e-7 rad against theta ~ 0.2 rad: alpha = theta - beta keeps ~9
    # digits of the positions, so the deflection is compared in absolute
    # terms against the bundle's scale of deflection
    a_g = o.ray_theta() - g["rays"][:, :, 1:3] / o.chi_s
    da = np.abs(a_g - o.alpha()).max() / np.abs(o.alpha()).max()
    if precision == "fp64":
        assert dm.max() < 1e-10 and da < 1e-7
    else:
        assert dm.max() < 1e-4 and da < 1e-5
    assert ctx.stats()["interactions"] == pytest.approx(o.n_pairs)


def test_device_variant_matches_host_call(P, cosmo):
    import torch
    cfg = inputs.config_c2(n_particles=5000, n_side=4, n_steps=10)
    ctx = ctx_for(P, P.MIXED)
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    kw = dict(n_ring=4, theta_r=cfg["theta_r"])
    g = ctx.multiplane(0, cfg["z_s"], cfg["theta"], slices=2, **kw)
    nb = cfg["theta"].shape[0]
    d_theta = torch.from_numpy(np.ascontiguousarray(cfg["theta"])).cuda()
    d_out = torch.zeros(nb * 6, dtype=torch.float64, device="cuda")
    ctx.multiplane_device(torch.cuda.current_stream().cuda_stream, 0, cfg["z_s"], nb, d_theta.data_ptr(),
                          d_out.data_ptr(), slices=2, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(d_out.view(nb, 6)[:, 0].cpu().numpy(), g["mu"])
    with pytest.raises(P.Rt3dError):
        ctx.multiplane(0, cfg["z_s"], cfg["theta"], slices=0, **kw)


def test_box_2e21_particles_full_size_sampled(P, cosmo):
    # the 2^21-particle 100/h Mpc box to z_s = 0.5, all 65,536 bundles through
    # one plane per replica; the oracle recomputes 16 sampled bundles
    cfg = inputs.config_c3(n_steps=10)
    ctx = ctx_for(P, P.MIXED)
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, box_length=cfg["L"], rot=cfg["rot"],
                       shift=cfg["shift"], mean_subtract=True)
    kw = dict(n_ring=4, theta_r=cfg["theta_r"])
    g = ctx.multiplane(0, cfg["z_s"], cfg["theta"], want_rays=True, **kw)
    nb = cfg["theta"].shape[0]
    assert np.all(g["flags"] & P.F_NONFINITE == 0)
    idx = np.linspace(0, nb - 1, 16).astype(int)
    f = oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"], replicated=True, L=cfg["L"], rot=cfg["rot"],
                         shift=cfg["shift"], mean_subtract=True)
    o = oracle.multiplane(cosmo, f, cfg["z_s"], cfg["theta"][idx], **kw)
    assert np.abs(g["mu"][idx] / o.mu - 1).max() < 1e-4
    a_g = o.ray_theta() - g["rays"][idx][:, :, 1:3] / o.chi_s
    assert (np.linalg.norm(a_g - o.alpha(), axis=-1) / np.linalg.norm(o.alpha(), axis=-1)).max() < 1e-5
    st = ctx.stats()
    assert st["interactions"] > nb * 5 * 2 ** 21 * 10

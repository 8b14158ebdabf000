"""Grid path (Sec. 3.3 CIC + zero-padded FFT, App. B interpolation) on the GPU
against the oracle's grid path: node values, interpolated field, and whole
traces through a gridded NFW halo."""
import ctypes

import numpy as np
import pytest

import inputs
import oracle
import oracle.grid as G
from _cases import rel_alpha, rel_mu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1110_4894_gb300 as P
    return P


def _cloud(n, seed, lo, span):
    g = inputs.rng(seed)
    pos = lo + g.uniform(-0.1 * span, 1.1 * span, (n, 3))  # some particles fall outside the grid
    mass = g.uniform(1e9, 5e10, n)
    return pos, mass


@pytest.mark.parametrize("eps,mean_subtract", [(0.05, False), (0.05, True), (0.0, False)])
def test_grid_nodes_match_oracle(P, eps, mean_subtract):
    n, h = 24, 0.1
    lo = np.array([-1.2, 0.3, 500.0])
    pos, mass = _cloud(3000, 17, lo, (n - 1) * h)
    ctx = P.Context(0, precision=P.FP64)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    ctx.load_grid(2, pos, mass, eps, lo, h, n, n_int=2, mean_subtract=mean_subtract)
    got = ctx.grid_nodes(2)
    ref = G.GridField(pos, mass, eps, lo, h, n, n_int=2, mean_subtract=mean_subtract).val
    for f in range(4):
        assert np.max(np.abs(got[f] - ref[f])) <= 1e-11 * np.max(np.abs(ref[f])), f
    # a mixed context keeps the same table rounded to FP32
    cm = P.Context(0, precision=P.MIXED)
    cm.set_cosmology(0.3, 0.7, 0.7)
    cm.load_grid(2, pos, mass, eps, lo, h, n, n_int=2, mean_subtract=mean_subtract)
    got32 = cm.grid_nodes(2)
    assert np.array_equal(got32, got.astype(np.float32).astype(np.float64)) or np.all(
        np.abs(got32 - got) <= 6e-8 * np.abs(got) + 1e-12 * np.max(np.abs(got)))


@pytest.mark.parametrize("n_int", [1, 2, 3, 4])
def test_grid_interpolation_matches_oracle(P, n_int):
    n, h = 20, 0.15
    lo = np.array([0.4, -1.0, 800.0])
    pos, mass = _cloud(2000, 23 + n_int, lo, (n - 1) * h)
    ref = G.GridField(pos, mass, 0.03, lo, h, n, n_int=n_int)
    g = inputs.rng(5 + n_int)
    span = (n - 1) * h
    pts = lo + g.uniform(-0.05 * span, 1.05 * span, (3000, 3))
    # nodes, faces and corners of the node range, and just outside it
    pts = np.concatenate([pts, lo + h * g.integers(0, n, (50, 3)), [lo, lo + span, lo + [span, 0, span / 2]],
                          [lo - [1e-9, 0, 0], lo + span + [0, 0, 1e-9]]])
    want = ref.eval(pts)
    # a mixed context keeps the node table in FP32 and interpolates in FP32
    for prec, tol in ((P.FP64, 1e-11), (P.MIXED, 2e-6)):
        ctx = P.Context(0, precision=prec)
        ctx.set_cosmology(0.3, 0.7, 0.7)
        ctx.load_grid(0, pos, mass, 0.03, lo, h, n, n_int=n_int)
        got = ctx.potential(0, pts)
        scale = np.max(np.abs(want), axis=0)
        assert np.all(np.abs(got - want) <= tol * scale), prec
        assert np.all(got[-2:] == 0.0)


def _nfw_grid_case(n_part=5000, n=48, n_steps=200, n_side=3):
    cfg = inputs.config_c2(n_particles=n_part, n_side=n_side, n_steps=n_steps)
    r200c = cfg["info"]["r200_phys"] * (1 + cfg["z_l"])  # comoving
    half = 2.2 * r200c
    h = 2 * half / (n - 1)
    lo = np.array([-half, -half, cfg["chi_l"] - half])
    return cfg, lo, h, n


def test_grid_trace_matches_oracle(P, cosmo):
    cfg, lo, h, n = _nfw_grid_case()
    gf = G.GridField(cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], n_steps=cfg["n_steps"],
              lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    o = oracle.trace(cosmo, gf.field(), cfg["z_s"], cfg["theta"], **kw)
    assert np.all(o.flags == 0)
    # the mixed path interpolates from the FP32 node table in FP32
    for prec, tol_mu, tol_a in ((P.FP64, 1e-9, 1e-9), (P.MIXED, 1e-6, 1e-6)):
        ctx = P.Context(0, precision=prec)
        ctx.set_cosmology(*cfg["cosmo"])
        ctx.load_grid(1, cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
        g = ctx.trace(1, cfg["z_s"], cfg["theta"], want_rays=True, **kw)
        assert np.array_equal(g["flags"], o.flags)
        assert np.array_equal(g["steps"], o.steps)
        assert rel_mu(g["mu"], o.mu).max() < tol_mu
        assert rel_alpha(g["rays"], o).max() < tol_a
        st = ctx.stats()
        assert st["variant"] == 6 and st["splits"] == 1


def test_grid_empty_field_is_empty_space(P):
    ctx = P.Context(0, precision=P.FP64)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    ctx.load_grid(0, np.zeros((0, 3)), np.zeros(0), 0.01, [-1, -1, 100], 0.1, 21)
    assert np.all(ctx.grid_nodes(0) == 0.0)
    r = ctx.trace(0, 0.3, [[1e-4, -2e-4], [0.0, 0.0]], n_ring=4, theta_r=1e-6, n_steps=50)
    assert np.allclose(r["mu"], 1.0, atol=1e-12)


def test_grid_errors(P):
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    pos, mass = np.zeros((1, 3)), np.ones(1) * 1e10
    for kw in (dict(n=3, n_int=2), dict(n=16, n_int=0), dict(n=16, n_int=5), dict(n=2000, n_int=2)):
        with pytest.raises(P.Rt3dError):
            ctx.load_grid(0, pos, mass, 0.01, [0, 0, 0], 0.1, **kw)
    with pytest.raises(P.Rt3dError):
        ctx.load_grid(0, pos, mass, 0.01, [0, 0, 0], 0.0, 16)
    with pytest.raises(P.Rt3dError):
        ctx.load_grid(0, pos, -mass, 0.01, [0, 0, 0], 0.1, 16)
    ctx.load_grid(0, pos, mass, 0.01, [0, 0, 0], 0.1, 16)
    ctx.load_particles(1, pos, mass, 0.01)
    buf = np.zeros(4)
    rc = ctx.L.rt3d_grid_nodes(ctx.h, 1, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == P._binding.EINVAL  # not a grid field


def _box(n_rep=3):
    L = inputs.box_length(20.0 / 0.7)
    pos, mass, _ = inputs.halo_box(3000, L, 8, inputs.BASE_SEED + 61)
    rot, shift = inputs.replicas(n_rep, L, inputs.BASE_SEED + 61)
    return pos, mass, rot, shift, L


def test_box_grid_matches_oracle(P, cosmo):
    pos, mass, rot, shift, L = _box()
    cubes, n, soft = 4, 16, 0.02
    bg = G.BoxGridField(pos, mass, soft, L, rot, shift, cubes=cubes, n=n)
    ctx = P.Context(0, precision=P.FP64)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    ctx.load_grid_box(0, pos, mass, soft, L, rot, shift, cubes, n)
    nodes = ctx.grid_nodes(0)
    for c, gf in enumerate(bg.grids):
        for f in range(4):
            assert np.max(np.abs(nodes[c, f] - gf.val[f])) <= 1e-11 * max(np.max(np.abs(gf.val[f])), 1e-300), (c, f)
    W = L / cubes
    g = inputs.rng(8)
    pts = np.stack([g.uniform(-0.6, 0.6, 400) * W, g.uniform(-0.6, 0.6, 400) * W, g.uniform(0, 3 * L, 400)], 1)
    want = oracle.potential(bg.field(), pts)
    got = ctx.potential(0, pts)
    assert np.all(np.abs(got - want) <= 1e-11 * np.max(np.abs(want), axis=0))
    # traces: bundles within the prism, crossing several cubes and replicas
    chi_s = 2.6 * L
    z_s = cosmo.z_of_chi(chi_s)
    th = g.uniform(-0.3, 0.3, (12, 2)) * W / chi_s
    kw = dict(n_ring=4, theta_r=4.8e-6, schedule=0, n_steps=150)
    o = oracle.trace(cosmo, bg.field(), z_s, th, **kw)
    for prec, tol_mu, tol_a in ((P.FP64, 1e-9, 1e-8), (P.MIXED, 1e-6, 1e-5)):
        c2 = P.Context(0, precision=prec)
        c2.set_cosmology(0.3, 0.7, 0.7)
        c2.load_grid_box(1, pos, mass, soft, L, rot, shift, cubes, n)
        r = c2.trace(1, z_s, th, want_rays=True, **kw)
        assert np.array_equal(r["flags"], o.flags) and np.array_equal(r["steps"], o.steps)
        assert rel_mu(r["mu"], o.mu).max() < tol_mu
        assert rel_alpha(r["rays"], o).max() < tol_a


def test_box_grid_errors(P):
    pos, mass, rot, shift, L = _box()
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    with pytest.raises(P.Rt3dError):
        ctx.load_grid_box(0, pos, mass, 0.02, L, rot, shift, 0, 16)
    with pytest.raises(P.Rt3dError):
        ctx.load_grid_box(0, pos + L, mass, 0.02, L, rot, shift, 4, 16)  # outside [0, L)


def test_batch_with_grid_cones(P, cosmo):
    # one persistent launch over an isolated grid, a replicated box on cube
    # grids and a particle field; each cone against the oracle on its own field
    cfg, lo, h, n = _nfw_grid_case(n_steps=120, n_side=2)
    pos, mass, rot, shift, L = _box()
    gf = G.GridField(cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    bg = G.BoxGridField(pos, mass, 0.02, L, rot, shift, cubes=4, n=16)
    W = L / 4
    chi_s = 2.6 * L
    z_box = cosmo.z_of_chi(chi_s)
    g = inputs.rng(12)
    th_box = g.uniform(-0.3, 0.3, (6, 2)) * W / chi_s
    kw = dict(n_ring=cfg["n_ring"], theta_r=cfg["theta_r"], schedule=cfg["schedule"], lens_chi=cfg["lens_chi"],
              asinh_s=cfg["asinh_s"])
    o_grid = oracle.trace(cosmo, gf.field(), cfg["z_s"], cfg["theta"], n_steps=120, **kw)
    o_box = oracle.trace(cosmo, bg.field(), z_box, th_box, n_steps=90, **kw)
    o_part = oracle.trace(cosmo, oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"]), cfg["z_s"], cfg["theta"],
                          n_steps=120, **kw)
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cfg["cosmo"])
    ctx.load_grid(0, cfg["pos"], cfg["mass"], cfg["soft"], lo, h, n, n_int=2)
    ctx.load_grid_box(1, pos, mass, 0.02, L, rot, shift, 4, 16)
    ctx.load_particles(2, cfg["pos"], cfg["mass"], cfg["soft"])
    res = ctx.trace_batch([dict(field_id=0, z_s=cfg["z_s"], theta=cfg["theta"], n_steps=120),
                           dict(field_id=1, z_s=z_box, theta=th_box, n_steps=90),
                           dict(field_id=2, z_s=cfg["z_s"], theta=cfg["theta"], n_steps=120)], want_rays=True, **kw)
    for r, o, tol_mu in ((res[0], o_grid, 1e-6), (res[1], o_box, 1e-6), (res[2], o_part, 1e-4)):
        assert np.array_equal(r["flags"], o.flags) and np.array_equal(r["steps"], o.steps)
        assert rel_mu(r["mu"], o.mu).max() < tol_mu
        assert rel_alpha(r["rays"], o).max() < 1e-5
    # the grid cones equal the single-field grid trace of the same bundles
    one = ctx.trace(0, cfg["z_s"], cfg["theta"], n_steps=120, **kw)
    assert rel_mu(res[0]["mu"], one["mu"]).max() < 1e-12

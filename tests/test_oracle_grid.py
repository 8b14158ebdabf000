"""Pins of the oracle's grid path (Sec. 3.3 CIC + zero-padded FFT convolution,
App. B spline interpolation) against definitions, library routines and
special cases that do not share its code."""
import numpy as np
import pytest

import oracle
import oracle.grid as G


def test_cic_special_cases_and_moments():
    lo, h, n = np.zeros(3), 0.5, 6
    # a particle on a node puts all its mass there
    M = G.cic([[1.0, 1.5, 2.0]], [3.0], lo, h, n)
    assert M[2, 3, 4] == 3.0 and M.sum() == 3.0
    # a particle at a cell centre splits its mass equally over the 8 corners
    M = G.cic([[1.25, 1.75, 0.25]], [8.0], lo, h, n)
    assert np.allclose(M[2:4, 3:5, 0:2], 1.0) and M.sum() == pytest.approx(8.0)
    # CIC keeps the mass and the centre of mass of particles inside the grid
    g = np.random.default_rng(3)
    pos = g.uniform(0.0, (n - 1) * h, (200, 3))
    m = g.uniform(1.0, 2.0, 200)
    M = G.cic(pos, m, lo, h, n)
    assert M.sum() == pytest.approx(m.sum(), rel=1e-14)
    idx = np.stack(np.meshgrid(*[np.arange(n) * h] * 3, indexing="ij"), -1)
    com = np.einsum("ijk,ijkc->c", M, idx) / M.sum()
    assert np.allclose(com, (m[:, None] * pos).sum(0) / m.sum(), rtol=1e-13)


def test_cic_drops_mass_outside_the_grid():
    M = G.cic([[-0.75, 0.2, 0.2], [0.2, 0.2, 0.2]], [5.0, 1.0], np.zeros(3), 0.5, 4)
    assert M.sum() == pytest.approx(1.0)


@pytest.mark.parametrize("eps", [0.0, 0.07])
def test_fft_convolution_equals_the_node_double_sum(eps):
    g = np.random.default_rng(7)
    n, h = 5, 0.3
    M = g.uniform(-1.0, 2.0, (n, n, n)) * 1e11
    fft = G.convolve(M, h, eps)
    ref = G.direct_node_sum(M, h, eps)
    assert np.max(np.abs(fft - ref)) < 1e-12 * np.max(np.abs(ref))


def test_single_mass_on_a_node_gives_the_plummer_field_on_the_nodes():
    n, h, eps = 8, 0.25, 0.1
    M = np.zeros((n, n, n))
    M[3, 4, 2] = 2e12
    val = G.convolve(M, h, eps)
    mu = oracle.mu_G()
    i = np.array([6, 1, 7])
    d = (i - np.array([3, 4, 2])) * h
    r2 = d @ d + eps * eps
    assert val[0][tuple(i)] == pytest.approx(-mu * 2e12 / np.sqrt(r2), rel=1e-12)
    assert np.allclose(val[1:, i[0], i[1], i[2]], mu * 2e12 * d / r2 ** 1.5, rtol=1e-11)


def test_spline_second_derivatives_match_scipy_natural_spline():
    interp = pytest.importorskip("scipy.interpolate")
    g = np.random.default_rng(11)
    for n in (2, 3, 4, 9, 40):
        y = g.normal(size=n)
        ref = interp.CubicSpline(np.arange(n), y, bc_type="natural")(np.arange(n), 2)
        assert np.allclose(G.spline_y2(y), ref, atol=1e-12)


def _grid_from(fun, n=12, h=0.2, lo=(1.0, -1.0, 0.5), n_int=2):
    lo = np.asarray(lo, np.float64)
    x = [lo[d] + h * np.arange(n) for d in range(3)]
    X = np.meshgrid(*x, indexing="ij")
    val = np.stack([fun(*X, f) for f in range(4)])
    return G.GridField(None, None, 0.0, lo, h, n, n_int=n_int, val=val), lo, h, n


def test_grid_eval_reproduces_nodes_and_linear_fields():
    gf, lo, h, n = _grid_from(lambda x, y, z, f: 1.0 + (f + 1) * x - 2.0 * y + 0.5 * f * z)
    g = np.random.default_rng(5)
    nodes = lo + h * g.integers(0, n, (20, 3))
    pts = lo + h * g.uniform(0, n - 1, (50, 3))
    for p in (nodes, pts):
        out = gf.eval(p)
        want = np.stack([1.0 + (f + 1) * p[:, 0] - 2.0 * p[:, 1] + 0.5 * f * p[:, 2] for f in range(4)], 1)
        assert np.allclose(out, want, atol=1e-12)


def test_grid_eval_along_x3_is_the_global_natural_spline():
    interp = pytest.importorskip("scipy.interpolate")
    gf, lo, h, n = _grid_from(lambda x, y, z, f: np.sin(3.0 * z + f) + 0.0 * x)
    zs = lo[2] + h * np.arange(n)
    p = np.array([[lo[0] + 0.37, lo[1] + 0.91, z] for z in np.linspace(lo[2], zs[-1], 33)])
    out = gf.eval(p)
    for f in range(4):
        cs = interp.CubicSpline(np.arange(n), np.sin(3.0 * zs + f), bc_type="natural")
        assert np.allclose(out[:, f], cs((p[:, 2] - lo[2]) / h), atol=1e-12)


@pytest.mark.parametrize("n_int", [1, 2, 3])
def test_grid_eval_along_x1_is_the_local_natural_spline(n_int):
    interp = pytest.importorskip("scipy.interpolate")
    gf, lo, h, n = _grid_from(lambda x, y, z, f: np.cos(2.0 * x - f), n_int=n_int)
    xs = lo[0] + h * np.arange(n)
    for u in (0.0, 0.3, 2.5, 5.99, 9.2, n - 1.0):
        p = np.array([[lo[0] + u * h, lo[1] + 0.33, lo[2] + 1.1]])
        s = min(max(int(np.floor(u)) - n_int + 1, 0), n - 2 * n_int)
        win = np.arange(s, s + 2 * n_int)
        out = gf.eval(p)[0]
        for f in range(4):
            cs = interp.CubicSpline(win, np.cos(2.0 * xs[win] - f), bc_type="natural")
            assert out[f] == pytest.approx(float(cs(u)), abs=1e-12)


@pytest.mark.parametrize("n_int", [1, 2, 3])
def test_grid_eval_along_x2_is_the_local_natural_spline(n_int):
    interp = pytest.importorskip("scipy.interpolate")
    gf, lo, h, n = _grid_from(lambda x, y, z, f: np.sin(1.7 * y + 0.3 * f), n_int=n_int)
    ys = lo[1] + h * np.arange(n)
    for u in (0.0, 0.45, 3.5, 7.25, n - 1.0):
        p = np.array([[lo[0] + 0.77, lo[1] + u * h, lo[2] + 0.9]])
        s = min(max(int(np.floor(u)) - n_int + 1, 0), n - 2 * n_int)
        win = np.arange(s, s + 2 * n_int)
        out = gf.eval(p)[0]
        for f in range(4):
            cs = interp.CubicSpline(win, np.sin(1.7 * ys[win] + 0.3 * f), bc_type="natural")
            assert out[f] == pytest.approx(float(cs(u)), abs=1e-12)


def test_grid_eval_of_a_product_field_is_the_tensor_product_of_the_splines():
    # f(x1, x2, x3) = g1(x1) g2(x2) g3(x3): App. B's three interpolations
    # factor, so the result is the product of the three one-dimensional splines
    interp = pytest.importorskip("scipy.interpolate")
    g1 = lambda x: np.cos(1.3 * x)
    g2 = lambda y: 1.0 + 0.5 * np.sin(2.1 * y)
    g3 = lambda z: np.exp(-0.4 * z)
    gf, lo, h, n = _grid_from(lambda x, y, z, f: (f + 1.0) * g1(x) * g2(y) * g3(z), n_int=2)
    nodes = [lo[d] + h * np.arange(n) for d in range(3)]
    rng = np.random.default_rng(9)
    for _ in range(10):
        u = rng.uniform(0, n - 1, 3)
        p = lo + h * u
        want = 1.0
        for d, gfun in enumerate((g1, g2)):
            s = min(max(int(np.floor(u[d])) - 1, 0), n - 4)
            win = np.arange(s, s + 4)
            want *= float(interp.CubicSpline(win, gfun(nodes[d][win]), bc_type="natural")(u[d]))
        want *= float(interp.CubicSpline(np.arange(n), g3(nodes[2]), bc_type="natural")(u[2]))
        out = gf.eval(p[None, :])[0]
        assert np.allclose(out, want * np.arange(1.0, 5.0), rtol=1e-11, atol=1e-13)


def test_grid_eval_is_zero_outside_the_nodes():
    gf, lo, h, n = _grid_from(lambda x, y, z, f: 1.0 + x * 0.0)
    out = gf.eval([[lo[0] - 1e-9, lo[1] + 0.5, lo[2] + 0.5], [lo[0] + 0.5, lo[1] + 0.5, lo[2] + (n - 1) * h + 1e-9]])
    assert np.all(out == 0.0)


def test_grid_eval_margin_extrapolates_the_end_cubics():
    # natural splines reproduce linear data, also beyond the end nodes, so a
    # linear field is exact up to the margin; farther out the field is zero
    n, h, lo = 10, 0.25, np.array([0.5, -1.0, 2.0])
    x = [lo[d] + h * np.arange(n) for d in range(3)]
    X = np.meshgrid(*x, indexing="ij")
    lin = lambda p, f: 0.3 + (f + 1.0) * p[..., 0] - 0.7 * p[..., 1] + 0.2 * (f - 1.5) * p[..., 2]
    val = np.stack([lin(np.stack(X, -1), f) for f in range(4)])
    gf = G.GridField(None, None, 0.0, lo, h, n, n_int=2, val=val, margin=1.0)
    span = (n - 1) * h
    inside = np.array([lo - 0.9 * h, lo + span + 0.6 * h, lo + [-0.99 * h, 0.5 * span, span + 0.3 * h]])
    out = gf.eval(inside)
    want = np.stack([lin(inside, f) for f in range(4)], 1)
    assert np.allclose(out, want, atol=1e-12)
    beyond = np.array([lo - [1.01 * h, 0.0, 0.0], lo + [0.0, span + 1.2 * h, 0.0]])
    assert np.all(gf.eval(beyond) == 0.0)
    # without a margin the same points just outside the nodes read zero
    g0 = G.GridField(None, None, 0.0, lo, h, n, n_int=2, val=val)
    assert np.all(g0.eval(inside[:2]) == 0.0)


def test_grid_field_converges_to_the_direct_sum():
    # a Plummer-softened particle: the grid field between the nodes approaches
    # the direct sum as the node spacing shrinks (App. B, Figs. nfwtests2)
    p0 = np.array([[0.5, 0.5, 0.5]])
    m0 = np.array([1e12])
    eps = 0.08
    pts = np.array([[0.71, 0.43, 0.62], [0.35, 0.58, 0.33], [0.52, 0.27, 0.55]])
    ref = oracle.potential(oracle.MassField(p0, m0, eps), pts)
    errs = []
    for n in (11, 21, 41):
        h = 1.0 / (n - 1)
        gf = G.GridField(p0, m0, eps, np.zeros(3), h, n, n_int=2)
        errs.append(np.max(np.abs(gf.eval(pts) - ref) / np.abs(ref).max(axis=0)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-3


def test_grid_trace_matches_direct_sum_for_a_smooth_lens(cosmo):
    # the whole trace through a gridded Plummer lens tends to the direct-sum trace
    import inputs
    cfg = inputs.config_c1(n_bundles=4, x_lo=2.0, x_hi=4.0, n_steps=400, extra_images=False)
    chi_l = cfg["chi_l"]
    eps = 3.0 * cfg["theta_E"] * chi_l
    pos, mass = cfg["pos"], cfg["mass"]
    kw = dict(n_ring=4, theta_r=cfg["theta_r"], schedule=1, n_steps=400, lens_chi=chi_l, asinh_s=eps)
    ref = oracle.trace(cosmo, oracle.MassField(pos, mass, eps), cfg["z_s"], cfg["theta"], **kw)
    n = 41
    half = 12.0 * eps
    h = 2.0 * half / (n - 1)
    lo = pos[0] - half
    gf = G.GridField(pos, mass, eps, lo, h, n, n_int=2)
    got = oracle.trace(cosmo, gf.field(), cfg["z_s"], cfg["theta"], **kw)
    assert np.all(got.flags == 0)
    # the grid holds the lens only within +-12 eps: the deflection outside is
    # missing, so compare the magnification, which is set near the lens
    assert np.max(np.abs(got.mu / ref.mu - 1)) < 2e-2
    assert np.max(np.abs(got.mu - 1) / np.abs(ref.mu - 1)) > 0.5


def _box_grid(cubes=4, n=12, n_rep=3):
    import inputs as I
    L = I.box_length(20.0 / 0.7)
    pos, mass, _ = I.halo_box(3000, L, 8, I.BASE_SEED + 61)
    rot, shift = I.replicas(n_rep, L, I.BASE_SEED + 61)
    return G.BoxGridField(pos, mass, 0.02, L, rot, shift, cubes=cubes, n=n), pos, mass, rot, shift, L


def test_replica_world_is_the_direct_sums_replica():
    bg, pos, mass, rot, shift, L = _box_grid()
    box = oracle.MassField(pos, mass, 0.02, replicated=True, L=L, rot=rot, shift=shift)
    j = 2
    w = oracle.replica_world(box, j)
    pts = np.array([[0.3, -1.1, (j + 0.4) * L], [-2.0, 0.7, (j + 0.9) * L]])
    a = oracle.potential(box, pts, np.array([j, j], np.int32))
    b = oracle.potential(oracle.MassField(w, mass, 0.02), pts)
    assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_box_grid_cubes_hold_the_prism_mass_and_select_by_x3():
    bg, pos, mass, rot, shift, L = _box_grid()
    W = L / bg.cubes
    box = oracle.MassField(pos, mass, 0.02, replicated=True, L=L, rot=rot, shift=shift)
    for j in range(bg.n_rep):
        w = oracle.replica_world(box, j)
        inside = (w[:, 0] >= -0.5 * W) & (w[:, 0] < 0.5 * W) & (w[:, 1] >= -0.5 * W) & (w[:, 1] < 0.5 * W)
        # every particle of the prism lands in exactly one cube, with all its mass (nodes on the faces)
        held = sum(bg.grids[j * bg.cubes + c].M_raw.sum() for c in range(bg.cubes))
        assert held == pytest.approx(mass[inside].sum(), rel=1e-12)
    g = np.random.default_rng(4)
    pts = np.stack([g.uniform(-0.4, 0.4, 30) * W, g.uniform(-0.4, 0.4, 30) * W, g.uniform(0, bg.n_rep * L, 30)], 1)
    got = oracle.potential(bg.field(), pts)
    for p, v in zip(pts, got):
        j = min(int(p[2] // L), bg.n_rep - 1)
        c = min(int((p[2] - j * L) // W), bg.cubes - 1)
        assert np.array_equal(v, bg.grids[j * bg.cubes + c].eval(p[None, :])[0])

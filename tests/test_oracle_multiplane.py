"""Pins of the oracle's multiple lens-plane comparison system (Sec. 3.1,
Eqs. defangleB, lenseqn, defangle):

- the uniform-rectangle deflection integral (mean subtraction of a slab)
  against two-dimensional quadrature, its far field (a point mass), its
  symmetry and its divergence (2 pi inside, 0 outside: the 2D Poisson equation);
- one plane with a point mass is the thin lens of App. C exactly (deflection
  theta_E^2/theta, mu = (1 - x^-4)^-1, |gamma| = x^-2, two-image total);
- one plane with a Plummer particle is the Plummer sphere's thin lens;
- two point masses on two planes follow the textbook multi-plane lens
  equation in angles and angular-diameter distances;
- an extended weak lens cut into more and more planes agrees with the 3D
  trace to second order in the field;
- the plane bookkeeping of a replicated box: slabs at their centres, the last
  one cut at the source, every particle in front of the source on exactly
  one plane; a mean-subtracted uniform lattice deflects (almost) nothing."""
import math

import numpy as np
import pytest
from scipy import integrate

import inputs
import oracle
from oracle import analytic as A


@pytest.mark.parametrize("x", [(0.3, -0.2), (2.5, 0.7), (-3.0, 4.0), (0.999, 0.0), (0.0, 0.0)])
def test_rect_deflection_matches_quadrature(x):
    # reference: the inner integral across the rectangle in closed form (an
    # arctangent), the outer one by adaptive quadrature with a breakpoint at
    # the point's own coordinate
    lo, hi = np.array([-1.0, -0.6]), np.array([1.0, 0.6])
    out = oracle.rect_deflection(lo, hi, [x])[0]

    def inner(c, t):
        o = 1 - c
        u = x[c] - t
        if u == 0.0:
            return 0.0
        return math.atan((x[o] - lo[o]) / u) - math.atan((x[o] - hi[o]) / u)

    ref = []
    for c in range(2):
        pts = [x[c]] if lo[c] < x[c] < hi[c] else None
        v, _ = integrate.quad(lambda t: inner(c, t), lo[c], hi[c], points=pts, limit=500, epsabs=1e-13)
        ref.append(v)
    assert np.allclose(out, ref, rtol=1e-9, atol=1e-11)


def test_rect_deflection_far_field_symmetry_and_divergence():
    lo, hi = np.array([-0.5, -0.5]), np.array([0.5, 0.5])
    # far away: the point mass of the same area
    x = np.array([[40.0, 25.0]])
    r = oracle.rect_deflection(lo, hi, x)[0]
    ref = x[0] / np.dot(x[0], x[0])
    assert np.allclose(r, ref, rtol=2e-3)
    # the centre of a square is a point of symmetry
    assert np.allclose(oracle.rect_deflection(lo, hi, [[0.0, 0.0]]), 0.0, atol=1e-14)
    # mirror symmetry
    a = oracle.rect_deflection(lo, hi, [[0.3, 0.2]])[0]
    b = oracle.rect_deflection(lo, hi, [[-0.3, 0.2]])[0]
    assert np.allclose([a[0], a[1]], [-b[0], b[1]], atol=1e-14)
    # div R = 2 pi inside the rectangle, 0 outside (2D Poisson equation)
    h = 1e-5
    for p, want in (((0.1, -0.2), 2 * math.pi), ((1.3, 0.4), 0.0), ((-0.2, 2.0), 0.0)):
        p = np.array(p)
        d = (oracle.rect_deflection(lo, hi, [p + [h, 0]])[0][0] - oracle.rect_deflection(lo, hi, [p - [h, 0]])[0][0]
             + oracle.rect_deflection(lo, hi, [p + [0, h]])[0][1] - oracle.rect_deflection(lo, hi, [p - [0, h]])[0][1])
        assert abs(d / (2 * h) - want) < 1e-5


@pytest.fixture(scope="module")
def c1_mp(cosmo):
    cfg = inputs.config_c1()
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    return cfg, oracle.multiplane(cosmo, f, cfg["z_s"], cfg["theta"], theta_r=cfg["theta_r"])


def test_one_plane_point_lens_deflection(cosmo, c1_mp):
    cfg, r = c1_mp
    assert r.planes.shape[0] == 1 and r.planes[0, 0] == cfg["pos"][0, 2]  # the plane holds the particle
    thE = A.theta_einstein(cosmo, cfg["M"], cfg["z_l"], cfg["z_s"])
    th = r.ray_theta()
    ref = A.point_deflection(th, thE)
    rel = np.linalg.norm(r.alpha() - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() < 1e-9  # the thin lens is exact here


@pytest.mark.parametrize("n_ring", [4, 8])
def test_one_plane_point_lens_magnification(cosmo, n_ring):
    cfg = inputs.config_c1()
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    r = oracle.multiplane(cosmo, f, cfg["z_s"], cfg["theta"], n_ring=n_ring, theta_r=cfg["theta_r"], phase=0.1)
    x = cfg["x"]
    ok = np.abs(np.abs(x) - 1) > 0.05
    with np.errstate(divide="ignore"):
        mu = A.schw_mu_image(np.abs(x))
    # only the bundle's finite size (theta_r = 1e-3 theta_E) separates it from the closed form
    assert np.abs(r.mu / mu - 1)[ok].max() < 3e-5
    far = np.abs(x) > 1.5
    assert np.abs(r.mu / mu - 1)[far].max() < 1e-6
    assert np.allclose(np.hypot(r.gamma1, r.gamma2)[far], A.schw_gamma(np.abs(x[far])), rtol=1e-6)
    # the bundle's finite size leaves kappa of order (theta_r / theta)^2 |gamma| ~ 2e-7
    assert np.all(np.abs(r.kappa[far]) < 1e-6)
    # a thin lens has a symmetric Jacobian: the fit's rotation is of the same finite-size order
    assert np.all(np.abs(r.omega) < 4 * (cfg["theta_r"] / np.abs(cfg["theta"][:, 0])) ** 2)
    assert np.all(((r.mu < 0) == (np.abs(x) < 1))[ok])
    assert abs((abs(r.mu[-2]) + abs(r.mu[-1])) / A.schw_mu_total(1.5) - 1) < 3e-5


def test_one_plane_plummer_lens(cosmo):
    M, zl, zs = 1e13, 0.25, 0.5
    chi_l = cosmo.chi(zl)
    thE = A.theta_einstein(cosmo, M, zl, zs)
    eps = 0.7 * thE * chi_l
    e = eps / chi_l
    pos, mass = inputs.plummer_particle(M, chi_l)
    x = np.array([0.3, 0.8, 1.6, 3.0])
    th = np.stack([x * thE * 0.6, x * thE * 0.8], 1)
    r = oracle.multiplane(cosmo, oracle.MassField(pos, mass, eps), zs, th, n_ring=8, theta_r=1e-3 * thE)
    ref = A.jacobian_to_mu_kappa_gamma(A.plummer_jacobian(th, thE, e))
    assert np.allclose(1 / r.mu, 1 / ref["mu"], rtol=0, atol=2e-6)
    assert np.allclose(r.kappa, A.plummer_kappa(x, e / thE), rtol=0, atol=2e-6)
    assert np.allclose(r.gamma1, ref["gamma1"], rtol=0, atol=2e-6)
    assert np.allclose(r.gamma2, ref["gamma2"], rtol=0, atol=2e-6)
    assert np.allclose(r.alpha()[:, 0], A.plummer_deflection(th, thE, e), rtol=1e-9)


def test_empty_field_and_rotation_symmetry(cosmo):
    th = np.array([[0.0, 0.0], [1e-3, -2e-3]])
    r = oracle.multiplane(cosmo, oracle.MassField(np.zeros((0, 3)), np.zeros(0), 0.0), 0.5, th, theta_r=1e-5)
    assert np.allclose(r.mu, 1.0, atol=1e-12) and np.allclose(r.alpha(), 0.0, atol=1e-15)
    # turning the particles and the bundles about the optical axis changes no mu, kappa
    g = inputs.rng(31)
    n = 200
    pos = np.array([0.0, 0.0, 900.0]) + g.normal(size=(n, 3)) * [0.3, 0.3, 2.0]
    m = g.uniform(0.5, 2, n) * 1e11
    th = g.normal(size=(6, 2)) * 3e-4
    psi = 0.7
    R = np.array([[math.cos(psi), -math.sin(psi)], [math.sin(psi), math.cos(psi)]])
    p2 = pos.copy()
    p2[:, :2] = pos[:, :2] @ R.T
    kw = dict(theta_r=1e-6, slices=3)
    a = oracle.multiplane(cosmo, oracle.MassField(pos, m, 0.01), 0.5, th, **kw)
    b = oracle.multiplane(cosmo, oracle.MassField(p2, m, 0.01), 0.5, th @ R.T, phase=psi, **kw)
    assert np.allclose(a.mu, b.mu, rtol=1e-9) and np.allclose(a.kappa, b.kappa, atol=1e-12)
    ga, gb = a.gamma1 + 1j * a.gamma2, b.gamma1 + 1j * b.gamma2
    assert np.allclose(gb, ga * np.exp(2j * psi), rtol=1e-7, atol=1e-12)


def test_thin_planes_approach_the_3d_trace(cosmo):
    # five softened clumps (eps = 100 kpc, so that the 3D trace converges in
    # its step count) spread over 3 Mpc along the line of sight: one plane at
    # the centre of their range already gives mu - 1 to 0.5 %, and cutting the
    # range into more slabs (planes nearer each clump) converges to the 3D
    # trace up to its weak-field terms of order phi ~ 1e-5
    zl, zs = 0.25, 0.5
    chi_l = cosmo.chi(zl)
    g = inputs.rng(77)
    dz = np.array([-1.5, -0.7, 0.0, 0.6, 1.4])
    pos = inputs.quantize(np.stack([g.uniform(-0.3, 0.3, 5), g.uniform(-0.3, 0.3, 5), chi_l + dz], 1))
    f = oracle.MassField(pos, np.full(5, 2e13), 0.1)
    th = g.uniform(-0.5, 0.5, (12, 2)) / chi_l
    tr = math.radians(1 / 3600)
    r3 = oracle.trace(cosmo, f, zs, th, theta_r=tr, schedule=1, n_steps=1000, lens_chi=chi_l, asinh_s=0.1)
    r3b = oracle.trace(cosmo, f, zs, th, theta_r=tr, schedule=1, n_steps=2000, lens_chi=chi_l, asinh_s=0.1)
    assert np.abs(r3b.mu / r3.mu - 1).max() < 1e-8  # the 3D reference is step-converged
    dev, dal = [], []
    for s_ in (1, 4, 256):
        rm = oracle.multiplane(cosmo, f, zs, th, theta_r=tr, slices=s_)
        dev.append((np.abs(rm.mu - r3b.mu) / np.abs(r3b.mu - 1)).max())
        dal.append((np.linalg.norm(rm.alpha()[:, 0] - r3b.alpha()[:, 0], axis=-1) /
                    np.linalg.norm(r3b.alpha()[:, 0], axis=-1)).max())
    assert dev[0] < 1e-2 and dal[0] < 2e-3
    assert dev[2] < dev[1] < dev[0] and dal[2] < dal[1] < dal[0]
    assert dev[2] < 3e-4 and dal[2] < 1e-4


def test_two_planes_match_the_angular_lens_equation(cosmo):
    # two point masses on two planes against the multi-plane lens equation in
    # its textbook angular form (Sec. 3.1, Eq. lenseqn): physical impact
    # parameters xi_i = D_i theta_i - p_i / (1 + z_i), deflections
    # 4 G M xi / |xi|^2, theta_2 = theta - (D_12 / D_2) alpha_1 and
    # beta = theta - sum_i (D_is / D_s) alpha_i, with the flat universe's
    # angular-diameter distances D_ij = (chi_j - chi_i) / (1 + z_j).  The
    # oracle works in comoving positions and slopes instead; a wrong distance
    # ratio, (1 + z) factor or plane order fails here.
    from scipy import optimize
    z_a, z_b, z_s = 0.2, 0.35, 0.6
    chi_a, chi_b, chi_s = cosmo.chi(z_a), cosmo.chi(z_b), cosmo.chi(z_s)
    M = np.array([2e13, 1e13])
    p = np.array([[0.0, 0.0], [0.05, -0.03]])
    pos = np.array([[p[0, 0], p[0, 1], chi_a], [p[1, 0], p[1, 1], chi_b]])
    # two slabs of the particles' x3 range, each projected onto its centre
    d = 0.5 * (chi_b - chi_a)
    chi_pl = np.array([chi_a + 0.5 * d, chi_a + 1.5 * d])
    z_pl = np.array([optimize.brentq(lambda z: cosmo.chi(z) - c, 0.0, 1.0, xtol=1e-15) for c in chi_pl])
    thE = A.theta_einstein(cosmo, M[0], z_a, z_s)
    th = np.array([[1.7, 0.4], [-1.1, 1.9], [2.6, -2.2], [0.3, -3.1], [4.0, 1.0]]) * thE
    r = oracle.multiplane(cosmo, oracle.MassField(pos, M, 0.0), z_s, th, n_ring=8, theta_r=1e-3 * thE, slices=2)
    assert np.allclose(r.planes[:, 0], chi_pl, rtol=1e-13) and np.array_equal(r.planes[:, 2], [1, 1])

    D = chi_pl / (1 + z_pl)
    D_s = chi_s / (1 + z_s)
    D_12 = (chi_pl[1] - chi_pl[0]) / (1 + z_pl[1])
    D_is = (chi_s - chi_pl) / (1 + z_s)
    G = oracle.mu_G()

    def deflection(i, t):
        xi = D[i] * t - p[i] / (1 + z_pl[i])
        return 4.0 * G * M[i] * xi / np.sum(xi * xi, axis=-1, keepdims=True)

    def beta(t):
        a1 = deflection(0, t)
        a2 = deflection(1, t - (D_12 / D[1]) * a1)
        return t - (D_is[0] / D_s) * a1 - (D_is[1] / D_s) * a2

    rays = r.ray_theta()
    want = beta(rays)
    assert np.max(np.linalg.norm(r.beta() - want, axis=-1) / np.linalg.norm(rays - want, axis=-1)) < 1e-12
    # the bundle's magnification against the Jacobian of the angular map
    h = 1e-6 * thE
    for b in range(th.shape[0]):
        jac = np.stack([(beta(th[b] + h * e) - beta(th[b] - h * e)) / (2 * h) for e in np.eye(2)], 1)
        mu = 1.0 / np.linalg.det(jac)
        assert abs(r.mu[b] / mu - 1) < 1e-6, (b, r.mu[b], mu)  # the bundle's finite size: ~1e-9


def test_box_planes_bookkeeping(cosmo):
    L = inputs.box_length(20.0 / 0.7)
    pos, mass, _ = inputs.halo_box(3000, L, 8, seed=81)
    z_s = 0.03
    chi_s = cosmo.chi(z_s)
    n_rep = int(math.ceil(chi_s / L)) + 1
    rot, shift = inputs.replicas(n_rep, L, seed=81)
    f = oracle.MassField(pos, mass, 0.02, replicated=True, L=L, rot=rot, shift=shift, mean_subtract=True)
    for slices in (1, 3):
        r = oracle.multiplane(cosmo, f, z_s, np.zeros((2, 2)), theta_r=1e-5, slices=slices)
        pl = r.planes
        d = L / slices
        n_full = int(chi_s // d)
        assert pl.shape[0] == n_full + 1
        assert np.allclose(pl[:n_full, 0], (np.arange(n_full) + 0.5) * d)
        assert np.allclose(pl[:n_full, 3], d)
        assert abs(pl[-1, 0] - 0.5 * (n_full * d + chi_s)) < 1e-9 and abs(pl[-1, 3] - (chi_s - n_full * d)) < 1e-9
        assert np.allclose(pl[:, 1], [cosmo.z_of_chi(c) for c in pl[:, 0]])
        # every particle in front of the source lands on one plane
        want = sum(int(np.sum(oracle.replica_world(f, j)[:, 2] < chi_s)) for j in range(n_rep))
        assert int(pl[:, 2].sum()) == want


def test_mean_subtracted_uniform_lattice_deflects_little(cosmo):
    # a cubic lattice filling the box is uniform on scales above its spacing:
    # minus the slab's mean surface density, the deflection near the axis is
    # a small fraction of either term alone
    L = inputs.box_length(10.0 / 0.7)
    k = 24
    g = (np.arange(k) + 0.5) * L / k
    pos = inputs.quantize(np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3))
    mass = np.full(len(pos), 1e10)
    rot = np.tile(np.eye(3, dtype=np.int32).ravel(), (3, 1))
    shift = np.zeros((3, 3))
    th = np.array([[1e-4, 2e-4], [-3e-4, 1e-4]])
    kw = dict(theta_r=1e-5, slices=1)
    sub = oracle.multiplane(cosmo, oracle.MassField(pos, mass, L / k, replicated=True, L=L, rot=rot, shift=shift,
                                                    mean_subtract=True), 0.008, th, **kw)
    raw = oracle.multiplane(cosmo, oracle.MassField(pos, mass, L / k, replicated=True, L=L, rot=rot, shift=shift),
                            0.008, th, **kw)
    a_sub = np.linalg.norm(sub.alpha()[:, 0], axis=-1)
    a_raw = np.linalg.norm(raw.alpha()[:, 0], axis=-1)
    assert np.all(a_sub < 0.05 * a_raw)  # a wrong sign or surface density would not cancel
    assert np.all(np.abs(sub.mu - 1) < 0.05 * np.abs(raw.mu - 1))

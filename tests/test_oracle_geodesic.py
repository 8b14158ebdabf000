"""Pins for the oracle's geodesic integration (Eq. geodesiceqn with App. A's
Christoffel symbols, RK4 with fixed steps and termination on x3, Sec. 3.4).

The Christoffel symbols are checked against symbols computed numerically
from the metric of Eq. expandingmetric; the integrator against invariants
(empty space, a(t) at the source, the null condition, symmetry) and against
its own convergence order.
"""
import math

import numpy as np
import pytest

import inputs
import oracle


def _metric(cosmo, t, x, phi_fn):
    a = cosmo.a_of_t(t)
    p = phi_fn(x)
    return np.diag([-(1 + 2 * p / a), a * a * (1 - 2 * p / a), a * a * (1 - 2 * p / a), a * a * (1 - 2 * p / a)])


def _christoffel_fd(cosmo, t, x, phi_fn, ht=0.5, hx=1e-5):
    X = np.concatenate([[t], x])
    dg = np.zeros((4, 4, 4))  # dg[k] = d g / d X^k
    for k in range(4):
        h = ht if k == 0 else hx
        e = np.zeros(4)
        e[k] = h
        gp = _metric(cosmo, (X + e)[0], (X + e)[1:], phi_fn)
        gm = _metric(cosmo, (X - e)[0], (X - e)[1:], phi_fn)
        dg[k] = (gp - gm) / (2 * h)
    g = _metric(cosmo, t, x, phi_fn)
    gi = np.linalg.inv(g)
    G = np.zeros((4, 4, 4))
    for al in range(4):
        for b in range(4):
            for c in range(4):
                G[al, b, c] = 0.5 * sum(gi[al, d] * (dg[b][d, c] + dg[c][d, b] - dg[d][b, c]) for d in range(4))
    return G


def _acc(G, u):
    return -np.einsum("abc,b,c->a", G, u, u)


def test_christoffel_symbols_from_metric(cosmo):
    # a smooth Plummer potential with |phi| ~ 2e-4: first-order terms dominate
    x0, eps, K = np.array([0.02, -0.01, 500.0]), 0.05, 1e-5

    def phi_fn(x):
        d = x - x0
        return -K / math.sqrt(d @ d + eps * eps)

    def field(x):
        d = x - x0
        q = d @ d + eps * eps
        return np.array([-K / math.sqrt(q), *(K * d / q ** 1.5)])

    t = 480.0
    x = np.array([0.03, 0.02, 500.01])
    F = field(x)
    a = cosmo.a_of_t(t)
    for v in (np.array([0.001, -0.002, 1.0 / a ** 2]), np.array([0.3, 0.1, 0.9]),
              np.array([F[2], -F[1], 0.0]) / np.hypot(F[1], F[2])):   # last: v perpendicular to grad phi
        vn = math.sqrt(v @ v)
        T = a * vn * math.sqrt((1 - 2 * F[0] / a) / (1 + 2 * F[0] / a))
        u = np.concatenate([[T], v])
        y = np.concatenate([[t], x, u])
        acc_fd = _acc(_christoffel_fd(cosmo, t, x, phi_fn), u)
        acc_bg = _acc(_christoffel_fd(cosmo, t, x, lambda q: 0.0), u)
        d_fd = acc_fd - acc_bg
        rhs_derived = oracle.geodesic_rhs(cosmo, y, F, christoffel=1)[4:]
        rhs_paper = oracle.geodesic_rhs(cosmo, y, F, christoffel=0)[4:]
        rhs_bg = oracle.geodesic_rhs(cosmo, y, np.zeros(4), christoffel=1)[4:]
        d_or = rhs_derived - rhs_bg
        # first-order symbols: the residual is O(phi) relative to the O(phi) part
        scale = np.abs(d_fd).max()
        assert np.all(np.abs(d_or - d_fd) < 3e-3 * scale), (d_or, d_fd)
        # App. A as printed differs only in Gamma^t_ij: a-dot (a + phi) vs a-dot (a - 3 phi)
        ad = cosmo.adot_of_t(t)
        assert np.allclose(rhs_paper[1:], rhs_derived[1:], rtol=0, atol=1e-12 * np.abs(rhs_derived).max())
        assert abs((rhs_paper[0] - rhs_derived[0]) - (-4 * ad * F[0] * (v @ v))) < 1e-9 * abs(4 * ad * F[0] * (v @ v))


def test_unperturbed_background_terms(cosmo):
    # FRW null ray: T = a|v|, d T/d l = -(a-dot/a) T^2, d v/d l = -2 (a-dot/a) T v
    t = 300.0
    a, ad = cosmo.a_of_t(t), cosmo.adot_of_t(t)
    v = np.array([1e-3, 2e-3, 1.0])
    T = a * math.sqrt(v @ v)
    dy = oracle.geodesic_rhs(cosmo, np.concatenate([[t, 0, 0, 10.0], [T], v]), np.zeros(4))
    assert abs(dy[4] / (-(ad / a) * T * T) - 1) < 1e-14
    assert np.allclose(dy[5:], -2 * (ad / a) * T * v, rtol=1e-14, atol=0)


def _empty_field():
    return oracle.MassField(np.zeros((0, 3)), np.zeros(0), 0.0)


def test_empty_space_is_unlensed(cosmo):
    th = np.array([[0.0, 0.0], [1e-3, -2e-3], [-0.02, 0.01]])
    for sched, n in ((0, 50), (1, 200)):
        r = oracle.trace(cosmo, _empty_field(), 0.5, th, theta_r=1e-6, schedule=sched, n_steps=n,
                         lens_chi=cosmo.chi(0.25), asinh_s=0.01)
        assert np.all(np.abs(r.mu - 1) < 1e-9)
        assert np.all(np.abs(r.kappa) < 1e-9) and np.all(np.abs(r.gamma1) < 1e-9)
        assert np.all(np.abs(r.gamma2) < 1e-9) and np.all(np.abs(r.omega) < 1e-9)
        assert np.all(np.abs(r.alpha()) < 1e-14)
        assert np.all(r.flags == 0)


@pytest.mark.parametrize("z_s", [0.3, 1.0])
def test_scale_factor_at_source_plane(cosmo, z_s):
    # the paper's sanity check: the integrated a(t) at x3 = chi(z) is 1/(1+z)
    th = np.array([[0.0, 0.0], [1e-2, 2e-2]])
    r = oracle.trace(cosmo, _empty_field(), z_s, th, schedule=0, n_steps=400)
    t_fin = r.rays[0, 0, 0]
    assert abs(cosmo.a_of_t(t_fin) * (1 + z_s) - 1) < 1e-11
    assert abs(r.rays[0, 0, 3] - cosmo.chi(z_s)) < 1e-9
    # an oblique ray meets the plane x3 = chi_s after a comoving path
    # chi_s sqrt(1 + theta^2), hence at a slightly higher redshift; it runs
    # slightly ahead of the step nodes, so it crosses inside its last step and
    # the linear interpolation of the termination rule (Sec. 3.4) adds an
    # O(step) error of order theta^2 (~1e-7 here)
    for b in range(2):
        for k in range(5):
            y = r.rays[b, k]
            path = cosmo.chi(z_s) * math.sqrt(y[5] ** 2 + y[6] ** 2 + y[7] ** 2) / y[7]
            assert abs(cosmo.a_of_t(y[0]) * (1 + cosmo.z_of_chi(path)) - 1) < (1e-11 if b == 0 else 5e-7)


def _plummer(cosmo, M=1e13, eps=0.02):
    chi_l = cosmo.chi(0.25)
    pos, mass = inputs.plummer_particle(M, chi_l)
    return oracle.MassField(pos, mass, eps), chi_l


def test_null_condition_is_kept(cosmo):
    # with the symbols derived from the metric the null condition holds to
    # O(phi^2); App. A's Gamma^t_ij = a-dot (a + phi) breaks it at O(a-dot phi L)
    f, chi_l = _plummer(cosmo)
    th = np.array([[2e-6, 1e-6], [5e-6, -4e-6]])
    drift = {}
    for ch in (0, 1):
        r = oracle.trace(cosmo, f, 0.5, th, theta_r=1e-7, schedule=1, n_steps=800, lens_chi=chi_l,
                         asinh_s=0.02, christoffel=ch)
        worst = 0.0
        for b in range(2):
            for k in range(5):
                y = r.rays[b, k]
                F = oracle.potential(f, y[1:4][None])[0]
                a = cosmo.a_of_t(y[0])
                g = -(1 + 2 * F[0] / a) * y[4] ** 2 + a * a * (1 - 2 * F[0] / a) * (y[5:] @ y[5:])
                worst = max(worst, abs(g) / y[4] ** 2)
        drift[ch] = worst
    assert drift[1] < 1e-9
    assert drift[0] < 1e-7
    assert drift[0] > 10 * drift[1]


def test_rk4_fourth_order(cosmo):
    f, chi_l = _plummer(cosmo, M=1e14, eps=0.05)
    th = np.array([[6e-6, 3e-6]])
    run = lambda n: oracle.trace(cosmo, f, 0.5, th, theta_r=1e-7, schedule=1, n_steps=n,
                                 lens_chi=chi_l, asinh_s=0.05)
    ref = run(3200)
    errs = []
    for n in (100, 200):
        r = run(n)
        errs.append((abs(r.mu[0] - ref.mu[0]), np.abs(r.alpha()[0, 0] - ref.alpha()[0, 0]).max()))
    for q in range(2):
        ratio = errs[0][q] / errs[1][q]
        assert 11.0 < ratio < 22.0, (q, errs)


def test_rotation_about_line_of_sight(cosmo):
    chi_l = cosmo.chi(0.25)
    g = inputs.rng(3)
    p = np.stack([g.normal(0, 0.05, 6), g.normal(0, 0.05, 6), chi_l + g.normal(0, 0.05, 6)], 1)
    m = g.uniform(1, 5, 6) * 1e12
    th = np.array([[4e-6, -1e-6], [-2e-6, 7e-6]])
    psi = 0.7
    R = np.array([[math.cos(psi), -math.sin(psi)], [math.sin(psi), math.cos(psi)]])
    p2 = p.copy()
    p2[:, :2] = p[:, :2] @ R.T
    kw = dict(theta_r=2e-7, schedule=1, n_steps=600, lens_chi=chi_l, asinh_s=0.03)
    r1 = oracle.trace(cosmo, oracle.MassField(p, m, 0.02), 0.5, th, **kw)
    r2 = oracle.trace(cosmo, oracle.MassField(p2, m, 0.02), 0.5, th @ R.T, phase=psi, **kw)
    assert np.allclose(r1.mu, r2.mu, rtol=1e-9)
    assert np.allclose(r1.kappa, r2.kappa, atol=1e-9)
    g1 = r1.gamma1 + 1j * r1.gamma2
    g2 = r2.gamma1 + 1j * r2.gamma2
    assert np.allclose(g2, np.exp(2j * psi) * g1, atol=1e-9)
    assert np.allclose(r2.alpha()[:, 0], r1.alpha()[:, 0] @ R.T, rtol=0, atol=1e-9 * np.abs(r1.alpha()).max())


def test_christoffel_variants_agree_to_order_phi(cosmo):
    cfg = inputs.config_c1(n_bundles=6)
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    kw = dict(theta_r=cfg["theta_r"], schedule=1, n_steps=1000, lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    a = oracle.trace(cosmo, f, 0.5, cfg["theta"], christoffel=0, **kw)
    b = oracle.trace(cosmo, f, 0.5, cfg["theta"], christoffel=1, **kw)
    d = np.abs(a.mu / b.mu - 1)
    assert d.max() < 1e-6

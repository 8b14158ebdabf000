"""Pins of the oracle's full trace against thin-lens closed forms:
Schwarzschild lens (App. C), Plummer sphere (one softened particle) and the
NFW lens (App. D, Eq. nfwprof), plus the App. D formulae themselves against
quadrature of the NFW profile."""
import math

import numpy as np
import pytest

import inputs
import oracle
from oracle import analytic as A

ARCSEC = math.pi / 180 / 3600


@pytest.fixture(scope="module")
def c1(cosmo):
    cfg = inputs.config_c1()
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    r = oracle.trace(cosmo, f, cfg["z_s"], cfg["theta"], n_ring=4, theta_r=cfg["theta_r"], schedule=1,
                     n_steps=cfg["n_steps"], lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    return cfg, r


def test_point_lens_deflection(cosmo, c1):
    # weak-field deflection 4GM/(c^2 b) -> reduced deflection theta_E^2 / theta
    cfg, r = c1
    thE = A.theta_einstein(cosmo, cfg["M"], cfg["z_l"], cfg["z_s"])
    assert abs(thE / cfg["theta_E"] - 1) < 1e-9
    th = r.ray_theta()
    al = r.alpha()
    ref = A.point_deflection(th, thE)
    rel = np.abs(al - ref).max(axis=-1) / np.linalg.norm(ref, axis=-1)
    # thin-lens, first-order weak field: agreement to O(GM/c^2 b) ~ 1e-5
    assert rel.max() < 1e-4
    # deflection points towards the lens (attractive)
    assert np.all(np.sign(al[:, 0, 0]) == np.sign(th[:, 0, 0]))


def test_point_lens_magnification(c1):
    cfg, r = c1
    x = cfg["x"]
    # x = 1 lies on the Einstein ring (infinite mu): a finite bundle cannot
    # resolve the critical curve, so the comparison skips its neighbourhood
    ok = np.abs(np.abs(x) - 1) > 0.05
    with np.errstate(divide="ignore"):
        mu = A.schw_mu_image(np.abs(x))
    rel = np.abs(r.mu / mu - 1)[ok]
    assert rel.max() < 3e-4
    assert abs(r.mu[np.argmin(np.abs(np.abs(x) - 1))]) > 100
    assert np.abs(r.mu / mu - 1)[np.abs(x) > 1.5].max() < 1e-5
    # images inside the Einstein ring have negative parity
    assert np.all(((r.mu < 0) == (np.abs(x) < 1))[ok])
    assert np.all((((r.flags & oracle.F_NEGPARITY) != 0) == (r.mu < 0)))


def test_point_lens_jacobian_components(cosmo, c1):
    cfg, r = c1
    thE = cfg["theta_E"]
    Aan = A.plummer_jacobian(cfg["theta"], thE, 0.0)
    ref = A.jacobian_to_mu_kappa_gamma(Aan)
    sel = np.abs(cfg["x"]) > 1.5
    assert np.all(np.abs(r.kappa[sel]) < 1e-5)
    assert np.allclose(r.gamma1[sel], ref["gamma1"][sel], rtol=1e-4, atol=1e-7)
    assert np.allclose(r.gamma2[sel], 0.0, atol=1e-8)
    # |gamma| = x^-2 (the form consistent with Eq. schwmu)
    assert np.allclose(np.hypot(r.gamma1, r.gamma2)[sel], A.schw_gamma(np.abs(cfg["x"][sel])), rtol=1e-4)
    assert np.all(np.abs(r.omega) < 1e-6)


def test_point_lens_two_image_total(c1):
    cfg, r = c1
    # the last two bundles are the images x+ = 2 and x- = -1/2 of u = 1.5
    mu_p, mu_m = r.mu[-2], r.mu[-1]
    assert cfg["x"][-2] == 2.0 and cfg["x"][-1] == -0.5
    tot = abs(mu_p) + abs(mu_m)
    assert abs(tot / A.schw_mu_total(1.5) - 1) < 3e-4


def test_point_lens_scale_invariance(cosmo):
    # the lens solution depends on theta/theta_E only (Sec. 4.1)
    out = []
    for M in (1e12, 1e13):
        cfg = inputs.config_c1(n_bundles=4, x_lo=1.5, x_hi=4.0, extra_images=False)
        chi_l = cfg["chi_l"]
        thE = inputs.theta_einstein_placement(M, cfg["z_l"], cfg["z_s"], 0.3, 0.7, 0.7)
        f = oracle.MassField(cfg["pos"], [M], 0.0)
        th = np.stack([cfg["x"] * thE, 0 * cfg["x"]], 1)
        r = oracle.trace(cosmo, f, 0.5, th, theta_r=1e-3 * thE, schedule=1, n_steps=1000,
                         lens_chi=chi_l, asinh_s=0.2 * thE * chi_l)
        out.append(r.mu)
    assert np.allclose(out[0], out[1], rtol=5e-5)


def test_plummer_lens(cosmo):
    M, zl, zs = 1e13, 0.25, 0.5
    chi_l = cosmo.chi(zl)
    thE = A.theta_einstein(cosmo, M, zl, zs)
    eps = 0.7 * thE * chi_l            # comoving softening = 0.7 theta_E at the lens
    e = eps / chi_l
    pos, mass = inputs.plummer_particle(M, chi_l)
    x = np.array([0.3, 0.8, 1.6, 3.0])
    th = np.stack([x * thE * 0.6, x * thE * 0.8], 1)
    r = oracle.trace(cosmo, oracle.MassField(pos, mass, eps), zs, th, theta_r=1e-3 * thE, schedule=1,
                     n_steps=1000, lens_chi=float(pos[0, 2]), asinh_s=eps)
    Aan = A.plummer_jacobian(th, thE, e)
    ref = A.jacobian_to_mu_kappa_gamma(Aan)
    # compare det A = 1/mu: thin-lens and weak-field errors enter A at O(phi) ~ 2e-5 here
    assert np.allclose(1 / r.mu, 1 / ref["mu"], rtol=0, atol=1e-4)
    assert np.allclose(r.kappa, A.plummer_kappa(x, e / thE), rtol=0, atol=1e-4 * np.abs(ref["kappa"]).max())
    assert np.allclose(r.gamma1, ref["gamma1"], rtol=0, atol=3e-5)
    assert np.allclose(r.gamma2, ref["gamma2"], rtol=0, atol=3e-5)
    al = r.alpha()[:, 0]
    assert np.allclose(al, A.plummer_deflection(th, thE, e), rtol=1e-4)


@pytest.mark.parametrize("x", [0.2, 0.7, 1.0, 1.3, 3.0, 8.0])
def test_nfw_closed_forms_match_profile_quadrature(cosmo, x):
    # App. D's K, C and G against direct quadrature of the NFW profile
    L = A.NFWLens(cosmo, 1e14, 5.0, 0.25, 0.5)
    R = x * L.rs
    big = 1e4 * L.rs
    sig = L.sigma_trunc(R, rt=big)
    # correction for the part of the untruncated profile beyond 'big': rho ~ r^-3
    tail = 2 * L.dc * L.rho_c * L.rs ** 3 / (2 * big ** 2)
    assert abs((sig + tail) / (L.rs * L.dc * L.rho_c * A.nfw_K(x)) - 1) < 1e-6
    mcyl = L.mcyl_trunc(R, rt=big)
    # mass of the untruncated profile between the sphere 'big' and the cylinder: analytic tail
    mc_ref = 4 * math.pi * L.rs ** 3 * L.dc * L.rho_c * A.nfw_C(x)
    assert abs(mcyl / mc_ref - 1) < 1e-3
    G = 4 * A.nfw_C(x) / (x * x) - A.nfw_K(x)
    assert abs(A.nfw_G(x) / G - 1) < 1e-12


def test_nfw_delta_c_definition(cosmo):
    # Eq. overdens: the mean density inside r200 is 200 rho_c
    L = A.NFWLens(cosmo, 1e14, 5.0, 0.25, 0.5)
    M = L.m3d(L.r200)
    assert abs(M / (200 * L.rho_c * 4 / 3 * math.pi * L.r200 ** 3) - 1) < 1e-12
    assert abs(M / 1e14 - 1) < 1e-12


def test_nfw_halo_deflection_and_magnification(cosmo):
    # a discretised, truncated NFW halo (Sec. 4.2): the traced deflection follows
    # the truncated analytic M_cyl; magnification to within shot noise
    n = 20000
    zl, zs = 0.25, 0.5
    chi_l = cosmo.chi(zl)
    pos, mass, info = inputs.nfw_halo(1e14, 5.0, zl, chi_l, n, seed=inputs.BASE_SEED + 2)
    L = A.NFWLens(cosmo, 1e14, 5.0, zl, zs)
    assert abs(info["r200_phys"] / L.r200 - 1) < 1e-6
    D_d, D_s, D_ds = A.thin_lens_distances(cosmo, zl, zs)
    b = np.array([0.3, 0.6, 1.0, 1.6]) * L.r200
    ang = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    th = np.array([[bb / D_d * math.cos(a), bb / D_d * math.sin(a)] for bb in b for a in ang])
    r = oracle.trace(cosmo, oracle.MassField(pos, mass, 5e-3), zs, th, theta_r=ARCSEC, schedule=1,
                     n_steps=300, lens_chi=chi_l, asinh_s=5e-3)
    al = np.linalg.norm(r.alpha()[:, 0], axis=1).reshape(len(b), len(ang)).mean(axis=1)
    mu = r.mu.reshape(len(b), len(ang)).mean(axis=1)
    for i, bb in enumerate(b):
        a_ref = D_ds / D_s * 4 * oracle.mu_G() * L.mcyl_trunc(bb) / bb
        assert abs(al[i] / a_ref - 1) < 0.02
        mu_ref = L.lens_trunc(bb / D_d)[2]
        assert abs(mu[i] / mu_ref - 1) < 0.03 * mu_ref

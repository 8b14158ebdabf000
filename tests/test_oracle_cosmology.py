"""Pins for the oracle's background cosmology (Sec. 3.5, Sec. 5.1, App. E).

Everything here is checked against scipy quadrature of the defining
integrals, against closed-form identities, or against numbers the paper
prints (tests/golden/paper_values.txt).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import analytic as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol, cos, _ = [s.strip() for s in line.split("|")]
        c = None if cos == "-" else tuple(float(x) for x in cos.split())
        out[name] = (float(val), float(tol), c)
    return out


def quad(f, a, b):
    v, _ = integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=200)
    return v


@pytest.mark.parametrize("z", [0.05, 0.25, 0.5, 1.0, 1.5])
def test_chi_matches_quadrature(cosmo, z):
    E = lambda x: math.sqrt(0.3 * (1 + x) ** 3 + 0.7)
    ref = quad(lambda x: 1 / E(x), 0, z) * 2997.92458 / 0.7
    assert abs(cosmo.chi(z) / ref - 1) < 1e-13
    assert abs(cosmo.z_of_chi(cosmo.chi(z)) - z) < 1e-13


@pytest.mark.parametrize("z", [0.1, 0.5, 1.5])
def test_empty_beam_distance_matches_quadrature(cosmo, z):
    E = lambda x: math.sqrt(0.3 * (1 + x) ** 3 + 0.7)
    ref = quad(lambda x: 1 / ((1 + x) ** 2 * E(x)), 0, z) * 2997.92458 / 0.7
    assert abs(cosmo.D_eb(z) / ref - 1) < 1e-13
    assert abs(cosmo.D_fb(z) - cosmo.chi(z) / (1 + z)) < 1e-12


def test_scale_factor_today_is_one(cosmo):
    # Eq. scalefac: a = R(t)/R(0); the corrected t0 of Eq. lookbacksingularity gives a(0) = 1
    assert abs(cosmo.a_of_t(0.0) - 1.0) < 1e-15
    # da/dt_lookback at t = 0 is -H0
    assert abs(cosmo.adot_of_t(0.0) / -cosmo.H0() - 1) < 1e-14


def test_printed_t0_is_garbled(cosmo):
    # the literal Eq. lookbacksingularity (asinh of OL/OM) would give a(0) != 1
    H0 = cosmo.H0()
    t0_lit = 2 / (3 * H0 * math.sqrt(0.7)) * math.asinh(0.7 / 0.3)
    a0 = (0.3 / 0.7 * math.sinh(1.5 * math.sqrt(0.7) * H0 * t0_lit) ** 2) ** (1 / 3)
    assert abs(a0 - 1) > 0.1
    assert abs(cosmo.t0() / (2 / (3 * H0 * math.sqrt(0.7)) * math.asinh(math.sqrt(0.7 / 0.3))) - 1) < 1e-15


@pytest.mark.parametrize("z", [0.1, 0.5, 1.0, 2.0])
def test_scale_factor_at_lookback_time(cosmo, z):
    # lookback time t(z) = int dz/((1+z) H) by quadrature; Eq. scalefac2 must give 1/(1+z)
    E = lambda x: math.sqrt(0.3 * (1 + x) ** 3 + 0.7)
    t = quad(lambda x: 1 / ((1 + x) * E(x)), 0, z) / cosmo.H0()
    assert abs(cosmo.a_of_t(t) * (1 + z) - 1) < 1e-12
    # da/dt from a central difference of a(t)
    h = 1e-3
    fd = (cosmo.a_of_t(t + h) - cosmo.a_of_t(t - h)) / (2 * h)
    assert abs(cosmo.adot_of_t(t) / fd - 1) < 1e-8


def test_schedule_sums_to_empty_beam_distance(cosmo):
    # d lambda = a^2 dx3 on the unperturbed ray, and int a^2 dchi = D_eb (App. E)
    chi_s = cosmo.chi(0.5)
    for kind, n in ((0, 7), (0, 1000), (1, 1000), (1, 2000)):
        dl, nodes = cosmo.schedule(chi_s, kind, n, cosmo.chi(0.25), 5e-3)
        assert nodes[0] == 0.0 and nodes[-1] == chi_s
        assert np.all(np.diff(nodes) > 0) and np.all(dl > 0)
        assert abs(dl.sum() / cosmo.D_eb(0.5) - 1) < 1e-12
        # each step: a^2 between the end-point values
        zs = [cosmo.z_of_chi(x) for x in nodes[:: max(1, n // 50)]]
        assert np.all(np.diff(zs) > 0)


def test_asinh_nodes_cluster_at_lens(cosmo):
    chi_s, chi_l, s = cosmo.chi(0.5), cosmo.chi(0.25), 2e-3
    dl, nodes = cosmo.schedule(chi_s, 1, 1000, chi_l, s)
    u = np.arcsinh((nodes - chi_l) / s)
    du = np.diff(u)
    assert np.allclose(du, du.mean(), rtol=1e-6, atol=1e-9)
    step = np.diff(nodes)
    k = np.argmin(np.abs(nodes[:-1] - chi_l))
    assert step[k] < 1e-3 * step.max()


def test_golden_full_beam_minimum_magnification():
    val, tol, cos = golden()["mu_fb_min_z0.5"]
    c = oracle.Cosmology(*cos)
    mu = (c.D_fb(0.5) / c.D_eb(0.5)) ** 2
    assert abs(mu / val - 1) < tol


def test_golden_angular_diameter_distance():
    val, tol, cos = golden()["D_A_z0.5_hinvMpc"]
    c = oracle.Cosmology(*cos)
    assert abs(c.D_fb(0.5) * cos[2] / val - 1) < tol


def test_golden_box_count():
    val, tol, cos = golden()["boxes_to_z0.5"]
    c = oracle.Cosmology(*cos)
    n = c.chi(0.5) * cos[2] / 50.0
    assert abs(n / val - 1) < tol


def test_golden_nfw_angular_size():
    val, tol, cos = golden()["nfw_2r200_arcsec"]
    c = oracle.Cosmology(*cos)
    r = A.r200(c, 1e14, 0.35)
    D_d = c.chi(0.35) / 1.35
    assert abs(2 * r / D_d * 206264.80624709636 / val - 1) < tol


def test_golden_einstein_radius():
    val, tol, cos = golden()["schw_theta_E_arcsec"]
    c = oracle.Cosmology(*cos)
    th = A.theta_einstein(c, 1e15, 0.35, 0.8) * 206264.80624709636
    assert abs(th / val - 1) < tol


def test_mu_G_value():
    # G Msun / c^2 = 1476.6 m  (IAU nominal GM_sun)
    assert abs(oracle.mu_G() * 3.0856775814913673e22 - 1476.6250385) < 1e-4

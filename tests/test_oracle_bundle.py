"""Pins of the oracle's bundle reducer for the paper's bundle: a central ray
and a regular polygon of rays (Sec. 3.1; 8 rays plus the anchor in Sec. 5.2),
reduced to the lens-map Jacobian of Eq. lensmap and mu, kappa, gamma of
Eq. magnification.

- For an exactly linear lens map the least-squares fit must return that map
  for any polygon (size, orientation, regular or not): this fixes the
  normal matrix and its normalisation independently of the ring size.
- Traced through a point lens and a Plummer sphere with rings of 8 at any
  orientation, the bundle must give the closed forms of App. C and of the
  Plummer sphere at the tolerances the rings of 4 meet.
- The polygon's orientation changes mu, kappa, |gamma| only at the bundle's
  nonlinear order (theta_r^2), and rotates nothing."""
import math

import numpy as np
import pytest

import inputs
import oracle
from oracle import analytic as A


def _fit(A0, dth, chi_s=1888.6, beta0=(3e-3, -1e-3)):
    n = dth.shape[0]
    xy = np.zeros((n + 1, 2))
    xy[0] = np.asarray(beta0) * chi_s
    xy[1:] = (np.asarray(beta0) + dth @ A0.T) * chi_s
    return oracle.bundle_jacobian(n, np.zeros(2), dth, xy.ravel(), chi_s)


def _expect(A0):
    det = A0[0, 0] * A0[1, 1] - A0[0, 1] * A0[1, 0]
    return np.array([1 / det, 1 - 0.5 * (A0[0, 0] + A0[1, 1]), 0.5 * (A0[1, 1] - A0[0, 0]),
                     -0.5 * (A0[0, 1] + A0[1, 0]), 0.5 * (A0[0, 1] - A0[1, 0])])


@pytest.mark.parametrize("n_ring", [3, 4, 5, 6, 7, 8])
def test_linear_map_is_recovered_exactly(n_ring):
    g = inputs.rng(400 + n_ring)
    for trial in range(6):
        A0 = np.eye(2) + g.normal(size=(2, 2)) * 0.4
        if trial % 2:
            A0[0] *= -1  # negative parity
        phase = g.uniform(0, 2 * np.pi)
        r = 10 ** g.uniform(-7, -3)
        ang = phase + 2 * np.pi * np.arange(n_ring) / n_ring
        dth = r * np.stack([np.cos(ang), np.sin(ang)], 1)
        out = _fit(A0, dth)
        exp = _expect(A0)
        assert np.allclose(out[:5], exp, rtol=1e-9, atol=1e-9 * np.abs(exp).max())
        # an irregular polygon of the same size: still the same map
        dth2 = dth * g.uniform(0.5, 1.5, (n_ring, 1)) + r * 0.2 * g.normal(size=(n_ring, 2))
        out2 = _fit(A0, dth2)
        assert np.allclose(out2[:5], exp, rtol=1e-9, atol=1e-9 * np.abs(exp).max())


def test_ring_of_two_is_rejected(cosmo):
    f = oracle.MassField(np.zeros((0, 3)), np.zeros(0), 0.0)
    with pytest.raises(ValueError):
        oracle.trace(cosmo, f, 0.5, np.zeros((1, 2)), n_ring=2, n_steps=8)


@pytest.fixture(scope="module")
def c1_ring8(cosmo):
    cfg = inputs.config_c1()
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    out = {}
    for phase in (0.0, 0.37, math.pi / 8):
        out[phase] = oracle.trace(cosmo, f, cfg["z_s"], cfg["theta"], n_ring=8, theta_r=cfg["theta_r"],
                                  phase=phase, schedule=1, n_steps=cfg["n_steps"], lens_chi=cfg["lens_chi"],
                                  asinh_s=cfg["asinh_s"])
    return cfg, out


@pytest.mark.parametrize("phase", [0.0, 0.37, math.pi / 8])
def test_ring_of_eight_point_lens(c1_ring8, phase):
    cfg, res = c1_ring8
    r = res[phase]
    x = cfg["x"]
    ok = np.abs(np.abs(x) - 1) > 0.05
    with np.errstate(divide="ignore"):
        mu = A.schw_mu_image(np.abs(x))
    assert np.abs(r.mu / mu - 1)[ok].max() < 3e-4
    far = np.abs(x) > 1.5
    assert np.abs(r.mu / mu - 1)[far].max() < 1e-5
    assert np.all(np.abs(r.kappa[far]) < 1e-5)
    assert np.allclose(np.hypot(r.gamma1, r.gamma2)[far], A.schw_gamma(np.abs(x[far])), rtol=1e-4)
    assert np.all(np.abs(r.omega) < 1e-6)
    assert np.all(((r.mu < 0) == (np.abs(x) < 1))[ok])
    # the two images of u = 1.5 add up to the total magnification
    assert abs((abs(r.mu[-2]) + abs(r.mu[-1])) / A.schw_mu_total(1.5) - 1) < 3e-4
    # the ring rays start on the polygon of radius theta_r at this orientation
    th = r.ray_theta()
    d = th[:, 1:] - th[:, :1]
    ang = np.arctan2(d[..., 1], d[..., 0])
    ref = phase + 2 * np.pi * np.arange(8) / 8
    assert np.allclose(np.angle(np.exp(1j * (ang - ref))), 0, atol=1e-9)
    assert np.allclose(np.linalg.norm(d, axis=-1), cfg["theta_r"], rtol=1e-9)


def test_ring_orientation_changes_only_nonlinear_order(c1_ring8):
    cfg, res = c1_ring8
    x = cfg["x"]
    ok = np.abs(np.abs(x) - 1) > 0.05
    r0 = res[0.0]
    for phase in (0.37, math.pi / 8):
        r = res[phase]
        # relative changes of order (theta_r / theta)^2 ~ 1e-6 at most here
        assert np.abs(r.mu / r0.mu - 1)[ok].max() < 1e-5
        g0, g = np.hypot(r0.gamma1, r0.gamma2), np.hypot(r.gamma1, r.gamma2)
        assert np.abs(g / g0 - 1)[ok].max() < 1e-5
        assert np.abs(r.kappa - r0.kappa)[ok].max() < 1e-8


def test_ring_of_four_and_eight_agree(cosmo, c1_ring8):
    cfg, res = c1_ring8
    f = oracle.MassField(cfg["pos"], cfg["mass"], 0.0)
    r4 = oracle.trace(cosmo, f, cfg["z_s"], cfg["theta"], n_ring=4, theta_r=cfg["theta_r"], schedule=1,
                      n_steps=cfg["n_steps"], lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    ok = np.abs(np.abs(cfg["x"]) - 1) > 0.05
    assert np.abs(res[0.0].mu / r4.mu - 1)[ok].max() < 1e-5


@pytest.mark.parametrize("phase", [0.0, 0.2])
def test_ring_of_eight_plummer_lens(cosmo, phase):
    M, zl, zs = 1e13, 0.25, 0.5
    chi_l = cosmo.chi(zl)
    thE = A.theta_einstein(cosmo, M, zl, zs)
    eps = 0.7 * thE * chi_l
    e = eps / chi_l
    pos, mass = inputs.plummer_particle(M, chi_l)
    x = np.array([0.3, 0.8, 1.6, 3.0])
    th = np.stack([x * thE * 0.6, x * thE * 0.8], 1)
    r = oracle.trace(cosmo, oracle.MassField(pos, mass, eps), zs, th, n_ring=8, phase=phase, theta_r=1e-3 * thE,
                     schedule=1, n_steps=1000, lens_chi=float(pos[0, 2]), asinh_s=eps)
    ref = A.jacobian_to_mu_kappa_gamma(A.plummer_jacobian(th, thE, e))
    assert np.allclose(1 / r.mu, 1 / ref["mu"], rtol=0, atol=1e-4)
    assert np.allclose(r.kappa, A.plummer_kappa(x, e / thE), rtol=0, atol=1e-4 * np.abs(ref["kappa"]).max())
    assert np.allclose(r.gamma1, ref["gamma1"], rtol=0, atol=3e-5)
    assert np.allclose(r.gamma2, ref["gamma2"], rtol=0, atol=3e-5)

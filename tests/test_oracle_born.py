"""Pins of the oracle's Born approximation (Sec. 6: convergence and shear from
the Hessian of psi along the unperturbed line of sight) and of the prism
Hessian used for its mean subtraction."""
import math

import numpy as np
import pytest

import inputs
import oracle
import oracle.analytic as A


@pytest.mark.parametrize("p", [[0.3, 0.7, 4.0], [3.5, -1.5, 8.5], [6.0, 1.0, 12.0]])
def test_prism_hessian_is_the_derivative_of_the_gradient(p):
    lo, hi, p = np.array([-3.0, -2.0, 1.0]), np.array([4.0, 5.0, 9.0]), np.array(p)
    H = oracle.prism_hessian(lo, hi, p)
    h = 1e-4
    num = np.zeros((3, 3))
    for j in range(3):
        d = np.zeros(3)
        d[j] = h
        num[:, j] = (oracle.prism(lo, hi, p + d)[1:] - oracle.prism(lo, hi, p - d)[1:]) / (2 * h)
    full = np.array([[H[0], H[1], H[2]], [H[1], H[3], H[4]], [H[2], H[4], H[5]]])
    assert np.max(np.abs(full - num)) < 1e-7
    inside = np.all((p > lo) & (p < hi))
    # Poisson: the trace is -4 pi inside the prism, 0 outside
    assert H[0] + H[3] + H[5] == pytest.approx(-4 * math.pi if inside else 0.0, abs=1e-12)


def test_born_of_a_plummer_lens_is_its_thin_lens_jacobian(cosmo):
    # one Plummer-softened particle: kappa and gamma of the straight-line
    # integral equal the thin Plummer lens (projected mass M R^2 / (R^2 + eps^2))
    M, zl, zs, eps = 1e13, 0.3, 1.0, 0.02
    chi_l = cosmo.chi(zl)
    thE = A.theta_einstein(cosmo, M, zl, zs)
    D_d = chi_l / (1 + zl)
    e = eps / (1 + zl) / D_d  # angular softening (eps is comoving)
    x = np.array([0.3, 1.0, 2.5, 6.0])
    phi = np.array([0.2, 1.1, 2.0, 4.0])
    th = np.stack([x * thE * np.cos(phi), x * thE * np.sin(phi)], 1)
    f = oracle.MassField(np.array([[0.0, 0.0, chi_l]]), np.array([M]), eps)
    b = oracle.born(cosmo, f, zs, th, schedule=1, n_steps=4000, lens_chi=chi_l, asinh_s=eps)
    Aj = A.plummer_jacobian(th, thE, e)
    kap = 1 - 0.5 * (Aj[:, 0, 0] + Aj[:, 1, 1])
    g1 = 0.5 * (Aj[:, 1, 1] - Aj[:, 0, 0])
    g2 = -0.5 * (Aj[:, 0, 1] + Aj[:, 1, 0])
    scale = np.abs(kap) + np.hypot(g1, g2)
    for got, want in ((b[:, 0], kap), (b[:, 1], g1), (b[:, 2], g2)):
        assert np.all(np.abs(got - want) < 2e-4 * scale)


def test_born_of_empty_space_is_zero(cosmo):
    f = oracle.MassField(np.zeros((0, 3)), np.zeros(0), 0.01)
    b = oracle.born(cosmo, f, 0.7, [[1e-3, 2e-3]], n_steps=50)
    assert np.all(b == 0.0)


def test_born_matches_the_traced_weak_lensing(cosmo):
    # a weak, extended lens (one Plummer sphere of 0.3 Mpc softening): the
    # ray-traced bundles' kappa and gamma agree with the Born values up to the
    # second-order terms the Born approximation drops, O(kappa^2)
    M, zl, zs, eps = 5e13, 0.3, 1.0, 0.3
    chi_l = cosmo.chi(zl)
    f = oracle.MassField(np.array([[0.0, 0.0, chi_l]]), np.array([M]), eps)
    th = np.array([[0.9, 0.0], [0.7, 0.7], [0.0, -1.5], [2.0, 1.0]]) * eps / chi_l
    kw = dict(schedule=1, n_steps=800, lens_chi=chi_l, asinh_s=eps)
    b = oracle.born(cosmo, f, zs, th, **kw)
    t = oracle.trace(cosmo, f, zs, th, n_ring=4, theta_r=1e-3 * eps / chi_l, **kw)
    assert np.all(t.kappa > 0.002) and np.all(t.kappa < 0.1)
    bound = 3.0 * (t.kappa ** 2 + t.gamma1 ** 2 + t.gamma2 ** 2) + 1e-5
    assert np.all(np.abs(b[:, 0] - t.kappa) < bound)
    assert np.all(np.abs(b[:, 1] - t.gamma1) < bound)
    assert np.all(np.abs(b[:, 2] - t.gamma2) < bound)

"""Closed-form thin-lens solutions the oracle is pinned against (test
infrastructure).

* Schwarzschild (point) lens: App. C, Eqs. Eangle, Eradius, schwmu; the
  weak-field deflection 4GM/(c^2 b) (Sec. 2); the two-image total
  magnification (u^2+2)/(u sqrt(u^2+4)).
* Plummer sphere (the potential of one softened particle): projected mass
  M R^2/(R^2+eps^2), textbook closed form.
* NFW lens: App. D, Eqs. nfwkappa-nfwgmore and Eq. overdens, plus the
  truncated profile by direct quadrature (the model lens is cut at 2 r200).

All distances here are thin-lens angular-diameter distances of a flat
universe built from the oracle's comoving distance (Eq. raytracedistance).
"""
import math

import numpy as np
from scipy import integrate

from . import Cosmology, mu_G


def thin_lens_distances(cosmo, z_l, z_s):
    cl, cs = cosmo.chi(z_l), cosmo.chi(z_s)
    return cl / (1 + z_l), cs / (1 + z_s), (cs - cl) / (1 + z_s)


def sigma_crit(cosmo, z_l, z_s):
    """Eq. sigmacrit in Msun / Mpc^2 (physical)"""
    D_d, D_s, D_ds = thin_lens_distances(cosmo, z_l, z_s)
    return D_s / (4.0 * math.pi * mu_G() * D_d * D_ds)


def theta_einstein(cosmo, M, z_l, z_s):
    """Eq. Eangle (rad)"""
    D_d, D_s, D_ds = thin_lens_distances(cosmo, z_l, z_s)
    return math.sqrt(4.0 * mu_G() * M * D_ds / (D_d * D_s))


def rho_crit(cosmo, z):
    """Eq. critdens in Msun / Mpc^3 (physical)"""
    H = cosmo.H0() * cosmo.E(z)
    return 3.0 * H * H / (8.0 * math.pi * mu_G())


def r200(cosmo, M, z):
    """physical radius with mean enclosed density 200 rho_c(z)"""
    return (3.0 * M / (4.0 * math.pi * 200.0 * rho_crit(cosmo, z))) ** (1.0 / 3.0)


# ---------------------------------------------------------------------------
# point lens and Plummer sphere: reduced deflection alpha(theta) and Jacobian
# ---------------------------------------------------------------------------
def point_deflection(theta, theta_E):
    """reduced deflection theta_E^2 theta/|theta|^2 (weak field 4GM/(c^2 b))"""
    theta = np.asarray(theta, np.float64)
    r2 = np.sum(theta * theta, axis=-1, keepdims=True)
    return theta_E ** 2 * theta / r2


def plummer_deflection(theta, theta_E, e):
    """reduced deflection of a Plummer sphere with angular scale e"""
    theta = np.asarray(theta, np.float64)
    r2 = np.sum(theta * theta, axis=-1, keepdims=True)
    return theta_E ** 2 * theta / (r2 + e * e)


def plummer_jacobian(theta, theta_E, e):
    """A = I - d alpha / d theta for the Plummer sphere (e = 0: point lens)"""
    theta = np.asarray(theta, np.float64)
    tx, ty = theta[..., 0], theta[..., 1]
    q = tx * tx + ty * ty + e * e
    k = theta_E ** 2
    A = np.empty(theta.shape[:-1] + (2, 2))
    A[..., 0, 0] = 1.0 - k * (1.0 / q - 2.0 * tx * tx / q ** 2)
    A[..., 1, 1] = 1.0 - k * (1.0 / q - 2.0 * ty * ty / q ** 2)
    A[..., 0, 1] = A[..., 1, 0] = k * 2.0 * tx * ty / q ** 2
    return A


def jacobian_to_mu_kappa_gamma(A):
    det = A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    return dict(mu=1.0 / det, kappa=1.0 - 0.5 * (A[..., 0, 0] + A[..., 1, 1]),
                gamma1=0.5 * (A[..., 1, 1] - A[..., 0, 0]), gamma2=-0.5 * (A[..., 0, 1] + A[..., 1, 0]))


def schw_mu_image(x):
    """Eq. schwmu: magnification of the image at x = theta/theta_E"""
    x = np.asarray(x, np.float64)
    return 1.0 / (1.0 - x ** -4)


def schw_gamma(x):
    """shear of a point lens at x = theta/theta_E.  READING: Eq. schwgamma prints
    gamma = x; the form consistent with Eq. schwmu and kappa = 0 is x^-2."""
    return np.asarray(x, np.float64) ** -2


def schw_mu_total(u):
    """total two-image magnification at source offset u"""
    u = np.asarray(u, np.float64)
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def plummer_kappa(x, e):
    """convergence of a Plummer sphere, x and e in theta_E units"""
    return e * e / (x * x + e * e) ** 2


# ---------------------------------------------------------------------------
# NFW lens (Sec. 4.2 Eq. nfwprof / overdens; App. D)
# ---------------------------------------------------------------------------
def nfw_delta_c(c):
    """Eq. overdens"""
    return 200.0 / 3.0 * c ** 3 / (math.log(1 + c) - c / (1 + c))


def nfw_K(x):
    """Eq. nfwK"""
    x = float(x)
    if x < 1:
        return 2.0 / (x * x - 1) * (1 - 2.0 / math.sqrt(1 - x * x) * math.atanh(math.sqrt((1 - x) / (1 + x))))
    if x == 1:
        return 2.0 / 3.0
    return 2.0 / (x * x - 1) * (1 - 2.0 / math.sqrt(x * x - 1) * math.atan(math.sqrt((x - 1) / (1 + x))))


def nfw_C(x):
    """Eq. nfwC"""
    x = float(x)
    if x < 1:
        return math.log(x / 2) + math.acosh(1 / x) / math.sqrt(1 - x * x)
    if x == 1:
        return math.log(x / 2) + 1.0
    return math.log(x / 2) + math.acos(1 / x) / math.sqrt(x * x - 1)


def nfw_G(x):
    """Eqs. nfwG, nfwgless, nfwgmore"""
    x = float(x)
    if x < 1:
        at = math.atanh(math.sqrt((1 - x) / (1 + x)))
        return (8 * at / (x * x * math.sqrt(1 - x * x)) + 4 / (x * x) * math.log(x / 2)
                - 2 / (x * x - 1) + 4 * at / ((x * x - 1) * math.sqrt(1 - x * x)))
    if x == 1:
        return 10.0 / 3.0 + 4 * math.log(0.5)
    at = math.atan(math.sqrt((x - 1) / (1 + x)))
    return (8 * at / (x * x * math.sqrt(x * x - 1)) + 4 / (x * x) * math.log(x / 2)
            - 2 / (x * x - 1) + 4 * at / (x * x - 1) ** 1.5)


class NFWLens:
    """Thin NFW lens (App. D) and the same profile truncated at r_t."""

    def __init__(self, cosmo, M200, conc, z_l, z_s, trunc=2.0):
        self.cosmo, self.z_l, self.z_s = cosmo, z_l, z_s
        self.rho_c = rho_crit(cosmo, z_l)
        self.r200 = r200(cosmo, M200, z_l)
        self.rs = self.r200 / conc
        self.dc = nfw_delta_c(conc)
        self.rt = trunc * self.r200
        self.Scr = sigma_crit(cosmo, z_l, z_s)
        self.D_d = thin_lens_distances(cosmo, z_l, z_s)[0]
        self.k0 = self.rs * self.dc * self.rho_c / self.Scr

    def rho(self, r):
        s = r / self.rs
        return self.dc * self.rho_c / (s * (1 + s) ** 2)

    # untruncated closed forms (App. D)
    def kappa_inf(self, R):
        return self.k0 * nfw_K(R / self.rs)

    def gamma_inf(self, R):
        return self.k0 * nfw_G(R / self.rs)

    def mcyl_inf(self, R):
        return 4 * math.pi * self.rs ** 3 * self.dc * self.rho_c * nfw_C(R / self.rs)

    # profile cut at r_t, by quadrature (independent of the closed forms)
    def sigma_trunc(self, R, rt=None):
        rt = self.rt if rt is None else rt
        if R >= rt:
            return 0.0
        zmax = math.sqrt(rt * rt - R * R)
        f = lambda z: self.rho(math.sqrt(R * R + z * z))
        brk = [p for p in (self.rs, R) if p < zmax]
        v, _ = integrate.quad(f, 0.0, zmax, points=brk or None, epsabs=0, epsrel=1e-12, limit=400)
        return 2.0 * v

    def m3d(self, r):
        s = r / self.rs
        return 4 * math.pi * self.dc * self.rho_c * self.rs ** 3 * (math.log1p(s) - s / (1 + s))

    def mcyl_trunc(self, R, rt=None):
        rt = self.rt if rt is None else rt
        if R >= rt:
            return self.m3d(rt)
        f = lambda r: 4 * math.pi * r * r * self.rho(r) * (1.0 - math.sqrt(1.0 - (R / r) ** 2))
        v, _ = integrate.quad(f, R, rt, epsabs=0, epsrel=1e-12, limit=400)
        return self.m3d(R) + v

    def lens_trunc(self, theta):
        """kappa, gamma, mu of the truncated lens at angle theta (rad)"""
        R = theta * self.D_d
        k = self.sigma_trunc(R) / self.Scr
        kb = self.mcyl_trunc(R) / (math.pi * R * R * self.Scr)
        g = kb - k
        return k, g, 1.0 / ((1 - k) ** 2 - g * g)

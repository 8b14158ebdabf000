"""FP64 CPU oracle for 3D ray-bundle lensing (Killedar et al. 2011).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library; the two meet only
through the seeded input generators of the ``inputs`` package.

The numerical work lives in ``orc.c`` (plain C, FP64, Neumaier sums); this
module marshals numpy arrays into it.  ``analytic`` holds the closed forms
(point lens, Plummer sphere, NFW) the oracle is pinned against.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class Cosmo(C.Structure):
    _fields_ = [("omega_m", C.c_double), ("omega_l", C.c_double), ("h", C.c_double)]


class Grid(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("lo", C.c_double * 3),
        ("h", C.c_double),
        ("n_int", C.c_int),
        ("val", C.POINTER(C.c_double)),
        ("y2", C.POINTER(C.c_double)),
        ("margin", C.c_double),
    ]


class Field(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("pos", C.POINTER(C.c_double)),
        ("mass", C.POINTER(C.c_double)),
        ("soft", C.POINTER(C.c_double)),
        ("soft_scalar", C.c_double),
        ("replicated", C.c_int),
        ("L", C.c_double),
        ("n_rep", C.c_int),
        ("rot", C.POINTER(C.c_int32)),
        ("shift", C.POINTER(C.c_double)),
        ("mean_subtract", C.c_int),
        ("grid", C.POINTER(Grid)),
        ("grid_cubes", C.c_int),
    ]


class TraceOpts(C.Structure):
    _fields_ = [
        ("n_ring", C.c_int),
        ("theta_r", C.c_double),
        ("phase", C.c_double),
        ("schedule", C.c_int),
        ("n_steps", C.c_int),
        ("lens_chi", C.c_double),
        ("asinh_s", C.c_double),
        ("max_extra", C.c_int),
        ("christoffel", C.c_int),
    ]


class HistOpts(C.Structure):
    _fields_ = [("bins", C.c_int), ("mu_min", C.c_double), ("mu_max", C.c_double)]


class MPOpts(C.Structure):
    _fields_ = [("n_ring", C.c_int), ("theta_r", C.c_double), ("phase", C.c_double), ("slices", C.c_int)]


F_NOCROSS, F_NONFINITE, F_NEGPARITY = 1, 2, 4

_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        pc = C.POINTER(Cosmo)
        for name in ("orc_E", "orc_chi", "orc_z_of_chi", "orc_a_of_t", "orc_adot_of_t",
                     "orc_D_fb", "orc_D_eb"):
            getattr(L, name).argtypes = [pc, C.c_double]
            getattr(L, name).restype = C.c_double
        for name in ("orc_t0", "orc_H0"):
            getattr(L, name).argtypes = [pc]
            getattr(L, name).restype = C.c_double
        L.orc_mu_G.argtypes = []
        L.orc_mu_G.restype = C.c_double
        L.orc_schedule.argtypes = [pc, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
        L.orc_schedule.restype = C.c_int
        L.orc_potential.argtypes = [C.POINTER(Field), C.c_int64, _dp, C.POINTER(C.c_int32), _dp, C.c_int]
        L.orc_potential.restype = C.c_int
        L.orc_prism.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_prism.restype = None
        L.orc_geodesic_rhs.argtypes = [pc, _dp, _dp, C.c_int, _dp]
        L.orc_geodesic_rhs.restype = None
        L.orc_trace.argtypes = [pc, C.POINTER(Field), C.c_double, C.c_int64, _dp, C.POINTER(TraceOpts),
                                _dp, _dp, C.POINTER(C.c_int32), _dp, C.c_int]
        L.orc_trace.restype = C.c_int
        L.orc_bundle_jacobian.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, _dp]
        L.orc_bundle_jacobian.restype = None
        L.orc_histogram.argtypes = [C.c_int64, _dp, C.POINTER(C.c_int32), C.POINTER(HistOpts),
                                    C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), _dp]
        L.orc_histogram.restype = C.c_int
        L.orc_replica_world.argtypes = [C.POINTER(Field), C.c_int, _dp]
        L.orc_replica_world.restype = None
        L.orc_prism_hessian.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_prism_hessian.restype = None
        L.orc_born.argtypes = [pc, C.POINTER(Field), C.c_double, C.c_int64, _dp, C.POINTER(TraceOpts), _dp, C.c_int]
        L.orc_born.restype = C.c_int
        L.orc_shear_histogram.argtypes = [C.c_int64, _dp, _dp, _dp, C.POINTER(C.c_int32), C.POINTER(HistOpts),
                                          C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), _dp]
        L.orc_shear_histogram.restype = C.c_int
        L.orc_spline_y2.argtypes = [C.c_int, _dp, C.c_int64, _dp]
        L.orc_spline_y2.restype = None
        L.orc_grid_y2.argtypes = [C.c_int, _dp, _dp]
        L.orc_grid_y2.restype = None
        L.orc_grid_eval.argtypes = [C.POINTER(Grid), _dp, _dp]
        L.orc_grid_eval.restype = None
        L.orc_rect_deflection.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_rect_deflection.restype = None
        L.orc_multiplane.argtypes = [pc, C.POINTER(Field), C.c_double, C.c_int64, _dp, C.POINTER(MPOpts), _dp, _dp,
                                     _dp, C.POINTER(C.c_int), _dp, C.c_int]
        L.orc_multiplane.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def default_threads():
    return max(1, os.cpu_count() or 1)


class Cosmology:
    """Flat LCDM background (Sec. 3.5, App. E)."""

    def __init__(self, omega_m=0.3, omega_l=0.7, h=0.7):
        self.c = Cosmo(omega_m, omega_l, h)
        self.omega_m, self.omega_l, self.h = omega_m, omega_l, h

    def _f(self, name, x):
        return getattr(lib(), name)(C.byref(self.c), float(x))

    E = lambda self, z: self._f("orc_E", z)
    chi = lambda self, z: self._f("orc_chi", z)
    z_of_chi = lambda self, chi: self._f("orc_z_of_chi", chi)
    a_of_t = lambda self, t: self._f("orc_a_of_t", t)
    adot_of_t = lambda self, t: self._f("orc_adot_of_t", t)
    D_fb = lambda self, z: self._f("orc_D_fb", z)
    D_eb = lambda self, z: self._f("orc_D_eb", z)

    def t0(self):
        return lib().orc_t0(C.byref(self.c))

    def H0(self):
        return lib().orc_H0(C.byref(self.c))

    def schedule(self, chi_s, kind, n_steps, chi_l=0.0, s=1.0):
        dl = np.zeros(n_steps)
        nodes = np.zeros(n_steps + 1)
        rc = lib().orc_schedule(C.byref(self.c), chi_s, int(kind), int(n_steps), chi_l, s, _p(dl), _p(nodes))
        if rc != 0:
            raise ValueError("orc_schedule failed: %d" % rc)
        return dl, nodes


def mu_G():
    return lib().orc_mu_G()


class MassField:
    """A particle mass distribution as the oracle sees it (Sec. 3.3, 5.2)."""

    def __init__(self, pos, mass, soft, replicated=False, L=0.0, rot=None, shift=None,
                 mean_subtract=False, grid=None, grid_cubes=0):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        n = self.pos.shape[0]
        self.mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (n,)))
        soft = np.asarray(soft, np.float64)
        self.soft = None if soft.ndim == 0 else np.ascontiguousarray(soft.reshape(n))
        self.soft_scalar = float(soft) if soft.ndim == 0 else 0.0
        self.replicated = bool(replicated)
        self.L = float(L)
        if replicated:
            self.rot = np.ascontiguousarray(np.asarray(rot, np.int32).reshape(-1, 9))
            self.shift = np.ascontiguousarray(np.asarray(shift, np.float64).reshape(-1, 3))
            self.n_rep = self.rot.shape[0]
        else:
            self.rot = np.zeros((1, 9), np.int32)
            self.shift = np.zeros((1, 3))
            self.n_rep = 1
        self.mean_subtract = bool(mean_subtract)
        self.f = Field(n, _p(self.pos), _p(self.mass),
                       _p(self.soft) if self.soft is not None else None, self.soft_scalar,
                       int(self.replicated), self.L, self.n_rep, _p(self.rot, C.c_int32), _p(self.shift),
                       int(self.mean_subtract), grid.pointer() if grid is not None else None, int(grid_cubes))
        self.grid = grid  # keeps the node arrays alive


def potential(field, pts, rep=None, nthreads=None):
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    n = pts.shape[0]
    rep = np.zeros(n, np.int32) if rep is None else np.ascontiguousarray(rep, np.int32)
    out = np.zeros((n, 4))
    rc = lib().orc_potential(C.byref(field.f), n, _p(pts), _p(rep, C.c_int32), _p(out),
                             nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_potential failed: %d" % rc)
    return out


def prism(lo, hi, r):
    lo, hi, r = (np.ascontiguousarray(x, np.float64) for x in (lo, hi, r))
    out = np.zeros(4)
    lib().orc_prism(_p(lo), _p(hi), _p(r), _p(out))
    return out


def geodesic_rhs(cosmo, y, F, christoffel=0):
    y = np.ascontiguousarray(y, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    dy = np.zeros(8)
    lib().orc_geodesic_rhs(C.byref(cosmo.c), _p(y), _p(F), int(christoffel), _p(dy))
    return dy


class TraceResult:
    def __init__(self, rays, bundles, steps, n_pairs, chi_s, theta, opts):
        self.rays = rays          # (n_b, nr, 8) final states at x3 = chi_s
        self.bundles = bundles    # (n_b, 6) mu, kappa, gamma1, gamma2, omega, flags
        self.steps = steps        # (n_b, nr) step at which each ray crossed
        self.n_pairs = n_pairs
        self.chi_s = chi_s
        self.theta = theta
        self.opts = opts

    mu = property(lambda s: s.bundles[:, 0])
    kappa = property(lambda s: s.bundles[:, 1])
    gamma1 = property(lambda s: s.bundles[:, 2])
    gamma2 = property(lambda s: s.bundles[:, 3])
    omega = property(lambda s: s.bundles[:, 4])
    flags = property(lambda s: s.bundles[:, 5].astype(np.int32))

    def beta(self):
        """source-plane tangent positions of every ray, (n_b, nr, 2)"""
        return self.rays[:, :, 1:3] / self.chi_s

    def ray_theta(self):
        o = self.opts
        nr = 1 + o.n_ring
        th = np.zeros((self.theta.shape[0], nr, 2))
        th[:, 0] = self.theta
        for k in range(1, nr):
            ang = o.phase + 2.0 * np.pi * (k - 1) / o.n_ring
            th[:, k, 0] = self.theta[:, 0] + o.theta_r * np.cos(ang)
            th[:, k, 1] = self.theta[:, 1] + o.theta_r * np.sin(ang)
        return th

    def alpha(self):
        """reduced deflection theta - beta of every ray, (n_b, nr, 2)"""
        return self.ray_theta() - self.beta()


def trace(cosmo, field, z_s, theta, n_ring=4, theta_r=1e-6, phase=0.0, schedule=0, n_steps=1000,
          lens_chi=0.0, asinh_s=1.0, max_extra=16, christoffel=0, nthreads=None):
    theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
    nb = theta.shape[0]
    nr = 1 + n_ring
    o = TraceOpts(n_ring, theta_r, phase, schedule, n_steps, lens_chi, asinh_s, max_extra, christoffel)
    rays = np.zeros((nb, nr, 8))
    bundles = np.zeros((nb, 6))
    steps = np.zeros((nb, nr), np.int32)
    npairs = C.c_double(0.0)
    rc = lib().orc_trace(C.byref(cosmo.c), C.byref(field.f), float(z_s), nb, _p(theta), C.byref(o),
                         _p(rays), _p(bundles), _p(steps, C.c_int32), C.byref(npairs),
                         nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_trace failed: %d" % rc)
    return TraceResult(rays, bundles, steps, npairs.value, cosmo.chi(z_s), theta, o)


def bundle_jacobian(n_ring, theta0, dtheta, xy, chi_s):
    theta0 = np.ascontiguousarray(theta0, np.float64)
    dtheta = np.ascontiguousarray(dtheta, np.float64)
    xy = np.ascontiguousarray(xy, np.float64)
    out = np.zeros(6)
    lib().orc_bundle_jacobian(int(n_ring), _p(theta0), _p(dtheta), _p(xy), float(chi_s), _p(out))
    return out


def histogram(mu, flags=None, bins=200, mu_min=0.5, mu_max=5.0):
    mu = np.ascontiguousarray(mu, np.float64)
    n = mu.shape[0]
    fl = None if flags is None else np.ascontiguousarray(flags, np.int32)
    counts = np.zeros(bins, np.uint64)
    wfix = np.zeros(bins, np.uint64)
    sc = np.zeros(8)
    o = HistOpts(bins, mu_min, mu_max)
    rc = lib().orc_histogram(n, _p(mu), _p(fl, C.c_int32) if fl is not None else None, C.byref(o),
                             _p(counts, C.c_uint64), _p(wfix, C.c_uint64), _p(sc))
    if rc != 0:
        raise ValueError("orc_histogram failed: %d" % rc)
    keys = ("n_used", "n_under", "n_over", "n_neg", "n_bad", "W_total", "mean_w", "sigma_w")
    return counts, wfix, dict(zip(keys, sc))


def shear_histogram(mu, gamma1, gamma2, flags=None, bins=200, g_min=1e-4, g_max=1.0):
    """shear PDF: bins in log10|gamma|, weight 1/|mu| (see orc.h)"""
    mu, g1, g2 = (np.ascontiguousarray(a, np.float64) for a in (mu, gamma1, gamma2))
    n = mu.shape[0]
    fl = None if flags is None else np.ascontiguousarray(flags, np.int32)
    counts = np.zeros(bins, np.uint64)
    wfix = np.zeros(bins, np.uint64)
    sc = np.zeros(8)
    o = HistOpts(bins, g_min, g_max)
    rc = lib().orc_shear_histogram(n, _p(mu), _p(g1), _p(g2), _p(fl, C.c_int32) if fl is not None else None,
                                   C.byref(o), _p(counts, C.c_uint64), _p(wfix, C.c_uint64), _p(sc))
    if rc != 0:
        raise ValueError("orc_shear_histogram failed: %d" % rc)
    keys = ("n_used", "n_under", "n_over", "n_neg", "n_bad", "W_total", "mean_w", "sigma_w")
    return counts, wfix, dict(zip(keys, sc))


def prism_hessian(lo, hi, r):
    lo, hi, r = (np.ascontiguousarray(x, np.float64) for x in (lo, hi, r))
    out = np.zeros(6)
    lib().orc_prism_hessian(_p(lo), _p(hi), _p(r), _p(out))
    return out


def born(cosmo, field, z_s, theta, schedule=0, n_steps=1000, lens_chi=0.0, asinh_s=1.0, nthreads=None):
    """Born-approximation (kappa, gamma1, gamma2) per line of sight, (n_b, 3)"""
    theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
    o = TraceOpts(4, 1e-6, 0.0, schedule, n_steps, lens_chi, asinh_s, 0, 0)
    out = np.zeros((theta.shape[0], 3))
    rc = lib().orc_born(C.byref(cosmo.c), C.byref(field.f), float(z_s), theta.shape[0], _p(theta), C.byref(o),
                        _p(out), nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_born failed: %d" % rc)
    return out


def replica_world(field, j):
    """world positions (n, 3) of replica j of a replicated MassField"""
    out = np.zeros((field.pos.shape[0], 3))
    lib().orc_replica_world(C.byref(field.f), int(j), _p(out))
    return out


def rect_deflection(lo, hi, x):
    """int over the rectangle [lo, hi] of (x - x') / |x - x'|^2 d^2x' (unit
    surface density), at the points x (n, 2)"""
    lo, hi = (np.ascontiguousarray(v, np.float64) for v in (lo, hi))
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 2)
    out = np.zeros_like(x)
    for i in range(x.shape[0]):
        xi = np.ascontiguousarray(x[i])
        o = np.zeros(2)
        lib().orc_rect_deflection(_p(lo), _p(hi), _p(xi), _p(o))
        out[i] = o
    return out


class MultiPlaneResult:
    def __init__(self, xs, bundles, planes, n_pairs, chi_s, theta, n_ring, theta_r, phase):
        self.xs = xs              # (n_b, nr, 2) comoving source-plane positions
        self.bundles = bundles    # (n_b, 6) mu, kappa, gamma1, gamma2, omega, flags
        self.planes = planes      # (n_planes, 4) chi, z, particles, slab thickness
        self.n_pairs = n_pairs
        self.chi_s = chi_s
        self.theta = theta
        self.n_ring, self.theta_r, self.phase = n_ring, theta_r, phase

    mu = property(lambda self: self.bundles[:, 0])
    kappa = property(lambda self: self.bundles[:, 1])
    gamma1 = property(lambda self: self.bundles[:, 2])
    gamma2 = property(lambda self: self.bundles[:, 3])
    omega = property(lambda self: self.bundles[:, 4])
    flags = property(lambda self: self.bundles[:, 5].astype(np.int32))

    def beta(self):
        return self.xs / self.chi_s

    def ray_theta(self):
        nr = 1 + self.n_ring
        th = np.zeros((self.theta.shape[0], nr, 2))
        th[:, 0] = self.theta
        for k in range(1, nr):
            ang = self.phase + 2.0 * np.pi * (k - 1) / self.n_ring
            th[:, k, 0] = self.theta[:, 0] + self.theta_r * np.cos(ang)
            th[:, k, 1] = self.theta[:, 1] + self.theta_r * np.sin(ang)
        return th

    def alpha(self):
        return self.ray_theta() - self.beta()


def multiplane(cosmo, field, z_s, theta, n_ring=4, theta_r=1e-6, phase=0.0, slices=1, nthreads=None):
    """the multiple lens-plane comparison system (Sec. 3.1): bundles traced
    through the field's projected slabs (see orc.c for the readings)"""
    theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
    n_b = theta.shape[0]
    nr = 1 + n_ring
    xs = np.zeros((n_b, nr, 2))
    bundles = np.zeros((n_b, 6))
    cap = (field.n_rep if field.replicated else 1) * slices
    planes = np.zeros((max(cap, 1), 4))
    npl = C.c_int(0)
    pairs = C.c_double(0.0)
    o = MPOpts(int(n_ring), float(theta_r), float(phase), int(slices))
    rc = lib().orc_multiplane(C.byref(cosmo.c), C.byref(field.f), float(z_s), n_b, _p(theta), C.byref(o), _p(xs),
                              _p(bundles), _p(planes), C.byref(npl), C.byref(pairs), nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_multiplane failed: %d" % rc)
    return MultiPlaneResult(xs, bundles, planes[:npl.value].copy(), pairs.value, cosmo.chi(z_s), theta, n_ring,
                            theta_r, phase)

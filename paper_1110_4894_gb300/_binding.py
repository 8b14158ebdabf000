"""ctypes marshalling for librt3d.so; names follow include/rt3d.h."""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTIMPL, ENOCOSMO, ENOFIELD = 0, -1, -2, -3, -4, -5, -6, -7
MIXED, FP64 = 0, 1
CHRISTOFFEL_PAPER, CHRISTOFFEL_DERIVED = 0, 1
SCHED_UNIFORM, SCHED_ASINH = 0, 1
F_NOCROSS, F_NONFINITE, F_NEGPARITY = 1, 2, 4


class Rt3dError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rt3d error %d: %s" % (code, msg))
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("christoffel", C.c_int), ("rays_per_thread", C.c_int),
                ("threads_per_block", C.c_int), ("splits", C.c_int), ("autotune", C.c_int),
                ("watchdog_s", C.c_double), ("time_kernels", C.c_int), ("variant", C.c_int),
                ("cluster", C.c_int)]


class Volume(C.Structure):
    _fields_ = [("replicated", C.c_int), ("box_length", C.c_double), ("n_replicas", C.c_int),
                ("rot", C.POINTER(C.c_int32)), ("shift", C.POINTER(C.c_double)), ("mean_subtract", C.c_int)]


class BundleOpts(C.Structure):
    _fields_ = [("n_ring", C.c_int), ("theta_r", C.c_double), ("phase", C.c_double), ("schedule", C.c_int),
                ("n_steps", C.c_int), ("lens_chi", C.c_double), ("asinh_s", C.c_double), ("max_extra", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint64)


class BundleResult(C.Structure):
    _fields_ = [("mu", _dp), ("kappa", _dp), ("gamma1", _dp), ("gamma2", _dp), ("omega", _dp),
                ("flags", _ip), ("ray_state", _dp), ("ray_steps", _ip)]


class HistOpts(C.Structure):
    _fields_ = [("bins", C.c_int), ("mu_min", C.c_double), ("mu_max", C.c_double)]


class Hist(C.Structure):
    _fields_ = [("counts", _up), ("wfix", _up), ("n_used", C.c_int64), ("n_under", C.c_int64),
                ("n_over", C.c_int64), ("n_neg", C.c_int64), ("n_bad", C.c_int64), ("W_total", C.c_double),
                ("mean_w", C.c_double), ("sigma_w", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("interactions", C.c_double), ("device_ms", C.c_double), ("force_ms", C.c_double),
                ("launches", C.c_int64), ("force_launches", C.c_int64), ("steps", C.c_int),
                ("rays_per_thread", C.c_int), ("threads_per_block", C.c_int), ("splits", C.c_int),
                ("variant", C.c_int), ("cluster", C.c_int)]


class GridOpts(C.Structure):
    _fields_ = [("n", C.c_int), ("lo", C.c_double * 3), ("h", C.c_double), ("n_int", C.c_int),
                ("mean_subtract", C.c_int)]


class Cone(C.Structure):
    _fields_ = [("field_id", C.c_int), ("z_s", C.c_double), ("n_bundles", C.c_int64), ("theta", _dp),
                ("n_steps", C.c_int)]


_lib = None


def library_path():
    return os.path.join(HERE, "librt3d.so")


def lib(build=True):
    """Load librt3d.so (building it from csrc/ with nvcc when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        from . import build as _b
        _b.build()
    path = library_path()
    if not os.path.exists(path):
        raise Rt3dError(ECUDA, "librt3d.so not found at %s; build it with __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "rt3d_create": ([C.POINTER(vp), C.c_int, C.POINTER(Options)], C.c_int),
        "rt3d_destroy": ([vp], C.c_int),
        "rt3d_set_cosmology": ([vp, C.c_double, C.c_double, C.c_double], C.c_int),
        "rt3d_load_particles": ([vp, C.c_int, C.c_int64, _dp, _dp, _dp, C.c_int, C.POINTER(Volume)], C.c_int),
        "rt3d_trace": ([vp, C.c_int, C.c_double, C.c_int64, _dp, C.POINTER(BundleOpts), C.POINTER(BundleResult)],
                       C.c_int),
        "rt3d_trace_device": ([vp, vp, C.c_int, C.c_double, C.c_int64, vp, C.POINTER(BundleOpts), vp, vp], C.c_int),
        "rt3d_trace_batch": ([vp, C.c_int, C.POINTER(Cone), C.POINTER(BundleOpts), C.POINTER(BundleResult)],
                             C.c_int),
        "rt3d_multiplane": ([vp, C.c_int, C.c_double, C.c_int64, _dp, C.POINTER(BundleOpts), C.c_int,
                             C.POINTER(BundleResult)], C.c_int),
        "rt3d_multiplane_device": ([vp, vp, C.c_int, C.c_double, C.c_int64, vp, C.POINTER(BundleOpts), C.c_int, vp,
                                    vp], C.c_int),
        "rt3d_trace_begin": ([vp, vp, C.c_int, C.c_double, C.c_int64, vp, C.POINTER(BundleOpts)], C.c_int),
        "rt3d_trace_advance": ([vp, vp, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "rt3d_trace_end": ([vp, vp, vp, vp], C.c_int),
        "rt3d_histogram": ([vp, C.c_int64, _dp, _ip, C.POINTER(HistOpts), C.POINTER(Hist)], C.c_int),
        "rt3d_histogram_combine": ([vp, C.c_int, C.c_int, C.POINTER(Hist), C.POINTER(Hist)], C.c_int),
        "rt3d_shear_histogram": ([vp, C.c_int64, _dp, _dp, _dp, _ip, C.POINTER(HistOpts), C.POINTER(Hist)],
                                 C.c_int),
        "rt3d_histogram_device": ([vp, vp, C.c_int64, vp, C.POINTER(HistOpts), vp, vp, vp], C.c_int),
        "rt3d_potential": ([vp, C.c_int, C.c_int64, _dp, _ip, _dp], C.c_int),
        "rt3d_born": ([vp, C.c_int, C.c_double, C.c_int64, _dp, C.POINTER(BundleOpts), _dp], C.c_int),
        "rt3d_watchdog_selftest": ([vp, C.c_double], C.c_int),
        "rt3d_load_grid": ([vp, C.c_int, C.c_int64, _dp, _dp, C.c_double, C.POINTER(GridOpts)], C.c_int),
        "rt3d_grid_nodes": ([vp, C.c_int, _dp], C.c_int),
        "rt3d_load_grid_box": ([vp, C.c_int, C.c_int64, _dp, _dp, C.c_double, C.POINTER(Volume), C.c_int,
                                C.POINTER(GridOpts)], C.c_int),
        "rt3d_schedule": ([vp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp], C.c_int),
        "rt3d_get_stats": ([vp, C.POINTER(Stats)], C.c_int),
        "rt3d_status_string": ([C.c_int], C.c_char_p),
        "rt3d_last_error": ([vp], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _p(a, ct=C.c_double):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


_HIST_KEYS = ("n_used", "n_under", "n_over", "n_neg", "n_bad", "W_total", "mean_w", "sigma_w")


def histogram_combine(parts):
    """rt3d_histogram_combine: the histogram of the union of disjoint sets of
    bundles from the parts' (counts, wfix, scalars); a host call of the
    library that needs no GPU and no context."""
    L = lib()
    keep = []
    arr = (Hist * len(parts))()
    bins = None
    for i, (c, w, sc) in enumerate(parts):
        c = np.ascontiguousarray(c, np.uint64)
        w = np.ascontiguousarray(np.asarray(w).view(np.uint64) if np.asarray(w).dtype == np.int64 else w, np.uint64)
        if bins is None:
            bins = c.shape[0]
        if c.shape[0] != bins or w.shape[0] != bins:
            raise ValueError("parts have different bin counts")
        keep += [c, w]
        arr[i] = Hist(_p(c, C.c_uint64), _p(w, C.c_uint64), *[int(sc[k]) for k in _HIST_KEYS[:5]],
                      *[float(sc[k]) for k in _HIST_KEYS[5:]])
    counts = np.zeros(bins, np.uint64)
    wfix = np.zeros(bins, np.uint64)
    h = Hist(_p(counts, C.c_uint64), _p(wfix, C.c_uint64))
    rc = L.rt3d_histogram_combine(None, len(parts), int(bins), arr, C.byref(h))
    if rc != 0:
        raise Rt3dError(rc, "rt3d_histogram_combine failed: %s" % L.rt3d_status_string(rc).decode())
    return counts, wfix, {k: getattr(h, k) for k in _HIST_KEYS}


class Context:
    """One library context on one CUDA device (rt3d_create ... rt3d_destroy)."""

    def __init__(self, device=0, precision=MIXED, christoffel=CHRISTOFFEL_PAPER, rays_per_thread=0,
                 threads_per_block=0, splits=0, autotune=0, watchdog_s=0.0, time_kernels=0, variant=0, cluster=0):
        self.L = lib()
        self.h = C.c_void_p()
        self.opt = Options(precision, christoffel, rays_per_thread, threads_per_block, splits, autotune,
                           watchdog_s, time_kernels, variant, cluster)
        rc = self.L.rt3d_create(C.byref(self.h), int(device), C.byref(self.opt))
        if rc != OK:
            raise Rt3dError(rc, self.L.rt3d_status_string(rc).decode())
        self._keep = {}

    def _check(self, rc):
        if rc != OK:
            raise Rt3dError(rc, self.L.rt3d_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.L.rt3d_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_cosmology(self, omega_m=0.3, omega_l=0.7, h=0.7):
        self._check(self.L.rt3d_set_cosmology(self.h, omega_m, omega_l, h))

    def load_particles(self, field_id, pos, mass, soft, replicated=False, box_length=0.0, rot=None, shift=None,
                       mean_subtract=False):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        n = pos.shape[0]
        mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (n,)))
        soft = np.asarray(soft, np.float64)
        pp = soft.ndim > 0 and soft.size == n and n > 1
        soft = np.ascontiguousarray(soft.reshape(-1) if pp else soft.reshape(-1)[:1])
        vol = None
        if replicated:
            rot = np.ascontiguousarray(np.asarray(rot, np.int32).reshape(-1, 9))
            shift = np.ascontiguousarray(np.asarray(shift, np.float64).reshape(-1, 3))
            vol = Volume(1, float(box_length), rot.shape[0], _p(rot, C.c_int32), _p(shift), int(bool(mean_subtract)))
        self._check(self.L.rt3d_load_particles(self.h, int(field_id), n, _p(pos), _p(mass), _p(soft), int(pp),
                                               C.byref(vol) if vol is not None else None))

    def load_grid(self, field_id, pos, mass, soft, lo, h, n, n_int=2, mean_subtract=False):
        """rt3d_load_grid: the grid path's field (CIC, zero-padded FFT, App. B splines)."""
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        npart = pos.shape[0]
        mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (npart,)))
        g = GridOpts(int(n), (C.c_double * 3)(*[float(v) for v in lo]), float(h), int(n_int), int(bool(mean_subtract)))
        self._grid_n = getattr(self, "_grid_n", {})
        self._grid_n[int(field_id)] = int(n)
        self._check(self.L.rt3d_load_grid(self.h, int(field_id), npart, _p(pos), _p(mass), float(soft), C.byref(g)))

    def load_grid_box(self, field_id, pos, mass, soft, box_length, rot, shift, cubes, n, n_int=2,
                      mean_subtract=True):
        """rt3d_load_grid_box: a replicated box on cube grids (n^3 nodes per cube)."""
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        npart = pos.shape[0]
        mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (npart,)))
        rot = np.ascontiguousarray(np.asarray(rot, np.int32).reshape(-1, 9))
        shift = np.ascontiguousarray(np.asarray(shift, np.float64).reshape(-1, 3))
        vol = Volume(1, float(box_length), rot.shape[0], _p(rot, C.c_int32), _p(shift), 0)
        g = GridOpts(int(n), (C.c_double * 3)(0.0, 0.0, 0.0), 0.0, int(n_int), int(bool(mean_subtract)))
        self._grid_n = getattr(self, "_grid_n", {})
        self._grid_n[int(field_id)] = (int(n), rot.shape[0] * int(cubes))
        self._check(self.L.rt3d_load_grid_box(self.h, int(field_id), npart, _p(pos), _p(mass), float(soft),
                                              C.byref(vol), int(cubes), C.byref(g)))

    def grid_nodes(self, field_id):
        """rt3d_grid_nodes: phi and grad phi on the nodes, (4, n, n, n) (boxes:
        (cells, 4, n, n, n))."""
        n = self._grid_n[int(field_id)]
        if isinstance(n, tuple):
            n, cells = n
            out = np.zeros((cells, 4, n, n, n))
            self._check(self.L.rt3d_grid_nodes(self.h, int(field_id), _p(out)))
            return out
        out = np.zeros((4, n, n, n))
        self._check(self.L.rt3d_grid_nodes(self.h, int(field_id), _p(out)))
        return out

    @staticmethod
    def bundle_opts(n_ring=4, theta_r=1e-6, phase=0.0, schedule=SCHED_UNIFORM, n_steps=1000, lens_chi=0.0,
                    asinh_s=1.0, max_extra=16):
        return BundleOpts(n_ring, theta_r, phase, schedule, n_steps, lens_chi, asinh_s, max_extra)

    def trace(self, field_id, z_s, theta, want_rays=False, **kw):
        theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
        nb = theta.shape[0]
        o = self.bundle_opts(**kw)
        nr = 1 + o.n_ring
        out = {k: np.zeros(nb) for k in ("mu", "kappa", "gamma1", "gamma2", "omega")}
        out["flags"] = np.zeros(nb, np.int32)
        rays = np.zeros((nb, nr, 8)) if want_rays else None
        steps = np.zeros((nb, nr), np.int32) if want_rays else None
        res = BundleResult(_p(out["mu"]), _p(out["kappa"]), _p(out["gamma1"]), _p(out["gamma2"]), _p(out["omega"]),
                           _p(out["flags"], C.c_int32), _p(rays), _p(steps, C.c_int32))
        self._check(self.L.rt3d_trace(self.h, int(field_id), float(z_s), nb, _p(theta), C.byref(o), C.byref(res)))
        if want_rays:
            out["rays"] = rays
            out["steps"] = steps
        return out

    def born(self, field_id, z_s, theta, **kw):
        """rt3d_born: Born-approximation (kappa, gamma1, gamma2) per line of sight, (n, 3)."""
        theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
        o = self.bundle_opts(**kw)
        out = np.zeros((theta.shape[0], 3))
        self._check(self.L.rt3d_born(self.h, int(field_id), float(z_s), theta.shape[0], _p(theta), C.byref(o),
                                     _p(out)))
        return out

    def watchdog_selftest(self, limit_s=0.2):
        """rt3d_watchdog_selftest: returns the status code (ETIMEOUT is the pass)."""
        return self.L.rt3d_watchdog_selftest(self.h, float(limit_s))

    def trace_device(self, stream, field_id, z_s, n_bundles, d_theta, d_bundle_out, d_ray_out=None, **kw):
        """Enqueue a trace on a CUDA stream with device pointers (integers)."""
        o = self.bundle_opts(**kw)
        self._check(self.L.rt3d_trace_device(self.h, C.c_void_p(stream), int(field_id), float(z_s), int(n_bundles),
                                             C.c_void_p(d_theta), C.byref(o), C.c_void_p(d_bundle_out),
                                             C.c_void_p(d_ray_out) if d_ray_out else None))

    def multiplane(self, field_id, z_s, theta, slices=1, want_rays=False, **kw):
        """rt3d_multiplane: the bundles through the field's lens planes (Sec. 3.1);
        the same result dict as trace ("rays": (n, nr, 8) source-plane states)."""
        theta = np.ascontiguousarray(theta, np.float64).reshape(-1, 2)
        nb = theta.shape[0]
        o = self.bundle_opts(**kw)
        nr = 1 + o.n_ring
        r = {k: np.zeros(nb) for k in ("mu", "kappa", "gamma1", "gamma2", "omega")}
        r["flags"] = np.zeros(nb, np.int32)
        rays = np.zeros((nb, nr, 8)) if want_rays else None
        res = BundleResult(_p(r["mu"]), _p(r["kappa"]), _p(r["gamma1"]), _p(r["gamma2"]), _p(r["omega"]),
                           _p(r["flags"], C.c_int32), _p(rays) if want_rays else None, None)
        self._check(self.L.rt3d_multiplane(self.h, int(field_id), float(z_s), nb, _p(theta), C.byref(o),
                                           int(slices), C.byref(res)))
        if want_rays:
            r["rays"] = rays
        return r

    def multiplane_device(self, stream, field_id, z_s, n_bundles, d_theta, d_bundle_out, slices=1, d_ray_out=None,
                          **kw):
        """rt3d_multiplane_device: enqueue the lens-plane system with device pointers."""
        o = self.bundle_opts(**kw)
        self._check(self.L.rt3d_multiplane_device(self.h, C.c_void_p(stream), int(field_id), float(z_s),
                                                  int(n_bundles), C.c_void_p(d_theta), C.byref(o), int(slices),
                                                  C.c_void_p(d_bundle_out), C.c_void_p(d_ray_out) if d_ray_out else None))

    def trace_begin(self, stream, field_id, z_s, n_bundles, d_theta, **kw):
        """rt3d_trace_begin: open a trace in pieces (step table, initialiser) on stream."""
        o = self.bundle_opts(**kw)
        self._check(self.L.rt3d_trace_begin(self.h, C.c_void_p(stream), int(field_id), float(z_s), int(n_bundles),
                                            C.c_void_p(d_theta), C.byref(o)))

    def trace_advance(self, stream, n_stages):
        """rt3d_trace_advance: enqueue the next n_stages RK4 stages; returns the stages left."""
        left = C.c_int(0)
        self._check(self.L.rt3d_trace_advance(self.h, C.c_void_p(stream), int(n_stages), C.byref(left)))
        return left.value

    def trace_end(self, stream, d_bundle_out, d_ray_out=None):
        """rt3d_trace_end: the remaining stages and the bundle reducer."""
        self._check(self.L.rt3d_trace_end(self.h, C.c_void_p(stream), C.c_void_p(d_bundle_out),
                                          C.c_void_p(d_ray_out) if d_ray_out else None))

    def trace_batch(self, cones, want_rays=False, **kw):
        """cones: list of dicts with field_id, z_s, theta, n_steps."""
        o = self.bundle_opts(**kw)
        arr = (Cone * len(cones))()
        outs = (BundleResult * len(cones))()
        keep, results = [], []
        for i, c in enumerate(cones):
            th = np.ascontiguousarray(c["theta"], np.float64).reshape(-1, 2)
            nb = th.shape[0]
            nr = 1 + o.n_ring
            r = {k: np.zeros(nb) for k in ("mu", "kappa", "gamma1", "gamma2", "omega")}
            r["flags"] = np.zeros(nb, np.int32)
            if want_rays:
                r["rays"] = np.zeros((nb, nr, 8))
                r["steps"] = np.zeros((nb, nr), np.int32)
            keep.append(th)
            results.append(r)
            arr[i] = Cone(int(c["field_id"]), float(c["z_s"]), nb, _p(th), int(c.get("n_steps", o.n_steps)))
            outs[i] = BundleResult(_p(r["mu"]), _p(r["kappa"]), _p(r["gamma1"]), _p(r["gamma2"]), _p(r["omega"]),
                                   _p(r["flags"], C.c_int32), _p(r.get("rays")), _p(r.get("steps"), C.c_int32))
        self._check(self.L.rt3d_trace_batch(self.h, len(cones), arr, C.byref(o), outs))
        return results

    def histogram(self, mu, flags=None, bins=200, mu_min=0.5, mu_max=5.0):
        mu = np.ascontiguousarray(mu, np.float64)
        fl = None if flags is None else np.ascontiguousarray(flags, np.int32)
        counts = np.zeros(bins, np.uint64)
        wfix = np.zeros(bins, np.uint64)
        h = Hist(_p(counts, C.c_uint64), _p(wfix, C.c_uint64))
        o = HistOpts(bins, mu_min, mu_max)
        self._check(self.L.rt3d_histogram(self.h, mu.shape[0], _p(mu), _p(fl, C.c_int32), C.byref(o), C.byref(h)))
        sc = dict(n_used=h.n_used, n_under=h.n_under, n_over=h.n_over, n_neg=h.n_neg, n_bad=h.n_bad,
                  W_total=h.W_total, mean_w=h.mean_w, sigma_w=h.sigma_w)
        return counts, wfix, sc

    def shear_histogram(self, mu, gamma1, gamma2, flags=None, bins=200, g_min=1e-4, g_max=1.0):
        """rt3d_shear_histogram: |gamma| in log10 bins, weight 1/|mu|."""
        mu, g1, g2 = (np.ascontiguousarray(a, np.float64) for a in (mu, gamma1, gamma2))
        fl = None if flags is None else np.ascontiguousarray(flags, np.int32)
        counts = np.zeros(bins, np.uint64)
        wfix = np.zeros(bins, np.uint64)
        h = Hist(_p(counts, C.c_uint64), _p(wfix, C.c_uint64))
        o = HistOpts(bins, g_min, g_max)
        self._check(self.L.rt3d_shear_histogram(self.h, mu.shape[0], _p(mu), _p(g1), _p(g2), _p(fl, C.c_int32),
                                                C.byref(o), C.byref(h)))
        sc = dict(n_used=h.n_used, n_under=h.n_under, n_over=h.n_over, n_neg=h.n_neg, n_bad=h.n_bad,
                  W_total=h.W_total, mean_w=h.mean_w, sigma_w=h.sigma_w)
        return counts, wfix, sc

    def histogram_device(self, stream, n, d_bundle_out, d_counts, d_wfix, d_scalars, bins=200, mu_min=0.5,
                         mu_max=5.0):
        o = HistOpts(bins, mu_min, mu_max)
        self._check(self.L.rt3d_histogram_device(self.h, C.c_void_p(stream), int(n), C.c_void_p(d_bundle_out),
                                                 C.byref(o), C.c_void_p(d_counts), C.c_void_p(d_wfix),
                                                 C.c_void_p(d_scalars)))

    def potential(self, field_id, pts, rep=None):
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        rep = None if rep is None else np.ascontiguousarray(rep, np.int32)
        out = np.zeros((pts.shape[0], 4))
        self._check(self.L.rt3d_potential(self.h, int(field_id), pts.shape[0], _p(pts), _p(rep, C.c_int32), _p(out)))
        return out

    def schedule(self, z_s, kind, n_steps, chi_l=0.0, s=1.0):
        dl = np.zeros(n_steps)
        chi = C.c_double(0.0)
        self._check(self.L.rt3d_schedule(self.h, float(z_s), int(kind), int(n_steps), float(chi_l), float(s),
                                         _p(dl), C.byref(chi)))
        return dl, chi.value

    def stats(self):
        s = Stats()
        self._check(self.L.rt3d_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}


def _potential_device_noalloc(self, stream, field_id, n, d_pts, d_rep, d_out):
    """rt3d_potential_device_noalloc: the pair sum on device arrays with no
    device allocation (scratch in a static device array); d_pts holds all x1,
    then all x2, then all x3; enqueued on stream."""
    fn = self.L.rt3d_potential_device_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    self._check(fn(self.h, C.c_void_p(stream), int(field_id), int(n), C.c_void_p(d_pts),
                   C.c_void_p(d_rep) if d_rep else None, C.c_void_p(d_out)))


Context.potential_device_noalloc = _potential_device_noalloc

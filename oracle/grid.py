"""Grid path of the oracle (Sec. 3.3 and App. B): the field of a particle
set computed on a regular node grid and interpolated at the ray positions.

TEST INFRASTRUCTURE, like the rest of ``oracle``.

Steps, in the paper's order:

1. Cloud-in-cell assignment of the particle masses to the nodes
   x = lo + h (i1, i2, i3), i = 0..n-1 (Sec. 3.3, Hockney & Eastwood CIC);
   mass that falls on nodes outside the grid is dropped.  Optionally the mean
   node mass is subtracted (Sec. 3.3 removes the mean density).
2. phi and grad phi on the nodes by a zero-padded FFT convolution (Eqs. psi,
   derivs with phi = a psi) of the node masses with the kernels
       K_phi(d) = -mu_G (|d|^2 + eps^2)^(-1/2),
       K_g(d)   =  mu_G d (|d|^2 + eps^2)^(-3/2),
   d = x_node - x_source_node; for eps = 0 the self term d = 0 is zero.  The
   FFT (numpy) is only a fast way to form the plain double sum over nodes,
   which a test checks on a small grid.
3. Natural cubic-spline second derivatives of every line along x3, once per
   mass distribution (App. B), and the App. B five-step evaluation, both in
   ``orc.c``.
"""
import ctypes as C

import numpy as np

from . import Grid, _p, lib, mu_G


def cic(pos, mass, lo, h, n):
    """node masses (n, n, n) [i1, i2, i3] from particles by cloud-in-cell"""
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    mass = np.broadcast_to(np.asarray(mass, np.float64), (pos.shape[0],))
    M = np.zeros((n, n, n))
    u = (pos - np.asarray(lo, np.float64)[None, :]) / h
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    for c1 in (0, 1):
        for c2 in (0, 1):
            for c3 in (0, 1):
                w = ((f[:, 0] if c1 else 1.0 - f[:, 0]) * (f[:, 1] if c2 else 1.0 - f[:, 1])
                     * (f[:, 2] if c3 else 1.0 - f[:, 2]))
                idx = i0 + np.array([c1, c2, c3])[None, :]
                ok = np.all((idx >= 0) & (idx < n), axis=1)
                np.add.at(M, (idx[ok, 0], idx[ok, 1], idx[ok, 2]), mass[ok] * w[ok])
    return M


def kernels(n, h, eps):
    """the four kernels on the zero-padded (2n)^3 grid, indexed by node
    displacement k (k < n: +k, k > n: k - 2n; k = n: unused, zero)"""
    P = 2 * n
    k = np.arange(P)
    d = np.where(k < n, k, k - P).astype(np.float64) * h
    valid = k != n
    dx, dy, dz = np.meshgrid(d, d, d, indexing="ij")
    ok = valid[:, None, None] & valid[None, :, None] & valid[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz + eps * eps
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(ok & (r2 > 0.0), 1.0 / np.sqrt(r2), 0.0)
    inv3 = inv * inv * inv
    m = mu_G()
    return [-m * inv, m * dx * inv3, m * dy * inv3, m * dz * inv3]


def convolve(M, h, eps):
    """phi, grad phi on the nodes: (4, n, n, n)"""
    n = M.shape[0]
    P = 2 * n
    Mp = np.zeros((P, P, P))
    Mp[:n, :n, :n] = M
    FM = np.fft.rfftn(Mp)
    out = np.empty((4, n, n, n))
    for f, K in enumerate(kernels(n, h, eps)):
        out[f] = np.fft.irfftn(FM * np.fft.rfftn(K), s=(P, P, P), axes=(0, 1, 2))[:n, :n, :n]
    return out


def direct_node_sum(M, h, eps):
    """the same node field as a plain double sum (small grids only)"""
    n = M.shape[0]
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    x = idx * h
    m = M.reshape(-1)
    out = np.zeros((4, n ** 3))
    mu = mu_G()
    for i in range(n ** 3):
        d = x[i][None, :] - x
        r2 = np.sum(d * d, axis=1) + eps * eps
        with np.errstate(divide="ignore"):
            inv = np.where(r2 > 0.0, 1.0 / np.sqrt(r2), 0.0)
        out[0, i] = -mu * np.sum(m * inv)
        for c in range(3):
            out[1 + c, i] = mu * np.sum(m * d[:, c] * inv ** 3)
    return out.reshape(4, n, n, n)


def spline_y2(y):
    """natural-spline second derivatives (unit spacing) of a 1-D array"""
    y = np.ascontiguousarray(y, np.float64)
    y2 = np.zeros_like(y)
    lib().orc_spline_y2(y.shape[0], _p(y), 1, _p(y2))
    return y2


class GridField:
    """A particle set on the App. B node grid, ready for the oracle's field
    evaluation and trace (pass ``grid=`` to ``MassField``)."""

    def __init__(self, pos, mass, soft, lo, h, n, n_int=2, mean_subtract=False, val=None, margin=0.0):
        self.n, self.h, self.n_int = int(n), float(h), int(n_int)
        self.lo = np.asarray(lo, np.float64).reshape(3)
        self.eps = float(soft)
        if val is None:
            M = cic(pos, mass, self.lo, self.h, self.n)
            self.M_raw = M
            if mean_subtract:
                M = M - M.mean()
            self.M = M
            val = convolve(M, self.h, self.eps)
        self.val = np.ascontiguousarray(val, np.float64)
        self.y2 = np.zeros_like(self.val)
        lib().orc_grid_y2(self.n, _p(self.val), _p(self.y2))
        self.g = Grid(self.n, (C.c_double * 3)(*self.lo), self.h, self.n_int, _p(self.val), _p(self.y2),
                      float(margin))

    def eval(self, pts):
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 4))
        for i in range(pts.shape[0]):
            lib().orc_grid_eval(C.byref(self.g), _p(pts[i]), _p(out[i]))
        return out

    def pointer(self):
        return C.pointer(self.g)

    def field(self):
        """an oracle MassField whose phi and grad phi come from this grid"""
        from . import MassField
        return MassField(np.zeros((0, 3)), np.zeros(0), 0.0, grid=self)


class BoxGridField:
    """A replicated box on cube grids (Sec. 5.2): the prism of each replica
    around the optical axis, |x1|, |x2| <= W/2 with W = L / cubes, is cut
    along x3 into `cubes` cubes of side W; the particles of each cube (half-
    open in every axis, the others dropped) go on that cube's own n^3 grid
    with nodes on its faces (spacing W / (n - 1)), minus the cube's mean node
    mass, and each cube's field is computed from its own mass only (Sec. 5.2:
    each box contributes its own structure).  A bundle uses the cube holding
    its central ray; points up to one node spacing outside the cube's nodes
    (the bundle's other rays near a face) take the end intervals' cubics."""

    def __init__(self, pos, mass, soft, L, rot, shift, cubes, n, n_int=2, mean_subtract=True):
        from . import MassField, replica_world
        self.L, self.cubes, self.n = float(L), int(cubes), int(n)
        W = self.L / self.cubes
        h = W / (self.n - 1)
        box = MassField(pos, mass, soft, replicated=True, L=L, rot=rot, shift=shift)
        mass = np.broadcast_to(np.asarray(mass, np.float64), (box.pos.shape[0],))
        self.rot, self.shift, self.n_rep = box.rot, box.shift, box.n_rep
        self.grids = []
        for j in range(self.n_rep):
            w = replica_world(box, j)
            for c in range(self.cubes):
                lo = np.array([-0.5 * W, -0.5 * W, j * self.L + c * W])
                inside = np.all((w >= lo) & (w < lo + W), axis=1)
                self.grids.append(GridField(w[inside], mass[inside], soft, lo, h, self.n, n_int=n_int,
                                            mean_subtract=mean_subtract, margin=1.0))
        self.array = (Grid * len(self.grids))(*[gf.g for gf in self.grids])

    def pointer(self):
        return C.cast(self.array, C.POINTER(Grid))

    def field(self):
        from . import MassField
        return MassField(np.zeros((0, 3)), np.zeros(0), 0.0, replicated=True, L=self.L,
                         rot=self.rot, shift=self.shift, grid=self, grid_cubes=self.cubes)

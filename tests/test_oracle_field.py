"""Pins for the oracle's potential (Eqs. psi, derivs, phicotophys as a
Plummer-softened direct sum), the uniform-prism background and the replica
placement (Sec. 5.2)."""
import math

import numpy as np
import pytest
from scipy import integrate

import inputs
import oracle

MU = 4.7854158422368954e-20  # G Msun / c^2 in Mpc, IAU nominal values


def test_single_particle_closed_form():
    p = np.array([[1.0, -2.0, 3.0]])
    f = oracle.MassField(p, [2.5e12], 0.01)
    r = np.array([[1.3, -1.9, 2.2], [1.0, -2.0, 3.0]])
    out = oracle.potential(f, r)
    for i in range(2):
        d = r[i] - p[0]
        q = d @ d + 1e-4
        assert abs(out[i, 0] / (-MU * 2.5e12 / math.sqrt(q)) - 1) < 1e-14
        g = MU * 2.5e12 * d / q ** 1.5
        assert np.allclose(out[i, 1:], g, rtol=1e-14, atol=1e-30)


def test_gradient_is_derivative_of_potential():
    g = inputs.rng(7)
    p = g.normal(size=(50, 3))
    f = oracle.MassField(p, g.uniform(1e10, 1e11, 50), g.uniform(0.05, 0.2, 50))
    r0 = np.array([0.3, -0.2, 0.1])
    h = 1e-5
    pts = [r0]
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        pts += [r0 + e, r0 - e]
    out = oracle.potential(f, np.array(pts))
    for k in range(3):
        fd = (out[1 + 2 * k, 0] - out[2 + 2 * k, 0]) / (2 * h)
        assert abs(fd / out[0, 1 + k] - 1) < 1e-6


def test_superposition():
    g = inputs.rng(8)
    p = g.normal(size=(6, 3))
    m = g.uniform(1, 2, 6) * 1e11
    r = g.normal(size=(5, 3)) * 2
    tot = oracle.potential(oracle.MassField(p, m, 0.1), r)
    parts = sum(oracle.potential(oracle.MassField(p[i:i + 1], m[i:i + 1], 0.1), r) for i in range(6))
    assert np.allclose(tot, parts, rtol=1e-13, atol=0)


def _prism_quad(lo, hi, r):
    f = lambda z, y, x: 1.0 / math.sqrt((x - r[0]) ** 2 + (y - r[1]) ** 2 + (z - r[2]) ** 2)
    v, _ = integrate.tplquad(f, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], epsabs=1e-11, epsrel=1e-11)
    return v


@pytest.mark.parametrize("r", [(3.0, 0.5, -0.7), (0.6, 2.5, 4.0), (-2.0, -1.5, 0.2)])
def test_prism_matches_quadrature_outside(r):
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 1.5])
    out = oracle.prism(lo, hi, np.array(r))
    assert abs(out[0] / _prism_quad(lo, hi, r) - 1) < 1e-9


def test_prism_matches_quadrature_inside():
    # split the box at the field point so the singular point sits on corners
    lo, hi, r = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 1.5]), np.array([0.3, 1.1, 0.4])
    ref = 0.0
    for ax in (0, 1):
        for ay in (0, 1):
            for az in (0, 1):
                l = [lo[0] if ax == 0 else r[0], lo[1] if ay == 0 else r[1], lo[2] if az == 0 else r[2]]
                h = [r[0] if ax == 0 else hi[0], r[1] if ay == 0 else hi[1], r[2] if az == 0 else hi[2]]
                ref += _prism_quad(l, h, r)
    out = oracle.prism(lo, hi, r)
    assert abs(out[0] / ref - 1) < 1e-8


@pytest.mark.parametrize("r", [(0.3, 1.1, 0.4), (3.0, 0.5, -0.7), (0.0, 1.0, 0.75), (1.0, 2.0, 0.3)])
def test_prism_gradient_is_derivative(r):
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 1.5])
    r = np.array(r, float)
    out = oracle.prism(lo, hi, r)
    on_face = np.any(r == lo) or np.any(r == hi)
    # across a face the second derivative jumps (the density does), so the
    # central difference there is only first order: use a smaller step
    h, tol = (1e-7, 1e-6) if on_face else (1e-5, 1e-8)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (oracle.prism(lo, hi, r + e)[0] - oracle.prism(lo, hi, r - e)[0]) / (2 * h)
        assert abs(fd - out[1 + k]) < tol * max(1.0, abs(out[1 + k]))


def test_prism_far_field_is_point_mass():
    lo, hi = np.array([-0.5, -0.5, -0.5]), np.array([0.5, 0.5, 0.5])
    r = np.array([30.0, 20.0, -10.0])
    d = math.sqrt(r @ r)
    out = oracle.prism(lo, hi, r)
    # a cube has no quadrupole: the first correction is O((a/d)^4) ~ 1e-8
    assert abs(out[0] * d - 1) < 1e-7
    assert np.allclose(out[1:], -r / d ** 3, rtol=1e-6)


def test_prism_centre_is_symmetric():
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    out = oracle.prism(lo, hi, np.zeros(3))
    assert np.all(np.abs(out[1:]) < 1e-13)


def _box_field(n_side=12, L=10.0, rep=None, shift=None):
    s = L / n_side
    g = (np.arange(n_side) + 0.5) * s
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n_rep = 3
    rot = np.tile(np.eye(3, dtype=np.int32), (n_rep, 1, 1)) if rep is None else rep
    sh = np.zeros((n_rep, 3)) if shift is None else shift
    return pos, s, rot, sh


def test_replica_placement_identity():
    pos, s, rot, sh = _box_field(4, 8.0)
    f = oracle.MassField(pos, np.full(len(pos), 1e10), 0.0, replicated=True, L=8.0, rot=rot, shift=sh)
    # one particle at a time: the field of replica j at the particle's expected
    # world position equals the softened self-field (phi = -mu m / eps)
    for j in range(3):
        for i in (0, 5, 37):
            fi = oracle.MassField(pos[i:i + 1], [1e10], 0.3, replicated=True, L=8.0, rot=rot, shift=sh)
            w = pos[i] - np.array([4.0, 4.0, 0.0]) + np.array([0, 0, 8.0 * j])
            out = oracle.potential(fi, w[None], np.array([j], np.int32))
            assert abs(out[0, 0] / (-MU * 1e10 / 0.3) - 1) < 1e-14
    assert f.n_rep == 3


def test_replica_rotation_and_shift_exact():
    L = 8.0
    rots, shift = inputs.replicas(4, L, 11)
    p = np.array([[1.25, 7.5, 0.5]])
    for j in range(4):
        fi = oracle.MassField(p, [1e10], 0.2, replicated=True, L=L, rot=rots, shift=shift)
        c = np.full(3, L / 2)
        q = np.mod(rots[j] @ (p[0] - c) + c + shift[j], L)
        w = np.array([q[0] - L / 2, q[1] - L / 2, q[2] + j * L])
        out = oracle.potential(fi, w[None], np.array([j], np.int32))
        assert abs(out[0, 0] / (-MU * 1e10 / 0.2) - 1) < 1e-14
        assert np.all(np.abs(out[0, 1:]) < 1e-30)


def test_mean_subtraction_cancels_uniform_lattice():
    # a softened cubic lattice is close to a uniform prism: the mean-subtracted
    # field deep inside is far smaller than either part
    L, n_side = 10.0, 16
    pos, s, rot, sh = _box_field(n_side, L)
    m = np.full(len(pos), 1e11)
    pts = np.array([[0.13, -0.21, 5.07], [1.9, 0.7, 3.3], [-2.1, 1.4, 6.2]])
    raw = oracle.MassField(pos, m, s, replicated=True, L=L, rot=rot, shift=sh, mean_subtract=False)
    net = oracle.MassField(pos, m, s, replicated=True, L=L, rot=rot, shift=sh, mean_subtract=True)
    a = oracle.potential(raw, pts, np.zeros(3, np.int32))
    b = oracle.potential(net, pts, np.zeros(3, np.int32))
    assert np.all(np.abs(b[:, 1:]) < 0.05 * np.abs(a[:, 1:]).max())
    # softening lowers every particle's potential by a near-constant amount, so
    # compare differences between points rather than values
    assert np.all(np.abs(np.diff(b[:, 0])) < 0.05 * np.abs(np.diff(a[:, 0])))


def test_replica_choice_follows_x3():
    # rep argument selects the replica block; a point in replica 1's volume
    # sees only that replica's copy
    L = 8.0
    pos = np.array([[4.0, 4.0, 4.0]])
    rot = np.tile(np.eye(3, dtype=np.int32), (3, 1, 1))
    f = oracle.MassField(pos, [1e10], 0.1, replicated=True, L=L, rot=rot, shift=np.zeros((3, 3)))
    r = np.array([[0.0, 0.0, 12.0]])
    o1 = oracle.potential(f, r, np.array([1], np.int32))
    o0 = oracle.potential(f, r, np.array([0], np.int32))
    assert abs(o1[0, 0] / (-MU * 1e10 / 0.1) - 1) < 1e-14
    assert abs(o0[0, 0] / (-MU * 1e10 / math.sqrt(64 + 0.01)) - 1) < 1e-14

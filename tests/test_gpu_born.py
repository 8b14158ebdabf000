"""Born approximation on the GPU (FP32 Hessian pair sums, FP64 weights and
prism) against the oracle's FP64 Born integral: a Plummer lens, a small NFW
halo, a replicated mean-subtracted box, empty space, and the errors."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1110_4894_gb300 as P
    return P


def _ctx(P, cosmo=(0.3, 0.7, 0.7)):
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(*cosmo)
    return ctx


def _close(got, want, rel):
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= rel * scale, (np.max(np.abs(got - want)) / scale)


def test_born_plummer_lens(P, cosmo):
    chi_l = cosmo.chi(0.3)
    pos, mass, eps = np.array([[0.0, 0.0, chi_l]]), np.array([1e13]), 0.02
    g = inputs.rng(31)
    th = g.normal(size=(40, 2)) * 3 * eps / chi_l
    kw = dict(schedule=1, n_steps=1500, lens_chi=chi_l, asinh_s=eps)
    want = oracle.born(cosmo, oracle.MassField(pos, mass, eps), 1.0, th, **kw)
    ctx = _ctx(P)
    ctx.load_particles(0, pos, mass, eps)
    got = ctx.born(0, 1.0, th, **kw)
    _close(got, want, 1e-5)


def test_born_nfw_halo(P, cosmo):
    cfg = inputs.config_c2(n_particles=5000, n_side=4, n_steps=300)
    kw = dict(schedule=1, n_steps=cfg["n_steps"], lens_chi=cfg["lens_chi"], asinh_s=cfg["asinh_s"])
    want = oracle.born(cosmo, oracle.MassField(cfg["pos"], cfg["mass"], cfg["soft"]), cfg["z_s"], cfg["theta"], **kw)
    ctx = _ctx(P)
    ctx.load_particles(0, cfg["pos"], cfg["mass"], cfg["soft"])
    got = ctx.born(0, cfg["z_s"], cfg["theta"], **kw)
    _close(got, want, 1e-5)


def test_born_replicated_box(P, cosmo):
    L = inputs.box_length(100.0 / 0.7)
    pos, mass, _ = inputs.halo_box(8000, L, 40, inputs.BASE_SEED + 35)
    rot, shift = inputs.replicas(6, L, inputs.BASE_SEED + 35)
    chi_s = 4.5 * L
    z_s = cosmo.z_of_chi(chi_s)
    g = inputs.rng(77)
    th = g.uniform(-0.4, 0.4, (24, 2)) * L / chi_s  # inside the replicas' transverse extent
    kw = dict(schedule=0, n_steps=120)
    soft = 0.016 / 0.7
    f = oracle.MassField(pos, mass, soft, replicated=True, L=L, rot=rot, shift=shift, mean_subtract=True)
    want = oracle.born(cosmo, f, z_s, th, **kw)
    ctx = _ctx(P)
    ctx.load_particles(0, pos, mass, soft, replicated=True, box_length=L, rot=rot, shift=shift, mean_subtract=True)
    got = ctx.born(0, z_s, th, **kw)
    _close(got, want, 2e-5)


def test_born_empty_and_errors(P):
    ctx = _ctx(P)
    ctx.load_particles(0, np.zeros((0, 3)), np.zeros(0), 0.01)
    assert np.all(ctx.born(0, 0.5, [[1e-3, 0.0]], n_steps=40) == 0.0)
    ctx.load_grid(1, np.zeros((1, 3)), np.ones(1) * 1e10, 0.01, [-1, -1, -1], 0.1, 21)
    with pytest.raises(P.Rt3dError):
        ctx.born(1, 0.5, [[1e-3, 0.0]], n_steps=40)
    with pytest.raises(P.Rt3dError):
        ctx.born(0, -0.5, [[1e-3, 0.0]], n_steps=40)

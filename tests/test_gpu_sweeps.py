"""Minimum-reliable-radius sweeps on the NFW halo (Sec. 4.2, Figs.
nfwtests1-3) as GPU tests: bundles at impact parameters log-spaced over
[0.05, 2] r200 around the NFW workload's halo (M200 = 1e14, c = 5, z_l = 0.25,
z_s = 0.5), one numerical parameter varied at a time, each setting's
magnification compared with the analytic truncated NFW lens (oracle.analytic)
per radial bin.  The assertions are the paper's qualitative findings:

- the particle mass sets the error: coarser particles, larger scatter at
  every radius (Fig. nfwtests3, the shot noise of the discrete halo);
- the RK4 step count (f_RK) does not matter once the lens is resolved
  (500 vs 4000 steps);
- the bundle radius barely matters (0.1" vs 1", Sec. 4.1-4.2);
- a larger softening smooths the shot noise and lowers the error;
- the grid path's accuracy at small radii depends on n_int (Fig. nfwtests1-2).
The minimum reliable radius (MRR) is the smallest bin edge outside which every
bin's mean |mu/mu_analytic - 1| is below 3 % (Sec. 4.2)."""
import math

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

ARCSEC = math.radians(1.0 / 3600.0)
BINS, PER_BIN = 8, 48
EDGES = np.logspace(math.log10(0.05), math.log10(2.0), BINS + 1)


@pytest.fixture(scope="module")
def lens():
    import oracle
    import oracle.analytic as A
    cosmo = oracle.Cosmology(0.3, 0.7, 0.7)
    L = A.NFWLens(cosmo, 1e14, 5.0, 0.25, 0.5)
    g = np.random.default_rng(2024)
    x = np.concatenate([np.exp(g.uniform(math.log(EDGES[i]), math.log(EDGES[i + 1]), PER_BIN)) for i in range(BINS)])
    ph = g.uniform(0, 2 * math.pi, x.size)
    theta = np.stack([x * L.r200 / L.D_d * np.cos(ph), x * L.r200 / L.D_d * np.sin(ph)], 1)
    mu_an = np.array([L.lens_trunc(t)[2] for t in x * L.r200 / L.D_d])
    return theta, mu_an


_halos = {}


def run(lens, n_part=100000, soft=5e-3, theta_r=ARCSEC, n_steps=2000, grid=None):
    import paper_1110_4894_gb300 as P
    theta, mu_an = lens
    if n_part not in _halos:
        _halos[n_part] = inputs.config_c2(n_particles=n_part, n_side=2)
    cfg = _halos[n_part]
    ctx = P.Context(0, precision=P.MIXED)
    ctx.set_cosmology(0.3, 0.7, 0.7)
    if grid is None:
        ctx.load_particles(0, cfg["pos"], cfg["mass"], soft)
    else:
        sp, ni = grid
        half = 2.2 * cfg["info"]["r200_phys"] * (1 + cfg["z_l"])
        hh = sp / 1000.0 / 0.7
        n = int(math.ceil(2 * half / hh)) + 1
        ctx.load_grid(0, cfg["pos"], cfg["mass"], soft, [-half, -half, cfg["chi_l"] - half], hh, n, n_int=ni)
    r = ctx.trace(0, cfg["z_s"], theta, n_ring=4, theta_r=theta_r, schedule=P.SCHED_ASINH, n_steps=n_steps,
                  lens_chi=cfg["chi_l"], asinh_s=max(soft, 1e-3))
    ctx.close()
    err = np.abs(r["mu"] / mu_an - 1)
    per_bin = err.reshape(BINS, PER_BIN).mean(axis=1)
    mrr = 2.0
    for i in range(BINS - 1, -1, -1):
        if per_bin[i] < 0.03:
            mrr = EDGES[i]
        else:
            break
    return per_bin, mrr


def test_particle_mass_sets_the_error(lens):
    e9, _ = run(lens, n_part=int(round(1.5534e14 / 1e9)))
    e10, _ = run(lens, n_part=int(round(1.5534e14 / 1e10)))
    e11, m11 = run(lens, n_part=int(round(1.5534e14 / 1e11)))
    inner = slice(0, 6)
    assert e9[inner].mean() < e10[inner].mean() < e11[inner].mean()
    assert e11[inner].mean() > 3 * e9[inner].mean()
    assert m11 > EDGES[1]  # 1e11 Msun particles lose the inner halo


def test_step_count_does_not_matter(lens):
    e500, m500 = run(lens, n_steps=500)
    e4000, m4000 = run(lens, n_steps=4000)
    assert abs(e500.mean() / e4000.mean() - 1) < 0.10
    assert m500 == m4000


def test_bundle_radius_barely_matters(lens):
    e1, m1 = run(lens, theta_r=ARCSEC)
    e01, m01 = run(lens, theta_r=0.1 * ARCSEC)
    # the smaller bundle samples finer shot noise: its mean error is within
    # 30 % of the 1" bundle's, and the MRR moves by at most one bin
    assert abs(e01.mean() / e1.mean() - 1) < 0.30
    assert abs(np.searchsorted(EDGES, m01) - np.searchsorted(EDGES, m1)) <= 1


def test_softening_lowers_shot_noise(lens):
    e1, _ = run(lens, soft=1e-3)
    e5, _ = run(lens, soft=5e-3)
    e20, _ = run(lens, soft=2e-2)
    assert e20.mean() < e5.mean() < e1.mean()


def test_grid_interpolation_order(lens):
    # on a 49/h kpc grid the App. B interpolation with n_int = 2 is more
    # accurate at small radii than with n_int = 1
    e1, m1 = run(lens, grid=(49.0, 1))
    e2, m2 = run(lens, grid=(49.0, 2))
    assert e2[:3].mean() < e1[:3].mean()
    assert m2 <= m1

"""Seeded generators for the synthetic workloads (point lens, NFW halo,
halo-plus-background boxes, replica transforms, bundle grids, light cones).

Conventions
-----------
* lengths: comoving Mpc; masses: solar masses.
* Every particle coordinate, box length and replica shift is a multiple of
  ``QUANTUM`` = 2^-22 Mpc (0.24 pc).  Such values are exactly representable in
  FP64, so periodic wrapping and replica placement are exact on every side.
* Streams: ``rng(seed, purpose, index)`` = numpy PCG64 seeded through a
  SeedSequence of the three integers; configuration k uses the base seed
  0x5EED0000 + k.

The small amount of background cosmology here (comoving distance, critical
density) only places and sizes the synthetic lenses; it is computed with
scipy quadrature and is not used by either implementation of the method.
"""
import math

import numpy as np
from scipy import integrate

QUANTUM = 2.0 ** -22
BASE_SEED = 0x5EED0000

# placement constants (G Msun / c^2 in Mpc; c in km/s)
_GMSUN, _C, _MPC, _CKMS = 1.32712440018e20, 299792458.0, 3.0856775814913673e22, 299792.458
MU_G_PLACEMENT = _GMSUN / (_C * _C) / _MPC

P_PARTICLES, P_HALO_MASS, P_HALO_CENTRE, P_REPLICA, P_CONE, P_BUNDLES = range(1, 7)

__all__ = [
    "QUANTUM", "BASE_SEED", "rng", "quantize", "chi_placement", "hubble_placement",
    "r200_physical", "point_lens", "nfw_halo", "plummer_particle", "halo_box", "proper_rotations",
    "replicas", "bundle_line", "bundle_grid", "config_c1", "config_c2", "config_c3",
    "config_c4", "config_c5", "config_prism", "box_length", "theta_einstein_placement",
]


def rng(seed, purpose=0, index=0):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(purpose), int(index)])))


def quantize(x):
    return np.round(np.asarray(x, np.float64) / QUANTUM) * QUANTUM


def box_length(L):
    """round a box length to a multiple of 2 QUANTUM (so L/2 is on the grid)"""
    return float(round(L / (2 * QUANTUM)) * 2 * QUANTUM)


def hubble_placement(z, om, ol, h):
    """H(z)/c in 1/Mpc (flat LCDM)"""
    return 100.0 * h / _CKMS * math.sqrt(om * (1 + z) ** 3 + ol)


def chi_placement(z, om, ol, h):
    """comoving distance (Mpc) used to place a lens at redshift z"""
    H0 = 100.0 * h / _CKMS
    v, _ = integrate.quad(lambda x: 1.0 / math.sqrt(om * (1 + x) ** 3 + ol), 0.0, z,
                          epsabs=0, epsrel=1e-13, limit=200)
    return v / H0


def r200_physical(M, z, om, ol, h):
    """radius inside which the mean density is 200 rho_crit(z) (physical Mpc)"""
    Hz = hubble_placement(z, om, ol, h)
    return (MU_G_PLACEMENT * M / (100.0 * Hz * Hz)) ** (1.0 / 3.0)


def theta_einstein_placement(M, z_l, z_s, om, ol, h):
    """point-lens Einstein angle (rad), used to lay out bundles"""
    cl, cs = chi_placement(z_l, om, ol, h), chi_placement(z_s, om, ol, h)
    return math.sqrt(4 * MU_G_PLACEMENT * M * (1 + z_l) * (cs - cl) / (cl * cs))


def point_lens(M, chi_l):
    pos = quantize(np.array([[0.0, 0.0, chi_l]]))
    return pos, np.array([float(M)])


def plummer_particle(M, chi_l, offset=(0.0, 0.0)):
    pos = quantize(np.array([[offset[0], offset[1], chi_l]]))
    return pos, np.array([float(M)])


def _nfw_m(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(g, n, x_t):
    """inverse-CDF radii (units of r_s) of an NFW profile truncated at x_t"""
    u = g.random(n) * _nfw_m(x_t)
    lo, hi = np.zeros(n), np.full(n, float(x_t))
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        below = _nfw_m(mid) < u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def _isotropic(g, n):
    ct = g.uniform(-1.0, 1.0, n)
    ph = g.uniform(0.0, 2.0 * np.pi, n)
    st = np.sqrt(1.0 - ct * ct)
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def nfw_halo(M200, conc, z_l, chi_l, n, seed, om=0.3, ol=0.7, h=0.7, trunc=2.0):
    """Equal-mass particles of an NFW halo (Eq. nfwprof) truncated at trunc*r200,
    centred at (0, 0, chi_l).  Radii by the continuous inverse CDF of the
    enclosed mass; isotropic directions.  Returns (pos, mass, info)."""
    g = rng(seed, P_PARTICLES, 0)
    r200 = r200_physical(M200, z_l, om, ol, h)
    rs = r200 / conc
    x_t = trunc * conc
    x = _nfw_radii(g, n, x_t)
    d = _isotropic(g, n)
    r_co = x * rs * (1.0 + z_l)
    pos = quantize(d * r_co[:, None] + np.array([0.0, 0.0, chi_l]))
    M_t = M200 * _nfw_m(x_t) / _nfw_m(conc)
    mass = np.full(n, M_t / n)
    info = dict(r200_phys=r200, rs_phys=rs, M_trunc=M_t, m_p=M_t / n, chi_l=chi_l, z_l=z_l,
                conc=conc, M200=M200, trunc=trunc)
    return pos, mass, info


def _wrap_grid(q, L):
    """snap to the grid, then wrap into [0, L) (exact: L is on the grid)"""
    q = np.mod(quantize(q), L)
    q[q >= L] -= L
    q[q < 0.0] += L
    return q


def halo_box(N, L, n_halos, seed, om=0.3, ol=0.7, h=0.7, m_min=1e11, m_max=1e15, slope=1.9,
             c0=5.0, c_exp=-0.1, f_bg=0.5, trunc=2.0):
    """Periodic box [0, L)^3 of N equal-mass particles: a fraction f_bg uniform,
    the rest in n_halos NFW halos with dN/dM ~ M^-slope on [m_min, m_max],
    c(M) = c0 (M/1e14)^c_exp, radii to trunc*r200 (z = 0), counts ~ M."""
    g = rng(seed, P_HALO_MASS, 0)
    a = 1.0 - slope
    u = g.random(n_halos)
    M = (m_min ** a + u * (m_max ** a - m_min ** a)) ** (1.0 / a)
    n_bg = int(round(N * f_bg))
    n_h_tot = N - n_bg
    share = M / M.sum() * n_h_tot
    counts = np.floor(share).astype(np.int64)
    rem = n_h_tot - counts.sum()
    if rem > 0:
        order = np.argsort(-(share - counts), kind="stable")
        counts[order[:rem]] += 1
    m_p = M.sum() / max(n_h_tot, 1)
    gc = rng(seed, P_HALO_CENTRE, 0)
    centres = gc.random((n_halos, 3)) * L
    parts = []
    gp = rng(seed, P_PARTICLES, 0)
    for i in range(n_halos):
        k = int(counts[i])
        if k == 0:
            continue
        c = c0 * (M[i] / 1e14) ** c_exp
        r200 = r200_physical(M[i], 0.0, om, ol, h)
        x = _nfw_radii(gp, k, trunc * c)
        parts.append(centres[i] + _isotropic(gp, k) * (x * r200 / c)[:, None])
    parts.append(gp.random((n_bg, 3)) * L)
    pos = _wrap_grid(np.concatenate(parts, axis=0), L)
    mass = np.full(N, m_p)
    info = dict(halo_mass=M, halo_counts=counts, m_p=m_p, n_bg=n_bg, L=L)
    return pos, mass, info


def proper_rotations():
    """the 24 proper rotations of the cube as signed permutation matrices"""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), np.int32)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return np.array(out)


def replicas(n_rep, L, seed):
    """random 90-degree rotation and periodic shift per replica (Sec. 5.2)"""
    g = rng(seed, P_REPLICA, 0)
    rots = proper_rotations()
    idx = g.integers(0, len(rots), n_rep)
    shift = _wrap_grid(g.random((n_rep, 3)) * L, L)
    return rots[idx].astype(np.int32), shift


def bundle_line(theta_lo, theta_hi, n):
    """bundle centres along the theta_x axis"""
    t = np.linspace(theta_lo, theta_hi, n)
    return np.stack([t, np.zeros(n)], axis=1)


def bundle_grid(lo, hi, n_side, tile=8):
    """n_side x n_side grid on [lo, hi]^2, ordered tile by tile so that
    consecutive bundles are neighbours on the sky"""
    t = np.linspace(lo, hi, n_side)
    ii, jj = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    ti, tj = ii // tile, jj // tile
    key = (ti * ((n_side + tile - 1) // tile) + tj) * tile * tile + (ii % tile) * tile + (jj % tile)
    order = np.argsort(key.ravel(), kind="stable")
    th = np.stack([t[ii.ravel()], t[jj.ravel()]], axis=1)
    return np.ascontiguousarray(th[order])


# ---------------------------------------------------------------------------
# the five workloads (cosmology 0.3 / 0.7 / 0.7)
# ---------------------------------------------------------------------------
COSMO = (0.3, 0.7, 0.7)


def config_c1(n_bundles=64, x_lo=0.5, x_hi=5.0, n_steps=1000, extra_images=True):
    """Single point lens M = 1e12 at z_l = 0.25, z_s = 0.5, bundles of a central
    ray + 4 at 1e-3 Einstein radii, centres along theta_x at x = theta/theta_E."""
    om, ol, h = COSMO
    M, zl, zs = 1e12, 0.25, 0.5
    chi_l = chi_placement(zl, om, ol, h)
    pos, mass = point_lens(M, chi_l)
    thE = theta_einstein_placement(M, zl, zs, om, ol, h)
    x = np.linspace(x_lo, x_hi, n_bundles)
    if extra_images:
        x = np.concatenate([x, [2.0, -0.5]])
    theta = np.stack([x * thE, np.zeros_like(x)], axis=1)
    return dict(name="c1_point_lens", cosmo=COSMO, z_s=zs, pos=pos, mass=mass, soft=0.0,
                theta=theta, x=x, theta_E=thE, n_ring=4, theta_r=1e-3 * thE, schedule=1,
                n_steps=n_steps, lens_chi=float(pos[0, 2]), asinh_s=max(0.0, 0.2 * thE * chi_l),
                M=M, z_l=zl, chi_l=chi_l, precision="fp64", replicated=False)


def config_c2(n_particles=100000, n_side=64, n_steps=2000, seed=BASE_SEED + 2):
    """NFW halo M200 = 1e14, c = 5, z_l = 0.25, n equal-mass particles to
    2 r200, Plummer softening 5 kpc (comoving); bundles on an n_side^2 grid
    of impact parameters in [0.05, 2] r200 (first quadrant)."""
    om, ol, h = COSMO
    zl, zs = 0.25, 0.5
    chi_l = chi_placement(zl, om, ol, h)
    pos, mass, info = nfw_halo(1e14, 5.0, zl, chi_l, n_particles, seed, om, ol, h)
    D_d = chi_l / (1 + zl)
    r200 = info["r200_phys"]
    lo, hi = 0.05 * r200 / D_d / math.sqrt(2), 2.0 * r200 / D_d / math.sqrt(2)
    theta = bundle_grid(lo, hi, n_side)
    eps = 5e-3
    return dict(name="c2_nfw", cosmo=COSMO, z_s=zs, pos=pos, mass=mass, soft=eps, theta=theta,
                n_ring=4, theta_r=math.radians(1.0 / 3600.0), schedule=1, n_steps=n_steps,
                lens_chi=chi_l, asinh_s=eps, info=info, chi_l=chi_l, z_l=zl,
                precision="mixed", replicated=False)


def _box_config(name, N, L_h, n_halos, zs, n_side, fov_deg, n_steps, seed, eps_h=0.016):
    om, ol, h = COSMO
    L = box_length(L_h / h)
    pos, mass, info = halo_box(N, L, n_halos, seed, om, ol, h)
    chi_s = chi_placement(zs, om, ol, h)
    n_rep = int(math.ceil(chi_s / L)) + 1
    rot, shift = replicas(n_rep, L, seed)
    half = math.radians(fov_deg)
    theta = bundle_grid(-half, half, n_side)
    return dict(name=name, cosmo=COSMO, z_s=zs, pos=pos, mass=mass, soft=eps_h / h, theta=theta,
                n_ring=4, theta_r=math.radians(1.0 / 3600.0), schedule=0, n_steps=n_steps,
                lens_chi=0.0, asinh_s=1.0, L=L, rot=rot, shift=shift, n_rep=n_rep, info=info,
                precision="mixed", replicated=True, mean_subtract=True)


def config_c3(N=2097152, n_side=256, n_steps=1000, n_halos=3000, seed=BASE_SEED + 3):
    """2^21 particles in a periodic 100/h Mpc box (3000 NFW halos + 50% uniform),
    replicated to z_s = 0.5 with random rotations/shifts; n_side^2 bundles in a
    +-1.95 degree field."""
    return _box_config("c3_box", N, 100.0, n_halos, 0.5, n_side, 1.95, n_steps, seed)


def config_c5(N=16777216, n_side=1024, n_steps=1000, n_halos=24000, seed=BASE_SEED + 5):
    """2^24 particles in a 200/h Mpc box, z_s = 1.0, n_side^2 bundles, +-2.3 deg."""
    return _box_config("c5_box", N, 200.0, n_halos, 1.0, n_side, 2.3, n_steps, seed)


def config_prism(N=16777216, n_side=176, n_steps=1000, n_halos=24000, cubes=8, grid_n=128, seed=BASE_SEED + 6):
    """The sampling region of Sec. 5.2: 256^3 particles in a periodic 50/h Mpc
    box, replicated to z_s = 0.5 (28 replicas), each replica's prism 6.25/h
    Mpc across cut into 8 cubes with 128^3-node grids; n_side^2 bundles on a
    grid inside 0.9 of the prism's half-width at the source plane."""
    om, ol, h = COSMO
    zs = 0.5
    L = box_length(50.0 / h)
    pos, mass, info = halo_box(N, L, n_halos, seed, om, ol, h)
    chi_s = chi_placement(zs, om, ol, h)
    n_rep = int(math.ceil(chi_s / L)) + 1
    rot, shift = replicas(n_rep, L, seed)
    half = 0.9 * 0.5 * (L / cubes) / chi_s
    theta = bundle_grid(-half, half, n_side)
    return dict(name="prism_box", cosmo=COSMO, z_s=zs, pos=pos, mass=mass, soft=0.016 / h, theta=theta,
                n_ring=4, theta_r=math.radians(1.0 / 3600.0), schedule=0, n_steps=n_steps,
                lens_chi=0.0, asinh_s=1.0, L=L, rot=rot, shift=shift, n_rep=n_rep, info=info, cubes=cubes,
                grid_n=grid_n, precision="mixed", replicated=True, mean_subtract=True)


def _cone(i, Nc, zs, nb, seed, n_steps, L, margin_h):
    """one light cone of config_c4 (its own seeded halo box and bundle grid)"""
    om, ol, h = COSMO
    n_halos = max(1, int(round(3000 * Nc / 2 ** 21)))
    pos, mass, info = halo_box(Nc, L, n_halos, seed * 1000 + i, om, ol, h)
    chi_s = chi_placement(zs, om, ol, h)
    n_rep = int(math.ceil(chi_s / L)) + 1
    rot, shift = replicas(n_rep, L, seed * 1000 + i)
    half = (0.5 * L - margin_h / h) / chi_s
    side = int(math.ceil(math.sqrt(nb)))
    theta = bundle_grid(-half, half, side)[:nb]
    return dict(pos=pos, mass=mass, soft=0.016 / h, z_s=zs, theta=theta, L=L, rot=rot,
                shift=shift, n_rep=n_rep, n_steps=n_steps, info=info)


def config_c4(n_cones=512, n_steps=1000, seed=BASE_SEED + 4, n_min=1000, n_max=1000000,
              b_min=256, b_max=4096, zs_lo=0.3, zs_hi=1.5, L_h=50.0, margin_h=5.0, workers=1):
    """Independent light cones: per cone a halo box with N_c log-uniform in
    [n_min, n_max], z_s uniform in [zs_lo, zs_hi], bundles log-uniform in
    [b_min, b_max] on a square grid inside the replica margin.  workers > 1
    draws the cones in that many spawned processes (same cones: each has its
    own seeds)."""
    om, ol, h = COSMO
    g = rng(seed, P_CONE, 0)
    L = box_length(L_h / h)
    draws = []
    for i in range(n_cones):
        Nc = int(round(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
        zs = float(g.uniform(zs_lo, zs_hi))
        nb = int(round(math.exp(g.uniform(math.log(b_min), math.log(b_max)))))
        draws.append((i, Nc, zs, nb, seed, n_steps, L, margin_h))
    if workers > 1 and n_cones > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            cones = list(ex.map(_cone, *zip(*draws), chunksize=4))
    else:
        cones = [_cone(*d) for d in draws]
    return dict(name="c4_cones", cosmo=COSMO, cones=cones, n_ring=4,
                theta_r=math.radians(1.0 / 3600.0), schedule=0, precision="mixed")

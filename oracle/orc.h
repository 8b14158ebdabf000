/*
 * orc.h -- plain FP64 CPU oracle for 3D ray-bundle tracing through a particle
 * mass distribution (Killedar, Lasky, Lewis & Fluke 2011, "Gravitational
 * Lensing with Three-Dimensional Ray Tracing").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the reference against which the
 * CUDA path is checked.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Units: comoving lengths in Mpc, time in Mpc (c = 1), masses in solar
 * masses.  G/c^2 is folded into ORC_MU_G (Mpc per solar mass).
 *
 * Every routine is a direct transcription of the paper's definitions, in
 * FP64, with naive loops and Neumaier-compensated sums; nothing is blocked,
 * fused or reordered beyond what the definition states.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- cosmology (Sec. 3.5, Sec. 5.1, App. E) ---------------------------- */
typedef struct {
    double omega_m; /* Omega_M,0 */
    double omega_l; /* Omega_Lambda,0 ; flat: omega_m + omega_l = 1 */
    double h;       /* H0 = 100 h km/s/Mpc */
} orc_cosmo;

double orc_mu_G(void);                              /* G Msun / c^2 in Mpc */
double orc_H0(const orc_cosmo *c);                  /* H0 / c in 1/Mpc */
double orc_E(const orc_cosmo *c, double z);         /* H(z)/H0 */
double orc_chi(const orc_cosmo *c, double z);       /* Eq. raytracedistance */
double orc_z_of_chi(const orc_cosmo *c, double chi);
double orc_t0(const orc_cosmo *c);                  /* Eq. lookbacksingularity (a(0)=1 reading) */
double orc_a_of_t(const orc_cosmo *c, double t);    /* Eq. scalefac2, t = lookback time */
double orc_adot_of_t(const orc_cosmo *c, double t); /* da/dt, t = lookback time */
double orc_D_fb(const orc_cosmo *c, double z);      /* Eq. angularDD12 */
double orc_D_eb(const orc_cosmo *c, double z);      /* Eq. DRempty */

/* step schedule (Eq. RKstepsize with the resolution length replaced by a
 * node table).  kind 0: uniform nodes in x3; kind 1: lens-centred asinh
 * nodes x3_k = chi_l + s sinh(u_k).  dlam[k] = int_{x3_k}^{x3_{k+1}} a^2 dchi
 * along the unperturbed ray.  nodes may be NULL. */
int orc_schedule(const orc_cosmo *c, double chi_s, int kind, int n_steps,
                 double chi_l, double s, double *dlam, double *nodes);

/* ---- mass distribution (Sec. 3.3, Sec. 5.2) ---------------------------- */
typedef struct {
    int64_t n;
    const double *pos;    /* n*3 comoving Mpc.  isolated: world frame;
                             replicated: box frame [0,L)^3 */
    const double *mass;   /* n, Msun */
    const double *soft;   /* n Plummer softening lengths (comoving Mpc), or NULL */
    double soft_scalar;   /* used when soft == NULL */
    int replicated;       /* 0 isolated field, 1 box replicated along x3 */
    double L;             /* box length (replicated only) */
    int n_rep;            /* number of replicas along the line of sight */
    const int32_t *rot;   /* n_rep * 9 row-major signed permutation matrices */
    const double *shift;  /* n_rep * 3 shifts in [0, L) */
    int mean_subtract;    /* subtract the field of the replica's uniform mean */
    const struct orc_grid *grid; /* non-NULL: phi and grad phi come from this
                                    gridded field; for replicated fields an array
                                    of n_rep * grid_cubes cube grids (below) */
    int grid_cubes;      /* replicated grid fields: cubes of side L / grid_cubes
                            along x3 per replica (Sec. 5.2: the prism of each box
                            split into cubes, each on its own grid) */
} orc_field;

/* ---- gridded field (Sec. 3.3 grid path, App. B interpolation) ---------- */
/* phi and grad phi on the nodes x = lo + h (i1, i2, i3), i = 0..n-1, stored
 * [f][i1][i2][i3] with f = (phi, dphi/dx1, dphi/dx2, dphi/dx3) and i3
 * fastest; y2 holds the natural-spline second derivatives of every line
 * along x3 in index units (App. B: computed once per mass distribution). */
typedef struct orc_grid {
    int n;
    double lo[3];
    double h;
    int n_int;          /* App. B: n_int nodes on either side per dimension */
    const double *val;  /* 4 n^3 */
    const double *y2;   /* 4 n^3 */
    double margin;      /* points up to margin node spacings outside the node
                           range take the end intervals' cubics (box cubes: 1,
                           so the rays of a bundle near a cube face keep their
                           field); farther out the field is zero */
} orc_grid;

/* second derivatives of the natural cubic spline through y[0..n-1] (unit
 * spacing, y'' = 0 at both ends); y and y2 strided by `stride` */
void orc_spline_y2(int n, const double *y, int64_t stride, double *y2);

/* y2 of every x3 line of val (4 n^3) */
void orc_grid_y2(int n, const double *val, double *y2);

/* App. B evaluation at r: out = (phi, grad phi); zero outside the node range */
void orc_grid_eval(const orc_grid *g, const double r[3], double out[4]);

/* world positions (n*3) of replica j of a replicated field (the transform the
 * direct sum uses): rotation about the box centre, periodic shift, the box
 * centred on the optical axis at x3 in [jL, (j+1)L) */
void orc_replica_world(const orc_field *f, int j, double *out);

/* phi and grad phi (Eqs. psi, derivs, phicotophys, as a Plummer-softened
 * direct sum) at n points; rep[i] selects the replica for point i (ignored
 * for isolated fields).  out: n*4 = (phi, dphi/dx1, dphi/dx2, dphi/dx3). */
int orc_potential(const orc_field *f, int64_t n, const double *pts,
                  const int32_t *rep, double *out, int nthreads);

/* Newtonian-form integral of a uniform rectangular prism:
 * I = int dV / |r - r'| over [lo, hi] and its gradient with respect to r.
 * out = (I, dI/dx1, dI/dx2, dI/dx3). */
void orc_prism(const double lo[3], const double hi[3], const double r[3], double out[4]);

/* second derivatives of the same integral: out = (xx, xy, xz, yy, yz, zz) */
void orc_prism_hessian(const double lo[3], const double hi[3], const double r[3], double out[6]);

/* ---- geodesic right-hand side (Eq. geodesiceqn, App. A) ---------------- */
/* y = (t, x1, x2, x3, dt/dl, dx1/dl, dx2/dl, dx3/dl); F = (phi, grad phi).
 * christoffel 0: App. A as printed; 1: Gamma^t_ij derived from the metric. */
void orc_geodesic_rhs(const orc_cosmo *c, const double y[8], const double F[4],
                      int christoffel, double dy[8]);

/* ---- full trace (Secs. 3.1, 3.4, 5.3) ---------------------------------- */
typedef struct {
    int n_ring;         /* rays on the bundle polygon (paper: 8; default 4) */
    double theta_r;     /* polygon radius, rad */
    double phase;       /* polygon orientation, rad */
    int schedule;       /* 0 uniform, 1 asinh */
    int n_steps;
    double lens_chi;    /* asinh centre */
    double asinh_s;     /* asinh scale */
    int max_extra;      /* extra steps of the last size after the table ends */
    int christoffel;    /* 0 paper App. A, 1 derived */
} orc_trace_opts;

enum { ORC_F_NOCROSS = 1, ORC_F_NONFINITE = 2, ORC_F_NEGPARITY = 4 };

/* ray_out: n_b*(1+n_ring)*8 final states at x3 = chi_s.
 * bundle_out: n_b*6 = (mu, kappa, gamma1, gamma2, omega, flags).
 * steps_out (optional): n_b*(1+n_ring) steps taken until the crossing.
 * Returns the number of (ray, particle) pair evaluations in *n_pairs. */
int orc_trace(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b,
              const double *theta, const orc_trace_opts *o, double *ray_out,
              double *bundle_out, int32_t *steps_out, double *n_pairs, int nthreads);

/* Jacobian of one bundle from its final states (Eqs. lensmap, magnification). */
void orc_bundle_jacobian(int n_ring, const double *theta0, const double *dtheta,
                         const double *xy_final, double chi_s, double out[6]);

/* ---- mu PDF (Eq. weighthisto) ------------------------------------------ */
typedef struct {
    int bins;
    double mu_min, mu_max;
} orc_hist_opts;

/* counts[bins], wfix[bins] = sum of round(2^32/|mu|) per bin,
 * scalars: (n_used, n_under, n_over, n_neg, n_bad, W_total, mean_w, sigma_w). */
int orc_histogram(int64_t n, const double *mu, const int32_t *flags,
                  const orc_hist_opts *o, uint64_t *counts, uint64_t *wfix,
                  double *scalars);

/* Born approximation (Sec. 6): kappa, gamma1, gamma2 of n_b lines of sight
 * theta (n_b*2) from the Hessian of psi along the unperturbed rays, over the
 * node table of o (schedule, n_steps, lens_chi, asinh_s); out = n_b*3. */
int orc_born(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b, const double *theta,
             const orc_trace_opts *o, double *out, int nthreads);

/* shear PDF (Sec. 5.4, Fig. RBMvsMudShear): as orc_histogram, but bins are
 * uniform in log10|gamma|, |gamma| = sqrt(gamma1^2 + gamma2^2), over
 * [o->mu_min, o->mu_max] read as the |gamma| range; each bundle still
 * carries the source-plane weight 1/|mu|; the moments are those of |gamma|
 * under that weight.  |gamma| = 0 counts as underflow. */
int orc_shear_histogram(int64_t n, const double *mu, const double *g1, const double *g2,
                        const int32_t *flags, const orc_hist_opts *o, uint64_t *counts,
                        uint64_t *wfix, double *scalars);

/* ---- multiple lens-plane comparison system (Sec. 3.1; Eqs. defangleB, lenseqn) */
typedef struct {
    int n_ring;         /* rays on the bundle polygon */
    double theta_r;     /* polygon radius, rad */
    double phase;       /* polygon orientation, rad */
    int slices;         /* slabs (planes) per replica, or per isolated field */
} orc_mp_opts;

/* deflection integral of a uniform unit surface density over the rectangle
 * [lo, hi]: out = int (x - x') / |x - x'|^2 d^2x' */
void orc_rect_deflection(const double lo[2], const double hi[2], const double x[2], double out[2]);

/* Bundles traced through the lens planes of f (see orc.c for the readings).
 * ray_out (optional): n_b*(1+n_ring)*2 comoving source-plane positions;
 * bundle_out: n_b*6 (mu, kappa, gamma1, gamma2, omega, flags);
 * planes_out (optional, room for n_rep*slices or slices planes): per plane
 * (chi, z, particles, slab thickness); *n_planes: planes used;
 * *n_pairs: (ray, particle) deflection terms. */
int orc_multiplane(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b, const double *theta,
                   const orc_mp_opts *o, double *ray_out, double *bundle_out, double *planes_out,
                   int *n_planes, double *n_pairs, int nthreads);

#ifdef __cplusplus
}
#endif
#endif

/*
 * orc.c -- plain FP64 CPU oracle (test infrastructure; see orc.h).
 *
 * Each function cites the passage of Killedar et al. (2011) it follows.
 * Readings where the paper is silent or garbled are marked READING and are
 * listed in the design notes of the repository.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* constants: IAU nominal G Msun, SI c, IAU parsec-based Mpc                 */
/* ------------------------------------------------------------------------ */
static const double GM_SUN_SI = 1.32712440018e20;   /* m^3 s^-2 */
static const double C_SI = 299792458.0;             /* m s^-1 */
static const double MPC_SI = 3.0856775814913673e22; /* m */
static const double C_KMS = 299792.458;             /* km s^-1 */

double orc_mu_G(void) { return GM_SUN_SI / (C_SI * C_SI) / MPC_SI; }
double orc_H0(const orc_cosmo *c) { return 100.0 * c->h / C_KMS; }

/* H(z)/H0 for a flat, radiation-free Lemaitre model (Sec. 3.5). */
double orc_E(const orc_cosmo *c, double z)
{
    double zp = 1.0 + z;
    return sqrt(c->omega_m * zp * zp * zp + c->omega_l);
}

/* ------------------------------------------------------------------------ */
/* composite 8-point Gauss-Legendre quadrature (library-grade primitive)    */
/* ------------------------------------------------------------------------ */
static const double GLX[4] = {0.1834346424956498, 0.5255324099163290,
                              0.7966664774136267, 0.9602898564975363};
static const double GLW[4] = {0.3626837833783620, 0.3137066458778873,
                              0.2223810344533745, 0.1012285362903763};

typedef double (*orc_fn)(const void *ctx, double x);

static double gl8(orc_fn f, const void *ctx, double a, double b, int panels)
{
    double h = (b - a) / panels, s = 0.0;
    for (int p = 0; p < panels; ++p) {
        double m = a + (p + 0.5) * h, r = 0.5 * h, ps = 0.0;
        for (int i = 0; i < 4; ++i)
            ps += GLW[i] * (f(ctx, m - r * GLX[i]) + f(ctx, m + r * GLX[i]));
        s += ps * r;
    }
    return s;
}

static double inv_E(const void *ctx, double z) { return 1.0 / orc_E((const orc_cosmo *)ctx, z); }
static double inv_E_zp2(const void *ctx, double z)
{
    double zp = 1.0 + z;
    return 1.0 / (zp * zp * orc_E((const orc_cosmo *)ctx, z));
}
static int panels_for(double z) { int p = (int)ceil(fabs(z) / 0.05); return p < 1 ? 1 : p; }

/* Eq. raytracedistance: D_C = c int_0^z dz / H(z). */
double orc_chi(const orc_cosmo *c, double z)
{
    if (z == 0.0) return 0.0;
    return gl8(inv_E, c, 0.0, z, panels_for(z)) / orc_H0(c);
}

/* inverse of orc_chi by Newton-Raphson, d chi/dz = 1/(H0 E). */
double orc_z_of_chi(const orc_cosmo *c, double chi)
{
    if (chi == 0.0) return 0.0;
    double H0 = orc_H0(c), z = chi * H0;
    for (int it = 0; it < 60; ++it) {
        double dz = (orc_chi(c, z) - chi) * H0 * orc_E(c, z);
        z -= dz;
        if (fabs(dz) <= 1e-16 * (1.0 + fabs(z))) break;
    }
    return z;
}

/* Eq. lookbacksingularity.  READING: the printed argument of sinh^-1 is
 * Omega_L/Omega_M, which gives a(0) != 1; the square root of that ratio
 * makes a(0) = 1 as Eq. scalefac defines, and is used here. */
double orc_t0(const orc_cosmo *c)
{
    return 2.0 / (3.0 * orc_H0(c) * sqrt(c->omega_l)) * asinh(sqrt(c->omega_l / c->omega_m));
}

/* Eq. scalefac2 with t the lookback time. */
double orc_a_of_t(const orc_cosmo *c, double t)
{
    double s = sinh(1.5 * sqrt(c->omega_l) * orc_H0(c) * (orc_t0(c) - t));
    return cbrt(c->omega_m / c->omega_l * s * s);
}

/* d a / d t for t the lookback time: the derivative of Eq. scalefac2,
 * written as -a H(a) (the Friedmann equation of the same model). */
double orc_adot_of_t(const orc_cosmo *c, double t)
{
    double a = orc_a_of_t(c, t);
    return -a * orc_H0(c) * sqrt(c->omega_m / (a * a * a) + c->omega_l);
}

/* Eq. angularDD12 (full beam = FLRW angular diameter distance). */
double orc_D_fb(const orc_cosmo *c, double z) { return orc_chi(c, z) / (1.0 + z); }

/* Eq. DRempty (empty beam, Dyer-Roeder alpha = 0). */
double orc_D_eb(const orc_cosmo *c, double z)
{
    if (z == 0.0) return 0.0;
    return gl8(inv_E_zp2, c, 0.0, z, panels_for(z)) / orc_H0(c);
}

/* ------------------------------------------------------------------------ */
/* step schedule (Eq. RKstepsize; READING: node table instead of grid size) */
/* ------------------------------------------------------------------------ */
typedef struct { const orc_cosmo *c; } a2_ctx;
static double a2_of_chi(const void *ctx, double chi)
{
    const orc_cosmo *c = ((const a2_ctx *)ctx)->c;
    double a = 1.0 / (1.0 + orc_z_of_chi(c, chi));
    return a * a;
}

int orc_schedule(const orc_cosmo *c, double chi_s, int kind, int n, double chi_l,
                 double s, double *dlam, double *nodes)
{
    if (n < 1 || !(chi_s > 0.0)) return -1;
    if (kind == 1 && !(s > 0.0)) return -1;
    double *x = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!x) return -2;
    if (kind == 0) {
        for (int k = 0; k <= n; ++k) x[k] = chi_s * (double)k / (double)n;
    } else {
        double u0 = asinh((0.0 - chi_l) / s), u1 = asinh((chi_s - chi_l) / s);
        for (int k = 0; k <= n; ++k) x[k] = chi_l + s * sinh(u0 + (u1 - u0) * (double)k / (double)n);
    }
    x[0] = 0.0;
    x[n] = chi_s;
    a2_ctx ctx = {c};
    /* unperturbed ray with dx3/dlambda = 1 at the observer: dlambda = a^2 dx3 */
    for (int k = 0; k < n; ++k) dlam[k] = gl8(a2_of_chi, &ctx, x[k], x[k + 1], 1);
    if (nodes) memcpy(nodes, x, sizeof(double) * (size_t)(n + 1));
    free(x);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Neumaier compensated summation                                           */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nval(nsum a) { return a.s + a.c; }

/* ------------------------------------------------------------------------ */
/* uniform prism: I(r) = int dV / |r - r'|  (Newtonian potential integral)   */
/* F is an antiderivative with d^3F/dx dy dz = 1/r; Hx = dF/dx.             */
/* ------------------------------------------------------------------------ */
/* log(a + r) where b2 = r^2 - a^2 > 0; the second form avoids cancellation */
static double log_a_plus_r(double a, double r, double b2)
{
    return a >= 0.0 ? log(a + r) : log(b2 / (r - a));
}

static double prism_F(double x, double y, double z)
{
    double x2 = x * x, y2 = y * y, z2 = z * z, r = sqrt(x2 + y2 + z2);
    double v = 0.0;
    if (x != 0.0 && y != 0.0) v += x * y * log_a_plus_r(z, r, x2 + y2);
    if (y != 0.0 && z != 0.0) v += y * z * log_a_plus_r(x, r, y2 + z2);
    if (z != 0.0 && x != 0.0) v += z * x * log_a_plus_r(y, r, z2 + x2);
    if (x != 0.0) v -= 0.5 * x2 * atan(y * z / (x * r));
    if (y != 0.0) v -= 0.5 * y2 * atan(z * x / (y * r));
    if (z != 0.0) v -= 0.5 * z2 * atan(x * y / (z * r));
    return v;
}

/* dF/dx (first argument); the other two follow by cyclic permutation */
static double prism_H(double x, double y, double z)
{
    double x2 = x * x, y2 = y * y, z2 = z * z, r = sqrt(x2 + y2 + z2);
    double v = 0.0;
    if (y != 0.0) v += y * log_a_plus_r(z, r, x2 + y2);
    if (z != 0.0) v += z * log_a_plus_r(y, r, x2 + z2);
    if (x != 0.0) v -= x * atan(y * z / (x * r));
    return v;
}

void orc_prism(const double lo[3], const double hi[3], const double r[3], double out[4])
{
    double X[2] = {lo[0] - r[0], hi[0] - r[0]};
    double Y[2] = {lo[1] - r[1], hi[1] - r[1]};
    double Z[2] = {lo[2] - r[2], hi[2] - r[2]};
    double I = 0, gx = 0, gy = 0, gz = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
                /* sign = s_a s_b s_d with s = +1 at the upper limit, -1 at the lower */
                double sgn = (a ? 1.0 : -1.0) * (b ? 1.0 : -1.0) * (d ? 1.0 : -1.0);
                I += sgn * prism_F(X[a], Y[b], Z[d]);
                /* X = corner - r, so d/dr = -d/dX */
                gx -= sgn * prism_H(X[a], Y[b], Z[d]);
                gy -= sgn * prism_H(Y[b], Z[d], X[a]);
                gz -= sgn * prism_H(Z[d], X[a], Y[b]);
            }
    out[0] = I;
    out[1] = gx;
    out[2] = gy;
    out[3] = gz;
}

/* second derivatives of the prism integral: the corner function has
 * d2F/dx2 = -atan(yz/(x r)) and d2F/dxdy = log(z + r) (cyclic); with X =
 * corner - r the sign of d2/dr2 is that of d2/dX2.  out = (xx, xy, xz, yy,
 * yz, zz). */
void orc_prism_hessian(const double lo[3], const double hi[3], const double r[3], double out[6])
{
    double X[2] = {lo[0] - r[0], hi[0] - r[0]};
    double Y[2] = {lo[1] - r[1], hi[1] - r[1]};
    double Z[2] = {lo[2] - r[2], hi[2] - r[2]};
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
                double sgn = (a ? 1.0 : -1.0) * (b ? 1.0 : -1.0) * (d ? 1.0 : -1.0);
                double x = X[a], y = Y[b], z = Z[d];
                double x2 = x * x, y2 = y * y, z2 = z * z, rr = sqrt(x2 + y2 + z2);
                double txx = x != 0.0 ? -atan(y * z / (x * rr)) : 0.0;
                double tyy = y != 0.0 ? -atan(z * x / (y * rr)) : 0.0;
                double tzz = z != 0.0 ? -atan(x * y / (z * rr)) : 0.0;
                out[0] += sgn * txx;
                out[1] += sgn * log_a_plus_r(z, rr, x2 + y2);
                out[2] += sgn * log_a_plus_r(y, rr, x2 + z2);
                out[3] += sgn * tyy;
                out[4] += sgn * log_a_plus_r(x, rr, y2 + z2);
                out[5] += sgn * tzz;
            }
}

/* ------------------------------------------------------------------------ */
/* mass distribution: world positions of a replica (Sec. 5.2)               */
/* READING: replica j is the box rotated about its centre by a proper 90-   */
/* degree rotation, shifted periodically, centred transversely on the       */
/* optical axis and placed at x3 in [jL, (j+1)L).                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int nrep;          /* replicas held (1 for isolated fields) */
    double **w;        /* nrep arrays of n*3 world positions */
    double *m;         /* n */
    double *eps2;      /* n */
    double rho_bar;    /* particle mean density of the box (Msun/Mpc^3) */
} prep_field;

static void replica_world(const orc_field *f, int j, double *w)
{
    double L = f->L, c = 0.5 * L;
    const int32_t *R = f->rot + 9 * j;
    const double *s = f->shift + 3 * j;
    for (int64_t i = 0; i < f->n; ++i) {
        const double *p = f->pos + 3 * i;
        double q[3];
        for (int r = 0; r < 3; ++r) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += (double)R[3 * r + k] * (p[k] - c);
            v = v + c + s[r];
            while (v >= L) v -= L;
            while (v < 0.0) v += L;
            q[r] = v;
        }
        w[3 * i + 0] = q[0] - c;
        w[3 * i + 1] = q[1] - c;
        w[3 * i + 2] = q[2] + (double)j * L;
    }
}

static int prep_make(const orc_field *f, prep_field *pf)
{
    memset(pf, 0, sizeof(*pf));
    pf->n = f->n;
    pf->nrep = f->replicated ? f->n_rep : 1;
    pf->w = (double **)calloc((size_t)pf->nrep, sizeof(double *));
    pf->m = (double *)malloc(sizeof(double) * (size_t)(f->n > 0 ? f->n : 1));
    pf->eps2 = (double *)malloc(sizeof(double) * (size_t)(f->n > 0 ? f->n : 1));
    if (!pf->w || !pf->m || !pf->eps2) return -2;
    nsum mt = {0, 0};
    for (int64_t i = 0; i < f->n; ++i) {
        double e = f->soft ? f->soft[i] : f->soft_scalar;
        pf->m[i] = f->mass[i];
        pf->eps2[i] = e * e;
        nadd(&mt, f->mass[i]);
    }
    if (f->replicated) pf->rho_bar = nval(mt) / (f->L * f->L * f->L);
    for (int j = 0; j < pf->nrep; ++j) {
        pf->w[j] = (double *)malloc(sizeof(double) * 3 * (size_t)(f->n > 0 ? f->n : 1));
        if (!pf->w[j]) return -2;
        if (f->replicated) replica_world(f, j, pf->w[j]);
        else memcpy(pf->w[j], f->pos, sizeof(double) * 3 * (size_t)f->n);
    }
    return 0;
}

static void prep_free(prep_field *pf)
{
    if (pf->w)
        for (int j = 0; j < pf->nrep; ++j) free(pf->w[j]);
    free(pf->w);
    free(pf->m);
    free(pf->eps2);
}

/* Eqs. psi and derivs with phi = a psi (Eq. phicotophys), evaluated as a
 * Plummer-softened sum over particles (comoving):
 *   phi(r)      = - mu_G sum_p m_p (|r - x_p|^2 + eps_p^2)^(-1/2)
 *   grad phi(r) =   mu_G sum_p m_p (r - x_p) (|r - x_p|^2 + eps_p^2)^(-3/2)
 * For mean-subtracted boxes the field of the replica's uniform mean density
 * is removed (Sec. 3.3: the mean density is subtracted from the field). */
static void field_eval(const orc_field *f, const prep_field *pf, int rep, const double *r,
                       double out[4], double *npairs)
{
    if (f->grid) {  /* grid path: the field interpolated from the nodes (App. B) */
        /* cube-tiled boxes: rep is the cell (replica, cube) the caller chose */
        orc_grid_eval(f->grid + (f->replicated ? rep : 0), r, out);
        return;
    }
    const double *w = pf->w[f->replicated ? rep : 0];
    nsum ph = {0, 0}, gx = {0, 0}, gy = {0, 0}, gz = {0, 0};
    for (int64_t i = 0; i < pf->n; ++i) {
        double dx = r[0] - w[3 * i], dy = r[1] - w[3 * i + 1], dz = r[2] - w[3 * i + 2];
        double r2 = dx * dx + dy * dy + dz * dz + pf->eps2[i];
        double inv = 1.0 / sqrt(r2);
        double mi = pf->m[i] * inv;
        double mi3 = mi * inv * inv;
        nadd(&ph, mi);
        nadd(&gx, mi3 * dx);
        nadd(&gy, mi3 * dy);
        nadd(&gz, mi3 * dz);
    }
    double mu = orc_mu_G();
    out[0] = -mu * nval(ph);
    out[1] = mu * nval(gx);
    out[2] = mu * nval(gy);
    out[3] = mu * nval(gz);
    if (npairs) *npairs += (double)pf->n;
    if (f->replicated && f->mean_subtract) {
        double L = f->L;
        double lo[3] = {-0.5 * L, -0.5 * L, (double)rep * L};
        double hi[3] = {0.5 * L, 0.5 * L, (double)(rep + 1) * L};
        double I[4];
        orc_prism(lo, hi, r, I);
        /* phi_bg = -mu_G rho I ; subtract it */
        double k = mu * pf->rho_bar;
        out[0] += k * I[0];
        out[1] += k * I[1];
        out[2] += k * I[2];
        out[3] += k * I[3];
    }
}

/* ------------------------------------------------------------------------ */
/* gridded field (Sec. 3.3 grid path; App. B "three-dimensional bicubic    */
/* spline"): natural cubic splines with unit node spacing.                  */
/* ------------------------------------------------------------------------ */
void orc_spline_y2(int n, const double *y, int64_t stride, double *y2)
{
    /* y2[0] = y2[n-1] = 0;  y2[i-1] + 4 y2[i] + y2[i+1] = 6 (y[i+1] - 2 y[i] + y[i-1]) */
    for (int i = 0; i < n; ++i) y2[i * stride] = 0.0;
    if (n < 3) return;
    double cp[4096], dp[4096];
    if (n - 2 >= 4096) return;
    cp[0] = 0.0;
    dp[0] = 0.0;  /* y2[0] = 0 enters the first row as a known value */
    for (int i = 1; i <= n - 2; ++i) {
        double d = 6.0 * (y[(i + 1) * stride] - 2.0 * y[i * stride] + y[(i - 1) * stride]);
        double den = 4.0 - cp[i - 1];
        cp[i] = 1.0 / den;
        dp[i] = (d - dp[i - 1]) / den;
    }
    y2[(n - 2) * stride] = dp[n - 2];
    for (int i = n - 3; i >= 1; --i) y2[i * stride] = dp[i] - cp[i] * y2[(i + 1) * stride];
}

void orc_grid_y2(int n, const double *val, double *y2)
{
    const int64_t lines = 4 * (int64_t)n * n;
    for (int64_t l = 0; l < lines; ++l) orc_spline_y2(n, val + l * n, 1, y2 + l * n);
}

/* cubic-spline value at u in [0, m-1] from values y and second derivatives y2 */
static double splint_unit(int m, const double *y, const double *y2, double u)
{
    int k = (int)floor(u);
    if (k > m - 2) k = m - 2;
    if (k < 0) k = 0;
    double A = (double)(k + 1) - u, B = u - (double)k;
    return A * y[k] + B * y[k + 1] + ((A * A * A - A) * y2[k] + (B * B * B - B) * y2[k + 1]) / 6.0;
}

void orc_grid_eval(const orc_grid *g, const double r[3], double out[4])
{
    const int n = g->n, w = 2 * g->n_int;
    double u[3];
    int s[3];
    for (int f = 0; f < 4; ++f) out[f] = 0.0;
    if (w < 2 || w > 16 || n < w) return;
    for (int d = 0; d < 3; ++d) {
        u[d] = (r[d] - g->lo[d]) / g->h;
        if (!(u[d] >= -g->margin && u[d] <= (double)(n - 1) + g->margin)) return;  /* outside: no field */
        s[d] = (int)floor(u[d]) - g->n_int + 1;
        if (s[d] > n - w) s[d] = n - w;
        if (s[d] < 0) s[d] = 0;
    }
    const int64_t n3 = (int64_t)n * n * n;
    for (int f = 0; f < 4; ++f) {
        const double *v = g->val + f * n3, *y2 = g->y2 + f * n3;
        double v1[16][16], v2[16], t[16], t2[16];
        /* step 1: along x3 on every (x1, x2) node of the window, global spline */
        for (int a = 0; a < w; ++a)
            for (int b = 0; b < w; ++b) {
                const int64_t line = ((int64_t)(s[0] + a) * n + (s[1] + b)) * n;
                v1[a][b] = splint_unit(n, v + line, y2 + line, u[2]);
            }
        /* steps 2-3: along x1, one local spline per x2 node */
        for (int b = 0; b < w; ++b) {
            for (int a = 0; a < w; ++a) t[a] = v1[a][b];
            orc_spline_y2(w, t, 1, t2);
            v2[b] = splint_unit(w, t, t2, u[0] - (double)s[0]);
        }
        /* steps 4-5: along x2 */
        orc_spline_y2(w, v2, 1, t2);
        out[f] = splint_unit(w, v2, t2, u[1] - (double)s[1]);
    }
}

/* READING (grid boxes): a bundle uses the cube holding its central ray's
 * stage position, as for replicas; the cell index is replica * cubes + cube */
static int cell_of(const orc_field *f, double x3)
{
    if (!f->replicated) return 0;
    double q = floor(x3 / f->L);
    int j = q < 0.0 ? 0 : (q > (double)(f->n_rep - 1) ? f->n_rep - 1 : (int)q);
    double W = f->L / (double)f->grid_cubes;
    double c = floor((x3 - (double)j * f->L) / W);
    int cc = c < 0.0 ? 0 : (c > (double)(f->grid_cubes - 1) ? f->grid_cubes - 1 : (int)c);
    return j * f->grid_cubes + cc;
}

void orc_replica_world(const orc_field *f, int j, double *out)
{
    replica_world(f, j, out);
}

static int rep_of(const orc_field *f, double x3)
{
    if (f->grid && f->replicated) return cell_of(f, x3);
    if (!f->replicated) return 0;
    double q = floor(x3 / f->L);
    if (q < 0.0) return 0;
    if (q > (double)(f->n_rep - 1)) return f->n_rep - 1;
    return (int)q;
}

int orc_potential(const orc_field *f, int64_t n, const double *pts, const int32_t *rep,
                  double *out, int nthreads)
{
    if (f->grid && f->replicated && f->grid_cubes < 1) return -1;
    prep_field pf;
    if (prep_make(f, &pf) != 0) { prep_free(&pf); return -2; }
    const int cubes = f->grid && f->replicated;  /* grid boxes: the point's own cell */
    for (int64_t i = 0; i < n; ++i)
        if (f->replicated && !cubes && (rep[i] < 0 || rep[i] >= f->n_rep)) { prep_free(&pf); return -1; }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t i = 0; i < n; ++i)
        field_eval(f, &pf, cubes ? cell_of(f, pts[3 * i + 2]) : (f->replicated ? rep[i] : 0), pts + 3 * i,
                   out + 4 * i, NULL);
    prep_free(&pf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* geodesic equation (Eq. geodesiceqn) with the Christoffel symbols of      */
/* App. A, contracted literally: d^2 x^a / dl^2 = -Gamma^a_bc u^b u^c.      */
/* index 0 = t, 1..3 = x, y, z.                                              */
/* ------------------------------------------------------------------------ */
void orc_geodesic_rhs(const orc_cosmo *c, const double y[8], const double F[4],
                      int christoffel, double dy[8])
{
    double a = orc_a_of_t(c, y[0]), ad = orc_adot_of_t(c, y[0]);
    double phi = F[0];
    const double *g = F + 1; /* phi_{,i} */
    double G[4][4][4];
    memset(G, 0, sizeof(G));
    for (int i = 1; i <= 3; ++i) {
        G[i][0][0] = g[i - 1] / (a * a * a);                 /* Gamma^i_tt */
        G[i][0][i] = G[i][i][0] = ad * (a + phi) / (a * a);   /* Gamma^i_ti */
        G[0][0][i] = G[0][i][0] = g[i - 1] / a;               /* Gamma^t_ti */
        G[0][i][i] = christoffel == 0 ? ad * (a + phi)        /* Gamma^t_ii, App. A */
                                      : ad * (a - 3.0 * phi); /* derived from the metric */
        for (int j = 1; j <= 3; ++j) {
            if (j == i) {
                G[i][i][i] = -g[i - 1] / a;                   /* Gamma^i_ii */
            } else {
                G[i][j][j] = g[i - 1] / a;                    /* Gamma^i_jj, j != i */
                G[i][i][j] = G[i][j][i] = -g[j - 1] / a;      /* Gamma^i_ij, j != i */
            }
        }
    }
    G[0][0][0] = -ad * phi / (a * a);                         /* Gamma^t_tt */
    const double *u = y + 4;
    for (int k = 0; k < 4; ++k) dy[k] = u[k];
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int b = 0; b < 4; ++b)
            for (int d = 0; d < 4; ++d) s += G[al][b][d] * u[b] * u[d];
        dy[4 + al] = -s;
    }
}

/* ------------------------------------------------------------------------ */
/* bundle Jacobian (Sec. 3.1 ray bundle; Eqs. lensmap, magnification).      */
/* READING: the ellipse fit is the least-squares linear map of the polygon  */
/* offsets, A = (sum dbeta dtheta^T)(sum dtheta dtheta^T)^-1.                */
/* ------------------------------------------------------------------------ */
void orc_bundle_jacobian(int n_ring, const double *theta0, const double *dtheta,
                         const double *xy, double chi_s, double out[6])
{
    (void)theta0;
    double M[2][2] = {{0, 0}, {0, 0}}, N[2][2] = {{0, 0}, {0, 0}};
    for (int k = 1; k <= n_ring; ++k) {
        double db[2] = {(xy[2 * k] - xy[0]) / chi_s, (xy[2 * k + 1] - xy[1]) / chi_s};
        const double *dt = dtheta + 2 * (k - 1);
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) {
                M[r][q] += db[r] * dt[q];
                N[r][q] += dt[r] * dt[q];
            }
    }
    double dn = N[0][0] * N[1][1] - N[0][1] * N[1][0];
    double Ni[2][2] = {{N[1][1] / dn, -N[0][1] / dn}, {-N[1][0] / dn, N[0][0] / dn}};
    double A[2][2];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) A[r][q] = M[r][0] * Ni[0][q] + M[r][1] * Ni[1][q];
    double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    out[0] = 1.0 / det;                          /* mu */
    out[1] = 1.0 - 0.5 * (A[0][0] + A[1][1]);    /* kappa */
    out[2] = 0.5 * (A[1][1] - A[0][0]);          /* gamma1 */
    out[3] = -0.5 * (A[0][1] + A[1][0]);         /* gamma2 */
    out[4] = 0.5 * (A[0][1] - A[1][0]);          /* omega (rotation) */
    out[5] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* full trace: RK4 with fixed steps in lambda (Sec. 3.4), terminated on x3, */
/* linear interpolation at the overshoot.                                    */
/* READING (initial conditions): t = 0, x = 0, direction (theta_x,          */
/* theta_y, 1) with dx3/dlambda = 1, dt/dlambda from the null condition.    */
/* READING (volume): at each stage the bundle uses the replica holding its  */
/* central ray's stage position.                                            */
/* ------------------------------------------------------------------------ */
int orc_trace(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b,
              const double *theta, const orc_trace_opts *o, double *ray_out,
              double *bundle_out, int32_t *steps_out, double *n_pairs, int nthreads)
{
    if (o->n_ring < 3 || o->n_ring > 8 || o->n_steps < 1 || !(z_s > 0.0)) return -1;
    if (f->grid && f->replicated && f->grid_cubes < 1) return -1;
    const int nr = 1 + o->n_ring;
    const double chi_s = orc_chi(c, z_s);
    double *dlam = (double *)malloc(sizeof(double) * (size_t)o->n_steps);
    if (!dlam) return -2;
    if (orc_schedule(c, chi_s, o->schedule, o->n_steps, o->lens_chi, o->asinh_s, dlam, NULL) != 0) {
        free(dlam);
        return -1;
    }
    prep_field pf;
    if (prep_make(f, &pf) != 0) { prep_free(&pf); free(dlam); return -2; }
    double total_pairs = 0.0;
    const double cs[4] = {0.0, 0.5, 0.5, 1.0};
    const int max_steps = o->n_steps + (o->max_extra > 0 ? o->max_extra : 0);

#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : total_pairs)
    for (int64_t b = 0; b < n_b; ++b) {
        double y[9][8], ys[9][8], kk[4][9][8], fin[9][8], th[9][2];
        int done[9], steps[9];
        double pairs = 0.0;
        th[0][0] = theta[2 * b];
        th[0][1] = theta[2 * b + 1];
        for (int k = 1; k < nr; ++k) {
            double ang = o->phase + 2.0 * M_PI * (double)(k - 1) / (double)o->n_ring;
            th[k][0] = th[0][0] + o->theta_r * cos(ang);
            th[k][1] = th[0][1] + o->theta_r * sin(ang);
        }
        for (int k = 0; k < nr; ++k) {
            double v[3] = {th[k][0], th[k][1], 1.0};
            y[k][0] = 0.0;
            y[k][1] = y[k][2] = y[k][3] = 0.0;
            y[k][5] = v[0];
            y[k][6] = v[1];
            y[k][7] = v[2];
            double F[4];
            field_eval(f, &pf, rep_of(f, 0.0), y[k] + 1, F, &pairs);
            double a = orc_a_of_t(c, 0.0), vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            /* null condition of Eq. expandingmetric with psi = phi/a */
            y[k][4] = a * vn * sqrt((1.0 - 2.0 * F[0] / a) / (1.0 + 2.0 * F[0] / a));
            done[k] = 0;
            steps[k] = -1;
        }
        for (int step = 0; step < max_steps; ++step) {
            double dl = dlam[step < o->n_steps ? step : o->n_steps - 1];
            for (int s = 0; s < 4; ++s) {
                for (int k = 0; k < nr; ++k)
                    for (int q = 0; q < 8; ++q)
                        ys[k][q] = s == 0 ? y[k][q] : y[k][q] + cs[s] * dl * kk[s - 1][k][q];
                int rep = rep_of(f, ys[0][3]);
                for (int k = 0; k < nr; ++k) {
                    double F[4];
                    field_eval(f, &pf, rep, ys[k] + 1, F, done[k] ? NULL : &pairs);
                    orc_geodesic_rhs(c, ys[k], F, o->christoffel, kk[s][k]);
                }
            }
            int all = 1;
            for (int k = 0; k < nr; ++k) {
                double yn[8];
                for (int q = 0; q < 8; ++q)
                    yn[q] = y[k][q] + dl / 6.0 * (kk[0][k][q] + 2.0 * kk[1][k][q] + 2.0 * kk[2][k][q] + kk[3][k][q]);
                if (!done[k] && yn[3] >= chi_s) {
                    double sfr = (chi_s - y[k][3]) / (yn[3] - y[k][3]);
                    for (int q = 0; q < 8; ++q) fin[k][q] = y[k][q] + sfr * (yn[q] - y[k][q]);
                    done[k] = 1;
                    steps[k] = step + 1;
                }
                for (int q = 0; q < 8; ++q) y[k][q] = yn[q];
                all &= done[k];
            }
            if (all) break;
        }
        int flags = 0;
        for (int k = 0; k < nr; ++k) {
            if (!done[k]) {
                flags |= ORC_F_NOCROSS;
                for (int q = 0; q < 8; ++q) fin[k][q] = y[k][q];
            }
            for (int q = 0; q < 8; ++q) {
                if (!isfinite(fin[k][q])) flags |= ORC_F_NONFINITE;
                ray_out[((size_t)b * nr + k) * 8 + q] = fin[k][q];
            }
            if (steps_out) steps_out[(size_t)b * nr + k] = steps[k];
        }
        double xy[18], dth[16];
        for (int k = 0; k < nr; ++k) {
            xy[2 * k] = fin[k][1];
            xy[2 * k + 1] = fin[k][2];
        }
        for (int k = 1; k < nr; ++k) {
            dth[2 * (k - 1)] = th[k][0] - th[0][0];
            dth[2 * (k - 1) + 1] = th[k][1] - th[0][1];
        }
        double J[6];
        orc_bundle_jacobian(o->n_ring, th[0], dth, xy, chi_s, J);
        if (!isfinite(J[0])) flags |= ORC_F_NONFINITE;
        if (J[0] < 0.0) flags |= ORC_F_NEGPARITY;
        J[5] = (double)flags;
        for (int q = 0; q < 6; ++q) bundle_out[(size_t)b * 6 + q] = J[q];
        total_pairs += pairs;
    }
    if (n_pairs) *n_pairs = total_pairs;
    prep_free(&pf);
    free(dlam);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* mu PDF (Sec. 5.3, Eq. weighthisto): counts weighted by 1/mu.             */
/* READING: bins uniform in log10|mu|; negative parity binned by |mu| and   */
/* counted; flagged (no-cross, non-finite) bundles are excluded.            */
/* ------------------------------------------------------------------------ */
int orc_histogram(int64_t n, const double *mu, const int32_t *flags, const orc_hist_opts *o,
                  uint64_t *counts, uint64_t *wfix, double *sc)
{
    if (o->bins < 1 || !(o->mu_min > 0.0) || !(o->mu_max > o->mu_min)) return -1;
    memset(counts, 0, sizeof(uint64_t) * (size_t)o->bins);
    memset(wfix, 0, sizeof(uint64_t) * (size_t)o->bins);
    double lmin = log10(o->mu_min);
    double dl = (log10(o->mu_max) - lmin) / (double)o->bins;
    int64_t used = 0, under = 0, over = 0, neg = 0, bad = 0;
    nsum W = {0, 0}, S1 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int fl = flags ? flags[i] : 0;
        if ((fl & (ORC_F_NOCROSS | ORC_F_NONFINITE)) || !isfinite(mu[i]) || mu[i] == 0.0) { ++bad; continue; }
        double m = fabs(mu[i]);
        if (mu[i] < 0.0) ++neg;
        double w = 1.0 / m;
        nadd(&W, w);
        nadd(&S1, w * m);
        double bb = floor((log10(m) - lmin) / dl);
        if (bb < 0.0) ++under;
        else if (bb >= (double)o->bins) ++over;
        else {
            int64_t k = (int64_t)bb;
            counts[k] += 1;
            wfix[k] += (uint64_t)llrint(ldexp(w, 32));
        }
        ++used;
    }
    double Wt = nval(W), mean = used ? nval(S1) / Wt : 0.0;
    nsum S2 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int fl = flags ? flags[i] : 0;
        if ((fl & (ORC_F_NOCROSS | ORC_F_NONFINITE)) || !isfinite(mu[i]) || mu[i] == 0.0) continue;
        double m = fabs(mu[i]), d = m - mean;
        nadd(&S2, d * d / m);
    }
    sc[0] = (double)used;
    sc[1] = (double)under;
    sc[2] = (double)over;
    sc[3] = (double)neg;
    sc[4] = (double)bad;
    sc[5] = Wt;
    sc[6] = mean;
    sc[7] = used ? sqrt(nval(S2) / Wt) : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* shear PDF (Sec. 5.4): |gamma| per bundle, source-plane weight 1/|mu|.     */
/* READING: the paper does not state the weighting of its shear PDF; the    */
/* 1/mu weight of Eq. weighthisto is used, bins uniform in log10|gamma|.     */
/* ------------------------------------------------------------------------ */
int orc_shear_histogram(int64_t n, const double *mu, const double *g1, const double *g2,
                        const int32_t *flags, const orc_hist_opts *o, uint64_t *counts,
                        uint64_t *wfix, double *sc)
{
    if (o->bins < 1 || !(o->mu_min > 0.0) || !(o->mu_max > o->mu_min)) return -1;
    memset(counts, 0, sizeof(uint64_t) * (size_t)o->bins);
    memset(wfix, 0, sizeof(uint64_t) * (size_t)o->bins);
    double lmin = log10(o->mu_min);
    double dl = (log10(o->mu_max) - lmin) / (double)o->bins;
    int64_t used = 0, under = 0, over = 0, neg = 0, bad = 0;
    nsum W = {0, 0}, S1 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int fl = flags ? flags[i] : 0;
        double g = sqrt(g1[i] * g1[i] + g2[i] * g2[i]);
        if ((fl & (ORC_F_NOCROSS | ORC_F_NONFINITE)) || !isfinite(mu[i]) || mu[i] == 0.0 || !isfinite(g)) {
            ++bad;
            continue;
        }
        if (mu[i] < 0.0) ++neg;
        double w = 1.0 / fabs(mu[i]);
        nadd(&W, w);
        nadd(&S1, w * g);
        double bb = floor((log10(g) - lmin) / dl);
        if (bb < 0.0) ++under;
        else if (bb >= (double)o->bins) ++over;
        else {
            int64_t k = (int64_t)bb;
            counts[k] += 1;
            wfix[k] += (uint64_t)llrint(ldexp(w, 32));
        }
        ++used;
    }
    double Wt = nval(W), mean = used ? nval(S1) / Wt : 0.0;
    nsum S2 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int fl = flags ? flags[i] : 0;
        double g = sqrt(g1[i] * g1[i] + g2[i] * g2[i]);
        if ((fl & (ORC_F_NOCROSS | ORC_F_NONFINITE)) || !isfinite(mu[i]) || mu[i] == 0.0 || !isfinite(g)) continue;
        double d = g - mean;
        nadd(&S2, d * d / fabs(mu[i]));
    }
    sc[0] = (double)used;
    sc[1] = (double)under;
    sc[2] = (double)over;
    sc[3] = (double)neg;
    sc[4] = (double)bad;
    sc[5] = Wt;
    sc[6] = mean;
    sc[7] = used ? sqrt(nval(S2) / Wt) : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Born approximation (Sec. 6): convergence and shear along the unperturbed */
/* line of sight x(chi) = (theta_x chi, theta_y chi, chi).  With A_ij =     */
/* d_ij - 2 int W d_i d_j psi dchi, W = chi (chi_s - chi) / chi_s, psi =    */
/* phi / a (Eq. phicotophys):                                               */
/*   kappa = int W (d11 + d22) psi,  gamma1 = int W (d11 - d22) psi,        */
/*   gamma2 = 2 int W d12 psi.                                              */
/* READING: the integral runs over the trace's node table (Eq. RKstepsize   */
/* reading) by the trapezoid rule in the node variable (uniform in chi, or  */
/* in u for the asinh nodes chi = chi_l + s sinh u); a(chi) = 1/(1+z(chi)); */
/* boxes use the replica holding the node, minus the mean-density prism.    */
/* ------------------------------------------------------------------------ */
static void hessian_eval(const orc_field *f, const prep_field *pf, int rep, const double *r, double h[6])
{
    const double *w = pf->w[f->replicated ? rep : 0];
    nsum s[6];
    for (int q = 0; q < 6; ++q) s[q].s = s[q].c = 0.0;
    for (int64_t i = 0; i < pf->n; ++i) {
        double d[3] = {r[0] - w[3 * i], r[1] - w[3 * i + 1], r[2] - w[3 * i + 2]};
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + pf->eps2[i];
        double inv = 1.0 / sqrt(r2);
        double i3 = pf->m[i] * inv * inv * inv, i5 = i3 * inv * inv;
        /* d_i d_j of -m / r: m (delta_ij / r^3 - 3 d_i d_j / r^5) */
        nadd(&s[0], i3 - 3.0 * d[0] * d[0] * i5);
        nadd(&s[1], -3.0 * d[0] * d[1] * i5);
        nadd(&s[2], -3.0 * d[0] * d[2] * i5);
        nadd(&s[3], i3 - 3.0 * d[1] * d[1] * i5);
        nadd(&s[4], -3.0 * d[1] * d[2] * i5);
        nadd(&s[5], i3 - 3.0 * d[2] * d[2] * i5);
    }
    double mu = orc_mu_G();
    for (int q = 0; q < 6; ++q) h[q] = mu * nval(s[q]);
    if (f->replicated && f->mean_subtract) {
        double L = f->L;
        double lo[3] = {-0.5 * L, -0.5 * L, (double)rep * L};
        double hi[3] = {0.5 * L, 0.5 * L, (double)(rep + 1) * L};
        double H[6];
        orc_prism_hessian(lo, hi, r, H);
        double k = mu * pf->rho_bar;  /* phi_bg = -mu_G rho I: its Hessian is removed */
        for (int q = 0; q < 6; ++q) h[q] += k * H[q];
    }
}

int orc_born(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b, const double *theta,
             const orc_trace_opts *o, double *out, int nthreads)
{
    if (o->n_steps < 1 || !(z_s > 0.0) || f->grid) return -1;
    const int n = o->n_steps;
    const double chi_s = orc_chi(c, z_s);
    double *x = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *dl = (double *)malloc(sizeof(double) * (size_t)n);
    double *wt = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!x || !dl || !wt) { free(x); free(dl); free(wt); return -2; }
    if (orc_schedule(c, chi_s, o->schedule, n, o->lens_chi, o->asinh_s, dl, x) != 0) {
        free(x); free(dl); free(wt);
        return -1;
    }
    /* trapezoid weights in the node variable times W / a */
    double du = o->schedule == 1 ? (asinh((chi_s - o->lens_chi) / o->asinh_s) - asinh(-o->lens_chi / o->asinh_s)) / n
                                 : chi_s / n;
    for (int k = 0; k <= n; ++k) {
        double jac = o->schedule == 1 ? sqrt(o->asinh_s * o->asinh_s + (x[k] - o->lens_chi) * (x[k] - o->lens_chi))
                                      : 1.0;
        double W = x[k] * (chi_s - x[k]) / chi_s;
        double inv_a = 1.0 + orc_z_of_chi(c, x[k]);
        wt[k] = (k == 0 || k == n ? 0.5 : 1.0) * du * jac * W * inv_a;
    }
    prep_field pf;
    if (prep_make(f, &pf) != 0) { prep_free(&pf); free(x); free(dl); free(wt); return -2; }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t b = 0; b < n_b; ++b) {
        nsum kap = {0, 0}, g1 = {0, 0}, g2 = {0, 0};
        for (int k = 0; k <= n; ++k) {
            if (wt[k] == 0.0) continue;
            double r[3] = {theta[2 * b] * x[k], theta[2 * b + 1] * x[k], x[k]};
            double h[6];
            hessian_eval(f, &pf, rep_of(f, x[k]), r, h);
            nadd(&kap, wt[k] * (h[0] + h[3]));
            nadd(&g1, wt[k] * (h[0] - h[3]));
            nadd(&g2, wt[k] * 2.0 * h[1]);
        }
        out[3 * b] = nval(kap);
        out[3 * b + 1] = nval(g1);
        out[3 * b + 2] = nval(g2);
    }
    prep_free(&pf);
    free(x); free(dl); free(wt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* multiple lens-plane comparison system (Sec. 3.1 "Multiple lens plane     */
/* methods"; Eqs. defangleB, lenseqn, defangle): the mass between observer  */
/* and source is cut into slabs along x3, each slab projected onto a plane  */
/* at its centre; a ray travels straight between planes and is deflected    */
/* only at them, by the matter of that plane.                               */
/* READING (planes): replicated fields: replica j's range [jL, (j+1)L) in  */
/* `slices` slabs of equal thickness, each cut at the source plane x3 =     */
/* chi_s; isolated fields: the particles' x3 range in `slices` slabs (one   */
/* particle, or slices = 1 with all particles at one x3: one plane there).  */
/* Particles beyond the source plane or behind the observer are left out.   */
/* READING (deflection): the projected Plummer particle deflects by the     */
/* thin-lens angle of Eq. defangleB for its Plummer-sphere surface density: */
/*   alpha_hat(x) = 4 mu_G (1 + z_k) sum_p m_p (x - x_p)/(|x - x_p|^2 + e_p^2) */
/* in comoving transverse coordinates (x = (1 + z_k) xi), which makes the  */
/* recursion below the multi-plane lens equation of Sec. 3.1 in a flat     */
/* universe (D_ij = (chi_j - chi_i) / (1 + z_j)).                            */
/* READING (mean): mean-subtracted boxes also remove the deflection of the  */
/* slab's uniform mean surface density rho_bar * thickness over the square  */
/* |x1|, |x2| < L/2 (the 2D analogue of the 3D path's prism).                */
/* READING (propagation): tangent-plane slopes as in the 3D trace's initial */
/* conditions; x(chi) = x_k + (chi - chi_k) theta between planes and        */
/* theta -> theta - alpha_hat at plane k (small angles).                    */
/* ------------------------------------------------------------------------ */
/* g(u, v) = u atan(v/u) + (v/2) ln(u^2 + v^2): d^2 g / du dv = u / (u^2 + v^2) */
static double rect_g(double u, double v)
{
    double q = u * u + v * v;
    if (q == 0.0) return 0.0;
    double a = u != 0.0 ? u * atan(v / u) : 0.0;
    return a + 0.5 * v * log(q);
}

void orc_rect_deflection(const double lo[2], const double hi[2], const double x[2], double out[2])
{
    /* int over [lo, hi] of (x - x') / |x - x'|^2 d^2x', with u = x - x' */
    double u1 = x[0] - lo[0], u0 = x[0] - hi[0];
    double v1 = x[1] - lo[1], v0 = x[1] - hi[1];
    out[0] = rect_g(u1, v1) - rect_g(u0, v1) - rect_g(u1, v0) + rect_g(u0, v0);
    out[1] = rect_g(v1, u1) - rect_g(v1, u0) - rect_g(v0, u1) + rect_g(v0, u0);
}

typedef struct {
    double chi, z, lo, hi;  /* plane position, its redshift, slab [lo, hi) */
    int rep;                /* replica (replicated fields) */
    int64_t n;              /* particles on the plane */
    double *x;              /* n*2 transverse positions */
    double *m, *e2;         /* n masses, n softening^2 */
} mp_plane;

static void mp_free(mp_plane *pl, int np)
{
    for (int k = 0; k < np; ++k) {
        free(pl[k].x);
        free(pl[k].m);
        free(pl[k].e2);
    }
    free(pl);
}

/* the planes of field f up to chi_s (see the readings above); returns the
 * count, or -1 on a bad option, -2 on allocation failure */
static int mp_planes(const orc_cosmo *c, const orc_field *f, double chi_s, int slices, mp_plane **out)
{
    *out = NULL;
    if (slices < 1 || f->grid) return -1;
    int nrep = f->replicated ? f->n_rep : 1;
    int np = nrep * slices;
    mp_plane *pl = (mp_plane *)calloc((size_t)np, sizeof(mp_plane));
    if (!pl) return -2;
    double xlo = 0.0, xhi = 0.0;
    if (!f->replicated && f->n > 0) {
        xlo = xhi = f->pos[2];
        for (int64_t i = 1; i < f->n; ++i) {
            if (f->pos[3 * i + 2] < xlo) xlo = f->pos[3 * i + 2];
            if (f->pos[3 * i + 2] > xhi) xhi = f->pos[3 * i + 2];
        }
    }
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)(f->n > 0 ? f->n : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)slices, sizeof(int64_t));
    if (!w || !cnt) { free(w); free(cnt); mp_free(pl, np); return -2; }
    int used = 0;
    for (int j = 0; j < nrep; ++j) {
        double a, b;
        if (f->replicated) {
            replica_world(f, j, w);
            a = (double)j * f->L;
            b = a + f->L;
        } else {
            memcpy(w, f->pos, sizeof(double) * 3 * (size_t)f->n);
            a = xlo;
            b = xhi;
        }
        double d = (b - a) / (double)slices;
        /* slab of each particle; -1: outside [0, chi_s) or the replica */
        memset(cnt, 0, sizeof(int64_t) * (size_t)slices);
        for (int64_t i = 0; i < f->n; ++i) {
            double x3 = w[3 * i + 2];
            int s = d > 0.0 ? (int)floor((x3 - a) / d) : 0;
            if (s >= slices) s = slices - 1;  /* the particle at the far end of an isolated range */
            if (s < 0 || x3 < 0.0 || x3 >= chi_s || (f->replicated && (x3 < a || x3 >= b))) continue;
            cnt[s]++;
        }
        for (int s = 0; s < slices; ++s) {
            double lo = d > 0.0 ? a + d * (double)s : a, hi = d > 0.0 ? a + d * (double)(s + 1) : a;
            if (hi > chi_s) hi = chi_s;
            if (lo < 0.0) lo = 0.0;
            if (f->replicated ? !(hi > lo) : (cnt[s] == 0)) continue;
            mp_plane *p = pl + used++;
            p->lo = lo;
            p->hi = hi;
            p->chi = 0.5 * (lo + hi);
            p->z = orc_z_of_chi(c, p->chi);
            p->rep = j;
            p->n = 0;
            p->x = (double *)malloc(sizeof(double) * 2 * (size_t)(cnt[s] > 0 ? cnt[s] : 1));
            p->m = (double *)malloc(sizeof(double) * (size_t)(cnt[s] > 0 ? cnt[s] : 1));
            p->e2 = (double *)malloc(sizeof(double) * (size_t)(cnt[s] > 0 ? cnt[s] : 1));
            if (!p->x || !p->m || !p->e2) { free(w); free(cnt); mp_free(pl, np); return -2; }
            for (int64_t i = 0; i < f->n; ++i) {
                double x3 = w[3 * i + 2];
                int s2 = d > 0.0 ? (int)floor((x3 - a) / d) : 0;
                if (s2 >= slices) s2 = slices - 1;
                if (s2 != s || x3 < 0.0 || x3 >= chi_s || (f->replicated && (x3 < a || x3 >= b))) continue;
                double e = f->soft ? f->soft[i] : f->soft_scalar;
                p->x[2 * p->n] = w[3 * i];
                p->x[2 * p->n + 1] = w[3 * i + 1];
                p->m[p->n] = f->mass[i];
                p->e2[p->n] = e * e;
                p->n++;
            }
        }
    }
    free(w);
    free(cnt);
    /* planes in order of distance (isolated slabs and replicas already are) */
    *out = pl;
    return used;
}

int orc_multiplane(const orc_cosmo *c, const orc_field *f, double z_s, int64_t n_b, const double *theta,
                   const orc_mp_opts *o, double *ray_out, double *bundle_out, double *planes_out,
                   int *n_planes, double *n_pairs, int nthreads)
{
    if (o->n_ring < 3 || o->n_ring > 8 || !(z_s > 0.0) || o->slices < 1) return -1;
    const int nr = 1 + o->n_ring;
    const double chi_s = orc_chi(c, z_s);
    mp_plane *pl = NULL;
    int np = mp_planes(c, f, chi_s, o->slices, &pl);
    if (np < 0) return np;
    double rho_bar = 0.0;
    if (f->replicated && f->mean_subtract) {
        nsum mt = {0, 0};
        for (int64_t i = 0; i < f->n; ++i) nadd(&mt, f->mass[i]);
        rho_bar = nval(mt) / (f->L * f->L * f->L);
    }
    const double mu4 = 4.0 * orc_mu_G();
    double total = 0.0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : total)
    for (int64_t b = 0; b < n_b; ++b) {
        double th[9][2], x[9][2], xs[18], dth[16];
        th[0][0] = theta[2 * b];
        th[0][1] = theta[2 * b + 1];
        for (int k = 1; k < nr; ++k) {
            double ang = o->phase + 2.0 * M_PI * (double)(k - 1) / (double)o->n_ring;
            th[k][0] = th[0][0] + o->theta_r * cos(ang);
            th[k][1] = th[0][1] + o->theta_r * sin(ang);
        }
        for (int k = 1; k < nr; ++k) {
            dth[2 * (k - 1)] = th[k][0] - th[0][0];
            dth[2 * (k - 1) + 1] = th[k][1] - th[0][1];
        }
        for (int k = 0; k < nr; ++k) {
            double t[2] = {th[k][0], th[k][1]}, chi = 0.0;
            x[k][0] = x[k][1] = 0.0;
            for (int q = 0; q < np; ++q) {
                const mp_plane *p = pl + q;
                x[k][0] += (p->chi - chi) * t[0];
                x[k][1] += (p->chi - chi) * t[1];
                chi = p->chi;
                nsum ax = {0, 0}, ay = {0, 0};
                for (int64_t i = 0; i < p->n; ++i) {
                    double dx = x[k][0] - p->x[2 * i], dy = x[k][1] - p->x[2 * i + 1];
                    double w = p->m[i] / (dx * dx + dy * dy + p->e2[i]);
                    nadd(&ax, w * dx);
                    nadd(&ay, w * dy);
                }
                total += (double)p->n;
                double a[2] = {nval(ax), nval(ay)};
                if (rho_bar > 0.0) {
                    double sig = rho_bar * (p->hi - p->lo);
                    double lo[2] = {-0.5 * f->L, -0.5 * f->L}, hi[2] = {0.5 * f->L, 0.5 * f->L}, r[2];
                    orc_rect_deflection(lo, hi, x[k], r);
                    a[0] -= sig * r[0];
                    a[1] -= sig * r[1];
                }
                double g = mu4 * (1.0 + p->z);
                t[0] -= g * a[0];
                t[1] -= g * a[1];
            }
            x[k][0] += (chi_s - chi) * t[0];
            x[k][1] += (chi_s - chi) * t[1];
            xs[2 * k] = x[k][0];
            xs[2 * k + 1] = x[k][1];
            if (ray_out) {
                ray_out[((size_t)b * nr + k) * 2] = x[k][0];
                ray_out[((size_t)b * nr + k) * 2 + 1] = x[k][1];
            }
        }
        double J[6];
        orc_bundle_jacobian(o->n_ring, th[0], dth, xs, chi_s, J);
        int flags = 0;
        for (int q = 0; q < 2 * nr; ++q)
            if (!isfinite(xs[q])) flags |= ORC_F_NONFINITE;
        if (!isfinite(J[0])) flags |= ORC_F_NONFINITE;
        if (J[0] < 0.0) flags |= ORC_F_NEGPARITY;
        J[5] = (double)flags;
        for (int q = 0; q < 6; ++q) bundle_out[(size_t)b * 6 + q] = J[q];
    }
    if (planes_out)
        for (int q = 0; q < np; ++q) {
            planes_out[4 * q] = pl[q].chi;
            planes_out[4 * q + 1] = pl[q].z;
            planes_out[4 * q + 2] = (double)pl[q].n;
            planes_out[4 * q + 3] = pl[q].hi - pl[q].lo;
        }
    if (n_planes) *n_planes = np;
    if (n_pairs) *n_pairs = total;
    mp_free(pl, f->replicated ? f->n_rep * o->slices : o->slices);
    return 0;
}

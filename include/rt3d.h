/*
 * rt3d.h -- C ABI of the GB300 (sm_103a) 3D ray-bundle lensing library.
 *
 * The library integrates bundles of null geodesics from the observer to a
 * source plane through a particle mass distribution, without the thin-lens
 * approximation, following Killedar, Lasky, Lewis & Fluke (2011),
 * "Gravitational Lensing with Three-Dimensional Ray Tracing":
 *   - metric: the weakly perturbed flat FRW metric, Eq. expandingmetric, with
 *     psi = phi / a (Eq. phicotophys);
 *   - potential: Eqs. psi / derivs evaluated as a Plummer-softened direct sum
 *     over the particles (comoving), optionally minus the field of the
 *     replica's uniform mean density (Sec. 3.3);
 *   - geodesic equation: Eq. geodesiceqn with the Christoffel symbols of
 *     App. A, classical RK4 with fixed steps in the affine parameter,
 *     terminated on the x3 coordinate with linear interpolation (Sec. 3.4);
 *   - scale factor: Eq. scalefac2 of the lookback time carried by each ray;
 *   - bundles: a central ray and a regular polygon of rays (Sec. 3.1); the
 *     lens-map Jacobian (Eq. lensmap) gives mu, kappa, gamma (Eq. magnification);
 *   - muPDF: counts weighted by 1/mu (Eq. weighthisto).
 *
 * Units: comoving Mpc for lengths, Mpc for time (c = 1), solar masses,
 * radians for angles.
 *
 * Conventions for every entry point:
 *   - return RT3D_OK (0) or a negative RT3D_E* code; nothing aborts or
 *     throws across the ABI; rt3d_last_error() holds a message per context;
 *   - host pointers are read during the call only; output arrays are owned
 *     by the caller and sized as stated; the context owns all device memory
 *     it allocates and frees it in rt3d_destroy();
 *   - one context per host thread; calls on one context are not reentrant;
 *   - entry points without "_device" are synchronous; the _device variants
 *     take device pointers and a cudaStream_t and only enqueue work.
 */
#ifndef RT3D_H
#define RT3D_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT3D_OK 0
#define RT3D_EINVAL (-1)   /* bad argument (NaN, negative mass, empty, out of range) */
#define RT3D_ENOMEM (-2)   /* device or host allocation failed */
#define RT3D_ECUDA (-3)    /* a CUDA runtime call failed */
#define RT3D_ETIMEOUT (-4) /* a device watchdog expired */
#define RT3D_ENOTIMPL (-5) /* option not implemented */
#define RT3D_ENOCOSMO (-6) /* trace before rt3d_set_cosmology */
#define RT3D_ENOFIELD (-7) /* field id not loaded */

#define RT3D_MIXED 0 /* FP32 pair sums with compensated accumulation, FP64 ray state */
#define RT3D_FP64 1  /* every step in FP64 */

#define RT3D_CHRISTOFFEL_PAPER 0   /* App. A as printed: Gamma^t_ii = a-dot (a + phi) */
#define RT3D_CHRISTOFFEL_DERIVED 1 /* from the metric to first order: a-dot (a - 3 phi) */

#define RT3D_SCHED_UNIFORM 0 /* nodes uniform in x3 */
#define RT3D_SCHED_ASINH 1   /* nodes x3_k = chi_l + s sinh(u_k), u uniform */

#define RT3D_F_NOCROSS 1   /* a ray did not reach x3 = chi_s within n_steps + max_extra */
#define RT3D_F_NONFINITE 2 /* a non-finite state or magnification */
#define RT3D_F_NEGPARITY 4 /* det A < 0 (image of negative parity) */

#define RT3D_MAX_FIELDS 1024

typedef struct rt3d_ctx rt3d_ctx;

typedef struct {
    int precision;         /* RT3D_MIXED (default) or RT3D_FP64 */
    int christoffel;       /* RT3D_CHRISTOFFEL_PAPER (default) or _DERIVED */
    int rays_per_thread;   /* force-kernel register blocking (1, 2, 4); 0 = tuned */
    int threads_per_block; /* force-kernel block size (64..512); 0 = tuned */
    int splits;            /* particle splits per ray block; 0 = tuned */
    int autotune;          /* 1: time candidate launch shapes once per size bucket */
    double watchdog_s;     /* limit for the persistent kernel's grid-barrier waits; 0 = 120 s */
    int time_kernels;      /* 1: bracket every pair-sum launch with CUDA events (stats.force_ms) */
    int variant;           /* pair-sum kernel: 0 = automatic (bundle-centric FP32x2 for traces:
                              5 for rings of 4 and 8, 3 otherwise; with autotune, the fastest of
                              3, 4, 5), 1 = scalar FP32, 2 = packed FP32x2 per ray, 3 = one bundle
                              per thread, 4 = two bundles per thread (rings of 4), 5 = two bundles
                              per thread with the ring separations expanded about the central ray
                              (rings of 4 and 8; rings of 8 in blocks of 64).  rt3d_trace_batch:
                              3 = bundle-centric items, 5 = expanded two-bundle items (64
                              threads; the default for rings of 4), 0 with autotune = the faster */
    int cluster;           /* variant 5, rings of 4: 4 = thread-block clusters of 4 splits add their
                              partials in distributed shared memory, 1 = no clusters, 0 = automatic
                              (none unless the autotuner finds clusters faster) */
} rt3d_options;

/* Mass distribution layout.
 * replicated = 0: an isolated field; positions are world coordinates.
 * replicated = 1: a periodic box [0, box_length)^3; replica j is the box
 *   rotated about its centre by rot[j] (a 3x3 signed permutation, row-major),
 *   shifted by shift[j] with periodic wrap, centred on the optical axis in
 *   x1, x2 and placed at x3 in [j L, (j+1) L) (Sec. 5.2).  A bundle uses the
 *   replica that holds its central ray's stage position. */
typedef struct {
    int replicated;
    double box_length;
    int n_replicas;
    const int32_t *rot;   /* n_replicas * 9 (host) */
    const double *shift;  /* n_replicas * 3 (host), in [0, box_length) */
    int mean_subtract;    /* subtract the field of the box's mean particle density */
} rt3d_volume;

typedef struct {
    int n_ring;      /* rays on the polygon (3..8; two rays would be collinear and fix no
                        Jacobian); the paper uses 8 (Sec. 3.1, Sec. 5.2), default 4 */
    double theta_r;  /* polygon radius (rad) */
    double phase;    /* polygon orientation (rad) */
    int schedule;    /* RT3D_SCHED_* */
    int n_steps;     /* RK4 steps in the node table */
    double lens_chi; /* asinh schedule: centre (comoving Mpc) */
    double asinh_s;  /* asinh schedule: scale (comoving Mpc) */
    int max_extra;   /* further steps of the last size for rays not yet across (<= 64) */
} rt3d_bundle_opts;

/* Per-bundle results (caller-owned host arrays of n_bundles; optional ones may be NULL). */
typedef struct {
    double *mu, *kappa, *gamma1, *gamma2, *omega;
    int32_t *flags;
    double *ray_state;  /* optional: n_bundles*(1+n_ring)*8 final (t,x1,x2,x3,dt,dx1,dx2,dx3) */
    int32_t *ray_steps; /* optional: n_bundles*(1+n_ring) step at which each ray crossed */
} rt3d_bundle_result;

typedef struct {
    int bins;      /* >= 1 */
    double mu_min; /* > 0 */
    double mu_max; /* > mu_min */
} rt3d_hist_opts;

typedef struct {
    uint64_t *counts; /* caller-owned [bins] */
    uint64_t *wfix;   /* caller-owned [bins]: sum of round(2^32 / |mu|) */
    int64_t n_used, n_under, n_over, n_neg, n_bad;
    double W_total, mean_w, sigma_w;
} rt3d_hist;

typedef struct {
    double interactions;  /* (ray, particle) pairs evaluated for rays not yet across */
    double device_ms;     /* device time of the last trace/batch (CUDA events) */
    double force_ms;      /* device time inside the pair-sum kernels */
    int64_t launches;     /* kernels launched by the last trace/batch */
    int64_t force_launches;
    int steps;            /* RK4 steps issued */
    int rays_per_thread, threads_per_block, splits; /* force launch shape used */
    int variant;          /* pair-sum kernel used: 0 packed, 1 scalar, 2 FP64, 3 bundle, 4 two bundles
                             per thread, 5 two bundles per thread, expanded separations, 6 grid path */
    int cluster;          /* thread-block cluster size along the splits (1: none); the
                             cluster's splits are added in distributed shared memory */
} rt3d_stats;

/* One light cone of a batch (Sec. 5): its field, source redshift, bundles and steps. */
typedef struct {
    int field_id;
    double z_s;
    int64_t n_bundles;
    const double *theta; /* host n_bundles*2 */
    int n_steps;
} rt3d_cone;

/* Create a context on CUDA device cuda_device; opt may be NULL (defaults).
 * The options select how the method of Sec. 3 is computed: opt->precision
 * RT3D_MIXED sums the pair terms of Eqs. psi / derivs in FP32 with
 * compensated accumulation and keeps the ray state of Eq. geodesiceqn, the
 * background of Sec. 3.5 and the Jacobian of Eq. lensmap in FP64; RT3D_FP64
 * computes every step in FP64.  RT3D_MIXED meets |dmu/mu| <= 1e-4 on softened
 * fields; it does not on an unsoftened point lens (eps = 0) traced with
 * bundles of 1e-3 Einstein radii (Sec. 4.1), whose ring-central deflection
 * difference is below FP32 resolution: use RT3D_FP64 there.
 * opt->christoffel selects App. A's symbols as printed or as derived.
 * Errors: RT3D_EINVAL (no such device, bad option), RT3D_ENOMEM, RT3D_ECUDA. */
int rt3d_create(rt3d_ctx **out, int cuda_device, const rt3d_options *opt);
/* Free every device allocation of the context (the paper has no counterpart:
 * resource management only).  The context may not be used afterwards. */
int rt3d_destroy(rt3d_ctx *ctx);

/* Flat LCDM background (Sec. 3.5): |omega_m + omega_l - 1| <= 1e-12, h > 0. */
int rt3d_set_cosmology(rt3d_ctx *ctx, double omega_m, double omega_l, double h);

/* The mass distribution of Sec. 3.3 (N-body particles, the potential of
 * Eqs. psi / derivs) and its replication along the line of sight of Sec. 5.2.
 * Copy a particle set to the device as field field_id (0..RT3D_MAX_FIELDS-1,
 * replacing any previous one).  pos: n*3, mass: n (> 0), soft: n Plummer
 * softening lengths if soft_per_particle, else soft[0] for all (>= 0).
 * Positions are stored as integers on a grid of 2^-e Mpc, the finest that
 * holds the field: 2^30 grid units for the largest distance of an isolated
 * field's particles from its centre, 2^31 for a replicated box's length.
 * Coordinates that are multiples of 2^-e Mpc are kept exactly; others are
 * rounded to the nearest multiple (at most 2^-(e+1) Mpc away).  Multiples of
 * 2^-22 Mpc are exact when that distance is at most 256 Mpc (box length at
 * most 512 Mpc); a wider field has e <= 21.  vol may be NULL (isolated
 * field). */
int rt3d_load_particles(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos,
                        const double *mass, const double *soft, int soft_per_particle,
                        const rt3d_volume *vol);

/* ---- grid path (Sec. 3.3 and App. B) --------------------------------------
 * The paper's own force path: the particle masses are assigned to a regular
 * node grid by cloud-in-cell, phi and grad phi are found on the nodes by a
 * zero-padded FFT convolution (no periodic images) with the kernels
 *   K_phi(d) = -mu_G (|d|^2 + soft^2)^(-1/2),  K_g(d) = mu_G d (|d|^2 + soft^2)^(-3/2)
 * (soft = 0: the d = 0 term is zero), and at every RK4 stage each ray reads
 * the field by App. B's interpolation: along x3 with the natural cubic spline
 * of the whole node line (second derivatives computed once at load), then
 * along x1 and x2 with natural cubic splines through the 2 n_int nodes
 * around the ray.  Outside the node range the field is zero.  Mass on nodes
 * outside the grid is dropped. */
typedef struct {
    int n;              /* nodes per side, 2 n_int .. 1024 */
    double lo[3];       /* position of node (0, 0, 0), comoving Mpc */
    double h;           /* node spacing, comoving Mpc (> 0) */
    int n_int;          /* interpolation nodes on either side, 1 .. 4 */
    int mean_subtract;  /* 1: subtract the mean node mass before the convolution */
} rt3d_grid_opts;

/* The grid force path of Sec. 3.3 and App. B (described above).
 * Build a gridded field in slot field_id from n particles (pos n*3, mass n,
 * one softening length soft for the kernels).  The library copies the
 * inputs; the grid's node table (per node the four values and their x3
 * spline second derivatives: 8 n^3 doubles in an RT3D_FP64 context, the same
 * rounded to 8 n^3 floats in an RT3D_MIXED context, which also interpolates in
 * FP32) stays on the device until the slot is reloaded or the context
 * destroyed.  The build (always FP64) needs (2n)^3 doubles, 8 n^3 doubles and
 * two (2n)^2 (n+1) complex FFT buffers of temporary device memory (a box
 * keeps four more, the kernels' spectra, where they fit in 8 GiB).  Traces,
 * rt3d_potential, rt3d_grid_nodes and rt3d_trace_batch cones on the slot then
 * use the grid (rt3d_grid_nodes of a mixed context returns the FP32 values);
 * rt3d_born rejects grid slots (RT3D_ENOTIMPL).  Errors: RT3D_EINVAL for a bad option or a
 * non-finite input, RT3D_ENOMEM, RT3D_ECUDA (including a cuFFT failure). */
int rt3d_load_grid(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos, const double *mass,
                   double soft, const rt3d_grid_opts *g);

/* Grid path for a replicated box (Sec. 5.2): each replica of the box (as in
 * rt3d_load_particles: rot[j] about the box centre, shift[j] with periodic
 * wrap, centred on the optical axis at x3 in [jL, (j+1)L)) is cut to the
 * prism |x1|, |x2| < W/2 around the optical axis, W = L / cubes, and the prism
 * into `cubes` cubes of side W along x3.  The particles of each cube (half-
 * open intervals; particles outside the prism are dropped) go on that cube's
 * own n^3 grid with nodes on its faces (spacing W / (n - 1)); with
 * g->mean_subtract the cube's mean node mass is removed; the cube's field
 * comes from its own mass only (zero-padded FFT).  A bundle reads the cube
 * holding its central ray's stage position (rt3d_potential: each point its
 * own cube); up to one node spacing beyond that cube's faces the end splines
 * are extrapolated (the other rays of a bundle that straddles a face),
 * further out the field is zero.  g->lo and g->h are not
 * used.  Positions must lie in [0, L).  Memory: one node table per cube (as
 * rt3d_load_grid: 8 n^3 doubles, or floats in a mixed context) stays on the
 * device.  Errors as rt3d_load_grid. */
int rt3d_load_grid_box(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos, const double *mass,
                       double soft, const rt3d_volume *vol, int cubes, const rt3d_grid_opts *g);

/* The node values of the grid of Sec. 3.3 (the field App. B interpolates).
 * Copy a grid slot's node values to out (host, 4 n^3 doubles, [f][i1][i2][i3]
 * with i3 fastest, f = phi, dphi/dx1, dphi/dx2, dphi/dx3; for a box grid,
 * n_replicas * cubes such blocks, replica-major). */
int rt3d_grid_nodes(rt3d_ctx *ctx, int field_id, double *out);

/* Trace n_bundles bundles with centres theta (n_bundles*2, tangent-plane
 * angles: direction (theta_x, theta_y, 1)) from the observer to the plane
 * x3 = chi(z_s), and fill out.  Each bundle is a central ray and a polygon of
 * b->n_ring rays of radius b->theta_r (Sec. 3.1); every ray integrates the
 * null geodesic equation (Eq. geodesiceqn, App. A symbols) by classical RK4
 * with fixed affine steps (Sec. 3.4, Eq. RKstepsize read as a node table) and
 * stops on the plane x3 = chi(z_s) (Sec. 5.1, Eq. raytracedistance) with
 * linear interpolation; the polygon's source positions give the lens-map
 * Jacobian (Eq. lensmap) and mu, kappa, gamma (Eq. magnification).  Errors:
 * RT3D_ENOCOSMO, RT3D_ENOFIELD, RT3D_EINVAL (z_s outside (0, 20], n_bundles
 * outside [1, 2^28], a non-finite theta, bad options), RT3D_ENOMEM,
 * RT3D_ECUDA.  Flags per bundle: RT3D_F_*. */
int rt3d_trace(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_bundles, const double *theta,
               const rt3d_bundle_opts *b, rt3d_bundle_result *out);

/* The trace of Sec. 3.1 / Sec. 3.4 as rt3d_trace, with device pointers,
 * enqueued on stream (a cudaStream_t; NULL = default stream) without host
 * synchronisation; the caller owns the device arrays.
 * d_theta: n_bundles*2; d_bundle_out: n_bundles*6 doubles
 * (mu, kappa, gamma1, gamma2, omega, flags as a double);
 * d_ray_out (optional): n_bundles*(1+n_ring)*8. */
int rt3d_trace_device(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_bundles,
                      const double *d_theta, const rt3d_bundle_opts *b, double *d_bundle_out,
                      double *d_ray_out);

/* The trace of Sec. 3.4 in pieces, with device pointers on a stream, for a
 * caller that wants to interleave its own work between RK4 stages or time them
 * (the trace itself is the same: rt3d_trace_device is begin + end).
 * rt3d_trace_begin enqueues the step table (Sec. 3.4, Eq. RKstepsize) and the
 * bundle initialiser (Sec. 3.1) and picks the pair-sum launch shape; d_theta
 * (n_bundles*2, device) must stay valid until rt3d_trace_end.
 * rt3d_trace_advance enqueues the next n_stages RK4 stages (4 per step: pair
 * sum of Eqs. psi / derivs, the Sec. 3.3 mean-density prism of mean-
 * subtracted boxes, the geodesic update of Eq. geodesiceqn); *stages_left
 * (may be NULL) receives the stages still to run, extra steps (max_extra)
 * included; stages past the end are no-ops.
 * rt3d_trace_end enqueues the remaining stages and the bundle reducer (Eq.
 * lensmap), writing d_bundle_out and d_ray_out as rt3d_trace_device.
 * One trace is open per context; its state lives in the context.
 * rt3d_trace_begin, rt3d_trace, rt3d_trace_device, rt3d_trace_batch,
 * rt3d_born, rt3d_schedule, and loading into the trace's field slot close it
 * (advance / end then return RT3D_EINVAL).  Enqueue every piece on one stream
 * (or streams ordered after it).  rt3d_get_stats counts from rt3d_trace_begin. */
int rt3d_trace_begin(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_bundles,
                     const double *d_theta, const rt3d_bundle_opts *b);
/* The next n_stages RK4 stages of the open trace (Sec. 3.4), as above. */
int rt3d_trace_advance(rt3d_ctx *ctx, void *stream, int n_stages, int *stages_left);
/* The rest of the open trace and its bundle reducer (Sec. 3.4, Eq. lensmap),
 * as above; the trace is closed. */
int rt3d_trace_end(rt3d_ctx *ctx, void *stream, double *d_bundle_out, double *d_ray_out);

/* Many lines of sight of Sec. 5 (each cone a mass distribution of Sec. 3.3
 * or 5.2 traced as in Sec. 3.4, with its own field, z_s, bundles and step
 * count) in one persistent launch recorded in a CUDA graph.  A cone's
 * field may be a particle field or a grid (isolated or cube-tiled box); all
 * cones share the bundle options b, each with its own n_steps.  An RT3D_FP64
 * context traces the cones one after another through rt3d_trace.
 * outs[i] receives cone i's results. */
int rt3d_trace_batch(rt3d_ctx *ctx, int n_cones, const rt3d_cone *cones,
                     const rt3d_bundle_opts *b, rt3d_bundle_result *outs);

/* ---- the multiple lens-plane comparison system (Sec. 3.1) ----------------
 * The paper's comparison method: the mass between observer and source is cut
 * into slabs along x3 -- each replica of a box into `slices` slabs of equal
 * thickness, the last one cut at the source plane x3 = chi(z_s); an isolated
 * field's x3 range into `slices` slabs -- and each slab is projected onto a
 * plane at its centre (Sec. 3.1 puts each box's plane at its centre as the
 * rule; slices = 1 is that).  A ray travels straight from
 * plane to plane and is deflected only at them, by the matter of that plane:
 * the thin-lens angle of Eq. defangleB of each projected Plummer particle,
 *   alpha_hat(x) = 4 G/c^2 (1 + z_k) sum_p m_p (x - x_p) / (|x - x_p|^2 + eps^2)
 * in comoving transverse coordinates, which makes the propagation the
 * multi-plane lens equation of Sec. 3.1 (flat universe); a mean-subtracted box
 * also removes the deflection of the slab's uniform mean surface density over
 * the replica's square cross-section.  Particles beyond the source plane are
 * left out.  The bundles (b->n_ring, theta_r, phase; the step options are not
 * used) and the least-squares Jacobian are those of rt3d_trace, so mu, kappa,
 * gamma and the muPDF of rt3d_histogram compare one to one with the 3D trace
 * (Sec. 5.4, Figs. RBMvsMudMag, RBMvsMudShear).  The pair sums are FP32 with
 * compensated accumulation (RT3D_MIXED) or FP64 (RT3D_FP64); the ray state,
 * deflection update and Jacobian are FP64.  out->ray_state (optional) holds
 * per ray (0, x1, x2, chi_s, 0, slope1, slope2, 1) at the source plane;
 * out->ray_steps (optional) is zeroed.  Errors: as rt3d_trace, plus
 * RT3D_ENOTIMPL for grid fields and RT3D_EINVAL for slices outside
 * [1, 4096] or more than 65536 planes. */
int rt3d_multiplane(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_bundles, const double *theta,
                    const rt3d_bundle_opts *b, int slices, rt3d_bundle_result *out);

/* The lens-plane system of Sec. 3.1 as rt3d_multiplane with device arrays
 * (d_theta n_bundles*2; d_bundle_out n_bundles*6 as rt3d_trace_device;
 * d_ray_out optional n_bundles*(1+n_ring)*8), enqueued on stream. */
int rt3d_multiplane_device(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_bundles,
                           const double *d_theta, const rt3d_bundle_opts *b, int slices, double *d_bundle_out,
                           double *d_ray_out);

/* muPDF of n magnifications (Eq. weighthisto): bins uniform in log10|mu|
 * (bin = floor((log10|mu| - log10 mu_min) / dl) in FP64), counts and
 * fixed-point weights round(2^32/|mu|); flagged (NOCROSS / NONFINITE) and
 * non-finite entries are excluded; flags may be NULL. */
int rt3d_histogram(rt3d_ctx *ctx, int64_t n, const double *mu, const int32_t *flags,
                   const rt3d_hist_opts *o, rt3d_hist *out);

/* The muPDF (Sec. 5.3, Eq. weighthisto) or shear PDF of the union of n_parts
 * disjoint sets of bundles -- the ranks of a run over several GPUs, each of
 * which binned its own bundles with the same bins and range -- from the
 * parts' histograms: counts and fixed-point weights add exactly, as do the
 * integer counters; the weighted mean is sum W_p mean_p / W and the weighted
 * spread comes from sum W_p (sigma_p^2 + (mean_p - mean)^2) / W (compensated
 * sums).  parts: n_parts histograms (host; counts, wfix of bins each); out:
 * caller-owned counts and wfix of bins, scalars written.  A host computation:
 * no device is touched, so it also runs where no GPU is present (ctx may be
 * NULL; then no error message is kept).  Errors: RT3D_EINVAL (null arrays,
 * n_parts or bins < 1, a negative or non-finite scalar). */
int rt3d_histogram_combine(rt3d_ctx *ctx, int n_parts, int bins, const rt3d_hist *parts, rt3d_hist *out);

/* Shear PDF (Sec. 5.4, Fig. RBMvsMudShear) of n bundles: bins uniform in
 * log10|gamma|, |gamma| = sqrt(gamma1^2 + gamma2^2), over [o->mu_min,
 * o->mu_max] read as the |gamma| range; every bundle keeps the source-plane
 * weight round(2^32/|mu|) of the muPDF; |gamma| = 0 counts as underflow; the
 * scalars are the 1/|mu|-weighted mean and spread of |gamma|.  Exclusions
 * as rt3d_histogram (and non-finite gamma).  The paper does not state its
 * shear-PDF weighting; this is the muPDF's. */
int rt3d_shear_histogram(rt3d_ctx *ctx, int64_t n, const double *mu, const double *gamma1,
                         const double *gamma2, const int32_t *flags, const rt3d_hist_opts *o,
                         rt3d_hist *out);

/* Born approximation (Sec. 6): convergence and shear of each line of sight
 * theta (n_bundles*2) from the Hessian of psi = phi / a along the unperturbed
 * ray x(chi) = (theta_x chi, theta_y chi, chi):
 *   kappa = int W (d11 + d22) psi,  gamma1 = int W (d11 - d22) psi,
 *   gamma2 = 2 int W d12 psi,  W = chi (chi_s - chi) / chi_s,
 * by the trapezoid rule over the node table of b (schedule, n_steps,
 * lens_chi, asinh_s; the other fields are not used) in its node variable;
 * a(chi) = 1 / (1 + z(chi)); boxes use the replica holding each node, minus
 * the mean-density prism.  out: n_bundles*3 (kappa, gamma1, gamma2), host.
 * The Hessian sums are FP32 with compensated accumulation, the rest FP64.
 * Particle fields only (grid fields: RT3D_ENOTIMPL). */
int rt3d_born(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_bundles, const double *theta,
              const rt3d_bundle_opts *b, double *out);

/* The pair sum of Eqs. psi / derivs (with the mean-density subtraction of
 * Sec. 3.3 when enabled): phi and grad phi (comoving) at n points: out = n*4 (phi, dphi/dx1, dphi/dx2, dphi/dx3).  rep: replica per
 * point (replicated fields; NULL = 0).  Uses the context's precision. */
int rt3d_potential(rt3d_ctx *ctx, int field_id, int64_t n, const double *pts, const int32_t *rep,
                   double *out);

/* Step table of a trace (Sec. 3.4, Eq. RKstepsize; chi_s of Sec. 5.1, Eq.
 * raytracedistance): chi_s = chi(z_s) and the n_steps affine-parameter steps
 * dlam (int of a^2 dchi between nodes on the unperturbed ray). */
int rt3d_schedule(rt3d_ctx *ctx, double z_s, int kind, int n_steps, double chi_l, double s,
                  double *dlam_out, double *chi_s_out);

/* muPDF (Sec. 5.3, Eq. weighthisto) of a device bundle-result array as
 * written by rt3d_trace_device
 * (n*6 doubles: mu at offset 0, flags at offset 5), enqueued on stream.
 * d_counts, d_wfix: device [bins] uint64; d_scalars: device 8 doubles
 * (n_used, n_under, n_over, n_neg, n_bad, W_total, mean_w, sigma_w). */
int rt3d_histogram_device(rt3d_ctx *ctx, void *stream, int64_t n, const double *d_bundle_out,
                          const rt3d_hist_opts *o, uint64_t *d_counts, uint64_t *d_wfix, double *d_scalars);

/* Watchdog self-test (the paper has no counterpart): one GPU thread runs the
 * bounded wait of the persistent kernel's grid barrier on a device word that
 * nothing changes.  The wait must give up after limit_s (0 < limit_s <= 10)
 * and report it, leaving the context usable: the call then returns
 * RT3D_ETIMEOUT, which is the passing outcome; RT3D_ECUDA if the wait ended
 * any other way. */
int rt3d_watchdog_selftest(rt3d_ctx *ctx, double limit_s);

/* ---- no-allocation variant ------------------------------------------------
 * rt3d_potential_device_noalloc: phi and grad phi of a loaded field at n
 * points, like rt3d_potential, but on device arrays and without allocating any
 * device memory during the call.  The paper has no counterpart to this entry
 * point; it exists for callers that cannot call cudaMalloc: a host process
 * whose device memory is already reserved in full by another framework's
 * pooling allocator (a new allocation would fail), or a loop that must not
 * pay the device-wide synchronisation that cudaMalloc and cudaFree can imply.
 *
 * Scratch: the split partial sums go to one static device array of
 * RT3D_NOALLOC_SCRATCH_BYTES (32 MiB), which every GPU that loads the library
 * holds until the process exits.  Limit: n <= RT3D_NOALLOC_SCRATCH_BYTES / 32
 * = 1048576 points per call (larger n returns RT3D_EINVAL); the number of
 * particle splits is reduced as needed to fit.  Every call shares that array
 * and it keeps the last call's contents; each entry a call reads is written
 * first by the same call, so nothing needs clearing.  Calls that overlap on
 * the GPU (two streams, two host threads) race on the array and give wrong
 * results: serialise them.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it; make that
 * first call before any stream capture begins.
 *
 * Arguments: ctx with field field_id loaded; stream = cudaStream_t (NULL =
 * default stream); d_pts = device n*3 doubles laid out as all x1, then all x2,
 * then all x3 (comoving Mpc, finite); d_rep = device n int32 replica indices
 * in [0, n_replicas) of the field (an isolated field has one, index 0) or
 * NULL (replica 0); d_out = device n*4 doubles (phi, dphi/dx1, dphi/dx2,
 * dphi/dx3 per point).  The call only enqueues work on stream, so the device
 * arrays are not checked on the host: a point whose replica index is out of
 * range or whose coordinates are not finite takes part in no pair sum and
 * gets NaN in all four outputs, and the other points are unaffected.  Points
 * are summed in blocks of consecutive indices, and a block makes one pass over
 * the particles for every replica its points use: group points by replica
 * (sorted rep) for the cost of one pass per point. */
#define RT3D_NOALLOC_SCRATCH_BYTES (32u << 20)
#define RT3D_NOALLOC_MAX_DEVICES 64
int rt3d_potential_device_noalloc(rt3d_ctx *ctx, void *stream, int field_id, int64_t n,
                                  const double *d_pts, const int32_t *d_rep, double *d_out);

/* Counters of the last trace or batch (the paper has no counterpart:
 * interactions and device time, for the throughput measurement). */
int rt3d_get_stats(rt3d_ctx *ctx, rt3d_stats *out);

/* Text of a status code (the paper has no counterpart). */
const char *rt3d_status_string(int status);
/* Message of the context's last failed call (the paper has no counterpart). */
const char *rt3d_last_error(rt3d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif

// multiplane.cu -- the multiple lens-plane comparison system (Sec. 3.1,
// "Multiple lens plane methods"; Eqs. defangleB, lenseqn, defangle).
//
// The mass between observer and source is cut into slabs along x3 (each
// replica of a box into `slices` slabs, the last one cut at the source plane;
// an isolated field's x3 range into `slices` slabs); every slab is projected
// onto a plane at its centre.  Rays travel straight between planes and are
// deflected only at them, by the matter of that plane:
//   alpha_hat(x) = 4 mu_G (1 + z_k) [ sum_p m_p (x - x_p) / (|x - x_p|^2 + eps^2)
//                                     - Sigma_bar R(x) ]
// in comoving transverse coordinates (the thin-lens angle of Eq. defangleB
// for a projected Plummer particle; for mean-subtracted boxes R is the
// deflection integral of the slab's uniform mean surface density over the
// replica's square cross-section).  theta -> theta - alpha_hat at a plane,
// x -> x + (chi_next - chi) theta between planes: the multi-plane lens
// equation of Sec. 3.1 in a flat universe.
//
// Per plane: k_mp_deflect2 (rings of 4 and 8, two bundles per thread in
// f32x2) or k_mp_deflect (other rings), the FP32 two-dimensional pair sum over
// the particles of the plane's slab (bundle-centric: the ring rays'
// separations expanded about the central ray's, compensated sums per chunk,
// partial sums per particle split), then k_mp_update in FP64 (split reduction, mean
// subtraction, deflection, propagation to the next plane).  The RT3D_FP64
// context runs k_mp_deflect64 (all FP64) instead.  The bundle reducer of the
// 3D trace fits the lens-map Jacobian at the source plane.
#include "force.cuh"
#include "trace_device.cuh"

namespace rt3d {

namespace {

constexpr int kMpNT = 128;     // bundles per block of the FP32 pair sum
constexpr int kMpChunk = 64;   // particles per compensated chunk
constexpr int kMpNT64 = 64;    // bundles per block of the FP64 pair sum

// one lens plane: position, 1 + z, slab [lo, hi) and its thickness, the next
// plane a ray travels to (or the source plane)
struct MPPlane {
    double chi, zp1, thick, lo, hi, next_chi;
    double a, b, d;  // the plane's replica / field spans [a, b); slab = floor((x3 - a) / d)
    int active, rep, slice, pad;
    long long qlo, qhi;  // grid z-coordinates (plane's frame) on the plane: [qlo, qhi]
};

// slab rule of a particle at world x3 against plane p, split in two
// predicates that are monotone in x3: below (x3 before the slab, or before
// the replica or the observer) and above (past the slab, the replica or the
// source).  A particle is on the plane when it is neither.
__device__ __forceinline__ double slab_index(const MPPlane &p, int slices, double x3)
{
    if (!(p.d > 0.0)) return 0.0;
    return fmin(floor((x3 - p.a) / p.d), (double)(slices - 1));
}
__device__ __forceinline__ bool slab_below(const MPPlane &p, int replicated, int slices, double x3)
{
    return x3 < 0.0 || (replicated && x3 < p.a) || slab_index(p, slices, x3) < (double)p.slice;
}
__device__ __forceinline__ bool slab_above(const MPPlane &p, int replicated, int slices, double x3, double chi_s)
{
    return x3 >= chi_s || (replicated && x3 >= p.b) || slab_index(p, slices, x3) > (double)p.slice;
}

// world x3 of grid z-coordinate gz in a frame whose origin has z = o2
__device__ __forceinline__ double grid_x3(long long gz, double delta, double o2) { return (double)gz * delta + o2; }

// The grid z-coordinates whose particles lie on plane p form one interval:
// x3 and the slab index never decrease as gz grows.  Both ends are found by
// bisection over the 32-bit coordinate range with the slab rule itself, so
// the pair sums test two integers per staged particle and select exactly the
// particles the rule selects.
__device__ void plane_q_range(MPPlane &p, int replicated, int slices, double chi_s, double delta, double o2)
{
    constexpr long long G0 = -2147483648LL, G1 = 2147483647LL;
    long long lo = G1 + 1, hi = G0 - 1;  // empty
    if (!slab_below(p, replicated, slices, grid_x3(G1, delta, o2))) {
        long long l = G0 - 1, h = G1;  // below(l) taken as true, below(h) false
        while (h - l > 1) {
            const long long m = l + (h - l) / 2;
            if (slab_below(p, replicated, slices, grid_x3(m, delta, o2))) l = m;
            else h = m;
        }
        lo = h;
    }
    if (!slab_above(p, replicated, slices, grid_x3(G0, delta, o2), chi_s)) {
        long long l = G0, h = G1 + 1;  // above(l) false, above(h) taken as true
        while (h - l > 1) {
            const long long m = l + (h - l) / 2;
            if (slab_above(p, replicated, slices, grid_x3(m, delta, o2), chi_s)) h = m;
            else l = m;
        }
        hi = l;
    }
    p.qlo = lo;
    p.qhi = hi;
}

// the plane table: chi_s in misc[0], the first plane's distance in misc[1]
__global__ void k_mp_table(Cosmo c, DevField f, double z_s, int slices, double a_iso, double b_iso, int n_pl,
                           MPPlane *pl, double *misc)
{
    __shared__ double s_chi;
    if (threadIdx.x == 0) {
        s_chi = comoving_distance(c, z_s);
        misc[0] = s_chi;
    }
    __syncthreads();
    const double chi_s = s_chi;
    const int replicated = f.replicated;
    const double L = f.L;
    for (int q = threadIdx.x; q < n_pl; q += blockDim.x) {
        const int j = q / slices, s = q % slices;
        double a, b;
        if (replicated) {
            a = (double)j * L;
            b = a + L;
        } else {
            a = a_iso;
            b = b_iso;
        }
        const double d = (b - a) / (double)slices;
        double lo = d > 0.0 ? a + d * (double)s : a, hi = d > 0.0 ? a + d * (double)(s + 1) : a;
        if (hi > chi_s) hi = chi_s;
        if (lo < 0.0) lo = 0.0;
        MPPlane p;
        p.lo = lo;
        p.hi = hi;
        p.thick = hi - lo;
        p.chi = 0.5 * (lo + hi);
        p.zp1 = 1.0 + redshift_at(c, p.chi);
        p.a = a;
        p.b = b;
        p.d = d;
        p.rep = j;
        p.slice = s;
        p.pad = 0;
        // an isolated field of one x3 (d = 0) has one plane; an empty slab of
        // an isolated field deflects nothing, so it may stay in the table
        p.active = (replicated || d > 0.0) ? (hi > lo) : (s == 0 && a >= 0.0 && a < chi_s);
        p.next_chi = chi_s;
        double o[3];
        frame_origin(f, replicated ? j : 0, o);
        plane_q_range(p, replicated, slices, chi_s, f.delta, o[2]);
        pl[q] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double next = chi_s;
        for (int q = n_pl - 1; q >= 0; --q) {
            pl[q].next_chi = next;
            if (pl[q].active) next = pl[q].chi;
        }
        misc[1] = next;  // the first plane a ray meets
    }
}

// ray state of the multi-plane trace: x1, x2 (comoving transverse position on
// the current plane) and t1, t2 (tangent-plane slopes), SoA FP64 in rs.y
__global__ void k_mp_init(TraceParams tp, const double *__restrict__ theta, RayState rs,
                          const double *__restrict__ misc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rs.n_rays) return;
    const int64_t b = i / rs.nr;
    const int k = (int)(i % rs.nr);
    double tx, ty;
    ray_theta(tp, theta, b, k, tx, ty);
    const double chi1 = misc[1];
    const int64_t n = rs.stride;
    rs.y[0 * n + i] = chi1 * tx;
    rs.y[1 * n + i] = chi1 * ty;
    rs.y[2 * n + i] = tx;
    rs.y[3 * n + i] = ty;
}

struct MPArgs {
    DevField f;
    const double *x;   // rs.y: x1 at [0, n_rays), x2 at [n_rays, 2 n_rays)
    int64_t n_b, n_rays;
    const MPPlane *pl;
    int q, slices;
    const double *misc;
    int64_t per_split;
    void *out;         // partials [split][output][bundle]
    unsigned long long *count;  // particles on the planes (interactions = rays x count)
};

// FP32 two-dimensional pair sum of one plane, one bundle per thread.
// d_c = r_c - p (central ray minus particle), e_k = r_k - r_c (FP64
// difference, rounded once), so d_k = d_c + e_k and
//   |d_k|^2 + eps^2 = (|d_c|^2 + eps^2) + (2 e_k . d_c + |e_k|^2),
//   sum w_k d_k = sum w_k d_c + e_k sum w_k,   w_k = m / (|d_k|^2 + eps^2).
// Outputs per bundle: (G_c x, G_c y), then per ring ray (G_k x, G_k y, S_k),
// each a compensated FP32 (hi, lo) pair; the update adds e_k S_k in FP64.
template <int NRING, bool REPL, bool PEPS, bool UMASS>
__global__ void __launch_bounds__(kMpNT) k_mp_deflect(MPArgs A)
{
    constexpr int NR = NRING + 1;
    constexpr int NQ = 2 + 3 * NRING;
    const MPPlane P = A.pl[A.q];
    if (!P.active) return;
    __shared__ float4 s_p[kTile];
    __shared__ float2 s_hl[NQ * kMpNT];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.x * kMpNT, b = b0 + tid;
    const bool valid = b < A.n_b;
    const int64_t n = A.n_rays;
    unsigned n_on = 0;  // staged particles on the plane (block column 0 counts)
    double o[3];
    frame_origin(f, REPL ? P.rep : 0, o);
    const int64_t ia = b0 * NR;  // anchor: the block's first central ray
    const long long ax = anchor_q(A.x[ia], o[0], f.inv_delta);
    const long long ay = anchor_q(A.x[n + ia], o[1], f.inv_delta);
    // central ray relative to the anchor, ring offsets e_k (2 e_k and |e_k|^2)
    float rcx = 0.f, rcy = 0.f;
    float ex2[NRING], ey2[NRING], ee[NRING];
#pragma unroll
    for (int k = 0; k < NRING; ++k) ex2[k] = ey2[k] = ee[k] = 0.f;
    if (valid) {
        const int64_t ic = b * NR;
        rcx = (float)(((A.x[ic] - o[0]) * f.inv_delta - (double)ax) * f.delta);
        rcy = (float)(((A.x[n + ic] - o[1]) * f.inv_delta - (double)ay) * f.delta);
#pragma unroll
        for (int k = 0; k < NRING; ++k) {
            const float ex = (float)(A.x[ic + 1 + k] - A.x[ic]), ey = (float)(A.x[n + ic + 1 + k] - A.x[n + ic]);
            ex2[k] = 2.f * ex;
            ey2[k] = 2.f * ey;
            ee[k] = fmaf(ex, ex, ey * ey);
        }
    } else {
        rcx = rcy = 1e30f;  // far sentinel: contributions vanish
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) s_hl[q * kMpNT + tid] = make_float2(0.f, 0.f);
    const int64_t p0 = (int64_t)blockIdx.y * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    const float dlt = (float)f.delta;
    for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
        __syncthreads();
        for (int qq = tid; qq < kTile; qq += kMpNT) {
            const int64_t pi = t0 + qq;
            float4 v = make_float4(1e18f, 1e18f, 0.f, 0.f);
            if (pi < p1) {
                const int4 pr = f.part[pi];
                long long g[3] = {pr.x, pr.y, pr.z};
                if (REPL) replica_q(f, P.rep, pr.x, pr.y, pr.z, g);
                if (g[2] >= P.qlo && g[2] <= P.qhi) {
                    ++n_on;
                    v.x = (float)(g[0] - ax) * dlt;
                    v.y = (float)(g[1] - ay) * dlt;
                    v.z = __int_as_float(pr.w);
                    v.w = PEPS ? f.eps2[pi] : f.eps2u;
                }
            }
            s_p[qq] = v;
        }
        __syncthreads();
        for (int c0 = 0; c0 < kTile; c0 += kMpChunk) {
            float cx = 0.f, cy = 0.f, gx[NRING], gy[NRING], gs[NRING];
#pragma unroll
            for (int k = 0; k < NRING; ++k) gx[k] = gy[k] = gs[k] = 0.f;
#pragma unroll 2
            for (int jj = c0; jj < c0 + kMpChunk; ++jj) {
                const float4 p = s_p[jj];
                const float dx = rcx - p.x, dy = rcy - p.y;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, p.w));
                float w;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(w) : "f"(r2));
                if (!UMASS) w *= p.z;
                cx = fmaf(dx, w, cx);
                cy = fmaf(dy, w, cy);
#pragma unroll
                for (int k = 0; k < NRING; ++k) {
                    const float s2 = r2 + fmaf(ex2[k], dx, fmaf(ey2[k], dy, ee[k]));
                    float wk;
                    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(wk) : "f"(s2));
                    if (!UMASS) wk *= p.z;
                    gs[k] += wk;
                    gx[k] = fmaf(dx, wk, gx[k]);
                    gy[k] = fmaf(dy, wk, gy[k]);
                }
            }
            // merge the chunk into the (hi, lo) sums: TwoSum on hi, errors into lo
            float v[NQ];
            v[0] = cx;
            v[1] = cy;
#pragma unroll
            for (int k = 0; k < NRING; ++k) {
                v[2 + 3 * k] = gx[k];
                v[3 + 3 * k] = gy[k];
                v[4 + 3 * k] = gs[k];
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float2 h = s_hl[q * kMpNT + tid];
                two_sum_into(h.x, h.y, v[q]);
                s_hl[q * kMpNT + tid] = h;
            }
        }
    }
    if (blockIdx.x == 0 && n_on) atomicAdd(A.count, (unsigned long long)n_on);
    if (!valid) return;
    float2 *out = (float2 *)A.out;
    const int64_t sn = (int64_t)blockIdx.y * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[(sn + q) * A.n_b + b] = s_hl[q * kMpNT + tid];
}

// The same sums with two bundles per thread (rings of 4 and 8): bundles A =
// b0 + tid and B = b0 + NT + tid form f32x2 pairs ray by ray, so every FP32
// operation is one f32x2 instruction.  Particles are staged negated and
// duplicated, (-x, -x, -y, -y) and (m, m, eps^2, eps^2), so that d = r - p is
// one f32x2 add; a uniform-mass field skips the mass product (the update
// applies it).  Per particle and bundle pair: 6 + 6 NRING f32x2 operations and
// 2 (1 + NRING) reciprocals.  Same outputs and layout as k_mp_deflect.
constexpr int kMp2NT = 64;

// (rings of 4 bounded for 8 blocks per SM, 128 registers; rings of 8, whose
// accumulators need more, for 4)
template <int NRING, bool REPL, bool PEPS, bool UMASS>
__global__ void __launch_bounds__(kMp2NT, NRING <= 4 ? 8 : 4) k_mp_deflect2(MPArgs A)
{
    constexpr int NR = NRING + 1;
    constexpr int NQ = 2 + 3 * NRING;
    const MPPlane P = A.pl[A.q];
    if (!P.active) return;
    __shared__ float4 s_a[kTile + 1];  // + 1: the particle loop reads one record ahead
    __shared__ float4 s_b[kTile + 1];
    __shared__ float2 s_hl[2 * NQ * kMp2NT];  // (hi, lo) of output q for the pair (A, B)
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.x * 2 * kMp2NT;
    const int64_t bb[2] = {b0 + tid, b0 + kMp2NT + tid};
    const bool valid[2] = {bb[0] < A.n_b, bb[1] < A.n_b};
    const int64_t n = A.n_rays;
    unsigned n_on = 0;  // staged particles on the plane (block column 0 counts)
    double o[3];
    frame_origin(f, REPL ? P.rep : 0, o);
    const int64_t ia = b0 * NR;  // anchor: the block's first central ray
    const long long ax = anchor_q(A.x[ia], o[0], f.inv_delta);
    const long long ay = anchor_q(A.x[n + ia], o[1], f.inv_delta);
    float rc[2][2], e2[2][NRING][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        rc[h][0] = rc[h][1] = 1e30f;  // far sentinel: contributions vanish
#pragma unroll
        for (int k = 0; k < NRING; ++k) e2[h][k][0] = e2[h][k][1] = e2[h][k][2] = 0.f;
        if (valid[h]) {
            const int64_t ic = bb[h] * NR;
            rc[h][0] = (float)(((A.x[ic] - o[0]) * f.inv_delta - (double)ax) * f.delta);
            rc[h][1] = (float)(((A.x[n + ic] - o[1]) * f.inv_delta - (double)ay) * f.delta);
#pragma unroll
            for (int k = 0; k < NRING; ++k) {
                const float ex = (float)(A.x[ic + 1 + k] - A.x[ic]), ey = (float)(A.x[n + ic + 1 + k] - A.x[n + ic]);
                e2[h][k][0] = 2.f * ex;
                e2[h][k][1] = 2.f * ey;
                e2[h][k][2] = fmaf(ex, ex, ey * ey);
            }
        }
    }
    const float2 RX = make_float2(rc[0][0], rc[1][0]), RY = make_float2(rc[0][1], rc[1][1]);
    float2 EX2[NRING], EY2[NRING], EE[NRING];
#pragma unroll
    for (int k = 0; k < NRING; ++k) {
        EX2[k] = make_float2(e2[0][k][0], e2[1][k][0]);
        EY2[k] = make_float2(e2[0][k][1], e2[1][k][1]);
        EE[k] = make_float2(e2[0][k][2], e2[1][k][2]);
    }
    float2 *s_hi = s_hl, *s_lo = s_hl + NQ * kMp2NT;
#pragma unroll
    for (int q = 0; q < NQ; ++q) s_hi[q * kMp2NT + tid] = s_lo[q * kMp2NT + tid] = make_float2(0.f, 0.f);
    const int64_t p0 = (int64_t)blockIdx.y * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    const float dlt = (float)f.delta;
    for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
        __syncthreads();
        for (int qq = tid; qq < kTile; qq += kMp2NT) {
            const int64_t pi = t0 + qq;
            float x = -1e18f, y = -1e18f, m = 0.f, e = 0.f;
            if (pi < p1) {
                const int4 pr = f.part[pi];
                long long g[3] = {pr.x, pr.y, pr.z};
                if (REPL) replica_q(f, P.rep, pr.x, pr.y, pr.z, g);
                if (g[2] >= P.qlo && g[2] <= P.qhi) {
                    ++n_on;
                    x = -(float)(g[0] - ax) * dlt;
                    y = -(float)(g[1] - ay) * dlt;
                    m = __int_as_float(pr.w);
                    e = PEPS ? f.eps2[pi] : f.eps2u;
                }
            }
            s_a[qq] = make_float4(x, x, y, y);
            s_b[qq] = make_float4(m, m, e, e);
        }
        __syncthreads();
        float2 cx = make_float2(0.f, 0.f), cy = cx, gx[NRING], gy[NRING], gs[NRING];
#pragma unroll
        for (int k = 0; k < NRING; ++k) gx[k] = gy[k] = gs[k] = make_float2(0.f, 0.f);
        // the next particle's records are read one iteration ahead (s_a and s_b
        // hold kTile + 1 records), so the shared-memory latency overlaps the
        // current particle's arithmetic
        float4 a_nx = s_a[0], b_nx = s_b[0];
#pragma unroll 1
        for (int jj = 0; jj < kTile; ++jj) {
            const float4 a = a_nx;
            const float4 b = b_nx;
            a_nx = s_a[jj + 1];
            b_nx = s_b[jj + 1];
            const float2 DX = __fadd2_rn(RX, make_float2(a.x, a.y));
            const float2 DY = __fadd2_rn(RY, make_float2(a.z, a.w));
            const float2 R2 = __ffma2_rn(DX, DX, __ffma2_rn(DY, DY, make_float2(b.z, b.w)));
            float2 w;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(w.x) : "f"(R2.x));
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(w.y) : "f"(R2.y));
            if (!UMASS) w = __fmul2_rn(w, make_float2(b.x, b.y));
            cx = __ffma2_rn(DX, w, cx);
            cy = __ffma2_rn(DY, w, cy);
#pragma unroll
            for (int k = 0; k < NRING; ++k) {
                const float2 s2 = __fadd2_rn(R2, __ffma2_rn(EX2[k], DX, __ffma2_rn(EY2[k], DY, EE[k])));
                float2 wk;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(wk.x) : "f"(s2.x));
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(wk.y) : "f"(s2.y));
                if (!UMASS) wk = __fmul2_rn(wk, make_float2(b.x, b.y));
                gs[k] = __fadd2_rn(gs[k], wk);
                gx[k] = __ffma2_rn(DX, wk, gx[k]);
                gy[k] = __ffma2_rn(DY, wk, gy[k]);
            }
        }
        // merge the tile into the (hi, lo) sums of both bundles
        float2 v[NQ];
        v[0] = cx;
        v[1] = cy;
#pragma unroll
        for (int k = 0; k < NRING; ++k) {
            v[2 + 3 * k] = gx[k];
            v[3 + 3 * k] = gy[k];
            v[4 + 3 * k] = gs[k];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 hi = s_hi[q * kMp2NT + tid], lo = s_lo[q * kMp2NT + tid];
            two_sum2_into(hi, lo, v[q]);
            s_hi[q * kMp2NT + tid] = hi;
            s_lo[q * kMp2NT + tid] = lo;
        }
    }
    if (blockIdx.x == 0 && n_on) atomicAdd(A.count, (unsigned long long)n_on);
    float2 *out = (float2 *)A.out;
    const int64_t sn = (int64_t)blockIdx.y * NQ;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!valid[h]) continue;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float2 hi = s_hi[q * kMp2NT + tid], lo = s_lo[q * kMp2NT + tid];
            out[(sn + q) * A.n_b + bb[h]] = h ? make_float2(hi.y, lo.y) : make_float2(hi.x, lo.x);
        }
    }
}

// the all-FP64 twin: plain FP64 sums, every ray on its own (outputs per ray:
// sum w d, two components), for the RT3D_FP64 context
template <int NRING, bool REPL, bool PEPS>
__global__ void __launch_bounds__(kMpNT64) k_mp_deflect64(MPArgs A)
{
    constexpr int NR = NRING + 1;
    const MPPlane P = A.pl[A.q];
    if (!P.active) return;
    __shared__ double4_16a s_p[kTile64];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t b = (int64_t)blockIdx.x * kMpNT64 + tid;
    const bool valid = b < A.n_b;
    const int64_t n = A.n_rays;
    unsigned n_on = 0;  // staged particles on the plane (block column 0 counts)
    double o[3];
    frame_origin(f, REPL ? P.rep : 0, o);
    double rx[NR], ry[NR], sx[NR], sy[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        rx[k] = valid ? A.x[b * NR + k] - o[0] : 1e150;
        ry[k] = valid ? A.x[n + b * NR + k] - o[1] : 1e150;
        sx[k] = sy[k] = 0.0;
    }
    const int64_t p0 = (int64_t)blockIdx.y * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    for (int64_t t0 = p0; t0 < p1; t0 += kTile64) {
        __syncthreads();
        for (int qq = tid; qq < kTile64; qq += kMpNT64) {
            const int64_t pi = t0 + qq;
            double4_16a v = make_double4_16a(1e100, 1e100, 0.0, 0.0);
            if (pi < p1) {
                const int4 pr = f.part[pi];
                long long g[3] = {pr.x, pr.y, pr.z};
                if (REPL) replica_q(f, P.rep, pr.x, pr.y, pr.z, g);
                if (g[2] >= P.qlo && g[2] <= P.qhi) {
                    ++n_on;
                    v = make_double4_16a((double)g[0] * f.delta, (double)g[1] * f.delta, f.m64[pi],
                                         PEPS ? f.eps2_64[pi] : f.eps2u64);
                }
            }
            s_p[qq] = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int jj = 0; jj < kTile64; ++jj) {
            const double4_16a p = s_p[jj];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const double dx = rx[k] - p.x, dy = ry[k] - p.y;
                const double w = p.z / (dx * dx + dy * dy + p.w);
                sx[k] += w * dx;
                sy[k] += w * dy;
            }
        }
    }
    if (blockIdx.x == 0 && n_on) atomicAdd(A.count, (unsigned long long)n_on);
    if (!valid) return;
    double *out = (double *)A.out;
    const int64_t sn = (int64_t)blockIdx.y * 2;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        out[(sn + 0) * n + b * NR + k] = sx[k];
        out[(sn + 1) * n + b * NR + k] = sy[k];
    }
}

// deflection integral of a uniform unit surface density over the square
// |x1|, |x2| < h (corner sum of g(u, v) = u atan(v/u) + (v/2) ln(u^2 + v^2))
__device__ __forceinline__ double mp_g(double u, double v)
{
    const double q = u * u + v * v;
    if (q == 0.0) return 0.0;
    return (u != 0.0 ? u * atan(v / u) : 0.0) + 0.5 * v * log(q);
}

__device__ __forceinline__ void mp_rect(double h, double x, double y, double r[2])
{
    const double u1 = x + h, u0 = x - h, v1 = y + h, v0 = y - h;
    r[0] = mp_g(u1, v1) - mp_g(u0, v1) - mp_g(u1, v0) + mp_g(u0, v0);
    r[1] = mp_g(v1, u1) - mp_g(v1, u0) - mp_g(v0, u1) + mp_g(v0, u0);
}

// FP64 update of one ray at plane q: the deflection from the split sums (and
// the slab's mean surface density), then the straight path to the next plane
template <int NRING>
__global__ void k_mp_update(MPArgs A, int S, int fp64, double mfac, double rho_term, double half_L, RayState rs)
{
    constexpr int NR = NRING + 1;
    constexpr int NQ = 2 + 3 * NRING;
    const MPPlane P = A.pl[A.q];
    if (!P.active) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rs.n_rays) return;
    const int64_t n = rs.stride;
    const int64_t b = i / NR;
    const int k = (int)(i % NR);
    const double x = rs.y[i], y = rs.y[n + i];
    double ax, ay;
    if (fp64) {
        const double *pd = (const double *)A.out;
        ax = ay = 0.0;
        for (int s = 0; s < S; ++s) {
            ax += pd[(2 * (int64_t)s + 0) * n + i];
            ay += pd[(2 * (int64_t)s + 1) * n + i];
        }
    } else {
        // (hi, lo) FP32 pairs added as double-float numbers, converted once
        const float2 *pm = (const float2 *)A.out;
        const int q0 = k == 0 ? 0 : 2 + 3 * (k - 1);
        const int nq = k == 0 ? 2 : 3;
        float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
        for (int s = 0; s < S; ++s)
            for (int c = 0; c < nq; ++c) {
                const float2 v = pm[((int64_t)s * NQ + q0 + c) * A.n_b + b];
                const float t = hi[c] + v.x;
                const float bb = t - hi[c];
                lo[c] += ((hi[c] - (t - bb)) + (v.x - bb)) + v.y;
                hi[c] = t;
            }
        ax = (double)hi[0] + (double)lo[0];
        ay = (double)hi[1] + (double)lo[1];
        if (k > 0) {  // + e_k S_k with the FP32 offsets the pair sum used
            const int64_t ic = b * NR;
            const float ex = (float)(x - rs.y[ic]), ey = (float)(y - rs.y[n + ic]);
            const double Sk = (double)hi[2] + (double)lo[2];
            ax += (double)ex * Sk;
            ay += (double)ey * Sk;
        }
    }
    const double sc = A.f.mscale_inv * mfac;  // stored masses are mu_G m 2^ms
    ax *= sc;
    ay *= sc;
    if (rho_term > 0.0) {
        double r[2];
        mp_rect(half_L, x, y, r);
        ax -= rho_term * P.thick * r[0];
        ay -= rho_term * P.thick * r[1];
    }
    const double g = 4.0 * P.zp1;
    const double tx = rs.y[2 * n + i] - g * ax, ty = rs.y[3 * n + i] - g * ay;
    const double dc = P.next_chi - P.chi;
    rs.y[2 * n + i] = tx;
    rs.y[3 * n + i] = ty;
    rs.y[i] = x + dc * tx;
    rs.y[n + i] = y + dc * ty;
}

// final state at the source plane in the trace's layout, for the reducer
__global__ void k_mp_finish(RayState rs, const double *__restrict__ misc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rs.n_rays) return;
    const int64_t n = rs.stride;
    const double v[8] = {0.0, rs.y[i], rs.y[n + i], misc[0], 0.0, rs.y[2 * n + i], rs.y[3 * n + i], 1.0};
#pragma unroll
    for (int q = 0; q < 8; ++q) rs.fin[q * n + i] = v[q];
    rs.done[i] = 1;
}

template <int NRING, bool REPL, bool PEPS, bool UMASS>
cudaError_t go_deflect(const MPArgs &A, int S, bool fp64, cudaStream_t st)
{
    if (fp64) {
        dim3 grid((unsigned)((A.n_b + kMpNT64 - 1) / kMpNT64), (unsigned)S);
        k_mp_deflect64<NRING, REPL, PEPS><<<grid, kMpNT64, 0, st>>>(A);
    } else {
        if constexpr (NRING == 4 || NRING == 8) {  // two bundles per thread, f32x2
            dim3 grid((unsigned)((A.n_b + 2 * kMp2NT - 1) / (2 * kMp2NT)), (unsigned)S);
            k_mp_deflect2<NRING, REPL, PEPS, UMASS><<<grid, kMp2NT, 0, st>>>(A);
        } else {
            dim3 grid((unsigned)((A.n_b + kMpNT - 1) / kMpNT), (unsigned)S);
            k_mp_deflect<NRING, REPL, PEPS, UMASS><<<grid, kMpNT, 0, st>>>(A);
        }
    }
    return cudaGetLastError();
}

template <int NRING>
cudaError_t deflect_ring(const MPArgs &A, int S, bool fp64, bool umass, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = fp64 ? A.f.eps2_64 != nullptr : A.f.eps2 != nullptr;
    if (repl) {
        if (peps) return umass ? go_deflect<NRING, true, true, true>(A, S, fp64, st)
                               : go_deflect<NRING, true, true, false>(A, S, fp64, st);
        return umass ? go_deflect<NRING, true, false, true>(A, S, fp64, st)
                     : go_deflect<NRING, true, false, false>(A, S, fp64, st);
    }
    if (peps) return umass ? go_deflect<NRING, false, true, true>(A, S, fp64, st)
                           : go_deflect<NRING, false, true, false>(A, S, fp64, st);
    return umass ? go_deflect<NRING, false, false, true>(A, S, fp64, st)
                 : go_deflect<NRING, false, false, false>(A, S, fp64, st);
}

template <int NRING>
cudaError_t plane_pass(const MPArgs &A, int S, bool fp64, bool umass, double rho_term, double half_L, RayState rs,
                       cudaStream_t st)
{
    cudaError_t e = deflect_ring<NRING>(A, S, fp64, umass, st);
    if (e != cudaSuccess) return e;
    const double mfac = (umass && !fp64) ? A.f.m_uniform : 1.0;
    k_mp_update<NRING><<<(unsigned)((rs.n_rays + 255) / 256), 256, 0, st>>>(A, S, fp64 ? 1 : 0, mfac, rho_term,
                                                                            half_L, rs);
    return cudaGetLastError();
}

}  // namespace

size_t mp_plane_bytes() { return sizeof(MPPlane); }

size_t mp_partials_bytes(int n_ring, int64_t n_b, int splits, bool fp64)
{
    return fp64 ? (size_t)splits * 2 * (size_t)(n_b * (1 + n_ring)) * sizeof(double)
                : (size_t)splits * (size_t)(2 + 3 * n_ring) * (size_t)n_b * sizeof(float2);
}

// the whole multi-plane trace of n_b bundles on stream st (tables, initial
// rays, one deflection pass and update per plane, final state, reducer)
cudaError_t mp_run(const Cosmo &c, const DevField &f, double z_s, int slices, double x3_lo, double x3_hi,
                   const TraceParams &tp, const double *d_theta, RayState rs, void *d_planes, int n_pl, void *partials,
                   int splits, bool fp64, bool umass, double *misc, unsigned long long *count, double *d_bout,
                   double *d_rout, cudaStream_t st)
{
    MPPlane *pl = (MPPlane *)d_planes;
    k_mp_table<<<1, 256, 0, st>>>(c, f, z_s, slices, x3_lo, x3_hi, n_pl, pl, misc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned rb = (unsigned)((rs.n_rays + 255) / 256);
    k_mp_init<<<rb, 256, 0, st>>>(tp, d_theta, rs, misc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    MPArgs A;
    A.f = f;
    A.x = rs.y;
    A.n_b = rs.n_b;
    A.n_rays = rs.n_rays;
    A.pl = pl;
    A.slices = slices;
    A.misc = misc;
    const int64_t tiles = std::max<int64_t>(1, (f.n + kTile - 1) / kTile);
    const int64_t tps = (tiles + splits - 1) / splits;
    A.per_split = tps * kTile;
    const int S = (int)((tiles + tps - 1) / tps);
    A.out = partials;
    A.count = count;
    if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    const double rho_term = (f.replicated && f.mean_subtract) ? f.rho_term : 0.0;
    for (int q = 0; q < n_pl; ++q) {
        A.q = q;
        switch (tp.n_ring) {
        case 3: e = plane_pass<3>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        case 4: e = plane_pass<4>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        case 5: e = plane_pass<5>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        case 6: e = plane_pass<6>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        case 7: e = plane_pass<7>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        case 8: e = plane_pass<8>(A, S, fp64, umass, rho_term, 0.5 * f.L, rs, st); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    k_mp_finish<<<rb, 256, 0, st>>>(rs, misc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_reduce(tp, d_theta, rs, misc, d_bout, d_rout, st);
}

}  // namespace rt3d

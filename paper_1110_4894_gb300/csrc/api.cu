// api.cu -- the C ABI (include/rt3d.h): context, particle staging, trace
// orchestration, histogram, potential and schedule entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "batch_layout.cuh"
#include "force.cuh"
#include "rt3d_internal.cuh"

namespace rt3d {
cudaError_t dispatch_mixed(const ForceArgs &A, const ForceShape &sh, cudaStream_t st);
cudaError_t dispatch_fp64(const ForceArgs &A, const ForceShape &sh, cudaStream_t st);
cudaError_t dispatch_packed(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st);
cudaError_t dispatch_bundle(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st);
cudaError_t dispatch_bundle2(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st);
cudaError_t dispatch_bundle2x(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st,
                              int *occ = nullptr);
struct BatchArgs;

// rays covered by one block of the pair-sum kernel of shape sh
inline int64_t rays_per_block(const ForceShape &sh)
{
    return (int64_t)sh.R * sh.NT * ((sh.variant == 4 || sh.variant == 5) ? 2 : 1);
}

// ---------------------------------------------------------------------------
// particle staging (S2): FP64 input -> integer grid + scaled masses
// ---------------------------------------------------------------------------
// One block: bounding box, largest and total mass (Kahan), in a fixed order.
__global__ void __launch_bounds__(1024) k_field_stats(int64_t n, const double *__restrict__ pos,
                                                      const double *__restrict__ mass, double *out)
{
    __shared__ double s[8][1024];
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300}, mm = 0.0, sum = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], pos[3 * i + d]);
            mx[d] = fmax(mx[d], pos[3 * i + d]);
        }
        mm = fmax(mm, mass[i]);
        const double y = mass[i] - c, t = sum + y;
        c = (t - sum) - y;
        sum = t;
    }
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    s[6][threadIdx.x] = mm;
    s[7][threadIdx.x] = sum;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + h]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + h]);
            }
            s[6][threadIdx.x] = fmax(s[6][threadIdx.x], s[6][threadIdx.x + h]);
            s[7][threadIdx.x] += s[7][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) out[threadIdx.x] = s[threadIdx.x][0];
}

// grid position q = round((p - O) 2^e) (isolated) or round(p 2^e) mod Lq
// (replicated box); mass mu_G m 2^ms in FP32 bits and FP64; eps^2 in grid units
__global__ void k_stage_particles(int64_t n, const double *__restrict__ pos, const double *__restrict__ mass,
                                  const double *__restrict__ soft, int soft_pp, double soft0, int replicated,
                                  long long Lq, double O0, double O1, double O2, double two_e, double mscale,
                                  int4 *part, double *m64, float *eps2, double *eps2_64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double O[3] = {O0, O1, O2};
    int q[3];
    for (int d = 0; d < 3; ++d) {
        long long v = __double2ll_rn((pos[3 * i + d] - O[d]) * two_e);
        if (replicated) {
            v %= Lq;
            if (v < 0) v += Lq;
        }
        q[d] = (int)v;
    }
    const double m = kMuG * mass[i] * mscale;
    part[i] = make_int4(q[0], q[1], q[2], __float_as_int((float)m));
    m64[i] = m;
    if (soft_pp) {  // Plummer softening squared, Mpc^2
        const double e = soft[i];
        eps2[i] = (float)(e * e);
        eps2_64[i] = e * e;
    }
    (void)soft0;
}

int force_max_splits(const ForceShape &, int64_t n_particles)
{
    const int64_t t = (n_particles + kTile - 1) / kTile;
    return (int)std::max<int64_t>(1, std::min<int64_t>(t, 65535));
}

size_t partials_bytes(const ForceShape &sh, int64_t n_rays, bool)
{
    return (size_t)sh.splits * 4 * (size_t)n_rays * 8;
}

}  // namespace rt3d

using namespace rt3d;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct FieldSlot {
    bool loaded = false;
    DevField df{};
    int4 *d_part = nullptr;
    float *d_eps2 = nullptr;
    double *d_m64 = nullptr, *d_eps2_64 = nullptr;
    int *d_rot = nullptr, *d_shift = nullptr;
    int64_t n = 0;
    bool is_grid = false;  // grid path: phi and grad phi interpolated from nodes
    GridDev gd;
    double x3_lo = 0.0, x3_hi = 0.0;  // x3 range of an isolated field's particles (lens planes)
};

// A trace open on the context: the ray state lives in the context's scratch
// between rt3d_trace_begin and rt3d_trace_end, so one trace is open at a time.
struct OpenTrace {
    bool open = false;
    const FieldSlot *fs = nullptr;
    const double *d_theta = nullptr;
    int64_t n_b = 0;
    rt3d_bundle_opts b{};
    TraceParams tp{};
    ForceShape sh{};
    RayState rs{};
    bool fp64 = false, use_prism = false, timed = false;
    int next = 0, total = 0;  // next global stage (4 per RK4 step) and their count
    int64_t launches = 0, flaunch = 0;
};

struct rt3d_ctx {
    int device = 0;
    int n_sm = 152;  // streaming multiprocessors of the device (queried at create)
    rt3d_options opt{};
    std::string err;
    bool have_cosmo = false;
    Cosmo cosmo{};
    std::vector<FieldSlot> fields;
    Scratch scr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    rt3d_stats stats{};
    double last_npart = 0.0;
    bool stats_pending = false;
    std::vector<cudaEvent_t> tev;  // per-launch timing events
    int tev_used = 0;
    double *atab = nullptr;  // a(t) table of the cosmology (device)
    size_t atab_n = 0;
    unsigned long long *d_hist_u64 = nullptr;  // bins*2 + 5
    double *d_hist_f64 = nullptr;              // 8
    int hist_cap = 0;
    double *d_io = nullptr;                    // staging for potential / histogram inputs
    size_t d_io_n = 0;
    OpenTrace trace;  // the trace between rt3d_trace_begin and rt3d_trace_end
    // launch shapes chosen by the autotuner, per size class
    std::map<std::tuple<int, int, int, int, int, int>, ForceShape> tuned;
    // batched trace: device scratch, the captured graph and its key
    struct Batch {
        void *cones = nullptr;
        size_t cones_n = 0;
        int4 *items = nullptr;
        size_t items_n = 0;
        int *rb2cone = nullptr;
        size_t rb_n = 0;
        double *state = nullptr;
        size_t state_n = 0;
        int *ints = nullptr;
        size_t ints_n = 0;
        double *theta = nullptr;
        size_t theta_n = 0;
        double *dlam = nullptr;
        size_t dlam_n = 0;
        float2 *partials = nullptr;
        size_t partials_n = 0;
        unsigned long long *cnt = nullptr;
        size_t cnt_n = 0;
        unsigned *bar = nullptr;  // [0] count, [1] generation, [2] error word, [4], [5] work queues
        double *bout = nullptr;
        size_t bout_n = 0;
        double *rout = nullptr;
        size_t rout_n = 0;
        double *prism = nullptr;
        size_t prism_n = 0;
        cudaGraphExec_t exec = nullptr;
        std::vector<long long> key;
        // (cones, log2 rays, log2 pairs) -> (NT, particles per item, kernel mode)
        std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> tuned;
    } batch;
};

static int fail(rt3d_ctx *c, int code, const char *msg)
{
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            char b_[256];                                                                     \
            snprintf(b_, sizeof b_, "%s failed: %s", #call, cudaGetErrorString(e_));          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RT3D_ENOMEM : RT3D_ECUDA, b_); \
        }                                                                                     \
    } while (0)

template <typename T>
static cudaError_t grow(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void **)&p, std::max<size_t>(need, 1) * sizeof(T));
    if (e == cudaSuccess) cap = need;
    return e;
}

static void free_field(FieldSlot &s)
{
    cudaFree(s.d_part);
    cudaFree(s.d_eps2);
    cudaFree(s.d_m64);
    cudaFree(s.d_eps2_64);
    cudaFree(s.d_rot);
    cudaFree(s.d_shift);
    grid_free(s.gd);
    s = FieldSlot{};
}

extern "C" const char *rt3d_status_string(int s)
{
    switch (s) {
    case RT3D_OK: return "ok";
    case RT3D_EINVAL: return "invalid argument";
    case RT3D_ENOMEM: return "out of memory";
    case RT3D_ECUDA: return "CUDA error";
    case RT3D_ETIMEOUT: return "device watchdog expired";
    case RT3D_ENOTIMPL: return "not implemented";
    case RT3D_ENOCOSMO: return "cosmology not set";
    case RT3D_ENOFIELD: return "field not loaded";
    default: return "unknown status";
    }
}

extern "C" const char *rt3d_last_error(rt3d_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int rt3d_create(rt3d_ctx **out, int dev, const rt3d_options *opt)
{
    if (!out) return RT3D_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev < 0 || dev >= ndev) return RT3D_EINVAL;
    rt3d_ctx *ctx = new (std::nothrow) rt3d_ctx();
    if (!ctx) return RT3D_ENOMEM;
    ctx->device = dev;
    if (opt) ctx->opt = *opt;
    if (ctx->opt.precision != RT3D_MIXED && ctx->opt.precision != RT3D_FP64) {
        delete ctx;
        return RT3D_EINVAL;
    }
    if (ctx->opt.christoffel != RT3D_CHRISTOFFEL_PAPER && ctx->opt.christoffel != RT3D_CHRISTOFFEL_DERIVED) {
        delete ctx;
        return RT3D_EINVAL;
    }
    if (ctx->opt.cluster != 0 && ctx->opt.cluster != 1 && ctx->opt.cluster != 4) {
        delete ctx;
        return RT3D_EINVAL;
    }
    ctx->fields.resize(RT3D_MAX_FIELDS);
    int rc = RT3D_OK;
    do {
        if (cudaSetDevice(dev) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || ctx->n_sm < 1) {
            rc = RT3D_ECUDA;
            break;
        }
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        if (cudaMalloc((void **)&ctx->scr.misc, 16 * sizeof(double)) != cudaSuccess) { rc = RT3D_ENOMEM; break; }
        if (cudaMalloc((void **)&ctx->scr.counters, 8 * sizeof(unsigned long long)) != cudaSuccess) { rc = RT3D_ENOMEM; break; }
    } while (0);
    if (rc != RT3D_OK) {
        rt3d_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return RT3D_OK;
}

extern "C" int rt3d_destroy(rt3d_ctx *ctx)
{
    if (!ctx) return RT3D_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &f : ctx->fields) free_field(f);
    Scratch &s = ctx->scr;
    cudaFree(s.partials);
    cudaFree(s.dlam);
    cudaFree(s.misc);
    cudaFree(s.counters);
    cudaFree(s.state);
    cudaFree(s.ints);
    cudaFree(s.theta);
    cudaFree(s.bout);
    cudaFree(s.rout);
    cudaFree(s.prism);
    cudaFree(s.planes);
    cudaFree(ctx->atab);
    cudaFree(ctx->d_hist_u64);
    cudaFree(ctx->d_hist_f64);
    cudaFree(ctx->d_io);
    for (auto e : ctx->tev) cudaEventDestroy(e);
    {
        auto &B = ctx->batch;
        if (B.exec) cudaGraphExecDestroy(B.exec);
        cudaFree(B.cones);
        cudaFree(B.items);
        cudaFree(B.rb2cone);
        cudaFree(B.state);
        cudaFree(B.ints);
        cudaFree(B.theta);
        cudaFree(B.dlam);
        cudaFree(B.partials);
        cudaFree(B.cnt);
        cudaFree(B.bar);
        cudaFree(B.bout);
        cudaFree(B.rout);
        cudaFree(B.prism);
    }
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return RT3D_OK;
}

extern "C" int rt3d_set_cosmology(rt3d_ctx *ctx, double om, double ol, double h)
{
    if (!ctx) return RT3D_EINVAL;
    if (!(om > 0.0) || !(ol > 0.0) || !(h > 0.0) || !isfinite(om + ol + h) || fabs(om + ol - 1.0) > 1e-12)
        return fail(ctx, RT3D_EINVAL, "cosmology must be flat with omega_m, omega_l, h > 0");
    Cosmo &c = ctx->cosmo;
    c.om = om;
    c.ol = ol;
    c.h = h;
    c.H0 = 100.0 * h / kCkms;
    // Eq. lookbacksingularity with the argument sqrt(OL/OM), so that a(0) = 1
    c.t0 = 2.0 / (3.0 * c.H0 * sqrt(ol)) * asinh(sqrt(ol / om));
    c.k = 1.5 * sqrt(ol) * c.H0;
    c.r = om / ol;
    // a(t) table up to the lookback time of z = 5 (a = 1/6):
    // t(a) = t0 - asinh(sqrt(a^3 / r)) / k
    CK(cudaSetDevice(ctx->device));
    const int n = 4096;
    const double t_max = c.t0 - asinh(sqrt(pow(1.0 / 6.0, 3.0) / c.r)) / c.k;
    CK(grow(ctx->atab, ctx->atab_n, (size_t)(2 * n)));
    c.atab = nullptr;  // the table is filled from the closed form
    CK(launch_atab(c, n, t_max / (n - 1), ctx->atab, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    c.atab = ctx->atab;
    c.atab_n = n;
    c.atab_h = t_max / (n - 1);
    c.atab_ih = 1.0 / c.atab_h;
    ctx->have_cosmo = true;
    return RT3D_OK;
}

extern "C" int rt3d_load_particles(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos, const double *mass,
                                   const double *soft, int soft_pp, const rt3d_volume *vol)
{
    if (ctx && field_id >= 0 && field_id < RT3D_MAX_FIELDS && ctx->trace.open &&
        ctx->trace.fs == &ctx->fields[field_id])
        ctx->trace.open = false;  // the open trace's field is replaced
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS) return fail(ctx, RT3D_EINVAL, "field id out of range");
    if (n < 0 || (n > 0 && (!pos || !mass)) || (!soft && n > 0)) return fail(ctx, RT3D_EINVAL, "null particle arrays");
    if (n >= (int64_t)1 << 40) return fail(ctx, RT3D_EINVAL, "too many particles");
    const bool repl = vol && vol->replicated;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(pos[3 * i]) || !isfinite(pos[3 * i + 1]) || !isfinite(pos[3 * i + 2]))
            return fail(ctx, RT3D_EINVAL, "non-finite particle position");
        if (!(mass[i] > 0.0) || !isfinite(mass[i])) return fail(ctx, RT3D_EINVAL, "particle masses must be > 0");
        const double e = soft_pp ? soft[i] : soft[0];
        if (!(e >= 0.0) || !isfinite(e)) return fail(ctx, RT3D_EINVAL, "softening must be >= 0");
    }
    if (n == 0 && soft && !(soft[0] >= 0.0)) return fail(ctx, RT3D_EINVAL, "softening must be >= 0");
    bool umass = n > 0;
    for (int64_t i = 1; i < n && umass; ++i) umass = mass[i] == mass[0];
    double L = 0.0;
    if (repl) {
        L = vol->box_length;
        if (!(L > 0.0) || !isfinite(L) || vol->n_replicas < 1 || !vol->rot || !vol->shift)
            return fail(ctx, RT3D_EINVAL, "replicated volume needs box_length > 0 and replica transforms");
        for (int j = 0; j < vol->n_replicas; ++j) {
            const int32_t *R = vol->rot + 9 * j;
            int colused = 0;
            for (int r = 0; r < 3; ++r) {
                int nz = 0;
                for (int k = 0; k < 3; ++k)
                    if (R[3 * r + k] != 0) {
                        if (R[3 * r + k] != 1 && R[3 * r + k] != -1) return fail(ctx, RT3D_EINVAL, "rot must be a signed permutation");
                        ++nz;
                        colused |= 1 << k;
                    }
                if (nz != 1) return fail(ctx, RT3D_EINVAL, "rot must be a signed permutation");
            }
            if (colused != 7) return fail(ctx, RT3D_EINVAL, "rot must be a signed permutation");
            for (int d = 0; d < 3; ++d)
                if (!(vol->shift[3 * j + d] >= 0.0) || !(vol->shift[3 * j + d] < L))
                    return fail(ctx, RT3D_EINVAL, "replica shift outside [0, L)");
        }
        for (int64_t i = 0; i < 3 * n; ++i)
            if (pos[i] < 0.0 || pos[i] > L) return fail(ctx, RT3D_EINVAL, "box positions outside [0, L]");
    }
    CK(cudaSetDevice(ctx->device));
    FieldSlot &slot = ctx->fields[field_id];
    CK(cudaStreamSynchronize(ctx->stream));
    free_field(slot);

    const int64_t nn = std::max<int64_t>(n, 1);
    double *d_pos = nullptr, *d_mass = nullptr, *d_soft = nullptr, *d_stats = nullptr;
    int rc = RT3D_OK;
    double st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    do {
        if (cudaMalloc((void **)&d_pos, 3 * nn * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&d_mass, nn * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&d_soft, (soft_pp ? nn : 1) * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&d_stats, 8 * sizeof(double)) != cudaSuccess) { rc = RT3D_ENOMEM; break; }
        if (n > 0) {
            if (cudaMemcpyAsync(d_pos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
                cudaMemcpyAsync(d_mass, mass, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
                cudaMemcpyAsync(d_soft, soft, (soft_pp ? n : 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) { rc = RT3D_ECUDA; break; }
            k_field_stats<<<1, 1024, 0, ctx->stream>>>(n, d_pos, d_mass, d_stats);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(st, d_stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        }
        // grid: the finest 2^-e that holds the field in 2^30 (isolated, centred)
        // or the box in 2^31 (replicated) grid units
        DevField &f = slot.df;
        f = DevField{};
        int e = 40;
        double O[3] = {0.0, 0.0, 0.0};
        long long Lq = 0;
        const double q22 = ldexp(1.0, -22);
        if (repl) {
            e = (int)floor(log2(2147483000.0 / L));
            if (e > 40) e = 40;
            Lq = llround(ldexp(L, e));
            if (Lq & 1) Lq += 1;
        } else if (n > 0) {
            double H = 0.0;
            for (int d = 0; d < 3; ++d) {
                O[d] = nearbyint(0.5 * (st[d] + st[3 + d]) / q22) * q22;
                H = std::max(H, std::max(fabs(st[3 + d] - O[d]), fabs(st[d] - O[d])));
            }
            if (H > 0.0) e = std::min(40, (int)floor(log2(1073741824.0 / H)));
        }
        const double two_e = ldexp(1.0, e);
        const double mmax = kMuG * st[6];
        const int ms = mmax > 0.0 ? -(int)nearbyint(log2(mmax)) : 0;
        const double mscale = ldexp(1.0, ms);
        if (cudaMalloc((void **)&slot.d_part, nn * sizeof(int4)) != cudaSuccess ||
            cudaMalloc((void **)&slot.d_m64, nn * sizeof(double)) != cudaSuccess) { rc = RT3D_ENOMEM; break; }
        if (soft_pp && (cudaMalloc((void **)&slot.d_eps2, nn * sizeof(float)) != cudaSuccess ||
                        cudaMalloc((void **)&slot.d_eps2_64, nn * sizeof(double)) != cudaSuccess)) { rc = RT3D_ENOMEM; break; }
        if (n > 0) {
            k_stage_particles<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
                n, d_pos, d_mass, d_soft, soft_pp, soft[0], repl ? 1 : 0, repl ? Lq : 0, O[0], O[1], O[2], two_e,
                mscale, slot.d_part, slot.d_m64, slot.d_eps2, slot.d_eps2_64);
            if (cudaGetLastError() != cudaSuccess) { rc = RT3D_ECUDA; break; }
        }
        if (repl) {
            std::vector<int> rot(9 * vol->n_replicas), sh(3 * vol->n_replicas);
            for (int j = 0; j < 9 * vol->n_replicas; ++j) rot[j] = vol->rot[j];
            for (int j = 0; j < 3 * vol->n_replicas; ++j) {
                long long v = llround(ldexp(vol->shift[j], e)) % Lq;
                sh[j] = (int)v;
            }
            if (cudaMalloc((void **)&slot.d_rot, rot.size() * sizeof(int)) != cudaSuccess ||
                cudaMalloc((void **)&slot.d_shift, sh.size() * sizeof(int)) != cudaSuccess) { rc = RT3D_ENOMEM; break; }
            if (cudaMemcpyAsync(slot.d_rot, rot.data(), rot.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
                cudaMemcpyAsync(slot.d_shift, sh.data(), sh.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        }
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { rc = RT3D_ECUDA; break; }
        f.part = slot.d_part;
        f.eps2 = slot.d_eps2;
        f.m64 = slot.d_m64;
        f.eps2_64 = slot.d_eps2_64;
        f.rot = slot.d_rot;
        f.shift = slot.d_shift;
        f.n = n;
        const double e0 = soft_pp ? 0.0 : soft[0];
        f.eps2u = (float)(e0 * e0);
        f.eps2u64 = e0 * e0;
        f.replicated = repl ? 1 : 0;
        f.mean_subtract = (repl && vol->mean_subtract) ? 1 : 0;
        f.n_rep = repl ? vol->n_replicas : 1;
        f.Lq = (int)Lq;
        f.delta = ldexp(1.0, -e);
        f.inv_delta = two_e;
        f.O[0] = O[0];
        f.O[1] = O[1];
        f.O[2] = O[2];
        f.L = repl ? (double)Lq * f.delta : 0.0;
        f.mscale_inv = ldexp(1.0, -ms);
        f.rho_term = repl ? kMuG * st[7] / (f.L * f.L * f.L) : 0.0;
        f.uniform_mass = umass ? 1 : 0;
        f.m_uniform = umass ? kMuG * mass[0] * mscale : 0.0;
        slot.n = n;
        if (!repl && n > 0) {
            slot.x3_lo = slot.x3_hi = pos[2];
            for (int64_t i = 1; i < n; ++i) {
                slot.x3_lo = std::min(slot.x3_lo, pos[3 * i + 2]);
                slot.x3_hi = std::max(slot.x3_hi, pos[3 * i + 2]);
            }
        }
        slot.loaded = true;
    } while (0);
    cudaFree(d_pos);
    cudaFree(d_mass);
    cudaFree(d_soft);
    cudaFree(d_stats);
    if (rc != RT3D_OK) {
        free_field(slot);
        return fail(ctx, rc, "particle staging failed");
    }
    return RT3D_OK;
}

// resident blocks per SM of shape sh's pair-sum kernel: queried for the
// two-bundle kernel (its launch bounds and shared memory set it), about five
// blocks of 128 threads for the others
static int resident_blocks(const DevField &f, const ForceShape &sh)
{
    if (sh.variant == 5) {
        ForceArgs A{};
        A.f = f;
        A.n = rays_per_block(sh);
        ForceShape q = sh;
        q.splits = q.cl;
        int occ = 0;
        if (dispatch_bundle2x(A, q, q.umass != 0, nullptr, &occ) == cudaSuccess && occ > 0) return occ;
    }
    return std::max(1, 640 / sh.NT);
}

// Particle splits for a launch of nrb ray blocks: about `waves` waves of
// resident blocks (wave = blocks the device holds at once), whole tiles per
// split.  A last wave that is only part full leaves SMs idle at the end of the
// launch, so up to twice that count the first split count whose blocks fill
// their last wave to 99 % is taken (else the fullest).
static int splits_for(int64_t nrb, int64_t wave, double waves, int tiles)
{
    auto balanced = [&](int64_t s) {
        s = std::max<int64_t>(1, std::min<int64_t>(s, tiles));
        const int64_t tps = (tiles + s - 1) / s;
        return (int)((tiles + tps - 1) / tps);
    };
    auto fill = [&](int s) {
        const int64_t b = nrb * s;
        return (double)b / (double)(((b + wave - 1) / wave) * wave);
    };
    const int s0 = balanced((int64_t)std::ceil(waves * (double)wave / (double)nrb));
    int best = s0;
    double bf = fill(s0);
    for (int s = s0 + 1; s <= std::min(2 * s0, tiles) && bf < 0.99; ++s) {
        const int sb = balanced(s);
        const double fb = fill(sb);
        if (fb > bf + 1e-12) {
            best = sb;
            bf = fb;
        }
    }
    return best;
}

// a clustered shape needs whole clusters along the splits; splits past the
// particles are empty and add zeros
static void round_to_clusters(ForceShape &sh)
{
    if (sh.cl > 1 && sh.splits < 2 * sh.cl) sh.cl = 1;  // too few splits to pair up
    if (sh.cl > 1) sh.splits = (sh.splits + sh.cl - 1) / sh.cl * sh.cl;
}

// ---------------------------------------------------------------------------
// launch shape
// ---------------------------------------------------------------------------
// group = rays per bundle for a trace (1 for arbitrary points).  Traces with
// rings of 4 or 8 use the bundle-centric kernel (R = rays per bundle, NT =
// bundles per block); other calls the packed kernel (R rays per thread).
static ForceShape choose_shape(rt3d_ctx *ctx, const DevField &f, int64_t n_points, bool fp64, int group = 1)
{
    const int64_t n_particles = f.n;
    ForceShape sh;
    sh.umass = 0;
    if (fp64) {
        sh.variant = 2;
        sh.R = 2;
        sh.NT = 128;
    } else if ((ctx->opt.variant == 0 || ctx->opt.variant >= 3) && (group == 5 || group == 9)) {
        // bundle-centric: two bundles per thread with the expanded separations
        // (variant 5, rings of 4 and 8), without them (4, rings of 4), or one
        // bundle per thread (3)
        if (group == 5)
            sh.variant = ctx->opt.variant == 3 || ctx->opt.variant == 4 ? ctx->opt.variant : 5;
        else
            sh.variant = ctx->opt.variant == 3 || ctx->opt.variant == 4 ? 3 : 5;
        sh.umass = f.uniform_mass ? 1 : 0;
        sh.R = group;
        const bool two = sh.variant == 4 || sh.variant == 5;
        sh.NT = ctx->opt.threads_per_block > 0 ? ctx->opt.threads_per_block : (two ? 64 : 128);
        if (two && sh.NT > 128) sh.NT = 128;
        if (sh.variant == 5 && group == 9) sh.NT = 64;  // the ring-of-8 kernel's only block size
    } else {
        sh.variant = ctx->opt.variant == 1 ? 1 : 0;
        sh.umass = (sh.variant == 0 && f.uniform_mass) ? 1 : 0;
        sh.R = ctx->opt.rays_per_thread > 0 ? ctx->opt.rays_per_thread : 4;
        sh.NT = ctx->opt.threads_per_block > 0 ? ctx->opt.threads_per_block : 128;
    }
    const int64_t per_block = rays_per_block(sh);
    const int64_t nrb = std::max<int64_t>(1, (n_points + per_block - 1) / per_block);
    const int tiles = force_max_splits(sh, n_particles);
    int S;
    if (ctx->opt.splits > 0) {
        S = std::min(ctx->opt.splits, tiles);
        // balance: whole tiles per split, then the number of splits actually used
        const int64_t tps = (tiles + S - 1) / S;
        S = (int)((tiles + tps - 1) / tps);
    } else {
        // about five waves of resident blocks: many small blocks balance the
        // SMs better than one exact wave
        S = splits_for(nrb, (int64_t)ctx->n_sm * resident_blocks(f, sh), 5.0, tiles);
    }
    sh.splits = std::max(1, S);
    // the expanded two-bundle kernel can add groups of 4 splits in a cluster
    // (off unless asked for: measured slower on the NFW workload, see the tuner)
    sh.cl = (sh.variant == 5 && group == 5 && ctx->opt.cluster == 4) ? 4 : 1;
    round_to_clusters(sh);
    return sh;
}

static int64_t per_split_of(const ForceShape &sh, int64_t n_particles)
{
    const int64_t tiles = std::max<int64_t>(1, (n_particles + kTile - 1) / kTile);
    return ((tiles + sh.splits - 1) / sh.splits) * kTile;
}

static cudaError_t run_force(rt3d_ctx *ctx, const DevField &f, const double *px, const double *py, const double *pz,
                             const int *rep, int group, int64_t n, const ForceShape &sh, bool fp64, void *partials,
                             const unsigned long long *gate, cudaStream_t st)
{
    ForceArgs A;
    A.f = f;
    A.px = px;
    A.py = py;
    A.pz = pz;
    A.rep = rep;
    A.group = group;
    A.n = n;
    A.per_split = per_split_of(sh, f.n);
    A.out = partials;
    A.gate = gate;
    (void)ctx;
    (void)fp64;
    if (sh.variant == 2) return dispatch_fp64(A, sh, st);
    if (sh.variant == 1) return dispatch_mixed(A, sh, st);
    if (sh.variant == 3) return dispatch_bundle(A, sh, sh.umass != 0, st);
    if (sh.variant == 4) return dispatch_bundle2(A, sh, sh.umass != 0, st);
    if (sh.variant == 5) return dispatch_bundle2x(A, sh, sh.umass != 0, st);
    return dispatch_packed(A, sh, sh.umass != 0, st);
}

// ---------------------------------------------------------------------------
// autotuner: time candidate launch shapes of the pair sum once per size class
// (variant, uniform mass, replicated, per-particle softening, log2 points,
// log2 particles) on the caller's data, keep the fastest.  Shapes differ only
// in how the FP32 partial sums are split, so results agree to rounding.
// ---------------------------------------------------------------------------
static int ilog2(int64_t v)
{
    int l = 0;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

static ForceShape with_splits(const rt3d_ctx *ctx, const DevField &f, ForceShape sh, int64_t n_points,
                              int64_t n_particles, int waves)
{
    const int64_t per_block = rays_per_block(sh);
    const int64_t nrb = std::max<int64_t>(1, (n_points + per_block - 1) / per_block);
    const int64_t wave = (int64_t)ctx->n_sm * resident_blocks(f, sh);
    sh.splits = splits_for(nrb, wave, (double)waves, force_max_splits(sh, n_particles));
    round_to_clusters(sh);
    return sh;
}

static int tuned_shape(rt3d_ctx *ctx, const FieldSlot &fs, const double *px, const double *py, const double *pz,
                       const int *rep, int group, int64_t n, bool fp64, cudaStream_t st, ForceShape &out)
{
    ForceShape base = choose_shape(ctx, fs.df, n, fp64, group);
    if (!ctx->opt.autotune || ctx->opt.rays_per_thread > 0 || ctx->opt.threads_per_block > 0 || ctx->opt.splits > 0) {
        out = base;
        return RT3D_OK;
    }
    const auto key = std::make_tuple(base.variant, base.umass, fs.df.replicated, fs.df.eps2 != nullptr ? 1 : 0,
                                     ilog2(n), ilog2(std::max<int64_t>(1, fs.n)));
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        out = with_splits(ctx, fs.df, it->second, n, fs.n, it->second.splits);  // splits slot holds the wave count
        return RT3D_OK;
    }
    // Launches beyond 2^37 interactions (~50 ms) are timed on a proxy: the
    // first rays (whole bundles, at most 16 waves of the largest block) against
    // a prefix of the particles (whole tiles), so that each timing launch stays
    // near 2^37 interactions.  Candidates cost the same per interaction on the
    // proxy as on the whole launch; the chosen shape is then sized for the
    // whole launch by its wave count.
    DevField dft = fs.df;
    int64_t n_t = n;
    const double cap = 137438953472.0;
    if ((double)n * (double)fs.n > cap) {
        const int64_t nb = n / group;
        const int64_t nb_t = std::min<int64_t>(nb, (int64_t)ctx->n_sm * 16 * 256);
        n_t = nb_t * group;
        const int64_t np_t = std::max<int64_t>(kTile, (int64_t)(cap / (double)n_t) / kTile * kTile);
        dft.n = std::min<int64_t>(dft.n, np_t);
    }
    std::vector<ForceShape> cand;
    std::vector<int> waves;
    const int rn[][2] = {{4, 128}, {4, 256}, {4, 64}, {8, 64}};
    const int rn64[][2] = {{2, 128}, {1, 128}};
    // bundle shapes: {variant, rays per bundle, threads per block, cluster size}
    const int rnb4[][4] = {{3, 5, 128, 1}, {3, 5, 64, 1}, {3, 5, 256, 1}, {4, 5, 64, 1}, {4, 5, 128, 1},
                           {5, 5, 64, 1}, {5, 5, 128, 1}, {5, 5, 64, 4}, {5, 5, 128, 4}};
    const int rnb8[][4] = {{3, 9, 128, 1}, {3, 9, 64, 1}, {3, 9, 256, 1}, {5, 9, 64, 1}};
    const int(*rnb)[4] = group == 5 ? rnb4 : rnb8;
    const bool bundles = base.variant >= 3;
    const int nrn = base.variant == 2 ? 2 : (bundles ? (group == 5 ? 9 : 4) : 4);
    for (int c = 0; c < nrn; ++c)
        for (int w : {2, 3, 5, 8, 16}) {
            ForceShape s = base;
            // a requested bundle kernel (or cluster size) is tuned over its own shapes only
            if (bundles && ctx->opt.variant >= 3 && rnb[c][0] != base.variant) continue;
            if (bundles && ctx->opt.cluster > 0 && rnb[c][3] != ctx->opt.cluster) continue;
            if (bundles) {
                s.variant = rnb[c][0];
                s.R = rnb[c][1];
                s.NT = rnb[c][2];
                s.cl = rnb[c][3];
            } else {
                const int *p = base.variant == 2 ? rn64[c] : rn[c];
                s.R = p[0];
                s.NT = p[1];
            }
            s = with_splits(ctx, dft, s, n_t, dft.n, w);
            bool dup = false;  // the same launch under another wave count
            for (const auto &c2 : cand)
                dup |= c2.variant == s.variant && c2.R == s.R && c2.NT == s.NT && c2.cl == s.cl && c2.splits == s.splits;
            if (dup) continue;
            cand.push_back(s);
            waves.push_back(w);
        }
    if (cand.empty()) {
        out = base;
        return RT3D_OK;
    }
    size_t need = 0;
    for (auto &s : cand) need = std::max(need, partials_bytes(s, n_t, fp64));
    CK(grow(*(char **)&ctx->scr.partials, ctx->scr.partials_bytes, need));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    size_t bi = 0;
    for (size_t c = 0; c < cand.size(); ++c) {
        CK(run_force(ctx, dft, px, py, pz, rep, group, n_t, cand[c], fp64, ctx->scr.partials, nullptr, st));
        for (int rep_t = 0; rep_t < 3; ++rep_t) {  // best of three: candidates are often within 1-2 %
            CK(cudaEventRecord(e0, st));
            CK(run_force(ctx, dft, px, py, pz, rep, group, n_t, cand[c], fp64, ctx->scr.partials, nullptr, st));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bi = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ForceShape keep = cand[bi];
    keep.splits = waves[bi];
    ctx->tuned[key] = keep;
    out = n_t == n && dft.n == fs.df.n ? cand[bi] : with_splits(ctx, fs.df, keep, n, fs.n, waves[bi]);
    return RT3D_OK;
}

// ---------------------------------------------------------------------------
// trace orchestration
// ---------------------------------------------------------------------------
static int check_bundle_opts(rt3d_ctx *ctx, const rt3d_bundle_opts *b)
{
    if (!b) return fail(ctx, RT3D_EINVAL, "null bundle options");
    if (b->n_ring < 3 || b->n_ring > 8) return fail(ctx, RT3D_EINVAL, "n_ring must be 3..8");
    if (!(b->theta_r > 0.0) || !isfinite(b->theta_r) || !isfinite(b->phase)) return fail(ctx, RT3D_EINVAL, "bad theta_r/phase");
    if (b->n_steps < 1 || b->n_steps > 10000000) return fail(ctx, RT3D_EINVAL, "n_steps out of range");
    if (b->max_extra < 0 || b->max_extra > 64) return fail(ctx, RT3D_EINVAL, "max_extra must be 0..64");
    if (b->schedule == RT3D_SCHED_ASINH) {
        if (!(b->asinh_s > 0.0) || !isfinite(b->lens_chi)) return fail(ctx, RT3D_EINVAL, "asinh schedule needs s > 0");
    } else if (b->schedule != RT3D_SCHED_UNIFORM) {
        return fail(ctx, RT3D_EINVAL, "unknown schedule");
    }
    return RT3D_OK;
}

static cudaEvent_t timing_event(rt3d_ctx *ctx)
{
    if (ctx->tev_used == (int)ctx->tev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->tev.push_back(e);
    }
    return ctx->tev[ctx->tev_used++];
}

static int ensure_trace_scratch(rt3d_ctx *ctx, int64_t n_b, int nr, int n_steps, const ForceShape &sh)
{
    Scratch &s = ctx->scr;
    const int64_t n_rays = n_b * nr;
    CK(grow(s.state, s.state_rays, (size_t)(32 * n_rays)));
    CK(grow(s.ints, s.ints_n, (size_t)(2 * n_rays + 2 * n_b)));
    CK(grow(s.dlam, s.dlam_n, (size_t)n_steps));
    size_t pb = partials_bytes(sh, n_rays, false);
    CK(grow(*(char **)&s.partials, s.partials_bytes, pb));
    return RT3D_OK;
}

static RayState make_state(rt3d_ctx *ctx, int64_t n_b, int nr)
{
    Scratch &s = ctx->scr;
    RayState rs;
    rs.n_rays = n_b * nr;
    rs.n_b = n_b;
    rs.nr = nr;
    rs.y = s.state;
    rs.ys = s.state + 8 * rs.n_rays;
    rs.ks = s.state + 16 * rs.n_rays;
    rs.fin = s.state + 24 * rs.n_rays;
    rs.done = s.ints;
    rs.steps = s.ints + rs.n_rays;
    rs.rep = s.ints + 2 * rs.n_rays;
    rs.stride = rs.n_rays;
    return rs;
}

// force shape of a grid-path trace: one "split" of interpolated values, no
// mass factor (variant 6 names the grid path in the statistics)
static ForceShape grid_shape()
{
    ForceShape sh;
    sh.R = 1;
    sh.NT = 128;
    sh.splits = 1;
    sh.variant = 6;
    sh.umass = 0;
    return sh;
}

// schedule (S0), bundle initialiser (S1), launch shape; the trace is then open
static int trace_begin(rt3d_ctx *ctx, const FieldSlot &fs, double z_s, int64_t n_b, const double *d_theta,
                       const rt3d_bundle_opts *b, cudaStream_t st, bool timed)
{
    OpenTrace &T = ctx->trace;
    T = OpenTrace{};
    T.fp64 = ctx->opt.precision == RT3D_FP64;
    const int nr = 1 + b->n_ring;
    const int64_t n_rays = n_b * nr;
    T.sh = fs.is_grid ? grid_shape() : choose_shape(ctx, fs.df, n_rays, T.fp64, nr);
    int rc = ensure_trace_scratch(ctx, n_b, nr, b->n_steps, T.sh);
    if (rc) return rc;
    T.rs = make_state(ctx, n_b, nr);
    const bool tune_pending = ctx->opt.autotune != 0 && !fs.is_grid;
    TraceParams &tp = T.tp;
    tp.cosmo = ctx->cosmo;
    tp.chi_s = 0.0;
    tp.n_ring = b->n_ring;
    tp.theta_r = b->theta_r;
    tp.phase = b->phase;
    tp.christoffel = ctx->opt.christoffel;
    tp.n_steps = b->n_steps;
    tp.max_extra = b->max_extra;
    Scratch &s = ctx->scr;
    ctx->tev_used = 0;
    CK(launch_schedule(ctx->cosmo, z_s, b->schedule, b->n_steps, b->lens_chi, b->asinh_s, s.dlam, s.misc, st));
    CK(launch_init(tp, fs.df, d_theta, T.rs, s.counters, st));
    T.launches = 2;
    if (tune_pending) {  // rays now sit at the observer: time shapes on this field
        rc = tuned_shape(ctx, fs, T.rs.ys + n_rays, T.rs.ys + 2 * n_rays, T.rs.ys + 3 * n_rays, T.rs.rep, nr, n_rays,
                         T.fp64, st, T.sh);
        if (rc) return rc;
        rc = ensure_trace_scratch(ctx, n_b, nr, b->n_steps, T.sh);
        if (rc) return rc;
        T.rs = make_state(ctx, n_b, nr);
    }
    // mean-subtracted boxes: the prism field once per bundle and stage (value,
    // gradient, Hessian), expanded to the bundle's other rays
    T.use_prism = !fs.is_grid && fs.df.replicated && fs.df.mean_subtract;
    if (T.use_prism) CK(grow(s.prism, s.prism_n, (size_t)(kPrismRec * n_b)));
    T.fs = &fs;
    T.d_theta = d_theta;
    T.n_b = n_b;
    T.b = *b;
    T.timed = timed;
    T.next = 0;
    T.total = 4 * (b->n_steps + b->max_extra);
    T.open = true;
    ctx->stats_pending = false;
    return RT3D_OK;
}

// the next n global RK4 stages (S2-S6): pair sum (or grid evaluation), the
// prism of mean-subtracted boxes, the integrator stage
static int trace_advance(rt3d_ctx *ctx, int n, cudaStream_t st)
{
    OpenTrace &T = ctx->trace;
    const FieldSlot &fs = *T.fs;
    const int64_t n_rays = T.rs.n_rays;
    const int nr = T.rs.nr;
    Scratch &s = ctx->scr;
    const int stop = std::min(T.total, T.next + n);
    for (; T.next < stop; ++T.next) {
        const int g = T.next, step = g / 4, stage = g % 4;
        // extra steps past the table run only while some ray is not across
        const unsigned long long *gate = step >= T.b.n_steps ? s.counters + ((step - 1) & 1) : nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (T.timed && !gate) {
            e0 = timing_event(ctx);
            e1 = timing_event(ctx);
            if (e0) CK(cudaEventRecord(e0, st));
        }
        if (fs.is_grid)
            CK(launch_grid_eval(fs.gd, T.rs.ys + n_rays, T.rs.ys + 2 * n_rays, T.rs.ys + 3 * n_rays, n_rays,
                                T.fp64 ? 1 : 0, s.partials, gate, st, nr));
        else
            CK(run_force(ctx, fs.df, T.rs.ys + n_rays, T.rs.ys + 2 * n_rays, T.rs.ys + 3 * n_rays,
                         T.rs.rep + (g & 1) * T.n_b, nr, n_rays, T.sh, T.fp64, s.partials, gate, st));
        if (e1) CK(cudaEventRecord(e1, st));
        if (T.use_prism) {
            CK(launch_prism(T.tp, fs.df, T.rs, step, stage, s.counters, s.prism, st));
            ++T.launches;
        }
        CK(launch_stage(T.tp, fs.df, T.rs, T.sh, T.fp64, s.partials, s.dlam, s.misc, step, stage, s.counters, st,
                        T.use_prism ? s.prism : nullptr));
        T.launches += 2;
        T.flaunch += gate ? 0 : 1;
    }
    ctx->stats.launches = T.launches;
    ctx->stats.force_launches = T.flaunch;
    ctx->stats.steps = (T.next + 3) / 4;
    ctx->stats.rays_per_thread = T.sh.R;
    ctx->stats.threads_per_block = T.sh.NT;
    ctx->stats.splits = T.sh.splits;
    ctx->stats.cluster = T.sh.cl;
    ctx->stats.variant = T.sh.variant;
    // grid path: one field evaluation per ray and stage counts as one
    ctx->last_npart = fs.is_grid ? 1.0 : (double)fs.n;
    ctx->stats_pending = true;
    return RT3D_OK;
}

// the remaining stages, then the bundle reducer (S7); the trace is closed
static int trace_end(rt3d_ctx *ctx, double *d_bout, double *d_rout, cudaStream_t st)
{
    OpenTrace &T = ctx->trace;
    int rc = trace_advance(ctx, T.total - T.next, st);
    if (rc) return rc;
    CK(launch_reduce(T.tp, T.d_theta, T.rs, ctx->scr.misc, d_bout, d_rout, st));
    T.launches += 1;
    ctx->stats.launches = T.launches;
    T.open = false;
    return RT3D_OK;
}

// enqueue one full trace on st: schedule, init, RK4 stages, reduce
static int enqueue_trace(rt3d_ctx *ctx, const FieldSlot &fs, double z_s, int64_t n_b, const double *d_theta,
                         const rt3d_bundle_opts *b, double *d_bout, double *d_rout, cudaStream_t st, bool timed)
{
    int rc = trace_begin(ctx, fs, z_s, n_b, d_theta, b, st, timed);
    if (rc) return rc;
    return trace_end(ctx, d_bout, d_rout, st);
}

static int finish_stats(rt3d_ctx *ctx)
{
    if (!ctx->stats_pending) return RT3D_OK;
    unsigned long long c[3];
    CK(cudaMemcpy(c, ctx->scr.counters, sizeof c, cudaMemcpyDeviceToHost));
    ctx->stats.interactions = (double)c[2] * ctx->last_npart;
    double fms = 0.0;
    for (int i = 0; i + 1 < ctx->tev_used; i += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->tev[i], ctx->tev[i + 1]) == cudaSuccess) fms += ms;
    }
    ctx->stats.force_ms = fms;
    ctx->stats_pending = false;
    return RT3D_OK;
}

static int check_trace_args(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_b, const rt3d_bundle_opts *b)
{
    if (!ctx->have_cosmo) return fail(ctx, RT3D_ENOCOSMO, "set the cosmology first");
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS || !ctx->fields[field_id].loaded)
        return fail(ctx, RT3D_ENOFIELD, "field not loaded");
    if (!(z_s > 0.0) || !isfinite(z_s) || z_s > 20.0) return fail(ctx, RT3D_EINVAL, "z_s must be in (0, 20]");
    if (n_b < 1 || n_b > ((int64_t)1 << 28)) return fail(ctx, RT3D_EINVAL, "n_bundles out of range");
    return check_bundle_opts(ctx, b);
}

extern "C" int rt3d_trace(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_b, const double *theta,
                          const rt3d_bundle_opts *b, rt3d_bundle_result *out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    int rc = check_trace_args(ctx, field_id, z_s, n_b, b);
    if (rc) return rc;
    if (!theta || !out || !out->mu) return fail(ctx, RT3D_EINVAL, "null theta or result arrays");
    for (int64_t i = 0; i < 2 * n_b; ++i)
        if (!isfinite(theta[i])) return fail(ctx, RT3D_EINVAL, "non-finite theta");
    CK(cudaSetDevice(ctx->device));
    const int nr = 1 + b->n_ring;
    const int64_t n_rays = n_b * nr;
    Scratch &s = ctx->scr;
    CK(grow(s.theta, s.theta_n, (size_t)(2 * n_b)));
    CK(grow(s.bout, s.bout_n, (size_t)(6 * n_b)));
    const bool want_rays = out->ray_state != nullptr;
    if (want_rays) CK(grow(s.rout, s.rout_n, (size_t)(8 * n_rays)));
    cudaStream_t st = ctx->stream;
    CK(cudaEventRecord(ctx->ev0, st));
    CK(cudaMemcpyAsync(s.theta, theta, 2 * n_b * sizeof(double), cudaMemcpyHostToDevice, st));
    rc = enqueue_trace(ctx, ctx->fields[field_id], z_s, n_b, s.theta, b, s.bout, want_rays ? s.rout : nullptr, st,
                       ctx->opt.time_kernels != 0);
    if (rc) return rc;
    std::vector<double> bo((size_t)(6 * n_b));
    CK(cudaMemcpyAsync(bo.data(), s.bout, 6 * n_b * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (want_rays) CK(cudaMemcpyAsync(out->ray_state, s.rout, 8 * n_rays * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (out->ray_steps)
        CK(cudaMemcpyAsync(out->ray_steps, ctx->scr.ints + n_rays, n_rays * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ctx->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->stats.device_ms = ms;
    rc = finish_stats(ctx);
    if (rc) return rc;
    for (int64_t i = 0; i < n_b; ++i) {
        out->mu[i] = bo[6 * i];
        if (out->kappa) out->kappa[i] = bo[6 * i + 1];
        if (out->gamma1) out->gamma1[i] = bo[6 * i + 2];
        if (out->gamma2) out->gamma2[i] = bo[6 * i + 3];
        if (out->omega) out->omega[i] = bo[6 * i + 4];
        if (out->flags) out->flags[i] = (int32_t)bo[6 * i + 5];
    }
    return RT3D_OK;
}

extern "C" int rt3d_trace_device(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_b,
                                 const double *d_theta, const rt3d_bundle_opts *b, double *d_bundle_out,
                                 double *d_ray_out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    int rc = check_trace_args(ctx, field_id, z_s, n_b, b);
    if (rc) return rc;
    if (!d_theta || !d_bundle_out) return fail(ctx, RT3D_EINVAL, "null device arrays");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    return enqueue_trace(ctx, ctx->fields[field_id], z_s, n_b, d_theta, b, d_bundle_out, d_ray_out, st,
                         ctx->opt.time_kernels != 0);
}

extern "C" int rt3d_trace_begin(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_b,
                                const double *d_theta, const rt3d_bundle_opts *b)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;
    int rc = check_trace_args(ctx, field_id, z_s, n_b, b);
    if (rc) return rc;
    if (!d_theta) return fail(ctx, RT3D_EINVAL, "null device theta");
    CK(cudaSetDevice(ctx->device));
    return trace_begin(ctx, ctx->fields[field_id], z_s, n_b, d_theta, b, (cudaStream_t)stream,
                       ctx->opt.time_kernels != 0);
}

extern "C" int rt3d_trace_advance(rt3d_ctx *ctx, void *stream, int n_stages, int *stages_left)
{
    if (!ctx) return RT3D_EINVAL;
    if (!ctx->trace.open) return fail(ctx, RT3D_EINVAL, "no open trace (rt3d_trace_begin first)");
    if (n_stages < 0) return fail(ctx, RT3D_EINVAL, "n_stages must be >= 0");
    CK(cudaSetDevice(ctx->device));
    int rc = trace_advance(ctx, n_stages, (cudaStream_t)stream);
    if (rc) {
        ctx->trace.open = false;
        return rc;
    }
    if (stages_left) *stages_left = ctx->trace.total - ctx->trace.next;
    return RT3D_OK;
}

extern "C" int rt3d_trace_end(rt3d_ctx *ctx, void *stream, double *d_bundle_out, double *d_ray_out)
{
    if (!ctx) return RT3D_EINVAL;
    if (!ctx->trace.open) return fail(ctx, RT3D_EINVAL, "no open trace (rt3d_trace_begin first)");
    if (!d_bundle_out) return fail(ctx, RT3D_EINVAL, "null device bundle output");
    CK(cudaSetDevice(ctx->device));
    int rc = trace_end(ctx, d_bundle_out, d_ray_out, (cudaStream_t)stream);
    ctx->trace.open = false;
    return rc;
}

// ---------------------------------------------------------------------------
// multiple lens-plane comparison system (Sec. 3.1)
// ---------------------------------------------------------------------------
static void unpack_bundles(const double *bo, int64_t nb, rt3d_bundle_result *out);

static int check_mp_args(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_b, const rt3d_bundle_opts *b, int slices)
{
    int rc = check_trace_args(ctx, field_id, z_s, n_b, b);
    if (rc) return rc;
    if (ctx->fields[field_id].is_grid)
        return fail(ctx, RT3D_ENOTIMPL, "the lens-plane system projects particle fields, not grid fields");
    if (slices < 1 || slices > 4096) return fail(ctx, RT3D_EINVAL, "slices must be 1..4096");
    const FieldSlot &fs = ctx->fields[field_id];
    if ((int64_t)(fs.df.replicated ? fs.df.n_rep : 1) * slices > 65536)
        return fail(ctx, RT3D_EINVAL, "at most 65536 lens planes");
    return RT3D_OK;
}

static int enqueue_multiplane(rt3d_ctx *ctx, const FieldSlot &fs, double z_s, int64_t n_b, const double *d_theta,
                              const rt3d_bundle_opts *b, int slices, double *d_bout, double *d_rout, cudaStream_t st)
{
    const bool fp64 = ctx->opt.precision == RT3D_FP64;
    const int nr = 1 + b->n_ring;
    const int64_t n_rays = n_b * nr;
    Scratch &s = ctx->scr;
    CK(grow(s.state, s.state_rays, (size_t)(32 * n_rays)));
    CK(grow(s.ints, s.ints_n, (size_t)(2 * n_rays + 2 * n_b)));
    RayState rs = make_state(ctx, n_b, nr);
    const int n_pl = (fs.df.replicated ? fs.df.n_rep : 1) * slices;
    CK(grow(*(char **)&s.planes, s.planes_bytes, (size_t)n_pl * mp_plane_bytes()));
    // particle splits: about five waves of blocks (128 bundles per block; 64 for FP64)
    const int64_t blocks = (n_b + (fp64 ? 63 : 127)) / (fp64 ? 64 : 128);
    const int64_t tiles = std::max<int64_t>(1, (fs.n + kTile - 1) / kTile);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)ctx->n_sm * 5 * 4 + blocks - 1) / blocks));
    CK(grow(*(char **)&s.partials, s.partials_bytes, mp_partials_bytes(b->n_ring, n_b, splits, fp64)));
    TraceParams tp{};
    tp.cosmo = ctx->cosmo;
    tp.n_ring = b->n_ring;
    tp.theta_r = b->theta_r;
    tp.phase = b->phase;
    tp.christoffel = ctx->opt.christoffel;
    tp.n_steps = 1;
    const bool umass = !fp64 && fs.df.uniform_mass;
    CK(mp_run(ctx->cosmo, fs.df, z_s, slices, fs.x3_lo, fs.x3_hi, tp, d_theta, rs, s.planes, n_pl, s.partials, splits,
              fp64, umass, s.misc, s.counters + 2, d_bout, d_rout, st));
    ctx->stats = rt3d_stats{};
    ctx->stats.launches = 4 + 2 * (int64_t)n_pl;
    ctx->stats.force_launches = n_pl;
    ctx->stats.splits = splits;
    ctx->stats.variant = 7;
    ctx->last_npart = (double)n_rays;  // interactions = rays x particles on the planes
    ctx->stats_pending = true;
    ctx->tev_used = 0;
    return RT3D_OK;
}

extern "C" int rt3d_multiplane(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_b, const double *theta,
                               const rt3d_bundle_opts *b, int slices, rt3d_bundle_result *out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    int rc = check_mp_args(ctx, field_id, z_s, n_b, b, slices);
    if (rc) return rc;
    if (!theta || !out || !out->mu) return fail(ctx, RT3D_EINVAL, "null theta or result arrays");
    for (int64_t i = 0; i < 2 * n_b; ++i)
        if (!isfinite(theta[i])) return fail(ctx, RT3D_EINVAL, "non-finite theta");
    CK(cudaSetDevice(ctx->device));
    const int64_t n_rays = n_b * (1 + b->n_ring);
    Scratch &s = ctx->scr;
    CK(grow(s.theta, s.theta_n, (size_t)(2 * n_b)));
    CK(grow(s.bout, s.bout_n, (size_t)(6 * n_b)));
    const bool want_rays = out->ray_state != nullptr;
    if (want_rays) CK(grow(s.rout, s.rout_n, (size_t)(8 * n_rays)));
    cudaStream_t st = ctx->stream;
    CK(cudaEventRecord(ctx->ev0, st));
    CK(cudaMemcpyAsync(s.theta, theta, 2 * n_b * sizeof(double), cudaMemcpyHostToDevice, st));
    rc = enqueue_multiplane(ctx, ctx->fields[field_id], z_s, n_b, s.theta, b, slices, s.bout,
                            want_rays ? s.rout : nullptr, st);
    if (rc) return rc;
    std::vector<double> bo((size_t)(6 * n_b));
    CK(cudaMemcpyAsync(bo.data(), s.bout, 6 * n_b * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (want_rays) CK(cudaMemcpyAsync(out->ray_state, s.rout, 8 * n_rays * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ctx->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    rc = finish_stats(ctx);
    if (rc) return rc;
    ctx->stats.device_ms = ms;
    unpack_bundles(bo.data(), n_b, out);
    if (out->ray_steps)
        for (int64_t i = 0; i < n_rays; ++i) out->ray_steps[i] = 0;
    return RT3D_OK;
}

extern "C" int rt3d_multiplane_device(rt3d_ctx *ctx, void *stream, int field_id, double z_s, int64_t n_b,
                                      const double *d_theta, const rt3d_bundle_opts *b, int slices,
                                      double *d_bundle_out, double *d_ray_out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    int rc = check_mp_args(ctx, field_id, z_s, n_b, b, slices);
    if (rc) return rc;
    if (!d_theta || !d_bundle_out) return fail(ctx, RT3D_EINVAL, "null device arrays");
    CK(cudaSetDevice(ctx->device));
    return enqueue_multiplane(ctx, ctx->fields[field_id], z_s, n_b, d_theta, b, slices, d_bundle_out, d_ray_out,
                              (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// batched trace (many cones, one persistent launch in a CUDA graph)
// ---------------------------------------------------------------------------
struct BatchPlan {
    int64_t T = 0, n_b_total = 0, dlam_total = 0, partials_total = 0;
    int max_steps = 0, g_end = 0;
    std::vector<int64_t> ray_base, b_base, dlam_off, part_off, per_split;
    std::vector<int> S;
    std::vector<int4> items;
    std::vector<int64_t> cost;  // rays x particles of each item (planning order)
    std::vector<int> rb2cone;
    size_t cone_bytes(int n) const { return sizeof(BatchCone) * (size_t)n; }
};

// Layout of a batch: each cone's rays padded to whole ray blocks of RB, its
// particles split into whole tiles of about per_item particles, one work item
// per (cone, ray block, split).
static int plan_batch(const FieldSlot *fields, int n_cones, const rt3d_cone *cones, int nr, int RB, int NT,
                      int64_t per_item, int max_extra, BatchPlan &p)
{
    p = BatchPlan{};
    for (int c = 0; c < n_cones; ++c) {
        const int64_t nb = cones[c].n_bundles, n_rays = nb * nr, N = fields[cones[c].field_id].n;
        const int64_t nrb = (n_rays + RB - 1) / RB;
        if (fields[cones[c].field_id].is_grid) {
            // a grid cone: one evaluation item per ray block, one split
            p.ray_base.push_back(p.T);
            p.b_base.push_back(p.n_b_total);
            p.dlam_off.push_back(p.dlam_total);
            p.part_off.push_back(p.partials_total);
            p.per_split.push_back(0);
            p.S.push_back(1);
            for (int64_t rb = 0; rb < nrb; ++rb) {
                p.items.push_back(make_int4(c, (int)rb, 0, 1));
                // about 500 FP32 operations and 1 KB of node reads per ray
                p.cost.push_back(25 * std::min<int64_t>(RB, n_rays - rb * RB));
                p.rb2cone.push_back(c);
            }
            p.T += nrb * RB;
            p.n_b_total += nb;
            p.dlam_total += cones[c].n_steps;
            p.partials_total += 4 * n_rays;
            p.max_steps = std::max(p.max_steps, cones[c].n_steps);
            p.g_end = std::max(p.g_end, 4 * (cones[c].n_steps + max_extra));
            continue;
        }
        const int64_t tiles = std::max<int64_t>(1, (N + kTile - 1) / kTile);
        int64_t S = std::max<int64_t>(1, (tiles * kTile + per_item - 1) / per_item);
        S = std::min(S, tiles);
        const int64_t tps = (tiles + S - 1) / S;
        S = (tiles + tps - 1) / tps;
        p.ray_base.push_back(p.T);
        p.b_base.push_back(p.n_b_total);
        p.dlam_off.push_back(p.dlam_total);
        p.part_off.push_back(p.partials_total);
        p.per_split.push_back(tps * kTile);
        p.S.push_back((int)S);
        for (int64_t rb = 0; rb < nrb; ++rb) {
            for (int64_t s = 0; s < S; ++s) p.items.push_back(make_int4(c, (int)rb, (int)s, 0));
            p.rb2cone.push_back(c);
        }
        p.T += nrb * RB;
        const FieldSlot &fs = fields[cones[c].field_id];
        if (fs.df.replicated && fs.df.mean_subtract) {
            // prism records: one item per block of NT bundles, costed as the
            // FP64 closed form (about 24 000 pair interactions per bundle)
            const int64_t nbb = (nb + NT - 1) / NT;
            for (int64_t q = 0; q < nbb; ++q) {
                p.items.push_back(make_int4(c, (int)q, -1, 0));
                p.cost.push_back(24000 * std::min<int64_t>(NT, nb - q * NT));
            }
        }
        for (int64_t rb = 0; rb < nrb; ++rb) {
            const int64_t rays = std::min<int64_t>(RB, n_rays - rb * RB);
            for (int64_t s = 0; s < S; ++s) {
                const int64_t parts = std::min<int64_t>(tps * kTile, N - s * tps * kTile);
                p.cost.push_back(rays * std::max<int64_t>(parts, 1));
            }
        }
        p.n_b_total += nb;
        p.dlam_total += cones[c].n_steps;
        p.partials_total += S * 4 * n_rays;
        p.max_steps = std::max(p.max_steps, cones[c].n_steps);
        p.g_end = std::max(p.g_end, 4 * (cones[c].n_steps + max_extra));
    }
    // the work queue hands out items in this order: largest first
    std::vector<size_t> order(p.items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return p.cost[a] > p.cost[b]; });
    std::vector<int4> sorted(p.items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = p.items[order[i]];
    p.items.swap(sorted);
    return RT3D_OK;
}

static void fill_cone_table(const FieldSlot *fields, const Cosmo &cosmo, int christoffel, int n_cones,
                            const rt3d_cone *cones, const rt3d_bundle_opts *b, const BatchPlan &p, double *state,
                            int *ints, double *theta, double *dlam, float2 *partials, unsigned long long *cnt,
                            double *rout, double *prism, std::vector<unsigned char> &table)
{
    table.assign(p.cone_bytes(n_cones), 0);
    BatchCone *T = (BatchCone *)table.data();
    const int nr = 1 + b->n_ring;
    for (int c = 0; c < n_cones; ++c) {
        BatchCone &C = T[c];
        const DevField &f = fields[cones[c].field_id].df;
        C.f = f;
        RayState &rs = C.rs;
        rs.stride = p.T;
        rs.y = state + p.ray_base[c];
        rs.ys = state + 8 * p.T + p.ray_base[c];
        rs.ks = state + 16 * p.T + p.ray_base[c];
        rs.fin = state + 24 * p.T + p.ray_base[c];
        rs.done = ints + p.ray_base[c];
        rs.steps = ints + p.T + p.ray_base[c];
        rs.rep = ints + 2 * p.T + 2 * p.b_base[c];
        rs.n_b = cones[c].n_bundles;
        rs.nr = nr;
        rs.n_rays = rs.n_b * nr;
        C.tp.cosmo = cosmo;
        C.tp.chi_s = 0.0;
        C.tp.n_ring = b->n_ring;
        C.tp.theta_r = b->theta_r;
        C.tp.phase = b->phase;
        C.tp.christoffel = christoffel;
        C.tp.n_steps = cones[c].n_steps;
        C.tp.max_extra = b->max_extra;
        C.theta = theta + 2 * p.b_base[c];
        C.dlam = dlam + p.dlam_off[c];
        C.partials = partials + p.part_off[c];
        C.cnt = cnt + 3 * c;
        C.rout = rout ? rout + 8 * nr * p.b_base[c] : nullptr;
        C.prism = (f.replicated && f.mean_subtract) ? prism + kPrismRec * p.b_base[c] : nullptr;
        C.chi_s = 0.0;
        C.z_s = cones[c].z_s;
        C.chi_l = b->lens_chi;
        C.s_asinh = b->asinh_s;
        C.kind = b->schedule;
        C.mfac = f.uniform_mass ? f.m_uniform : 1.0;
        C.per_split = p.per_split[c];
        C.ray_base = p.ray_base[c];
        C.b_base = p.b_base[c];
        C.S = p.S[c];
        C.flags = (f.replicated ? 1 : 0) | (f.eps2 ? 2 : 0) | (f.uniform_mass ? 4 : 0);
        C.total_steps = cones[c].n_steps + b->max_extra;
        C.grid = fields[cones[c].field_id].is_grid ? 1 : 0;
        C.g = fields[cones[c].field_id].gd;
    }
}

static void unpack_bundles(const double *bo, int64_t nb, rt3d_bundle_result *out)
{
    for (int64_t i = 0; i < nb; ++i) {
        out->mu[i] = bo[6 * i];
        if (out->kappa) out->kappa[i] = bo[6 * i + 1];
        if (out->gamma1) out->gamma1[i] = bo[6 * i + 2];
        if (out->gamma2) out->gamma2[i] = bo[6 * i + 3];
        if (out->omega) out->omega[i] = bo[6 * i + 4];
        if (out->flags) out->flags[i] = (int32_t)bo[6 * i + 5];
    }
}

// rays per ray block of the batched kernel: 2 NT bundles (expanded
// two-bundle kernel, rings of 4), NT bundles (bundle-centric kernel, rings of
// 4 or 8) or 2 kBatchP rays per thread (packed kernel); all multiples of 32
constexpr int kBatchP = 2;
static int batch_rays_per_block(int nr, int NT, int MODE)
{
    return MODE == 5 ? 2 * NT * nr : ((nr == 5 || nr == 9) ? NT * nr : 2 * kBatchP * NT);
}

// Build the batch layout for launch shape (NT, particles per work item),
// upload it, and run (or replay) the graph.  g_limit > 0 runs only that many
// global stages (autotuner timing); then nothing is read back.
static int batch_run(rt3d_ctx *ctx, int n_cones, const rt3d_cone *cones, const rt3d_bundle_opts *b, int NT,
                     int64_t per_item, int MODE, int g_limit, bool want_rays, float *ms_out)
{
    auto &BS = ctx->batch;
    const int P = kBatchP;
    const int nr = 1 + b->n_ring;
    const int RB = batch_rays_per_block(nr, NT, MODE);
    BatchPlan plan;
    int rc = plan_batch(ctx->fields.data(), n_cones, cones, nr, RB, NT, per_item, b->max_extra, plan);
    if (rc) return fail(ctx, rc, "invalid cone list");
    const int64_t T = plan.T;
    CK(grow(*(char **)&BS.cones, BS.cones_n, plan.cone_bytes(n_cones)));
    CK(grow(BS.items, BS.items_n, plan.items.size()));
    CK(grow(BS.rb2cone, BS.rb_n, plan.rb2cone.size()));
    CK(grow(BS.state, BS.state_n, (size_t)(32 * T)));
    CK(grow(BS.ints, BS.ints_n, (size_t)(2 * T + 2 * plan.n_b_total)));
    CK(grow(BS.theta, BS.theta_n, (size_t)(2 * plan.n_b_total)));
    CK(grow(BS.dlam, BS.dlam_n, (size_t)plan.dlam_total));
    CK(grow(BS.partials, BS.partials_n, (size_t)plan.partials_total));
    CK(grow(BS.cnt, BS.cnt_n, (size_t)(3 * n_cones)));
    size_t bar_n = BS.bar ? 8 : 0;
    CK(grow(BS.bar, bar_n, 8));
    CK(grow(BS.bout, BS.bout_n, (size_t)(6 * plan.n_b_total)));
    if (want_rays) CK(grow(BS.rout, BS.rout_n, (size_t)(8 * nr * plan.n_b_total)));
    std::vector<unsigned char> table;
    CK(grow(BS.prism, BS.prism_n, (size_t)(kPrismRec * plan.n_b_total)));
    fill_cone_table(ctx->fields.data(), ctx->cosmo, ctx->opt.christoffel, n_cones, cones, b, plan, BS.state, BS.ints,
                    BS.theta, BS.dlam, BS.partials, BS.cnt, want_rays ? BS.rout : nullptr, BS.prism, table);
    cudaStream_t st = ctx->stream;
    for (int c = 0; c < n_cones; ++c)
        CK(cudaMemcpyAsync(BS.theta + 2 * plan.b_base[c], cones[c].theta, 2 * cones[c].n_bundles * sizeof(double),
                           cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(BS.cones, table.data(), table.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(BS.items, plan.items.data(), plan.items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(BS.rb2cone, plan.rb2cone.data(), plan.rb2cone.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(BS.bar, 0, 8 * sizeof(unsigned), st));
    int grid = 0;
    CK(batch_resident_blocks(NT, MODE, &grid));
    if (grid < 1) return fail(ctx, RT3D_ECUDA, "persistent kernel cannot be resident");
    BatchArgs A = make_batch_args(BS.cones, n_cones, BS.items, (int64_t)plan.items.size(), BS.rb2cone, T, RB,
                                  g_limit > 0 ? g_limit : plan.g_end, BS.bar, (int *)(BS.bar + 2),
                                  ctx->opt.watchdog_s > 0 ? ctx->opt.watchdog_s : 120.0, BS.bout);
    // the graph is keyed by everything its launches capture
    std::vector<long long> key = {n_cones, T, (long long)plan.items.size(), A.g_end, NT, MODE, per_item, grid,
                                  plan.max_steps, plan.n_b_total, (long long)(intptr_t)BS.cones,
                                  (long long)(intptr_t)BS.items, (long long)(intptr_t)BS.bout,
                                  (long long)(intptr_t)BS.prism};
    CK(cudaEventRecord(ctx->ev0, st));
    bool use_graph = g_limit == 0;
    if (use_graph && (BS.key != key || !BS.exec)) {
        if (BS.exec) {
            cudaGraphExecDestroy(BS.exec);
            BS.exec = nullptr;
        }
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = batch_launch(A, NT, MODE, grid, plan.max_steps, plan.n_b_total, st);
        cudaError_t ce = cudaStreamEndCapture(st, &gr);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            use_graph = false;  // capture unsupported here: launch directly
        } else {
            cudaError_t ie = cudaGraphInstantiate(&BS.exec, gr, 0);
            cudaGraphDestroy(gr);
            if (ie != cudaSuccess) {
                BS.exec = nullptr;
                cudaGetLastError();
                use_graph = false;
            } else {
                BS.key = key;
            }
        }
    }
    if (use_graph) CK(cudaGraphLaunch(BS.exec, st));
    else CK(batch_launch(A, NT, MODE, grid, plan.max_steps, plan.n_b_total, st));
    CK(cudaEventRecord(ctx->ev1, st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (ms_out) *ms_out = ms;
    unsigned err = 0;
    CK(cudaMemcpy(&err, BS.bar + 2, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(ctx, RT3D_ETIMEOUT, "persistent kernel: a grid barrier wait exceeded the watchdog");
    ctx->stats.device_ms = ms;
    ctx->stats.launches = 4;
    ctx->stats.force_launches = 1;
    ctx->stats.steps = plan.max_steps + b->max_extra;
    ctx->stats.rays_per_thread = (nr == 5 || nr == 9) ? nr : 2 * P;
    ctx->stats.threads_per_block = NT;
    ctx->stats.variant = MODE == 5 ? 5 : ((nr == 5 || nr == 9) ? 3 : 0);
    ctx->stats.cluster = 1;
    ctx->stats.splits = (int)per_item;
    ctx->stats.force_ms = ms;
    ctx->stats_pending = false;
    if (g_limit > 0) return RT3D_OK;
    std::vector<unsigned long long> cnt((size_t)(3 * n_cones));
    CK(cudaMemcpy(cnt.data(), BS.cnt, cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    double inter = 0.0;
    // grid cones count one field evaluation per ray and stage
    for (int c = 0; c < n_cones; ++c) {
        const FieldSlot &fs = ctx->fields[cones[c].field_id];
        inter += (double)cnt[3 * c + 2] * (fs.is_grid ? 1.0 : (double)fs.n);
    }
    ctx->stats.interactions = inter;
    return RT3D_OK;
}

extern "C" int rt3d_trace_batch(rt3d_ctx *ctx, int n_cones, const rt3d_cone *cones, const rt3d_bundle_opts *b,
                                rt3d_bundle_result *outs)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    if (n_cones < 1 || !cones || !outs) return fail(ctx, RT3D_EINVAL, "need n_cones >= 1, cones and outputs");
    int rc = check_bundle_opts(ctx, b);
    if (rc) return rc;
    if (!ctx->have_cosmo) return fail(ctx, RT3D_ENOCOSMO, "set the cosmology first");
    for (int c = 0; c < n_cones; ++c) {
        const rt3d_cone &k = cones[c];
        if (k.field_id < 0 || k.field_id >= RT3D_MAX_FIELDS || !ctx->fields[k.field_id].loaded)
            return fail(ctx, RT3D_ENOFIELD, "cone field not loaded");
        if (!(k.z_s > 0.0) || k.z_s > 20.0 || k.n_bundles < 1 || !k.theta || k.n_steps < 1 || k.n_steps > 10000000)
            return fail(ctx, RT3D_EINVAL, "cone needs z_s in (0, 20], n_bundles >= 1, theta, n_steps >= 1");
        if (!outs[c].mu) return fail(ctx, RT3D_EINVAL, "null mu output");
        for (int64_t i = 0; i < 2 * k.n_bundles; ++i)
            if (!isfinite(k.theta[i])) return fail(ctx, RT3D_EINVAL, "non-finite theta");
    }
    CK(cudaSetDevice(ctx->device));
    if (ctx->opt.precision == RT3D_FP64) {
        // the all-FP64 reference path: one cone per launch sequence
        double ms = 0.0, inter = 0.0;
        for (int c = 0; c < n_cones; ++c) {
            rt3d_bundle_opts bc = *b;
            bc.n_steps = cones[c].n_steps;
            rc = rt3d_trace(ctx, cones[c].field_id, cones[c].z_s, cones[c].n_bundles, cones[c].theta, &bc, &outs[c]);
            if (rc) return rc;
            ms += ctx->stats.device_ms;
            inter += ctx->stats.interactions;
        }
        ctx->stats.device_ms = ms;
        ctx->stats.interactions = inter;
        return RT3D_OK;
    }
    bool want_rays = false;
    for (int c = 0; c < n_cones; ++c) want_rays |= outs[c].ray_state != nullptr || outs[c].ray_steps != nullptr;
    // launch shape: kernel, block size and particles per work item (autotuned
    // per size class).  Rings of 4 default to the expanded two-bundle kernel
    // (64 threads: its compensated sums fill the static shared memory), other
    // rings to the bundle-centric or packed kernel; variant 3 asks for the
    // bundle-centric kernel, variant 5 for the two-bundle one.
    const int nr = 1 + b->n_ring;
    const int mode_plain = nr == 5 ? 4 : (nr == 9 ? 8 : 0);
    int NT = ctx->opt.threads_per_block == 64 || ctx->opt.threads_per_block == 256 ? ctx->opt.threads_per_block : 128;
    if (NT == 256 && b->n_ring == 8) NT = 128;
    int MODE = mode_plain;
    if (nr == 5 && ctx->opt.variant != 3 && (ctx->opt.threads_per_block <= 0 || ctx->opt.threads_per_block == 64)) {
        MODE = 5;
        NT = 64;
    }
    int64_t per_item = ctx->opt.splits > 0 ? (int64_t)ctx->opt.splits * kTile : 16 * kTile;
    if (ctx->opt.autotune && ctx->opt.threads_per_block <= 0 && ctx->opt.splits <= 0) {
        int64_t rays = 0;
        double pairs = 0.0;
        for (int c = 0; c < n_cones; ++c) {
            rays += cones[c].n_bundles * (1 + b->n_ring);
            pairs += (double)cones[c].n_bundles * (1 + b->n_ring) * (double)ctx->fields[cones[c].field_id].n;
        }
        const auto key = std::make_tuple(n_cones, ilog2(rays), ilog2((int64_t)std::max(1.0, pairs)));
        auto it = ctx->batch.tuned.find(key);
        if (it != ctx->batch.tuned.end()) {
            std::tie(NT, per_item, MODE) = it->second;
        } else {
            float best = 1e30f;
            // (threads, kernel mode) candidates
            std::vector<std::pair<int, int>> shapes;
            if (nr == 5 && ctx->opt.variant != 3) shapes.push_back({64, 5});
            if (!(nr == 5 && ctx->opt.variant == 5))
                for (int nt : {128, 256, 64})
                    if (!(nt == 256 && b->n_ring == 8)) shapes.push_back({nt, mode_plain});
            for (const auto &sh : shapes)
                for (int tiles : {8, 16, 32}) {
                    float ms = 0.0f;
                    rc = batch_run(ctx, n_cones, cones, b, sh.first, (int64_t)tiles * kTile, sh.second, 8, false, &ms);
                    if (rc) return rc;
                    if (ms < best) {
                        best = ms;
                        NT = sh.first;
                        MODE = sh.second;
                        per_item = (int64_t)tiles * kTile;
                    }
                }
            ctx->batch.tuned[key] = std::make_tuple(NT, (int)per_item, MODE);
        }
    }
    rc = batch_run(ctx, n_cones, cones, b, NT, per_item, MODE, 0, want_rays, nullptr);
    if (rc) return rc;
    // read back per cone
    auto &BS = ctx->batch;
    int64_t nbt = 0;
    for (int c = 0; c < n_cones; ++c) nbt += cones[c].n_bundles;
    std::vector<double> bo((size_t)(6 * nbt));
    CK(cudaMemcpy(bo.data(), BS.bout, bo.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> ro;
    if (want_rays) {
        ro.resize((size_t)(8 * nr * nbt));
        CK(cudaMemcpy(ro.data(), BS.rout, ro.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    int64_t off = 0;
    for (int c = 0; c < n_cones; ++c) {
        const int64_t nb = cones[c].n_bundles;
        unpack_bundles(bo.data() + 6 * off, nb, &outs[c]);
        if (want_rays && outs[c].ray_state)
            memcpy(outs[c].ray_state, ro.data() + 8 * nr * off, 8 * nr * nb * sizeof(double));
        off += nb;
    }
    if (want_rays) {
        // crossing steps: read each cone's done/steps view
        std::vector<int> steps;
        int64_t T = 0;
        const int RB = batch_rays_per_block(nr, NT, MODE);
        for (int c = 0; c < n_cones; ++c) T += ((cones[c].n_bundles * nr + RB - 1) / RB) * RB;
        steps.resize((size_t)T);
        CK(cudaMemcpy(steps.data(), BS.ints + T, T * sizeof(int), cudaMemcpyDeviceToHost));
        int64_t base = 0;
        for (int c = 0; c < n_cones; ++c) {
            const int64_t n = cones[c].n_bundles * nr;
            if (outs[c].ray_steps) memcpy(outs[c].ray_steps, steps.data() + base, n * sizeof(int));
            base += ((n + RB - 1) / RB) * RB;
        }
    }
    return RT3D_OK;
}

static int ensure_hist(rt3d_ctx *ctx, int bins)
{
    if (bins > ctx->hist_cap) {
        cudaFree(ctx->d_hist_u64);
        cudaFree(ctx->d_hist_f64);
        ctx->d_hist_u64 = nullptr;
        ctx->d_hist_f64 = nullptr;
        ctx->hist_cap = 0;
        CK(cudaMalloc((void **)&ctx->d_hist_u64, (2 * (size_t)bins + 8) * sizeof(unsigned long long)));
        CK(cudaMalloc((void **)&ctx->d_hist_f64, 8 * sizeof(double)));
        ctx->hist_cap = bins;
    }
    return RT3D_OK;
}

static int check_hist(rt3d_ctx *ctx, const rt3d_hist_opts *o)
{
    if (!o || o->bins < 1 || o->bins > (1 << 20) || !(o->mu_min > 0.0) || !(o->mu_max > o->mu_min) ||
        !isfinite(o->mu_max))
        return fail(ctx, RT3D_EINVAL, "histogram needs bins >= 1 and 0 < mu_min < mu_max");
    return RT3D_OK;
}

extern "C" int rt3d_histogram(rt3d_ctx *ctx, int64_t n, const double *mu, const int32_t *flags,
                              const rt3d_hist_opts *o, rt3d_hist *out)
{
    if (!ctx) return RT3D_EINVAL;
    int rc = check_hist(ctx, o);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !mu) || !out || !out->counts || !out->wfix) return fail(ctx, RT3D_EINVAL, "null arrays");
    CK(cudaSetDevice(ctx->device));
    rc = ensure_hist(ctx, o->bins);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    const size_t need = (size_t)std::max<int64_t>(n, 1) * 2;
    CK(grow(ctx->d_io, ctx->d_io_n, need));
    double *d_mu = ctx->d_io;
    int *d_fl = flags ? (int *)(ctx->d_io + std::max<int64_t>(n, 1)) : nullptr;
    if (n > 0) CK(cudaMemcpyAsync(d_mu, mu, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (flags && n > 0) CK(cudaMemcpyAsync(d_fl, flags, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    unsigned long long *cnt = ctx->d_hist_u64, *wf = cnt + o->bins, *sc = wf + o->bins;
    CK(launch_histogram(n, d_mu, 1, d_fl, nullptr, o->bins, o->mu_min, o->mu_max, cnt, wf, sc, ctx->d_hist_f64, st));
    double o8[8];
    CK(cudaMemcpyAsync(out->counts, cnt, o->bins * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out->wfix, wf, o->bins * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(o8, ctx->d_hist_f64, sizeof o8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->n_used = (int64_t)o8[0];
    out->n_under = (int64_t)o8[1];
    out->n_over = (int64_t)o8[2];
    out->n_neg = (int64_t)o8[3];
    out->n_bad = (int64_t)o8[4];
    out->W_total = o8[5];
    out->mean_w = o8[6];
    out->sigma_w = o8[7];
    return RT3D_OK;
}

extern "C" int rt3d_shear_histogram(rt3d_ctx *ctx, int64_t n, const double *mu, const double *gamma1,
                                    const double *gamma2, const int32_t *flags, const rt3d_hist_opts *o,
                                    rt3d_hist *out)
{
    if (!ctx) return RT3D_EINVAL;
    int rc = check_hist(ctx, o);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!mu || !gamma1 || !gamma2)) || !out || !out->counts || !out->wfix)
        return fail(ctx, RT3D_EINVAL, "null arrays");
    CK(cudaSetDevice(ctx->device));
    rc = ensure_hist(ctx, o->bins);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    const int64_t m = std::max<int64_t>(n, 1);
    CK(grow(ctx->d_io, ctx->d_io_n, (size_t)(4 * m)));
    double *d_mu = ctx->d_io, *d_g1 = ctx->d_io + m, *d_g2 = ctx->d_io + 2 * m;
    int *d_fl = flags ? (int *)(ctx->d_io + 3 * m) : nullptr;
    if (n > 0) {
        CK(cudaMemcpyAsync(d_mu, mu, n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_g1, gamma1, n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_g2, gamma2, n * sizeof(double), cudaMemcpyHostToDevice, st));
        if (flags) CK(cudaMemcpyAsync(d_fl, flags, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    unsigned long long *cnt = ctx->d_hist_u64, *wf = cnt + o->bins, *sc = wf + o->bins;
    CK(launch_histogram(n, d_mu, 1, d_fl, nullptr, o->bins, o->mu_min, o->mu_max, cnt, wf, sc, ctx->d_hist_f64, st,
                        d_g1, d_g2));
    double o8[8];
    CK(cudaMemcpyAsync(out->counts, cnt, o->bins * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out->wfix, wf, o->bins * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(o8, ctx->d_hist_f64, sizeof o8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->n_used = (int64_t)o8[0];
    out->n_under = (int64_t)o8[1];
    out->n_over = (int64_t)o8[2];
    out->n_neg = (int64_t)o8[3];
    out->n_bad = (int64_t)o8[4];
    out->W_total = o8[5];
    out->mean_w = o8[6];
    out->sigma_w = o8[7];
    return RT3D_OK;
}

// Sum of x into (s, c) by Neumaier's compensated addition.
static void neumaier_add(double &s, double &c, double x)
{
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

extern "C" int rt3d_histogram_combine(rt3d_ctx *ctx, int n_parts, int bins, const rt3d_hist *parts, rt3d_hist *out)
{
    if (n_parts < 1 || bins < 1 || !parts || !out || !out->counts || !out->wfix)
        return fail(ctx, RT3D_EINVAL, "need n_parts >= 1, bins >= 1, parts and output arrays");
    for (int p = 0; p < n_parts; ++p) {
        const rt3d_hist &h = parts[p];
        if (!h.counts || !h.wfix) return fail(ctx, RT3D_EINVAL, "null counts or weights in a part");
        if (h.n_used < 0 || h.n_under < 0 || h.n_over < 0 || h.n_neg < 0 || h.n_bad < 0 || !(h.W_total >= 0.0) ||
            !isfinite(h.W_total) || !isfinite(h.mean_w) || !(h.sigma_w >= 0.0) || !isfinite(h.sigma_w))
            return fail(ctx, RT3D_EINVAL, "a part's scalars are negative or not finite");
    }
    std::vector<uint64_t> c((size_t)bins, 0), w((size_t)bins, 0);
    rt3d_hist r{};
    double W = 0.0, Wc = 0.0, M = 0.0, Mc = 0.0;
    for (int p = 0; p < n_parts; ++p) {
        const rt3d_hist &h = parts[p];
        for (int k = 0; k < bins; ++k) {
            c[k] += h.counts[k];
            w[k] += h.wfix[k];
        }
        r.n_used += h.n_used;
        r.n_under += h.n_under;
        r.n_over += h.n_over;
        r.n_neg += h.n_neg;
        r.n_bad += h.n_bad;
        neumaier_add(W, Wc, h.W_total);
        neumaier_add(M, Mc, h.W_total * h.mean_w);
    }
    W += Wc;
    const double mean = W > 0.0 ? (M + Mc) / W : 0.0;
    // spread of the union: each part's weighted square deviation about its own
    // mean plus its weight times the square distance of that mean from the union's
    double V = 0.0, Vc = 0.0;
    for (int p = 0; p < n_parts; ++p) {
        const rt3d_hist &h = parts[p];
        const double d = h.mean_w - mean;
        neumaier_add(V, Vc, h.W_total * (h.sigma_w * h.sigma_w + d * d));
    }
    r.W_total = W;
    r.mean_w = mean;
    r.sigma_w = W > 0.0 ? sqrt((V + Vc) / W) : 0.0;
    r.counts = out->counts;
    r.wfix = out->wfix;
    for (int k = 0; k < bins; ++k) {
        out->counts[k] = c[k];
        out->wfix[k] = w[k];
    }
    *out = r;
    return RT3D_OK;
}

extern "C" int rt3d_histogram_device(rt3d_ctx *ctx, void *stream, int64_t n, const double *d_bundle_out,
                                     const rt3d_hist_opts *o, uint64_t *d_counts, uint64_t *d_wfix,
                                     double *d_scalars)
{
    if (!ctx) return RT3D_EINVAL;
    int rc = check_hist(ctx, o);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !d_bundle_out) || !d_counts || !d_wfix || !d_scalars)
        return fail(ctx, RT3D_EINVAL, "null device arrays");
    CK(cudaSetDevice(ctx->device));
    rc = ensure_hist(ctx, o->bins);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *sc = ctx->d_hist_u64 + 2 * o->bins;
    CK(launch_histogram(n, d_bundle_out, 6, nullptr, d_bundle_out + 5, o->bins, o->mu_min, o->mu_max,
                        (unsigned long long *)d_counts, (unsigned long long *)d_wfix, sc, d_scalars, st));
    return RT3D_OK;
}

extern "C" int rt3d_load_grid(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos, const double *mass,
                              double soft, const rt3d_grid_opts *g)
{
    if (ctx && field_id >= 0 && field_id < RT3D_MAX_FIELDS && ctx->trace.open &&
        ctx->trace.fs == &ctx->fields[field_id])
        ctx->trace.open = false;  // the open trace's field is replaced
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS) return fail(ctx, RT3D_EINVAL, "field id out of range");
    if (!g) return fail(ctx, RT3D_EINVAL, "null grid options");
    if (g->n_int < 1 || g->n_int > 4) return fail(ctx, RT3D_EINVAL, "n_int must be 1..4");
    if (g->n < 2 * g->n_int || g->n > 1024) return fail(ctx, RT3D_EINVAL, "grid n must be in [2 n_int, 1024]");
    if (!(g->h > 0.0) || !isfinite(g->h) || !isfinite(g->lo[0]) || !isfinite(g->lo[1]) || !isfinite(g->lo[2]))
        return fail(ctx, RT3D_EINVAL, "grid needs h > 0 and a finite origin");
    if (!(soft >= 0.0) || !isfinite(soft)) return fail(ctx, RT3D_EINVAL, "softening must be >= 0");
    if (n < 0 || (n > 0 && (!pos || !mass))) return fail(ctx, RT3D_EINVAL, "null particle arrays");
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(pos[3 * i]) || !isfinite(pos[3 * i + 1]) || !isfinite(pos[3 * i + 2]))
            return fail(ctx, RT3D_EINVAL, "non-finite particle position");
        if (!(mass[i] > 0.0) || !isfinite(mass[i])) return fail(ctx, RT3D_EINVAL, "particle masses must be > 0");
    }
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    FieldSlot &fs = ctx->fields[field_id];
    free_field(fs);
    fs.gd.n = g->n;
    fs.gd.n_int = g->n_int;
    fs.gd.h = g->h;
    for (int d = 0; d < 3; ++d) fs.gd.lo[d] = g->lo[d];
    int rc = grid_build(fs.gd, n, pos, mass, soft, g->mean_subtract ? 1 : 0, ctx->opt.precision == RT3D_FP64,
                        ctx->stream, ctx->err);
    if (rc != RT3D_OK) {
        free_field(fs);
        return rc;
    }
    DevField &df = fs.df;
    df = DevField{};
    df.n = n;
    df.n_rep = 1;
    df.mscale_inv = 1.0;
    df.delta = 1.0;
    df.inv_delta = 1.0;
    fs.n = n;
    fs.is_grid = true;
    fs.loaded = true;
    return RT3D_OK;
}

extern "C" int rt3d_load_grid_box(rt3d_ctx *ctx, int field_id, int64_t n, const double *pos, const double *mass,
                                  double soft, const rt3d_volume *vol, int cubes, const rt3d_grid_opts *g)
{
    if (ctx && field_id >= 0 && field_id < RT3D_MAX_FIELDS && ctx->trace.open &&
        ctx->trace.fs == &ctx->fields[field_id])
        ctx->trace.open = false;  // the open trace's field is replaced
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS) return fail(ctx, RT3D_EINVAL, "field id out of range");
    if (!g || !vol || !vol->replicated) return fail(ctx, RT3D_EINVAL, "a replicated volume and grid options are needed");
    if (g->n_int < 1 || g->n_int > 4) return fail(ctx, RT3D_EINVAL, "n_int must be 1..4");
    if (g->n < 2 * g->n_int || g->n > 512) return fail(ctx, RT3D_EINVAL, "grid n must be in [2 n_int, 512]");
    const double L = vol->box_length;
    if (!(L > 0.0) || !isfinite(L) || vol->n_replicas < 1 || !vol->rot || !vol->shift)
        return fail(ctx, RT3D_EINVAL, "replicated volume needs box_length > 0 and replica transforms");
    if (cubes < 1 || cubes > 64) return fail(ctx, RT3D_EINVAL, "cubes per replica must be 1..64");
    if (!(soft >= 0.0) || !isfinite(soft)) return fail(ctx, RT3D_EINVAL, "softening must be >= 0");
    if (n < 0 || (n > 0 && (!pos || !mass))) return fail(ctx, RT3D_EINVAL, "null particle arrays");
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d)
            if (!(pos[3 * i + d] >= 0.0 && pos[3 * i + d] < L)) return fail(ctx, RT3D_EINVAL, "positions must be in [0, L)");
        if (!(mass[i] > 0.0) || !isfinite(mass[i])) return fail(ctx, RT3D_EINVAL, "particle masses must be > 0");
    }
    const int R = vol->n_replicas;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    FieldSlot &fs = ctx->fields[field_id];
    free_field(fs);
    GridDev &G = fs.gd;
    G.n = g->n;
    G.n_int = g->n_int;
    G.cubes = cubes;
    G.n_rep = R;
    G.L = L;
    G.W = L / cubes;
    G.h = G.W / (g->n - 1);
    G.margin = 1.0;
    int rc = grid_build_box(G, n, pos, mass, soft, vol->rot, vol->shift, g->mean_subtract ? 1 : 0,
                            ctx->opt.precision == RT3D_FP64, ctx->stream, ctx->err);
    if (rc != RT3D_OK) {
        free_field(fs);
        return rc;
    }
    DevField &df = fs.df;
    df = DevField{};
    df.n = n;
    df.n_rep = 1;
    df.mscale_inv = 1.0;
    df.delta = 1.0;
    df.inv_delta = 1.0;
    fs.n = n;
    fs.is_grid = true;
    fs.loaded = true;
    return RT3D_OK;
}

extern "C" int rt3d_grid_nodes(rt3d_ctx *ctx, int field_id, double *out)
{
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS || !ctx->fields[field_id].loaded)
        return fail(ctx, RT3D_ENOFIELD, "field not loaded");
    const FieldSlot &fs = ctx->fields[field_id];
    if (!fs.is_grid) return fail(ctx, RT3D_EINVAL, "not a grid field");
    if (!out) return fail(ctx, RT3D_EINVAL, "null output");
    CK(cudaSetDevice(ctx->device));
    const size_t n3 = (size_t)fs.gd.n * fs.gd.n * fs.gd.n;
    const size_t cells = fs.gd.cubes > 0 ? (size_t)fs.gd.cubes * fs.gd.n_rep : 1;
    std::vector<double> tab(fs.gd.tab ? kGridRec * n3 : 0);
    std::vector<float> tab32(fs.gd.tab ? 0 : kGridRec * n3);
    for (size_t c = 0; c < cells; ++c) {
        if (fs.gd.tab)
            CK(cudaMemcpyAsync(tab.data(), fs.gd.tab + c * kGridRec * n3, tab.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
        else
            CK(cudaMemcpyAsync(tab32.data(), fs.gd.tab32 + c * kGridRec * n3, tab32.size() * sizeof(float),
                               cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        double *o = out + c * 4 * n3;
        for (size_t i = 0; i < n3; ++i)
            for (int f = 0; f < 4; ++f)
                o[f * n3 + i] = fs.gd.tab ? tab[kGridRec * i + f] : (double)tab32[kGridRec * i + f];
    }
    return RT3D_OK;
}

extern "C" int rt3d_born(rt3d_ctx *ctx, int field_id, double z_s, int64_t n_b, const double *theta,
                         const rt3d_bundle_opts *b, double *out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    int rc = check_trace_args(ctx, field_id, z_s, n_b, b);
    if (rc) return rc;
    if (!theta || !out) return fail(ctx, RT3D_EINVAL, "null theta or output");
    for (int64_t i = 0; i < 2 * n_b; ++i)
        if (!isfinite(theta[i])) return fail(ctx, RT3D_EINVAL, "non-finite theta");
    const FieldSlot &fs = ctx->fields[field_id];
    if (fs.is_grid) return fail(ctx, RT3D_ENOTIMPL, "the Born approximation takes particle fields");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int n = b->n_steps;
    // node chunks of about 2^18 points; particle splits for about five waves
    const int K = (int)std::max<int64_t>(1, std::min<int64_t>(n + 1, ((int64_t)1 << 18) / n_b));
    const int64_t blocks = ((int64_t)K * n_b + 511) / 512;
    const int64_t tiles = std::max<int64_t>(1, (fs.n + kTile - 1) / kTile);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)ctx->n_sm * 4 * 5 + blocks - 1) / blocks));
    Scratch &sc = ctx->scr;
    CK(grow(sc.theta, sc.theta_n, (size_t)(2 * n_b)));
    CK(grow(sc.bout, sc.bout_n, (size_t)(6 * n_b)));
    const size_t need = born_scratch_bytes(n_b, n, K, splits);
    CK(grow(*(char **)&sc.partials, sc.partials_bytes, need));
    CK(cudaMemcpyAsync(sc.theta, theta, 2 * n_b * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(born_run(ctx->cosmo, fs.df, fs.n, z_s, n_b, sc.theta, b->schedule, n, b->lens_chi, b->asinh_s, K, splits,
                sc.partials, sc.bout, st));
    CK(cudaMemcpyAsync(out, sc.bout, 3 * n_b * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RT3D_OK;
}

extern "C" int rt3d_watchdog_selftest(rt3d_ctx *ctx, double limit_s)
{
    if (!ctx) return RT3D_EINVAL;
    if (!(limit_s > 0.0) || limit_s > 10.0) return fail(ctx, RT3D_EINVAL, "limit must be in (0, 10] s");
    CK(cudaSetDevice(ctx->device));
    unsigned *d = nullptr;
    CK(cudaMalloc(&d, 2 * sizeof(unsigned)));
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = launch_watchdog_probe(d, (int *)(d + 1), limit_s, st);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d + 1, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    CK(e);
    if (err) return fail(ctx, RT3D_ETIMEOUT, "watchdog self-test: the bounded wait expired as intended");
    return fail(ctx, RT3D_ECUDA, "watchdog self-test: the wait ended without the watchdog");
}

extern "C" int rt3d_potential(rt3d_ctx *ctx, int field_id, int64_t n, const double *pts, const int32_t *rep,
                              double *out)
{
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS || !ctx->fields[field_id].loaded)
        return fail(ctx, RT3D_ENOFIELD, "field not loaded");
    if (n < 1 || !pts || !out) return fail(ctx, RT3D_EINVAL, "need n >= 1 points");
    const FieldSlot &fs = ctx->fields[field_id];
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(pts[3 * i]) || !isfinite(pts[3 * i + 1]) || !isfinite(pts[3 * i + 2]))
            return fail(ctx, RT3D_EINVAL, "non-finite point");
        if (rep && (rep[i] < 0 || rep[i] >= fs.df.n_rep)) return fail(ctx, RT3D_EINVAL, "replica index out of range");
    }
    CK(cudaSetDevice(ctx->device));
    const bool fp64 = ctx->opt.precision == RT3D_FP64;
    ForceShape sh = choose_shape(ctx, fs.df, n, fp64);
    Scratch &s = ctx->scr;
    CK(grow(*(char **)&s.partials, s.partials_bytes, partials_bytes(sh, n, fp64)));
    CK(grow(ctx->d_io, ctx->d_io_n, (size_t)(3 * n + 4 * n + n)));
    double *d_pts = ctx->d_io, *d_out = ctx->d_io + 3 * n;
    int *d_rep = rep ? (int *)(ctx->d_io + 7 * n) : nullptr;
    std::vector<double> soa((size_t)(3 * n));
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) soa[d * n + i] = pts[3 * i + d];
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(d_pts, soa.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (rep) CK(cudaMemcpyAsync(d_rep, rep, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (fs.is_grid) {
        CK(launch_grid_eval(fs.gd, d_pts, d_pts + n, d_pts + 2 * n, n, 2, d_out, nullptr, st));
    } else {
        CK(run_force(ctx, fs.df, d_pts, d_pts + n, d_pts + 2 * n, d_rep, 1, n, sh, fp64, s.partials, nullptr, st));
        CK(launch_stage_field(fs.df, sh, fp64, s.partials, d_pts, d_rep, n, d_out, st));
    }
    CK(cudaMemcpyAsync(out, d_out, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RT3D_OK;
}

extern "C" int rt3d_schedule(rt3d_ctx *ctx, double z_s, int kind, int n_steps, double chi_l, double s,
                             double *dlam_out, double *chi_s_out)
{
    if (!ctx) return RT3D_EINVAL;
    ctx->trace.open = false;  // this call reuses the open trace's scratch
    if (!ctx->have_cosmo) return fail(ctx, RT3D_ENOCOSMO, "set the cosmology first");
    if (!(z_s > 0.0) || n_steps < 1 || !dlam_out || (kind != RT3D_SCHED_UNIFORM && kind != RT3D_SCHED_ASINH) ||
        (kind == RT3D_SCHED_ASINH && !(s > 0.0)))
        return fail(ctx, RT3D_EINVAL, "bad schedule arguments");
    CK(cudaSetDevice(ctx->device));
    Scratch &sc = ctx->scr;
    CK(grow(sc.dlam, sc.dlam_n, (size_t)n_steps));
    cudaStream_t st = ctx->stream;
    CK(launch_schedule(ctx->cosmo, z_s, kind, n_steps, chi_l, s, sc.dlam, sc.misc, st));
    CK(cudaMemcpyAsync(dlam_out, sc.dlam, n_steps * sizeof(double), cudaMemcpyDeviceToHost, st));
    double chi = 0.0;
    CK(cudaMemcpyAsync(&chi, sc.misc, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (chi_s_out) *chi_s_out = chi;
    return RT3D_OK;
}

extern "C" int rt3d_get_stats(rt3d_ctx *ctx, rt3d_stats *out)
{
    if (!ctx || !out) return RT3D_EINVAL;
    CK(cudaSetDevice(ctx->device));
    if (ctx->stats_pending) {
        CK(cudaDeviceSynchronize());
        int rc = finish_stats(ctx);
        if (rc) return rc;
    }
    *out = ctx->stats;
    return RT3D_OK;
}

// ---------------------------------------------------------------------------
// rt3d_potential_device_noalloc: the pair sum with its split partials in a
// static device array instead of context scratch, for callers that cannot
// allocate device memory.  The paper has no counterpart to this entry point.
// ---------------------------------------------------------------------------
#include <mutex>

// Split-K scratch of the no-allocation entry point.  It exists on every device
// that loads this library, for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT3D_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[RT3D_NOALLOC_MAX_DEVICES];

// Device address of g_noalloc_scratch on the current device (set up once per
// device).  In host code the symbol is only a host-side handle, so its device
// address must come from cudaGetSymbolAddress with that device current.
static cudaError_t noalloc_scratch(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

extern "C" int rt3d_potential_device_noalloc(rt3d_ctx *ctx, void *stream, int field_id, int64_t n,
                                             const double *d_pts, const int32_t *d_rep, double *d_out)
{
    if (!ctx) return RT3D_EINVAL;
    if (field_id < 0 || field_id >= RT3D_MAX_FIELDS || !ctx->fields[field_id].loaded)
        return fail(ctx, RT3D_ENOFIELD, "field not loaded");
    if (ctx->fields[field_id].is_grid)
        return fail(ctx, RT3D_ENOTIMPL, "the no-allocation entry point takes particle fields, not grid fields");
    if (n < 1 || !d_pts || !d_out) return fail(ctx, RT3D_EINVAL, "need n >= 1 points and device arrays");
    const int64_t max_points = (int64_t)(RT3D_NOALLOC_SCRATCH_BYTES / 32);
    if (n > max_points) return fail(ctx, RT3D_EINVAL, "rt3d_potential_device_noalloc: at most 1048576 points per call");
    if (ctx->device < 0 || ctx->device >= RT3D_NOALLOC_MAX_DEVICES)
        return fail(ctx, RT3D_EINVAL, "device index beyond the no-allocation table");
    CK(cudaSetDevice(ctx->device));
    void *scratch = nullptr;
    CK(noalloc_scratch(ctx->device, &scratch));
    const FieldSlot &fs = ctx->fields[field_id];
    const bool fp64 = ctx->opt.precision == RT3D_FP64;
    ForceShape sh = choose_shape(ctx, fs.df, n, fp64);
    // keep splits * 4 outputs * n points * 8 bytes inside the static array
    const int64_t cap = (int64_t)(RT3D_NOALLOC_SCRATCH_BYTES / ((size_t)32 * (size_t)n));
    if (sh.splits > cap) {
        const int64_t tiles = std::max<int64_t>(1, (fs.n + kTile - 1) / kTile);
        const int64_t tps = (tiles + cap - 1) / cap;
        sh.splits = (int)std::max<int64_t>(1, (tiles + tps - 1) / tps);
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(run_force(ctx, fs.df, d_pts, d_pts + n, d_pts + 2 * n, (const int *)d_rep, 1, n, sh, fp64, scratch, nullptr, st));
    CK(launch_stage_field(fs.df, sh, fp64, scratch, d_pts, (const int *)d_rep, n, d_out, st));
    return RT3D_OK;
}

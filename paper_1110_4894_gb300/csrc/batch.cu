// batch.cu -- many independent light cones (each with its own particle field,
// source redshift, bundles and step table) traced in one persistent launch.
//
// The persistent kernel is a cooperative launch of one resident grid.  For
// every global RK4 stage it runs two phases separated by grid barriers:
//   force phase: every (cone, ray block, particle split) work item of the
//                cones still in flight, taken from a work queue (an atomic
//                counter) by whichever block is free, largest items first;
//   stage phase: the FP64 integrator stage of every ray of those cones.
// Cones whose rays have all crossed their source plane drop out; cones with
// fewer steps simply finish earlier.  The barrier waits are bounded by a
// %globaltimer watchdog: on expiry the kernel sets an error word and returns,
// and the host reports RT3D_ETIMEOUT.
#include "batch_layout.cuh"
#include "grid_device.cuh"
#include "force.cuh"
#include "trace_device.cuh"

namespace rt3d {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *word differs from old; give up when *err is set or limit_ns
// has elapsed (then set *err, so every other waiter stops too).  True if
// the word changed.
__device__ __forceinline__ bool bounded_wait(const volatile unsigned *word, unsigned old, int *err,
                                             unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    while (*word == old) {
        if (*(volatile int *)err) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

// Grid-wide barrier of a cooperative launch; every wait is bounded.
__device__ __forceinline__ bool grid_sync(const BatchArgs &B)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = B.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(B.bar, 1u) == gridDim.x - 1) {
            atomicExch(B.bar, 0u);
            __threadfence();
            atomicAdd(B.bar + 1, 1u);
        } else {
            bounded_wait(gen, g0, B.err, B.limit_ns);
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)B.err == 0;
}

// Watchdog check: one thread waits, with the barrier's bounded wait, on a
// word that nothing changes; the wait must end after limit_ns with *err set.
__global__ void k_watchdog_probe(unsigned *word, int *err, unsigned long long limit_ns)
{
    bounded_wait(word, *(volatile unsigned *)word, err, limit_ns);
}

cudaError_t launch_watchdog_probe(unsigned *d_word, int *d_err, double limit_s, cudaStream_t st)
{
    k_watchdog_probe<<<1, 1, 0, st>>>(d_word, d_err, (unsigned long long)(limit_s * 1e9));
    return cudaGetLastError();
}

__device__ __forceinline__ bool cone_active(const BatchCone &C, int step)
{
    if (step >= C.total_steps) return false;
    if (step < C.tp.n_steps) return true;
    return *(volatile unsigned long long *)&C.cnt[(step - 1) & 1] != 0ull;
}

__global__ void k_batch_schedule(BatchArgs B)
{
    BatchCone &C = B.cones[blockIdx.y];
    __shared__ double s_chi;
    if (threadIdx.x == 0) {
        s_chi = comoving_distance(C.tp.cosmo, C.z_s);
        if (blockIdx.x == 0) C.chi_s = s_chi;
    }
    __syncthreads();
    const int n = C.tp.n_steps;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        C.dlam[k] = schedule_step(C.tp.cosmo, C.kind, n, k, s_chi, C.chi_l, C.s_asinh);
}

__global__ void k_batch_init(BatchArgs B)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.T) return;
    const BatchCone &C = B.cones[B.rb2cone[r / B.RB]];
    const int64_t local = r - C.ray_base;
    if (local >= C.rs.n_rays) return;
    if (local == 0) C.cnt[0] = C.cnt[1] = C.cnt[2] = 0ull;
    init_ray(C.tp, C.f, C.theta, C.rs, local);
}

// MODE 4 / 8: bundle-centric kernel for rings of 4 / 8 rays; MODE 5: the
// expanded two-bundle kernel for rings of 4 (block = 2 NT bundles); MODE 0:
// packed
template <int P, int NT, int MODE>
__device__ __forceinline__ void batch_item(const BatchCone &C, int4 item, int g, float4 *s_a, float4 *s_b,
                                           float2 *s_e, float2 *s_hl)
{
    const int64_t p0 = (int64_t)item.z * C.per_split;
    const int64_t p1 = min(C.f.n, p0 + C.per_split);
    const int64_t st = C.rs.stride;
    const double *px = C.rs.ys + st, *py = C.rs.ys + 2 * st, *pz = C.rs.ys + 3 * st;
    const int *rep = C.rs.rep + (g & 1) * C.rs.n_b;
    if constexpr (MODE == 5) {
        const int64_t b0 = (int64_t)item.y * 2 * NT;
#define RT3D_XITEM(R_, E_, U_)                                                                                   \
    bundle2x_block_sum<NT, 4, R_, E_, U_, 1, false>(C.f, px, py, pz, rep, C.rs.n_b, C.rs.n_rays, b0, p0, p1,      \
                                                    item.z, C.partials, s_a, s_b, (float *)s_e, s_hl)
        switch (C.flags) {
        case 0: RT3D_XITEM(false, false, false); break;
        case 1: RT3D_XITEM(true, false, false); break;
        case 2: RT3D_XITEM(false, true, false); break;
        case 3: RT3D_XITEM(true, true, false); break;
        case 4: RT3D_XITEM(false, false, true); break;
        case 5: RT3D_XITEM(true, false, true); break;
        case 6: RT3D_XITEM(false, true, true); break;
        default: RT3D_XITEM(true, true, true); break;
        }
#undef RT3D_XITEM
        return;
    }
    if (MODE != 0) {  // bundle-centric: block = NT bundles
        const int64_t b0 = (int64_t)item.y * NT;
#define RT3D_BITEM(NRING_, R_, E_, U_)                                                                          \
    bundle_block_sum<NT, NRING_, R_, E_, U_>(C.f, px, py, pz, rep, C.rs.n_b, C.rs.n_rays, b0, p0, p1, item.z,   \
                                             C.partials, s_a, (float *)s_e)
#define RT3D_BFLAGS(NRING_)                                          \
    switch (C.flags) {                                               \
    case 0: RT3D_BITEM(NRING_, false, false, false); break;          \
    case 1: RT3D_BITEM(NRING_, true, false, false); break;           \
    case 2: RT3D_BITEM(NRING_, false, true, false); break;           \
    case 3: RT3D_BITEM(NRING_, true, true, false); break;            \
    case 4: RT3D_BITEM(NRING_, false, false, true); break;           \
    case 5: RT3D_BITEM(NRING_, true, false, true); break;            \
    case 6: RT3D_BITEM(NRING_, false, true, true); break;            \
    default: RT3D_BITEM(NRING_, true, true, true); break;            \
    }
        RT3D_BFLAGS(MODE == 8 ? 8 : 4)
#undef RT3D_BFLAGS
#undef RT3D_BITEM
        return;
    }
    const int64_t base = (int64_t)item.y * (NT * 2 * P);
#define RT3D_ITEM(R_, E_, U_)                                                                                   \
    packed_block_sum<P, NT, R_, E_, U_>(C.f, px, py, pz, rep, C.rs.nr, C.rs.n_rays, base, p0, p1, item.z,        \
                                        C.partials, s_a, s_b, s_e)
    switch (C.flags) {
    case 0: RT3D_ITEM(false, false, false); break;
    case 1: RT3D_ITEM(true, false, false); break;
    case 2: RT3D_ITEM(false, true, false); break;
    case 3: RT3D_ITEM(true, true, false); break;
    case 4: RT3D_ITEM(false, false, true); break;
    case 5: RT3D_ITEM(true, false, true); break;
    case 6: RT3D_ITEM(false, true, true); break;
    default: RT3D_ITEM(true, true, true); break;
    }
#undef RT3D_ITEM
}

// The grid evaluation of ray block rb of a grid cone into its one split of
// partials.  Not inlined: its registers stay out of the pair-sum code's
// allocation.
__device__ __noinline__ void batch_grid_item(const BatchCone &C, int rb, int RB, int NT)
{
    const int64_t st = C.rs.stride;
    const int64_t r1 = min(C.rs.n_rays, (int64_t)(rb + 1) * RB);
    for (int64_t i = (int64_t)rb * RB + threadIdx.x; i < r1; i += NT) {
        float F[4];
        grid_eval32_any(C.g, C.rs.ys + st, C.rs.ys + 2 * st, C.rs.ys + 3 * st, i, C.rs.nr, F);
#pragma unroll
        for (int o = 0; o < 4; ++o) C.partials[(int64_t)o * C.rs.n_rays + i] = make_float2(-F[o], 0.0f);
    }
}

template <int P, int NT, int MODE>
__global__ void __launch_bounds__(NT, MODE == 5 ? 6 : 1) k_batch_run(BatchArgs B)
{
    __shared__ float4 s_a[kTile];
    __shared__ float4 s_b[kTile];
    __shared__ float2 s_e[kTile];
    __shared__ float2 s_hl[MODE == 5 ? 2 * (5 * 3 + 4) * NT : 1];
    __shared__ unsigned s_it;
    const int64_t nthreads = (int64_t)gridDim.x * NT;
    for (int g = 0; g < B.g_end; ++g) {
        const int step = g >> 2, stage = g & 3;
        // work queue of this stage's force items (largest first, as planned):
        // each block takes the next item when it is free.  The counter of the
        // next stage is the one stage g-1 used, finished before the barriers
        // that ended it, so it is reset here.
        unsigned *queue = B.bar + 4;
        if (blockIdx.x == 0 && threadIdx.x == 0) queue[(g + 1) & 1] = 0u;
        for (;;) {
            if (threadIdx.x == 0) s_it = atomicAdd(&queue[g & 1], 1u);
            __syncthreads();
            const int64_t it = s_it;
            __syncthreads();
            if (it >= B.n_items) break;
            const int4 item = B.items[it];
            const BatchCone &C = B.cones[item.x];
            if (!cone_active(C, step)) continue;  // uniform across the block
            if (item.z < 0) {  // the prism records of NT bundles (FP64)
                const int64_t b = (int64_t)item.y * NT + threadIdx.x;
                if (b < C.rs.n_b) bundle_prism(C.f, C.rs, g, b, C.prism);
                continue;
            }
            if (item.w == 1) {  // a grid cone: App. B evaluation of one ray block (one split)
                batch_grid_item(C, item.y, B.RB, NT);
                continue;
            }
            batch_item<P, NT, MODE>(C, item, g, s_a, s_b, s_e, s_hl);
        }
        if (!grid_sync(B)) return;
        for (int64_t r = (int64_t)blockIdx.x * NT + threadIdx.x; r < B.T; r += nthreads) {
            const int c = B.rb2cone[r / B.RB];
            const BatchCone &C = B.cones[c];
            const int64_t local = r - C.ray_base;
            bool act = false;
            if (local < C.rs.n_rays) {
                if (stage == 0 && local == 0) C.cnt[step & 1] = 0ull;
                if (cone_active(C, step))
                    act = stage_ray(C.tp, C.f, C.rs, C.S, false, C.mfac, C.partials, C.dlam, C.chi_s, step, stage,
                                    C.cnt, local, nullptr, C.prism);
            }
            // ray blocks are multiples of 32 rays, so a warp never spans two cones
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if ((threadIdx.x & 31) == 0 && m) atomicAdd(&C.cnt[2], (unsigned long long)__popc(m));
        }
        if (!grid_sync(B)) return;
    }
}

__global__ void k_batch_reduce(BatchArgs B, int64_t n_b_total)
{
    const int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= n_b_total) return;
    int lo = 0, hi = B.n_cones - 1;
    while (lo < hi) {  // last cone whose first bundle is <= gb
        const int mid = (lo + hi + 1) / 2;
        if (B.cones[mid].b_base <= gb) lo = mid;
        else hi = mid - 1;
    }
    const BatchCone &C = B.cones[lo];
    const int64_t b = gb - C.b_base;
    reduce_bundle(C.tp, C.theta, C.rs, C.chi_s, b, B.bout + 6 * gb, C.rout);
}

// ---------------------------------------------------------------------------
// launch wrappers (the host orchestration lives in api.cu)
// ---------------------------------------------------------------------------
template <int NT, int MODE>
static cudaError_t batch_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_run<2, NT, MODE>, NT, 0);
}

template <int NT, int MODE>
static cudaError_t batch_coop(const cudaLaunchConfig_t &cfg, const BatchArgs &B)
{
    return cudaLaunchKernelEx(&cfg, k_batch_run<2, NT, MODE>, B);
}

#define RT3D_BATCH_SHAPES(F, ...)                                              \
    if (NT == 64 && MODE == 5) e = F<64, 5>(__VA_ARGS__);                      \
    else if (NT == 128 && MODE == 4) e = F<128, 4>(__VA_ARGS__);               \
    else if (NT == 256 && MODE == 4) e = F<256, 4>(__VA_ARGS__);               \
    else if (NT == 64 && MODE == 4) e = F<64, 4>(__VA_ARGS__);                 \
    else if (NT == 128 && MODE == 8) e = F<128, 8>(__VA_ARGS__);               \
    else if (NT == 64 && MODE == 8) e = F<64, 8>(__VA_ARGS__);                 \
    else if (NT == 128 && MODE == 0) e = F<128, 0>(__VA_ARGS__);               \
    else if (NT == 256 && MODE == 0) e = F<256, 0>(__VA_ARGS__);               \
    else if (NT == 64 && MODE == 0) e = F<64, 0>(__VA_ARGS__);                 \
    else e = cudaErrorInvalidConfiguration;

cudaError_t batch_resident_blocks(int NT, int MODE, int *out)
{
    int dev = 0, sms = 0, per = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    RT3D_BATCH_SHAPES(batch_occupancy, &per)
    if (e != cudaSuccess) return e;
    *out = per * sms;
    return cudaSuccess;
}

cudaError_t batch_launch(const BatchArgs &B, int NT, int MODE, int grid, int max_sched_steps, int64_t n_b_total,
                         cudaStream_t st)
{
    cudaError_t e;
    {
        int bx = (max_sched_steps + 127) / 128;
        if (bx > 64) bx = 64;
        k_batch_schedule<<<dim3((unsigned)std::max(bx, 1), (unsigned)B.n_cones), 128, 0, st>>>(B);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_batch_init<<<(unsigned)((B.T + 255) / 256), 256, 0, st>>>(B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RT3D_BATCH_SHAPES(batch_coop, cfg, B)
    if (e != cudaSuccess) return e;
    k_batch_reduce<<<(unsigned)((n_b_total + 127) / 128), 128, 0, st>>>(B, n_b_total);
    return cudaGetLastError();
}
#undef RT3D_BATCH_SHAPES

}  // namespace rt3d

// force_bundle2x.cu -- launch dispatch of the two-bundles-per-thread pair sum
// with ring separations expanded about the central ray (rings of 4 and 8).
#include "force.cuh"

namespace rt3d {

template <int NT, int NRING, bool UMASS, bool REPL, bool PEPS, int T, int CL, bool AHEAD>
static cudaError_t go_one(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    const auto kern = k_force_bundle2x<NT, NRING, REPL, PEPS, UMASS, T, CL, AHEAD>;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, NT, 0);
    if (CL == 1) {
        kern<<<grid, NT, 0, st>>>(A);
        return cudaGetLastError();
    }
    // thread-block clusters of CL consecutive splits of one bundle block
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CL;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A);
}

template <int NT, int NRING, bool UMASS, int T, int CL, bool AHEAD>
static cudaError_t go_fields(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) return go_one<NT, NRING, UMASS, true, true, T, CL, AHEAD>(A, grid, st, occ);
    if (repl) return go_one<NT, NRING, UMASS, true, false, T, CL, AHEAD>(A, grid, st, occ);
    if (peps) return go_one<NT, NRING, UMASS, false, true, T, CL, AHEAD>(A, grid, st, occ);
    return go_one<NT, NRING, UMASS, false, false, T, CL, AHEAD>(A, grid, st, occ);
}

// Rings of 4, both block sizes: bounded for 384 resident threads per SM (168
// registers, no spills).  With the particle records read one iteration ahead,
// three warps per scheduler keep the FP32 pipe busier than four at 128
// registers, where the read-ahead spills (on the 2^24-particle box, 128-thread
// blocks: 0.778 of the FP32 peak against 0.770 for 512 threads without the
// read-ahead, 0.745 with it, and 0.746 for 384 threads without it)
template <int NT, bool UMASS, int CL>
static cudaError_t go_bundle2x(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    return go_fields<NT, 4, UMASS, 384, CL, true>(A, grid, st, occ);
}

// Rings of 8 (the paper's bundle of 8 rays around the central one): 64
// threads, no clusters; the 35 compensated sums and 32 ring-offset registers
// per bundle pair need about twice the registers of a ring of 4, so the
// bound is 256 resident threads (255 registers; at 320 or 384 the allocation
// falls to 168 and spills).  Without the read-ahead: 0.732 of the FP32 peak
// against 0.723 with it on 65,536 bundles of the 2^24-particle box.
constexpr int kRing8Threads = 256;
constexpr bool kRing8Ahead = false;
template <bool UMASS>
static cudaError_t go_bundle2x8(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    return go_fields<64, 8, UMASS, kRing8Threads, 1, kRing8Ahead>(A, grid, st, occ);
}

// rings of 4 (R = 5) or 8 (R = 9): grid.x counts blocks of 2 NT bundles,
// grid.y the splits (a multiple of sh.cl).  With occ set nothing is launched:
// *occ receives the kernel's resident blocks per SM.
cudaError_t dispatch_bundle2x(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st, int *occ)
{
    if ((sh.R != 5 && sh.R != 9) || sh.splits % sh.cl != 0) return cudaErrorInvalidConfiguration;
    const int64_t n_b = A.n / sh.R;
    const dim3 grid((unsigned)((n_b + 2 * sh.NT - 1) / (2 * sh.NT)), (unsigned)sh.splits);
    if (sh.R == 9) {
        if (sh.NT != 64 || sh.cl != 1) return cudaErrorInvalidConfiguration;
        return umass ? go_bundle2x8<true>(A, grid, st, occ) : go_bundle2x8<false>(A, grid, st, occ);
    }
    switch ((sh.NT * 2 + (umass ? 1 : 0)) * 8 + sh.cl) {
    case 128 * 8 + 1: return go_bundle2x<64, false, 1>(A, grid, st, occ);
    case 129 * 8 + 1: return go_bundle2x<64, true, 1>(A, grid, st, occ);
    case 256 * 8 + 1: return go_bundle2x<128, false, 1>(A, grid, st, occ);
    case 257 * 8 + 1: return go_bundle2x<128, true, 1>(A, grid, st, occ);
    case 128 * 8 + 4: return go_bundle2x<64, false, 4>(A, grid, st, occ);
    case 129 * 8 + 4: return go_bundle2x<64, true, 4>(A, grid, st, occ);
    case 256 * 8 + 4: return go_bundle2x<128, false, 4>(A, grid, st, occ);
    case 257 * 8 + 4: return go_bundle2x<128, true, 4>(A, grid, st, occ);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace rt3d

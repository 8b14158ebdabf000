// force_bundle2x.cu -- launch dispatch of the two-bundles-per-thread pair sum
// with ring separations expanded about the central ray.
#include "force.cuh"

namespace rt3d {

template <int NT, bool UMASS, bool REPL, bool PEPS, int T, int CL>
static cudaError_t go_one(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_force_bundle2x<NT, 4, REPL, PEPS, UMASS, T, CL>,
                                                                  NT, 0);
    if (CL == 1) {
        k_force_bundle2x<NT, 4, REPL, PEPS, UMASS, T, 1><<<grid, NT, 0, st>>>(A);
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
    return cudaLaunchKernelEx(&cfg, k_force_bundle2x<NT, 4, REPL, PEPS, UMASS, T, CL>, A);
}

// Both block sizes are bounded for 384 resident threads per SM (168
// registers, no spills).  With the particle records read one iteration ahead,
// three warps per scheduler keep the FP32 pipe busier than four at 128
// registers, where the read-ahead spills (on the 2^24-particle box, 128-thread
// blocks: 0.778 of the FP32 peak against 0.770 for 512 threads without the
// read-ahead, 0.745 with it, and 0.746 for 384 threads without it)
template <int NT, bool UMASS, int CL>
static cudaError_t go_bundle2x(const ForceArgs &A, dim3 grid, cudaStream_t st, int *occ)
{
    constexpr int T = 384;
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) return go_one<NT, UMASS, true, true, T, CL>(A, grid, st, occ);
    if (repl) return go_one<NT, UMASS, true, false, T, CL>(A, grid, st, occ);
    if (peps) return go_one<NT, UMASS, false, true, T, CL>(A, grid, st, occ);
    return go_one<NT, UMASS, false, false, T, CL>(A, grid, st, occ);
}

// rings of 4: grid.x counts blocks of 2 NT bundles, grid.y the splits (a
// multiple of sh.cl).  With occ set nothing is launched: *occ receives the
// kernel's resident blocks per SM.
cudaError_t dispatch_bundle2x(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st, int *occ)
{
    const int64_t n_b = A.n / 5;
    const dim3 grid((unsigned)((n_b + 2 * sh.NT - 1) / (2 * sh.NT)), (unsigned)sh.splits);
    if (sh.R != 5 || sh.splits % sh.cl != 0) return cudaErrorInvalidConfiguration;
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

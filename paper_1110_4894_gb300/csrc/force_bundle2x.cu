// force_bundle2x.cu -- launch dispatch of the two-bundles-per-thread pair sum
// with ring separations expanded about the central ray.
#include "force.cuh"

namespace rt3d {

// 64-thread blocks are bounded for 6 blocks per SM (168 registers), 128-thread
// blocks for 2 (no spills): the tuner times both register regimes
template <int NT, bool UMASS>
static cudaError_t go_bundle2x(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    constexpr int T = NT == 64 ? 384 : 256;
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_force_bundle2x<NT, 4, true, true, UMASS, T><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_bundle2x<NT, 4, true, false, UMASS, T><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_bundle2x<NT, 4, false, true, UMASS, T><<<grid, NT, 0, st>>>(A);
    else k_force_bundle2x<NT, 4, false, false, UMASS, T><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

// rings of 4: grid.x counts blocks of 2 NT bundles
cudaError_t dispatch_bundle2x(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st)
{
    const int64_t n_b = A.n / 5;
    const dim3 grid((unsigned)((n_b + 2 * sh.NT - 1) / (2 * sh.NT)), (unsigned)sh.splits);
    if (sh.R != 5) return cudaErrorInvalidConfiguration;
    switch (sh.NT * 2 + (umass ? 1 : 0)) {
    case 128: return go_bundle2x<64, false>(A, grid, st);
    case 129: return go_bundle2x<64, true>(A, grid, st);
    case 256: return go_bundle2x<128, false>(A, grid, st);
    case 257: return go_bundle2x<128, true>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace rt3d

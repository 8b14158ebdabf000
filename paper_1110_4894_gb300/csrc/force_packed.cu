// force_packed.cu -- launch dispatch of the packed (FP32x2) pair-sum kernel.
#include "force.cuh"

namespace rt3d {

template <int P, int NT, bool UMASS>
static cudaError_t go_packed(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_force_packed<P, NT, true, true, UMASS><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_packed<P, NT, true, false, UMASS><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_packed<P, NT, false, true, UMASS><<<grid, NT, 0, st>>>(A);
    else k_force_packed<P, NT, false, false, UMASS><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

template <bool UMASS>
static cudaError_t pick(const ForceArgs &A, const ForceShape &sh, dim3 grid, cudaStream_t st)
{
    switch (sh.R * 1000 + sh.NT) {
    case 4064: return go_packed<2, 64, UMASS>(A, grid, st);
    case 4128: return go_packed<2, 128, UMASS>(A, grid, st);
    case 4256: return go_packed<2, 256, UMASS>(A, grid, st);
    case 8064: return go_packed<4, 64, UMASS>(A, grid, st);
    case 8128: return go_packed<4, 128, UMASS>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t dispatch_packed(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st)
{
    const int64_t per_block = (int64_t)sh.R * sh.NT;
    const dim3 grid((unsigned)((A.n + per_block - 1) / per_block), (unsigned)sh.splits);
    return umass ? pick<true>(A, sh, grid, st) : pick<false>(A, sh, grid, st);
}

}  // namespace rt3d

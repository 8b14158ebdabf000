// force_mixed.cu -- launch dispatch of the mixed-precision pair-sum kernel.
#include "force.cuh"

namespace rt3d {

template <int R, int NT>
static cudaError_t go_mixed(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_force_mixed<R, NT, true, true><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_mixed<R, NT, true, false><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_mixed<R, NT, false, true><<<grid, NT, 0, st>>>(A);
    else k_force_mixed<R, NT, false, false><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t dispatch_mixed(const ForceArgs &A, const ForceShape &sh, cudaStream_t st)
{
    const int64_t per_block = (int64_t)sh.R * sh.NT;
    const dim3 grid((unsigned)((A.n + per_block - 1) / per_block), (unsigned)sh.splits);
    switch (sh.R * 1000 + sh.NT) {
    case 1128: return go_mixed<1, 128>(A, grid, st);
    case 2128: return go_mixed<2, 128>(A, grid, st);
    case 2256: return go_mixed<2, 256>(A, grid, st);
    case 4064: return go_mixed<4, 64>(A, grid, st);
    case 4128: return go_mixed<4, 128>(A, grid, st);
    case 4256: return go_mixed<4, 256>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace rt3d

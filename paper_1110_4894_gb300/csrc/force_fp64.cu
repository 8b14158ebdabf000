// force_fp64.cu -- launch dispatch of the all-FP64 pair-sum kernel.
#include "force.cuh"

namespace rt3d {

template <int R, int NT>
static cudaError_t go_fp64(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2_64 != nullptr;
    if (repl && peps) k_force_fp64<R, NT, true, true><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_fp64<R, NT, true, false><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_fp64<R, NT, false, true><<<grid, NT, 0, st>>>(A);
    else k_force_fp64<R, NT, false, false><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t dispatch_fp64(const ForceArgs &A, const ForceShape &sh, cudaStream_t st)
{
    const int64_t per_block = (int64_t)sh.R * sh.NT;
    const dim3 grid((unsigned)((A.n + per_block - 1) / per_block), (unsigned)sh.splits);
    switch (sh.R * 1000 + sh.NT) {
    case 1128: return go_fp64<1, 128>(A, grid, st);
    case 2128: return go_fp64<2, 128>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace rt3d

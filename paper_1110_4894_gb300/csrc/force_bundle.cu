// force_bundle.cu -- launch dispatch of the bundle-centric pair-sum kernel.
#include "force.cuh"

namespace rt3d {

template <int NT, int NRING, bool UMASS>
static cudaError_t go_bundle(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_force_bundle<NT, NRING, true, true, UMASS><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_bundle<NT, NRING, true, false, UMASS><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_bundle<NT, NRING, false, true, UMASS><<<grid, NT, 0, st>>>(A);
    else k_force_bundle<NT, NRING, false, false, UMASS><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

template <int NRING, bool UMASS>
static cudaError_t pick(const ForceArgs &A, const ForceShape &sh, dim3 grid, cudaStream_t st)
{
    switch (sh.NT) {
    case 64: return go_bundle<64, NRING, UMASS>(A, grid, st);
    case 128: return go_bundle<128, NRING, UMASS>(A, grid, st);
    case 256: return go_bundle<256, NRING, UMASS>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

template <int NT, bool UMASS>
static cudaError_t go_bundle2(const ForceArgs &A, dim3 grid, cudaStream_t st)
{
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_force_bundle2<NT, 4, true, true, UMASS><<<grid, NT, 0, st>>>(A);
    else if (repl) k_force_bundle2<NT, 4, true, false, UMASS><<<grid, NT, 0, st>>>(A);
    else if (peps) k_force_bundle2<NT, 4, false, true, UMASS><<<grid, NT, 0, st>>>(A);
    else k_force_bundle2<NT, 4, false, false, UMASS><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

// two bundles per thread (rings of 4): grid.x counts blocks of 2 NT bundles
cudaError_t dispatch_bundle2(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st)
{
    const int64_t n_b = A.n / 5;
    const dim3 grid((unsigned)((n_b + 2 * sh.NT - 1) / (2 * sh.NT)), (unsigned)sh.splits);
    if (sh.R != 5) return cudaErrorInvalidConfiguration;
    switch (sh.NT * 2 + (umass ? 1 : 0)) {
    case 128: return go_bundle2<64, false>(A, grid, st);
    case 129: return go_bundle2<64, true>(A, grid, st);
    case 256: return go_bundle2<128, false>(A, grid, st);
    case 257: return go_bundle2<128, true>(A, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

// sh.R carries the rays per bundle (5 or 9); grid.x counts bundle blocks
cudaError_t dispatch_bundle(const ForceArgs &A, const ForceShape &sh, bool umass, cudaStream_t st)
{
    const int64_t n_b = A.n / sh.R;
    const dim3 grid((unsigned)((n_b + sh.NT - 1) / sh.NT), (unsigned)sh.splits);
    if (sh.R == 5) return umass ? pick<4, true>(A, sh, grid, st) : pick<4, false>(A, sh, grid, st);
    if (sh.R == 9) return umass ? pick<8, true>(A, sh, grid, st) : pick<8, false>(A, sh, grid, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace rt3d

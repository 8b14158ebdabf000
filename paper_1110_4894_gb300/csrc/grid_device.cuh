// grid_device.cuh -- the mixed path's App. B evaluation of one point from a
// grid's FP32 node table, shared by the grid kernel and the batched kernel.
#pragma once
#include "rt3d_internal.cuh"

namespace rt3d {

// Weights c of the natural cubic spline through W unit-spaced values y,
// evaluated at u in [0, W-1], in FP32: S(u) = sum_j c[j] y[j].  The second
// derivatives of the spline through the unit vector e_j solve
// z[i-1] + 4 z[i] + z[i+1] = 6 (e[i+1] - 2 e[i] + e[i-1]) with z = 0 at the
// ends; they are constants of W.
template <int W>
__device__ __forceinline__ void spline_weights_f(float u, float (&c)[W])
{
    int k = (int)floorf(u);
    k = k > W - 2 ? W - 2 : k;
    k = k < 0 ? 0 : k;
    const float A = (float)(k + 1) - u, B = u - (float)k;
    const float cA = (A * A * A - A) * (1.0f / 6.0f), cB = (B * B * B - B) * (1.0f / 6.0f);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        float z[W];
        z[0] = 0.0f;
        z[W - 1] = 0.0f;
        if (W >= 3) {
            float den[W], dp = 0.0f, cp = 0.0f;
#pragma unroll
            for (int i = 1; i <= W - 2; ++i) {
                const float e = (i + 1 == j ? 1.0f : 0.0f) - 2.0f * (i == j ? 1.0f : 0.0f) + (i - 1 == j ? 1.0f : 0.0f);
                den[i] = 4.0f - cp;
                cp = 1.0f / den[i];
                dp = (6.0f * e - dp) / den[i];
                z[i] = dp;
            }
#pragma unroll
            for (int i = W - 3; i >= 1; --i) z[i] = z[i] - z[i + 1] / den[i];
        }
        float zk = z[0], zk1 = z[1];
#pragma unroll
        for (int i = 1; i < W - 1; ++i)
            if (k == i) {
                zk = z[i];
                zk1 = z[i + 1];
            }
        c[j] = (j == k ? A : 0.0f) + (j == k + 1 ? B : 0.0f) + (cA * zk + cB * zk1);
    }
}

// phi and grad phi (F[0..3]) at point i from the FP32 node table: App. B's
// interpolation with FP32 weights and sums; the cube (box grids: the one
// holding the x3 of the first point of i's group, the bundle's central ray),
// node window and fractional offsets come from FP64 coordinates.  Zero
// outside the node range widened by g.margin.
template <int NI>
__device__ __forceinline__ void grid_eval32_point(const GridDev &g, const double *__restrict__ px,
                                                  const double *__restrict__ py, const double *__restrict__ pz,
                                                  int64_t i, int group, float F[4])
{
    constexpr int W = 2 * NI;
    const int n = g.n;
    const double r[3] = {px[i], py[i], pz[i]};
    double lo[3] = {g.lo[0], g.lo[1], g.lo[2]};
    const float *tab = g.tab32;
    if (g.cubes > 0) {
        const double x3 = pz[(i / group) * group];
        double q = floor(x3 / g.L);
        const int j = q < 0.0 ? 0 : (q > (double)(g.n_rep - 1) ? g.n_rep - 1 : (int)q);
        double cq = floor((x3 - (double)j * g.L) / g.W);
        const int c = cq < 0.0 ? 0 : (cq > (double)(g.cubes - 1) ? g.cubes - 1 : (int)cq);
        lo[0] = -0.5 * g.W;
        lo[1] = -0.5 * g.W;
        lo[2] = (double)j * g.L + (double)c * g.W;
        tab += ((int64_t)j * g.cubes + c) * kGridRec * (int64_t)n * n * n;
    }
    double u[3];
    int s[3];
    bool inside = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        u[d] = (r[d] - lo[d]) / g.h;
        inside = inside && (u[d] >= -g.margin && u[d] <= (double)(n - 1) + g.margin);
        int sd = inside ? (int)floor(u[d]) - NI + 1 : 0;
        sd = sd > n - W ? n - W : sd;
        s[d] = sd < 0 ? 0 : sd;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) F[f] = 0.0f;
    if (!inside) return;
    int k3 = (int)floor(u[2]);
    k3 = k3 > n - 2 ? n - 2 : k3;
    k3 = k3 < 0 ? 0 : k3;
    const float B = (float)(u[2] - (double)k3), A = 1.0f - B;
    const float cA = (A * A * A - A) * (1.0f / 6.0f), cB = (B * B * B - B) * (1.0f / 6.0f);
    float c1[W], c2[W];
    spline_weights_f<W>((float)(u[0] - (double)s[0]), c1);
    spline_weights_f<W>((float)(u[1] - (double)s[1]), c2);
#pragma unroll
    for (int b = 0; b < W; ++b) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < W; ++a) {
            // along x3 on node line (s1 + a, s2 + b): the global spline from
            // nodes k3 and k3 + 1 (values, then second derivatives)
            const int64_t node = ((int64_t)(s[0] + a) * n + (s[1] + b)) * n + k3;
            const float4 *p = reinterpret_cast<const float4 *>(tab + kGridRec * node);
            const float4 v = __ldg(p), y = __ldg(p + 1), w = __ldg(p + 2), z = __ldg(p + 3);
            // along x1
            acc[0] += c1[a] * (A * v.x + B * w.x + (cA * y.x + cB * z.x));
            acc[1] += c1[a] * (A * v.y + B * w.y + (cA * y.y + cB * z.y));
            acc[2] += c1[a] * (A * v.z + B * w.z + (cA * y.z + cB * z.z));
            acc[3] += c1[a] * (A * v.w + B * w.w + (cA * y.w + cB * z.w));
        }
        // along x2
#pragma unroll
        for (int f = 0; f < 4; ++f) F[f] += c2[b] * acc[f];
    }
}

// grid_eval32_point for the grid's n_int (1..4)
__device__ __forceinline__ void grid_eval32_any(const GridDev &g, const double *__restrict__ px,
                                                const double *__restrict__ py, const double *__restrict__ pz,
                                                int64_t i, int group, float F[4])
{
    switch (g.n_int) {
    case 1: grid_eval32_point<1>(g, px, py, pz, i, group, F); break;
    case 2: grid_eval32_point<2>(g, px, py, pz, i, group, F); break;
    case 3: grid_eval32_point<3>(g, px, py, pz, i, group, F); break;
    default: grid_eval32_point<4>(g, px, py, pz, i, group, F); break;
    }
}

}  // namespace rt3d

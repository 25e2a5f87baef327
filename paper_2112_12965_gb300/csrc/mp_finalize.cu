// K4: finalisation of the dictionary AB-join.
//
// Per query window i it
//   1. reduces the column groups' partial maxima of q = C * invstd_b (the
//      element-wise minimum of Algorithm 2, Sec. 3.2, over the distance
//      d^2 = 2m - 2 invstd_a q), keeping the lowest window index on ties;
//   2. applies the constant-window convention (a constant window normalises
//      to the zero vector: d = sqrt(m) against a non-constant window, 0
//      against a constant one);
//   3. recomputes the chosen pair's distance from its definition,
//      sqrt(sum_k (z_a[k] - z_b[k])^2), so the reported value carries no
//      error from the recurrence or the tensor-core products, only from the
//      choice of the pair.
// One warp per query window: the lanes split the m terms of the sum.
#include <math.h>

#include "mp_internal.cuh"

namespace mpd {
namespace {

// Exact-as-practical distance of query window i and dictionary window g.
__device__ __forceinline__ double pair_distance(const float *a, int64_t i, double mu_a, double is_a, const float *b,
                                                int64_t g, double mu_b, double is_b, int m, int lane)
{
    // Split each FP64 mean into two floats so the centring is accurate to
    // FP32 relative to the centred values, even for series with big offsets.
    const float ma_hi = (float)mu_a, ma_lo = (float)(mu_a - (double)ma_hi);
    const float mb_hi = (float)mu_b, mb_lo = (float)(mu_b - (double)mb_hi);
    const float sa = (float)is_a, sb = (float)is_b;
    float acc = 0.f;
    for (int k = lane; k < m; k += 32) {
        const float za = ((a[i + k] - ma_hi) - ma_lo) * sa;
        const float zb = ((b[g + k] - mb_hi) - mb_lo) * sb;
        const float d = za - zb;
        acc = fmaf(d, d, acc);
    }
    double t = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return sqrt(t);
}

__device__ __forceinline__ double pair_distance(const double *a, int64_t i, double mu_a, double is_a,
                                                const double *b, int64_t g, double mu_b, double is_b, int m, int lane)
{
    double acc = 0.0;
    for (int k = lane; k < m; k += 32) {
        const double d = (a[i + k] - mu_a) * is_a - (b[g + k] - mu_b) * is_b;
        acc = fma(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return sqrt(acc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_finalize(int64_t nq, int32_t m, int32_t n_groups,
                                                  const Partial<T> *__restrict__ part, const T *__restrict__ a,
                                                  const double *__restrict__ mean_a,
                                                  const double *__restrict__ invstd_a,
                                                  const uint8_t *__restrict__ cflag_a, const T *__restrict__ b,
                                                  const double *__restrict__ mean_b,
                                                  const double *__restrict__ invstd_b, int64_t g_const,
                                                  int64_t g_first, double *__restrict__ out_dist,
                                                  int64_t *__restrict__ out_idx)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sqrt_m = sqrt((double)m);
    for (int64_t i = warp_global; i < nq; i += nwarps) {
        // 1. reduce the column groups: largest q, then lowest g
        T q = T(-INFINITY);
        int32_t g = -1;
        for (int k = lane; k < n_groups; k += 32) {
            const Partial<T> v = part[(int64_t)k * nq + i];
            if (v.g >= 0 && (g < 0 || v.q > q || (v.q == q && v.g < g))) {
                q = v.q;
                g = v.g;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T q2 = __shfl_xor_sync(0xffffffffu, q, o);
            const int32_t g2 = __shfl_xor_sync(0xffffffffu, g, o);
            if (g2 >= 0 && (g < 0 || q2 > q || (q2 == q && g2 < g))) {
                q = q2;
                g = g2;
            }
        }
        // 2. constant-window convention and 3. exact distance of the pick
        double d = INFINITY;
        int64_t gi = -1;
        if (g_first >= 0) {
            if (cflag_a[i]) {
                if (g_const >= 0) {
                    d = 0.0;
                    gi = g_const;
                } else {
                    d = sqrt_m;
                    gi = g_first;
                }
            } else {
                if (g >= 0) {
                    d = pair_distance(a, i, mean_a[i], invstd_a[i], b, g, mean_b[g], invstd_b[g], m, lane);
                    gi = g;
                }
                if (g_const >= 0 && (gi < 0 || sqrt_m < d || (sqrt_m == d && g_const < gi))) {
                    d = sqrt_m;
                    gi = g_const;
                }
            }
        }
        if (lane == 0) {
            out_dist[i] = d;
            out_idx[i] = gi;
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_finalize(int64_t nq, int32_t m, int32_t n_groups, const Partial<T> *part, const T *a,
                            const double *mean_a, const double *invstd_a, const uint8_t *cflag_a, const T *b,
                            const double *mean_b, const double *invstd_b, int64_t g_const, int64_t g_first,
                            double *out_dist, int64_t *out_idx, cudaStream_t st)
{
    if (nq <= 0) return cudaSuccess;
    int64_t grid = (nq + 7) / 8;  // 8 warps (rows) per CTA
    if (grid > 152 * 32) grid = 152 * 32;
    k_finalize<T><<<(unsigned)grid, 256, 0, st>>>(nq, m, n_groups, part, a, mean_a, invstd_a, cflag_a, b, mean_b,
                                                  invstd_b, g_const, g_first, out_dist, out_idx);
    return cudaGetLastError();
}

template cudaError_t launch_finalize<float>(int64_t, int32_t, int32_t, const Partial<float> *, const float *,
                                            const double *, const double *, const uint8_t *, const float *,
                                            const double *, const double *, int64_t, int64_t, double *, int64_t *,
                                            cudaStream_t);
template cudaError_t launch_finalize<double>(int64_t, int32_t, int32_t, const Partial<double> *, const double *,
                                             const double *, const double *, const uint8_t *, const double *,
                                             const double *, const double *, int64_t, int64_t, double *, int64_t *,
                                             cudaStream_t);

}  // namespace mpd

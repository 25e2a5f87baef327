// K1: per-window statistics for the z-normalised distance.
//
// The z-normalised Euclidean distance (Sec. 2.1) needs each window's mean and
// population standard deviation. They are kept in FP64 because sums of
// squares cancel badly in FP32 when a series carries a large offset (random
// walks). Each CTA handles a tile of consecutive windows:
//   1. the tile's samples are read with coalesced 16-byte vector loads,
//      shifted by the tile's first sample (the statistics are shift
//      invariant, and the shift keeps the prefix sums small) and staged in
//      shared memory;
//   2. a block-wide prefix sum gives, for every window, sum(y) and sum(y^2)
//      over its m samples in O(1);
//   3. an integer prefix count of neighbouring samples that differ gives the
//      exact constant-window flag.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "mp_internal.cuh"

namespace mpd {
namespace {

constexpr int kStatsThreads = 256;
constexpr int kStatsTile = 1024;  // windows per CTA (halved down to 128 while the grid is small)

__device__ __forceinline__ double block_exclusive_scan(double v, double *warp_tot, double *total)
{
    __syncthreads();  // warp_tot may still be read by the previous scan
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        double w = lane < (kStatsThreads / 32) ? warp_tot[lane] : 0.0;
        double wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (kStatsThreads / 32)) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == (kStatsThreads / 32) - 1) *total = wi;
    }
    __syncthreads();
    return warp_tot[wid] + incl - v;
}

__device__ __forceinline__ int block_exclusive_scan_int(int v, int *warp_tot)
{
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (kStatsThreads / 32) ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (kStatsThreads / 32)) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    return warp_tot[wid] + incl - v;
}

// 1/sqrt(v) to FP64 accuracy: FP32 estimate refined by two Newton steps.
__device__ __forceinline__ double rsqrt_fp64(double v)
{
    double y = (double)rsqrtf((float)v);
    y = y * (1.5 - 0.5 * v * y * y);
    y = y * (1.5 - 0.5 * v * y * y);
    return y;
}

template <typename T>
__global__ void __launch_bounds__(kStatsThreads) k_window_stats(const T *__restrict__ x, int64_t n, int32_t m,
                                                                 double *__restrict__ mean,
                                                                 double *__restrict__ invstd,
                                                                 uint8_t *__restrict__ cflag,
                                                                 vec4_t<T> *__restrict__ rs,
                                                                 Split<T> *__restrict__ ms, int32_t tile)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t nw = n - m + 1;
    const int64_t w0 = (int64_t)blockIdx.x * tile;
    const int tw = (nw - w0 < tile) ? (int)(nw - w0) : tile;
    // Samples e = 0 .. E-1 hold x[w0 - 1 + e]; e = 0 is the sample before the
    // tile (needed for the previous window's mean), absent for the first tile.
    const int E = tw + m;
    double *ys = reinterpret_cast<double *>(smem_raw);  // E + 1 entries, reused as prefix of y
    double *p2 = ys + (E + 1);                           // E + 1 entries: prefix of y^2
    int *pc = reinterpret_cast<int *>(p2 + (E + 1));     // E + 1 entries: prefix of "differs from next"
    __shared__ double warp_tot[kStatsThreads / 32];
    __shared__ int warp_tot_i[kStatsThreads / 32];
    __shared__ double tot;

    // The tile's samples, read with 16-byte vector loads (the ragged ends,
    // samples outside [0, n) and unaligned series take scalar loads): each
    // thread shifts its samples and compares each with the next (the next
    // vector's first sample is one more, cached, load).
    constexpr int V = 16 / sizeof(T);
    using VecT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const double shift = (double)x[w0];
    const int64_t base = w0 - 1;  // sample of e = 0
    const bool vec_ok = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    const int64_t a0 = (base >= 0 ? base : base - (V - 1)) / V * V;  // base rounded down to a vector
    const int nvec = (int)((base + E - a0 + V - 1) / V);
    for (int v = threadIdx.x; v < nvec; v += kStatsThreads) {
        const int64_t g = a0 + (int64_t)v * V;
        T vals[V + 1];
        if (vec_ok && g >= 0 && g + V <= n) {
            const VecT u = *reinterpret_cast<const VecT *>(x + g);
            memcpy(vals, &u, sizeof u);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) vals[k] = (g + k >= 0 && g + k < n) ? x[g + k] : T(0);
        }
        vals[V] = (g + V >= 0 && g + V < n) ? x[g + V] : T(0);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int64_t e = g + k - base, j = g + k;
            if (e >= 0 && e < E) {
                ys[e] = (j >= 0 && j < n) ? (double)vals[k] - shift : 0.0;
                pc[e] = (e + 1 < E && j >= 0 && j + 1 < n && vals[k] != vals[k + 1]) ? 1 : 0;
            }
        }
    }
    __syncthreads();

    // Each thread owns a contiguous chunk of the E samples.
    const int per = (E + kStatsThreads - 1) / kStatsThreads;
    const int e_lo = min(E, (int)threadIdx.x * per), e_hi = min(E, e_lo + per);
    double s1 = 0.0, s2 = 0.0;
    int sc = 0;
    for (int e = e_lo; e < e_hi; ++e) {
        const double y = ys[e];
        s1 += y;
        s2 += y * y;
        sc += pc[e];
    }
    const double o1 = block_exclusive_scan(s1, warp_tot, &tot);
    const double o2 = block_exclusive_scan(s2, warp_tot, &tot);
    const int oc = block_exclusive_scan_int(sc, warp_tot_i);
    // Local values are still needed: compute the exclusive prefixes in
    // registers first, write them after a barrier (ys is overwritten in place).
    __syncthreads();
    {
        double a1 = o1, a2 = o2;
        int ac = oc;
        for (int e = e_lo; e < e_hi; ++e) {
            const double y = ys[e];
            const int d = pc[e];
            ys[e] = a1;  // exclusive prefix: sum of y over [0, e)
            p2[e] = a2;
            pc[e] = ac;
            a1 += y;
            a2 += y * y;
            ac += d;
        }
        if (e_hi == E && e_lo < e_hi) {
            ys[E] = a1;
            p2[E] = a2;
            pc[E] = ac;
        }
    }
    __syncthreads();

    const double inv_m = 1.0 / (double)m;
    for (int t = threadIdx.x; t < tw; t += kStatsThreads) {
        const int64_t i = w0 + t;
        // window i covers e in [t + 1, t + 1 + m)
        const double S1 = ys[t + 1 + m] - ys[t + 1];
        const double S2 = p2[t + 1 + m] - p2[t + 1];
        const int nchg = pc[t + m] - pc[t + 1];
        const double mu_s = S1 * inv_m;  // mean relative to the shift
        double var = S2 * inv_m - mu_s * mu_s;
        const bool is_const = (nchg == 0);
        if (!is_const && !(var > 1e-4 * (S2 * inv_m + 1e-300))) {
            // The one-pass formula cancelled more than four digits (a window
            // whose spread is tiny next to its distance from the tile's
            // shift): redo it with two passes over the window's samples.
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += (double)x[i + k] - shift;
            const double mu2 = s * inv_m;
            double v = 0.0;
            for (int k = 0; k < m; ++k) {
                const double d = ((double)x[i + k] - shift) - mu2;
                v += d * d;
            }
            var = v * inv_m;
        }
        double inv_s = 0.0;
        if (!is_const && var > 0.0) inv_s = (var > 1e-30 && var < 1e30) ? rsqrt_fp64(var) : 1.0 / sqrt(var);
        const double mu = shift + mu_s;
        mean[i] = mu;
        invstd[i] = inv_s;
        cflag[i] = is_const ? 1 : 0;
        if (ms) {
            Split<T> sp;
            sp.hi = (T)mu;
            sp.lo = (T)(mu - (double)sp.hi);
            ms[i] = sp;
        }
        if (rs) {
            vec4_t<T> r;
            if (i == 0) {
                r.x = T(0);
                r.y = T(0);
            } else {
                // previous window i-1 covers e in [t, t + m)
                const double mu_prev_s = (ys[t + m] - ys[t]) * inv_m;
                const double y_new = ys[t + 1 + m] - ys[t + m];  // sample i+m-1, shifted
                const double y_old = ys[t + 1] - ys[t];          // sample i-1, shifted
                r.x = T(0.5 * (y_new - y_old));
                r.y = T((y_new - mu_s) + (y_old - mu_prev_s));
            }
            r.z = T(inv_s);
            r.w = is_const ? T(-INFINITY) : T(0);
            rs[i] = r;
        }
    }
}

template <typename T>
__global__ void k_check_finite(const T *__restrict__ x, int64_t n, int32_t *bad)
{
    bool ok = true;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ok &= isfinite((double)x[i]);
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

// Positions of the concatenated dictionary whose window crosses a segment end
// (or lies in a segment shorter than m) are not dictionary windows (Def. 8):
// give them score weight 0 and penalty -inf so that no kernel can select them.
template <typename T>
__global__ void k_mark_invalid(vec4_t<T> *__restrict__ rs, int64_t npos, const int64_t *__restrict__ offs,
                               int32_t nseg, int32_t m)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < npos; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nseg;  // find s with offs[s] <= g < offs[s+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offs[mid] <= g) lo = mid; else hi = mid;
        }
        if (g + m > offs[lo + 1]) {
            vec4_t<T> v = rs[g];
            v.z = T(0);
            v.w = T(-INFINITY);
            rs[g] = v;
        }
    }
}

__global__ void k_dict_specials(const Span *__restrict__ spans, int32_t n_spans, const uint8_t *__restrict__ cflag,
                                unsigned long long *out)
{
    for (int s = blockIdx.x; s < n_spans; s += gridDim.x) {
        const Span sp = spans[s];
        if (threadIdx.x == 0 && sp.ncols > 0) atomicMin(&out[1], (unsigned long long)sp.g0);
        for (int c = threadIdx.x; c < sp.ncols; c += blockDim.x)
            if (cflag[sp.g0 + c]) atomicMin(&out[0], (unsigned long long)(sp.g0 + c));
    }
}

}  // namespace

template <typename T>
cudaError_t launch_window_stats(const T *x, int64_t n, int32_t m, double *mean, double *invstd, uint8_t *cflag,
                                vec4_t<T> *rs, Split<T> *ms, cudaStream_t st)
{
    const int64_t nw = n - m + 1;
    if (nw <= 0) return cudaSuccess;
    // smaller tiles for short series, so that a short query's statistics
    // spread over many SMs instead of running in one CTA
    int tile = kStatsTile;
    while (tile > 128 && (nw + tile - 1) / tile < 512) tile >>= 1;
    const int64_t grid = (nw + tile - 1) / tile;
    const int E = tile + m;
    const size_t smem = (size_t)(E + 1) * (2 * sizeof(double) + sizeof(int));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_window_stats<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_window_stats<T><<<(unsigned)grid, kStatsThreads, smem, st>>>(x, n, m, mean, invstd, cflag, rs, ms, tile);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const T *x, int64_t n, int32_t *bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_check_finite<T><<<(unsigned)grid, 256, 0, st>>>(x, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_dict_specials(const Span *spans, int32_t n_spans, const uint8_t *cflag, int64_t *out,
                                 cudaStream_t st)
{
    // out[] must hold INT64_MAX-like sentinels (all ones) before the call.
    if (n_spans <= 0) return cudaSuccess;
    k_dict_specials<<<n_spans < 1024 ? n_spans : 1024, 256, 0, st>>>(spans, n_spans, cflag,
                                                                      reinterpret_cast<unsigned long long *>(out));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mark_invalid(vec4_t<T> *rs, int64_t npos, const int64_t *seg_offsets, int32_t n_segments,
                                int32_t m, cudaStream_t st)
{
    if (npos <= 0 || n_segments <= 0) return cudaSuccess;
    int64_t grid = (npos + 255) / 256;
    if (grid > 8192) grid = 8192;
    k_mark_invalid<T><<<(unsigned)grid, 256, 0, st>>>(rs, npos, seg_offsets, n_segments, m);
    return cudaGetLastError();
}
template cudaError_t launch_mark_invalid<float>(float4 *, int64_t, const int64_t *, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_mark_invalid<double>(dvec4 *, int64_t, const int64_t *, int32_t, int32_t, cudaStream_t);

template cudaError_t launch_window_stats<float>(const float *, int64_t, int32_t, double *, double *, uint8_t *,
                                                float4 *, Split<float> *, cudaStream_t);
template cudaError_t launch_window_stats<double>(const double *, int64_t, int32_t, double *, double *, uint8_t *,
                                                 dvec4 *, Split<double> *, cudaStream_t);
template cudaError_t launch_check_finite<float>(const float *, int64_t, int32_t *, cudaStream_t);
template cudaError_t launch_check_finite<double>(const double *, int64_t, int32_t *, cudaStream_t);

}  // namespace mpd

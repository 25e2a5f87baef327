// Kernels of dictionary learning (Algorithm 1, Sec. 3.1).
//
// Algorithm 1 starts from the self-join matrix profile P_B of the training
// series T_B (computed by the plain join kernels with an exclusion zone) and
// repeats: take the window j that minimises P_B - S outside the exclusion
// zones of the windows already taken, add it (with context) to the
// dictionary, and fold the distance profile of T_B against window j into S
// by an element-wise minimum. The kernels here are the per-iteration steps:
//   k_learn_argmin   argmin over i of P_B[i] - S[i] (+inf where excluded),
//                    lowest i on ties;
//   k_learn_profile  S'[i] = d(T_B window i, T_B window j) for every i, then
//                    S = S' (first iteration) or min(S, S'), and max(S);
// and the suffix table used by the self-join's constant-window rule:
//   next_const[x] = the lowest constant window >= x, or -1.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "mp_internal.cuh"

namespace mpd {
namespace {

constexpr int kNcBlock = 1024;

// Order-preserving map of a float to an unsigned key (larger float, larger key).
__device__ __forceinline__ uint32_t float_key(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Pass 1: per block of kNcBlock positions, the lowest constant position >= x
// inside the block (INT64_MAX if none), and the block's first constant.
__global__ void __launch_bounds__(kNcBlock) k_nc_local(const uint8_t *__restrict__ cflag, int64_t npos,
                                                       int64_t *__restrict__ local, int64_t *__restrict__ first)
{
    __shared__ int64_t v[kNcBlock];
    const int t = threadIdx.x;
    const int64_t x = (int64_t)blockIdx.x * kNcBlock + t;
    v[t] = (x < npos && cflag[x]) ? x : INT64_MAX;
    __syncthreads();
    // suffix minimum within the block
    for (int off = 1; off < kNcBlock; off <<= 1) {
        const int64_t o = t + off < kNcBlock ? v[t + off] : INT64_MAX;
        __syncthreads();
        if (o < v[t]) v[t] = o;
        __syncthreads();
    }
    if (x < npos) local[x] = v[t];
    if (t == 0) first[blockIdx.x] = v[0];
}

// Pass 2 (one thread): after[b] = the lowest constant position in blocks > b.
__global__ void k_nc_blocks(const int64_t *__restrict__ first, int64_t nblk, int64_t *__restrict__ after)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t run = INT64_MAX;
    for (int64_t b = nblk - 1; b >= 0; --b) {
        after[b] = run;
        if (first[b] < run) run = first[b];
    }
}

// Pass 3: combine.
__global__ void k_nc_final(const int64_t *__restrict__ local, const int64_t *__restrict__ after, int64_t npos,
                           int64_t *__restrict__ next_const)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= npos) return;
    int64_t v = local[x];
    if (v == INT64_MAX) v = after[x / kNcBlock];
    next_const[x] = v == INT64_MAX ? -1 : v;
}

// argmin over i < n of (excluded[i] ? +inf : P[i] - S[i]) into *best as the
// packed key (order key of the value << 32) | i; *best must start at ~0.
__global__ void __launch_bounds__(256) k_learn_argmin(const double *__restrict__ P, const float *__restrict__ S,
                                                      const uint8_t *__restrict__ excluded, int64_t n,
                                                      unsigned long long *__restrict__ best)
{
    unsigned long long mine = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (excluded[i]) continue;
        const float v = (float)(P[i] - (double)S[i]);
        if (!(v < INFINITY)) continue;  // +inf (a row without any window) or NaN: not a candidate
        const unsigned long long k = ((unsigned long long)float_key(v) << 32) | (unsigned long long)(uint32_t)i;
        if (k < mine) mine = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k = __shfl_xor_sync(0xffffffffu, mine, o);
        if (k < mine) mine = k;
    }
    if ((threadIdx.x & 31) == 0 && mine != ~0ull) atomicMin(best, mine);
}

// S'[i] = d(window i, window j) of one series from its statistics; S becomes
// S' (first) or min(S, S'); *smax (order key) receives the largest S[i].
// The dot products are FP32 on centred samples: window j is centred on its
// mean (split) in shared memory, window i is shifted by its mean's hi part,
// and sum_k (x_i - hi_i)(x_j - mu_j) = cov + (mu_i - hi_i) sum_k (x_j - mu_j).
__global__ void __launch_bounds__(256) k_learn_profile(const float *__restrict__ x, int64_t nq, int32_t m,
                                                       const Split<float> *__restrict__ ms,
                                                       const float4 *__restrict__ rs, const uint8_t *__restrict__ cflag,
                                                       int64_t j, float *__restrict__ S, int32_t first,
                                                       uint32_t *__restrict__ smax)
{
    extern __shared__ float qc[];  // window j, centred
    __shared__ float qsum_s;
    const Split<float> mj = ms[j];
    for (int k = threadIdx.x; k < m; k += blockDim.x) qc[k] = (x[j + k] - mj.hi) - mj.lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < m; ++k) t += qc[k];
        qsum_s = t;
    }
    __syncthreads();
    const float qsum = qsum_s;
    const bool cj = cflag[j] != 0;
    const float isj = rs[j].z;
    const float sqrt_m = sqrtf((float)m);
    uint32_t mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        float d;
        const bool ci = cflag[i] != 0;
        if (ci || cj) {
            d = (ci && cj) ? 0.f : sqrt_m;  // the zero-vector convention for constant windows
        } else {
            const Split<float> mi = ms[i];
            const float *xi = x + i;
            float acc = 0.f;
            for (int k = 0; k < m; ++k) acc = fmaf(xi[k] - mi.hi, qc[k], acc);
            const float cov = acc - mi.lo * qsum;
            const float rho = cov * rs[i].z * isj / (float)m;
            d = sqrtf(fmaxf(0.f, 2.f * (float)m * (1.f - rho)));
        }
        const float s = first ? d : fminf(S[i], d);
        S[i] = s;
        const uint32_t k = float_key(s);
        if (k > mx) mx = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t k = __shfl_xor_sync(0xffffffffu, mx, o);
        if (k > mx) mx = k;
    }
    if ((threadIdx.x & 31) == 0 && mx != 0) atomicMax(smax, mx);
}

}  // namespace

cudaError_t launch_next_const(const uint8_t *cflag, int64_t npos, int64_t *next_const, int64_t *scratch,
                              cudaStream_t st)
{
    if (npos <= 0) return cudaSuccess;
    const int64_t nblk = (npos + kNcBlock - 1) / kNcBlock;
    int64_t *local = scratch, *first = scratch + npos, *after = first + nblk;
    k_nc_local<<<(unsigned)nblk, kNcBlock, 0, st>>>(cflag, npos, local, first);
    k_nc_blocks<<<1, 1, 0, st>>>(first, nblk, after);
    k_nc_final<<<(unsigned)((npos + 255) / 256), 256, 0, st>>>(local, after, npos, next_const);
    return cudaGetLastError();
}

size_t next_const_scratch_elems(int64_t npos) { return (size_t)npos + 2 * (size_t)((npos + kNcBlock - 1) / kNcBlock); }

cudaError_t launch_learn_argmin(const double *P, const float *S, const uint8_t *excluded, int64_t n,
                                unsigned long long *best, int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(best, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)sm_count * 8) grid = (int64_t)sm_count * 8;
    k_learn_argmin<<<(unsigned)std::max<int64_t>(1, grid), 256, 0, st>>>(P, S, excluded, n, best);
    return cudaGetLastError();
}

float learn_key_float(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

cudaError_t launch_learn_profile(const float *x, int64_t nq, int32_t m, const Split<float> *ms, const float4 *rs,
                                 const uint8_t *cflag, int64_t j, float *S, bool first, uint32_t *smax, int sm_count,
                                 cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    int64_t grid = (nq + 255) / 256;
    if (grid > (int64_t)sm_count * 16) grid = (int64_t)sm_count * 16;
    const size_t smem = sizeof(float) * (size_t)m;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_learn_profile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_learn_profile<<<(unsigned)std::max<int64_t>(1, grid), 256, smem, st>>>(x, nq, m, ms, rs, cflag, j, S,
                                                                             first ? 1 : 0, smax);
    return cudaGetLastError();
}

}  // namespace mpd

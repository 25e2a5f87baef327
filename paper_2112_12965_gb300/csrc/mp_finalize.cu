// K4: finalisation of the dictionary AB-join.
//
// Per query window i it
//   1. reduces the column groups' partial maxima of q = C * invstd_b (the
//      element-wise minimum of Algorithm 2, Sec. 3.2, over the distance
//      d^2 = 2m - 2 invstd_a q), keeping the lowest window index on ties;
//   2. re-scores the kChunk dictionary windows of the winning chunk with
//      direct dot products (the join kernels keep only a running maximum and
//      the chunk that raised it) and takes their argmax, lowest g on ties;
//      with the plain kernel's near-tie records it re-scores every chunk whose
//      approximate score came within the near-tie width of the best as well;
//   3. applies the constant-window convention (a constant window normalises
//      to the zero vector: d = sqrt(m) against a non-constant window, 0
//      against a constant one);
//   4. recomputes the chosen pair's distance from its definition,
//      sqrt(sum_k (z_a[k] - z_b[k])^2), so the reported value carries no
//      error from the recurrence or the tensor-core products, only from the
//      choice of the pair.
// For m <= 512 (k_finalize_blk) a CTA takes blocks of consecutive query
// windows: steps 1 and 3 run one thread per window, step 2 one warp per
// window; for longer windows (k_finalize) one warp takes each window.
#include <math.h>

#include "mp_internal.cuh"

namespace mpd {
namespace {

// Distance of query window i and dictionary window g from the definition,
// sqrt(sum_k (z_a[k] - z_b[k])^2). Samples are centred with the split means
// (hi, then lo), so the centring is accurate to T's relative precision even
// for series with large offsets; lanes split the m terms.
template <typename T>
__device__ __forceinline__ double pair_distance(const T *a, int64_t i, Split<T> ma, T is_a, const T *b, int64_t g,
                                                Split<T> mb, T is_b, int m, int lane)
{
    T acc = T(0);
    for (int k = lane; k < m; k += 32) {
        const T za = ((a[i + k] - ma.hi) - ma.lo) * is_a;
        const T zb = ((b[g + k] - mb.hi) - mb.lo) * is_b;
        const T d = za - zb;
        acc = fma(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return (double)sqrt(acc);
}

// k values staged per pass of the re-scoring, and the padded shared-memory
// index (one pad slot every 16 values: lanes reading with a stride of 16
// values hit distinct banks).
constexpr int kFinChunk = 256;
__device__ __forceinline__ int fpad(int e) { return e + (e >> 4); }
constexpr int kFinWarpVals = (kFinChunk + kChunk) + ((kFinChunk + kChunk) >> 4) + 1;

template <typename T>
__device__ __forceinline__ bool better(T q1, int32_t g1, T q2, int32_t g2)
{
    // (q1, g1) beats (q2, g2): valid, larger score, or equal score and lower index
    return g1 >= 0 && (g2 < 0 || q1 > q2 || (q1 == q2 && g1 < g2));
}

// The warp's best (score, window) under better(), in every lane: the largest
// score, then the lowest window; (-inf, -1) when no lane has a candidate. The
// scores hold no NaN. FP32 scores take two reductions (redux.sync) of a key
// whose unsigned order is the floats' order, with 0 for no candidate; FP64
// scores a butterfly of shuffles.
template <typename T>
__device__ __forceinline__ void warp_best(T &sc, int32_t &gw)
{
    if constexpr (sizeof(T) == 4) {
        const uint32_t u = __float_as_uint(sc + 0.0f);  // -0 becomes +0: the keys then order as better() does
        const uint32_t key = gw < 0 ? 0u : ((u & 0x80000000u) ? ~u : (u | 0x80000000u));
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
        const int32_t gmin = __reduce_min_sync(0xffffffffu, key == kmax ? gw : 0x7fffffff);
        const uint32_t ub = (kmax & 0x80000000u) ? (kmax & 0x7fffffffu) : ~kmax;
        sc = kmax == 0u ? T(-INFINITY) : __uint_as_float(ub);
        gw = kmax == 0u ? -1 : gmin;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T s2 = __shfl_xor_sync(0xffffffffu, sc, o);
            const int32_t g2 = __shfl_xor_sync(0xffffffffu, gw, o);
            if (better(s2, g2, sc, gw)) {
                sc = s2;
                gw = g2;
            }
        }
    }
}

// Self-join helpers (excl > 0; the dictionary is the one series, so every
// position 0 .. npos_b - 1 is a valid window): the lowest constant window and
// the lowest window outside query window i's exclusion zone, -1 if none.
// With excl = 0 they are the dictionary's g_const and g_first.
template <typename T>
__device__ __forceinline__ int64_t const_outside(const FinalizeParams<T> &p, int64_t i)
{
    if (p.excl == 0 || p.g_const < 0) return p.g_const;
    if (p.g_const <= i - p.excl) return p.g_const;  // the lowest constant window lies before the zone
    const int64_t x = i + p.excl;
    return x < p.npos_b ? p.next_const[x] : -1;
}
template <typename T>
__device__ __forceinline__ int64_t first_outside(const FinalizeParams<T> &p, int64_t i)
{
    if (p.excl == 0 || p.g_first < 0) return p.g_first;
    if (p.g_first <= i - p.excl) return p.g_first;
    const int64_t x = i + p.excl;
    return x < p.npos_b ? x : -1;
}


// Re-score the kChunk windows g .. g + kChunk - 1 of one chunk (dictionary
// samples pb) against query window i (samples pa, split mean ma) with direct
// dot products and return (in every lane) the largest score cov * invstd_b
// among its valid non-constant windows and that window, lowest g on ties
// (-inf / -1 if none). The warp stages the shifted query
// window and the candidates' samples in shared memory (wa, wb) with
// coalesced loads, kFinChunk values of k at a time. Each half-warp takes 8
// candidates; lane l of a half sums the products of a contiguous run of k
// for its 8 candidates (a sliding window of dictionary samples in
// registers), and a transposing butterfly leaves candidate 8 * half + (l & 7)'s
// total in lane l.
template <typename T>
__device__ __forceinline__ void rescore_chunk(const T *__restrict__ pa, const T *__restrict__ pb, int64_t nb,
                                              int64_t npos_b, int m, const Split<T> *__restrict__ ms_b,
                                              const vec4_t<T> *__restrict__ rs_b, int64_t i, int32_t g,
                                              const Split<T> ma, int lane, T *wa, T *wb, T &sc_out,
                                              int32_t &g_out, int excl)
{
    const T sa = ma.hi, sb = ms_b[g].hi;
    const int half = lane >> 4, lg = lane & 15;
    T acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = T(0);
    for (int kc = 0; kc < m; kc += kFinChunk) {
        const int len = min(kFinChunk, m - kc);
        for (int e = lane; e < len; e += 32) wa[fpad(e)] = pa[i + kc + e] - sa;
        for (int e = lane; e < len + kChunk; e += 32) {
            const int64_t j = (int64_t)g + kc + e;
            wb[fpad(e)] = (j < nb) ? pb[j] - sb : T(0);
        }
        __syncwarp();
        const int kpl = (len + 15) >> 4;
        const int k0 = lg * kpl;
        const int k1 = min(len, k0 + kpl);
        T bw[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) bw[c] = (k0 < k1) ? wb[fpad(8 * half + k0 + c)] : T(0);
        for (int kb = k0; kb < k1; kb += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = kb + u;
                if (k < k1) {
                    const T av = wa[fpad(k)];
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[c] = fma(av, bw[(c + u) & 7], acc[c]);
                    bw[u] = wb[fpad(8 * half + k + 8)];
                }
            }
        }
        __syncwarp();  // the next pass (or chunk) overwrites the staged samples
    }
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
#pragma unroll
        for (int c = 0; c < s; ++c) {
            const bool up = (lane & s) != 0;
            const T send = up ? acc[c] : acc[c + s];
            const T keep = up ? acc[c + s] : acc[c];
            acc[c] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 8);  // the two k-halves of the 16 lanes
    const int cand = 8 * half + (lane & 7);
    const int64_t gc = (int64_t)g + cand;
    bool ok = gc < npos_b && (excl == 0 || (gc - i >= excl || i - gc >= excl));
    vec4_t<T> r;
    if (ok) {
        r = rs_b[gc];
        ok = r.w == T(0);
    }
    T sc = T(-INFINITY);
    if (ok) {
        // sum_k (a - sa)(b - sb) = cov + m (mean_a - sa)(mean_b - sb)
        const Split<T> mb = ms_b[gc];
        const T cov = acc[0] - T(m) * ma.lo * ((mb.hi - sb) + mb.lo);
        sc = cov * r.z;
        ok = sc == sc;  // NaN (products that overflowed): not a candidate
        sc = ok ? sc : T(-INFINITY);
    }
    // with NaN out, better() is a total order and every lane ends with the
    // same (score, window)
    int32_t gw = ok ? (int32_t)gc : -1;
    warp_best(sc, gw);
    sc_out = sc;
    g_out = gw;
}

// Entry e of query window i's near-tie candidates, with per = S + 1 entries per
// column group k = e / per: entry 0 is the group's winning chunk, entry u > 0
// its record u - 1. Returns the chunk if it differs from the overall winner g
// and its approximate score reaches lim, else -1; sets ovf if group k's
// records overflowed (tested at entry 1).
template <typename T>
__device__ __forceinline__ int32_t near_entry(const FinalizeParams<T> &p, int64_t i, int64_t e, int per, int64_t tot,
                                              int32_t g, T lim, bool &ovf)
{
    if (e >= tot) return -1;
    const int64_t k = e / per;
    const int u = (int)(e - k * per);
    if (u == 0) {
        const Partial<T> v = p.part[k * p.nq + i];
        return (v.g >= 0 && v.g != g && v.q >= lim) ? v.g : -1;
    }
    const NearSlot *h = p.near.head(k, i);
    const int32_t f = h->g;
    if (u == 1 && (f & kNearOverflow)) ovf = true;
    if (u - 1 >= (f & kNearCountMask)) return -1;
    const NearSlot sl = h[(int64_t)u * p.near.ld];
    return (sl.g != g && T(sl.q) >= lim) ? sl.g : -1;
}

// Near-tie width of query window i in units of its score q, the width the
// join used (NearRec): the plain form's rho m std_a, or the tensor-core
// forms' bound 2 u m sqrt(std_a^2 + da^2) F_b, da = mean_a - s_a with s_a the
// shift of the window's CTA of kTcRows windows.
template <typename T>
__device__ __forceinline__ T near_width(const FinalizeParams<T> &p, int64_t i, T isa, const Split<T> &ma)
{
    if (p.near.fb == nullptr) return T(p.near.rho) * T(p.m) / isa;
    const T s_a = p.ms_a[(i / kTcRows) * kTcRows].hi;
    const T da = (ma.hi - s_a) + ma.lo;
    const T sd = T(1) / isa;
    return T(2) * T(p.near.u) * T(p.m) * sqrt(fma(sd, sd, da * da)) * T(*p.near.fb);
}

// The window range [g_lo, g_hi) of column group k's chunks (its spans or
// tiles in increasing order), as the join kernel saw it for the overflow mask.
template <typename T>
__device__ __forceinline__ void group_range(const FinalizeParams<T> &p, int k, int64_t &g_lo, int64_t &g_hi)
{
    const int s0 = p.cgroup_start[k], s1 = p.cgroup_start[k + 1];
    g_lo = s0 < s1 ? p.cspans[s0].g0 : 0;
    g_hi = s0 < s1 ? p.cspans[s1 - 1].g0 + p.cspans[s1 - 1].ncols : 0;
}

// Add a CTA's counters (shared) to the global ones; every thread calls it.
__device__ __forceinline__ void flush_counters(unsigned long long *ctr, unsigned long long *s_ctr)
{
    __syncthreads();
    if (ctr != nullptr && threadIdx.x < kFinCounters && s_ctr[threadIdx.x] != 0)
        atomicAdd(&ctr[threadIdx.x], s_ctr[threadIdx.x]);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 4) k_finalize(FinalizeParams<T> p)
{
    __shared__ T fin_smem[8][2 * kFinWarpVals];
    __shared__ unsigned long long s_ctr[kFinCounters];
    if (threadIdx.x < kFinCounters) s_ctr[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    T *wa = fin_smem[threadIdx.x >> 5];
    T *wb = wa + kFinWarpVals;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sqrt_m = sqrt((double)p.m);
    const int m = p.m;
    if (p.err != nullptr && *p.err != 0) {
        // a bounded wait of a tensor-core kernel ran out: the partials are incomplete
        for (int64_t i = warp_global; i < p.nq; i += nwarps)
            if (lane == 0) {
                p.out_dist[i] = NAN;
                p.out_idx[i] = -1;
            }
        return;
    }
    for (int64_t i = warp_global; i < p.nq; i += nwarps) {
        // 1. reduce the column groups: largest q, then lowest chunk start
        T q = T(-INFINITY);
        int32_t g = -1;
        for (int k = lane; k < p.n_groups; k += 32) {
            const Partial<T> v = p.part[(int64_t)k * p.nq + i];
            if (better(v.q, v.g, q, g)) {
                q = v.q;
                g = v.g;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T q2 = __shfl_xor_sync(0xffffffffu, q, o);
            const int32_t g2 = __shfl_xor_sync(0xffffffffu, g, o);
            if (better(q2, g2, q, g)) {
                q = q2;
                g = g2;
            }
        }
        double d = INFINITY;
        int64_t gi = -1;
        if (p.g_first >= 0) {
            if (p.cflag_a[i]) {
                // 3. a constant query window is 0 from a constant window, sqrt(m) from the rest
                const int64_t gc = const_outside(p, i), gf = first_outside(p, i);
                if (gc >= 0) {
                    d = 0.0;
                    gi = gc;
                } else if (gf >= 0) {
                    d = sqrt_m;
                    gi = gf;
                }
            } else {
                if (g >= 0) {
                    // 2. re-score the winning chunk, and every chunk whose
                    // approximate score came within the near-tie width of the
                    // best (other groups' winners and the plain kernel's
                    // near-tie records), so that the recurrence's rounding
                    // cannot decide between near-tied windows
                    const Split<T> ma = p.ms_a[i];
                    T sc;
                    int32_t gw;
                    rescore_chunk<T>(p.a, p.b, p.nb, p.npos_b, m, p.ms_b, p.rs_b, i, g, ma, lane, wa, wb, sc,
                                     gw, p.excl);
                    if (p.near.rec != nullptr) {
                        const T lim = q - near_width(p, i, p.rs_a[i].z, ma);  // the row is not constant: z > 0
                        auto consider = [&](int32_t cu) {
                            T s2;
                            int32_t g2;
                            rescore_chunk<T>(p.a, p.b, p.nb, p.npos_b, m, p.ms_b, p.rs_b, i, cu, ma, lane, wa, wb,
                                             s2, g2, p.excl);
                            if (better(s2, g2, sc, gw)) {
                                sc = s2;
                                gw = g2;
                            }
                        };
                        // other groups' winners and the records, one (group, entry) per lane
                        const int per = p.near.S + 1;
                        const int64_t tot = (int64_t)p.n_groups * per;
                        bool ovf = false;
                        unsigned extra = 0;
                        for (int64_t e0 = 0; e0 < tot; e0 += 32) {
                            const int32_t c = near_entry(p, i, e0 + lane, per, tot, g, lim, ovf);
                            unsigned pend = __ballot_sync(0xffffffffu, c >= 0);
                            while (pend) {
                                const int src = __ffs(pend) - 1;
                                pend &= pend - 1;
                                consider(__shfl_sync(0xffffffffu, c, src));
                                ++extra;
                            }
                        }
                        unsigned ochunks = 0;
                        const bool any_ovf = __any_sync(0xffffffffu, ovf);
                        if (any_ovf) {
                            // a record within the width was dropped: every chunk of that group
                            for (int k = 0; k < p.n_groups; ++k) {
                                const NearSlot h = *p.near.head(k, i);
                                if (!(h.g & kNearOverflow)) continue;
                                const uint32_t mask = __float_as_uint(h.q);
                                int64_t g_lo, g_hi;
                                group_range(p, k, g_lo, g_hi);
                                for (int sp = p.cgroup_start[k]; sp < p.cgroup_start[k + 1]; ++sp) {
                                    const Span span = p.cspans[sp];
                                    for (int c0 = 0; c0 < span.ncols; c0 += kChunk) {
                                        const int32_t cu = (int32_t)(span.g0 + c0);
                                        // a chunk whose windows meet a marked run
                                        const uint32_t b0 = near_run(cu, g_lo, g_hi);
                                        const uint32_t b1 = near_run(cu + kChunk - 1, g_lo, g_hi);
                                        const uint32_t runs = (b1 >= 31 ? 0xffffffffu : ((2u << b1) - 1u)) &
                                                              ~((1u << b0) - 1u);
                                        if (cu == g || !(mask & runs)) continue;
                                        consider(cu);
                                        ++ochunks;
                                    }
                                }
                            }
                        }
                        if (lane == 0 && (extra > 0 || any_ovf)) {
                            atomicAdd(&s_ctr[0], extra > 0 ? 1ull : 0ull);
                            atomicAdd(&s_ctr[1], (unsigned long long)extra);
                            atomicAdd(&s_ctr[2], any_ovf ? 1ull : 0ull);
                            atomicAdd(&s_ctr[3], (unsigned long long)ochunks);
                        }
                    }
                    if (gw >= 0) {
                        // 4. the chosen pair's distance from its definition
                        d = pair_distance<T>(p.a, i, ma, p.rs_a[i].z, p.b, gw, p.ms_b[gw], p.rs_b[gw].z, m, lane);
                        gi = gw;
                    }
                }
                const int64_t gcst = const_outside(p, i);
                if (gcst >= 0 && (gi < 0 || sqrt_m < d || (sqrt_m == d && gcst < gi))) {
                    d = sqrt_m;
                    gi = gcst;
                }
            }
        }
        if (lane == 0) {
            p.out_dist[i] = p.out_corr ? (gi >= 0 ? 1.0 - d * d / (2.0 * m) : -INFINITY) : d;
            p.out_idx[i] = gi;
        }
    }
    flush_counters(p.ctr, s_ctr);
}

// ---------------------------------------------------------------------------
// Block form for m <= kFinMaxM. A CTA takes a block of fin_warps<T>() * wpw
// consecutive query windows at a time (wpw = 1 .. 32 windows per warp, 32 for
// large joins, fewer for short ones so that they still fill the GPU), in three
// phases:
//   1. one thread per window: the reduction of the column groups' partials,
//      the near-tie candidates, the constant-window cases and the window's
//      statistics, with loads that are coalesced across the block and no
//      per-window shuffles; the results go to shared memory;
//   2. one warp per window (each warp takes wpw of the block's windows): the
//      re-scoring of the winning chunk and of the candidates, and the chosen
//      pair's distance from the staged samples;
//   3. one thread per window again: the constant-window rule and the output.
// In phase 2 lane lg of half-warp h sums k in [lg * KPL, (lg + 1) * KPL) for
// candidates 8h .. 8h + 7, with KPL a multiple of 8 (compile-time, so that
// every loop unrolls) and both buffers zero-filled past their data, so the
// inner loop runs in unmasked steps of 8. Shared memory is padded by one
// value per 32 (qidx): a run of 8 starting at a multiple of 8 never crosses a
// pad, and the lanes' start offsets fall in distinct banks for KPL = 8 .. 32.
// ---------------------------------------------------------------------------
constexpr int kFinMaxM = 512;
// warps per CTA: the per-warp buffers stay within 48 KB of static shared memory
template <typename T> constexpr int fin_warps() { return sizeof(T) == 8 ? 2 : 4; }
__device__ __forceinline__ int qidx(int e) { return e + (e >> 5); }
// near-tie candidates kept per window in shared memory; a window with more
// scans the column groups' records again in phase 2
constexpr int kFinMaxCand = 8;

__host__ __device__ constexpr int fin_kpl(int m) { return ((m + 15) / 16 + 7) / 8 * 8; }

// Stage chunk g's samples b[g ..] - mean_hi(b_g) into wb (zero past the
// dictionary), for every value the lanes of rescore_staged read.
template <typename T, int KPL>
__device__ __forceinline__ T stage_chunk(const T *__restrict__ pb, int64_t nb, const Split<T> *__restrict__ ms_b,
                                         int32_t g, int lane, T *wb)
{
    constexpr int NBV = 16 * KPL + kChunk;
    __syncwarp();  // earlier reads of wb are done
    const T sb = ms_b[g].hi;
    const T *bg = pb + g;
    // value e = lane + 32 u sits at qidx(e) = lane + 33 u
    if (g + NBV <= nb) {
#pragma unroll
        for (int u = 0; u < (NBV + 31) / 32; ++u)
            if (32 * (u + 1) <= NBV || lane + 32 * u < NBV) wb[lane + 33 * u] = bg[lane + 32 * u] - sb;
    } else {  // the chunk's samples run past the dictionary: zeros there
        const int64_t lim = nb - g;
#pragma unroll
        for (int u = 0; u < (NBV + 31) / 32; ++u) {
            const int e = lane + 32 * u;
            if (e < NBV) wb[lane + 33 * u] = e < lim ? bg[e] - sb : T(0);
        }
    }
    __syncwarp();
    return sb;
}

// The terms of the chunk window this lane scores in rescore_staged (window
// g + 8 (lane / 16) + lane % 8, clamped into range): 1/std, penalty (0 or
// -inf) and split mean. Loaded before the chunk is staged, so that their
// latency overlaps the staging.
template <typename T> struct CandTerms {
    T z, w, mhi, mlo;
};
template <typename T>
__device__ __forceinline__ CandTerms<T> load_cand(const vec4_t<T> *__restrict__ rs_b,
                                                  const Split<T> *__restrict__ ms_b, int64_t npos_b, int32_t g,
                                                  int lane)
{
    const int64_t gc = (int64_t)g + 8 * (lane >> 4) + (lane & 7);
    const int64_t gcl = gc < npos_b ? gc : npos_b - 1;
    const vec4_t<T> rv = rs_b[gcl];
    const Split<T> mb = ms_b[gcl];
    return CandTerms<T>{rv.z, rv.w, mb.hi, mb.lo};
}

// Re-score chunk g against the staged query window qa (= a - mean_hi(a)) and
// the staged chunk wb (= b - mean_hi(b_g)); returns the chunk's best (score,
// window) in every lane as rescore_chunk.
template <typename T, int KPL>
__device__ __forceinline__ void rescore_staged(int64_t npos_b, int m, const CandTerms<T> &ct, T sb, const T *qa,
                                               T da, int32_t g, int lane, const T *wb, T &sc_out, int32_t &g_out,
                                               int64_t i, int excl)
{
    const int half = lane >> 4, lg = lane & 15;
    const int k0 = lg * KPL;
    T acc[8], bw[8];
    {
        const T *b0 = wb + qidx(8 * half + k0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[c] = T(0);
            bw[c] = b0[c];
        }
    }
#pragma unroll
    for (int kb = 0; kb < KPL; kb += 8) {
        const T *qp = qa + qidx(k0 + kb);
        const T *bp = wb + qidx(8 * half + k0 + kb + 8);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const T av = qp[u];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = fma(av, bw[(c + u) & 7], acc[c]);
            bw[u] = bp[u];
        }
    }
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
#pragma unroll
        for (int c = 0; c < s; ++c) {
            const bool up = (lane & s) != 0;
            const T send = up ? acc[c] : acc[c + s];
            const T keep = up ? acc[c + s] : acc[c];
            acc[c] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 8);
    // lanes l and l ^ 8 now hold the same candidate's total
    const int cand = 8 * half + (lane & 7);
    const int64_t gc = (int64_t)g + cand;
    const bool ok = gc < npos_b && (excl == 0 || (gc - i >= excl || i - gc >= excl)) && ct.w == T(0);
    // sum_k (a - sa)(b - sb) = cov + m (mean_a - sa)(mean_b - sb)
    T sc = ok ? (acc[0] - T(m) * da * ((ct.mhi - sb) + ct.mlo)) * ct.z : T(-INFINITY);
    // a NaN score (products that overflowed) is no candidate: better() is then
    // a total order, so every lane ends with the same (score, window) and the
    // branches on it below stay warp-uniform
    const bool num = sc == sc;
    sc = num ? sc : T(-INFINITY);
    int32_t gw = ok && num ? (int32_t)gc : -1;
    warp_best(sc, gw);
    sc_out = sc;
    g_out = gw;
}

template <typename T, int KPL>
__global__ void __launch_bounds__(32 * fin_warps<T>(), sizeof(T) == 8 ? 4 : 8)
    k_finalize_blk(FinalizeParams<T> p, int wpw)
{
    constexpr int kW = fin_warps<T>();
    constexpr int kNB = 32 * kW;                                   // threads, and the most windows per block
    constexpr int kQV = 16 * KPL + (16 * KPL) / 32 + 1;             // staged query window
    constexpr int kBV = (16 * KPL + kChunk) + (16 * KPL + kChunk) / 32 + 1;  // staged chunk
    __shared__ T f_buf[kW][kQV + kBV];
    __shared__ int32_t s_g[kNB];                 // winning chunk to re-score, -1: none
    __shared__ int32_t s_nc[kNB];                // near-tie candidates found
    __shared__ int32_t s_cand[kFinMaxCand][kNB];
    __shared__ int32_t s_gi[kNB];                // phase 2's window (-1: none)
    __shared__ T s_mhi[kNB], s_mlo[kNB], s_isa[kNB], s_lim[kNB], s_d[kNB];
    __shared__ unsigned long long s_ctr[kFinCounters];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kFinCounters) s_ctr[tid] = 0;  // published by the first block's barrier
    T *const qa = f_buf[warp];
    T *const wb = qa + kQV;
    const int m = p.m;
    const double sqrt_m = sqrt((double)m);
    if (p.err != nullptr && *p.err != 0) {
        // a bounded wait of a tensor-core kernel ran out: the partials are incomplete
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < p.nq; i += (int64_t)gridDim.x * blockDim.x) {
            p.out_dist[i] = NAN;
            p.out_idx[i] = -1;
        }
        return;
    }
    // wpw (1..32) query windows per warp: a block is kW * wpw windows, so that
    // short joins still spread over many CTAs
    const int nb = kW * wpw;
    const int64_t nblk = (p.nq + nb - 1) / nb;
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int64_t i0 = blk * nb;
        const bool mine = tid < nb;  // this thread has a window of the block
        const int64_t i = i0 + tid;
        // ---- phase 1: this thread's window ----
        double d = INFINITY;
        int64_t gi = -1, gcst = -1;
        int32_t g = -1;
        int nc = 0;
        bool ovf = false;   // a column group's records overflowed for this window
        bool resc = false;  // phase 2 re-scores this window
        if (mine && i < p.nq && p.g_first >= 0) {
            if (p.cflag_a[i]) {
                // a constant query window is 0 from a constant window, sqrt(m) from the rest
                const int64_t gc = const_outside(p, i), gf = first_outside(p, i);
                if (gc >= 0) {
                    d = 0.0;
                    gi = gc;
                } else if (gf >= 0) {
                    d = sqrt_m;
                    gi = gf;
                }
            } else {
                // the column groups: largest q, then lowest chunk start
                // (the record headers are read in the same pass, so that the
                // near-tie pass below re-reads only what this one brought into
                // L1 and walks the headers again only for windows with records)
                T q = T(-INFINITY);
                int32_t hdr = 0;  // OR of the groups' header words: any slot in use, any overflow
                const bool rec = p.near.rec != nullptr;
#pragma unroll 4
                for (int k = 0; k < p.n_groups; ++k) {
                    const Partial<T> v = p.part[(int64_t)k * p.nq + i];
                    if (rec) hdr |= p.near.head(k, i)->g;
                    if (better(v.q, v.g, q, g)) {
                        q = v.q;
                        g = v.g;
                    }
                }
                gcst = const_outside(p, i);
                if (g >= 0) {
                    resc = true;
                    const Split<T> ma = p.ms_a[i];
                    const T isa = p.rs_a[i].z;  // the row is not constant: isa > 0
                    s_mhi[tid] = ma.hi;
                    s_mlo[tid] = ma.lo;
                    s_isa[tid] = isa;
                    if (p.near.rec != nullptr) {
                        // every other chunk whose approximate score came within the
                        // near-tie width of the best (other groups' winners and the
                        // join's near-tie records) is re-scored too, so that the
                        // join's rounding cannot decide between near ties
                        const T lim = q - near_width(p, i, isa, ma);
                        s_lim[tid] = lim;
                        const int S = p.near.S;
                        ovf = (hdr & kNearOverflow) != 0;
#pragma unroll 4
                        for (int k = 0; k < p.n_groups; ++k) {
                            const Partial<T> v = p.part[(int64_t)k * p.nq + i];
                            if (v.g >= 0 && v.g != g && v.q >= lim) {
                                if (nc < kFinMaxCand) s_cand[nc][tid] = v.g;
                                ++nc;
                            }
                        }
                        if (hdr & kNearCountMask) {  // some group recorded near ties for this window
                            for (int k = 0; k < p.n_groups; ++k) {
                                const NearSlot *h = p.near.head(k, i);
                                const int n = h->g & kNearCountMask;
                                for (int u = 1; u <= n && u <= S; ++u) {
                                    const NearSlot sl = h[(int64_t)u * p.near.ld];
                                    if (sl.g != g && T(sl.q) >= lim) {
                                        if (nc < kFinMaxCand) s_cand[nc][tid] = sl.g;
                                        ++nc;
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }
        s_g[tid] = resc ? g : -1;
        s_nc[tid] = ovf ? -1 : nc;  // -1: scan the records again and re-score the overflowed groups
        __syncthreads();

        // ---- phase 2: this warp's 32 windows, one at a time ----
        for (int w = 0; w < wpw; ++w) {
            const int t = warp * wpw + w;
            const int32_t g0 = s_g[t];
            if (g0 < 0) continue;
            const int64_t iw = i0 + t;
            const Split<T> ma{s_mhi[t], s_mlo[t]};
            CandTerms<T> ct = load_cand(p.rs_b, p.ms_b, p.npos_b, g0, lane);
            const T *ai = p.a + iw;
            // 16 * KPL values over 32 lanes; qidx(lane + 32 u) = lane + 33 u
            if (m == 16 * KPL) {
#pragma unroll
                for (int u = 0; u < KPL / 2; ++u) qa[lane + 33 * u] = ai[lane + 32 * u] - ma.hi;
            } else {
#pragma unroll
                for (int u = 0; u < KPL / 2; ++u) {
                    const int e = lane + 32 * u;
                    qa[lane + 33 * u] = e < m ? ai[e] - ma.hi : T(0);
                }
            }
            T sb = stage_chunk<T, KPL>(p.b, p.nb, p.ms_b, g0, lane, wb);
            T sc;
            int32_t gw;
            rescore_staged<T, KPL>(p.npos_b, m, ct, sb, qa, ma.lo, g0, lane, wb, sc, gw, iw, p.excl);
            int32_t staged = g0;  // the chunk whose samples wb holds (and whose terms ct and sb are)
            int32_t win = g0;     // the chunk of the best window so far
            unsigned extra = 0, ochunks = 0;
            auto consider = [&](int32_t cu) {
                T s2;
                int32_t g2;
                ct = load_cand(p.rs_b, p.ms_b, p.npos_b, cu, lane);
                sb = stage_chunk<T, KPL>(p.b, p.nb, p.ms_b, cu, lane, wb);
                rescore_staged<T, KPL>(p.npos_b, m, ct, sb, qa, ma.lo, cu, lane, wb, s2, g2, iw, p.excl);
                staged = cu;
                if (better(s2, g2, sc, gw)) {
                    sc = s2;
                    gw = g2;
                    win = cu;
                }
            };
            const int ncw = s_nc[t];
            if (ncw > 0 && ncw <= kFinMaxCand) {
                for (int c = 0; c < ncw; ++c) consider(s_cand[c][t]);
                extra = ncw;
            } else if (ncw != 0) {
                // more candidates than the shared list holds, or overflowed
                // records: scan the entries again, one (group, entry) per lane
                const T lim = s_lim[t];
                const int per = p.near.S + 1;
                const int64_t tot = (int64_t)p.n_groups * per;
                bool o = false;
                for (int64_t e0 = 0; e0 < tot; e0 += 32) {
                    const int32_t c = near_entry(p, iw, e0 + lane, per, tot, g0, lim, o);
                    unsigned pend = __ballot_sync(0xffffffffu, c >= 0);
                    while (pend) {
                        const int src = __ffs(pend) - 1;
                        pend &= pend - 1;
                        consider(__shfl_sync(0xffffffffu, c, src));
                        ++extra;
                    }
                }
                if (ncw < 0) {
                    // a record within the width was dropped: every chunk of that group
                    for (int k = 0; k < p.n_groups; ++k) {
                        const NearSlot h = *p.near.head(k, iw);
                        if (!(h.g & kNearOverflow)) continue;
                        const uint32_t mask = __float_as_uint(h.q);
                        int64_t g_lo, g_hi;
                        group_range(p, k, g_lo, g_hi);
                        for (int sp = p.cgroup_start[k]; sp < p.cgroup_start[k + 1]; ++sp) {
                            const Span span = p.cspans[sp];
                            for (int c0 = 0; c0 < span.ncols; c0 += kChunk) {
                                const int32_t cu = (int32_t)(span.g0 + c0);
                                // a chunk whose windows meet a marked run
                                const uint32_t b0 = near_run(cu, g_lo, g_hi);
                                const uint32_t b1 = near_run(cu + kChunk - 1, g_lo, g_hi);
                                const uint32_t runs =
                                    (b1 >= 31 ? 0xffffffffu : ((2u << b1) - 1u)) & ~((1u << b0) - 1u);
                                if (cu == g0 || !(mask & runs)) continue;
                                consider(cu);
                                ++ochunks;
                            }
                        }
                    }
                }
            }
            if (lane == 0 && (extra > 0 || ncw < 0)) {
                atomicAdd(&s_ctr[0], extra > 0 ? 1ull : 0ull);
                atomicAdd(&s_ctr[1], (unsigned long long)extra);
                atomicAdd(&s_ctr[2], ncw < 0 ? 1ull : 0ull);
                atomicAdd(&s_ctr[3], (unsigned long long)ochunks);
            }
            T dw = T(INFINITY);
            if (gw >= 0) {
                // the chosen pair's distance from its definition, on the staged samples
                if (staged != win) {
                    ct = load_cand(p.rs_b, p.ms_b, p.npos_b, win, lane);
                    sb = stage_chunk<T, KPL>(p.b, p.nb, p.ms_b, win, lane, wb);
                }
                // the winner's terms from the lane that scored it (lanes 16 (o / 8) + o % 8)
                const int ow = gw - win, src = 16 * (ow >> 3) + (ow & 7);
                const T is_b = __shfl_sync(0xffffffffu, ct.z, src);
                const T db = (__shfl_sync(0xffffffffu, ct.mhi, src) - sb) + __shfl_sync(0xffffffffu, ct.mlo, src);
                const T is_a = s_isa[t];
                // z_a - z_b = (qa - lo_a) is_a - (wb - db) is_b: each difference is
                // taken before its scaling, so no large term is rounded (db, the
                // mean difference within the chunk, can be far above the spread)
                const T *wo = wb + qidx(gw - win + lane);  // value gw - win + lane + 32 u sits at wo[33 u]
                // the scalar form: (qa - lo) is_a - (wb - db) is_b, squared and summed
                auto dist2 = [&]() {
                    T a = T(0);
#pragma unroll
                    for (int u = 0; u < KPL / 2; ++u) {
                        if (lane + 32 * u < m) {
                            const T dd = fma(qa[lane + 33 * u] - ma.lo, is_a, -((wo[33 * u] - db) * is_b));
                            a = fma(dd, dd, a);
                        }
                    }
                    return a;
                };
                T acc;
                if constexpr (sizeof(T) == 4) {
                    if (m == 16 * KPL) {
                        // every value in use: the same operations on pairs of them
                        const float2 nlo = make_float2(-ma.lo, -ma.lo), ia = make_float2(is_a, is_a);
                        const float2 ndb = make_float2(-db, -db), nib = make_float2(-is_b, -is_b);
                        float2 a2 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < KPL / 2; u += 2) {
                            const float2 q2 = make_float2(qa[lane + 33 * u], qa[lane + 33 * (u + 1)]);
                            const float2 w2 = make_float2(wo[33 * u], wo[33 * (u + 1)]);
                            const float2 wz = __fmul2_rn(__fadd2_rn(w2, ndb), nib);
                            const float2 dd = __ffma2_rn(__fadd2_rn(q2, nlo), ia, wz);
                            a2 = __ffma2_rn(dd, dd, a2);
                        }
                        acc = a2.x + a2.y;
                    } else {
                        acc = dist2();
                    }
                } else {
                    acc = dist2();
                }
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
                dw = sqrt(acc);
            }
            if (lane == 0) {
                s_d[t] = dw;
                s_gi[t] = gw;
            }
            __syncwarp();  // the next window rewrites qa and wb
        }
        __syncthreads();

        // ---- phase 3: this thread's window ----
        if (mine && i < p.nq) {
            if (resc) {
                d = (double)s_d[tid];
                gi = s_gi[tid];
            }
            if (gcst >= 0 && (gi < 0 || sqrt_m < d || (sqrt_m == d && gcst < gi))) {
                d = sqrt_m;
                gi = gcst;
            }
            p.out_dist[i] = p.out_corr ? (gi >= 0 ? 1.0 - d * d / (2.0 * m) : -INFINITY) : d;
            p.out_idx[i] = gi;
        }
        __syncthreads();  // the next block rewrites the per-window arrays
    }
    flush_counters(p.ctr, s_ctr);
}

template <typename T, int KPL> cudaError_t launch_blk(const FinalizeParams<T> &p, cudaStream_t st)
{
    constexpr int kNB = 32 * fin_warps<T>();
    // windows per warp: 32, unless that leaves fewer than about eight CTAs per
    // SM, as for the short requests of the serving path
    const int64_t sms = p.sm_count > 0 ? p.sm_count : 1;
    const int64_t per = (p.nq + sms * 8 * fin_warps<T>() - 1) / (sms * 8 * fin_warps<T>());
    const int wpw = (int)(per < 1 ? 1 : (per > 32 ? 32 : per));
    const int nb = fin_warps<T>() * wpw;
    int64_t grid = (p.nq + nb - 1) / nb;  // one block of query windows per CTA and pass
    if (grid > sms * 64) grid = sms * 64;
    k_finalize_blk<T, KPL><<<(unsigned)grid, kNB, 0, st>>>(p, wpw);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_finalize(const FinalizeParams<T> &p, cudaStream_t st)
{
    if (p.nq <= 0) return cudaSuccess;
    if (p.m <= kFinMaxM) {
        switch (fin_kpl(p.m)) {
        case 8: return launch_blk<T, 8>(p, st);
        case 16: return launch_blk<T, 16>(p, st);
        case 24: return launch_blk<T, 24>(p, st);
        default: return launch_blk<T, 32>(p, st);
        }
    }
    int64_t grid = (p.nq + 7) / 8;  // 8 warps (rows) per CTA
    const int64_t sms = p.sm_count > 0 ? p.sm_count : 1;
    if (grid > sms * 64) grid = sms * 64;
    k_finalize<T><<<(unsigned)grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_finalize<float>(const FinalizeParams<float> &, cudaStream_t);
template cudaError_t launch_finalize<double>(const FinalizeParams<double> &, cudaStream_t);

}  // namespace mpd

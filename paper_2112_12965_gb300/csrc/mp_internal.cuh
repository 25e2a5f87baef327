// Internal declarations shared by the translation units of libmpdict.
// Nothing here is part of the public C ABI (include/mpdict.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpd {

// Vector types holding the per-window recurrence statistics.
struct __align__(32) dvec4 {
    double x, y, z, w;
};
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dvec4; };
template <typename T> using vec4_t = typename Vec4<T>::type;

// A window mean split into two values of the join's arithmetic type,
// hi = mean rounded to T and lo = (mean - hi) rounded to T, so that kernels
// can centre samples to T's relative precision without FP64 arithmetic
// (FP64 throughput on GB300 is a small fraction of FP32's).
template <typename T> struct __align__(2 * sizeof(T)) Split {
    T hi, lo;
};

// A run of consecutive valid dictionary windows inside one segment:
// global windows g0 .. g0 + ncols - 1.
struct Span {
    int64_t g0;
    int32_t ncols;
    int32_t pad;
};

// Launch geometry of the plain diagonal kernel.
constexpr int kPlainRowsPerLane = 20;  // query windows owned by one lane (k_plain, FP32)
// Short FP32 joins with seeds computed in the kernel (at most kPlainShortMaxRows
// query windows) use kPlainRowsShort rows per lane instead: a CTA's time is
// then its warps' seed dot products, which fall with the rows per lane.
constexpr int kPlainRowsShort = 4;
constexpr int64_t kPlainShortMaxRows = 4096;
constexpr int kServeRowsPerLane = 16;  // the same in the batched serving kernel (two CTAs per SM)
constexpr int kPlainColBlock = 256;    // dictionary windows staged per block
constexpr int kChunk = 16;             // windows per chunk of the lazy argmax
static_assert(kChunk % 2 == 0, "the plain kernel folds the scores of two columns per maximum");

// Per-window statistics of a series for one window length m (kernel K1).
//   mean[i], invstd[i]   FP64 mean and 1/population-std (0 for a constant window)
//   cflag[i]             1 if the window's samples all compare equal
//   rs[i]                recurrence terms for the diagonal kernel, in the join's
//                        arithmetic type T:
//                          x = df[i] = (x[i+m-1] - x[i-1]) / 2          (0 for i = 0)
//                          y = dg[i] = (x[i+m-1] - mean[i]) + (x[i-1] - mean[i-1])  (0 for i = 0)
//                          z = invstd[i] rounded to T
//                          w = 0, or -inf for a constant window (excludes it from
//                              the maximum of the correlation score); for a
//                              dictionary, launch_mark_invalid also sets -inf
//                              (and z = 0) on every position whose window
//                              crosses a segment end
template <typename T>
cudaError_t launch_mark_invalid(vec4_t<T> *rs, int64_t npos, const int64_t *seg_offsets, int32_t n_segments,
                                int32_t m, cudaStream_t st);
// ms[i] (may be null): mean[i] split into hi + lo of type T.
template <typename T>
cudaError_t launch_window_stats(const T *x, int64_t n, int32_t m, double *mean, double *invstd, uint8_t *cflag,
                                vec4_t<T> *rs, Split<T> *ms, cudaStream_t st);

// Checks every sample is finite; sets *bad to 1 otherwise (bad must be zeroed).
template <typename T>
cudaError_t launch_check_finite(const T *x, int64_t n, int32_t *bad, cudaStream_t st);

// Lowest constant window and lowest valid window among the spans (int64 out[2], -1 if none).
cudaError_t launch_dict_specials(const Span *spans, int32_t n_spans, const uint8_t *cflag, int64_t *out,
                                 cudaStream_t st);

// Partial result of one column group for one query window: the largest
// correlation score q = cov * invstd_b over the group's valid non-constant
// windows, and the first window g of the kChunk-window chunk (inside one
// segment) where that maximum was first reached (-1 if none). The
// finalisation re-scores windows g .. g + kChunk - 1 to find the exact one.
template <typename T> struct Partial {
    T q;
    int32_t g;
};

// Near-tie records of a join for one (column group, query window): up to S
// chunks (first window g and approximate score q) whose score came within the
// near-tie width below the running best, or that were the best until
// overtaken by less than the width. The join's rounding (the FP32 recurrence,
// or the tensor cores' operand rounding) can misorder such chunks; the
// finalisation re-scores each of them exactly, so the pick does not depend on
// that rounding. A record is dropped only when all S slots are in use; if the
// dropped score may still lie within the width of the final best, the
// overflow bit is set and the finalisation re-scores every chunk of that
// column group for that window.
struct NearSlot {
    int32_t g;
    float q;
};
constexpr int32_t kNearCountMask = 0x3f;  // header bits 0-5: slots in use
constexpr int32_t kNearOverflow = 0x80;   // header bit 7: a record within the width was dropped
constexpr int kNearMaxSlots = 63;
struct NearRec {
    // [n_groups][1 + S][ld]: entry (k, 0, r) is the header of (group k, row r):
    // its g holds the slots in use | kNearOverflow, its q the bits of an
    // overflow mask (bit b: a dropped record lay in the b-th of 32 equal runs
    // of the group's window range, see near_run); the join zeroes the headers
    // of its rows. Entries (k, 1 + u, r) are the slots. Null: no records.
    NearSlot *rec;
    int64_t ld;       // row stride
    int32_t S;        // slots per (group, row), 1 .. kNearMaxSlots
    float rho;        // plain form: width in Pearson correlation
    const float *fb;  // tensor-core forms (rho unused): the dictionary's column factor F_b, below
    float u;          // tensor-core forms: bound on the relative error of the products and their sum
    __host__ __device__ NearSlot *head(int64_t k, int64_t r) const { return rec + k * (S + 1) * ld + r; }
};

// The run of a group's window range [g_lo, g_hi) that window g lies in, for
// the overflow mask: 32 runs of ceil((g_hi - g_lo) / 32) windows.
__host__ __device__ inline uint32_t near_run(int64_t g, int64_t g_lo, int64_t g_hi)
{
    const int64_t len = (g_hi - g_lo + 31) / 32;
    const int64_t b = len > 0 ? (g - g_lo) / len : 0;
    return (uint32_t)(b < 0 ? 0 : (b > 31 ? 31 : b));
}
// Width of the plain FP32 recurrence, in correlation: 8x the largest drift
// measured by a float32 model of the recurrence on the benchmark data (about
// 1e-6 to 5e-6 over the up to 640-step diagonals between seeds, 32 lanes x 20
// rows).
constexpr float kNearRhoFP32 = 4e-5f;
// Tensor-core forms: a bound, not a measurement. The product sum S of the
// shifted operands a' = a - s_a, b' = b - s_b (per-CTA and per-tile shifts)
// errs by at most u * sum_k |a'_k b'_k| <= u ||a'|| ||b'|| (Cauchy-Schwarz),
// with u the relative error of one product plus that of the FP32 sum. In
// units of the score q = C / std_b this is u m sqrt(std_a^2 + da^2) F_b, where
// da = mean_a - s_a and F_b = max over the dictionary's windows of
// sqrt(1 + ((mean_b - s_b) / std_b)^2). The width is twice that (two chunks
// err in opposite directions), so a chunk left out is surely not the best.
//   single TF32 product: operands rounded to 11 significant bits (2^-11 each)
//   split BF16 (hi*hi + hi*lo + lo*hi): hi + lo within 2^-18 of each operand,
//     lo*lo left out: 3 * 2^-18
//   FP32 sum of the m (TF32) or 3m (split BF16) products: 2^-23 per product
//   single BF16 product: operands rounded to 8 significant bits (2^-9 each)
constexpr float kTcUnitTF32 = 9.7752e-4f;    // 2^-10 + 2^-21
constexpr float kTcUnitBF16X3 = 1.1445e-5f;  // 3 * 2^-18
constexpr float kTcUnitBF16 = 3.9101e-3f;    // 2^-8 + 2^-17
constexpr int kNearSlotsPlain = 4;
constexpr int kNearSlotsTC = 63;
constexpr int kTcRows = 128;  // query windows per CTA of the tensor-core join (one per TMEM lane)

#ifdef __CUDACC__
// Record chunk g with approximate score q for (group k, row r). floor_q is
// the running best minus the width: a record below it can never come within
// the width of the final best, so dropping it needs no overflow mark. The
// caller owns (k, r) exclusively for the whole join. With all S slots in use,
// kEvict replaces the lowest-scoring slot if q is higher, and the record
// dropped (that one, or q) sets the overflow bit if it may still matter;
// without kEvict q is dropped (less code, for the plain kernel's hot loop).
// The overflow marks the run of the dropped record's window in the header's
// mask when the group's window range [g_lo, g_hi) is given (g_hi > g_lo), and
// every run otherwise.
template <bool kEvict>
__device__ __forceinline__ void near_add(const NearRec &nr, int64_t k, int64_t r, int32_t g, float q, float floor_q,
                                         int64_t g_lo = 0, int64_t g_hi = 0)
{
    NearSlot *h = nr.head(k, r);
    const int32_t f = h->g;
    const int n = f & kNearCountMask;
    if (n < nr.S) {
        h[(int64_t)(n + 1) * nr.ld] = NearSlot{g, q};
        h->g = f + 1;
        return;
    }
    float dropped = q;
    int32_t dropped_g = g;
    if (kEvict) {
        int lo = 1;
        float qlo = h[nr.ld].q;
        for (int u = 2; u <= nr.S; ++u) {
            const float qu = h[(int64_t)u * nr.ld].q;
            if (qu < qlo) {
                qlo = qu;
                lo = u;
            }
        }
        if (q > qlo) {
            dropped = qlo;
            dropped_g = h[(int64_t)lo * nr.ld].g;
            h[(int64_t)lo * nr.ld] = NearSlot{g, q};
        }
    }
    if (dropped >= floor_q) {
        const uint32_t bits = g_hi > g_lo ? (1u << near_run(dropped_g, g_lo, g_hi)) : 0xffffffffu;
        h->g = f | kNearOverflow;
        h->q = __uint_as_float(__float_as_uint(h->q) | bits);
    }
}
#endif

struct PlainLaunch {
    int64_t nq;            // query windows
    int32_t m;
    int32_t n_row_blocks;
    int32_t n_groups;      // column groups
    int32_t warps;         // warps per CTA (rows per CTA = warps * 32 * rows per lane)
    int32_t rows_per_lane = 0;  // 0: plain_rows_per_lane<T>(); kPlainRowsShort: the short form (FP32, no K2s seeds)
    int64_t ld_part = 0;   // row stride of the partial results and near-tie records (0: nq)
    int64_t row0 = 0;      // self-join: series position of query window 0
    int32_t excl = 0;      // self-join: exclusion zone half-width (0: an AB-join)
};

// Plain diagonal-recurrence join (kernel K2). Writes part[group * ld_part + row]
// (ld_part = L.ld_part, or nq): a join may run in row chunks, each launch
// given its rows' query, statistics and partial results by pointer offsets.
// spans[group_start[k] .. group_start[k+1]) are the spans of column group k.
// seed_top (may be null): the centred covariances of each warp's first query
// window, row r / (32 * rows per lane) at column g, row stride seed_ld (as
// written by tc_seeds); null makes the kernel compute them itself.
// left (null exactly when seed_top is): the left seeds of every span s and
// query window r of the launch at left[s * left_ld + r] (as written by
// tc_left_seeds). near (near.rec may be null; FP32 only): near-tie records of
// every query window; near.ld must equal the partial results' row stride.
template <typename T>
cudaError_t launch_plain(const PlainLaunch &L, const T *a, int64_t na, const vec4_t<T> *rs_a, const Split<T> *ms_a,
                         const T *b, int64_t nb, const vec4_t<T> *rs_b, const Split<T> *ms_b, const Span *spans,
                         const int32_t *group_start, Partial<T> *part, const T *seed_top, int64_t seed_ld,
                         const T *left, int64_t left_ld, const NearRec &near, cudaStream_t st);
template <typename T> constexpr int plain_rows_per_lane() { return sizeof(T) == 4 ? kPlainRowsPerLane : 8; }
template <typename T> size_t plain_smem_bytes(int warps, int m, int rows_per_lane = plain_rows_per_lane<T>());
// Resident CTAs per SM of the plain kernel for this shape (occupancy API).
template <typename T> int plain_ctas_per_sm(int warps, int m, int rows_per_lane = plain_rows_per_lane<T>());

// Serving: one request of a persistent batched launch (FP32 data). The layout
// mirrors the kernel's parameter block.
struct PlainRequest {
    const float *a;
    int64_t na;
    int64_t nq;
    int32_t m;
    int32_t n_groups;
    const float4 *rs_a;
    const Split<float> *ms_a;
    const float *b;
    int64_t nb;
    const float4 *rs_b;
    const Split<float> *ms_b;
    const Span *spans;
    const int32_t *group_start;
    Partial<float> *part;
    const float *seed_top;  // always null: batched work computes its own seeds
    int64_t seed_ld;
    const float *left;      // always null
    int64_t left_ld;
    NearRec near;           // near-tie records (required), ld = nq
    int64_t ld_part;        // nq
    int64_t row0;           // 0
    int32_t excl;           // 0: serving joins are AB-joins
};
struct BatchItem {
    int32_t req;  // index into the request array
    int32_t grp;  // column group
    int64_t rb;   // row block
};
// Launch `grid` persistent CTAs of `warps` warps over items[0 .. n_items);
// *counter must be 0. Every request in the batch must have m <= max_m and use
// `warps` warps per row block.
cudaError_t launch_plain_batched(const PlainRequest *reqs_dev, const BatchItem *items, int32_t n_items,
                                 int32_t *counter, int warps, int max_m, int grid, cudaStream_t st);

// Finalisation (kernel K4): reduce the column groups, re-score the winning
// chunk, apply the constant-window convention, recompute the chosen pair's
// distance exactly and write the output.
template <typename T> struct FinalizeParams {
    int64_t nq;
    int32_t m;
    int32_t n_groups;
    const Partial<T> *part;   // [n_groups][nq]
    const T *a;               // query samples
    const vec4_t<T> *rs_a;    // query recurrence terms (z = 1/std)
    const Split<T> *ms_a;     // query window means, split
    const uint8_t *cflag_a;
    const T *b;               // dictionary samples
    int64_t nb;               // dictionary sample count
    int64_t npos_b;           // window positions of the concatenated dictionary (nb - m + 1)
    const vec4_t<T> *rs_b;    // dictionary recurrence terms (z = 1/std, w = 0 or -inf)
    const Split<T> *ms_b;     // dictionary window means, split
    int64_t g_const;          // lowest constant valid dictionary window, or -1
    int64_t g_first;          // lowest valid dictionary window, or -1 (no window at all)
    double *out_dist;
    int64_t *out_idx;
    const int32_t *err;       // may be null; if *err != 0 a tensor-core wait ran out: NaN / -1 everywhere
    NearRec near;             // near-tie records of the join (near.rec null: none), ld = nq
    // chunk layout of the column groups, for windows whose records overflowed:
    // chunks g0 + 16 j of cspans[cgroup_start[k] .. cgroup_start[k+1]) are group k's
    const Span *cspans;
    const int32_t *cgroup_start;
    unsigned long long *ctr;  // may be null; kFinCounters counters, added to (see below)
    int32_t sm_count;         // the device's SMs (launch shape)
    int32_t out_corr;         // 1: write rho = 1 - d^2 / (2m) (Pearson's r for non-constant windows), -inf if none
    // Self-join of one series (dictionary learning): windows g with |g - i| < excl are
    // trivial matches of query window i and are left out; next_const[x] is the lowest
    // constant window >= x (-1 if none), over the npos_b positions. excl = 0: an AB-join.
    int32_t excl;
    const int64_t *next_const;
};
// Finalisation counters (FinalizeParams::ctr): query windows with near-tie
// candidates re-scored, near-tie chunks re-scored, windows whose records
// overflowed, chunks re-scored for them.
constexpr int kFinCounters = 4;
template <typename T> cudaError_t launch_finalize(const FinalizeParams<T> &p, cudaStream_t st);

// Dictionary learning (Algorithm 1) kernels, mp_learn.cu.
// next_const[x] = the lowest position >= x with cflag set, or -1; scratch holds
// next_const_scratch_elems(npos) int64 values.
cudaError_t launch_next_const(const uint8_t *cflag, int64_t npos, int64_t *next_const, int64_t *scratch,
                              cudaStream_t st);
size_t next_const_scratch_elems(int64_t npos);
// *best = (order key of min_i (P[i] - S[i]) << 32) | argmin over the positions not
// excluded (lowest i on ties); ~0 if there is none.
cudaError_t launch_learn_argmin(const double *P, const float *S, const uint8_t *excluded, int64_t n,
                                unsigned long long *best, int sm_count, cudaStream_t st);
// The float of an order key (host).
float learn_key_float(uint32_t key);
// S'[i] = d(window i, window j) of series x (FP32 statistics ms, rs, cflag of its
// nq windows); S = S' if first, else min(S, S'); *smax = order key of max S.
cudaError_t launch_learn_profile(const float *x, int64_t nq, int32_t m, const Split<float> *ms, const float4 *rs,
                                 const uint8_t *cflag, int64_t j, float *S, bool first, uint32_t *smax, int sm_count,
                                 cudaStream_t st);

}  // namespace mpd

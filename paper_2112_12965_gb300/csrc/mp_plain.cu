// K2: the plain form of the dictionary AB-join -- a diagonal recurrence on the
// FP32 pipes (FP64 for float64 data).
//
// Algorithm 2 (Sec. 3.2) joins the query with every dictionary segment and
// keeps the element-wise minimum. For one segment the join is an exact AB-join
// (the paper uses the method of its ref. "Matrix Profile XIV" for it): along a
// diagonal (i, g) -> (i+1, g+1) the centred covariance
//     C(i, g) = sum_k (a[i+k] - mean_a[i]) * (b[g+k] - mean_b[g])
// changes by O(1) work:
//     C(i, g) = C(i-1, g-1) + df_a[i] * dg_b[g] + df_b[g] * dg_a[i]
// with df[i] = (x[i+m-1] - x[i-1]) / 2 and
//      dg[i] = (x[i+m-1] - mean[i]) + (x[i-1] - mean[i-1])
// (expanding both means around the previous window proves it). The distance
// follows from the Pearson correlation rho = C * invstd_a * invstd_b / m as
// d^2 = 2 m (1 - rho), so for one query window the nearest non-constant
// dictionary window is the one with the largest q = C * invstd_b.
//
// Layout of the work. A CTA owns a block of consecutive query windows (rows);
// each lane owns kRows consecutive rows and keeps their C values in registers.
// The CTA walks the dictionary windows (columns) of a column group in
// increasing g. Moving one column to the right moves every diagonal one row
// down, so each lane shifts its registers by one row and takes the top one
// from the lane above with a warp shuffle. The first row of each warp has no
// row above inside the warp: its value comes from a "top seed", the centred
// covariance of that row with the column's window. FP32 joins of at least
// 2^31 pairs take the top seeds from the tensor-core kernel K2s (a dense
// product, computed once per join); the other joins compute them here as
// direct dot products per column block. At the first column of each span (a
// run of columns inside one segment) every row gets a "left seed": from the
// tensor-core kernel K2l for those FP32 joins, else a direct dot product.
// Short FP32 joins run with fewer rows per lane (kPlainRowsShort), which
// shortens each warp's seed dot products. Dictionary
// windows never cross a segment (Def. 8) because spans never do. Each lane
// keeps, for its rows, the running maximum of q per 16-column chunk and the
// chunk that raised it (plus near-tie records); the partial result per (row,
// column group) is reduced by the finalisation kernel, which re-scores the
// chunk's windows.
//
// Seeds computed here use shifted samples (query minus a per-CTA constant,
// dictionary minus a per-block constant), which keeps the FP32 products small
// for series with large offsets; the exact mean correction m * da * db is
// applied afterwards from the split means.
#include <math.h>

#include "mp_internal.cuh"

namespace mpd {
namespace {

template <typename T> struct PlainParams {
    const T *a;
    int64_t na;
    int64_t nq;
    int32_t m;
    int32_t n_groups;
    const vec4_t<T> *rs_a;
    const Split<T> *ms_a;
    const T *b;
    int64_t nb;
    const vec4_t<T> *rs_b;
    const Split<T> *ms_b;
    const Span *spans;
    const int32_t *group_start;
    Partial<T> *part;
    const T *seed_top;  // top seeds from the tensor cores, or null
    int64_t seed_ld;
    const T *left;      // left seeds from the tensor cores, [span][left_ld] (with seed_top), or null
    int64_t left_ld;
    NearRec near;       // near-tie records (near.ld = ld_part), or near.rec null
    int64_t ld_part;    // row stride of part and near (>= nq)
    int64_t row0;       // self-join: position in the series of query window 0
    int32_t excl;       // self-join: pairs with |g - (row0 + r)| < excl are left out (0: none)
};

// Asynchronous copy of one element from global to shared memory; zero-fills
// the destination when !valid (src is then not read).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t n = valid ? (uint32_t)sizeof(T) : 0u;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Padded shared-memory index: one pad slot every P elements, so that lanes
// reading with a stride of P (or P+...) hit distinct banks.
template <int P> __device__ __forceinline__ int pad(int e) { return e + e / P; }

// One work item: query rows [rb * rows_cta, (rb + 1) * rows_cta) against the
// spans of column group grp.
// Covariances C of a lane's kRows rows with their recurrence terms, and one
// step of the recurrence (one column to the right). The generic form is
// scalar. The FP32 form packs rows j and j + kRows/2 into one float2, so
// that one packed FMA (fma.rn.f32x2: each half rounded once, exactly as
// fmaf) advances two rows: moving one column right shifts every row down by
// one, which maps pair k-1 onto pair k, and only pair 0 takes new inputs
// (the row above the lane, and row kRows/2 - 1). The packed form pays off in
// k_plain; the batched serving kernel, at 8 warps per SM, cannot hide the
// packed FMA's longer pipe occupancy and stays scalar.
template <typename T, int kRows, bool kPacked> struct Rows {
    T C[kRows], df[kRows], dg[kRows];
    __device__ __forceinline__ void set_terms(int j, T f, T g)
    {
        df[j] = f;
        dg[j] = g;
    }
    __device__ __forceinline__ void set(int j, T v) { C[j] = v; }
    __device__ __forceinline__ T last() const { return C[kRows - 1]; }
    // x, y: df_b, dg_b of the new column; up: the row above the lane's first
    __device__ __forceinline__ void step(T x, T y, T up, bool take_seed, T seed)
    {
#pragma unroll
        for (int j = kRows - 1; j >= 1; --j) C[j] = fma(df[j], y, fma(x, dg[j], C[j - 1]));
        const T c0 = fma(df[0], y, fma(x, dg[0], up));
        C[0] = take_seed ? seed : c0;
    }
    // cm[j] = max(cm[j], C[j] * z + w)
    __device__ __forceinline__ void score_max(T z, T w, T *cm) const
    {
#pragma unroll
        for (int j = 0; j < kRows; ++j) cm[j] = fmax(cm[j], fma(C[j], z, w));
    }
    // two columns per 3-input maximum, as in the packed form below
    __device__ __forceinline__ void score(T z, T w, T *q) const
    {
#pragma unroll
        for (int j = 0; j < kRows; ++j) q[j] = fma(C[j], z, w);
    }
    __device__ __forceinline__ void score_max2(T z, T w, const T *q0, T *cm) const
    {
#pragma unroll
        for (int j = 0; j < kRows; ++j) cm[j] = fmax(cm[j], fmax(q0[j], fma(C[j], z, w)));
    }
    // the same, leaving out rows inside the column's exclusion zone
    // (|d0 - j| < excl, d0 = column window - the lane's first row)
    __device__ __forceinline__ void score_max_excl(T z, T w, T *cm, int d0, int excl) const
    {
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const T q = fma(C[j], z, w);
            cm[j] = fmax(cm[j], abs(d0 - j) < excl ? T(-INFINITY) : q);
        }
    }
};

template <int kRows> struct Rows<float, kRows, true> {
    static constexpr int H = kRows / 2;
    float2 C[H], df[H], dg[H];
    __device__ __forceinline__ void set_terms(int j, float f, float g)
    {
        if (j < H) {
            df[j].x = f;
            dg[j].x = g;
        } else {
            df[j - H].y = f;
            dg[j - H].y = g;
        }
    }
    __device__ __forceinline__ void set(int j, float v)
    {
        if (j < H)
            C[j].x = v;
        else
            C[j - H].y = v;
    }
    __device__ __forceinline__ float last() const { return C[H - 1].y; }
    // X = (df_b, df_b), Y = (dg_b, dg_b) of the new column
    __device__ __forceinline__ void step(float2 X, float2 Y, float up, bool take_seed, float seed)
    {
        const float2 in0 = make_float2(up, C[H - 1].x);
#pragma unroll
        for (int k = H - 1; k >= 1; --k) C[k] = __ffma2_rn(df[k], Y, __ffma2_rn(X, dg[k], C[k - 1]));
        C[0] = __ffma2_rn(df[0], Y, __ffma2_rn(X, dg[0], in0));
        C[0].x = take_seed ? seed : C[0].x;
    }
    // Z = (1/std_b, 1/std_b), W = (penalty, penalty)
    __device__ __forceinline__ void score_max(float2 Z, float2 W, float *cm) const
    {
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float2 q = __ffma2_rn(C[k], Z, W);
            cm[k] = fmaxf(cm[k], q.x);
            cm[k + H] = fmaxf(cm[k + H], q.y);
        }
    }
    // One column's recurrence step and its scores in one pass over the row
    // pairs: for the first column of a pair of columns the scores go to q, for
    // the second they fold with q into the running maxima. The same
    // arithmetic as step() followed by score() / score_max2(); this order lets
    // the compiler interleave each pair's multiply and maximum with the next
    // pair's recurrence (1 % faster than the two passes).
    template <bool kSecond>
    __device__ __forceinline__ void step_score(float2 X, float2 Y, float up, bool take_seed, float seed, float2 Z,
                                               float2 *q, float *cm)
    {
        const float2 in0 = make_float2(up, C[H - 1].x);
#pragma unroll
        for (int k = H - 1; k >= 0; --k) {
            C[k] = __ffma2_rn(df[k], Y, __ffma2_rn(X, dg[k], k > 0 ? C[k - 1] : in0));
            if (k == 0) C[0].x = take_seed ? seed : C[0].x;
            const float2 s = __fmul2_rn(C[k], Z);
            if (kSecond) {
                cm[k] = fmaxf(cm[k], fmaxf(q[k].x, s.x));
                cm[k + H] = fmaxf(cm[k + H], fmaxf(q[k].y, s.y));
            } else {
                q[k] = s;
            }
        }
    }
    // Two columns share one 3-input maximum per row: score() keeps the first
    // column's scores in q, score_max2() folds them with the second's. Here Z
    // is NaN on a column that may not be selected (constant window or
    // padding): the score C * Z is then NaN, which the maximum ignores, so a
    // packed multiply replaces the multiply-add with the penalty.
    __device__ __forceinline__ void score(float2 Z, float2 *q) const
    {
#pragma unroll
        for (int k = 0; k < H; ++k) q[k] = __fmul2_rn(C[k], Z);
    }
    __device__ __forceinline__ void score_max2(float2 Z, const float2 *q0, float *cm) const
    {
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float2 q = __fmul2_rn(C[k], Z);
            cm[k] = fmaxf(cm[k], fmaxf(q0[k].x, q.x));
            cm[k + H] = fmaxf(cm[k + H], fmaxf(q0[k].y, q.y));
        }
    }
    __device__ __forceinline__ void score_max_excl(float2 Z, float2 W, float *cm, int d0, int excl) const
    {
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float2 q = __ffma2_rn(C[k], Z, W);
            cm[k] = fmaxf(cm[k], abs(d0 - k) < excl ? -INFINITY : q.x);
            cm[k + H] = fmaxf(cm[k + H], abs(d0 - k - H) < excl ? -INFINITY : q.y);
        }
    }
};

// kSeeds: the top seeds come from p.seed_top (the tensor cores) instead of
// direct dot products; kNear: near ties are recorded in p.near; kPacked
// (FP32 only): packed FMA on row pairs; kSelf: a self-join whose trivial
// matches (|g - i| < p.excl) are left out, in the column blocks that reach
// them. All are compile-time so that each form carries only its own code.
template <typename T, int kRows, bool kSeeds, bool kNear, bool kPacked, bool kSelf = false>
__device__ __forceinline__ void plain_item(const PlainParams<T> &p, int64_t rb, int grp, unsigned char *smem_raw)
{
    constexpr int CB = kPlainColBlock;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int rows_cta = nwarps * 32 * kRows;
    const int64_t R0 = rb * rows_cta;
    const int m = p.m;
    const int m_up8 = (m + 7) & ~7;
    const int m_up16 = (m + 15) & ~15;

    // sa: shifted query samples a[R0 + e] - shift_a, e in [0, NA)
    const int NA = rows_cta + m_up16 + 32;
    T *sa = reinterpret_cast<T *>(smem_raw);
    const int NA_pad = pad<16>(NA) + 1;
    // sb: shifted dictionary samples of the current column block
    const int NB = CB + m_up8 + 16;
    T *sb = sa + NA_pad;
    const int NB_pad = pad<8>(NB) + 1;
    // stop: top seeds, one per (warp, column of the block)
    T *stop = sb + NB_pad;
    // scs: recurrence terms of the block's columns (padded to whole chunks),
    // (df, dg, 1/std, penalty), one vec4 per column (32 bytes for FP64 data,
    // 16 for FP32), 32-byte aligned. The packed form builds its operand pairs
    // (x, x) from one 128-bit load per column: storing the pairs themselves
    // (two loads per column) cost 14 % of the kernel's time, and two columns'
    // worth of spilled registers. Offset arithmetic on smem_raw keeps the
    // shared address space visible to the compiler (shared, not generic, loads).
    const size_t scs_off = ((size_t)(reinterpret_cast<unsigned char *>(stop + nwarps * CB) - smem_raw) + 31) &
                           ~static_cast<size_t>(31);
    vec4_t<T> *scs = reinterpret_cast<vec4_t<T> *>(smem_raw + scs_off);
    float4 *scs2 = reinterpret_cast<float4 *>(smem_raw + scs_off);

    const T shift_a = p.ms_a[R0 < p.nq ? R0 : p.nq - 1].hi;
    for (int e = threadIdx.x; e < NA; e += blockDim.x) {
        const int64_t j = R0 + e;
        sa[pad<16>(e)] = (j < p.na) ? (p.a[j] - shift_a) : T(0);
    }

    const int64_t r_w = R0 + (int64_t)warp * 32 * kRows;  // first row of this warp
    const int64_t r0 = r_w + (int64_t)lane * kRows;       // first row of this lane
    constexpr bool kPack = kPacked && sizeof(T) == 4;
    Rows<T, kRows, kPack> R;
    T best[kRows];
    int32_t bchunk[kRows];  // first window of the chunk holding the row's best score
    T sig_max = T(0);       // largest std of the lane's (non-constant) rows
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
        const int64_t r = r0 + j;
        if (r < p.nq) {
            const vec4_t<T> v = p.rs_a[r];
            R.set_terms(j, v.x, v.y);
            if (kNear) {
                if (v.z > T(0)) sig_max = fmax(sig_max, T(1) / v.z);
                *p.near.head(grp, r) = NearSlot{0, 0.f};  // no records yet, empty overflow mask
            }
        } else {
            R.set_terms(j, T(0), T(0));
        }
        R.set(j, T(0));
        best[j] = T(-INFINITY);
        bchunk[j] = -1;
    }
    // near-tie width in units of the score q = C * invstd_b (q = rho * m * std_a),
    // taken with the lane's largest std so that it covers every row of the lane
    const T tq = T(p.near.rho) * T(m) * sig_max;
    const Split<T> mw = p.ms_a[r_w < p.nq ? r_w : p.nq - 1];
    const T da_w = (mw.hi - shift_a) + mw.lo;
    const int sa_w = warp * 32 * kRows;      // sa index of this warp's first row
    const int sa_l = sa_w + lane * kRows;    // sa index of this lane's first row

    const int s_lo = p.group_start[grp], s_hi = p.group_start[grp + 1];
    for (int s = s_lo; s < s_hi; ++s) {
        const Span sp = p.spans[s];
        for (int cb = 0; cb < sp.ncols; cb += CB) {
            const int ncb = min(CB, sp.ncols - cb);
            const int64_t gblk = sp.g0 + cb;
            const T shift_b = p.ms_b[gblk].hi;
            // top seeds from the tensor cores: this warp's row of them for the
            // block's columns, copied to shared memory asynchronously so the
            // latency overlaps the staging (zeros past the block / the rows)
            if (kSeeds) {
                __syncwarp();  // lane 0 has read this warp's seeds of the previous block
                const bool wok = r_w < p.nq;
                const T *src = p.seed_top + (wok ? r_w / (32 * kRows) : 0) * p.seed_ld + gblk;
#pragma unroll
                for (int t = 0; t < CB / 32; ++t) {
                    const int c = lane + 32 * t;
                    const bool v = wok && c < ncb;
                    cp_async_elem(&stop[warp * CB + c], v ? src + c : p.seed_top, v);
                }
            }
            __syncthreads();  // previous block's sb / stop no longer in use
            for (int e = threadIdx.x; e < NB; e += blockDim.x) {
                const int64_t j = gblk + e;
                sb[pad<8>(e)] = (j < p.nb) ? (p.b[j] - shift_b) : T(0);
            }
            const int ncb_up = (ncb + kChunk - 1) / kChunk * kChunk;
            for (int c = threadIdx.x; c < ncb_up; c += blockDim.x) {
                vec4_t<T> v;
                if (c < ncb) {
                    v = p.rs_b[gblk + c];
                } else {  // padding columns: no recurrence change, never selected
                    v.x = T(0);
                    v.y = T(0);
                    v.z = T(0);
                    v.w = T(-INFINITY);
                }
                if constexpr (kPack) {
                    // z = NaN where the penalty is -inf (the packed scores are C * z)
                    scs2[c] = make_float4(v.x, v.y, v.w < T(0) ? __int_as_float(0x7fc00000) : v.z, v.w);
                } else {
                    scs[c] = v;
                }
            }
            __syncthreads();

            // ---- top seeds: C(r_w, gblk + c) for c in [8*lane, 8*lane + 8) ----
            if (kSeeds) {
                cp_async_wait_all();  // the __syncwarp below publishes them to lane 0
            } else {
                T acc[8], bw[8];
                const int c0 = 8 * lane;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    acc[t] = T(0);
                    bw[t] = sb[pad<8>(c0 + t)];
                }
                for (int k0 = 0; k0 < m_up8; k0 += 8) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = k0 + u;
                        const T xk = (k < m) ? sa[pad<16>(sa_w + k)] : T(0);
#pragma unroll
                        for (int t = 0; t < 8; ++t) acc[t] = fma(xk, bw[(t + u) & 7], acc[t]);
                        bw[u] = sb[pad<8>(c0 + 8 + k)];
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int c = c0 + t;
                    if (c < ncb) {
                        const Split<T> mb = p.ms_b[gblk + c];
                        const T db = (mb.hi - shift_b) + mb.lo;
                        stop[warp * CB + c] = acc[t] - T(m) * da_w * db;
                    } else {
                        stop[warp * CB + c] = T(0);
                    }
                }
            }

            // ---- left seeds at the first column of the span ----
            if (kSeeds && cb == 0) {
                // from the tensor cores: the centred covariances of the lane's
                // rows with the span's first window
                const T *lp = p.left + (int64_t)s * p.left_ld + r0;
#pragma unroll
                for (int j = 0; j < kRows; ++j) R.set(j, r0 + j < p.nq ? lp[j] : T(0));
            } else if (cb == 0) {
                T acc[kRows];
#pragma unroll
                for (int j = 0; j < kRows; ++j) acc[j] = T(0);
                // rows in passes of up to 16, each with a sliding window of 16 query samples
#pragma unroll
                for (int j0 = 0; j0 < kRows; j0 += 16) {
                    T aw[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) aw[t] = sa[pad<16>(sa_l + j0 + t)];
                    for (int k0 = 0; k0 < m_up16; k0 += 16) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int k = k0 + u;
                            const T bk = (k < m) ? sb[pad<8>(k)] : T(0);
#pragma unroll
                            for (int j = j0; j < kRows && j < j0 + 16; ++j)
                                acc[j] = fma(aw[(j - j0 + u) & 15], bk, acc[j]);
                            aw[u] = sa[pad<16>(sa_l + j0 + 16 + k)];
                        }
                    }
                }
                const T db0 = p.ms_b[gblk].lo;  // shift_b is this window's mean rounded
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const int64_t r = r0 + j;
                    const Split<T> ma = p.ms_a[r < p.nq ? r : p.nq - 1];
                    const T da = (ma.hi - shift_a) + ma.lo;
                    R.set(j, acc[j] - T(m) * da * db0);
                }
            }
            __syncwarp();

            // ---- main loop: one dictionary window (column) per step, in
            // chunks of kChunk columns. Only the running maximum of each
            // row's score is kept per step; the chunk that raised it is
            // recorded, and the finalisation re-scores that chunk's
            // windows to find the exact one.
            const T *stop_w = stop + warp * CB;
            // self-join: does this block reach the exclusion zone of any of the CTA's rows?
            bool band = false;
            int d_lane = 0;  // column gblk - this lane's first row, clamped (only compared with small values)
            if (kSelf) {
                const int64_t a0 = p.row0 + R0;
                band = gblk < a0 + rows_cta - 1 + p.excl && gblk + ncb - 1 > a0 - p.excl;
                const int64_t dl = gblk - (p.row0 + r0);
                d_lane = (int)(dl > (1 << 30) ? (1 << 30) : (dl < -(1 << 30) ? -(1 << 30) : dl));
            }
            for (int c0 = 0; c0 < ncb; c0 += kChunk) {
                T cm[kRows];
#pragma unroll
                for (int j = 0; j < kRows; ++j) cm[j] = T(-INFINITY);
                if constexpr (kPack && !kSelf) {
                    // packed form: columns in pairs, one 3-input maximum per row and pair
                    float2 q0[kRows / 2];
#pragma unroll
                    for (int u = 0; u < kChunk; ++u) {
                        const int c = c0 + u;
                        const float4 cv = scs2[c];
                        if (cb > 0 || c > 0) {
                            const float up = __shfl_up_sync(0xffffffffu, R.last(), 1);
                            if ((u & 1) == 0)
                                R.template step_score<false>(make_float2(cv.x, cv.x), make_float2(cv.y, cv.y), up,
                                                             lane == 0, stop_w[c], make_float2(cv.z, cv.z), q0, cm);
                            else
                                R.template step_score<true>(make_float2(cv.x, cv.x), make_float2(cv.y, cv.y), up,
                                                            lane == 0, stop_w[c], make_float2(cv.z, cv.z), q0, cm);
                        } else if ((u & 1) == 0) {  // a span's first column holds its left seeds: no step
                            R.score(make_float2(cv.z, cv.z), q0);
                        } else {
                            R.score_max2(make_float2(cv.z, cv.z), q0, cm);
                        }
                    }
                } else if constexpr (!kPack && !kSelf && sizeof(T) == 4) {
                    // scalar FP32 form (serving): the same pairing of columns
                    T q0[kRows];
#pragma unroll
                    for (int u = 0; u < kChunk; ++u) {
                        const int c = c0 + u;
                        const vec4_t<T> cs = scs[c];
                        if (cb > 0 || c > 0) {
                            const T up = __shfl_up_sync(0xffffffffu, R.last(), 1);
                            R.step(cs.x, cs.y, up, lane == 0, stop_w[c]);
                        }
                        if ((u & 1) == 0)
                            R.score(cs.z, cs.w, q0);
                        else
                            R.score_max2(cs.z, cs.w, q0, cm);
                    }
                } else
#pragma unroll
                for (int u = 0; u < kChunk; ++u) {
                    const int c = c0 + u;
                    if constexpr (kPack) {
                        const float4 cv = scs2[c];
                        const float4 cxy = make_float4(cv.x, cv.x, cv.y, cv.y);
                        const float4 czw = make_float4(cv.z, cv.z, cv.w, cv.w);
                        if (cb > 0 || c > 0) {
                            const float up = __shfl_up_sync(0xffffffffu, R.last(), 1);
                            R.step(make_float2(cxy.x, cxy.y), make_float2(cxy.z, cxy.w), up, lane == 0, stop_w[c]);
                        }
                        if (kSelf && band)
                            R.score_max_excl(make_float2(czw.x, czw.y), make_float2(czw.z, czw.w), cm, d_lane + c,
                                             p.excl);
                        else
                            R.score_max(make_float2(czw.x, czw.y), make_float2(czw.z, czw.w), cm);
                    } else {
                        const vec4_t<T> cs = scs[c];
                        if (cb > 0 || c > 0) {
                            const T up = __shfl_up_sync(0xffffffffu, R.last(), 1);
                            R.step(cs.x, cs.y, up, lane == 0, stop_w[c]);
                        }
                        if (kSelf && band)
                            R.score_max_excl(cs.z, cs.w, cm, d_lane + c, p.excl);
                        else
                            R.score_max(cs.z, cs.w, cm);
                    }
                }
                const int32_t gch = (int32_t)(gblk + c0);
                if (kNear) {
                    // near ties: a chunk within tq below the running best, or a
                    // best overtaken by less than tq (-inf on either side gives
                    // inf or NaN, which fmin skips: no tie). One test per row,
                    // one branch per chunk.
                    T mn = T(INFINITY);
#pragma unroll
                    for (int j = 0; j < kRows; ++j) mn = fmin(mn, fabs(cm[j] - best[j]));
                    if (mn <= tq) {
#pragma unroll
                        for (int j = 0; j < kRows; ++j) {
                            if (fabs(cm[j] - best[j]) <= tq && r0 + j < p.nq) {
                                const bool upd = cm[j] > best[j];
                                // with all slots in use the new record is dropped (an
                                // eviction loop in each of the kRows unrolled copies
                                // cost 6 % of the kernel's time)
                                near_add<false>(p.near, grp, r0 + j, upd ? bchunk[j] : gch,
                                                (float)(upd ? best[j] : cm[j]), (float)(fmax(cm[j], best[j]) - tq));
                            }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const bool upd = cm[j] > best[j];
                    best[j] = upd ? cm[j] : best[j];
                    bchunk[j] = upd ? gch : bchunk[j];
                }
            }
        }
    }

#pragma unroll
    for (int j = 0; j < kRows; ++j) {
        const int64_t r = r0 + j;
        if (r < p.nq) {
            Partial<T> v;
            v.q = best[j];
            v.g = bchunk[j];
            p.part[(int64_t)grp * p.ld_part + r] = v;
        }
    }
}

// Three CTAs (12 warps) per SM for FP32 data, with 20 rows per lane in 168
// registers and no spills. More rows per lane spread the per-column work
// (shuffle, column terms, seed select) and the per-chunk argmax over more
// pairs, and mean fewer top seeds; that gained more than the 16 warps of 16
// rows per lane at 128 registers hid.
// The short form (kPlainRowsShort rows per lane) takes 6 CTAs per SM.
template <typename T, int kRows, bool kSeeds, bool kNear, bool kSelf = false>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (kRows <= kPlainRowsShort ? 6 : 3) : 1) k_plain(PlainParams<T> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    plain_item<T, kRows, kSeeds, kNear, true, kSelf>(p, blockIdx.x / p.n_groups, blockIdx.x % p.n_groups, smem_raw);
}

// Persistent batched form for serving: the CTAs walk a list of work items that
// may belong to different requests (different query, dictionary and m). Items
// are claimed in list order with a global counter.
template <typename T, int kRows, bool kNear>
__global__ void __launch_bounds__(128, 2) k_plain_batched(const PlainParams<T> *__restrict__ reqs,
                                                       const BatchItem *__restrict__ items, int32_t n_items,
                                                       int32_t *__restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t next;
    for (;;) {
        __syncthreads();  // every thread has read the previous `next`
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int32_t it = next;
        if (it >= n_items) break;
        const BatchItem bi = items[it];
        const PlainParams<T> p = reqs[bi.req];
        plain_item<T, kRows, false, kNear, false>(p, bi.rb, bi.grp, smem_raw);  // seeds computed here, scalar FMA
    }
}

}  // namespace

template <typename T>
size_t plain_smem_bytes(int warps, int m, int rows_per_lane)
{
    const int rows_cta = warps * 32 * rows_per_lane;
    const int m_up8 = (m + 7) & ~7, m_up16 = (m + 15) & ~15;
    const int NA = rows_cta + m_up16 + 32;
    const int NB = kPlainColBlock + m_up8 + 16;
    const size_t scalars = (size_t)(NA + NA / 16 + 1) + (size_t)(NB + NB / 8 + 1) + (size_t)warps * kPlainColBlock;
    // + 32: the column-term array (up to 32 bytes per column) is aligned up to 32 bytes
    return sizeof(T) * scalars + 32 + 32 * (size_t)kPlainColBlock;
}

template <typename T>
cudaError_t launch_plain(const PlainLaunch &L, const T *a, int64_t na, const vec4_t<T> *rs_a, const Split<T> *ms_a,
                         const T *b, int64_t nb, const vec4_t<T> *rs_b, const Split<T> *ms_b, const Span *spans,
                         const int32_t *group_start, Partial<T> *part, const T *seed_top, int64_t seed_ld,
                         const T *left, int64_t left_ld, const NearRec &near, cudaStream_t st)
{
    PlainParams<T> p{};
    p.a = a;
    p.na = na;
    p.nq = L.nq;
    p.m = L.m;
    p.n_groups = L.n_groups;
    p.rs_a = rs_a;
    p.ms_a = ms_a;
    p.b = b;
    p.nb = nb;
    p.rs_b = rs_b;
    p.ms_b = ms_b;
    p.spans = spans;
    p.group_start = group_start;
    p.part = part;
    p.seed_top = seed_top;
    p.seed_ld = seed_ld;
    p.left = left;
    p.left_ld = left_ld;
    p.near = near;
    p.ld_part = L.ld_part > 0 ? L.ld_part : L.nq;
    p.row0 = L.row0;
    p.excl = L.excl;
    constexpr int R = plain_rows_per_lane<T>();
    const bool short_form = sizeof(T) == 4 && L.rows_per_lane == kPlainRowsShort;
    if (L.rows_per_lane != 0 && L.rows_per_lane != R && !short_form) return cudaErrorInvalidValue;
    const size_t smem = plain_smem_bytes<T>(L.warps, L.m, short_form ? kPlainRowsShort : R);
    const int64_t grid = (int64_t)L.n_row_blocks * L.n_groups;
    auto launch = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, 32 * L.warps, smem, st>>>(p);
        return cudaGetLastError();
    };
    if constexpr (sizeof(T) == 8) {
        // FP64 data: seeds from direct dot products, no near-tie records
        if (seed_top != nullptr || left != nullptr || near.rec != nullptr || L.excl > 0) return cudaErrorInvalidValue;
        return launch(k_plain<T, R, false, false>);
    } else {
        if (near.rec != nullptr && (near.ld != p.ld_part || near.S < 1 || near.S > kNearMaxSlots))
            return cudaErrorInvalidValue;
        if ((seed_top == nullptr) != (left == nullptr)) return cudaErrorInvalidValue;  // both seeds, or neither
        if (short_form) {
            // short join: seeds computed in the kernel, 4 rows per lane
            if (seed_top != nullptr || L.excl > 0) return cudaErrorInvalidValue;
            return near.rec != nullptr ? launch(k_plain<T, kPlainRowsShort, false, true>)
                                       : launch(k_plain<T, kPlainRowsShort, false, false>);
        }
        if (L.excl > 0) {
            // self-join (dictionary learning): tensor-core seeds and near-tie records
            if (seed_top == nullptr || near.rec == nullptr) return cudaErrorInvalidValue;
            return launch(k_plain<T, R, true, true, true>);
        }
        if (seed_top != nullptr)
            return near.rec != nullptr ? launch(k_plain<T, R, true, true>) : launch(k_plain<T, R, true, false>);
        return near.rec != nullptr ? launch(k_plain<T, R, false, true>) : launch(k_plain<T, R, false, false>);
    }
}

cudaError_t launch_plain_batched(const PlainRequest *reqs_dev, const BatchItem *items, int32_t n_items,
                                 int32_t *counter, int warps, int max_m, int grid, cudaStream_t st)
{
    static_assert(sizeof(PlainRequest) == sizeof(PlainParams<float>), "request layout");
    const size_t smem = plain_smem_bytes<float>(warps, max_m, kServeRowsPerLane);
    auto kern = k_plain_batched<float, kServeRowsPerLane, true>;  // every request carries near-tie slots
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * warps, smem, st>>>(reinterpret_cast<const PlainParams<float> *>(reqs_dev), items, n_items,
                                         counter);
    return cudaGetLastError();
}

template <typename T>
int plain_ctas_per_sm(int warps, int m, int rows_per_lane)
{
    int n = 0;
    constexpr int R = plain_rows_per_lane<T>();
    const bool short_form = sizeof(T) == 4 && rows_per_lane == kPlainRowsShort;
    const size_t smem = plain_smem_bytes<T>(warps, m, short_form ? kPlainRowsShort : R);
    cudaError_t e;
    if constexpr (sizeof(T) == 8)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain<T, R, false, false>, 32 * warps, smem);
    else if (short_form)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain<T, kPlainRowsShort, false, true>, 32 * warps,
                                                          smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain<T, R, true, true>, 32 * warps, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template int plain_ctas_per_sm<float>(int, int, int);
template int plain_ctas_per_sm<double>(int, int, int);
template size_t plain_smem_bytes<float>(int, int, int);
template size_t plain_smem_bytes<double>(int, int, int);
template cudaError_t launch_plain<float>(const PlainLaunch &, const float *, int64_t, const float4 *,
                                         const Split<float> *, const float *, int64_t, const float4 *,
                                         const Split<float> *, const Span *, const int32_t *, Partial<float> *,
                                         const float *, int64_t, const float *, int64_t, const NearRec &,
                                         cudaStream_t);
template cudaError_t launch_plain<double>(const PlainLaunch &, const double *, int64_t, const dvec4 *,
                                          const Split<double> *, const double *, int64_t, const dvec4 *,
                                          const Split<double> *, const Span *, const int32_t *, Partial<double> *,
                                          const double *, int64_t, const double *, int64_t, const NearRec &,
                                          cudaStream_t);

}  // namespace mpd

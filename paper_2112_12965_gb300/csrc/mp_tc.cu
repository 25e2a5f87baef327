// K3: the tensor-core form of the dictionary AB-join (tcgen05, sm_103a).
//
// The join's dot products QT[i, g] = sum_k a[i+k] * b[g+k] (Algorithm 2's
// per-segment AB-join, Sec. 3.2) form, for a block of 128 query windows and N
// dictionary windows, a dense product of two Hankel matrices with K = m:
//     QT = A * B^T,  A[r, k] = a[i0 + r + k],  B[n, k] = b[g0 + n + k].
// A CTA owns 128 query windows (the 128 TMEM lanes) and walks tiles of up to
// 256 dictionary windows that never cross a segment (Def. 8). Accumulators are
// FP32 in TMEM; the products are either one TF32 product or three BF16
// products of a hi/lo split (x = hi + lo: hi*hi + hi*lo + lo*hi).
//
// Hankel operands in shared memory. The MMA reads K-major operands in 128-byte
// swizzled rows (64 BF16 or 32 TF32 values of K per row). Row rho of a
// "row-shifted Hankel" buffer holds samples [base + rho, base + rho + E),
// E = values per row. The operand of K-block q (K values [qE, qE + E)) is then
// the same buffer starting at row qE, so one buffer of (K-blocks - 1) E + rows
// rows serves every K-block: its descriptor start moves by qE rows (a multiple
// of 8 rows = 1024 bytes, so the swizzle phase is unchanged), and the four
// MMAs inside a 128-byte row step the start address by 32 bytes.
//
// The query operand is built once per CTA for all of K. The dictionary operand
// is built per tile and per K-group (a run of K-blocks sized to fit shared
// memory). After the last K-group the epilogue reads the accumulators with
// tcgen05.ld (one query window per thread), removes the shifts, scales by the
// dictionary windows' 1/std, masks invalid and constant windows and keeps the
// running maximum per 16-window chunk, as the plain kernel does, with the same
// near-tie records (their width covers the products' rounding: the TF32 form's
// 11-bit operands need a wider one than the split-BF16 form).
//
// Every wait on the tensor core is bounded: on timeout the CTA records an
// error, waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>
#include <stddef.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "../../include/mpdict.h"
#include "mp_tc.cuh"

namespace mpd {
namespace {

constexpr int kTcMaxN = 256;           // TMEM columns (FP32 accumulators) per CTA
constexpr long long kTcWaitCycles = 4000000000LL;  // bound of a wait, about 2 s
constexpr size_t kTcSmemLimit = 225 * 1024;

struct TcTile {
    int64_t g0;      // first dictionary window of the tile
    int32_t nvalid;  // valid windows in the tile
    int32_t nmma;    // MMA N: nvalid rounded up to 16
};

struct TcArgs {
    const float *a;
    int64_t na, nq;
    int32_t m;
    int32_t n_groups;
    const Split<float> *ms_a;  // query window means, split
    const float *b;
    int64_t nb;
    const Split<float> *ms_b;  // dictionary window means, split
    const float4 *rs_b;        // z = 1/std (0: constant or invalid), w = 0 or -inf
    const TcTile *tiles;
    const int32_t *group_start;
    Partial<float> *part;
    const float4 *rs_a;  // query terms (z = 1/std, 0 for a constant window)
    NearRec near;        // near-tie records (ld = nq), or near.rec null
    int32_t *err;
    int32_t ra_rows;   // rows of the query Hankel buffer
    int32_t nmax;      // widest tile
    int32_t nkb;       // K-blocks
    int32_t qg;        // K-blocks per stage (one stage = one tile's K-group)
    int32_t rb_rows;   // rows of a stage buffer: (qg - 1) * values-per-row + nmax
    int32_t n_stages;  // stage buffers in flight (1 or 2)
    long long wait_cycles;  // bound of the roles' waits on each other (clocks)
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a phase of the barrier: false after about `cycles` clocks.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);      // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                        // 128-byte swizzle
    return d;
}

template <int VARIANT>
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    // D = F32 (bits 4-5), A/B format (bits 7-9, 10-12): BF16 = 1, TF32 = 2;
    // both K-major; N >> 3 at bits 17-22; M >> 4 at bits 24-28 (M = 128).
    const uint32_t fmt = (VARIANT == 0 || VARIANT == 3) ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int VARIANT>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (VARIANT == 0 || VARIANT == 3)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Write one 16-byte chunk (EPC values) of an operand row: BF16 hi and lo
// halves (VARIANT 0), TF32 values (1), TF32 hi and lo halves (2), or BF16
// values (3).
template <int VARIANT>
__device__ __forceinline__ void put_chunk(const float *x, unsigned char *hi, unsigned char *lo, uint32_t off)
{
    if (VARIANT == 0) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            // packed conversions: two values per instruction
            const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
            const __nv_bfloat162 ll =
                __floats2bfloat162_rn(x[2 * e] - __low2float(hh), x[2 * e + 1] - __high2float(hh));
            h[e] = *reinterpret_cast<const uint32_t *>(&hh);
            l[e] = *reinterpret_cast<const uint32_t *>(&ll);
        }
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    } else if (VARIANT == 1) {
        *reinterpret_cast<float4 *>(hi + off) = make_float4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
    } else if (VARIANT == 3) {
        uint32_t h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
            h[e] = *reinterpret_cast<const uint32_t *>(&hh);
        }
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    } else {
        // TF32 hi and lo halves (x - hi is exact in FP32)
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = to_tf32(x[e]);
            l[e] = to_tf32(x[e] - h[e]);
        }
        *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// Build rows [0, rows) of a row-shifted Hankel buffer from staged samples
// raw[0 ..]: row rho, value j = raw[rho + j]. 16-byte chunk c of row rho is
// stored at chunk position c ^ (rho & 7) (the 128-byte swizzle). Thread t of
// nthr (a multiple of 8) owns chunk column c = t % 8 of a contiguous run of
// rows and slides a register window down them: one shared-memory load per
// chunk instead of one per value.
template <int VARIANT>
__device__ __forceinline__ void build_hankel(const float *raw, int rows, unsigned char *hi, unsigned char *lo, int t,
                                             int nthr)
{
    constexpr int EPC = (VARIANT == 0 || VARIANT == 3) ? 8 : 4;  // values per 16-byte chunk
    const int c = t & 7, groups = nthr >> 3, rg = t >> 3;
    const int rpg = (rows + groups - 1) / groups;
    const int r0 = rg * rpg, r1 = min(rows, r0 + rpg);
    if (r0 >= r1) return;
    float w[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) w[e] = raw[r0 + c * EPC + e];
    for (int rb = r0; rb < r1; rb += EPC) {
#pragma unroll
        for (int u = 0; u < EPC; ++u) {
            const int rho = rb + u;
            if (rho < r1) {
                float x[EPC];
#pragma unroll
                for (int e = 0; e < EPC; ++e) x[e] = w[(u + e) % EPC];
                put_chunk<VARIANT>(x, hi, lo, (uint32_t)rho * 128u + (uint32_t)((c ^ (rho & 7)) << 4));
                // slot u held raw[rho + c*EPC]; replace it with the value row rho + EPC needs last
                w[u] = raw[rho + c * EPC + EPC];
            }
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Two bulk asynchronous copies of `bytes` each (a multiple of 16; every
// address 16-byte aligned) from global to this CTA's shared memory, both
// completing on `bar`, which this call arms with their byte count.
__device__ __forceinline__ void bulk_copy2_g2s(void *dst0, const void *src0, void *dst1, const void *src1,
                                               uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(2u * bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst0)),
                 "l"(src0), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst1)),
                 "l"(src1), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bulk asynchronous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on `bar`,
// which this call arms with the expected byte count (one arrival).
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ANDs a predicate over its threads, so that every
// thread of a role takes the same branch after a wait that may have failed.
__device__ __forceinline__ bool named_sync_and(int id, int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Bounded wait (about `limit` clocks) that also gives up as soon as another
// role has aborted.
__device__ __forceinline__ bool role_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Warp roles of the pipelined kernel.
constexpr int kMmaWarp = 0;                  // TMEM owner; lane 0 issues the MMAs
constexpr int kBuildWarp0 = 1;               // warps 1..8 build operand stages (two groups of 4)
constexpr int kEpiWarp0 = 9;                 // warps 9..12 read the accumulators
constexpr int kTcThreadsP = 13 * 32;
constexpr int kRoleThreads = 128;            // threads of one builder group / of the epilogue
constexpr int kBuildThreads = 256;           // all builders
constexpr int kBarBuild = 1, kBarGroup0 = 2, kBarEpi = 4;  // named barriers (group g uses kBarGroup0 + g)
constexpr uint32_t kTmemCols = 2 * kTcMaxN;  // two accumulators of 256 FP32 columns

// The join of 128 query windows (one CTA) against the tiles of one column
// group. A stage holds the dictionary operand of one tile for one K-block
// (64 BF16 / 32 TF32 values of K); builders fill stage s while the MMAs read
// the other; each tile's accumulator alternates between two TMEM buffers so
// that the epilogue of tile t overlaps the MMAs of tile t + 1.
template <int VARIANT>
__global__ void __launch_bounds__(kTcThreadsP, 1) k_tc(TcArgs p)
{
    // VARIANT 0: split BF16 (3 products), 1: TF32, 3: single BF16 product
    constexpr bool kBF = VARIANT == 0 || VARIANT == 3;
    constexpr int EPR = kBF ? 64 : 32;       // K values per 128-byte row (one K-block)
    constexpr int KSTEP = kBF ? 16 : 8;      // K values per MMA
    constexpr int NHL = VARIANT == 0 ? 2 : 1;  // hi/lo buffers

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int NS = p.n_stages;
    const uint32_t a_bytes = (uint32_t)p.ra_rows * 128u, st_bytes = (uint32_t)p.rb_rows * 128u;
    unsigned char *ha[2] = {base, base + a_bytes};
    unsigned char *hb = base + NHL * a_bytes;  // stage s, half h at hb + (s * NHL + h) * st_bytes
    float *raw = reinterpret_cast<float *>(hb + NS * NHL * st_bytes);  // query staging, then two tile stagings
    const int raw_tile = p.nmax + p.m + EPR;  // samples a tile's stages read
    const int raw_a = p.ra_rows + EPR;
    // a tile buffer also holds the bulk copy's alignment slack (up to 3 values
    // before the tile, rounding to 4 after): raw_tile + 8 values, 16-byte aligned
    const int raw_tb = raw_tile + 8;
    float *raw_b[2] = {raw + raw_a, raw + raw_a + raw_tb};
    float4 *colp = reinterpret_cast<float4 *>(raw + ((raw_a + 2 * raw_tb + 3) & ~3));
    uint64_t *bars = reinterpret_cast<uint64_t *>(colp + kTcMaxN);
    uint64_t *full_a = bars + 0;
    uint64_t *full_b = bars + 1;     // [2]
    uint64_t *empty_b = bars + 3;    // [2]
    uint64_t *acc_full = bars + 5;   // [2]
    uint64_t *acc_empty = bars + 7;  // [2]
    uint64_t *drain = bars + 9;
    uint64_t *copy_b = bars + 10;    // [2]: bulk copies of the tile samples
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 12);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t rb = blockIdx.x / p.n_groups;
    const int grp = blockIdx.x % p.n_groups;
    const int64_t i0 = rb * 128;
    const int m = p.m;
    const int t_lo = p.group_start[grp], t_hi = p.group_start[grp + 1];

    if (warp == kMmaWarp) tmem_alloc(tmem_slot, kTmemCols);
    if (tid == 0) {
        *abort_flag = 0;
        mbar_init(full_a, kBuildThreads);
        for (int s = 0; s < 2; ++s) {
            // two stages: each is built by one builder group; one stage: by both
            mbar_init(&full_b[s], NS == 2 ? kRoleThreads : kBuildThreads);
            mbar_init(&empty_b[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kRoleThreads);
        }
        mbar_init(drain, 1);
        mbar_init(&copy_b[0], 1);
        mbar_init(&copy_b[1], 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    if (warp == kMmaWarp) {
        // ---------------- MMA issue (one lane) ----------------
        if (lane == 0) {
            bool ok = role_wait(full_a, 0, abort_flag, p.wait_cycles);
            tc_fence_after();
            const uint32_t a0 = smem_u32(ha[0]), a1 = smem_u32(ha[NHL - 1]);
            int j = 0;  // stage counter
            for (int t = t_lo; ok && t < t_hi; ++t) {
                const TcTile tile = p.tiles[t];
                const int ab = (t - t_lo) & 1;
                const int k_t = (t - t_lo) >> 1;
                if (k_t >= 1 && !(ok = role_wait(&acc_empty[ab], (k_t - 1) & 1, abort_flag, p.wait_cycles))) break;
                tc_fence_after();
                const uint32_t d_tmem = taddr + (uint32_t)(ab * kTcMaxN);
                const uint32_t idesc = instr_desc<VARIANT>(tile.nmma);
                for (int q0 = 0; q0 < p.nkb; q0 += p.qg, ++j) {
                    const int q1 = min(p.nkb, q0 + p.qg);
                    const int s = j % NS;
                    if (!(ok = role_wait(&full_b[s], (j / NS) & 1, abort_flag, p.wait_cycles))) break;
                    tc_fence_after();
                    const uint32_t b0 = smem_u32(hb + (s * NHL) * st_bytes);
                    const uint32_t b1 = smem_u32(hb + (s * NHL + NHL - 1) * st_bytes);
                    for (int q = q0; q < q1; ++q) {
                        const uint32_t ao = (uint32_t)(q * EPR) * 128u, bo = (uint32_t)((q - q0) * EPR) * 128u;
                        const int ksteps = min(EPR, m - q * EPR) / KSTEP;
                        for (int k = 0; k < ksteps; ++k) {
                            const uint32_t acc0 = (q == 0 && k == 0) ? 0u : 1u;
                            mma<VARIANT>(d_tmem, smem_desc(a0 + ao + 32u * k), smem_desc(b0 + bo + 32u * k), idesc,
                                         acc0);
                            if (VARIANT == 0) {
                                mma<VARIANT>(d_tmem, smem_desc(a0 + ao + 32u * k), smem_desc(b1 + bo + 32u * k),
                                             idesc, 1u);
                                mma<VARIANT>(d_tmem, smem_desc(a1 + ao + 32u * k), smem_desc(b0 + bo + 32u * k),
                                             idesc, 1u);
                            }
                        }
                    }
                    mma_commit(&empty_b[s]);  // stage s is free once these MMAs are done
                }
                if (!ok) break;
                mma_commit(&acc_full[ab]);  // tile t's accumulator is complete
            }
            // every MMA issued so far must finish before the TMEM is released
            mma_commit(drain);
            // (a bound of its own, never shortened: the TMEM is freed only after it)
            role_wait(drain, 0, abort_flag, p.wait_cycles) || mbar_wait(drain, 0, kTcWaitCycles);
        }
        __syncwarp();
    } else if (warp < kEpiWarp0) {
        // ---------------- operand builders ----------------
        // Two groups of four warps. With two stage buffers, group g builds
        // stage buffer g (every other stage), so each group has two stages'
        // worth of MMA time per build; with one buffer both groups build it.
        const int bt = tid - kBuildWarp0 * 32;  // 0 .. 255
        const int bgrp = bt >> 7, gt = bt & (kRoleThreads - 1);
        // Each tile's samples b[g0 .. g0 + nmma + m + values-per-row) are staged
        // once in shared memory (two tile buffers). One builder copies the
        // next tile's samples with a bulk asynchronous copy (cp.async.bulk,
        // completing on an mbarrier) at the top of the current tile, so that
        // the copy overlaps the current tile's builds and MMAs; at the tile's
        // end the builders shift them in place by the next tile's mean.
        constexpr int kPre = 6;  // covers nmax + m + values-per-row <= kPre * 256
        float pre[kPre];
        int issued0 = 0, issued1 = 0;  // bt == 0: copies issued into each buffer
        auto issue_copy = [&](int t) {
            const TcTile tl = p.tiles[t];
            const int buf = (t - t_lo) & 1;
            const int64_t a = tl.g0 & ~(int64_t)3;  // 16-byte aligned source
            int64_t c = (tl.g0 - a + raw_tile + 3) & ~(int64_t)3;
            const int64_t lim = (p.nb + 16 - a) & ~(int64_t)3;  // the dictionary buffer's readable end
            if (c > lim) c = lim;
            fence_async_smem();  // the buffer's earlier (generic) accesses come first
            bulk_copy_g2s(raw_b[buf], p.b + a, (uint32_t)c * 4u, &copy_b[buf]);
            issued0 += buf == 0;
            issued1 += buf == 1;
        };
        // wait for tile t's copy and shift its samples to the start of the
        // buffer (zeros past the dictionary); false if a wait gave up
        auto land_tile = [&](int t) -> bool {
            const int buf = (t - t_lo) & 1;
            const bool w = role_wait(&copy_b[buf], ((t - t_lo) >> 1) & 1, abort_flag, p.wait_cycles);
            if (!named_sync_and(kBarBuild, kBuildThreads, w)) return false;
            const TcTile tl = p.tiles[t];
            const float sb = p.ms_b[tl.g0].hi;
            const int o = (int)(tl.g0 & 3);
            float *dst = raw_b[buf];
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                const int e = bt + k * kBuildThreads;
                pre[k] = (e < raw_tile && tl.g0 + e < p.nb) ? dst[o + e] - sb : 0.f;
            }
            named_sync(kBarBuild, kBuildThreads);
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                const int e = bt + k * kBuildThreads;
                if (e < raw_tile) dst[e] = pre[k];
            }
            return true;
        };
        if (bt == 0 && t_lo < t_hi) issue_copy(t_lo);
        const float s_a = p.ms_a[i0 < p.nq ? i0 : p.nq - 1].hi;
        for (int e = bt; e < raw_a; e += kBuildThreads) {
            const int64_t jj = i0 + e;
            raw[e] = (jj < p.na) ? p.a[jj] - s_a : 0.f;
        }
        named_sync(kBarBuild, kBuildThreads);
        build_hankel<VARIANT>(raw, p.ra_rows, ha[0], ha[1], bt, kBuildThreads);
        fence_async_smem();
        mbar_arrive(full_a);
        bool ok = t_lo >= t_hi || land_tile(t_lo);
        named_sync(kBarBuild, kBuildThreads);
        const int nthr = NS == 2 ? kRoleThreads : kBuildThreads;
        const int tt = NS == 2 ? gt : bt;
        const int bar_id = NS == 2 ? kBarGroup0 + bgrp : kBarBuild;
        int j = 0;
        for (int t = t_lo; ok && t < t_hi; ++t) {
            const TcTile tile = p.tiles[t];
            const float *rt = raw_b[(t - t_lo) & 1];
            // the other buffer's last tile (t - 1) is built: it takes tile t + 1
            if (bt == 0 && t + 1 < t_hi) issue_copy(t + 1);
            j = (t - t_lo) * ((p.nkb + p.qg - 1) / p.qg);  // stages before this tile
            bool gok = true;
            for (int q0 = 0; q0 < p.nkb; q0 += p.qg, ++j) {
                const int s = j % NS;
                if (NS == 2 && s != bgrp) continue;  // the other group's stage
                const int q1 = min(p.nkb, q0 + p.qg);
                if (j >= NS) {
                    const bool w = role_wait(&empty_b[s], ((j / NS) - 1) & 1, abort_flag, p.wait_cycles);
                    if (!(gok = named_sync_and(bar_id, nthr, w))) break;
                }
                const int rows = (q1 - q0 - 1) * EPR + tile.nmma;
                build_hankel<VARIANT>(rt + q0 * EPR, rows, hb + (s * NHL) * st_bytes,
                                      hb + (s * NHL + NHL - 1) * st_bytes, tt, nthr);
                fence_async_smem();
                mbar_arrive(&full_b[s]);
            }
            // every builder takes the same branch (j is recomputed per tile below)
            if (!(ok = named_sync_and(kBarBuild, kBuildThreads, gok))) break;
            if (t + 1 < t_hi && !(ok = land_tile(t + 1))) break;
            named_sync(kBarBuild, kBuildThreads);
        }
        // a copy still in flight (a wait gave up) must land before the shared
        // memory is released: its own bound, never shortened
        if (bt == 0 && issued0 > 0) mbar_wait(&copy_b[0], (uint32_t)((issued0 - 1) & 1), kTcWaitCycles);
        if (bt == 0 && issued1 > 0) mbar_wait(&copy_b[1], (uint32_t)((issued1 - 1) & 1), kTcWaitCycles);
    } else {
        // ---------------- epilogue: one query window per thread ----------------
        const int quad = warp & 3;                 // TMEM lanes this warp may read
        const int row_in = quad * 32 + lane;       // query window within the CTA
        const int et = tid - kEpiWarp0 * 32;
        const int64_t row = i0 + row_in;
        const float s_a = p.ms_a[i0 < p.nq ? i0 : p.nq - 1].hi;
        float da = 0.f;
        if (row < p.nq) {
            const Split<float> ma = p.ms_a[row];
            da = (ma.hi - s_a) + ma.lo;
        }
        float best = -INFINITY;
        int32_t bchunk = -1;
        // near-tie width of this row in units of the score q = rho * m * std_a
        // (negative: no records, for rows past the end and constant rows)
        float tq = -1.f;
        // the group's window range, for the overflow mask's runs
        const int64_t g_lo = t_lo < t_hi ? p.tiles[t_lo].g0 : 0;
        const int64_t g_hi = t_lo < t_hi ? p.tiles[t_hi - 1].g0 + p.tiles[t_hi - 1].nvalid : 0;
        if (row < p.nq && p.near.rec != nullptr) {
            *p.near.head(grp, row) = NearSlot{0, 0.f};
            const float za = p.rs_a[row].z;
            if (za > 0.f) {
                // twice the products' error bound: u m sqrt(std_a^2 + da^2) F_b
                const float sd = 1.f / za;
                tq = 2.f * p.near.u * (float)m * sqrtf(fmaf(sd, sd, da * da)) * *p.near.fb;
            }
        }
        bool ok = true;
        for (int t = t_lo; ok && t < t_hi; ++t) {
            const TcTile tile = p.tiles[t];
            const int ab = (t - t_lo) & 1;
            const int k_t = (t - t_lo) >> 1;
            // column terms: w = m (mean_b - s_b), z = 1/std, penalty 0 / -inf
            const float s_b = p.ms_b[tile.g0].hi;
            for (int n = et; n < kTcMaxN; n += kRoleThreads) {
                float4 v = make_float4(0.f, 0.f, -INFINITY, 0.f);
                if (n < tile.nvalid) {
                    const int64_t g = tile.g0 + n;
                    const float4 r = p.rs_b[g];
                    const Split<float> mb = p.ms_b[g];
                    v.x = (float)m * ((mb.hi - s_b) + mb.lo);
                    v.y = r.z;
                    v.z = r.w;
                }
                colp[n] = v;
            }
            named_sync(kBarEpi, kRoleThreads);
            ok = role_wait(&acc_full[ab], k_t & 1, abort_flag, p.wait_cycles);
            if (!(ok = named_sync_and(kBarEpi, kRoleThreads, ok))) break;
            tc_fence_after();
            const uint32_t t_lane = taddr + (uint32_t)(ab * kTcMaxN) + ((uint32_t)(quad * 32) << 16);
            const int ncols = (tile.nmma + 31) & ~31;
            for (int c32 = 0; c32 < ncols; c32 += 32) {
                uint32_t v[32];
                tmem_ld32(t_lane + (uint32_t)c32, v);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float cm = -INFINITY;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const float4 cp = colp[c32 + 16 * h + u];
                        const float cov = fmaf(-da, cp.x, __uint_as_float(v[16 * h + u]));
                        cm = fmaxf(cm, fmaf(cov, cp.y, cp.z));
                    }
                    const int32_t gch = (int32_t)(tile.g0 + c32 + 16 * h);
                    // near ties: a chunk within tq below the running best, or a best
                    // overtaken by less than tq (-inf on either side: no record)
                    if (fabsf(cm - best) <= tq) {
                        const bool upd = cm > best;
                        near_add<true>(p.near, grp, row, upd ? bchunk : gch, upd ? best : cm, fmaxf(cm, best) - tq,
                                       g_lo, g_hi);
                    }
                    if (cm > best) {
                        best = cm;
                        bchunk = gch;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[ab]);
            named_sync(kBarEpi, kRoleThreads);  // colp is rewritten for the next tile
        }
        if (ok && !*abort_flag && row < p.nq) {
            Partial<float> pv;
            pv.q = best;
            pv.g = bchunk;
            p.part[(int64_t)grp * p.nq + row] = pv;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && *abort_flag) atomicExch(p.err, 1);
    if (warp == kMmaWarp) tmem_dealloc(taddr, kTmemCols);
}

// ---------------------------------------------------------------------------
// K2s: the plain kernel's top seeds on the tensor cores
// ---------------------------------------------------------------------------
// The plain recurrence (kernel K2) starts the diagonals of each warp's first
// query window from a direct dot product per dictionary window. Those "top
// seeds" form a dense product: for the query windows r_s = s * stride (s = 0,
// 1, ...) and every valid dictionary window g,
//     S[s, g] = sum_k (a[r_s + k] - mean_a[r_s]) * (b[g + k] - mean_b[g]),
// the centred covariance of the two windows (the C of Sec. 3.2's per-segment
// AB-join). A CTA owns 128 seed rows (the TMEM lanes) and walks the tiles of
// one column group. Per tile and K-block (32 values of k) the 128 query
// windows' samples are gathered into a K-major operand and the tile's
// dictionary samples form a row-shifted Hankel operand as in K3 (the samples of
// the next stage are loaded into registers while the MMAs run). The products
// are TF32 with a hi/lo split of both operands (hi*hi + hi*lo + lo*hi): each
// value is split with a residual below 2^-22 of it, so a seed carries about
// FP32's error, not the 2^-16 of a BF16 split; the recurrence adds its own
// rounding to that seed for up to 32 * 20 rows. The epilogue removes the
// shifts and stores S in FP32, transposed through shared memory so that the
// stores are row-contiguous. A CTA (8 warps) builds and multiplies in turn;
// two CTAs share an SM, so one CTA's operand build overlaps the other's MMAs,
// and 16 warps per SM hide the latency of the builds' conversion chains.
struct SeedArgs {
    const float *a;
    int64_t nq;
    int32_t m;
    int32_t n_groups;
    int32_t stride;   // query windows from one seed row to the next
    int64_t n_srows;  // seed rows: ceil(nq / stride)
    const Split<float> *ms_a;
    const float *b;
    int64_t nb;
    const Split<float> *ms_b;
    const TcTile *tiles;
    const int32_t *group_start;
    float *seeds;  // [n_srows][ld]; column = global dictionary window g
    int64_t ld;
    int32_t *err;
};

constexpr int kSeedVariant = 2;  // TF32 hi/lo
constexpr int kSeedThreads = 256;
constexpr int kSeedRows = 128;
constexpr int kSeedRowStep = kSeedThreads / 8;          // query rows one pass of the threads fills
constexpr int kSeedRowsPer = kSeedRows / kSeedRowStep;  // query rows per thread
constexpr int kSeedEpr = 32;  // TF32 values of K per 128-byte operand row
constexpr int kSeedRawPer = (kTcMaxN + kSeedEpr + kSeedThreads - 1) / kSeedThreads;  // staged samples per thread
constexpr int kSeedColPer = (kTcMaxN + kSeedThreads - 1) / kSeedThreads;             // column terms per thread
constexpr int kHalves = kSeedThreads / kSeedRows;  // groups of 4 warps sharing the TMEM lanes in the epilogue
static_assert(kSeedThreads % kSeedRows == 0 && kSeedRows == 128, "the epilogue splits columns over groups of 4 warps");
static_assert(kSeedRows % kSeedRowStep == 0, "query rows per thread");
constexpr int kSeedKstep = 8;  // K per MMA
constexpr long long kSeedWaitCycles = 4000000000LL;  // about 2 s

size_t seed_smem_bytes()
{
    // 1024-byte alignment slack, query operand (hi, lo), dictionary operand
    // (hi, lo), staged samples, column terms, barrier and TMEM slot
    return 1024 + 2 * (size_t)kSeedRows * 128 + 2 * (size_t)kTcMaxN * 128 + (kTcMaxN + kSeedEpr + 8) * 4 +
           kTcMaxN * 4 + 16;
}

__global__ void __launch_bounds__(kSeedThreads, 2) k_seed(SeedArgs p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *a_hi = base, *a_lo = base + kSeedRows * 128;
    unsigned char *b_hi = base + 2 * kSeedRows * 128, *b_lo = b_hi + kTcMaxN * 128;
    float *raw = reinterpret_cast<float *>(b_lo + kTcMaxN * 128);  // a tile's samples for one K-block
    float *colp = raw + kTcMaxN + kSeedEpr + 8;                     // m * (mean_b - s_b) per column
    uint64_t *bar = reinterpret_cast<uint64_t *>(colp + kTcMaxN);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    float *ost = reinterpret_cast<float *>(base);  // epilogue staging (operands are idle then): kHalves x 128 x 33

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t rb = blockIdx.x / p.n_groups;
    const int grp = blockIdx.x % p.n_groups;
    const int m = p.m;
    const int nkb = (m + kSeedEpr - 1) / kSeedEpr;
    const int t_lo = p.group_start[grp], t_hi = p.group_start[grp + 1];

    if (warp == 0) tmem_alloc(tmem_slot, kTcMaxN);
    if (tid == 0) mbar_init(bar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;

    // Query operand: this thread fills 16-byte chunk c of rows rho_i = tid / 8 + kSeedRowStep i
    // (4 values of k each); the rows are centred on their own mean's hi part.
    const int c = tid & 7;
    int64_t r_i[kSeedRowsPer];
    float sa_i[kSeedRowsPer];
#pragma unroll
    for (int i = 0; i < kSeedRowsPer; ++i) {
        const int64_t sr = rb * kSeedRows + (tid >> 3) + kSeedRowStep * i;
        r_i[i] = sr < p.n_srows ? sr * p.stride : -1;
        sa_i[i] = r_i[i] >= 0 ? p.ms_a[r_i[i]].hi : 0.f;
    }
    const bool a16 = (reinterpret_cast<uintptr_t>(p.a) & 15) == 0;
    // Raw samples of one stage (tile t, K-block q) and, for a tile's first
    // stage, its column terms, loaded into registers one stage ahead. Nothing
    // consumes them until the next stage, so their latency overlaps the MMAs.
    // Positions past m or past the series hold the shift itself (x - shift = 0).
    float xa[kSeedRowsPer][4], xb[kSeedRawPer];
    Split<float> mbv[kSeedColPer];
    TcTile tl_next;
    float sb_next = 0.f;
    const int n_st = (t_hi - t_lo) * nkb;
    auto load_stage = [&](int j) {
        tl_next = p.tiles[t_lo + j / nkb];
        const int k0 = (j % nkb) * kSeedEpr;
#pragma unroll
        for (int i = 0; i < kSeedRowsPer; ++i) {
            const int k = k0 + 4 * c;
            if (r_i[i] >= 0 && a16 && k + 3 < m) {
                const float4 v = *reinterpret_cast<const float4 *>(p.a + r_i[i] + k);
                xa[i][0] = v.x;
                xa[i][1] = v.y;
                xa[i][2] = v.z;
                xa[i][3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) xa[i][e] = (r_i[i] >= 0 && k + e < m) ? p.a[r_i[i] + k + e] : sa_i[i];
            }
        }
        sb_next = p.ms_b[tl_next.g0].hi;
#pragma unroll
        for (int u = 0; u < kSeedRawPer; ++u) {
            const int e = tid + u * kSeedThreads;
            const int64_t jj = tl_next.g0 + k0 + e;
            xb[u] = (e < tl_next.nmma + kSeedEpr && jj < p.nb) ? p.b[jj] : sb_next;
        }
        if (j % nkb == 0) {
#pragma unroll
            for (int u = 0; u < kSeedColPer; ++u) {
                const int n = tid + u * kSeedThreads;
                mbv[u] = n < tl_next.nvalid ? p.ms_b[tl_next.g0 + n] : Split<float>{sb_next, 0.f};
            }
        }
    };
    if (n_st > 0) load_stage(0);

    // the accumulator row this thread reads back: TMEM lane tid % 128 (a warp reads
    // the lane quarter warp % 4); the two groups of 4 warps take alternate column groups
    const int lrow = tid & (kSeedRows - 1), half = tid / kSeedRows;
    const int64_t srow = rb * kSeedRows + lrow;
    const float da = srow < p.n_srows ? p.ms_a[srow * p.stride].lo : 0.f;  // mean - hi = lo

    uint32_t phase = 0;
    bool ok = true;
    int j = 0;
    for (int t = t_lo; ok && t < t_hi; ++t) {
        const TcTile tile = tl_next;  // loaded with the tile's first stage
        const float s_b = sb_next;
#pragma unroll
        for (int u = 0; u < kSeedColPer; ++u)
            if (tid + u * kSeedThreads < kTcMaxN)
                colp[tid + u * kSeedThreads] = (float)m * ((mbv[u].hi - s_b) + mbv[u].lo);
        const uint32_t idesc = instr_desc<kSeedVariant>(tile.nmma);
        for (int q = 0; q < nkb; ++q, ++j) {
            const int k0 = q * kSeedEpr;
            // write this stage's operands from the registers
#pragma unroll
            for (int i = 0; i < kSeedRowsPer; ++i) {
                const int rho = (tid >> 3) + kSeedRowStep * i;
                float x[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) x[e] = xa[i][e] - sa_i[i];
                put_chunk<kSeedVariant>(x, a_hi, a_lo, (uint32_t)rho * 128u + (uint32_t)((c ^ (rho & 7)) << 4));
            }
#pragma unroll
            for (int u = 0; u < kSeedRawPer; ++u) {
                const int e = tid + u * kSeedThreads;
                if (e < kTcMaxN + kSeedEpr) raw[e] = xb[u] - s_b;
            }
            __syncthreads();
            build_hankel<kSeedVariant>(raw, tile.nmma, b_hi, b_lo, tid, kSeedThreads);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = smem_u32(a_hi), a1 = smem_u32(a_lo);
                const uint32_t b0 = smem_u32(b_hi), b1 = smem_u32(b_lo);
                // the query operand is 0 past m
                const int ksteps = (min(kSeedEpr, m - k0) + kSeedKstep - 1) / kSeedKstep;
                for (int k = 0; k < ksteps; ++k) {
                    const uint32_t acc = (q == 0 && k == 0) ? 0u : 1u;
                    mma<kSeedVariant>(taddr, smem_desc(a0 + 32u * k), smem_desc(b0 + 32u * k), idesc, acc);
                    mma<kSeedVariant>(taddr, smem_desc(a0 + 32u * k), smem_desc(b1 + 32u * k), idesc, 1u);
                    mma<kSeedVariant>(taddr, smem_desc(a1 + 32u * k), smem_desc(b0 + 32u * k), idesc, 1u);
                }
                mma_commit(bar);
            }
            if (j + 1 < n_st) load_stage(j + 1);  // overlaps the MMAs
            // the next stage rewrites the operands: wait for these MMAs
            const bool w = mbar_wait(bar, phase, kSeedWaitCycles);
            phase ^= 1u;
            ok = __syncthreads_and(w ? 1 : 0) != 0;
            tc_fence_after();
            if (!ok) break;
        }
        if (!ok) break;
        // epilogue: accumulator row lrow, 32 columns per TMEM load, staged in
        // shared memory (one buffer per group of 4 warps) so that each warp
        // stores contiguous runs of a row; group `half` takes the column
        // groups c32 = 32 (kHalves j + half), and both groups pass the same
        // barriers
        const uint32_t t_lane = taddr + ((uint32_t)((warp & 3) * 32) << 16);
        const int ncols = (tile.nmma + 31) & ~31;
        float *const osth = ost + half * kSeedRows * 33;
        for (int cg = 0; cg < ncols; cg += 32 * kHalves) {
            const int c32 = cg + 32 * half;
            const bool act = c32 < ncols;  // the same for the whole group of warps
            if (act) {
                uint32_t v[32];
                tmem_ld32(t_lane + (uint32_t)c32, v);
#pragma unroll
                for (int u = 0; u < 32; ++u) osth[lrow * 33 + u] = fmaf(-da, colp[c32 + u], __uint_as_float(v[u]));
            }
            __syncthreads();
            if (act) {
                const int n = c32 + lane;
                for (int rr = warp & 3; rr < kSeedRows; rr += 4) {
                    const int64_t sr = rb * kSeedRows + rr;
                    if (sr < p.n_srows && n < tile.nvalid) p.seeds[sr * p.ld + tile.g0 + n] = osth[rr * 33 + lane];
                }
            }
            __syncthreads();  // ost is rewritten by the next group (or the next tile's operands)
        }
        // TMEM and colp are read before the next tile's MMAs and column terms
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        // a wait ran out: give the MMAs in flight time to finish before the
        // TMEM and shared memory are released, and report the error
        mbar_wait(bar, phase ^ 1u, kSeedWaitCycles);
        if (tid == 0) atomicExch(p.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, kTcMaxN);
}

// ---------------------------------------------------------------------------
// K2l: the plain kernel's left seeds on the tensor cores
// ---------------------------------------------------------------------------
// Each span (a run of dictionary windows inside one segment) starts the plain
// recurrence's diagonals from "left seeds": the centred covariance of every
// query window r with the span's first window g_s,
//     L[s, r] = sum_k (a[r + k] - mean_a[r]) * (b[g_s + k] - mean_b[g_s]).
// For 128 consecutive query windows (the TMEM lanes) and up to 128 spans this
// is a dense product with K = m. The spans' operand does not depend on the
// query: k_left_operand builds it once per (dictionary, m, column grouping),
// in the MMA's swizzled K-major layout (each first window centred on its own
// mean's hi part, zero past m, TF32 hi and lo), one 32 KB block per span tile
// and K-block (32 values of k). A CTA stages its windows' samples for every
// K-block once (shifted by its first window's mean, hi part). Per K-block it
// copies the span block's rows in use (hi and lo) into shared memory with bulk
// asynchronous copies (the next block's copies overlap the current MMAs) and
// builds the query's row-shifted Hankel operand from the staged samples. The products
// are TF32 hi/lo as in K2s, so a left seed carries about FP32's error. The
// epilogue removes the shifts and stores L[s][r]: for one span, consecutive
// threads hold consecutive query windows, so the stores are coalesced as they
// come.
constexpr int kLeftThreads = 256;
constexpr int kLeftRows = 128;
constexpr int kLeftSpans = 128;                     // spans per CTA (TMEM columns, MMA N <= 128)
constexpr uint32_t kLeftHalf = kLeftSpans * 128;    // bytes of one (hi or lo) span operand block
constexpr uint32_t kLeftBlock = 2 * kLeftHalf;      // hi then lo
// query samples a CTA stages: its 128 windows' samples for every K-block
__host__ __device__ constexpr int left_raw(int m) { return kLeftRows + (m + kSeedEpr - 1) / kSeedEpr * kSeedEpr; }

struct LeftArgs {
    const float *a;
    int64_t nq;
    int32_t m;
    const Split<float> *ms_a;
    const Split<float> *ms_b;
    const Span *spans;
    int32_t n_spans;
    const unsigned char *ops;  // [span tile][K-block] blocks of kLeftBlock bytes (k_left_operand)
    float *left;               // [n_spans][ld]
    int64_t ld;
    int32_t *err;
};

// The spans' operand blocks: grid (span tiles, K-blocks), 256 threads.
__global__ void __launch_bounds__(256) k_left_operand(const Span *spans, int32_t n_spans, int32_t m,
                                                      const float *b, int64_t nb, const Split<float> *ms_b,
                                                      unsigned char *ops)
{
    const int tile = blockIdx.x, q = blockIdx.y, nkb = gridDim.y;
    unsigned char *hi = ops + ((size_t)tile * nkb + q) * kLeftBlock, *lo = hi + kLeftHalf;
    const int k0 = q * kSeedEpr;
    for (int idx = threadIdx.x; idx < kLeftSpans * 8; idx += blockDim.x) {
        const int n = idx >> 3, c = idx & 7, s = tile * kLeftSpans + n;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (s < n_spans) {
            const int64_t g0 = spans[s].g0;
            const float sb = ms_b[g0].hi;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + 4 * c + e;
                x[e] = (k < m && g0 + k < nb) ? b[g0 + k] - sb : 0.f;
            }
        }
        put_chunk<kSeedVariant>(x, hi, lo, (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) << 4));
    }
}

size_t left_smem_bytes(int m)
{
    // 1024-byte alignment slack, query operand (hi, lo), two span operand
    // blocks, staged query samples, column terms, barriers and TMEM slot
    return 1024 + 2 * (size_t)kLeftRows * 128 + 2 * (size_t)kLeftBlock + (left_raw(m) + 8) * 4 + kLeftSpans * 4 +
           3 * 8 + 16;
}

__global__ void __launch_bounds__(kLeftThreads, 2) k_left_seed(LeftArgs p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *a_hi = base, *a_lo = base + kLeftRows * 128;
    unsigned char *bst[2] = {base + 2 * kLeftRows * 128, base + 2 * kLeftRows * 128 + kLeftBlock};
    const int n_raw = left_raw(p.m);
    float *raw = reinterpret_cast<float *>(bst[1] + kLeftBlock);
    float *colp = raw + n_raw + 8;  // m * (mean_b - s_b) = m * mean's lo part, per span
    uint64_t *bar = reinterpret_cast<uint64_t *>(colp + kLeftSpans);  // MMAs done
    uint64_t *cbar = bar + 1;                                         // [2] span blocks landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 3);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t R0 = (int64_t)blockIdx.x * kLeftRows;  // first query window
    const int tile = blockIdx.y, s0 = tile * kLeftSpans;  // first span
    const int ns = min(kLeftSpans, p.n_spans - s0);
    const int nmma = (ns + 15) & ~15;
    const int m = p.m;
    const int nkb = (m + kSeedEpr - 1) / kSeedEpr;
    const unsigned char *ops = p.ops + (size_t)tile * nkb * kLeftBlock;

    if (warp == 0) tmem_alloc(tmem_slot, kLeftSpans);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(&cbar[0], 1);
        mbar_init(&cbar[1], 1);
    }
    for (int n = tid; n < kLeftSpans; n += kLeftThreads)
        colp[n] = n < ns ? (float)m * p.ms_b[p.spans[s0 + n].g0].lo : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tmem_slot;
    // a span block's hi and lo rows [0, nmma): two bulk copies on one mbarrier
    const uint32_t cbytes = (uint32_t)nmma * 128u;
    auto copy_block = [&](int q, int buf) {
        const unsigned char *src = ops + (size_t)q * kLeftBlock;
        bulk_copy2_g2s(bst[buf], src, bst[buf] + kLeftHalf, src + kLeftHalf, cbytes, &cbar[buf]);
    };
    if (tid == 0) copy_block(0, 0);

    // the CTA's query samples for every K-block, shifted (zeros past the
    // series), while the first span block is in flight
    const float s_a = p.ms_a[R0 < p.nq ? R0 : p.nq - 1].hi;
    const int64_t na = p.nq + m - 1;
    for (int e = tid; e < n_raw; e += kLeftThreads) {
        const int64_t j = R0 + e;
        raw[e] = j < na ? p.a[j] - s_a : 0.f;
    }
    const uint32_t idesc = instr_desc<kSeedVariant>(nmma);
    uint32_t phase = 0;
    int copies = 1;  // bulk copies issued
    bool ok = true;
    __syncthreads();  // the staged samples
    for (int q = 0; q < nkb; ++q) {
        // the query's Hankel operand of this K-block (the previous MMAs are done)
        build_hankel<kSeedVariant>(raw + q * kSeedEpr, kLeftRows, a_hi, a_lo, tid, kLeftThreads);
        fence_async_smem();
        const bool w = mbar_wait(&cbar[q & 1], (uint32_t)((q >> 1) & 1), kSeedWaitCycles);
        if (!(ok = __syncthreads_and(w ? 1 : 0) != 0)) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(a_hi), a1 = smem_u32(a_lo);
            const uint32_t b0 = smem_u32(bst[q & 1]), b1 = b0 + kLeftHalf;
            // the span operand is 0 past m
            const int ksteps = (min(kSeedEpr, m - q * kSeedEpr) + kSeedKstep - 1) / kSeedKstep;
            for (int k = 0; k < ksteps; ++k) {
                const uint32_t acc = (q == 0 && k == 0) ? 0u : 1u;
                mma<kSeedVariant>(taddr, smem_desc(a0 + 32u * k), smem_desc(b0 + 32u * k), idesc, acc);
                mma<kSeedVariant>(taddr, smem_desc(a0 + 32u * k), smem_desc(b1 + 32u * k), idesc, 1u);
                mma<kSeedVariant>(taddr, smem_desc(a1 + 32u * k), smem_desc(b0 + 32u * k), idesc, 1u);
            }
            mma_commit(bar);
            // the other block's last MMAs (K-block q - 1) are done: it takes K-block q + 1
            if (q + 1 < nkb) {
                fence_async_smem();
                copy_block(q + 1, (q + 1) & 1);
                ++copies;
            }
        }
        // the next K-block rewrites the query operand: wait for these MMAs
        const bool wm = mbar_wait(bar, phase, kSeedWaitCycles);
        phase ^= 1u;
        ok = __syncthreads_and(wm ? 1 : 0) != 0;
        tc_fence_after();
        if (!ok) break;
    }
    if (ok) {
        // epilogue: thread tid % 128 reads its query window's accumulator row (a
        // warp reads the TMEM lane quarter warp % 4); the two groups of 4 warps
        // take alternate 32-span groups
        const int lrow = tid & (kLeftRows - 1), half = tid / kLeftRows;
        const int64_t r = R0 + lrow;
        float da = 0.f;
        if (r < p.nq) {
            const Split<float> ma = p.ms_a[r];
            da = (ma.hi - s_a) + ma.lo;
        }
        const uint32_t t_lane = taddr + ((uint32_t)((warp & 3) * 32) << 16);
        for (int c32 = 32 * half; c32 < nmma; c32 += 64) {
            uint32_t v[32];
            tmem_ld32(t_lane + (uint32_t)c32, v);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int n = c32 + u;
                if (n < ns && r < p.nq)
                    p.left[(int64_t)(s0 + n) * p.ld + r] = fmaf(-da, colp[n], __uint_as_float(v[u]));
            }
        }
    } else {
        // a wait ran out: the MMAs and the copies in flight must finish before
        // the TMEM and shared memory are released (their own bounds); report it
        if (tid == 0) {
            mbar_wait(bar, phase ^ 1u, kSeedWaitCycles);
            const int last = copies - 1;  // the last copy went to block last & 1, its use (last >> 1)
            mbar_wait(&cbar[last & 1], (uint32_t)((last >> 1) & 1), kSeedWaitCycles);
            atomicExch(p.err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, kLeftSpans);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcPlan {
    int variant;
    int m;
    int epr, kstep, nhl, nprod;
    int nkb, ra_rows, nmax, qg, rb_rows, n_stages;
    size_t smem;
};

size_t plan_smem(const TcPlan &P)
{
    const size_t raw = (size_t)(P.ra_rows + P.epr) + 2 * (size_t)(P.nmax + P.m + P.epr + 8);
    return 1024 + (size_t)P.nhl * 128 * ((size_t)P.ra_rows + (size_t)P.n_stages * P.rb_rows) +
           ((raw + 3) & ~(size_t)3) * 4 + kTcMaxN * sizeof(float4) + 13 * 8 + 16;
}

// Estimated SM clocks per tile: the MMAs (or the shared-memory traffic they
// and the builders cause, if larger) plus, with one stage, the builders'
// time that cannot overlap the MMAs. The traffic term takes 64 bytes per
// clock: measured kernels whose MMAs (M = 128, one SM) read 12 KB of operands
// each ran at 60-68 bytes per clock of operand reads plus operand writes, not
// at the 128 of ordinary shared-memory loads.
constexpr double kTcSmemBytesPerClk = 64.0;
double plan_clocks(const TcPlan &P, int m)
{
    const double ksteps = (double)m / P.kstep;
    const double mma = ksteps * P.nprod * 128.0 * P.nmax / 256.0;
    const double reads = ksteps * P.nprod * (128.0 + P.nmax) * 32.0;
    const int groups = (P.nkb + P.qg - 1) / P.qg;
    const double writes = (double)groups * P.rb_rows * 128.0 * P.nhl;
    const double build = (double)groups * P.rb_rows * 8.0 / kBuildThreads * (P.variant == 1 ? 10.0 : 16.0);
    const double smem = (reads + writes) / kTcSmemBytesPerClk;
    return std::max(mma, smem) + (P.n_stages == 1 ? build : 0.0);
}

bool make_plan(int variant, int m, TcPlan *out)
{
    TcPlan P;
    P.variant = variant;
    P.m = m;
    P.epr = variant == 1 ? 32 : 64;
    P.kstep = variant == 1 ? 8 : 16;
    P.nhl = variant == 0 ? 2 : 1;
    P.nprod = variant == 0 ? 3 : 1;
    if (m < P.kstep || m % P.kstep != 0) return false;
    P.nkb = (m + P.epr - 1) / P.epr;
    P.ra_rows = (P.nkb - 1) * P.epr + 128;
    // one CTA per SM: the two accumulators use all 512 TMEM columns
    bool found = false;
    double best = 1e300;
    TcPlan bestP{};
    for (int nmax : {256, 128}) {
        for (int ns : {2, 1}) {
            for (int qg = 1; qg <= P.nkb; ++qg) {
                TcPlan C = P;
                C.nmax = nmax;
                C.n_stages = ns;
                C.qg = qg;
                C.rb_rows = (qg - 1) * P.epr + nmax;
                // at least 120 KB, so that two CTAs never share an SM
                C.smem = std::max<size_t>(plan_smem(C), 120 * 1024);
                if (C.smem > kTcSmemLimit) break;
                if (nmax + m + P.epr > 6 * kBuildThreads) continue;  // the builders' tile prefetch
                const double per_col = plan_clocks(C, m) / nmax;
                if (per_col < best) {
                    best = per_col;
                    bestP = C;
                    found = true;
                }
            }
        }
    }
    if (found) *out = bestP;
    return found;
}

struct TcPack {
    int nmax = 0, n_groups = 0;
    TcTile *tiles = nullptr;
    int32_t *group_start = nullptr;
    int32_t n_tiles = 0;
    float *fb = nullptr;  // the dictionary's column factor F_b for these tiles' shifts
};

// F_b = max over the tiles' valid windows g of sqrt(1 + ((mean_b[g] - s_b) /
// std_b[g])^2), s_b the tile's shift (its first window's mean, hi part), as
// the tensor-core join's epilogue forms them; *fb must start at 1. One CTA
// per tile.
__global__ void __launch_bounds__(256) k_tile_colfactor(const TcTile *tiles, int32_t n_tiles,
                                                        const Split<float> *ms_b, const float4 *rs_b, float *fb)
{
    if ((int)blockIdx.x >= n_tiles) return;
    const TcTile tile = tiles[blockIdx.x];
    const float s_b = ms_b[tile.g0].hi;
    float f = 1.f;
    for (int n = threadIdx.x; n < tile.nvalid; n += blockDim.x) {
        const int64_t g = tile.g0 + n;
        const Split<float> mb = ms_b[g];
        const float dz = ((mb.hi - s_b) + mb.lo) * rs_b[g].z;
        f = fmaxf(f, sqrtf(fmaf(dz, dz, 1.f)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f = fmaxf(f, __shfl_xor_sync(0xffffffffu, f, o));
    // f >= 1: the order of positive floats is that of their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(fb), __float_as_int(f));
}

struct TcPacks {
    std::vector<TcPack> packs;
};

// Tiles of up to nmax consecutive windows that never cross a segment.
std::vector<TcTile> make_tiles(const Span *seg_spans, int32_t n_seg, int nmax)
{
    std::vector<TcTile> tiles;
    for (int32_t s = 0; s < n_seg; ++s)
        for (int32_t c = 0; c < seg_spans[s].ncols; c += nmax) {
            TcTile t;
            t.g0 = seg_spans[s].g0 + c;
            t.nvalid = std::min(nmax, seg_spans[s].ncols - c);
            t.nmma = (t.nvalid + 15) & ~15;
            tiles.push_back(t);
        }
    return tiles;
}

// The device tile table of this tile width split into ng column groups
// (cached per dictionary and m); nullptr if device memory runs out or a CUDA
// call fails. Synchronises `st` once, when it is built.
TcPack *get_pack(TcPacks *pk, const std::vector<TcTile> &tiles, int nmax, int ng, cudaStream_t st)
{
    for (auto &p : pk->packs)
        if (p.nmax == nmax && p.n_groups == ng) return &p;
    const int n_tiles = (int)tiles.size();
    TcPack np;
    np.nmax = nmax;
    np.n_groups = ng;
    np.n_tiles = n_tiles;
    std::vector<int32_t> gs(ng + 1);
    for (int k = 0; k <= ng; ++k) gs[k] = (int32_t)((int64_t)n_tiles * k / ng);
    if (cudaMalloc(&np.tiles, std::max<size_t>(1, tiles.size()) * sizeof(TcTile)) != cudaSuccess ||
        cudaMalloc(&np.group_start, gs.size() * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(np.tiles);
        return nullptr;
    }
    const bool ok = (n_tiles == 0 || cudaMemcpyAsync(np.tiles, tiles.data(), tiles.size() * sizeof(TcTile),
                                                     cudaMemcpyHostToDevice, st) == cudaSuccess) &&
                    cudaMemcpyAsync(np.group_start, gs.data(), gs.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;  // the sources are host vectors
    if (!ok) {
        cudaGetLastError();
        cudaFree(np.tiles);
        cudaFree(np.group_start);
        return nullptr;
    }
    pk->packs.push_back(np);
    return &pk->packs.back();
}

// The column factor F_b of a pack's tiles, computed at its first use by the
// join (synchronising `st` once); false if a CUDA call fails.
bool pack_colfactor(TcPack *pk, const void *ms_b, const void *rs_b, cudaStream_t st)
{
    if (pk->fb) return true;
    float *fb = nullptr;
    if (cudaMalloc(&fb, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const float one = 1.f;
    bool ok = cudaMemcpyAsync(fb, &one, sizeof one, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok && pk->n_tiles > 0) {
        k_tile_colfactor<<<pk->n_tiles, 256, 0, st>>>(pk->tiles, pk->n_tiles, (const Split<float> *)ms_b,
                                                      (const float4 *)rs_b, fb);
        ok = cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;  // ready for every later join, on any stream
    if (!ok) {
        cudaGetLastError();
        cudaFree(fb);
        return false;
    }
    pk->fb = fb;
    return true;
}

}  // namespace

bool tc_supported(int variant, int m)
{
    TcPlan P;
    return make_plan(variant, m, &P);
}

int tc_groups_bound(int sm_count, int64_t nq)
{
    const int64_t rbk = (nq + 127) / 128;
    return (int)std::max<int64_t>(1, (2 * sm_count + rbk - 1) / rbk);
}

void tc_free_pack(void *pack)
{
    TcPacks *pk = (TcPacks *)pack;
    if (!pk) return;
    for (auto &p : pk->packs) {
        cudaFree(p.tiles);
        cudaFree(p.group_start);
        cudaFree(p.fb);
    }
    delete pk;
}

int tc_join(int sm_count, int variant, void **pack, const float *b, int64_t nb, const Span *seg_spans, int32_t n_seg,
            const void *ms_b, const void *rs_b, const float *a, int64_t n, int32_t m, const void *ms_a,
            const void *rs_a, Partial<float> *part, NearRec *near, int32_t *err, int *n_groups_out,
            const Span **cspans_out, const int32_t **cgroup_start_out, long long wait_cycles, cudaStream_t st,
            fail_fn fail)
{
    static_assert(sizeof(TcTile) == sizeof(Span) && offsetof(TcTile, g0) == offsetof(Span, g0) &&
                      offsetof(TcTile, nvalid) == offsetof(Span, ncols),
                  "a tile reads as the span of its valid windows");
    TcPlan P;
    if (!make_plan(variant, m, &P)) return fail(MP_E_ARG, "tensor-core join does not support m=%d", m);
    const int64_t nq = n - m + 1;
    const int64_t n_row_blocks = (nq + 127) / 128;
    if (!*pack) *pack = new TcPacks();
    TcPacks *pk = (TcPacks *)*pack;
    const std::vector<TcTile> tiles = make_tiles(seg_spans, n_seg, P.nmax);
    const int n_tiles = (int)tiles.size();
    int ng = (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (2 * sm_count + n_row_blocks - 1) / n_row_blocks));
    TcPack *use = get_pack(pk, tiles, P.nmax, ng, st);
    if (!use) return fail(MP_E_NOMEM, "tensor-core tile table");
    if (near->rec != nullptr) {
        if (!pack_colfactor(use, ms_b, rs_b, st)) return fail(MP_E_CUDA, "tensor-core column factor");
        // the products' error bound: one product's rounding plus the FP32 sum's
        near->fb = use->fb;
        near->u = variant == 1   ? kTcUnitTF32 + (float)m * 0x1p-23f
                  : variant == 2 ? kTcUnitBF16 + (float)m * 0x1p-23f
                                 : kTcUnitBF16X3 + 3.f * (float)m * 0x1p-23f;
    }
    TcArgs A;
    A.a = a;
    A.na = n;
    A.nq = nq;
    A.m = m;
    A.n_groups = ng;
    A.ms_a = (const Split<float> *)ms_a;
    A.b = b;
    A.nb = nb;
    A.ms_b = (const Split<float> *)ms_b;
    A.rs_b = (const float4 *)rs_b;
    A.tiles = use->tiles;
    A.group_start = use->group_start;
    A.part = part;
    A.rs_a = (const float4 *)rs_a;
    A.near = *near;
    if (near->rec != nullptr && (near->ld != nq || near->S < 1 || near->S > kNearMaxSlots))
        return fail(MP_E_INTERNAL, "tensor-core join: near-tie record layout");
    A.err = err;
    A.ra_rows = P.ra_rows;
    A.nmax = P.nmax;
    A.nkb = P.nkb;
    A.qg = P.qg;
    A.rb_rows = P.rb_rows;
    A.n_stages = P.n_stages;
    A.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    cudaError_t e;
    auto launch = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
        if (e == cudaSuccess) {
            kern<<<(unsigned)(n_row_blocks * ng), kTcThreadsP, P.smem, st>>>(A);
            e = cudaGetLastError();
        }
    };
    if (variant == 0)
        launch(k_tc<0>);
    else if (variant == 1)
        launch(k_tc<1>);
    else
        launch(k_tc<3>);
    if (e != cudaSuccess) return fail(MP_E_CUDA, "tensor-core kernel launch: %s", cudaGetErrorString(e));
    *n_groups_out = ng;
    // the column groups' chunks, for the finalisation of overflowed records
    *cspans_out = reinterpret_cast<const Span *>(use->tiles);
    *cgroup_start_out = use->group_start;
    return MP_OK;
}

int tc_seeds(void **pack, const float *b, int64_t nb, const Span *seg_spans, int32_t n_seg,
             const void *ms_b, const float *a, int64_t n, int32_t m, const void *ms_a, int32_t stride, float *seeds,
             int64_t ld, int32_t *err, cudaStream_t st, fail_fn fail)
{
    if (m < 1 || stride < 1) return fail(MP_E_ARG, "tensor-core seeds: bad m or stride");
    const int64_t nq = n - m + 1;
    const int64_t n_srows = (nq + stride - 1) / stride;
    const int64_t n_rb = (n_srows + kSeedRows - 1) / kSeedRows;
    if (!*pack) *pack = new TcPacks();
    TcPacks *pk = (TcPacks *)*pack;
    const std::vector<TcTile> tiles = make_tiles(seg_spans, n_seg, kTcMaxN);
    const int n_tiles = (int)tiles.size();
    if (n_tiles == 0 || n_srows <= 0) return MP_OK;
    // one tile per CTA: short CTAs of equal work, which the hardware scheduler
    // packs without a tail (groups of 2-3 tiles, about four waves, took 5 %
    // longer on the 2^20-window ECG join)
    const int ng = std::max(1, n_tiles);
    TcPack *use = get_pack(pk, tiles, kTcMaxN, ng, st);
    if (!use) return fail(MP_E_NOMEM, "tensor-core tile table");
    SeedArgs A;
    A.a = a;
    A.nq = nq;
    A.m = m;
    A.n_groups = ng;
    A.stride = stride;
    A.n_srows = n_srows;
    A.ms_a = (const Split<float> *)ms_a;
    A.b = b;
    A.nb = nb;
    A.ms_b = (const Split<float> *)ms_b;
    A.tiles = use->tiles;
    A.group_start = use->group_start;
    A.seeds = seeds;
    A.ld = ld;
    A.err = err;
    const size_t smem = seed_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_seed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_seed<<<(unsigned)(n_rb * ng), kSeedThreads, smem, st>>>(A);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(MP_E_CUDA, "tensor-core seed kernel launch: %s", cudaGetErrorString(e));
    return MP_OK;
}

size_t tc_left_operand_bytes(int32_t n_spans, int32_t m)
{
    const int64_t tiles = (n_spans + kLeftSpans - 1) / kLeftSpans, nkb = (m + kSeedEpr - 1) / kSeedEpr;
    return (size_t)(tiles * nkb) * kLeftBlock;
}

int tc_left_operand(const float *b, int64_t nb, const void *ms_b, const Span *spans, int32_t n_spans, int32_t m,
                    unsigned char *ops, cudaStream_t st, fail_fn fail)
{
    if (n_spans <= 0 || m < 1) return MP_OK;
    const dim3 grid((unsigned)((n_spans + kLeftSpans - 1) / kLeftSpans), (unsigned)((m + kSeedEpr - 1) / kSeedEpr));
    k_left_operand<<<grid, 256, 0, st>>>(spans, n_spans, m, b, nb, (const Split<float> *)ms_b, ops);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MP_E_CUDA, "left-seed operand kernel launch: %s", cudaGetErrorString(e));
    return MP_OK;
}

int tc_left_seeds(const float *a, int64_t n, int32_t m, const void *ms_a, const void *ms_b, const Span *spans,
                  int32_t n_spans, const unsigned char *ops, float *left, int64_t ld, int32_t *err, cudaStream_t st,
                  fail_fn fail)
{
    const int64_t nq = n - m + 1;
    if (m < 1 || nq <= 0 || n_spans <= 0) return MP_OK;
    if (ld < nq) return fail(MP_E_INTERNAL, "left seeds: row stride %lld below %lld rows", (long long)ld, (long long)nq);
    LeftArgs A;
    A.a = a;
    A.nq = nq;
    A.m = m;
    A.ms_a = (const Split<float> *)ms_a;
    A.ms_b = (const Split<float> *)ms_b;
    A.spans = spans;
    A.n_spans = n_spans;
    A.ops = ops;
    A.left = left;
    A.ld = ld;
    A.err = err;
    const size_t smem = left_smem_bytes(m);
    if (smem > kTcSmemLimit) return fail(MP_E_ARG, "left seeds: m=%d needs %zu bytes of shared memory", m, smem);
    cudaError_t e = cudaFuncSetAttribute(k_left_seed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)((nq + kLeftRows - 1) / kLeftRows), (unsigned)((n_spans + kLeftSpans - 1) / kLeftSpans));
        k_left_seed<<<grid, kLeftThreads, smem, st>>>(A);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(MP_E_CUDA, "tensor-core left-seed kernel launch: %s", cudaGetErrorString(e));
    return MP_OK;
}

}  // namespace mpd

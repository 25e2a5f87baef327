// Host runtime of libmpdict: the C ABI of include/mpdict.h.
//
//   * mp_ctx   -- one device, one stream for synchronous calls, a growable
//                 workspace, the resident dictionaries and the serving
//                 scheduler.
//   * mp_dict  -- dictionary samples resident in HBM plus, per window length
//                 m, the cached window statistics (kernel K1), the spans of
//                 valid windows (windows never cross a segment, Def. 8) and
//                 the two special windows used by the constant-window rule.
//   * join     -- K1 on the query, then the join form (plain K2, with its top
//                 seeds from the tensor-core kernel K2s for FP32 data, in row
//                 chunks when the seed matrix would pass its cap; or the
//                 tensor-core join K3), then K4 (reduction over column groups,
//                 re-scoring of the winning and near-tied chunks, exact
//                 distance of the picked pair), all enqueued on one stream.
//   * serving  -- mp_submit queues a request; a scheduler thread admits
//                 requests while slots and the memory budget allow, stages
//                 them, and runs every admitted request's join work in one
//                 persistent batched launch; completion is detected with
//                 events, so batches overlap on the device.
//   * more     -- the correlation form and the streaming join (on the same
//                 join path), e_max and discords, the autotuner, the join
//                 without device allocation, and dictionary learning
//                 (Algorithm 1: the self-join form of K2/K4 plus the kernels
//                 of mp_learn.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/mpdict.h"
#include "mp_internal.cuh"
#include "mp_tc.cuh"

using namespace mpd;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) return fail(MP_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                                           __FILE__, __LINE__);                                     \
    } while (0)

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Window lengths every call accepts (MP_E_ARG outside).
constexpr int kMinM = 4, kMaxM = 8192;

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
struct DictStats {
    int32_t m = 0;
    double *mean = nullptr;     // per window position of the concatenated buffer
    double *invstd = nullptr;
    uint8_t *cflag = nullptr;
    void *rs = nullptr;         // float4 / dvec4 recurrence terms
    void *ms = nullptr;         // Split<float> / Split<double> window means
    std::vector<Span> seg_spans;  // one span per segment with at least one window
    Span *d_seg_spans = nullptr;  // the same on the device
    int64_t n_windows = 0;        // W
    int64_t g_const = -1, g_first = -1;
    // column grouping cache: n_groups -> (device spans, device group_start)
    struct Grouping {
        Span *spans = nullptr;
        int32_t *group_start = nullptr;
        int32_t n_spans = 0;
        unsigned char *left_ops = nullptr;  // the spans' operand of the left-seed kernel (built at first use)
    };
    std::map<int, Grouping> groupings;
    void *tc_pack = nullptr;   // tensor-core operand cache (owned by the tc module)
};

struct mp_dict {
    mp_ctx *ctx = nullptr;
    int32_t dtype = MP_F32;
    int64_t nb = 0;
    std::vector<int64_t> offs;
    void *d_samples = nullptr;
    std::map<int, std::unique_ptr<DictStats>> stats;
    std::atomic<int> refs{0};
};

struct Request {
    uint64_t ticket = 0;
    mp_dict *dict = nullptr;
    int32_t dtype = MP_F32;
    int64_t n = 0;
    int32_t m = 0;
    // pinned staging: the query at submit, then the result (dist, idx) until
    // the host copies it to out_dist / out_idx at completion
    void *h_stage = nullptr;
    size_t stage_bytes = 0;
    bool no_windows = false;  // dictionary without a window of length m
    double *out_dist = nullptr;
    int64_t *out_idx = nullptr;
    double t_submit = 0, t_done = 0;
    int32_t state = MP_PENDING;
    // device side
    size_t bytes = 0;
    void *dmem = nullptr;
};

struct Batch {
    std::vector<std::shared_ptr<Request>> reqs;
    cudaEvent_t done = nullptr;
    cudaStream_t stream = nullptr;
    void *dmem = nullptr;  // batch-level buffers (request table, items, counter)
};

// Autotuner decisions: join form and column groups per (dtype, m, log2 of the
// dictionary windows, log2 of the query windows).
struct TuneKey {
    int dtype, m, wlog, qlog;
    bool operator<(const TuneKey &o) const
    {
        if (dtype != o.dtype) return dtype < o.dtype;
        if (m != o.m) return m < o.m;
        if (wlog != o.wlog) return wlog < o.wlog;
        return qlog < o.qlog;
    }
};
struct TuneVal {
    int kernel, groups;
    double ms;
    double tolerance = 0;  // the tolerance it was tuned for (recorded with the choice)
};
static int ilog2(int64_t x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        ++l;
    }
    return l;
}

struct mp_ctx {
    int32_t device = 0;
    int32_t sm_count = 0;
    int32_t kernel = MP_KERNEL_AUTO;
    mp_config cfg{};
    cudaStream_t stream = nullptr;
    std::mutex mu;  // serialises synchronous calls and dictionary changes
    void *ws = nullptr;
    size_t ws_size = 0;
    std::set<mp_dict *> dicts;

    // serving
    std::mutex smu;
    std::condition_variable scv;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    std::vector<Batch> inflight;
    size_t mem_budget = 0, mem_used = 0;
    int32_t n_inflight_reqs = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // serving streams: 0 and 1 (the device's greatest priority) take the
    // batches of small requests, 2 and 3 (its least) the large requests that
    // run alone, so that a small request's kernels are dispatched as soon as
    // SMs free up instead of after every CTA of a large join in flight
    static constexpr int kServeStreams = 4;
    cudaStream_t sstreams[kServeStreams] = {nullptr, nullptr, nullptr, nullptr};
    // the serving path's stream-ordered allocations; it keeps freed memory
    // for reuse (bounded by the admission budget) instead of returning it to
    // the driver at every synchronisation
    cudaMemPool_t pool = nullptr;
    // requests' memory is returned to the pool on this stream, which has no
    // other work: the host frees only memory whose work it has seen complete,
    // so each free completes at once and the pool can reuse the memory for the
    // next admission on any stream, without making that stream wait
    cudaStream_t fstream = nullptr;
    int next_small = 0, next_large = 0;

    // tracing
    bool profiling = false;
    struct Mark {
        int phase;
        cudaEvent_t t0, t1;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[MP_PHASE_COUNT] = {};
    int64_t prof_n[MP_PHASE_COUNT] = {};

    // pinned staging buffers, free lists by power-of-two size class
    std::map<size_t, std::vector<void *>> pinned_free;  // staging buffers by size class
    std::vector<void *> pinned_slabs;                   // the pinned allocations they are cut from

    // autotuner
    std::map<TuneKey, TuneVal> tune;
    std::string tune_path;
    int force_groups = 0;  // set while the autotuner times a candidate

    // finalisation counters (kFinCounters, summed on the device by every join)
    unsigned long long *d_counters = nullptr;

    // testing hooks (mp_test_hook)
    int64_t hook_fail_alloc = 0;  // serving allocations still to fail (under smu)
    long long hook_tc_wait = 0;   // tensor-core role-wait bound in clocks (0: the default)

    // CUDA graphs of repeated small synchronous joins (under mu; see ab_join_host)
    struct GraphKey {
        const mp_dict *d;
        int32_t dtype, m, kernel, corr;
        int64_t n;
        bool operator<(const GraphKey &o) const
        {
            return std::tie(d, dtype, m, kernel, corr, n) < std::tie(o.d, o.dtype, o.m, o.kernel, o.corr, o.n);
        }
    };
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        unsigned char *h_io = nullptr;  // pinned: the query, then dist, idx and the error word
        size_t out_off = 0;
        void *ws = nullptr;  // the workspace the graph was captured with
        int calls = 0;
        bool failed = false;  // capture did not work for this shape: never again
    };
    std::map<GraphKey, GraphEntry> graphs;
};

static void tune_load(mp_ctx *ctx, const char *path);

// Event pair around one phase of a join (no-op unless tracing is on).
struct PhaseTimer {
    mp_ctx *ctx;
    int phase;
    cudaStream_t st;
    cudaEvent_t t0 = nullptr;
    static cudaEvent_t take(mp_ctx *c)
    {
        if (!c->ev_pool.empty()) {
            cudaEvent_t e = c->ev_pool.back();
            c->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    PhaseTimer(mp_ctx *c, int ph, cudaStream_t s) : ctx(c), phase(ph), st(s)
    {
        if (ctx->profiling) {
            t0 = take(ctx);
            cudaEventRecord(t0, st);
        }
    }
    ~PhaseTimer()
    {
        if (t0) {
            cudaEvent_t t1 = take(ctx);
            cudaEventRecord(t1, st);
            ctx->marks.push_back(mp_ctx::Mark{phase, t0, t1});
        }
    }
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int dtype_size(int32_t dtype) { return dtype == MP_F64 ? 8 : 4; }

// No NaN or Inf among n samples: a value is non-finite exactly when its
// exponent bits are all ones. Branch-free within blocks of 4096 values so
// that the compiler vectorises the test; one exit test per block.
template <typename U>
static bool all_exponents_finite(const unsigned char *x, int64_t n, U exp_mask)
{
    constexpr int64_t kBlock = 4096;
    for (int64_t i0 = 0; i0 < n; i0 += kBlock) {
        const int64_t i1 = std::min(n, i0 + kBlock);
        U bad = 0;
        for (int64_t i = i0; i < i1; ++i) {
            U u;
            memcpy(&u, x + i * sizeof(U), sizeof(U));
            bad |= (U)((u & exp_mask) == exp_mask);
        }
        if (bad) return false;
    }
    return true;
}

static bool host_all_finite(const void *x, int32_t dtype, int64_t n)
{
    const unsigned char *p = (const unsigned char *)x;
    if (dtype == MP_F64) return all_exponents_finite<uint64_t>(p, n, 0x7ff0000000000000ull);
    return all_exponents_finite<uint32_t>(p, n, 0x7f800000u);
}

static int check_join_args(mp_ctx *ctx, const mp_dict *dict, const void *q, int32_t dtype, int64_t n, int32_t m)
{
    if (!ctx || !dict || !q) return fail(MP_E_ARG, "null argument");
    if (dtype != MP_F32 && dtype != MP_F64) return fail(MP_E_ARG, "unknown dtype %d", dtype);
    if (dtype != dict->dtype) return fail(MP_E_ARG, "query dtype differs from the dictionary's");
    if (m < kMinM || m > kMaxM) return fail(MP_E_ARG, "m=%d outside [%d, %d]", m, kMinM, kMaxM);
    if (n < m) return fail(MP_E_ARG, "query length %lld shorter than m=%d", (long long)n, m);
    if (n >= ((int64_t)1 << 40)) return fail(MP_E_ARG, "query too long");
    if (dict->ctx != ctx) return fail(MP_E_ARG, "dictionary belongs to another context");
    return MP_OK;
}

static void graph_entry_free(mp_ctx::GraphEntry &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.h_io) cudaFreeHost(e.h_io);
    e.exec = nullptr;
    e.h_io = nullptr;
}

// Drop the cached graphs (of one dictionary, or all when d is null): they hold
// its device pointers, the workspace's, and the launch geometry of the kernel
// setting and tuning they were captured under. Caller holds ctx->mu.
static void graphs_clear(mp_ctx *ctx, const mp_dict *d = nullptr)
{
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
        if (d == nullptr || it->first.d == d) {
            graph_entry_free(it->second);
            it = ctx->graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// Grow the context workspace to at least `bytes` (synchronises the stream).
static int ensure_ws(mp_ctx *ctx, size_t bytes)
{
    if (ctx->ws_size >= bytes) return MP_OK;
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    graphs_clear(ctx);  // they point into the old workspace
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    size_t sz = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&ctx->ws, sz) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_E_NOMEM, "workspace of %zu bytes", sz);
    }
    ctx->ws_size = sz;
    return MP_OK;
}

// Statistics of the dictionary for window length m (computed on first use).
static int get_stats(mp_ctx *ctx, mp_dict *d, int32_t m, DictStats **out)
{
    auto it = d->stats.find(m);
    if (it != d->stats.end()) {
        *out = it->second.get();
        return MP_OK;
    }
    std::unique_ptr<DictStats> s(new DictStats());
    s->m = m;
    for (size_t k = 0; k + 1 < d->offs.size(); ++k) {
        const int64_t L = d->offs[k + 1] - d->offs[k];
        if (L >= m) {
            Span sp;
            sp.g0 = d->offs[k];
            sp.ncols = (int32_t)(L - m + 1);
            sp.pad = 0;
            s->seg_spans.push_back(sp);
            s->n_windows += sp.ncols;
        }
    }
    const int64_t npos = d->nb - m + 1;
    if (npos > 0) {
        const bool f64 = d->dtype == MP_F64;
        const size_t rs_sz = (size_t)npos * (f64 ? sizeof(dvec4) : sizeof(float4));
        const size_t ms_sz = (size_t)npos * (f64 ? sizeof(Split<double>) : sizeof(Split<float>));
        if (cudaMalloc(&s->mean, npos * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s->invstd, npos * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s->cflag, npos) != cudaSuccess || cudaMalloc(&s->rs, rs_sz) != cudaSuccess ||
            cudaMalloc(&s->ms, ms_sz) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(s->mean);
            cudaFree(s->invstd);
            cudaFree(s->cflag);
            cudaFree(s->rs);
            cudaFree(s->ms);
            return fail(MP_E_NOMEM, "dictionary statistics for m=%d", m);
        }
        cudaError_t e;
        if (f64)
            e = launch_window_stats<double>((const double *)d->d_samples, d->nb, m, s->mean, s->invstd, s->cflag,
                                            (dvec4 *)s->rs, (Split<double> *)s->ms, ctx->stream);
        else
            e = launch_window_stats<float>((const float *)d->d_samples, d->nb, m, s->mean, s->invstd, s->cflag,
                                           (float4 *)s->rs, (Split<float> *)s->ms, ctx->stream);
        CUDA_TRY(e);
        {
            int64_t *doffs = nullptr;
            const size_t ob = d->offs.size() * sizeof(int64_t);
            CUDA_TRY(cudaMalloc(&doffs, ob));
            CUDA_TRY(cudaMemcpyAsync(doffs, d->offs.data(), ob, cudaMemcpyHostToDevice, ctx->stream));
            if (d->dtype == MP_F64)
                e = launch_mark_invalid<double>((dvec4 *)s->rs, npos, doffs, (int32_t)d->offs.size() - 1, m,
                                                ctx->stream);
            else
                e = launch_mark_invalid<float>((float4 *)s->rs, npos, doffs, (int32_t)d->offs.size() - 1, m,
                                               ctx->stream);
            CUDA_TRY(e);
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            cudaFree(doffs);
        }
        if (!s->seg_spans.empty()) {
            Span *dsp = nullptr;
            int64_t *dsv = nullptr;
            CUDA_TRY(cudaMalloc(&dsp, s->seg_spans.size() * sizeof(Span)));
            s->d_seg_spans = dsp;  // kept: the join without allocation cuts its column groups from it
            CUDA_TRY(cudaMalloc(&dsv, 2 * sizeof(int64_t)));
            CUDA_TRY(cudaMemcpyAsync(dsp, s->seg_spans.data(), s->seg_spans.size() * sizeof(Span),
                                     cudaMemcpyHostToDevice, ctx->stream));
            CUDA_TRY(cudaMemsetAsync(dsv, 0xFF, 2 * sizeof(int64_t), ctx->stream));
            CUDA_TRY(launch_dict_specials(dsp, (int32_t)s->seg_spans.size(), s->cflag, dsv, ctx->stream));
            int64_t hv[2];
            CUDA_TRY(cudaMemcpyAsync(hv, dsv, sizeof hv, cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            cudaFree(dsv);
            s->g_const = hv[0];
            s->g_first = hv[1];
        }
    }
    *out = s.get();
    d->stats[m] = std::move(s);
    return MP_OK;
}

// Cut the dictionary's valid windows into n_groups column groups of nearly
// equal size; a span never crosses a segment. Cached per n_groups.
// Column groups cut the dictionary's windows at chunk starts. A segment's
// windows form chunks of kChunk windows from its first window on (the plain
// and tensor-core kernels keep one approximate score per chunk, and the
// finalisation re-scores a chunk with its first window's mean as the shift),
// and a chunk belongs to group floor(p / T), p the position of its first
// window among all the dictionary's windows and T = ceil(windows / groups).
// So a window lies in the same chunk, scored with the same shift, whatever
// the number of groups, and the join's results do not depend on it. With
// T >= kChunk every group meets at least one chunk.
static int64_t group_target(int64_t n_windows, int n_groups)
{
    return (std::max<int64_t>(1, n_windows) + n_groups - 1) / n_groups;
}
// groups that a segment's chunks meet (cum: windows before the segment)
__host__ __device__ static inline int64_t segment_pieces(int64_t cum, int64_t ncols, int64_t T)
{
    if (ncols <= 0) return 0;
    const int64_t last = cum + (ncols - 1) / kChunk * kChunk;  // position of the last chunk's first window
    return last / T - cum / T + 1;
}
// the first chunk index (within the segment) whose start lies at or past
// position p, for chunk starts cum, cum + kChunk, ...
__host__ __device__ static inline int64_t chunk_at_or_after(int64_t cum, int64_t p)
{
    return p <= cum ? 0 : (p - cum + kChunk - 1) / kChunk;
}

static int get_grouping(mp_ctx *ctx, DictStats *s, int n_groups, DictStats::Grouping **out)
{
    auto it = s->groupings.find(n_groups);
    if (it != s->groupings.end()) {
        *out = &it->second;
        return MP_OK;
    }
    std::vector<Span> spans;
    std::vector<int32_t> gstart(1, 0);
    const int64_t T = group_target(s->n_windows, n_groups);
    int64_t cum = 0;
    for (const Span &seg : s->seg_spans) {
        const int64_t nch = (seg.ncols + kChunk - 1) / kChunk;
        for (int64_t j = 0; j < nch;) {
            const int64_t k = (cum + j * kChunk) / T;                       // this chunk's group
            const int64_t j_end = std::min(nch, chunk_at_or_after(cum, (k + 1) * T));  // first chunk of a later group
            while ((int64_t)gstart.size() <= k) gstart.push_back((int32_t)spans.size());  // group k starts here
            Span sp;
            sp.g0 = seg.g0 + j * kChunk;
            sp.ncols = (int32_t)(std::min<int64_t>(seg.ncols, j_end * kChunk) - j * kChunk);
            sp.pad = 0;
            spans.push_back(sp);
            j = j_end;
        }
        cum += seg.ncols;
    }
    while ((int)gstart.size() < n_groups + 1) gstart.push_back((int32_t)spans.size());
    DictStats::Grouping g;
    g.n_spans = (int32_t)spans.size();
    CUDA_TRY(cudaMalloc(&g.spans, std::max<size_t>(1, spans.size()) * sizeof(Span)));
    CUDA_TRY(cudaMalloc(&g.group_start, gstart.size() * sizeof(int32_t)));
    if (!spans.empty())
        CUDA_TRY(cudaMemcpyAsync(g.spans, spans.data(), spans.size() * sizeof(Span), cudaMemcpyHostToDevice,
                                 ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(g.group_start, gstart.data(), gstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    s->groupings[n_groups] = g;
    *out = &s->groupings[n_groups];
    return MP_OK;
}

static void free_stats(DictStats *s)
{
    cudaFree(s->d_seg_spans);
    cudaFree(s->mean);
    cudaFree(s->invstd);
    cudaFree(s->cflag);
    cudaFree(s->rs);
    cudaFree(s->ms);
    for (auto &kv : s->groupings) {
        cudaFree(kv.second.spans);
        cudaFree(kv.second.group_start);
        cudaFree(kv.second.left_ops);
    }
    tc_free_pack(s->tc_pack);
}

template <typename T>
static FinalizeParams<T> fin_params(mp_ctx *ctx, int64_t nq, int32_t m, int n_groups, const Partial<T> *part, const T *a,
                                    const vec4_t<T> *rs_a, const Split<T> *ms_a, const uint8_t *cf_a,
                                    const mp_dict *d, const DictStats *s, double *dist, int64_t *idx)
{
    FinalizeParams<T> f;
    f.nq = nq;
    f.m = m;
    f.n_groups = n_groups;
    f.part = part;
    f.a = a;
    f.rs_a = rs_a;
    f.ms_a = ms_a;
    f.cflag_a = cf_a;
    f.b = (const T *)d->d_samples;
    f.nb = d->nb;
    f.npos_b = d->nb - m + 1;
    f.rs_b = (const vec4_t<T> *)s->rs;
    f.ms_b = (const Split<T> *)s->ms;
    f.g_const = s->g_const;
    f.g_first = s->g_first;
    f.out_dist = dist;
    f.out_idx = idx;
    f.err = nullptr;
    f.near = NearRec{};
    f.cspans = nullptr;
    f.cgroup_start = nullptr;
    f.ctr = ctx->d_counters;
    f.sm_count = ctx->sm_count;
    f.out_corr = 0;
    f.excl = 0;
    f.next_const = nullptr;
    return f;
}

// Launch geometry of the plain kernel for nq rows and W columns.
struct Geometry {
    int warps, n_row_blocks, n_groups;
    int rows_per_lane = 0;  // the geometry's rows per lane
};

// Resident CTAs per SM of the plain kernel, from the occupancy API, cached per
// (dtype, warps, m, rows per lane): the serving scheduler sizes every request with it.
static int plain_ctas_cached(bool f64, int warps, int m, int rows_per_lane)
{
    static std::mutex mu;
    static std::map<std::tuple<bool, int, int, int>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(f64, warps, m, rows_per_lane);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int n = f64 ? plain_ctas_per_sm<double>(warps, m) : plain_ctas_per_sm<float>(warps, m, rows_per_lane);
    cache[key] = n;
    return n;
}

// tc_seeds: the FP32 plain kernel loads its left seeds (computed on the
// tensor cores) instead of computing them; batched: the serving kernel, where
// a request's column groups share the GPU with other requests' work.
static Geometry plain_geometry(const mp_ctx *ctx, int64_t nq, int64_t W, int rows_per_lane, int dtype = -1,
                               int m = 0, int64_t n_segments = 1, bool tc_seeds = false, bool batched = false)
{
    Geometry g;
    const int64_t rows_warp = 32 * rows_per_lane;
    g.warps = nq <= rows_warp ? 1 : (nq <= 2 * rows_warp ? 2 : 4);
    const int64_t rows_cta = rows_warp * g.warps;
    g.n_row_blocks = (int)((nq + rows_cta - 1) / rows_cta);
    // Column groups, chosen by a cost model of whole waves: a launch of
    // n_row_blocks * ng CTAs takes ceil(CTAs / resident CTAs) waves, each as
    // long as one CTA's columns plus its fixed work (staging the query rows
    // and a first column block, about (m + 64) / 4 columns' worth) plus its
    // left seeds per span (about m/4 columns' work when computed in the
    // kernel, 8 when loaded), plus the finalisation's walk over the groups'
    // partial results (about 5 columns' worth per group: its loads of a row's
    // groups follow one another). The smallest ng within 2 % of the cheapest
    // wins. A group keeps at least 16 columns (one chunk of the lazy argmax);
    // a batched request's groups keep enough columns that their fixed work
    // stays within a quarter of the request's, since other requests fill the
    // GPU.
    const double fixed = (double)(std::max(m, 16) + 64) / 4.0;
    const double span_cost = tc_seeds ? 8.0 : (double)std::max(m, 16) / 4.0;
    const int64_t min_cols = batched ? (int64_t)(4.0 * (fixed + span_cost)) : 16;
    const int64_t max_g = std::max<int64_t>(1, std::min<int64_t>(1024, W / min_cols));
    const int per_sm = m > 0 ? plain_ctas_cached(dtype == MP_F64, g.warps, m, rows_per_lane) : 4;
    const double slots = (double)ctx->sm_count * per_sm;
    const double nseg = std::max<double>(1.0, (double)n_segments);
    auto cost = [&](int64_t k) {
        const double waves = std::ceil((double)g.n_row_blocks * (double)k / slots);
        return waves * ((double)W / (double)k + fixed + span_cost * (nseg / (double)k + 1.0)) + 5.0 * (double)k;
    };
    double best_c = 1e300;
    for (int64_t k = 1; k <= max_g; ++k) best_c = std::min(best_c, cost(k));
    int64_t ng = 1;
    while (ng < max_g && cost(ng) > 1.02 * best_c) ++ng;
    if (ctx->force_groups > 0) {
        ng = ctx->force_groups;
    } else if (dtype >= 0 && ctx->kernel == MP_KERNEL_AUTO) {
        auto it = ctx->tune.find(TuneKey{dtype, m, ilog2(W), ilog2(nq)});
        if (it != ctx->tune.end() && it->second.kernel == MP_KERNEL_PLAIN) ng = it->second.groups;
    }
    // at most one group per chunk's worth of windows (T >= kChunk: no group
    // without a chunk), also for a grouping taken from the tuning cache
    g.n_groups = (int)std::max<int64_t>(1, std::min<int64_t>(ng, W / kChunk));
    g.rows_per_lane = rows_per_lane;
    return g;
}

// Top seeds of the plain FP32 kernel computed on the tensor cores: one row
// per warp of query windows (every 32 * kPlainRowsPerLane-th window), one
// column per dictionary window position. A join whose seed matrix would
// exceed kSeedCapBytes runs in row chunks (whole CTAs: multiples of
// 4 * 32 * kPlainRowsPerLane query windows), each with its own seeds in the
// same buffer.
constexpr size_t kSeedCapBytes = (size_t)2 << 30;

struct SeedGeo {
    int64_t n_srows;     // seed rows of one chunk
    int64_t ld;          // row stride (dictionary positions rounded up to 4)
    int64_t chunk_rows;  // query windows per chunk (all of them without chunking)
    size_t bytes;        // seed bytes of one chunk
};

static SeedGeo seed_geometry(int64_t nq, int64_t npos_b)
{
    SeedGeo g;
    const int64_t stride = 32 * kPlainRowsPerLane;
    g.ld = (std::max<int64_t>(1, npos_b) + 3) & ~(int64_t)3;
    const size_t row_bytes = (size_t)g.ld * sizeof(float);
    const int64_t full = (nq + stride - 1) / stride;
    if ((size_t)full * row_bytes <= kSeedCapBytes) {
        g.n_srows = full;
        g.chunk_rows = nq;
    } else {
        // whole CTAs of 4 warps (4 seed rows) per chunk
        g.n_srows = std::max<int64_t>(4, (int64_t)(kSeedCapBytes / row_bytes) & ~(int64_t)3);
        g.chunk_rows = g.n_srows * stride;
    }
    g.bytes = (size_t)g.n_srows * row_bytes;
    return g;
}

// Query windows per launch of the plain join (chunks only for FP32 with seeds).
static int64_t plain_chunk_rows(const mp_dict *d, int32_t dtype, int64_t nq, int32_t m, bool seeds)
{
    if (!seeds || dtype != MP_F32) return nq;
    return seed_geometry(nq, d->nb - m + 1).chunk_rows;
}

// Workspace layout of one join.
struct JoinWs {
    size_t off_err, off_mean, off_inv, off_cflag, off_rs, off_ms, off_part, off_near, off_seed, off_left, total;
    int near_slots;
};

// Near-tie record slots per (column group, query window) a join form uses.
static bool is_tc(int kernel)
{
    return kernel == MP_KERNEL_TC_BF16X3 || kernel == MP_KERNEL_TC_TF32 || kernel == MP_KERNEL_TC_BF16;
}
// tc_join's variant of a tensor-core form
static int tc_variant(int kernel) { return kernel == MP_KERNEL_TC_TF32 ? 1 : (kernel == MP_KERNEL_TC_BF16 ? 2 : 0); }
static int near_slots_for(int kernel) { return is_tc(kernel) ? kNearSlotsTC : kNearSlotsPlain; }

// near_slots: record slots per (column group, query window) of FP32 joins.
static JoinWs join_ws_layout(int64_t nq, int32_t dtype, int n_groups, size_t extra_front, size_t seed_bytes = 0,
                             int near_slots = kNearSlotsPlain, size_t left_bytes = 0)
{
    JoinWs w;
    // error word of the tensor-core kernels at the front
    const size_t e = dtype == MP_F64 ? 8 : 4;
    size_t o = align_up(extra_front, 256);
    w.off_err = o;
    o += 256;
    w.off_mean = o;
    o = align_up(o + nq * 8, 256);
    w.off_inv = o;
    o = align_up(o + nq * 8, 256);
    w.off_cflag = o;
    o = align_up(o + nq, 256);
    w.off_rs = o;
    o = align_up(o + nq * 4 * e, 256);
    w.off_ms = o;
    o = align_up(o + nq * 2 * e, 256);
    w.off_part = o;
    o = align_up(o + (size_t)n_groups * nq * (e == 8 ? sizeof(Partial<double>) : sizeof(Partial<float>)), 256);
    // near-tie records of FP32 joins: a header and near_slots slots per
    // (column group, query window)
    w.near_slots = dtype == MP_F32 ? near_slots : 0;
    w.off_near = o;
    if (dtype == MP_F32) o = align_up(o + (size_t)n_groups * (w.near_slots + 1) * nq * sizeof(NearSlot), 256);
    w.off_seed = o;
    o = align_up(o + seed_bytes, 256);
    // left seeds of the FP32 plain join (row chunk of the query windows)
    w.off_left = o;
    o = align_up(o + left_bytes, 256);
    w.total = o;
    return w;
}

// The near-tie records of a join laid out by w, for query windows of stride
// ld (the tensor-core join adds its width's terms, fb and u).
static NearRec near_rec(unsigned char *base, const JoinWs &w, int64_t ld)
{
    NearRec r{};
    r.rec = (NearSlot *)(base + w.off_near);
    r.ld = ld;
    r.S = w.near_slots;
    r.rho = kNearRhoFP32;
    return r;
}

// Seed bytes a join of this shape reserves (FP32 joins that may take the
// plain kernel with tensor-core seeds).
static size_t join_seed_bytes(const mp_dict *d, int32_t dtype, int64_t nq, int32_t m, bool seeds)
{
    if (!seeds || dtype != MP_F32) return 0;
    return seed_geometry(nq, d->nb - m + 1).bytes;
}

// Spans get_grouping cuts the dictionary's windows into for n_groups column
// groups (a segment contributes one span per group it meets).
static int64_t grouping_spans(const DictStats *s, int n_groups)
{
    const int64_t T = group_target(s->n_windows, n_groups);
    int64_t n = 0, cum = 0;
    for (const Span &seg : s->seg_spans) {
        n += segment_pieces(cum, seg.ncols, T);
        cum += seg.ncols;
    }
    return n;
}

// Row stride of the left seeds: the query windows of one row chunk, rounded up
// to 4 (16-byte rows).
static int64_t left_ld_for(int64_t crow) { return (crow + 3) & ~(int64_t)3; }

// Geometry of the plain join of nq query windows (row chunks included); seeds:
// the tensor-core seeds are taken (join_device's decision). A short FP32 join
// computing its seeds in the kernel takes the short form's rows per lane.
static Geometry join_plain_geometry(const mp_ctx *ctx, const mp_dict *d, const DictStats *s, int32_t dtype,
                                    int64_t nq, int32_t m, bool seeds)
{
    int rpl = dtype == MP_F64 ? plain_rows_per_lane<double>() : plain_rows_per_lane<float>();
    if (dtype == MP_F32 && !seeds && nq <= kPlainShortMaxRows) rpl = kPlainRowsShort;
    return plain_geometry(ctx, plain_chunk_rows(d, dtype, nq, m, seeds), std::max<int64_t>(1, s->n_windows), rpl,
                          dtype, m, (int64_t)s->seg_spans.size(), seeds && dtype == MP_F32);
}

// The workspace layout join_device uses for this form: the plain form's column
// groups with its near-tie slots, or the tensor-core forms' groups with theirs.
static JoinWs join_layout(const mp_ctx *ctx, const mp_dict *d, const DictStats *s, int32_t dtype, int64_t nq,
                          int32_t m, int kernel, bool seeds)
{
    if (is_tc(kernel))
        return join_ws_layout(nq, dtype, tc_groups_bound(ctx->sm_count, nq), 0,
                              join_seed_bytes(d, dtype, nq, m, seeds), near_slots_for(kernel));
    const int groups = join_plain_geometry(ctx, d, s, dtype, nq, m, seeds).n_groups;
    size_t left = 0;
    if (seeds && dtype == MP_F32)
        left = (size_t)grouping_spans(s, groups) * left_ld_for(plain_chunk_rows(d, dtype, nq, m, seeds)) * 4;
    return join_ws_layout(nq, dtype, groups, 0, join_seed_bytes(d, dtype, nq, m, seeds), near_slots_for(kernel),
                          left);
}

// Whether an FP32 plain join of nq query windows takes its top and left seeds
// from the tensor-core kernels (K2s, K2l) rather than computing them in the
// plain kernel. The two seed kernels cost a few tens of microseconds whatever
// the size (their tiles run one after another inside a CTA); computing the
// seeds in the plain kernel costs about a seventh of its column work plus
// m/4 columns per span and CTA. Below about 2^31 pairs the in-kernel seeds
// are cheaper.
constexpr double kTcSeedMinPairs = 2147483648.0;
static bool tc_seeds_pay(const DictStats *s, int32_t dtype, int64_t nq)
{
    return dtype == MP_F32 && (double)nq * (double)std::max<int64_t>(1, s->n_windows) >= kTcSeedMinPairs;
}

// The join on device buffers; `base` is a device workspace of at least
// join_layout(...).total bytes (join_ws_bytes covers every form). Everything is enqueued on `st`.
// With `seeds`, an FP32 plain join takes its top seeds from the tensor cores
// (the workspace then holds join_seed_bytes(..., true) more bytes). The
// error word at the front of the workspace is zeroed first; tensor-core
// kernels set it when a bounded wait runs out.
// excl > 0 makes it the self-join of one series (the query is the dictionary's
// only segment): pairs with |g - i| < excl are trivial matches and are left
// out; next_const is the series' next-constant-window table (launch_next_const).
static int join_device(mp_ctx *ctx, mp_dict *d, DictStats *s, const void *dq, int32_t dtype, int64_t n, int32_t m,
                       double *d_dist, int64_t *d_idx, cudaStream_t st, unsigned char *base, int kernel,
                       bool seeds = true, bool corr = false, int32_t excl = 0, const int64_t *next_const = nullptr)
{
    if (excl > 0 && (dtype != MP_F32 || !seeds || kernel != MP_KERNEL_PLAIN || !next_const))
        return fail(MP_E_INTERNAL, "the self-join runs the FP32 plain kernel with tensor-core seeds");
    const int64_t nq = n - m + 1;
    if (s->n_windows == 0) return fail(MP_E_INTERNAL, "empty dictionary must be handled by the caller");
    // a small join computes its seeds in the plain kernel (the self-join's kernel needs the tensor-core seeds)
    if (excl == 0) seeds = seeds && tc_seeds_pay(s, dtype, nq);
    const int64_t crow = plain_chunk_rows(d, dtype, nq, m, seeds);  // query windows per plain launch
    const Geometry geo = join_plain_geometry(ctx, d, s, dtype, nq, m, seeds);
    const bool tc = is_tc(kernel);
    const JoinWs w = join_layout(ctx, d, s, dtype, nq, m, kernel, seeds);
    int32_t *err = (int32_t *)(base + w.off_err);
    CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    double *mean_a = (double *)(base + w.off_mean);
    double *inv_a = (double *)(base + w.off_inv);
    uint8_t *cf_a = (uint8_t *)(base + w.off_cflag);
    DictStats::Grouping *gr = nullptr;
    int rc = get_grouping(ctx, s, geo.n_groups, &gr);
    if (rc) return rc;
    PlainLaunch L;
    L.nq = nq;
    L.m = m;
    L.n_row_blocks = geo.n_row_blocks;
    L.n_groups = geo.n_groups;
    L.warps = geo.warps;
    L.rows_per_lane = dtype == MP_F32 ? geo.rows_per_lane : 0;
    if (dtype == MP_F64) {
        const double *a = (const double *)dq;
        dvec4 *rs_a = (dvec4 *)(base + w.off_rs);
        Split<double> *ms_a = (Split<double> *)(base + w.off_ms);
        Partial<double> *part = (Partial<double> *)(base + w.off_part);
        {
            PhaseTimer t(ctx, MP_PHASE_STATS, st);
            CUDA_TRY(launch_window_stats<double>(a, n, m, mean_a, inv_a, cf_a, rs_a, ms_a, st));
        }
        {
            PhaseTimer t(ctx, MP_PHASE_JOIN, st);
            CUDA_TRY(launch_plain<double>(L, a, n, rs_a, ms_a, (const double *)d->d_samples, d->nb,
                                          (const dvec4 *)s->rs, (const Split<double> *)s->ms, gr->spans,
                                          gr->group_start, part, nullptr, 0, nullptr, 0, NearRec{}, st));
        }
        {
            PhaseTimer t(ctx, MP_PHASE_FINALIZE, st);
            FinalizeParams<double> f =
                fin_params<double>(ctx, nq, m, geo.n_groups, part, a, rs_a, ms_a, cf_a, d, s, d_dist, d_idx);
            f.out_corr = corr ? 1 : 0;
            CUDA_TRY(launch_finalize<double>(f, st));
        }
    } else {
        const float *a = (const float *)dq;
        float4 *rs_a = (float4 *)(base + w.off_rs);
        Split<float> *ms_a = (Split<float> *)(base + w.off_ms);
        {
            PhaseTimer t(ctx, MP_PHASE_STATS, st);
            CUDA_TRY(launch_window_stats<float>(a, n, m, mean_a, inv_a, cf_a, rs_a, ms_a, st));
        }
        if (tc) {
            Partial<float> *part = (Partial<float> *)(base + w.off_part);
            NearRec near = near_rec(base, w, nq);
            int ng = 1;
            const Span *cspans = nullptr;
            const int32_t *cgs = nullptr;
            {
                PhaseTimer t(ctx, MP_PHASE_JOIN, st);
                int rc = tc_join(ctx->sm_count, tc_variant(kernel), &s->tc_pack,
                                 (const float *)d->d_samples, d->nb, s->seg_spans.data(),
                                 (int32_t)s->seg_spans.size(), s->ms, s->rs, a, n, m, ms_a, rs_a, part, &near, err,
                                 &ng, &cspans, &cgs, ctx->hook_tc_wait, st, fail);
                if (rc) return rc;
            }
            {
                PhaseTimer t(ctx, MP_PHASE_FINALIZE, st);
                FinalizeParams<float> f =
                    fin_params<float>(ctx, nq, m, ng, part, a, rs_a, ms_a, cf_a, d, s, d_dist, d_idx);
                f.err = err;
                f.near = near;
                f.cspans = cspans;
                f.cgroup_start = cgs;
                f.out_corr = corr ? 1 : 0;
                CUDA_TRY(launch_finalize<float>(f, st));
            }
            return MP_OK;
        }
        Partial<float> *part = (Partial<float> *)(base + w.off_part);
        const NearRec near = near_rec(base, w, nq);
        float *seed_top = nullptr, *left = nullptr;
        const SeedGeo sg = seed_geometry(nq, d->nb - m + 1);
        const int64_t left_ld = left_ld_for(crow);
        if (seeds) {
            seed_top = (float *)(base + w.off_seed);
            left = (float *)(base + w.off_left);
            if (gr->n_spans != grouping_spans(s, geo.n_groups))
                return fail(MP_E_INTERNAL, "left-seed layout: %d spans, %lld expected", gr->n_spans,
                            (long long)grouping_spans(s, geo.n_groups));
            if (!gr->left_ops) {
                // the spans' operand of the left-seed kernel: once per (dictionary, m, grouping);
                // synchronised, so that joins on any stream find it complete
                unsigned char *ops = nullptr;
                if (cudaMalloc(&ops, tc_left_operand_bytes(gr->n_spans, m)) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(MP_E_NOMEM, "left-seed operand");
                }
                int rc2 = tc_left_operand((const float *)d->d_samples, d->nb, s->ms, gr->spans, gr->n_spans, m, ops, st,
                                          fail);
                if (rc2 == MP_OK && cudaStreamSynchronize(st) != cudaSuccess)
                    rc2 = fail(MP_E_CUDA, "left-seed operand: %s", cudaGetErrorString(cudaGetLastError()));
                if (rc2) {
                    cudaFree(ops);
                    return rc2;
                }
                gr->left_ops = ops;
            }
        }
        // row chunks (one chunk unless the seed matrix would exceed its cap)
        for (int64_t r0 = 0; r0 < nq; r0 += crow) {
            const int64_t rows = std::min<int64_t>(crow, nq - r0);
            if (seeds) {
                {
                    PhaseTimer t(ctx, MP_PHASE_SEEDS, st);
                    int rc = tc_seeds(&s->tc_pack, (const float *)d->d_samples, d->nb,
                                      s->seg_spans.data(), (int32_t)s->seg_spans.size(), s->ms, a + r0, rows + m - 1,
                                      m, ms_a + r0, 32 * kPlainRowsPerLane, seed_top, sg.ld, err, st, fail);
                    if (rc) return rc;
                }
                PhaseTimer t(ctx, MP_PHASE_LEFT_SEEDS, st);
                int rc = tc_left_seeds(a + r0, rows + m - 1, m, ms_a + r0, s->ms, gr->spans, gr->n_spans, gr->left_ops,
                                       left, left_ld, err, st, fail);
                if (rc) return rc;
            }
            PhaseTimer t(ctx, MP_PHASE_JOIN, st);
            PlainLaunch Lc = L;
            const int64_t rows_cta = (int64_t)geo.warps * 32 * geo.rows_per_lane;
            Lc.nq = rows;
            Lc.n_row_blocks = (int32_t)((rows + rows_cta - 1) / rows_cta);
            Lc.ld_part = nq;
            Lc.row0 = r0;
            Lc.excl = excl;
            NearRec nc = near;  // this chunk's rows
            nc.rec += r0;
            CUDA_TRY(launch_plain<float>(Lc, a + r0, rows + m - 1, rs_a + r0, ms_a + r0, (const float *)d->d_samples,
                                         d->nb, (const float4 *)s->rs, (const Split<float> *)s->ms, gr->spans,
                                         gr->group_start, part + r0, seed_top, seeds ? sg.ld : 0, left,
                                         seeds ? left_ld : 0, nc, st));
        }
        {
            PhaseTimer t(ctx, MP_PHASE_FINALIZE, st);
            FinalizeParams<float> f =
                fin_params<float>(ctx, nq, m, geo.n_groups, part, a, rs_a, ms_a, cf_a, d, s, d_dist, d_idx);
            f.err = seeds ? err : nullptr;
            f.near = near;
            f.cspans = gr->spans;
            f.cgroup_start = gr->group_start;
            f.out_corr = corr ? 1 : 0;
            f.excl = excl;
            f.next_const = next_const;
            CUDA_TRY(launch_finalize<float>(f, st));
        }
    }
    return MP_OK;
}

static size_t join_ws_bytes(const mp_ctx *ctx, const mp_dict *d, const DictStats *s, int32_t dtype, int64_t n,
                            int32_t m, bool seeds = true)
{
    const int64_t nq = n - m + 1;
    // the plain form with the seeds the join may take (join_device leaves out
    // the tensor-core seeds of a small join), or a tensor-core form
    size_t b = join_layout(ctx, d, s, dtype, nq, m, MP_KERNEL_PLAIN, false).total;
    if (seeds) b = std::max(b, join_layout(ctx, d, s, dtype, nq, m, MP_KERNEL_PLAIN, true).total);
    if (dtype == MP_F32) b = std::max(b, join_layout(ctx, d, s, dtype, nq, m, MP_KERNEL_TC_BF16X3, seeds).total);
    return b;
}

static int resolve_kernel(const mp_ctx *ctx, int32_t dtype, int32_t m, const DictStats *s, int64_t nq)
{
    if (dtype == MP_F64) return MP_KERNEL_PLAIN;
    int k = ctx->kernel;
    if (k == MP_KERNEL_AUTO) {
        // the autotuner's choice for this shape, else the plain form (the
        // fastest on every workload measured without a tuning run)
        k = MP_KERNEL_PLAIN;
        auto it = ctx->tune.find(TuneKey{dtype, m, ilog2(std::max<int64_t>(1, s->n_windows)), ilog2(nq)});
        if (it != ctx->tune.end()) k = it->second.kernel;
    }
    if (k == MP_KERNEL_TC_BF16X3 && !tc_supported(0, m)) k = MP_KERNEL_PLAIN;
    if (k == MP_KERNEL_TC_TF32 && !tc_supported(1, m)) k = MP_KERNEL_PLAIN;
    if (k == MP_KERNEL_TC_BF16 && !tc_supported(2, m)) k = MP_KERNEL_PLAIN;
    return k;
}

// ---------------------------------------------------------------------------
// serving scheduler
// ---------------------------------------------------------------------------
// Geometry of one request in the batched serving kernel: kServeRowsPerLane
// rows per lane, 4 warps per CTA. The request's memory is sized and laid out
// with this one function, so the two always agree.
static Geometry serve_geometry(const mp_ctx *ctx, int64_t nq, const DictStats *s, int32_t dtype, int32_t m)
{
    Geometry geo =
        plain_geometry(ctx, nq, std::max<int64_t>(1, s->n_windows), kServeRowsPerLane, dtype, m,
                       (int64_t)s->seg_spans.size(), false, true);
    geo.warps = 4;
    geo.n_row_blocks = (int)((nq + 4 * 32 * kServeRowsPerLane - 1) / (4 * 32 * kServeRowsPerLane));
    return geo;
}

// Device bytes of a request: its query, its outputs (dist, idx) and a
// workspace for either way it may run (alone through join_device, or in the
// batched kernel).
// Query windows from which a serving request of FP32 data runs alone, in a
// batch of such requests on a low-priority stream, with the headline join's
// kernels (tensor-core top seeds and the packed plain kernel at three CTAs per
// SM), rather than as items of the batched kernel (its own scalar seeds, two
// CTAs per SM). Such a request fills the GPU by itself: 2^16 windows are 26
// row blocks in each column group.
constexpr int64_t kServeAloneRows = (int64_t)1 << 16;
static bool serve_alone(const Request &r) { return r.n - r.m + 1 >= kServeAloneRows; }

static size_t request_ws_bytes(const mp_ctx *ctx, const Request &r, const DictStats *s)
{
    const int64_t nq = r.n - r.m + 1;
    size_t ws = join_ws_bytes(ctx, r.dict, s, r.dtype, r.n, r.m, r.dtype == MP_F32 && serve_alone(r));
    if (s->n_windows > 0 && r.dtype == MP_F32)
        ws = std::max(ws, join_ws_layout(nq, r.dtype, serve_geometry(ctx, nq, s, r.dtype, r.m).n_groups, 0).total);
    return ws;
}

static size_t request_bytes(const mp_ctx *ctx, const Request &r, const DictStats *s)
{
    const int64_t nq = r.n - r.m + 1;
    return align_up((size_t)r.n * dtype_size(r.dtype), 256) + align_up(nq * 16, 256) + request_ws_bytes(ctx, r, s);
}

// Pinned host buffer of at least `bytes` (caller holds ctx->smu or is the
// only user of the pool at that time).
static size_t pinned_class(size_t bytes)
{
    size_t c = 1 << 16;
    while (c < bytes) c <<= 1;
    return c;
}

// A pinned allocation costs tens of microseconds whatever its size, so
// staging buffers of one class are cut from slabs of at least 4 MB.
static void *pinned_take(mp_ctx *ctx, size_t bytes)
{
    const size_t c = pinned_class(bytes);
    auto &fl = ctx->pinned_free[c];
    if (fl.empty()) {
        const size_t slab = std::max(c, (size_t)4 << 20);
        void *p = nullptr;
        if (cudaHostAlloc(&p, slab, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->pinned_slabs.push_back(p);
        for (size_t o = 0; o + c <= slab; o += c) fl.push_back((unsigned char *)p + o);
    }
    void *p = fl.back();
    fl.pop_back();
    return p;
}

static void pinned_give(mp_ctx *ctx, void *p, size_t bytes)
{
    if (p) ctx->pinned_free[pinned_class(bytes)].push_back(p);
}

// The request's work has completed (or failed) on the device: the caller
// has seen its batch's event or synchronised its stream.
static void finish_request(mp_ctx *ctx, Request &r, int32_t state)
{
    if (state == MP_DONE) {
        // the result waits in the pinned staging buffer: dist then idx
        const int64_t nq = r.n - r.m + 1;
        if (r.no_windows) {
            for (int64_t i = 0; i < nq; ++i) {
                r.out_dist[i] = INFINITY;
                r.out_idx[i] = -1;
            }
        } else {
            memcpy(r.out_dist, r.h_stage, (size_t)nq * 8);
            memcpy(r.out_idx, (char *)r.h_stage + (size_t)nq * 8, (size_t)nq * 8);
        }
    }
    pinned_give(ctx, r.h_stage, r.stage_bytes);
    r.h_stage = nullptr;
    r.t_done = now_s();
    r.state = state;
    // stream-ordered free: no device-wide synchronisation in the serving loop
    if (r.dmem) cudaFreeAsync(r.dmem, ctx->fstream);
    r.dmem = nullptr;
    ctx->mem_used -= r.bytes;
    ctx->n_inflight_reqs -= 1;
    r.dict->refs.fetch_sub(1);
}

// Stage and launch one batch of admitted requests on stream `st`, from the
// scheduler thread. The context lock (ctx->mu) is held only while the
// requests' dictionary statistics and column groupings are resolved (they may
// be built then) and while requests that run alone are enqueued; the batched
// requests' copies and launches follow without it, so that submissions and
// synchronous joins on the context do not wait for them.
static int launch_batch(mp_ctx *ctx, Batch &bt)
{
    cudaStream_t st = bt.stream;
    std::vector<PlainRequest> preqs;
    std::vector<BatchItem> items;
    int max_m = 0;
    struct Post {
        Request *r;
        DictStats *s;
        const DictStats::Grouping *gr;
        int n_groups;
        unsigned char *base;
        float *a;
        double *dist;
        int64_t *idx;
    };
    std::vector<Post> post;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (auto &rp : bt.reqs) {
            Request &r = *rp;
            DictStats *s = nullptr;
            int rc = get_stats(ctx, r.dict, r.m, &s);
            if (rc) return rc;
            const int64_t nq = r.n - r.m + 1;
            unsigned char *p = (unsigned char *)r.dmem;
            unsigned char *q = p;
            p += align_up((size_t)r.n * dtype_size(r.dtype), 256);
            double *dist = (double *)p;
            int64_t *idx = (int64_t *)(p + nq * 8);
            p += align_up(nq * 16, 256);
            const int kern = s->n_windows > 0 ? resolve_kernel(ctx, r.dtype, r.m, s, nq) : MP_KERNEL_PLAIN;
            if (s->n_windows == 0) {
                r.no_windows = true;  // +inf / -1, written at completion
                continue;
            }
            if (r.dtype == MP_F64 || kern != MP_KERNEL_PLAIN || serve_alone(r)) {
                // Requests that do not fit the batched FP32 plain kernel, and
                // large ones, run alone on the batch's stream.
                CUDA_TRY(cudaMemcpyAsync(q, r.h_stage, (size_t)r.n * dtype_size(r.dtype), cudaMemcpyHostToDevice, st));
                rc = join_device(ctx, r.dict, s, q, r.dtype, r.n, r.m, dist, idx, st, p, kern,
                                 r.dtype == MP_F32 && serve_alone(r));
                if (rc) return rc;
                CUDA_TRY(cudaMemcpyAsync(r.h_stage, dist, (size_t)nq * 16, cudaMemcpyDeviceToHost, st));
                continue;
            }
            const Geometry geo = serve_geometry(ctx, nq, s, r.dtype, r.m);
            DictStats::Grouping *gr = nullptr;
            rc = get_grouping(ctx, s, geo.n_groups, &gr);
            if (rc) return rc;
            JoinWs w = join_ws_layout(nq, r.dtype, geo.n_groups, 0);
            // the layout must lie inside the request's memory (sized by request_bytes)
            if ((size_t)(p - (unsigned char *)r.dmem) + w.total > r.bytes)
                return fail(MP_E_INTERNAL, "serving workspace of %zu bytes exceeds the request's %zu", w.total,
                            r.bytes);
            PlainRequest pr{};  // seed_top null: the batched kernel computes its seeds
            pr.a = (const float *)q;
            pr.na = r.n;
            pr.nq = nq;
            pr.m = r.m;
            pr.n_groups = geo.n_groups;
            pr.rs_a = (float4 *)(p + w.off_rs);
            pr.ms_a = (Split<float> *)(p + w.off_ms);
            pr.b = (const float *)r.dict->d_samples;
            pr.nb = r.dict->nb;
            pr.rs_b = (const float4 *)s->rs;
            pr.ms_b = (const Split<float> *)s->ms;
            pr.spans = gr->spans;
            pr.group_start = gr->group_start;
            pr.part = (Partial<float> *)(p + w.off_part);
            pr.near = near_rec(p, w, nq);
            pr.ld_part = nq;
            const int ridx = (int)preqs.size();
            preqs.push_back(pr);
            for (int64_t rb = 0; rb < geo.n_row_blocks; ++rb)
                for (int g2 = 0; g2 < geo.n_groups; ++g2) items.push_back(BatchItem{ridx, g2, rb});
            max_m = std::max(max_m, (int)r.m);
            post.push_back(Post{&r, s, gr, geo.n_groups, p, (float *)q, dist, idx});
        }
    }
    if (!preqs.empty()) {
        // each batched request's query and statistics (K1)
        for (Post &ps : post) {
            Request &r = *ps.r;
            const int64_t nq = r.n - r.m + 1;
            JoinWs w = join_ws_layout(nq, r.dtype, ps.n_groups, 0);
            CUDA_TRY(cudaMemcpyAsync(ps.a, r.h_stage, (size_t)r.n * dtype_size(r.dtype), cudaMemcpyHostToDevice, st));
            CUDA_TRY(launch_window_stats<float>(ps.a, r.n, r.m, (double *)(ps.base + w.off_mean),
                                                (double *)(ps.base + w.off_inv), (uint8_t *)(ps.base + w.off_cflag),
                                                (float4 *)(ps.base + w.off_rs), (Split<float> *)(ps.base + w.off_ms),
                                                st));
        }
        const size_t sz_req = align_up(preqs.size() * sizeof(PlainRequest), 256);
        const size_t sz_items = align_up(items.size() * sizeof(BatchItem), 256);
        if (cudaMallocFromPoolAsync(&bt.dmem, sz_req + sz_items + 256, ctx->pool, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(MP_E_NOMEM, "batch tables");
        }
        unsigned char *bp = (unsigned char *)bt.dmem;
        CUDA_TRY(cudaMemcpyAsync(bp, preqs.data(), preqs.size() * sizeof(PlainRequest), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(bp + sz_req, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                 st));
        int32_t *counter = (int32_t *)(bp + sz_req + sz_items);
        CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
        const int grid = (int)std::min<int64_t>((int64_t)items.size(), (int64_t)ctx->sm_count * 2);
        CUDA_TRY(launch_plain_batched((const PlainRequest *)bp, (const BatchItem *)(bp + sz_req),
                                      (int32_t)items.size(), counter, 4, max_m, grid, st));
        for (Post &ps : post) {
            Request &r = *ps.r;
            const int64_t nq = r.n - r.m + 1;
            JoinWs w = join_ws_layout(nq, r.dtype, ps.n_groups, 0);
            FinalizeParams<float> f =
                fin_params<float>(ctx, nq, r.m, ps.n_groups, (const Partial<float> *)(ps.base + w.off_part), ps.a,
                                  (const float4 *)(ps.base + w.off_rs), (const Split<float> *)(ps.base + w.off_ms),
                                  (const uint8_t *)(ps.base + w.off_cflag), r.dict, ps.s, ps.dist, ps.idx);
            f.near = near_rec(ps.base, w, nq);
            f.cspans = ps.gr->spans;
            f.cgroup_start = ps.gr->group_start;
            CUDA_TRY(launch_finalize<float>(f, st));
            CUDA_TRY(cudaMemcpyAsync(r.h_stage, ps.dist, (size_t)nq * 16, cudaMemcpyDeviceToHost, st));
        }
    }
    CUDA_TRY(cudaEventRecord(bt.done, st));
    return MP_OK;
}

static void scheduler_loop(mp_ctx *ctx)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->smu);
    while (true) {
        // 1. retire finished batches
        for (size_t k = 0; k < ctx->inflight.size();) {
            Batch &bt = ctx->inflight[k];
            cudaError_t q = cudaEventQuery(bt.done);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            const int32_t state = (q == cudaSuccess) ? MP_DONE : MP_FAILED;
            if (q != cudaSuccess) cudaGetLastError();
            for (auto &r : bt.reqs) finish_request(ctx, *r, state);
            cudaEventDestroy(bt.done);
            if (bt.dmem) cudaFreeAsync(bt.dmem, ctx->fstream);
            ctx->inflight.erase(ctx->inflight.begin() + k);
        }
        if (ctx->stop && ctx->pending.empty() && ctx->inflight.empty()) break;
        // 2. admit: FIFO, while a slot and the memory budget allow. Large
        // requests (they run alone, see serve_alone) go to a batch of their
        // own on a low-priority stream, the rest to a batch on a high-priority
        // stream.
        Batch bs, bl;
        bs.stream = ctx->sstreams[ctx->next_small];
        bl.stream = ctx->sstreams[2 + ctx->next_large];
        while (!ctx->pending.empty() && (int)(bs.reqs.size() + bl.reqs.size()) < ctx->cfg.max_batch &&
               ctx->n_inflight_reqs < ctx->cfg.max_inflight) {
            std::shared_ptr<Request> r = ctx->pending.front();
            if (ctx->mem_used + r->bytes > ctx->mem_budget && ctx->n_inflight_reqs > 0) break;
            ctx->pending.pop_front();
            Batch &bt = serve_alone(*r) ? bl : bs;
            const bool injected = ctx->hook_fail_alloc > 0;  // a testing hook: fail as if out of memory
            if (injected) --ctx->hook_fail_alloc;
            if (injected || cudaMallocFromPoolAsync(&r->dmem, r->bytes, ctx->pool, bt.stream) != cudaSuccess) {
                cudaGetLastError();
                pinned_give(ctx, r->h_stage, r->stage_bytes);
                r->h_stage = nullptr;
                r->t_done = now_s();
                r->state = MP_FAILED;
                r->dict->refs.fetch_sub(1);
                continue;
            }
            ctx->mem_used += r->bytes;
            ctx->n_inflight_reqs += 1;
            bt.reqs.push_back(r);
        }
        bool launched = false;
        for (Batch *b : {&bs, &bl}) {  // the small requests' work is enqueued first
            if (b->reqs.empty()) continue;
            launched = true;
            (b == &bs ? ctx->next_small : ctx->next_large) ^= 1;
            Batch &bt = *b;
            cudaEventCreateWithFlags(&bt.done, cudaEventDisableTiming);
            lk.unlock();
            const int rc = launch_batch(ctx, bt);  // takes ctx->mu itself, for what needs it
            lk.lock();
            if (rc != MP_OK) {
                cudaStreamSynchronize(bt.stream);
                for (auto &r : bt.reqs) finish_request(ctx, *r, MP_FAILED);
                cudaEventDestroy(bt.done);
                if (bt.dmem) cudaFreeAsync(bt.dmem, ctx->fstream);
            } else {
                ctx->inflight.push_back(std::move(bt));
            }
        }
        if (launched) continue;
        // 3. nothing to admit: wait for a submission or poll the device
        if (ctx->inflight.empty())
            ctx->scv.wait(lk, [&] { return ctx->stop || !ctx->pending.empty(); });
        else
            ctx->scv.wait_for(lk, std::chrono::microseconds(50));
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *mp_last_error(void) { return g_err.c_str(); }

int mp_config_default(mp_config *cfg)
{
    if (!cfg) return fail(MP_E_ARG, "null cfg");
    memset(cfg, 0, sizeof *cfg);
    cfg->device = 0;
    cfg->kernel = MP_KERNEL_AUTO;
    cfg->max_inflight = 8;
    cfg->max_batch = 64;
    cfg->mem_budget = 0;
    cfg->tune_cache = nullptr;
    cfg->max_pending = 1 << 16;
    return MP_OK;
}

int mp_init(mp_ctx **out, const mp_config *cfg_in)
{
    g_err.clear();
    if (!out) return fail(MP_E_ARG, "null ctx pointer");
    mp_config cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        mp_config_default(&cfg);
    if (cfg.kernel < MP_KERNEL_AUTO || cfg.kernel > MP_KERNEL_TC_BF16) return fail(MP_E_ARG, "unknown kernel");
    if (cfg.max_inflight <= 0) cfg.max_inflight = 8;
    if (cfg.max_batch <= 0) cfg.max_batch = 64;
    if (cfg.max_pending <= 0) cfg.max_pending = 1 << 16;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (cfg.device < 0 || cfg.device >= ndev) return fail(MP_E_ARG, "device %d of %d", cfg.device, ndev);
    CUDA_TRY(cudaSetDevice(cfg.device));
    std::unique_ptr<mp_ctx> c(new mp_ctx());
    c->device = cfg.device;
    c->cfg = cfg;
    c->kernel = cfg.kernel;
    CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cfg.device));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    {
        int least = 0, greatest = 0;
        CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int k = 0; k < mp_ctx::kServeStreams; ++k)
            CUDA_TRY(cudaStreamCreateWithPriority(&c->sstreams[k], cudaStreamNonBlocking, k < 2 ? greatest : least));
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&c->fstream, cudaStreamNonBlocking));
    {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = cfg.device;
        CUDA_TRY(cudaMemPoolCreate(&c->pool, &props));
        uint64_t keep = UINT64_MAX;
        CUDA_TRY(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        // reuse only memory whose free has completed: the pool may otherwise
        // make an allocation's stream wait for the stream that freed the
        // memory, and a small request on a high-priority stream would then
        // wait for a large join on a low-priority one
        int no = 0;
        CUDA_TRY(cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no));
    }
    CUDA_TRY(cudaMalloc(&c->d_counters, kFinCounters * sizeof(unsigned long long)));
    CUDA_TRY(cudaMemset(c->d_counters, 0, kFinCounters * sizeof(unsigned long long)));
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    c->mem_budget = cfg.mem_budget ? cfg.mem_budget : fr / 2;
    if (cfg.tune_cache) tune_load(c.get(), cfg.tune_cache);

    mp_ctx *p = c.release();
    p->worker = std::thread(scheduler_loop, p);
    *out = p;
    return MP_OK;
}

int mp_shutdown(mp_ctx *ctx)
{
    g_err.clear();
    if (!ctx) return fail(MP_E_ARG, "null ctx");
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->stop = true;
    }
    ctx->scv.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    graphs_clear(ctx);
    for (mp_dict *d : ctx->dicts) {
        for (auto &kv : d->stats) free_stats(kv.second.get());
        cudaFree(d->d_samples);
        delete d;
    }
    if (ctx->ws) cudaFree(ctx->ws);
    cudaFree(ctx->d_counters);
    for (auto &mk : ctx->marks) {
        cudaEventDestroy(mk.t0);
        cudaEventDestroy(mk.t1);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (void *p : ctx->pinned_slabs) cudaFreeHost(p);
    for (cudaStream_t st : ctx->sstreams) cudaStreamSynchronize(st);
    cudaStreamSynchronize(ctx->fstream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    cudaStreamDestroy(ctx->stream);
    for (cudaStream_t st : ctx->sstreams) cudaStreamDestroy(st);
    cudaStreamDestroy(ctx->fstream);
    delete ctx;
    return MP_OK;
}

int mp_set_kernel(mp_ctx *ctx, int32_t kernel)
{
    g_err.clear();
    if (!ctx) return fail(MP_E_ARG, "null ctx");
    if (kernel < MP_KERNEL_AUTO || kernel > MP_KERNEL_TC_BF16) return fail(MP_E_ARG, "unknown kernel %d", kernel);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->kernel = kernel;
    graphs_clear(ctx);
    return MP_OK;
}

int mp_dict_load(mp_ctx *ctx, const void *samples, int32_t dtype, const int64_t *offs, int32_t n_segments,
                 const int32_t *ms, int32_t n_ms, mp_dict **out)
{
    g_err.clear();
    if (!ctx || !offs || !out || n_segments < 0) return fail(MP_E_ARG, "null argument");
    if (dtype != MP_F32 && dtype != MP_F64) return fail(MP_E_ARG, "unknown dtype %d", dtype);
    if (offs[0] != 0) return fail(MP_E_ARG, "seg_offsets[0] must be 0");
    for (int32_t s = 0; s < n_segments; ++s)
        if (offs[s + 1] < offs[s]) return fail(MP_E_ARG, "seg_offsets not sorted at %d", s);
    const int64_t nb = offs[n_segments];
    if (nb >= ((int64_t)1 << 31)) return fail(MP_E_ARG, "dictionary larger than 2^31 samples");
    if (nb > 0 && !samples) return fail(MP_E_ARG, "null samples");
    if (!host_all_finite(samples, dtype, nb)) return fail(MP_E_ARG, "dictionary has NaN or Inf samples");
    if (n_ms < 0 || (n_ms > 0 && !ms)) return fail(MP_E_ARG, "bad ms");
    for (int32_t k = 0; k < n_ms; ++k)
        if (ms[k] < kMinM || ms[k] > kMaxM) return fail(MP_E_ARG, "m=%d outside [%d, %d]", ms[k], kMinM, kMaxM);
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::unique_ptr<mp_dict> d(new mp_dict());
    d->ctx = ctx;
    d->dtype = dtype;
    d->nb = nb;
    d->offs.assign(offs, offs + n_segments + 1);
    const size_t bytes = std::max<int64_t>(nb, 1) * dtype_size(dtype) + 64;
    if (cudaMalloc(&d->d_samples, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(MP_E_NOMEM, "dictionary of %zu bytes", bytes);
    }
    CUDA_TRY(cudaMemsetAsync(d->d_samples, 0, bytes, ctx->stream));
    if (nb > 0)
        CUDA_TRY(cudaMemcpyAsync(d->d_samples, samples, nb * dtype_size(dtype), cudaMemcpyHostToDevice, ctx->stream));
    for (int32_t k = 0; k < n_ms; ++k) {
        DictStats *s;
        int rc = get_stats(ctx, d.get(), ms[k], &s);
        if (rc) {
            for (auto &kv : d->stats) free_stats(kv.second.get());
            cudaFree(d->d_samples);
            return rc;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = d.get();
    ctx->dicts.insert(d.release());
    return MP_OK;
}

int mp_dict_free(mp_ctx *ctx, mp_dict *d)
{
    g_err.clear();
    if (!ctx || !d) return fail(MP_E_ARG, "null argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->dicts.count(d)) return fail(MP_E_ARG, "unknown dictionary");
    if (d->refs.load() > 0) return fail(MP_E_BUSY, "dictionary referenced by %d requests in flight", d->refs.load());
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    graphs_clear(ctx, d);
    for (auto &kv : d->stats) free_stats(kv.second.get());
    cudaFree(d->d_samples);
    ctx->dicts.erase(d);
    delete d;
    return MP_OK;
}

int mp_dict_windows(const mp_dict *d, int32_t m, int64_t *n_windows)
{
    g_err.clear();
    if (!d || !n_windows || m < 1) return fail(MP_E_ARG, "bad argument");
    int64_t w = 0;
    for (size_t k = 0; k + 1 < d->offs.size(); ++k) w += std::max<int64_t>(0, d->offs[k + 1] - d->offs[k] - m + 1);
    *n_windows = w;
    return MP_OK;
}

int mp_ab_join_device(mp_ctx *ctx, const mp_dict *dict, const void *d_query, int32_t dtype, int64_t n, int32_t m,
                      double *d_dist, int64_t *d_idx, void *stream)
{
    g_err.clear();
    int rc = check_join_args(ctx, dict, d_query, dtype, n, m);
    if (rc) return rc;
    if (!d_dist || !d_idx) return fail(MP_E_ARG, "null output");
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    mp_dict *d = const_cast<mp_dict *>(dict);
    DictStats *s;
    rc = get_stats(ctx, d, m, &s);
    if (rc) return rc;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    const int64_t nq = n - m + 1;
    if (s->n_windows == 0) {
        // No dictionary window: +inf and index -1 (Algorithm 2's initial value).
        std::vector<double> inf(nq, INFINITY);
        std::vector<int64_t> neg(nq, -1);
        CUDA_TRY(cudaMemcpyAsync(d_dist, inf.data(), nq * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(d_idx, neg.data(), nq * 8, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return MP_OK;
    }
    rc = ensure_ws(ctx, join_ws_bytes(ctx, d, s, dtype, n, m));
    if (rc) return rc;
    if (st != ctx->stream) {
        // the workspace may still be in use by earlier work on the context stream
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(ev, ctx->stream));
        CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
        cudaEventDestroy(ev);
    }
    rc = join_device(ctx, d, s, d_query, dtype, n, m, d_dist, d_idx, st, (unsigned char *)ctx->ws,
                     resolve_kernel(ctx, dtype, m, s, nq));
    if (rc) return rc;
    if (st != ctx->stream) {
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(ev, st));
        CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ev, 0));
        cudaEventDestroy(ev);
    }
    return MP_OK;
}

// CUDA graphs of repeated synchronous joins: joins of at most this many query
// windows (larger ones are bound by their kernels), at most this many cached
// shapes per context (the cache is emptied when it is full).
constexpr int64_t kGraphMaxWindows = (int64_t)1 << 18;
constexpr size_t kGraphMaxEntries = 16;

// The synchronous join with host buffers; corr: report rho = 1 - d^2 / (2m)
// (-inf where the dictionary has no window) instead of d.
static int ab_join_host(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
                        double *out_dist, int64_t *out_idx, bool corr)
{
    g_err.clear();
    int rc = check_join_args(ctx, dict, query, dtype, n, m);
    if (rc) return rc;
    if (!out_dist || !out_idx) return fail(MP_E_ARG, "null output");
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    mp_dict *d = const_cast<mp_dict *>(dict);
    DictStats *s;
    rc = get_stats(ctx, d, m, &s);
    if (rc) return rc;
    const int64_t nq = n - m + 1;
    if (s->n_windows == 0) {
        if (!host_all_finite(query, dtype, n)) return fail(MP_E_ARG, "query has NaN or Inf samples");
        for (int64_t i = 0; i < nq; ++i) {
            out_dist[i] = corr ? -INFINITY : INFINITY;
            out_idx[i] = -1;
        }
        return MP_OK;
    }
    const size_t qbytes = align_up((size_t)n * dtype_size(dtype), 256);
    const size_t obytes = align_up((size_t)nq * 8, 256);
    const size_t jb = join_ws_bytes(ctx, d, s, dtype, n, m);
    rc = ensure_ws(ctx, qbytes + 2 * obytes + jb);
    if (rc) return rc;
    unsigned char *base = (unsigned char *)ctx->ws;
    void *dq = base;
    double *dd = (double *)(base + qbytes);
    int64_t *di = (int64_t *)(base + qbytes + obytes);
    int32_t *d_err = (int32_t *)(base + qbytes + 2 * obytes);  // the tensor-core kernels' error word (join_device)
    cudaStream_t st = ctx->stream;
    const int kern = resolve_kernel(ctx, dtype, m, s, nq);
    const size_t es = dtype_size(dtype);

    // A small join repeated with the same shape (a streaming append, a loop of
    // short queries) is bound by its launches, not its kernels: from its second
    // call on it runs as one CUDA graph captured from the same enqueue sequence
    // (copy in from a pinned staging buffer, the join, copies out), replayed
    // with one launch. Off while tracing (the phase events are not captured).
    mp_ctx::GraphEntry *ge = nullptr;
    if (!ctx->profiling && nq <= kGraphMaxWindows) {
        const mp_ctx::GraphKey key{d, dtype, m, kern, corr ? 1 : 0, n};
        auto it = ctx->graphs.find(key);
        if (it == ctx->graphs.end() && ctx->graphs.size() >= kGraphMaxEntries) graphs_clear(ctx);
        ge = &ctx->graphs[key];
        if (ge->failed || (ge->exec == nullptr && ++ge->calls < 2)) ge = nullptr;  // first call: the normal path
    }
    if (ge && ge->exec && ge->ws != ctx->ws) {  // (graphs_clear runs when the workspace moves; kept as a guard)
        graph_entry_free(*ge);
    }
    if (ge && ge->exec == nullptr) {
        // capture this call's enqueue sequence
        ge->out_off = align_up((size_t)n * es, 256);
        const size_t io = ge->out_off + (size_t)nq * 16 + 16;
        bool ok = cudaHostAlloc((void **)&ge->h_io, io, cudaHostAllocPortable) == cudaSuccess;
        cudaGraph_t graph = nullptr;
        if (ok) ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            bool enq = cudaMemcpyAsync(dq, ge->h_io, (size_t)n * es, cudaMemcpyHostToDevice, st) == cudaSuccess;
            enq = enq && join_device(ctx, d, s, dq, dtype, n, m, dd, di, st, base + qbytes + 2 * obytes, kern, true,
                                     corr) == MP_OK;
            unsigned char *ho = ge->h_io + ge->out_off;
            enq = enq && cudaMemcpyAsync(ho, dd, (size_t)nq * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
            enq = enq && cudaMemcpyAsync(ho + (size_t)nq * 8, di, (size_t)nq * 8, cudaMemcpyDeviceToHost, st) ==
                             cudaSuccess;
            enq = enq && cudaMemcpyAsync(ho + (size_t)nq * 16, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st) ==
                             cudaSuccess;
            const bool ended = cudaStreamEndCapture(st, &graph) == cudaSuccess;
            ok = enq && ended && graph != nullptr &&
                 cudaGraphInstantiate(&ge->exec, graph, 0) == cudaSuccess;
        }
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            // this shape cannot be captured (something in its path synchronises
            // or allocates): join it the normal way from now on
            cudaGetLastError();
            g_err.clear();
            graph_entry_free(*ge);
            ge->failed = true;
            ge = nullptr;
        } else {
            ge->ws = ctx->ws;
        }
    }
    if (ge) {
        memcpy(ge->h_io, query, (size_t)n * es);
        CUDA_TRY(cudaGraphLaunch(ge->exec, st));
        // the NaN/Inf check runs while the device joins; nothing is copied out unless it passes
        const bool finite = host_all_finite(query, dtype, n);
        CUDA_TRY(cudaStreamSynchronize(st));
        if (!finite) return fail(MP_E_ARG, "query has NaN or Inf samples");
        const unsigned char *ho = ge->h_io + ge->out_off;
        int32_t err = 0;
        memcpy(&err, ho + (size_t)nq * 16, sizeof err);
        if (err) return fail(MP_E_TIMEOUT, "a tensor-core wait timed out on the device; results are invalid");
        memcpy(out_dist, ho, (size_t)nq * 8);
        memcpy(out_idx, ho + (size_t)nq * 8, (size_t)nq * 8);
        return MP_OK;
    }

    CUDA_TRY(cudaMemcpyAsync(dq, query, (size_t)n * es, cudaMemcpyHostToDevice, st));
    rc = join_device(ctx, d, s, dq, dtype, n, m, dd, di, st, base + qbytes + 2 * obytes, kern, true, corr);
    if (rc) return rc;
    // The query is checked for NaN and Inf here, while the device joins it.
    // A join of such samples is wasted but harmless: the kernels take every
    // index from the launch geometry or from valid chunks, never from sample
    // values, and the finalisation's re-scoring drops NaN scores before its
    // lane reductions, so its branches stay warp-uniform. Nothing is copied
    // out unless the check passes.
    if (!host_all_finite(query, dtype, n)) {
        cudaStreamSynchronize(st);
        return fail(MP_E_ARG, "query has NaN or Inf samples");
    }
    CUDA_TRY(cudaMemcpyAsync(out_dist, dd, nq * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(out_idx, di, nq * 8, cudaMemcpyDeviceToHost, st));
    int32_t err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (err) return fail(MP_E_TIMEOUT, "a tensor-core wait timed out on the device; results are invalid");
    return MP_OK;
}

int mp_ab_join(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
               double *out_dist, int64_t *out_idx)
{
    return ab_join_host(ctx, dict, query, dtype, n, m, out_dist, out_idx, false);
}

int mp_ab_join_corr(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
                    double *out_corr, int64_t *out_idx)
{
    return ab_join_host(ctx, dict, query, dtype, n, m, out_corr, out_idx, true);
}

int mp_window_stats(mp_ctx *ctx, const void *d_x, int32_t dtype, int64_t n, int32_t m, double *d_mean,
                    double *d_invstd, uint8_t *d_const, void *stream)
{
    g_err.clear();
    if (!ctx || !d_x || !d_mean || !d_invstd || !d_const) return fail(MP_E_ARG, "null argument");
    if (dtype != MP_F32 && dtype != MP_F64) return fail(MP_E_ARG, "unknown dtype");
    if (m < kMinM || m > kMaxM || n < m) return fail(MP_E_ARG, "bad n/m (m in [%d, %d], n >= m)", kMinM, kMaxM);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    // the context's stream is shared with the synchronous joins (which may be
    // capturing it into a graph): enqueue on it under the context lock
    std::unique_lock<std::mutex> lk(ctx->mu, std::defer_lock);
    if (st == ctx->stream) lk.lock();
    if (dtype == MP_F64)
        CUDA_TRY(launch_window_stats<double>((const double *)d_x, n, m, d_mean, d_invstd, d_const, nullptr, nullptr,
                                             st));
    else
        CUDA_TRY(launch_window_stats<float>((const float *)d_x, n, m, d_mean, d_invstd, d_const, nullptr, nullptr,
                                            st));
    return MP_OK;
}

int mp_submit(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
              double *out_dist, int64_t *out_idx, uint64_t *ticket)
{
    g_err.clear();
    int rc = check_join_args(ctx, dict, query, dtype, n, m);
    if (rc) return rc;
    if (!out_dist || !out_idx || !ticket) return fail(MP_E_ARG, "null output");
    if (!host_all_finite(query, dtype, n)) return fail(MP_E_ARG, "query has NaN or Inf samples");
    mp_dict *d = const_cast<mp_dict *>(dict);
    auto r = std::make_shared<Request>();
    r->dict = d;
    r->dtype = dtype;
    r->n = n;
    r->m = m;
    const int64_t nq = n - m + 1;
    r->out_dist = out_dist;
    r->out_idx = out_idx;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        CUDA_TRY(cudaSetDevice(ctx->device));
        DictStats *s;
        rc = get_stats(ctx, d, m, &s);
        if (rc) return rc;
        r->bytes = request_bytes(ctx, *r, s);
    }
    if (r->bytes > ctx->mem_budget) return fail(MP_E_NOMEM, "request needs %zu bytes, budget %zu", r->bytes,
                                                 ctx->mem_budget);
    r->stage_bytes = std::max((size_t)n * dtype_size(dtype), (size_t)nq * 16);
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if ((int64_t)ctx->pending.size() >= ctx->cfg.max_pending)
            return fail(MP_E_BUSY, "%zu requests wait for admission (max_pending %d)", ctx->pending.size(),
                        ctx->cfg.max_pending);
        r->h_stage = pinned_take(ctx, r->stage_bytes);
    }
    if (!r->h_stage) return fail(MP_E_NOMEM, "pinned staging of %zu bytes", r->stage_bytes);
    memcpy(r->h_stage, query, (size_t)n * dtype_size(dtype));
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if ((int64_t)ctx->pending.size() >= ctx->cfg.max_pending) {  // filled while the query was copied
            pinned_give(ctx, r->h_stage, r->stage_bytes);
            return fail(MP_E_BUSY, "%zu requests wait for admission (max_pending %d)", ctx->pending.size(),
                        ctx->cfg.max_pending);
        }
        d->refs.fetch_add(1);
        r->ticket = ctx->next_ticket++;
        r->t_submit = now_s();
        ctx->tickets[r->ticket] = r;
        ctx->pending.push_back(r);
        *ticket = r->ticket;
    }
    ctx->scv.notify_all();
    return MP_OK;
}

int mp_poll(mp_ctx *ctx, uint64_t ticket, int32_t *state, double *latency_s)
{
    g_err.clear();
    if (!ctx || !state) return fail(MP_E_ARG, "null argument");
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(MP_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request &r = *it->second;
    *state = r.state;
    if (r.state != MP_PENDING) {
        if (latency_s) *latency_s = r.t_done - r.t_submit;
        ctx->tickets.erase(it);
    }
    return MP_OK;
}

int mp_plan_join(mp_ctx *ctx, const mp_dict *dict, int32_t dtype, int64_t n, int32_t m, mp_join_plan *plan)
{
    g_err.clear();
    if (!plan) return fail(MP_E_ARG, "null argument");
    const char dummy = 0;  // the plan reads no query
    int rc = check_join_args(ctx, dict, &dummy, dtype, n, m);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    mp_dict *d = const_cast<mp_dict *>(dict);
    DictStats *s;
    rc = get_stats(ctx, d, m, &s);
    if (rc) return rc;
    const int64_t nq = n - m + 1;
    *plan = mp_join_plan{};
    plan->kernel = s->n_windows > 0 ? resolve_kernel(ctx, dtype, m, s, nq) : MP_KERNEL_PLAIN;
    if (s->n_windows == 0) return MP_OK;  // nothing runs: +inf and -1 are written directly
    const bool seeds = tc_seeds_pay(s, dtype, nq);  // as join_device decides for the plain form
    const Geometry geo = join_plain_geometry(ctx, d, s, dtype, nq, m, seeds);
    const int64_t crow = plain_chunk_rows(d, dtype, nq, m, seeds);
    plan->column_groups = geo.n_groups;
    plan->spans = grouping_spans(s, geo.n_groups);
    plan->row_chunks = (nq + crow - 1) / crow;
    plan->tc_seeds = seeds && plan->kernel == MP_KERNEL_PLAIN ? 1 : 0;
    plan->workspace_bytes = (int64_t)join_ws_bytes(ctx, d, s, dtype, n, m);
    return MP_OK;
}

int mp_profile(mp_ctx *ctx, int32_t enable)
{
    g_err.clear();
    if (!ctx) return fail(MP_E_ARG, "null ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->profiling = enable != 0;
    return MP_OK;
}

int mp_profile_read(mp_ctx *ctx, double *ms, int64_t *launches, int32_t reset)
{
    g_err.clear();
    if (!ctx) return fail(MP_E_ARG, "null ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    for (auto &mk : ctx->marks) {
        CUDA_TRY(cudaEventSynchronize(mk.t1));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, mk.t0, mk.t1));
        ctx->prof_ms[mk.phase] += t;
        ctx->prof_n[mk.phase] += 1;
        ctx->ev_pool.push_back(mk.t0);
        ctx->ev_pool.push_back(mk.t1);
    }
    ctx->marks.clear();
    for (int k = 0; k < MP_PHASE_COUNT; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_n[k];
        if (reset) {
            ctx->prof_ms[k] = 0;
            ctx->prof_n[k] = 0;
        }
    }
    return MP_OK;
}

int mp_test_hook(mp_ctx *ctx, int32_t hook, int64_t value)
{
    g_err.clear();
    if (!ctx || value < 0) return fail(MP_E_ARG, "bad argument");
    if (hook == MP_HOOK_FAIL_ALLOC) {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->hook_fail_alloc = value;
    } else if (hook == MP_HOOK_TC_WAIT) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->hook_tc_wait = (long long)value;
        graphs_clear(ctx);  // a captured join carries the wait bound it was launched with
    } else {
        return fail(MP_E_ARG, "unknown hook %d", hook);
    }
    return MP_OK;
}

int mp_counters(mp_ctx *ctx, int64_t *values, int32_t reset)
{
    g_err.clear();
    if (!ctx || !values) return fail(MP_E_ARG, "null argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    static_assert(MP_COUNTER_COUNT == kFinCounters, "counter layout");
    unsigned long long h[kFinCounters];
    CUDA_TRY(cudaDeviceSynchronize());  // every stream's joins, serving batches included
    CUDA_TRY(cudaMemcpy(h, ctx->d_counters, sizeof h, cudaMemcpyDeviceToHost));
    for (int k = 0; k < kFinCounters; ++k) values[k] = (int64_t)h[k];
    if (reset) CUDA_TRY(cudaMemset(ctx->d_counters, 0, sizeof h));
    return MP_OK;
}

int mp_drain(mp_ctx *ctx, double timeout_s)
{
    g_err.clear();
    if (!ctx) return fail(MP_E_ARG, "null ctx");
    const double t_end = now_s() + timeout_s;
    while (true) {
        {
            std::lock_guard<std::mutex> lk(ctx->smu);
            // admitted requests are counted from admission to completion; a
            // batch being launched is in neither the queue nor the list
            if (ctx->pending.empty() && ctx->inflight.empty() && ctx->n_inflight_reqs == 0) return MP_OK;
        }
        if (now_s() > t_end) return fail(MP_E_TIMEOUT, "requests still in flight after %.3f s", timeout_s);
        ctx->scv.notify_all();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// e_max and discords (Sec. 2.1 and Sec. 3.3, on top of the join)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Streaming join (Sec. 1's online use: arriving data joined against a resident
// normal dictionary). The stream keeps the last m - 1 samples; each append
// joins [kept | new] on the device and returns the windows that end in the new
// samples.
// ---------------------------------------------------------------------------
struct mp_stream {
    mp_ctx *ctx;
    const mp_dict *dict;
    int32_t dtype;
    int32_t m;
    std::vector<unsigned char> tail;  // the last min(m - 1, seen) samples
    int64_t n_seen = 0;               // samples appended so far
};

extern "C" int mp_stream_open(mp_ctx *ctx, const mp_dict *dict, int32_t dtype, int32_t m, mp_stream **out)
{
    g_err.clear();
    if (!ctx || !dict || !out || m < kMinM || m > kMaxM || (dtype != MP_F32 && dtype != MP_F64))
        return fail(MP_E_ARG, "bad argument");
    if (dtype != dict->dtype) return fail(MP_E_ARG, "stream dtype must match the dictionary's");
    mp_stream *st = new mp_stream();
    st->ctx = ctx;
    st->dict = dict;
    st->dtype = dtype;
    st->m = m;
    *out = st;
    return MP_OK;
}

extern "C" int mp_stream_append(mp_stream *st, const void *samples, int64_t n_new, double *out_dist, int64_t *out_idx,
                                int64_t *n_out, int64_t *first_window)
{
    g_err.clear();
    if (!st || !n_out || n_new < 0 || (n_new > 0 && (!samples || !out_dist || !out_idx)))
        return fail(MP_E_ARG, "bad argument");
    const size_t es = dtype_size(st->dtype);
    const int64_t kept = (int64_t)(st->tail.size() / es);
    const int64_t n = kept + n_new;
    *n_out = 0;
    if (first_window) *first_window = std::max<int64_t>(0, st->n_seen - st->m + 1);
    std::vector<unsigned char> buf(st->tail);
    buf.insert(buf.end(), (const unsigned char *)samples, (const unsigned char *)samples + (size_t)n_new * es);
    if (n >= st->m) {
        int rc = ab_join_host(st->ctx, st->dict, buf.data(), st->dtype, n, st->m, out_dist, out_idx, false);
        if (rc) return rc;
        *n_out = n - st->m + 1;
    }
    // keep the last m - 1 samples
    const int64_t keep = std::min<int64_t>(n, st->m - 1);
    st->tail.assign(buf.end() - (ptrdiff_t)(keep * (int64_t)es), buf.end());
    st->n_seen += n_new;
    return MP_OK;
}

extern "C" int mp_stream_submit(mp_stream *st, const void *samples, int64_t n_new, double *out_dist,
                                int64_t *out_idx, uint64_t *ticket, int64_t *n_out, int64_t *first_window)
{
    g_err.clear();
    if (!st || !n_out || !ticket || n_new < 0 || (n_new > 0 && (!samples || !out_dist || !out_idx)))
        return fail(MP_E_ARG, "bad argument");
    const size_t es = dtype_size(st->dtype);
    const int64_t kept = (int64_t)(st->tail.size() / es);
    const int64_t n = kept + n_new;
    *n_out = 0;
    *ticket = 0;
    const int64_t first = std::max<int64_t>(0, st->n_seen - st->m + 1);
    std::vector<unsigned char> buf(st->tail);
    buf.insert(buf.end(), (const unsigned char *)samples, (const unsigned char *)samples + (size_t)n_new * es);
    if (n >= st->m) {
        // a serving request of [kept | new]: batched with the stream's other
        // appends and any other requests; the query is copied at submission
        int rc = mp_submit(st->ctx, st->dict, buf.data(), st->dtype, n, st->m, out_dist, out_idx, ticket);
        if (rc) return rc;
        *n_out = n - st->m + 1;
    }
    if (first_window) *first_window = first;
    const int64_t keep = std::min<int64_t>(n, st->m - 1);
    st->tail.assign(buf.end() - (ptrdiff_t)(keep * (int64_t)es), buf.end());
    st->n_seen += n_new;
    return MP_OK;
}

extern "C" int mp_stream_close(mp_stream *st)
{
    g_err.clear();
    delete st;
    return MP_OK;
}

// ---------------------------------------------------------------------------
// Self-join and dictionary learning (Algorithm 1, Sec. 3.1)
// ---------------------------------------------------------------------------
namespace {
// A device allocation freed at scope exit.
struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
    int alloc(size_t bytes)
    {
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(MP_E_NOMEM, "%zu bytes of device memory", bytes);
        }
        return MP_OK;
    }
};
}  // namespace

// The self-join profile of the series that dictionary d holds as its only
// segment, into device outputs (caller holds ctx->mu).
static int self_join_dev(mp_ctx *ctx, mp_dict *d, int32_t m, int32_t excl, double *dd, int64_t *di)
{
    DictStats *s = nullptr;
    int rc = get_stats(ctx, d, m, &s);
    if (rc) return rc;
    const int64_t n = d->nb, nq = n - m + 1;
    DevBuf nc, scr;
    if ((rc = nc.alloc((size_t)nq * sizeof(int64_t))) || (rc = scr.alloc(next_const_scratch_elems(nq) * 8)))
        return rc;
    CUDA_TRY(launch_next_const(s->cflag, nq, (int64_t *)nc.p, (int64_t *)scr.p, ctx->stream));
    rc = ensure_ws(ctx, join_ws_bytes(ctx, d, s, MP_F32, n, m));
    if (rc) return rc;
    rc = join_device(ctx, d, s, d->d_samples, MP_F32, n, m, dd, di, ctx->stream, (unsigned char *)ctx->ws,
                     MP_KERNEL_PLAIN, true, false, excl, (const int64_t *)nc.p);
    if (rc) return rc;
    int32_t err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, ctx->ws, sizeof err, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (err) return fail(MP_E_TIMEOUT, "a tensor-core wait timed out on the device; results are invalid");
    return MP_OK;
}

static int check_series(mp_ctx *ctx, const void *x, int32_t dtype, int64_t n, int32_t m)
{
    if (!ctx || !x) return fail(MP_E_ARG, "null argument");
    if (dtype != MP_F32) return fail(MP_E_ARG, "the self-join and dictionary learning take float32 samples");
    if (m < kMinM || m > kMaxM) return fail(MP_E_ARG, "m=%d outside [%d, %d]", m, kMinM, kMaxM);
    if (n < m) return fail(MP_E_ARG, "series shorter than m");
    return MP_OK;
}

extern "C" int mp_self_join(mp_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m, int32_t excl,
                            double *out_dist, int64_t *out_idx)
{
    g_err.clear();
    int rc = check_series(ctx, series, dtype, n, m);
    if (rc) return rc;
    if (excl < 1 || !out_dist || !out_idx) return fail(MP_E_ARG, "bad argument");
    const int64_t offs[2] = {0, n};
    mp_dict *d = nullptr;
    rc = mp_dict_load(ctx, series, dtype, offs, 1, &m, 1, &d);
    if (rc) return rc;
    const int64_t nq = n - m + 1;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        DevBuf dd, di;
        if (!(rc = dd.alloc((size_t)nq * 8)) && !(rc = di.alloc((size_t)nq * 8)) &&
            !(rc = self_join_dev(ctx, d, m, excl, (double *)dd.p, (int64_t *)di.p))) {
            if (cudaMemcpy(out_dist, dd.p, (size_t)nq * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(out_idx, di.p, (size_t)nq * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = fail(MP_E_CUDA, "copying the self-join back");
        }
    }
    mp_dict_free(ctx, d);
    return rc;
}

// Merge overlapping intervals [start, end) (sorted by start); returns the samples they cover.
static int64_t merge_intervals(std::vector<std::pair<int64_t, int64_t>> iv, std::vector<std::pair<int64_t, int64_t>> *out)
{
    std::sort(iv.begin(), iv.end());
    out->clear();
    int64_t total = 0;
    for (const auto &x : iv) {
        if (!out->empty() && x.first < out->back().second)
            out->back().second = std::max(out->back().second, x.second);
        else
            out->push_back(x);
    }
    for (const auto &x : *out) total += x.second - x.first;
    return total;
}

extern "C" int mp_learn_dictionary(mp_ctx *ctx, const void *t_b, int32_t dtype, int64_t n_b, int32_t m,
                                   double k_context, int32_t term_kind, double term_value, int32_t max_elements,
                                   int64_t *seg_start, int64_t *seg_len, int32_t *n_segments, double *err_bound,
                                   int64_t *chosen, int32_t *n_chosen)
{
    g_err.clear();
    int rc = check_series(ctx, t_b, dtype, n_b, m);
    if (rc) return rc;
    if (!(k_context >= 1.0) || max_elements < 1 || !seg_start || !seg_len || !n_segments ||
        (term_kind != MP_LEARN_MEMORY && term_kind != MP_LEARN_EMAX))
        return fail(MP_E_ARG, "bad argument");
    const int64_t offs[2] = {0, n_b};
    mp_dict *d = nullptr;
    rc = mp_dict_load(ctx, t_b, dtype, offs, 1, &m, 1, &d);
    if (rc) return rc;
    const int64_t nq = n_b - m + 1;
    const int32_t half = m / 2;
    const int64_t pad = (int64_t)std::floor((k_context - 1.0) * m / 2.0);
    std::vector<std::pair<int64_t, int64_t>> elems, merged;
    std::vector<int64_t> picks;
    float smax_v = INFINITY;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaStream_t st = ctx->stream;
        DevBuf P, I, S, ex, key;
        DictStats *s = nullptr;
        if ((rc = P.alloc((size_t)nq * 8)) || (rc = I.alloc((size_t)nq * 8)) || (rc = S.alloc((size_t)nq * 4)) ||
            (rc = ex.alloc((size_t)nq)) || (rc = key.alloc(16)))
            goto done;
        // line 3: the self-join matrix profile P_B, trivial matches |g - i| < ceil(m/2) left out
        if ((rc = self_join_dev(ctx, d, m, (m + 1) / 2, (double *)P.p, (int64_t *)I.p))) goto done;
        if ((rc = get_stats(ctx, d, m, &s))) goto done;
        if (cudaMemsetAsync(S.p, 0, (size_t)nq * 4, st) != cudaSuccess ||
            cudaMemsetAsync(ex.p, 0, (size_t)nq, st) != cudaSuccess) {
            rc = fail(MP_E_CUDA, "clearing the learning state");
            goto done;
        }
        for (int32_t it = 0; it < max_elements; ++it) {
            // lines 7-11: j = argmin (P_B - S) outside the taken elements' zones
            unsigned long long best = ~0ull;
            if (launch_learn_argmin((const double *)P.p, (const float *)S.p, (const uint8_t *)ex.p, nq,
                                    (unsigned long long *)key.p, ctx->sm_count, st) != cudaSuccess ||
                cudaMemcpyAsync(&best, key.p, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = fail(MP_E_CUDA, "argmin of the processed profile");
                goto done;
            }
            if (best == ~0ull) break;  // every window is taken or excluded
            const int64_t j = (int64_t)(best & 0xffffffffull);
            // line 12: add T_B[j : j + m] with its context (k m samples in all)
            picks.push_back(j);
            elems.emplace_back(std::max<int64_t>(0, j - pad), std::min<int64_t>(n_b, j + m + pad));
            // line 10 for the next iterations: the zone [j - m/2, j + m/2)
            const int64_t z0 = std::max<int64_t>(0, j - half), z1 = std::min<int64_t>(nq, j + half);
            // lines 15-19: S = S' or ElementwiseMin(S, S'), S' the distance profile of window j
            uint32_t smax = 0;
            if ((z1 > z0 && cudaMemsetAsync((uint8_t *)ex.p + z0, 1, (size_t)(z1 - z0), st) != cudaSuccess) ||
                launch_learn_profile((const float *)d->d_samples, nq, m, (const Split<float> *)s->ms,
                                     (const float4 *)s->rs, s->cflag, j, (float *)S.p, it == 0,
                                     (uint32_t *)key.p + 2, ctx->sm_count, st) != cudaSuccess ||
                cudaMemcpyAsync(&smax, (uint32_t *)key.p + 2, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = fail(MP_E_CUDA, "distance profile of the new element");
                goto done;
            }
            smax_v = learn_key_float(smax);
            // lines 13-14: the terminal condition
            const int64_t total = merge_intervals(elems, &merged);
            if (term_kind == MP_LEARN_MEMORY && (double)total >= term_value) break;
            if (term_kind == MP_LEARN_EMAX && (double)smax_v <= term_value) break;
        }
        merge_intervals(elems, &merged);
    }
done:
    mp_dict_free(ctx, d);
    if (rc) return rc;
    *n_segments = (int32_t)merged.size();
    for (size_t k = 0; k < merged.size(); ++k) {
        seg_start[k] = merged[k].first;
        seg_len[k] = merged[k].second - merged[k].first;
    }
    if (err_bound) *err_bound = (double)smax_v;
    if (n_chosen) *n_chosen = (int32_t)picks.size();
    if (chosen)
        for (size_t k = 0; k < picks.size(); ++k) chosen[k] = picks[k];
    return MP_OK;
}

extern "C" int mp_emax(mp_ctx *ctx, const mp_dict *dict, const void *t_b, int32_t dtype, int64_t n_b, int32_t m,
                       double *e_max, int64_t *argmax)
{
    g_err.clear();
    if (!e_max) return fail(MP_E_ARG, "null output");
    const int64_t nq = n_b - m + 1;
    if (nq <= 0) return fail(MP_E_ARG, "series shorter than m");
    std::vector<double> dist((size_t)nq);
    std::vector<int64_t> idx((size_t)nq);
    int rc = mp_ab_join(ctx, dict, t_b, dtype, n_b, m, dist.data(), idx.data());
    if (rc) return rc;
    // e_max = max over the windows of T_B of NNDist(window, D_{B,m})
    int64_t best = 0;
    for (int64_t i = 1; i < nq; ++i)
        if (dist[i] > dist[best]) best = i;
    *e_max = dist[best];
    if (argmax) *argmax = best;
    return MP_OK;
}

extern "C" int mp_top_discords(const double *profile, int64_t n, int32_t k, int64_t excl, double e_max, int64_t *idx,
                               double *val, int32_t *n_found, int32_t *top1_certified)
{
    g_err.clear();
    if (!profile || !idx || !val || n < 0 || k < 0 || excl < 0) return fail(MP_E_ARG, "bad argument");
    // repeatedly take the largest finite value not excluded; exclude +-excl around it
    std::vector<uint8_t> blocked((size_t)n, 0);
    int32_t found = 0;
    for (int32_t j = 0; j < k; ++j) {
        int64_t b = -1;
        for (int64_t i = 0; i < n; ++i)
            if (!blocked[i] && std::isfinite(profile[i]) && (b < 0 || profile[i] > profile[b])) b = i;
        if (b < 0) break;
        idx[j] = b;
        val[j] = profile[b];
        ++found;
        for (int64_t i = std::max<int64_t>(0, b - excl); i <= std::min<int64_t>(n - 1, b + excl); ++i) blocked[i] = 1;
    }
    if (n_found) *n_found = found;
    if (top1_certified) {
        // Guarantee 2: the true profile lies in [P_hat - e_max, P_hat], so a
        // lead larger than e_max over every other candidate is certain.
        double runner_up = -INFINITY;
        if (found >= 1)
            for (int64_t i = 0; i < n; ++i)
                if (std::llabs(i - idx[0]) > excl && std::isfinite(profile[i])) runner_up = std::max(runner_up, profile[i]);
        *top1_certified = (found >= 1 && e_max >= 0 && val[0] - runner_up > e_max) ? 1 : 0;
    }
    return MP_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
static void tune_load(mp_ctx *ctx, const char *path)
{
    ctx->tune_path = path;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        TuneKey k;
        TuneVal v;
        if (sscanf(line, "{\"dtype\": %d, \"m\": %d, \"wlog\": %d, \"qlog\": %d, \"kernel\": %d, \"groups\": %d, \"ms\": %lf",
                   &k.dtype, &k.m, &k.wlog, &k.qlog, &v.kernel, &v.groups, &v.ms) == 7 &&
            v.kernel >= MP_KERNEL_PLAIN && v.kernel <= MP_KERNEL_TC_BF16 && v.groups >= 1)
            ctx->tune[k] = v;  // a later line overrides an earlier one
    }
    fclose(f);
}

static void tune_save(const mp_ctx *ctx, const TuneKey &k, const TuneVal &v)
{
    if (ctx->tune_path.empty()) return;
    FILE *f = fopen(ctx->tune_path.c_str(), "a");
    if (!f) return;
    fprintf(f,
            "{\"dtype\": %d, \"m\": %d, \"wlog\": %d, \"qlog\": %d, \"kernel\": %d, \"groups\": %d, \"ms\": %.4f, "
            "\"tolerance\": %.3g}\n",
            k.dtype, k.m, k.wlog, k.qlog, v.kernel, v.groups, v.ms, v.tolerance);
    fclose(f);
}

extern "C" int mp_autotune(mp_ctx *ctx, const mp_dict *dict, int32_t m, int64_t n, double tolerance,
                           int32_t *kernel_out, int32_t *groups_out, double *ms_out)
{
    g_err.clear();
    if (!ctx || !dict) return fail(MP_E_ARG, "null argument");
    if (m < kMinM || m > kMaxM || n < m) return fail(MP_E_ARG, "bad n/m (m in [%d, %d], n >= m)", kMinM, kMaxM);
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    mp_dict *d = const_cast<mp_dict *>(dict);
    DictStats *s;
    int rc = get_stats(ctx, d, m, &s);
    if (rc) return rc;
    if (s->n_windows == 0) return fail(MP_E_ARG, "the dictionary has no window of length %d", m);
    const int64_t nq = n - m + 1;
    const int dtype = d->dtype;
    const size_t esz = dtype_size(dtype);
    // synthetic query of length n: the dictionary's samples repeated
    void *dq = nullptr, *dout = nullptr;
    if (cudaMalloc(&dq, (size_t)n * esz) != cudaSuccess || cudaMalloc(&dout, (size_t)nq * 16) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dq);
        return fail(MP_E_NOMEM, "autotune buffers");
    }
    for (int64_t o = 0; o < n; o += d->nb)
        CUDA_TRY(cudaMemcpyAsync((char *)dq + o * esz, d->d_samples, (size_t)std::min<int64_t>(d->nb, n - o) * esz,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
    double *dd = (double *)dout;
    int64_t *di = (int64_t *)((char *)dout + (size_t)nq * 8);
    // candidates: the plain form at several column-group counts, then the
    // tensor-core forms: every form picks exactly (near ties re-scored within
    // its error bound), so each meets any tolerance the plain form meets
    struct Cand {
        int kernel, groups;
    };
    std::vector<Cand> cands;
    const int64_t max_g = std::max<int64_t>(1, s->n_windows / 1024);
    for (int g : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32})
        if (g <= max_g) cands.push_back(Cand{MP_KERNEL_PLAIN, g});
    if (dtype == MP_F32 && tc_supported(0, m)) cands.push_back(Cand{MP_KERNEL_TC_BF16X3, 1});
    if (dtype == MP_F32 && tc_supported(1, m)) cands.push_back(Cand{MP_KERNEL_TC_TF32, 1});
    const int saved_kernel = ctx->kernel;
    // the workspace of the largest candidate: each forced grouping with its left seeds, and every form
    size_t wsb = join_ws_bytes(ctx, d, s, dtype, n, m);
    for (const Cand &c : cands) {
        if (c.kernel != MP_KERNEL_PLAIN) continue;
        const size_t left = dtype == MP_F32 ? (size_t)grouping_spans(s, c.groups) *
                                                  left_ld_for(plain_chunk_rows(d, dtype, nq, m, true)) * 4
                                            : 0;
        wsb = std::max(wsb, join_ws_layout(nq, dtype, c.groups, 0, join_seed_bytes(d, dtype, nq, m, true),
                                           kNearSlotsPlain, left)
                                .total);
    }
    rc = ensure_ws(ctx, wsb);
    if (rc) {
        cudaFree(dq);
        cudaFree(dout);
        return rc;
    }
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    Cand best{MP_KERNEL_PLAIN, 1};
    double best_ms = 1e300;
    for (const Cand &c : cands) {
        ctx->kernel = c.kernel;
        ctx->force_groups = c.kernel == MP_KERNEL_PLAIN ? c.groups : 0;
        double t_min = 1e300;
        for (int rep = 0; rep < 4 && rc == MP_OK; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            rc = join_device(ctx, d, s, dq, dtype, n, m, dd, di, ctx->stream, (unsigned char *)ctx->ws, c.kernel);
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(MP_E_CUDA, "autotune run failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t_min = std::min(t_min, (double)ms);  // the first run warms up
        }
        if (rc) break;
        if (t_min < best_ms) {
            best_ms = t_min;
            best = c;
        }
    }
    ctx->kernel = saved_kernel;
    ctx->force_groups = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dq);
    cudaFree(dout);
    if (rc) return rc;
    const TuneKey key{dtype, m, ilog2(s->n_windows), ilog2(nq)};
    const TuneVal val{best.kernel, best.groups, best_ms, tolerance};
    ctx->tune[key] = val;
    graphs_clear(ctx);  // cached graphs carry the launch geometry of the old choice
    tune_save(ctx, key, val);
    if (kernel_out) *kernel_out = best.kernel;
    if (groups_out) *groups_out = best.groups;
    if (ms_out) *ms_out = best_ms;
    return MP_OK;
}

// ---------------------------------------------------------------------------
// Join without device allocation
//
// Some callers cannot allocate device memory while they serve a request:
// services that reserve all of the GPU's memory up front and forbid
// allocation on the request path (cudaMalloc and cudaFree can synchronise the
// device and add latency jitter), and host applications that own the device
// allocator (a caching allocator or memory pool whose accounting a foreign
// cudaMalloc would break). mp_ab_join_noalloc serves them: its scratch lives
// in the fixed array below, which every GPU that loads this library holds
// until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocMaxWindows = (int64_t)1 << 19;   // query windows per call
constexpr int64_t kNoAllocMaxPartials = (int64_t)1 << 20;  // column groups x query windows
constexpr int64_t kNoAllocMaxSpans = (int64_t)1 << 16;     // runs of dictionary windows
constexpr size_t kNoAllocMeanOff = 0;
constexpr size_t kNoAllocInvOff = kNoAllocMeanOff + kNoAllocMaxWindows * sizeof(double);
constexpr size_t kNoAllocFlagOff = kNoAllocInvOff + kNoAllocMaxWindows * sizeof(double);
constexpr size_t kNoAllocRsOff = kNoAllocFlagOff + kNoAllocMaxWindows;
constexpr size_t kNoAllocMsOff = kNoAllocRsOff + kNoAllocMaxWindows * sizeof(float4);
constexpr size_t kNoAllocPartOff = kNoAllocMsOff + kNoAllocMaxWindows * sizeof(Split<float>);
constexpr int kNoAllocNearSlots = 2;                        // near-tie record slots per (group, window)
constexpr size_t kNoAllocNearOff = kNoAllocPartOff + kNoAllocMaxPartials * sizeof(Partial<float>);
constexpr size_t kNoAllocSpanOff = kNoAllocNearOff + kNoAllocMaxPartials * (kNoAllocNearSlots + 1) * sizeof(NearSlot);
constexpr size_t kNoAllocGroupOff = kNoAllocSpanOff + kNoAllocMaxSpans * sizeof(Span);
constexpr size_t kNoAllocBytes = kNoAllocGroupOff + (kNoAllocMaxSpans + 1) * sizeof(int32_t);
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

// About 56 MB: statistics of 2^19 query windows, 2^20 partial results with
// their near-tie records, and 2^16 spans. Host code must not use this name as
// an address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static unsigned char *g_noalloc_dev[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on `device` (which must be current).
// Resolved once per device, at that device's first call.
static int noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(MP_E_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(MP_E_CUDA, "cudaGetSymbolAddress of the no-allocation scratch: %s", cudaGetErrorString(e));
        g_noalloc_dev[device] = (unsigned char *)p;
    }
    *out = g_noalloc_dev[device];
    return MP_OK;
}

// The dictionary's valid windows cut into column groups on the device, as
// get_grouping cuts them on the host: in the order of the segments, windows
// [k T, (k + 1) T) of that order form group k, and a span never crosses a
// segment or a group. One CTA of 1024 threads, each taking a run of
// segments: block scans give each segment's first window in that order and its
// first span. Writes spans[0 .. total) and gstart[0 .. n_groups].
__device__ int64_t block_excl_scan(int64_t v, int64_t *tmp, int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) tmp[lane] = w;  // inclusive sums per warp
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? tmp[warp - 1] : 0) + x - v;
    *total = tmp[nw - 1];
    __syncthreads();  // tmp is reused by the next scan
    return before;
}

__global__ void __launch_bounds__(1024) k_noalloc_groups(const Span *seg, int32_t n_seg, int64_t T, int32_t n_groups,
                                                         int32_t n_spans_total, Span *spans, int32_t *gstart)
{
    __shared__ int64_t tmp[32];
    const int per = (n_seg + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min(n_seg, (int)threadIdx.x * per), s1 = min(n_seg, s0 + per);
    for (int k = threadIdx.x; k <= n_groups; k += blockDim.x) gstart[k] = n_spans_total;
    int64_t cols = 0;
    for (int s = s0; s < s1; ++s) cols += seg[s].ncols;
    int64_t tot;
    const int64_t cum0 = block_excl_scan(cols, tmp, &tot);
    // spans of each segment: one per group its chunks meet (the cut of get_grouping)
    int64_t pieces = 0, cum = cum0;
    for (int s = s0; s < s1; ++s) {
        pieces += segment_pieces(cum, seg[s].ncols, T);
        cum += seg[s].ncols;
    }
    int64_t idx = block_excl_scan(pieces, tmp, &tot);  // also orders the gstart initialisation before the writes
    cum = cum0;
    // the group of the previous segment's last chunk (-1 before the first segment)
    int64_t prev_k = -1;
    if (s0 > 0 && s0 < s1) {
        const int64_t n = seg[s0 - 1].ncols, c = cum0 - n;
        prev_k = n > 0 ? (c + (n - 1) / kChunk * kChunk) / T : -1;
    }
    for (int s = s0; s < s1; ++s) {
        const Span sg = seg[s];
        const int64_t nch = (sg.ncols + kChunk - 1) / kChunk;
        for (int64_t j = 0; j < nch;) {
            const int64_t k = (cum + j * kChunk) / T;
            const int64_t j_end = min(nch, chunk_at_or_after(cum, (k + 1) * T));
            spans[idx] = Span{sg.g0 + j * kChunk, (int32_t)(min((int64_t)sg.ncols, j_end * kChunk) - j * kChunk), 0};
            if (j > 0 || prev_k < k) gstart[k] = (int32_t)idx;  // group k's first chunk
            prev_k = k;
            ++idx;
            j = j_end;
        }
        cum += sg.ncols;
    }
}

extern "C" int mp_ab_join_noalloc(mp_ctx *ctx, const mp_dict *dict, const void *d_query, int32_t dtype, int64_t n,
                                  int32_t m, double *d_out_dist, int64_t *d_out_idx, void *stream)
{
    g_err.clear();
    int rc = check_join_args(ctx, dict, d_query, dtype, n, m);
    if (rc) return rc;
    if (!d_out_dist || !d_out_idx) return fail(MP_E_ARG, "null output");
    if (dtype != MP_F32) return fail(MP_E_ARG, "the no-allocation join takes float32 samples only");
    const int64_t nq = n - m + 1;
    if (nq > kNoAllocMaxWindows)
        return fail(MP_E_ARG, "query of %lld windows exceeds the no-allocation limit of %lld windows (n - m + 1)",
                    (long long)nq, (long long)kNoAllocMaxWindows);
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->mu);
    mp_dict *d = const_cast<mp_dict *>(dict);
    auto it = d->stats.find(m);
    if (it == d->stats.end())
        return fail(MP_E_ARG, "dictionary statistics for m=%d are not resident; list m when loading the dictionary "
                              "(computing them would allocate)", m);
    DictStats *s = it->second.get();
    unsigned char *base = nullptr;
    rc = noalloc_scratch(ctx->device, &base);
    if (rc) return rc;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    const float *a = (const float *)d_query;
    double *mean_a = (double *)(base + kNoAllocMeanOff);
    double *inv_a = (double *)(base + kNoAllocInvOff);
    uint8_t *cf_a = (uint8_t *)(base + kNoAllocFlagOff);
    float4 *rs_a = (float4 *)(base + kNoAllocRsOff);
    Split<float> *ms_a = (Split<float> *)(base + kNoAllocMsOff);
    Partial<float> *part = (Partial<float> *)(base + kNoAllocPartOff);
    CUDA_TRY(launch_window_stats<float>(a, n, m, mean_a, inv_a, cf_a, rs_a, ms_a, st));
    int n_groups = 0;
    NearRec near{};
    Span *d_spans = (Span *)(base + kNoAllocSpanOff);
    int32_t *d_gstart = (int32_t *)(base + kNoAllocGroupOff);
    if (s->n_windows > 0) {
        Geometry geo = plain_geometry(ctx, nq, s->n_windows, kPlainRowsPerLane, MP_F32, m,
                                      (int64_t)s->seg_spans.size());
        geo.n_groups = (int)std::max<int64_t>(1, std::min<int64_t>(geo.n_groups, kNoAllocMaxPartials / nq));
        // the cut into column groups of get_grouping, built on the device from
        // the dictionary's resident segment table (no host copy per call)
        const int64_t target = group_target(s->n_windows, geo.n_groups);
        const int64_t n_spans = grouping_spans(s, geo.n_groups);
        if (n_spans > kNoAllocMaxSpans)
            return fail(MP_E_ARG, "dictionary needs %lld spans, above the no-allocation limit of %lld",
                        (long long)n_spans, (long long)kNoAllocMaxSpans);
        k_noalloc_groups<<<1, 1024, 0, st>>>(s->d_seg_spans, (int32_t)s->seg_spans.size(), target, geo.n_groups,
                                             (int32_t)n_spans, d_spans, d_gstart);
        CUDA_TRY(cudaGetLastError());
        PlainLaunch L;
        L.nq = nq;
        L.m = m;
        L.n_row_blocks = geo.n_row_blocks;
        L.n_groups = geo.n_groups;
        L.warps = geo.warps;
        near.rec = (NearSlot *)(base + kNoAllocNearOff);
        near.ld = nq;
        near.S = kNoAllocNearSlots;
        near.rho = kNearRhoFP32;
        CUDA_TRY(launch_plain<float>(L, a, n, rs_a, ms_a, (const float *)d->d_samples, d->nb, (const float4 *)s->rs,
                                     (const Split<float> *)s->ms, d_spans, d_gstart, part, nullptr, 0, nullptr, 0,
                                     near, st));
        n_groups = geo.n_groups;
    }
    // with no dictionary window (n_groups = 0, g_first = -1) this writes +inf / -1
    FinalizeParams<float> f =
        fin_params<float>(ctx, nq, m, n_groups, part, a, rs_a, ms_a, cf_a, d, s, d_out_dist, d_out_idx);
    f.near = near;
    f.cspans = d_spans;
    f.cgroup_start = d_gstart;
    CUDA_TRY(launch_finalize<float>(f, st));
    return MP_OK;
}

/*
 * mpdict -- dictionary AB-join of time series on one NVIDIA GB300 (sm_103a).
 *
 * The library computes the approximate inter-time-series similarity join of
 * Yeh et al., "Error-bounded Approximate Time Series Joins Using Compact
 * Dictionary Representations of Time Series" (SDM 2022):
 *
 *   P_hat[i] = min over dictionary windows g of d(T_A[i : i+m], D_B[g : g+m])
 *   I_hat[i] = the g that attains it
 *
 * for every length-m window i of a query series T_A (Def. 2, Def. 3), where d
 * is the z-normalised Euclidean distance (Sec. 2.1) and the dictionary windows
 * slide inside each dictionary element (segment) and never cross a segment
 * boundary (Def. 8). This is Algorithm 2 (Sec. 3.2): the profile starts at
 * +inf and each segment's 1NN join is merged in by an element-wise minimum.
 * The inputs follow the problem statement (Sec. 2.1): the query T_A, the
 * dictionary D_B and the window length m.
 *
 * Conventions shared by every call:
 *   - Indices are 0-based (the paper's are 1-based).
 *   - The neighbour index is the global window index g: the start offset of
 *     the window in the concatenated segment buffer. Its segment s is the one
 *     with seg_offsets[s] <= g < seg_offsets[s+1].
 *   - The standard deviation is the population one (divide by m), so
 *     0 <= d <= 2 sqrt(m).
 *   - A window whose m samples all compare equal is constant. It normalises
 *     to the zero vector, so d(constant, non-constant) = sqrt(m) and
 *     d(constant, constant) = 0 (the paper leaves this case open).
 *   - On equal distances the lowest g wins.
 *   - A dictionary with no window of length m (every segment shorter than m)
 *     is not an error: every row gets +inf and index -1, the initial value of
 *     Algorithm 2.
 *   - Query and dictionary must have the same sample type. F32 data is joined
 *     in FP32 arithmetic with FP64 window statistics; F64 data in FP64.
 *     Products of centred F32 samples must stay within float32 range: with
 *     sample spreads near 1e17 or more they can overflow, and the distances
 *     and indices of the windows concerned are then unspecified.
 *
 * Errors: every call returns MP_OK (0) or a negative MP_E_* code and, on
 * error, leaves a message for mp_last_error(). Invalid arguments (null
 * pointers, m outside [4, 8192], n < m, NaN or Inf samples, unsorted offsets,
 * unknown dtype) give MP_E_ARG and change nothing. A CUDA failure gives
 * MP_E_CUDA. Every call that takes a window length accepts 4 <= m <= 8192.
 *
 * Threads: a context may be used from several host threads; calls on one
 * context are serialised internally. Distinct contexts are independent.
 */
#ifndef MPDICT_H
#define MPDICT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MP_OK 0
#define MP_E_ARG (-1)      /* invalid argument */
#define MP_E_NOMEM (-2)    /* device or host allocation failed, or request larger than the memory budget */
#define MP_E_CUDA (-3)     /* a CUDA call failed */
#define MP_E_NOTFOUND (-4) /* unknown ticket */
#define MP_E_BUSY (-5)     /* object still referenced by requests in flight */
#define MP_E_TIMEOUT (-6)  /* a bounded wait ran out */
#define MP_E_INTERNAL (-7) /* a device-side consistency check failed */

/* sample types */
#define MP_F32 0
#define MP_F64 1

/* join forms (mp_config.kernel, mp_set_kernel) */
#define MP_KERNEL_AUTO 0      /* the autotuner's choice for (m, dictionary size, dtype) */
#define MP_KERNEL_PLAIN 1     /* diagonal recurrence on the FP32 (F64 data: FP64) pipes */
#define MP_KERNEL_TC_BF16X3 2 /* tcgen05 Hankel tiles, split-BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulation */
#define MP_KERNEL_TC_TF32 3   /* tcgen05 Hankel tiles, one TF32 product, FP32 accumulation */
#define MP_KERNEL_TC_BF16 4   /* tcgen05 Hankel tiles, one BF16 product, FP32 accumulation */
/* Every form picks each row's window exactly: the join kernels keep an
 * approximate score per 16-window chunk and record every chunk that comes
 * within the form's error of the best (the tensor-core forms bound that error
 * from their operands' rounding), and the finalisation re-scores those chunks
 * and recomputes the chosen pair's distance from its definition. The forms
 * differ in speed, and in how many chunks they leave to re-score. */

/* request states (mp_poll) */
#define MP_PENDING 0
#define MP_DONE 1
#define MP_FAILED 2

typedef struct mp_ctx mp_ctx;
typedef struct mp_dict mp_dict;
typedef struct mp_stream mp_stream;

/* Context configuration. Fill with mp_config_default() and override fields. */
typedef struct mp_config {
    int32_t device;        /* CUDA device ordinal */
    int32_t kernel;        /* MP_KERNEL_*; F64 data always uses MP_KERNEL_PLAIN */
    int32_t max_inflight;  /* serving: requests whose work may be on the device at once */
    int32_t max_batch;     /* serving: requests merged into one persistent launch */
    size_t mem_budget;     /* serving: device bytes that admitted requests may hold; 0 = half the free memory at init */
    const char *tune_cache;/* autotuner cache file (JSON lines, see mp_autotune), or NULL for none */
    int32_t max_pending;   /* serving: submitted requests that may wait for admission; mp_submit gives
                              MP_E_BUSY beyond (default 65536) */
} mp_config;

/* Default configuration (device 0, AUTO kernel, 8 in flight, batch 64, 65536 pending). */
int mp_config_default(mp_config *cfg);

/* Create a context on cfg->device (NULL cfg: defaults). *ctx receives the handle. */
int mp_init(mp_ctx **ctx, const mp_config *cfg);

/* Destroy a context: waits for requests in flight, frees dictionaries and
 * device memory it owns. */
int mp_shutdown(mp_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). The pointer
 * stays valid until the thread's next library call. */
const char *mp_last_error(void);

/* Select the join form used by later calls on this context (MP_KERNEL_*). */
int mp_set_kernel(mp_ctx *ctx, int32_t kernel);

/*
 * Load a dictionary D_B (Sec. 3.1 output, Algorithm 2 input) onto the device.
 *   samples      host pointer, seg_offsets[n_segments] samples of type dtype
 *   seg_offsets  host, n_segments + 1 non-decreasing int64 offsets starting at 0;
 *                segment s is samples[seg_offsets[s] .. seg_offsets[s+1])
 *   ms, n_ms     window lengths whose statistics are computed now (others are
 *                computed on first use); may be NULL / 0
 *   out          receives the handle
 * The samples are copied; the caller may free its buffers on return. The
 * total sample count must be below 2^31.
 */
int mp_dict_load(mp_ctx *ctx, const void *samples, int32_t dtype, const int64_t *seg_offsets, int32_t n_segments,
                 const int32_t *ms, int32_t n_ms, mp_dict **out);

/* Free a dictionary. MP_E_BUSY while submitted requests still reference it. */
int mp_dict_free(mp_ctx *ctx, mp_dict *dict);

/* Number of valid dictionary windows W for window length m (windows inside one segment). */
int mp_dict_windows(const mp_dict *dict, int32_t m, int64_t *n_windows);

/*
 * Synchronous join with host buffers (Algorithm 2).
 *   query     host, n samples of type dtype (must match the dictionary's)
 *   out_dist  host, n - m + 1 doubles: P_hat
 *   out_idx   host, n - m + 1 int64: global window index g, or -1
 * Copies the query to the device, joins, copies the result back and returns.
 * From the second call with the same shape (dictionary, dtype, n, m, form)
 * on, a join of at most 2^18 query windows runs as one captured CUDA graph
 * through pinned staging memory that the context keeps (up to 16 shapes; a
 * shape's graph is dropped when its dictionary is freed or the kernel setting
 * changes). The results are the same either way.
 */
int mp_ab_join(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
               double *out_dist, int64_t *out_idx);

/*
 * The join of mp_ab_join reported as a bounded similarity (Sec. 2.1 names the
 * Pearson correlation coefficient as the alternative to the distance; with it
 * the profile keeps the largest value and Guarantee 1 reads P_hat <= P).
 *   out_corr  host, n - m + 1 doubles: rho = 1 - d^2 / (2m) for the nearest
 *             window, which is Pearson's r of the two windows when neither is
 *             constant; under the zero-vector convention for constant windows
 *             it is 0.5 between a constant and a non-constant window and 1
 *             between two constant ones. -inf where the dictionary has no
 *             window of length m.
 *   out_idx   host, n - m + 1 int64: the same window index as mp_ab_join's
 *             (the largest rho is the smallest d).
 */
int mp_ab_join_corr(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
                    double *out_corr, int64_t *out_idx);

/*
 * Streaming join (Sec. 1: arriving data compared with a resident "normal"
 * dictionary, flagging windows without a close neighbour). A stream joins
 * windows of length m as samples arrive; each window is joined once, when
 * its last sample arrives.
 *   mp_stream_open    the stream of one dictionary, dtype (the dictionary's)
 *                     and m (4 .. 8192); the dictionary must outlive the stream.
 *   mp_stream_append  appends n_new host samples and joins the windows that
 *                     end in them: *n_out of them (n_new once m - 1 samples
 *                     have been seen before; fewer at the start), written to
 *                     out_dist / out_idx (host, room for n_new values each) as
 *                     mp_ab_join writes them. *first_window (may be NULL) is
 *                     the stream index of out_dist[0]: windows are numbered
 *                     from the stream's first sample. The samples are copied;
 *                     the call is synchronous. Errors as mp_ab_join; on error
 *                     nothing of the append is kept.
 *   mp_stream_close   frees the stream (the last m - 1 samples it keeps).
 */
int mp_stream_open(mp_ctx *ctx, const mp_dict *dict, int32_t dtype, int32_t m, mp_stream **out);
int mp_stream_append(mp_stream *stream, const void *samples, int64_t n_new, double *out_dist, int64_t *out_idx,
                     int64_t *n_out, int64_t *first_window);
int mp_stream_close(mp_stream *stream);
/*
 * The append of mp_stream_append without waiting for the result: the windows
 * that end in the new samples become one serving request (see mp_submit), so
 * that appends of this stream and of other streams are batched on the device
 * while the caller keeps appending. out_dist / out_idx (host, room for n_new
 * values) must stay valid until mp_poll(*ticket) reports MP_DONE or
 * MP_FAILED; *n_out and *first_window are set at once; *ticket is 0 when no
 * window ended (fewer than m samples seen so far). The samples are copied.
 * Errors as mp_submit (MP_E_BUSY when the admission queue is full); on error
 * nothing of the append is kept.
 */
int mp_stream_submit(mp_stream *stream, const void *samples, int64_t n_new, double *out_dist, int64_t *out_idx,
                     uint64_t *ticket, int64_t *n_out, int64_t *first_window);

/*
 * Self-join matrix profile of one float32 series (the input of Algorithm 1,
 * Sec. 3.1): for every window i the nearest window g with |g - i| >= excl
 * (closer windows are trivial matches of i), its distance and index, with the
 * conventions of mp_ab_join (a constant window is 0 from a constant window
 * outside its zone and sqrt(m) from the rest). Host buffers of n - m + 1
 * values; +inf / -1 where no window lies outside the zone. excl >= 1,
 * 4 <= m <= 8192. Allocates and synchronises.
 */
int mp_self_join(mp_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m, int32_t excl,
                 double *out_dist, int64_t *out_idx);

/* terminal conditions of mp_learn_dictionary (Algorithm 1, lines 13-14) */
#define MP_LEARN_MEMORY 0 /* stop once the merged dictionary holds >= term_value samples */
#define MP_LEARN_EMAX 1   /* stop once the running bound max_i S[i] is <= term_value */

/*
 * Dictionary learning, Algorithm 1 (Sec. 3.1), on the GPU, for a float32
 * training series t_b of n_b samples and window length m (4 <= m <= 8192).
 *   1. P_B = mp_self_join(t_b, m, excl = ceil(m/2)).
 *   2. Repeat: j = argmin over i of P_B[i] - S[i] outside the zones
 *      [j' - m/2, j' + m/2) of the windows j' taken before (S = 0 at first);
 *      add T_B[j : j + m] with floor((k_context - 1) m / 2) samples of
 *      context on each side (clipped to the series), so an element holds
 *      k_context * m samples; S = the distance profile of T_B against
 *      T_B[j : j + m] (first time) or its element-wise minimum with S.
 *   3. Stop at the terminal condition (term_kind, term_value), after
 *      max_elements elements, or when no window is left.
 * Overlapping elements are merged (Sec. 3.1, Fig. 5). Outputs (host):
 *   seg_start, seg_len  the merged elements as positions in t_b, sorted,
 *                       *n_segments of them (capacity max_elements each);
 *                       the dictionary is t_b[seg_start[s] : seg_start[s] +
 *                       seg_len[s]] concatenated, offsets the prefix sums
 *   err_bound           (may be NULL) max_i S[i] at the end. Every window of
 *                       t_b is at most this far from a taken window, so it
 *                       bounds the learned dictionary's e_max (Sec. 3.3)
 *   chosen, n_chosen    (may be NULL) the taken windows j in order
 * Allocates and synchronises.
 */
int mp_learn_dictionary(mp_ctx *ctx, const void *t_b, int32_t dtype, int64_t n_b, int32_t m, double k_context,
                        int32_t term_kind, double term_value, int32_t max_elements, int64_t *seg_start,
                        int64_t *seg_len, int32_t *n_segments, double *err_bound, int64_t *chosen,
                        int32_t *n_chosen);

/*
 * The same join on device buffers, enqueued on `stream` (a cudaStream_t; NULL
 * = the context's own stream). d_query, d_out_dist and d_out_idx are device
 * pointers with the sizes of mp_ab_join. The call returns once the work is
 * enqueued; the outputs are ready when the stream reaches that point. The
 * query buffer must stay unchanged until then. Scratch memory comes from the
 * context's workspace, so calls on one context must not overlap on the GPU
 * (the context serialises them on the host; use one context per concurrent
 * stream). The tensor-core kernels bound every wait on the device; if one runs
 * out (about 2 s), every output distance is NaN and every index -1 (mp_ab_join
 * returns MP_E_TIMEOUT instead).
 */
int mp_ab_join_device(mp_ctx *ctx, const mp_dict *dict, const void *d_query, int32_t dtype, int64_t n, int32_t m,
                      double *d_out_dist, int64_t *d_out_idx, void *stream);

/*
 * The join of mp_ab_join_device without any device allocation (the paper has
 * no counterpart; this is a service of the library). It is meant for callers
 * that must not allocate device memory while they serve a request: services
 * that reserve all GPU memory up front and forbid allocation on the request
 * path, because cudaMalloc/cudaFree can synchronise the device and add
 * latency jitter, and applications that own the device allocator (a caching
 * allocator or pool whose accounting a foreign cudaMalloc would break).
 *
 * Its scratch is one fixed array of about 56 MB inside this library, held by
 * every GPU that loads the library until the process exits. Limits: float32
 * samples only, at most 2^19 query windows (n - m + 1), and a dictionary cut
 * into at most 2^16 runs of windows; larger calls return MP_E_ARG with a
 * message and do nothing. The dictionary's statistics for m must already be
 * resident (list m in mp_dict_load), since computing them would allocate.
 * The caller passes the device query and outputs as for mp_ab_join_device.
 *
 * The first call on a device resolves the scratch array's device address
 * (cudaGetSymbolAddress, with that device current). Every call shares the
 * array and it keeps the last call's contents; everything a call reads from
 * it is written by that call first. Calls whose work overlaps on the GPU (other streams, other
 * contexts, other threads) race on the array and give undefined results:
 * serialise them.
 */
int mp_ab_join_noalloc(mp_ctx *ctx, const mp_dict *dict, const void *d_query, int32_t dtype, int64_t n, int32_t m,
                       double *d_out_dist, int64_t *d_out_idx, void *stream);

/*
 * Window statistics (the first pass of the join) of a device series:
 * mean, 1/std (0 for a constant window) and the constant flag of each of the
 * n - m + 1 windows, in FP64, enqueued on `stream`.
 */
int mp_window_stats(mp_ctx *ctx, const void *d_x, int32_t dtype, int64_t n, int32_t m, double *d_mean,
                    double *d_invstd, uint8_t *d_const, void *stream);

/*
 * Serving: submit a join request. The query is copied before the call
 * returns. out_dist / out_idx are host buffers (n - m + 1 entries) that must
 * stay valid until mp_poll reports MP_DONE or MP_FAILED. Requests are admitted
 * to the device in arrival order as slots and memory free up. Float32
 * requests of at least 2^16 query windows run alone with the synchronous
 * join's kernels, on streams of the device's least priority; the others are
 * batched into persistent launches on streams of its greatest priority, so a
 * short request is not held up by a long one already running. Each result is
 * identical to what mp_ab_join returns for the same inputs. *ticket receives
 * the request id.
 */
int mp_submit(mp_ctx *ctx, const mp_dict *dict, const void *query, int32_t dtype, int64_t n, int32_t m,
              double *out_dist, int64_t *out_idx, uint64_t *ticket);

/*
 * Non-blocking state of a request: *state = MP_PENDING, MP_DONE or MP_FAILED;
 * *latency_s (may be NULL) = submit-to-completion time once done. A ticket
 * can be polled until it has been reported done or failed once; later polls
 * give MP_E_NOTFOUND.
 */
int mp_poll(mp_ctx *ctx, uint64_t ticket, int32_t *state, double *latency_s);

/* Block until every submitted request has finished or timeout_s passes (MP_E_TIMEOUT). */
int mp_drain(mp_ctx *ctx, double timeout_s);

/*
 * e_max of Sec. 3.3: the largest distance from a length-m window of the
 * series T_B the dictionary was learned from to its nearest dictionary window,
 * e_max = max_i NNDist(T_B[i : i+m], D_{B,m}), computed with the join
 * (mp_ab_join of T_B against the dictionary). By Lemma 2 every approximate
 * profile value exceeds the exact one by at most e_max when the dictionary's
 * windows are windows of T_B (Proposition 1). t_b is a host series of n_b
 * samples; *argmax (may be NULL) receives the window attaining the maximum.
 */
int mp_emax(mp_ctx *ctx, const mp_dict *dict, const void *t_b, int32_t dtype, int64_t n_b, int32_t m, double *e_max,
            int64_t *argmax);

/*
 * Discords of a (host) matrix profile of n values: the k largest finite
 * values, each followed by an exclusion of +-excl windows around it (the
 * paper excludes +-m/2 as trivial matches, Algorithm 1), written to idx / val
 * in decreasing order; *n_found (may be NULL) receives how many were found.
 * *top1_certified (may be NULL) is the certificate of Sec. 2.1 for an
 * approximate profile: 1 when the top value exceeds every value outside its
 * exclusion zone by more than e_max (Guarantee 2), so that the top discord of
 * the exact profile is the same subsequence. Host computation only.
 */
int mp_top_discords(const double *profile, int64_t n, int32_t k, int64_t excl, double e_max, int64_t *idx, double *val,
                    int32_t *n_found, int32_t *top1_certified);

/*
 * Autotuner: chooses the join form and the plain kernel's column grouping for
 * one shape (dictionary, m, query length n). It builds a synthetic query of n
 * samples from the dictionary's own samples, times the plain form at several
 * column-group counts and the split-BF16 and TF32 tensor-core forms, and
 * keeps the fastest. Every form picks each row's window exactly (see the join
 * forms above), so each meets the same distance tolerance; `tolerance` (the
 * caller's absolute distance tolerance) is recorded with the choice. The
 * single-BF16 form is not timed: its wide error bound leaves many chunks to
 * re-score. The choice applies to later joins on this context
 * whose kernel is MP_KERNEL_AUTO and whose shape falls in the same bucket
 * (same dtype and m, same floor(log2) of the dictionary windows and of the
 * query windows); with mp_config.tune_cache set it is also appended to that
 * file as one JSON line, and mp_init reloads the file. Outputs (may be
 * NULL): the chosen MP_KERNEL_* form, its column groups and its time in ms.
 * The call allocates and synchronises; it is meant for set-up, not serving.
 */
int mp_autotune(mp_ctx *ctx, const mp_dict *dict, int32_t m, int64_t n, double tolerance, int32_t *kernel,
                int32_t *groups, double *ms);

/*
 * The plan of a join (Algorithm 2) of n query samples at window length m on
 * this context, as mp_ab_join_device would run it now: the form (after the
 * kernel setting, the autotuner's cache and the form's m limits), the plain
 * form's column groups, the dictionary spans those groups cut (a span is one
 * segment's run of windows inside one group; the left seeds hold one value per
 * span and query window), the plain launches the query's windows take (row
 * chunks), whether the FP32 plain join takes its seeds from the tensor cores
 * (joins of at least 2^31 pairs; smaller ones compute them in the plain kernel),
 * and the workspace bytes the context reserves for the join. It computes the
 * dictionary's statistics for m if they are not resident (that allocates) and
 * launches nothing else. Errors: MP_E_ARG as for mp_ab_join_device.
 */
typedef struct mp_join_plan {
    int32_t kernel;          /* MP_KERNEL_* the join runs */
    int32_t column_groups;   /* column groups of the plain form */
    int64_t spans;           /* dictionary spans of those groups */
    int64_t row_chunks;      /* plain launches over the query's windows */
    int32_t tc_seeds;        /* 1: top and left seeds on the tensor cores (FP32 plain form) */
    int32_t pad;
    int64_t workspace_bytes; /* device workspace the join reserves (every form) */
} mp_join_plan;
int mp_plan_join(mp_ctx *ctx, const mp_dict *dict, int32_t dtype, int64_t n, int32_t m, mp_join_plan *plan);

/* Phases of a join, for mp_profile_read. */
#define MP_PHASE_STATS 0    /* window statistics of the query (K1) */
#define MP_PHASE_JOIN 1     /* the join kernel: plain (K2) or tensor-core (K3) */
#define MP_PHASE_FINALIZE 2 /* reduction, constant-window rule and exact distance of the pick (K4) */
#define MP_PHASE_SEEDS 3    /* the plain join's top seeds on the tensor cores (K2s; FP32 plain joins of >= 2^31 pairs) */
#define MP_PHASE_LEFT_SEEDS 4 /* the plain join's left seeds on the tensor cores (K2l; the same joins) */
#define MP_PHASE_COUNT 5

/*
 * Tracing: with enable = 1, synchronous and device joins on this context
 * record a CUDA event pair around each phase, on the stream the phase runs
 * on. mp_profile_read waits for the recorded work and returns the summed
 * device milliseconds and launch counts per phase (arrays of MP_PHASE_COUNT;
 * either may be NULL); reset = 1 clears the sums.
 */
int mp_profile(mp_ctx *ctx, int32_t enable);
int mp_profile_read(mp_ctx *ctx, double *ms, int64_t *launches, int32_t reset);

/* Counters of the finalisation step of Algorithm 2's element-wise minimum (Sec. 3.2), for mp_counters. */
#define MP_COUNTER_NEAR_ROWS 0      /* query windows that re-scored near-tied chunks besides the winner */
#define MP_COUNTER_NEAR_CHUNKS 1    /* near-tied chunks (16 dictionary windows each) re-scored */
#define MP_COUNTER_OVERFLOW_ROWS 2  /* query windows whose near-tie records of a column group overflowed */
#define MP_COUNTER_OVERFLOW_CHUNKS 3 /* chunks re-scored because of those overflows (whole column groups) */
#define MP_COUNTER_COUNT 4

/*
 * Counters summed over every join of this context (synchronous, device,
 * no-allocation and serving) since the last reset. The join kernels keep an
 * approximate score per 16-window chunk; the finalisation re-scores exactly
 * the winning chunk and every chunk whose approximate score came within the
 * form's near-tie width of the best (the kernels record up to a fixed number
 * of such chunks per column group and query window; when a record that might
 * matter has to be dropped, the finalisation re-scores that whole column
 * group for that window instead). values: MP_COUNTER_COUNT int64 (host).
 * Waits for all work on the context's device; reset = 1 zeroes them.
 */
int mp_counters(mp_ctx *ctx, int64_t *values, int32_t reset);

/* Testing hooks: host-side fault injection for the tests of the failure paths
 * (the paper has no counterpart). */
#define MP_HOOK_FAIL_ALLOC 0 /* the next `value` device allocations of serving requests fail as if the device
                                were out of memory: those requests end MP_FAILED */
#define MP_HOOK_TC_WAIT 1    /* bound, in SM clocks, of the tensor-core join's waits of one of its roles on
                                another (0: the default, about 2 s); a bound too short for the work makes the
                                join time out (mp_ab_join: MP_E_TIMEOUT; device calls: NaN and index -1). The
                                kernel's last wait, for its own tensor-core work before it frees the tensor
                                memory, keeps the default */
int mp_test_hook(mp_ctx *ctx, int32_t hook, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* MPDICT_H */

// Tensor-core form of the join (kernel K3): declarations used by the runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mp_internal.cuh"

namespace mpd {

typedef int (*fail_fn)(int, const char *, ...);

// Whether the tensor-core kernel handles window length m (variants 0: split
// BF16 and 2: single BF16, m a multiple of 16, up to about 600 and 1100;
// variant 1: TF32, m a multiple of 8, up to about 1100 -- the query operand
// of all m stays in shared memory).
bool tc_supported(int variant, int m);
// Upper bound of the column groups tc_join uses for nq query windows.
int tc_groups_bound(int sm_count, int64_t nq);
// Free the per-(dictionary, m) tile tables created by tc_join.
void tc_free_pack(void *pack);

// Launch the tensor-core join (kernel K3) of an FP32 query whose window
// statistics are computed (ms_*: Split<float> means, rs_*: float4 terms);
// writes part[group * nq + row] (the same partial format as the plain kernel),
// the near-tie records of every row (near->rec may be null; near->ld = nq;
// the call sets near->fb and near->u, the width's terms) and
// *n_groups_out; *cspans_out / *cgroup_start_out receive the column groups'
// chunk layout (valid until the dictionary is freed). *err is set to 1 on a
// device-side timeout. variant: 0 = split BF16 (3 products), 1 = TF32, 2 = one
// BF16 product.
// The caller sizes part and near for tc_groups_bound groups. wait_cycles
// bounds the kernel's waits of one role on another (<= 0: about 2 s); the
// final wait for the MMAs before the TMEM is freed keeps its own bound.
int tc_join(int sm_count, int variant, void **pack, const float *b, int64_t nb, const Span *seg_spans, int32_t n_seg,
            const void *ms_b, const void *rs_b, const float *a, int64_t n, int32_t m, const void *ms_a,
            const void *rs_a, Partial<float> *part, NearRec *near, int32_t *err, int *n_groups_out,
            const Span **cspans_out, const int32_t **cgroup_start_out, long long wait_cycles, cudaStream_t st,
            fail_fn fail);

// Top seeds of the plain kernel (K2s) on the tensor cores: for the query
// windows r_s = s * stride, s < ceil(nq / stride), and every valid dictionary
// window g, seeds[s * ld + g] = the centred covariance
// sum_k (a[r_s + k] - mean_a[r_s]) (b[g + k] - mean_b[g]) in FP32 (three TF32
// products of a hi/lo split). Positions g of windows that cross a segment end
// are not written; ld >= nb - m + 1. *err is set to 1 on a device-side
// timeout. Any m >= 1.
int tc_seeds(void **pack, const float *b, int64_t nb, const Span *seg_spans, int32_t n_seg,
             const void *ms_b, const float *a, int64_t n, int32_t m, const void *ms_a, int32_t stride, float *seeds,
             int64_t ld, int32_t *err, cudaStream_t st, fail_fn fail);

// Left seeds of the plain kernel (K2l) on the tensor cores: for every query
// window r < n - m + 1 and span s < n_spans (device spans, the column groups'
// runs of windows), left[s * ld + r] = the centred covariance
// sum_k (a[r + k] - mean_a[r]) (b[g_s + k] - mean_b[g_s]) with g_s the span's
// first window, in FP32 (three TF32 products of a hi/lo split). ops is the
// spans' operand (tc_left_operand_bytes bytes) that tc_left_operand builds
// once for the dictionary, m and spans. ld >= the query windows. *err is set
// to 1 on a device-side timeout. Any m >= 1.
size_t tc_left_operand_bytes(int32_t n_spans, int32_t m);
int tc_left_operand(const float *b, int64_t nb, const void *ms_b, const Span *spans, int32_t n_spans, int32_t m,
                    unsigned char *ops, cudaStream_t st, fail_fn fail);
int tc_left_seeds(const float *a, int64_t n, int32_t m, const void *ms_a, const void *ms_b, const Span *spans,
                  int32_t n_spans, const unsigned char *ops, float *left, int64_t ld, int32_t *err, cudaStream_t st,
                  fail_fn fail);

}  // namespace mpd

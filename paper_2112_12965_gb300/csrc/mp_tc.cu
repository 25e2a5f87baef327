// Tensor-core form of the join (kernel K3).
#include "../../include/mpdict.h"
#include "mp_tc.cuh"

namespace mpd {

bool tc_supported(int) { return false; }
int tc_autotune_choice(int, int64_t) { return MP_KERNEL_PLAIN; }
void tc_load_tune_cache(const char *) {}
void tc_free_pack(void *) {}
int tc_join(int, int, void **, const float *, int64_t, const Span *, int32_t, const double *, const double *,
            const void *, const float *, int64_t, int32_t, const double *, const double *, const uint8_t *, int64_t,
            int64_t, double *, int64_t *, cudaStream_t, fail_fn fail)
{
    return fail(MP_E_INTERNAL, "tensor-core join not available");
}

}  // namespace mpd

// Batched persistent launch of many Langevin systems (placeholder until the
// batched kernel lands).
#include "internal.cuh"

extern "C" int ld_run_batched(ld_system* sys, int n_sys, int64_t n_steps, const int* tune,
                              ld_stats* out, void* stream)
{
    (void)sys; (void)n_sys; (void)n_steps; (void)tune; (void)out; (void)stream;
    return gb::fail(GBRNG_EINVAL, "ld_run_batched is not available in this build");
}

// Reverse-time adjoint (placeholder until the adjoint kernels land).
#include "internal.cuh"

extern "C" int ld_backward(ld_system* sys, int64_t n_steps, int ckpt_every, float* dK_per,
                           double* dgamma, double* dkT, double* loss, void* stream)
{
    (void)sys; (void)n_steps; (void)ckpt_every; (void)dK_per; (void)dgamma; (void)dkT;
    (void)loss; (void)stream;
    return gb::fail(GBRNG_EINVAL, "ld_backward is not available in this build");
}

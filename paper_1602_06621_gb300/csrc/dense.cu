// Dense operator: products with +-1 probe blocks on the tensor cores.

#include <cuda_runtime.h>

#include "sme_internal.cuh"

namespace sme {

void dense_destroy(sme_op op) { op->dense = nullptr; }

sme_status dense_equilibrate(sme_op op, const sme_equil_params *p, float *u, float *v, float *ub, float *vb,
                             cudaStream_t s)
{
    (void)op; (void)p; (void)u; (void)v; (void)ub; (void)vb; (void)s;
    set_error("dense operators: not built yet");
    return SME_ERR_UNSUPPORTED;
}

sme_status dense_estimate(sme_op op, const float *u, const float *v, int t, int k, uint64_t seed, int sb, float *zu,
                          float *zv, cudaStream_t s)
{
    (void)op; (void)u; (void)v; (void)t; (void)k; (void)seed; (void)sb; (void)zu; (void)zv; (void)s;
    set_error("dense operators: not built yet");
    return SME_ERR_UNSUPPORTED;
}

}  // namespace sme

extern "C" sme_status sme_op_create_dense(sme_op *out, int64_t m, int64_t n, const void *A, int64_t lda,
                                          sme_dtype dtype, const float *row_scales, int on_device, void *stream)
{
    (void)m; (void)n; (void)A; (void)lda; (void)dtype; (void)row_scales; (void)on_device; (void)stream;
    if (out) *out = nullptr;
    sme::set_error("sme_op_create_dense: not built yet");
    return SME_ERR_UNSUPPORTED;
}

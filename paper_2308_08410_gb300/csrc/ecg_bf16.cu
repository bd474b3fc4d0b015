// ecg_bf16.cu -- BF16 tensor-core lead-field contraction (placeholder until
// the tcgen05 kernel lands: the entry point reports "not supported").
#include "gbp_internal.cuh"

namespace gbp {

cudaError_t prepare_leadfield_bf16(gbp_ctx *c)
{
    (void)c;
    return cudaSuccess;
}

cudaError_t launch_ecg_forward_bf16(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg)
{
    (void)c; (void)phi; (void)t; (void)ecg;
    return cudaErrorNotSupported;
}

}  // namespace gbp

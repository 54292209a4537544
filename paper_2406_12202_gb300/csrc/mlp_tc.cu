// mlp_tc.cu -- tensor-core (tcgen05) form of the NeRF MLP (placeholder until
// the fused kernel lands: BF16 / FP8 precisions report MCL_ERR_UNSUPPORTED).
#include "internal.cuh"

namespace mcl {

int mlp_tc_prepare(mcl_map* m, const float* host_blob) {
    (void)m; (void)host_blob;
    return MCL_OK;
}

void mlp_tc_free(mcl_map* m) { (void)m; }

cudaError_t mlp_tc(mcl_map* m, int precision, const Ray* rays, const float* gd, const float* z,
                   int S, int n_rays, float4* out, cudaStream_t s) {
    (void)m; (void)precision; (void)rays; (void)gd; (void)z; (void)S; (void)n_rays; (void)out; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace mcl

// k_mlp_tc.cu -- per-element network on tcgen05 tensor cores (BF16 / FP8).
#include "nnp_host.h"

namespace nnp {

int mlp_tc_init(nnp_ctx* ctx) {
  return ctx->fail(NNP_ERR_UNSUPPORTED, "tensor-core network not built yet");
}
int mlp_tc_set_weights(nnp_ctx*, int, const float*) { return NNP_OK; }
void mlp_tc_free(nnp_ctx*) {}
int launch_mlp_tc(nnp_ctx* ctx, cudaStream_t, long long) {
  return ctx->fail(NNP_ERR_UNSUPPORTED, "tensor-core network not built yet");
}

}  // namespace nnp

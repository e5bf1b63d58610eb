// BF16 tensor-core path (placeholder until the tcgen05 kernels land).
#include "paths.cuh"

namespace xmgn {
bool bf16_supported(const ParamPlan& p) { return false && p.H == 128; }
void bf16_sizes(const ParamPlan&, int64_t, int64_t, size_t* ws, size_t* ckpt) { *ws = *ckpt = 256; }
xmgn_status bf16_forward(const ParamPlan&, const float*, const xmgn_graph&, const float*, const float*,
                         const float*, float*, float*, void*, size_t, void*, size_t, cudaStream_t) {
  return fail(XMGN_ERR_UNSUPPORTED, "bf16 path not built");
}
xmgn_status bf16_backward(const ParamPlan&, const float*, const xmgn_graph&, const float*, const float*,
                          const float*, const void*, size_t, float*, float*, void*, size_t, cudaStream_t) {
  return fail(XMGN_ERR_UNSUPPORTED, "bf16 path not built");
}
}  // namespace xmgn

// D3Q19 step kernels with bf16 reference-offset storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_bf16(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, __nv_bfloat16>(p, fin, fout, st);
}
}  // namespace lbmsc

// D3Q19 step kernels with bf16 rest-offset storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_bf16_rest(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, bf16_rest>(p, fin, fout, st);
}
}  // namespace lbmsc

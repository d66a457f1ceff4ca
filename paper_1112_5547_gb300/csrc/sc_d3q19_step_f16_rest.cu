// D3Q19 step kernels with fp16 rest-offset storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_f16_rest(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, f16_rest>(p, fin, fout, st);
}
}  // namespace lbmsc

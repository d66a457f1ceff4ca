// D3Q19 step kernels with FP32 storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_f32(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, float>(p, fin, fout, st);
}
}  // namespace lbmsc

// D3Q19 step kernels with fp16 reference-offset storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_f16(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, __half>(p, fin, fout, st);
}
}  // namespace lbmsc

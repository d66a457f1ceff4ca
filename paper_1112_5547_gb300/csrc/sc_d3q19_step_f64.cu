// D3Q19 step kernels with FP64 storage (one translation unit per precision).
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step_f64(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_typed<D3Q19, double>(p, fin, fout, st);
}
}  // namespace lbmsc

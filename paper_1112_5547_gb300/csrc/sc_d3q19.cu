// D3Q19 instantiations of the fused Shan-Chen kernels.
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_any<D3Q19>(p, fin, fout, st);
}
cudaError_t d3q19_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st) {
    return init_any<D3Q19>(p, rA, rB, u, fout, st);
}
cudaError_t d3q19_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    return moments_any<D3Q19>(p, fin, o, st);
}
}  // namespace lbmsc

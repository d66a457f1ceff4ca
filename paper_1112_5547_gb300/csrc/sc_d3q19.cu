// D3Q19 instantiations of the fused Shan-Chen kernels: init and moments here;
// the step kernels of each storage precision in their own translation unit
// (sc_d3q19_step_*.cu) so that they compile in parallel.
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d3q19_step(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    switch (p.precision) {
        case 0: return d3q19_step_f64(p, fin, fout, st);
        case 1: return d3q19_step_f32(p, fin, fout, st);
        case 2: return d3q19_step_bf16(p, fin, fout, st);
        case 3: return d3q19_step_f16(p, fin, fout, st);
        case 4: return d3q19_step_bf16_rest(p, fin, fout, st);
        case 5: return d3q19_step_f16_rest(p, fin, fout, st);
    }
    return cudaErrorInvalidValue;
}
cudaError_t d3q19_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st,
                      int zlo, int zhi) {
    return init_any<D3Q19>(p, rA, rB, u, fout, st, zlo, zhi);
}
cudaError_t d3q19_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    return moments_any<D3Q19>(p, fin, o, st);
}
}  // namespace lbmsc

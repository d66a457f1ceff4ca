// D2Q9 instantiations of the fused Shan-Chen kernels.
#include "sc_instantiate.cuh"

namespace lbmsc {
cudaError_t d2q9_step(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    return step_any<D2Q9>(p, fin, fout, st);
}
cudaError_t d2q9_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st,
                      int zlo, int zhi) {
    return init_any<D2Q9>(p, rA, rB, u, fout, st, zlo, zhi);
}
cudaError_t d2q9_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    return moments_any<D2Q9>(p, fin, o, st);
}
cudaError_t diag_finish(const double* partials, long long nparts, double* out, cudaStream_t st) {
    sc_diag_finish_kernel<256><<<1, 256, 0, st>>>(partials, nparts, out);
    return cudaGetLastError();
}
}  // namespace lbmsc

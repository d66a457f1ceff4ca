// Typed launch helpers shared by the per-lattice translation units.
#pragma once

#include "sc_kernels.cuh"
#include "sc_launch.cuh"

namespace lbmsc {

template <class S> LatticeArgs<S> make_args(const Plan& p, const void* fin, void* fout) {
    using C = typename Codec<S>::C;
    LatticeArgs<S> a;
    a.fin = static_cast<const S*>(fin);
    a.fout = static_cast<S*>(fout);
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.zchunk = p.zchunk;
    a.N = p.N;
    a.omega_A = (C)(1.0 / p.tau_A);
    a.omega_B = (C)(1.0 / p.tau_B);
    a.tau_A = (C)p.tau_A;
    a.tau_B = (C)p.tau_B;
    a.G = (C)p.G;
    a.ref_A = Codec<S>::kOffset ? (C)p.ref_A : (C)0;
    a.ref_B = Codec<S>::kOffset ? (C)p.ref_B : (C)0;
    return a;
}

// Minimum CTAs per SM requested from the register allocator: two 256-thread
// CTAs for 32-bit compute, one for FP64 (whose 76 live doubles would spill).
template <class S> struct MinBlocks { static constexpr int value = 2; };
template <> struct MinBlocks<double> { static constexpr int value = 1; };

template <class L, class S> cudaError_t step_typed(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    using C = typename Codec<S>::C;
    const LatticeArgs<S> a = make_args<S>(p, fin, fout);
    FieldArgs<C> fo{};
    sc_fused_kernel<L, S, kTX, kTY, kModeStep, MinBlocks<S>::value>
        <<<fused_grid(p), dim3(kTX, kTY), 0, st>>>(a, fo);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t init_typed(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st) {
    using C = typename Codec<S>::C;
    const LatticeArgs<S> a = make_args<S>(p, nullptr, fout);
    long long blocks = (p.N + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    sc_init_kernel<L, S><<<(unsigned)blocks, 256, 0, st>>>(a, static_cast<const C*>(rA), static_cast<const C*>(rB),
                                                          static_cast<const C*>(u));
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t moments_typed(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    using C = typename Codec<S>::C;
    const LatticeArgs<S> a = make_args<S>(p, fin, nullptr);
    FieldArgs<C> fo;
    fo.rhoA = static_cast<C*>(o.rhoA);
    fo.rhoB = static_cast<C*>(o.rhoB);
    fo.u = static_cast<C*>(o.u);
    fo.p = static_cast<C*>(o.p);
    fo.partials = o.partials;
    fo.win_c[0] = o.win[0];
    fo.win_c[1] = o.win[1];
    fo.win_c[2] = o.win[2];
    fo.r_in2 = o.win[3] < 0 ? -1.0 : o.win[3] * o.win[3];
    fo.r_out2 = o.win[4] * o.win[4];
    sc_fused_kernel<L, S, kTX, kTY, kModeMoments, 1><<<fused_grid(p), dim3(kTX, kTY), 0, st>>>(a, fo);
    return cudaGetLastError();
}

template <class L> cudaError_t step_any(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    switch (p.precision) {
        case 0: return step_typed<L, double>(p, fin, fout, st);
        case 1: return step_typed<L, float>(p, fin, fout, st);
        case 2: return step_typed<L, __nv_bfloat16>(p, fin, fout, st);
        case 3: return step_typed<L, __half>(p, fin, fout, st);
    }
    return cudaErrorInvalidValue;
}

template <class L>
cudaError_t init_any(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st) {
    switch (p.precision) {
        case 0: return init_typed<L, double>(p, rA, rB, u, fout, st);
        case 1: return init_typed<L, float>(p, rA, rB, u, fout, st);
        case 2: return init_typed<L, __nv_bfloat16>(p, rA, rB, u, fout, st);
        case 3: return init_typed<L, __half>(p, rA, rB, u, fout, st);
    }
    return cudaErrorInvalidValue;
}

template <class L> cudaError_t moments_any(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    switch (p.precision) {
        case 0: return moments_typed<L, double>(p, fin, o, st);
        case 1: return moments_typed<L, float>(p, fin, o, st);
        case 2: return moments_typed<L, __nv_bfloat16>(p, fin, o, st);
        case 3: return moments_typed<L, __half>(p, fin, o, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbmsc

// Kernel arguments of one lattice from its host-side plan.
#pragma once

#include <cudaTypedefs.h>

#include "sc_common.cuh"
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
    a.zbase = 0;
    a.zend = p.nz;
    a.N = p.N;
    a.px = p.px;
    a.py = p.py;
    a.gxo = p.gxo;
    a.gyo = p.gyo;
    a.Np = p.Np;
    a.omega_A = (C)(1.0 / p.tau_A);
    a.omega_B = (C)(1.0 / p.tau_B);
    a.tau_A = (C)p.tau_A;
    a.tau_B = (C)p.tau_B;
    a.G = (C)p.G;
    a.ref_A = Codec<S>::kOffset ? (C)p.ref_A : (C)0;
    a.ref_B = Codec<S>::kOffset ? (C)p.ref_B : (C)0;
    a.body_A = (C)p.body_A;
    a.forcing = p.forcing;
    a.model = p.model;
    a.kappa = (C)p.kappa;
    a.gamma = (C)p.gamma;
    a.wait_probe = p.wait_probe;
    return a;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

constexpr CUtensorMapL2promotion kPromotion[4] = {CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B};

// Tensor map of the population planes of one buffer as a 4-D array: x and y
// of the ghost-padded plane, z, and the plane index (s*Q + i, or i for the
// paired rest-offset words; planes = 0 means 2 Q); boxes of bx x by x 1 x 1
// values of elem_bytes (4: FP32 or a paired rest-offset word, 2: 16-bit
// storage copied as raw 16-bit words).  The box x start of a tile at x0 is x0 + gxo - 16 bytes
// of values, so gxo and the row pitch must be whole 16-byte units for it to be
// 16-byte aligned, as tensor copies require.  promo indexes kPromotion (the
// L2 fetch granularity on a miss).
inline cudaError_t encode_population_map(const Plan& p, const void* fin, int bx, int by, CUtensorMap* map,
                                         int promo = 3, int elem_bytes = 4, int planes = 0) {
    const int e = elem_bytes;
    if ((e != 4 && e != 2) || p.gxo * e < 16 || (p.gxo * e) % 16 != 0 || ((long long)p.px * e) % 16 != 0 ||
        (bx * e) % 16 != 0)
        return cudaErrorInvalidValue;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const int q2 = planes > 0 ? planes : 2 * (p.lattice == 0 ? 9 : 19);
    const cuuint64_t dims[4] = {(cuuint64_t)p.px, (cuuint64_t)p.py, (cuuint64_t)p.nz, (cuuint64_t)q2};
    const cuuint64_t strides[3] = {(cuuint64_t)p.px * e, (cuuint64_t)p.px * p.py * e, (cuuint64_t)p.Np * e};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(map, e == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(fin),
            dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, kPromotion[promo & 3],
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

// Tensor map of the float2 density plane of a rest-offset buffer (rho_base =
// its first pair) as floats: x (two floats per node), y, z, and a unit fourth
// dimension; boxes of 2 bx floats (bx nodes) x by x 1 x 1.  A box starting at
// node x0 - 2 of a tile is 16-byte aligned when gxo and x0 are even.
inline cudaError_t encode_rho_map(const Plan& p, const float2* rho_base, int bx, int by, CUtensorMap* map,
                                  int promo = 3) {
    if ((p.px * 8) % 16 != 0 || (bx * 8) % 16 != 0 || p.gxo < 2 || (p.gxo - 2) % 2 != 0)
        return cudaErrorInvalidValue;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)p.px * 2, (cuuint64_t)p.py, (cuuint64_t)p.nz, 1};
    const cuuint64_t strides[3] = {(cuuint64_t)p.px * 8, (cuuint64_t)p.px * p.py * 8, (cuuint64_t)p.Np * 8};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * bx), (cuuint32_t)by, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(rho_base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, kPromotion[promo & 3],
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace lbmsc

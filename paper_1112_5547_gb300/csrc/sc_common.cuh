// Shared device-side definitions of the Shan-Chen LBM kernels: velocity sets,
// storage codecs and kernel argument blocks.
//
// Velocity sets (GPU order; opposite directions are adjacent):
//   D2Q9 : rest, (+-1,0), (0,+-1), (1,1),(-1,-1), (1,-1),(-1,1)
//          weights 4/9, 1/9, 1/36
//   D3Q19: rest, (+-1,0,0), (0,+-1,0), (0,0,+-1), then the 12 edge vectors
//          weights 1/3, 1/18, 1/36
// Both satisfy sum_i w_i c_ia c_ib = cs2 delta_ab and the fourth-order isotropy
// condition with cs2 = 1/3 required by Sec. 2.1 of the paper.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmsc {

struct D2Q9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr signed char t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},
                                         {0, 1, 0},  {0, -1, 0},  {1, 1, 0},
                                         {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D3Q19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr signed char t[19][3] = {
            {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
            {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
            {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// Storage codecs: load/store one population value.  16-bit types hold the
// offset h = f - w_i rho_ref (the caller passes the offset w_i rho_ref).
// The rest-offset types (kRest) pair the two species in one word per
// direction and offset from the storing node's own density (see bf16_rest).
template <class S> struct Codec;

template <> struct Codec<double> {
    using C = double;
    static constexpr bool kOffset = false;
    static constexpr bool kRest = false;
    __device__ __forceinline__ static C load(const double* p, C) { return __ldg(p); }
    __device__ __forceinline__ static void store(double* p, C v, C) { __stcs(p, v); }
};

template <> struct Codec<float> {
    using C = float;
    static constexpr bool kOffset = false;
    static constexpr bool kRest = false;
    __device__ __forceinline__ static C load(const float* p, C) { return __ldg(p); }
    __device__ __forceinline__ static void store(float* p, C v, C) { __stcs(p, v); }
};

template <> struct Codec<__nv_bfloat16> {
    using C = float;
    static constexpr bool kOffset = true;
    static constexpr bool kRest = false;
    __device__ __forceinline__ static C decode(__nv_bfloat16 v, C off) { return __fadd_rn(__bfloat162float(v), off); }
    __device__ __forceinline__ static C load(const __nv_bfloat16* p, C off) { return decode(__ldg(p), off); }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, C v, C off) {
        *p = __float2bfloat16_rn(__fsub_rn(v, off));
    }
};

template <> struct Codec<__half> {
    using C = float;
    static constexpr bool kOffset = true;
    static constexpr bool kRest = false;
    __device__ __forceinline__ static C decode(__half v, C off) { return __fadd_rn(__half2float(v), off); }
    __device__ __forceinline__ static C load(const __half* p, C off) { return decode(__ldg(p), off); }
    __device__ __forceinline__ static void store(__half* p, C v, C off) {
        *p = __float2half_rn(__fsub_rn(v, off));
    }
};

// Species-paired 16-bit rest-offset storage.  One 32-bit word per node and
// direction holds the offsets of both species, species A in the low 16 bits
// and species B in the high 16 bits (bf16 or fp16):
//   h_is(n) = f_is(n) - w_i rho_s(n),
// rho_s(n) the density of the node n the word is stored at, which is kept in
// FP32 beside the populations (rest_rho: one float2 (rho_A, rho_B) per node).
// Encoding and decoding take one fused multiply-add per value,
//   h = round16(fma(-w_i, rho_s(n), f)),   f = fma(w_i, rho_s(n), h),
// so a value pulled from n gets back exactly the product it was offset by.
// Pairing the species halves the load, store and conversion instructions of
// the unpaired 16-bit layout (one word, one pack, one density pair per
// direction instead of two of each).
struct bf16_rest {
    uint32_t v;
};
struct f16_rest {
    uint32_t v;
};

template <> struct Codec<bf16_rest> {
    using C = float;
    static constexpr bool kOffset = true;
    static constexpr bool kRest = true;
    __device__ __forceinline__ static C lo(uint32_t v) { return __uint_as_float(v << 16); }
    __device__ __forceinline__ static C hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
    // (a, b) -> one word, a in the low half (round to nearest even)
    __device__ __forceinline__ static uint32_t pack(C a, C b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
    }
};

template <> struct Codec<f16_rest> {
    using C = float;
    static constexpr bool kOffset = true;
    static constexpr bool kRest = true;
    __device__ __forceinline__ static C lo(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu))); }
    __device__ __forceinline__ static C hi(uint32_t v) { return __half2float(__ushort_as_half((unsigned short)(v >> 16))); }
    __device__ __forceinline__ static uint32_t pack(C a, C b) {
        const __half2 h = __floats2half2_rn(a, b);
        return (uint32_t)__half_as_ushort(h.x) | ((uint32_t)__half_as_ushort(h.y) << 16);
    }
};

// Decode and encode of one paired rest-offset word (the species' densities r.x, r.y of the storing node).
template <class S>
__device__ __forceinline__ void rest_decode(uint32_t v, float w, float2 r, float& fA, float& fB) {
    fA = __fmaf_rn(w, r.x, Codec<S>::lo(v));
    fB = __fmaf_rn(w, r.y, Codec<S>::hi(v));
}
template <class S> __device__ __forceinline__ uint32_t rest_encode(float fA, float fB, float w, float2 r) {
    return Codec<S>::pack(__fmaf_rn(-w, r.x, fA), __fmaf_rn(-w, r.y, fB));
}

// Density plane of a rest-offset population buffer: it follows the Q paired
// population planes, one float2 (rho_A, rho_B) per node, same ghost-padded
// geometry (node index cell()).
template <class L, class S> __host__ __device__ __forceinline__ float2* rest_rho(S* buf, long long Np) {
    return reinterpret_cast<float2*>(buf + (size_t)L::Q * (size_t)Np);
}
template <class L, class S> __host__ __device__ __forceinline__ const float2* rest_rho(const S* buf, long long Np) {
    return reinterpret_cast<const float2*>(buf + (size_t)L::Q * (size_t)Np);
}

// Per-lattice arguments of the step / moments kernels (compute type C).
template <class S> struct LatticeArgs {
    using C = typename Codec<S>::C;
    const S* fin;       // populations at the current time (pulled along -c_i)
    S* fout;            // populations after collision (same node, not pushed)
    int nx, ny, nz;
    int zchunk;         // planes per CTA along z (D3Q19)
    int zbase, zend;    // planes [zbase, zend) covered by a moments launch (0, nz otherwise)
    long long N;        // nx * ny * nz
    // Population storage is ghost-padded: each z plane of a population is
    // py rows of px values, node (x, y) at column x + gxo, row y + gyo.  The
    // columns x = -1, nx and rows y = -1, ny hold the periodic images of the
    // opposite edge (written by every store), so pulls never wrap in x or y.
    int px, py, gxo, gyo;
    long long Np;       // values per population plane: px * py * nz
    C omega_A, omega_B; // 1 / tau_s
    C tau_A, tau_B;
    C G;
    C ref_A, ref_B;     // rho_ref_s of the 16-bit offsets (0 otherwise)
    C body_A;           // amplitude A of the Kolmogorov forcing (Eq. kolmo); 0 = none
    int forcing;        // kForcingShift (Sec. 2.1) or kForcingGuo (Sec. 2.3)
    int model;          // kModelSC (Sec. 2.1) or kModelFE (Sec. 2.2: species 0 = f, 1 = g)
    C kappa, gamma;     // FE gradient coefficient and Gamma (mobility Gamma (tau_g - 1/2))
    int wait_probe;     // > 0: the TMA kernels' first CTA waits this many tries on a barrier
                        // nothing arrives on (failure-detection test hook); 0 = off
};

// How forces enter the collision (lbm_forcing), and the model (lbm_model).
constexpr int kForcingShift = 0, kForcingGuo = 1;
constexpr int kModelSC = 0, kModelFE = 1;
// Compile-time collision choice of the TMA kernel: the two forcing schemes, or the FE model.
constexpr int kSchemeFE = 2;

// Outputs of the moments kernel (any pointer may be null).
template <class C> struct FieldArgs {
    C* rhoA;
    C* rhoB;
    C* u;    // D planes of N
    C* p;
    double* partials;  // per-CTA diagnostics partial sums (kNumDiag each), or null
    double win_c[3];   // window centre
    double r_in2, r_out2;  // squared window radii (r_in2 < 0: no inner window)
};

// Order of the diagnostics partials (matches lbm_sc_diag).
enum DiagSlot {
    kMassA = 0, kMassB, kMomX, kMomY, kMomZ, kKE, kMaxSpeed, kMinRhoA, kMinRhoB, kNonFinite,
    kInCount, kInRhoA, kInP, kOutCount, kOutRhoA, kOutP, kDropNodes, kNumDiag
};

// Explicitly rounded arithmetic.  The node update is written with these so the
// compiler cannot contract or reorder it: every kernel (register-pipelined,
// cp.async, moments) produces bit-identical results, and the FP32 result can
// be reproduced operation for operation on a CPU.
template <class C> struct Ar;
template <> struct Ar<float> {
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ __forceinline__ static float rcp(float a) { return __frcp_rn(a); }
};
template <> struct Ar<double> {
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ __forceinline__ static double rcp(double a) { return __drcp_rn(a); }
};

// Storage index of cell (x, y, z), x in [-gxo, px - gxo), y in [-gyo, py - gyo).
template <class Args> __device__ __forceinline__ size_t cell(const Args& a, int x, int y, int z) {
    return (size_t)(x + a.gxo) + (size_t)a.px * ((size_t)(y + a.gyo) + (size_t)a.py * (size_t)z);
}

__device__ __forceinline__ int wrap_dec(int x, int n) { return x == 0 ? n - 1 : x - 1; }
__device__ __forceinline__ int wrap_inc(int x, int n) { return x == n - 1 ? 0 : x + 1; }

}  // namespace lbmsc

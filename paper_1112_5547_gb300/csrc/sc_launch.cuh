// Host-side launchers of the Shan-Chen kernels, one instantiation per lattice
// (sc_d2q9.cu, sc_d3q19.cu) so the two compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "sc_common.cuh"

namespace lbmsc {

// Everything a launcher needs to know about one lattice.
struct Plan {
    int lattice;    // 0 D2Q9, 1 D3Q19
    int precision;  // lbm_precision
    int nx, ny, nz;
    long long N;
    int zchunk;     // planes per CTA along z (D3Q19)
    double tau_A, tau_B, G, ref_A, ref_B;
};

// Tile of one CTA (threads = TX * TY, one (x, y) column each).
constexpr int kTX = 32;
constexpr int kTY = 8;

struct MomentsOut {
    void* rhoA;
    void* rhoB;
    void* u;
    void* p;
    double* partials;       // per-CTA diagnostics, or null
    double win[5];          // cx, cy, cz, r_in, r_out (r_in < 0: no inner window)
};

inline dim3 fused_grid(const Plan& p) {
    return dim3((unsigned)((p.nx + kTX - 1) / kTX), (unsigned)((p.ny + kTY - 1) / kTY),
                (unsigned)(p.lattice == 1 ? (p.nz + p.zchunk - 1) / p.zchunk : 1));
}

inline long long fused_blocks(const Plan& p) {
    const dim3 g = fused_grid(p);
    return (long long)g.x * g.y * g.z;
}

cudaError_t d2q9_step(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d2q9_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout,
                      cudaStream_t st);
cudaError_t d2q9_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st);
cudaError_t d3q19_step(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout,
                       cudaStream_t st);
cudaError_t d3q19_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st);
cudaError_t diag_finish(const double* partials, long long nparts, double* out, cudaStream_t st);

}  // namespace lbmsc

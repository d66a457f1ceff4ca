// lbm_sc_diagnostics_noalloc: the diagnostics reduction for callers that
// cannot allocate device memory.  Its per-CTA partial sums live in a
// file-scope static device array instead of a caller workspace; everything
// else (kernels, layout, arithmetic) is the library's existing diagnostics
// path, launched with that array as its scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm_sc.h"
#include "sc_launch.cuh"

namespace {

// Largest diagnostics grid the static scratch holds: one slot of kNumDiag
// doubles per CTA of the moments kernel (2.1 MiB in total on every device that
// loads the library, held until the process exits).
constexpr long long kStaticDiagSlots = 16384;

__device__ __align__(256) double g_diag_scratch[kStaticDiagSlots * lbmsc::kNumDiag];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
cudaError_t device_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_diag_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" LBM_SC_API lbm_status lbm_sc_diagnostics_noalloc(const lbm_sc_params* p, const void* d_populations,
                                                            const lbm_sc_window* window, lbm_sc_diag* d_out,
                                                            void* cuda_stream) {
    if (!p || !d_populations || !d_out) return LBM_ERR_INVALID_ARG;
    if (lbm_sc_workspace_bytes(p) == 0) return LBM_ERR_INVALID_ARG;  // the library's own validation

    lbmsc::Plan pl = {};
    pl.lattice = p->lattice;
    pl.precision = p->precision;
    pl.nx = p->nx;
    pl.ny = p->ny;
    pl.nz = p->nz;
    pl.N = (long long)p->nx * p->ny * p->nz;
    pl.zchunk = p->lattice == LBM_D3Q19 ? p->nz : 1;  // one CTA per tile column: fewest partials
    pl.step_tile = 0;
    pl.step_zchunk = pl.zchunk;
    pl.sm_count = 152;
    pl.tau_A = p->tau_A;
    pl.tau_B = p->tau_B;
    pl.G = p->G;
    pl.ref_A = p->rho_ref_A;
    pl.ref_B = p->rho_ref_B;
    pl.body_A = p->body_A;
    pl.forcing = p->forcing;
    pl.model = p->model;
    pl.kappa = p->kappa;
    pl.gamma = p->gamma;
    lbmsc::storage_geometry(p->nx, p->ny, p->nz, lbmsc::storage_elem_bytes(p->precision), pl.px, pl.py, pl.gxo, pl.gyo, pl.Np);
    pl.err = nullptr;

    const long long parts = lbmsc::fused_blocks(pl);
    if (parts > kStaticDiagSlots) return LBM_ERR_INVALID_ARG;  // larger than the static scratch

    double* scratch = nullptr;
    if (device_scratch(&scratch) != cudaSuccess) return LBM_ERR_CUDA;

    lbmsc::MomentsOut o;
    o.rhoA = o.rhoB = o.u = o.p = nullptr;
    o.partials = scratch;
    if (window) {
        o.win[0] = window->cx;
        o.win[1] = window->cy;
        o.win[2] = window->cz;
        o.win[3] = window->r_in;
        o.win[4] = window->r_out;
    } else {
        o.win[0] = o.win[1] = o.win[2] = 0.0;
        o.win[3] = -1.0;
        o.win[4] = 1e300;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = p->lattice == LBM_D2Q9 ? lbmsc::d2q9_moments(pl, d_populations, o, st)
                                           : lbmsc::d3q19_moments(pl, d_populations, o, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    // lbm_sc_diag is kNumDiag doubles in the fold's slot order
    static_assert(sizeof(lbm_sc_diag) == lbmsc::kNumDiag * sizeof(double), "diag layout");
    e = lbmsc::diag_finish(scratch, parts, reinterpret_cast<double*>(d_out), st);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// C-ABI of the GB300 Shan-Chen lattice Boltzmann library (declared in
// include/lbm_sc.h).  Host code only: validation, workspace carving, stream
// handling and dispatch to the per-lattice launchers.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/lbm_sc.h"
#include "sc_launch.cuh"

using lbmsc::Plan;

// Slabs of z planes lbm_sc_run_host overlaps its host copies with (at most).
constexpr int kIoSlabs = 8;

struct lbm_sc_handle {
    lbm_sc_params params;
    Plan plan;
    char* ws;
    size_t ws_bytes;
    void* buf[2];
    int cur;              // buffer holding the current populations
    double* partials;     // per-CTA diagnostics partials
    double* result;       // folded diagnostics (kNumDiag doubles)
    cudaStream_t stream;
    // lbm_sc_run_host's copy stream and events, created on its first call
    bool io_ready;
    cudaStream_t io_stream;
    cudaEvent_t io_start, io_done, io_in[kIoSlabs], io_out[kIoSlabs];
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int q_of(int lattice) { return lattice == LBM_D2Q9 ? 9 : 19; }
int d_of(int lattice) { return lattice == LBM_D2Q9 ? 2 : 3; }

size_t store_bytes(int precision) { return (size_t)lbmsc::storage_elem_bytes(precision); }

bool rest_offsets(int precision) { return lbmsc::rest_precision(precision); }

size_t compute_bytes(int precision) { return precision == LBM_F64 ? 8 : 4; }

bool valid(const lbm_sc_params* p) {
    if (!p) return false;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return false;
    if (store_bytes(p->precision) == 0) return false;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
    if (p->lattice == LBM_D2Q9 && p->nz != 1) return false;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N >= (1LL << 31)) return false;
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5)) return false;
    if (!(p->G == p->G) || !(p->rho_ref_A == p->rho_ref_A) || !(p->rho_ref_B == p->rho_ref_B)) return false;
    if (!(p->body_A - p->body_A == 0.0)) return false;  // finite
    if (p->forcing != LBM_FORCING_SHIFT && p->forcing != LBM_FORCING_GUO) return false;
    if (p->model != LBM_MODEL_SC && p->model != LBM_MODEL_FE) return false;
    if (p->model == LBM_MODEL_FE) {
        if (p->precision != LBM_F64 && p->precision != LBM_F32) return false;
        if (p->forcing != LBM_FORCING_SHIFT || p->body_A != 0.0) return false;
        if (!(p->kappa - p->kappa == 0.0) || !(p->gamma - p->gamma == 0.0)) return false;  // finite
    }
    return true;
}

// Planes per CTA along z: enough work items to fill the 152 SMs several times
// over, at least min_planes planes per chunk so the two extra density planes
// of each chunk stay cheap.
int pick_zchunk(const lbm_sc_params* p, int tx = lbmsc::kTX, int ty = lbmsc::kTY, long long target = 152LL * 2 * 8,
                int min_planes = 16) {
    if (p->lattice == LBM_D2Q9) return 1;
    const long long tiles = (long long)((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty);
    long long chunks = (target + tiles - 1) / tiles;
    long long max_chunks = p->nz / min_planes;
    if (max_chunks < 1) max_chunks = 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    return (int)((p->nz + chunks - 1) / chunks);
}

Plan make_plan(const lbm_sc_params* p) {
    Plan pl;
    pl.lattice = p->lattice;
    pl.precision = p->precision;
    pl.nx = p->nx;
    pl.ny = p->ny;
    pl.nz = p->nz;
    pl.N = (long long)p->nx * p->ny * p->nz;
    pl.zchunk = pick_zchunk(p);
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
    // a negative kappa selects the gradient coefficient of Eq. FEtau, g cs2^2 / 4
    pl.kappa = p->kappa < 0.0 ? p->G / 36.0 : p->kappa;
    pl.gamma = p->gamma;
    lbmsc::storage_geometry(p->nx, p->ny, p->nz, (int)store_bytes(p->precision), pl.px, pl.py, pl.gxo, pl.gyo,
                            pl.Np);
    return pl;
}

// One population buffer: 2 species x Q ghost-padded planes (Q paired planes
// and one float2 density plane for the rest-offset precisions).
size_t population_bytes(const lbm_sc_params* p) {
    int px, py, gxo, gyo;
    long long Np;
    lbmsc::storage_geometry(p->nx, p->ny, p->nz, (int)store_bytes(p->precision), px, py, gxo, gyo, Np);
    return (size_t)lbmsc::population_planes(p->lattice, p->precision) * (size_t)Np * store_bytes(p->precision) +
           (rest_offsets(p->precision) ? (size_t)Np * 8 : 0);
}

size_t partial_bytes(const Plan& pl) {
    return (size_t)lbmsc::fused_blocks(pl) * lbmsc::kNumDiag * sizeof(double);
}

lbm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

cudaError_t launch_step(const Plan& pl, const void* fin, void* fout, cudaStream_t st) {
    return pl.lattice == LBM_D2Q9 ? lbmsc::d2q9_step(pl, fin, fout, st) : lbmsc::d3q19_step(pl, fin, fout, st);
}

cudaError_t launch_init(const Plan& pl, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st) {
    return pl.lattice == LBM_D2Q9 ? lbmsc::d2q9_init(pl, rA, rB, u, fout, st)
                                  : lbmsc::d3q19_init(pl, rA, rB, u, fout, st);
}

cudaError_t launch_moments(const Plan& pl, const void* fin, const lbmsc::MomentsOut& o, cudaStream_t st) {
    return pl.lattice == LBM_D2Q9 ? lbmsc::d2q9_moments(pl, fin, o, st) : lbmsc::d3q19_moments(pl, fin, o, st);
}

}  // namespace

extern "C" {

size_t lbm_sc_workspace_bytes(const lbm_sc_params* p) {
    if (!valid(p)) return 0;
    const Plan pl = make_plan(p);
    // each population buffer is followed by at least kAlign bytes of padding, so a
    // 4-byte-word read around the last 16-bit value stays inside the buffer's span
    return 2 * align_up(population_bytes(p) + kAlign) + align_up(partial_bytes(pl)) +
           align_up(lbmsc::kNumDiag * sizeof(double)) + kAlign /* error word */;
}

lbm_status lbm_sc_create(const lbm_sc_params* p, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                         lbm_sc_handle** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid(p) || !d_workspace) return LBM_ERR_INVALID_ARG;
    if (((uintptr_t)d_workspace) % kAlign != 0) return LBM_ERR_INVALID_ARG;
    const size_t need = lbm_sc_workspace_bytes(p);
    if (workspace_bytes < need) return LBM_ERR_OUT_OF_MEMORY;
    lbm_sc_handle* h = static_cast<lbm_sc_handle*>(malloc(sizeof(lbm_sc_handle)));
    if (!h) return LBM_ERR_OUT_OF_MEMORY;
    memset(h, 0, sizeof(*h));
    h->params = *p;
    h->plan = make_plan(p);
    h->ws = static_cast<char*>(d_workspace);
    h->ws_bytes = workspace_bytes;
    const size_t pb = align_up(population_bytes(p) + kAlign);
    h->buf[0] = h->ws;
    h->buf[1] = h->ws + pb;
    h->partials = reinterpret_cast<double*>(h->ws + 2 * pb);
    h->result = reinterpret_cast<double*>(h->ws + 2 * pb + align_up(partial_bytes(h->plan)));
    h->plan.err = reinterpret_cast<int*>(h->ws + 2 * pb + align_up(partial_bytes(h->plan)) +
                                         align_up(lbmsc::kNumDiag * sizeof(double)));
    h->cur = 0;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    {
        // multiprocessor count for persistent grids (host query, no allocation); keep
        // the default when no device is present (host-only use)
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            h->plan.sm_count = sms;
        else
            cudaGetLastError();
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_sc_set_tuning(lbm_sc_handle* h, const lbm_sc_tuning* t) {
    if (!h || !t || t->zchunk < 0) return LBM_ERR_INVALID_ARG;
    if (!lbmsc::tile_fits(t->tile, h->plan)) return LBM_ERR_INVALID_ARG;
    const lbmsc::TileShape ts = lbmsc::kTiles[t->tile];
    h->plan.step_tile = t->tile;
    int zc = t->zchunk != 0 ? t->zchunk : pick_zchunk(&h->params, ts.tx, ts.ty);
    if (h->params.lattice == LBM_D2Q9 || zc > h->params.nz) zc = h->params.lattice == LBM_D2Q9 ? 1 : h->params.nz;
    h->plan.step_zchunk = zc;
    return LBM_OK;
}

lbm_status lbm_sc_get_tuning(const lbm_sc_handle* h, lbm_sc_tuning* t) {
    if (!h || !t) return LBM_ERR_INVALID_ARG;
    t->tile = h->plan.step_tile;
    t->zchunk = h->plan.step_zchunk;
    return LBM_OK;
}

lbm_status lbm_sc_set_wait_probe(lbm_sc_handle* h, int tries) {
    if (!h || tries < 0) return LBM_ERR_INVALID_ARG;
    h->plan.wait_probe = tries;
    return LBM_OK;
}

lbm_status lbm_sc_error_word(lbm_sc_handle* h, int* host_out) {
    if (!h || !host_out) return LBM_ERR_INVALID_ARG;
    int w = 0;
    if (cudaMemcpyAsync(&w, h->plan.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    *host_out = w;
    return LBM_OK;
}

lbm_status lbm_sc_set_stream(lbm_sc_handle* h, void* cuda_stream) {
    if (!h) return LBM_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

lbm_status lbm_sc_init_fields(lbm_sc_handle* h, const void* d_rhoA, const void* d_rhoB, const void* d_u) {
    if (!h || !d_rhoA || !d_rhoB) return LBM_ERR_INVALID_ARG;
    h->cur = 0;
    if (cudaMemsetAsync(h->plan.err, 0, sizeof(int), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    return cuda_status(launch_init(h->plan, d_rhoA, d_rhoB, d_u, h->buf[0], h->stream));
}

lbm_status lbm_sc_step(lbm_sc_handle* h, int nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_INVALID_ARG;
    for (int t = 0; t < nsteps; ++t) {
        const cudaError_t e = launch_step(h->plan, h->buf[h->cur], h->buf[1 - h->cur], h->stream);
        if (e != cudaSuccess) return LBM_ERR_CUDA;
        h->cur = 1 - h->cur;
    }
    return LBM_OK;
}

lbm_status lbm_sc_moments(lbm_sc_handle* h, void* d_rhoA, void* d_rhoB, void* d_u, void* d_p) {
    if (!h) return LBM_ERR_INVALID_ARG;
    if (!d_rhoA && !d_rhoB && !d_u && !d_p) return LBM_OK;
    lbmsc::MomentsOut o;
    o.rhoA = d_rhoA;
    o.rhoB = d_rhoB;
    o.u = d_u;
    o.p = d_p;
    o.partials = nullptr;
    o.win[0] = o.win[1] = o.win[2] = 0.0;
    o.win[3] = -1.0;
    o.win[4] = 1e300;
    return cuda_status(launch_moments(h->plan, h->buf[h->cur], o, h->stream));
}

lbm_status lbm_sc_diagnostics(lbm_sc_handle* h, const lbm_sc_window* window, lbm_sc_diag* host_out) {
    if (!h || !host_out) return LBM_ERR_INVALID_ARG;
    lbmsc::MomentsOut o;
    o.rhoA = o.rhoB = o.u = o.p = nullptr;
    o.partials = h->partials;
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
    cudaError_t e = launch_moments(h->plan, h->buf[h->cur], o, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    e = lbmsc::diag_finish(h->partials, lbmsc::fused_blocks(h->plan), h->result, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    double r[lbmsc::kNumDiag];
    int err_word = 0;
    e = cudaMemcpyAsync(r, h->result, sizeof(r), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    e = cudaMemcpyAsync(&err_word, h->plan.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    host_out->mass_A = r[lbmsc::kMassA];
    host_out->mass_B = r[lbmsc::kMassB];
    host_out->momentum[0] = r[lbmsc::kMomX];
    host_out->momentum[1] = r[lbmsc::kMomY];
    host_out->momentum[2] = r[lbmsc::kMomZ];
    host_out->kinetic_energy = r[lbmsc::kKE];
    host_out->max_speed = r[lbmsc::kMaxSpeed];
    host_out->min_rho_A = r[lbmsc::kMinRhoA];
    host_out->min_rho_B = r[lbmsc::kMinRhoB];
    host_out->nonfinite = r[lbmsc::kNonFinite];
    host_out->in_count = r[lbmsc::kInCount];
    host_out->in_rho_A = r[lbmsc::kInRhoA];
    host_out->in_p = r[lbmsc::kInP];
    host_out->out_count = r[lbmsc::kOutCount];
    host_out->out_rho_A = r[lbmsc::kOutRhoA];
    host_out->out_p = r[lbmsc::kOutP];
    host_out->droplet_nodes = r[lbmsc::kDropNodes];
    if (err_word != 0) return LBM_ERR_TIMEOUT;
    if (host_out->nonfinite > 0 || !(host_out->min_rho_A > 0) || !(host_out->min_rho_B > 0))
        return LBM_ERR_UNSTABLE;
    return LBM_OK;
}

size_t lbm_sc_host_staging_bytes(const lbm_sc_params* p) {
    if (!valid(p)) return 0;
    const size_t field = align_up((size_t)p->nx * p->ny * p->nz * compute_bytes(p->precision));
    return field * (size_t)(3 + d_of(p->lattice));
}

namespace {

// The copy stream and events of lbm_sc_run_host (no device memory), made once per handle.
cudaError_t io_setup(lbm_sc_handle* h) {
    if (h->io_ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking);
    cudaEvent_t* evs[2 + 2 * kIoSlabs];
    int n = 0;
    evs[n++] = &h->io_start;
    evs[n++] = &h->io_done;
    for (int k = 0; k < kIoSlabs; ++k) {
        evs[n++] = &h->io_in[k];
        evs[n++] = &h->io_out[k];
    }
    for (int k = 0; k < n && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(evs[k], cudaEventDisableTiming);
    if (e == cudaSuccess) h->io_ready = true;
    return e;
}

void io_release(lbm_sc_handle* h) {
    if (!h->io_ready) return;
    cudaEventDestroy(h->io_start);
    cudaEventDestroy(h->io_done);
    for (int k = 0; k < kIoSlabs; ++k) {
        cudaEventDestroy(h->io_in[k]);
        cudaEventDestroy(h->io_out[k]);
    }
    cudaStreamDestroy(h->io_stream);
    h->io_ready = false;
}

}  // namespace

namespace {

// Driver calls of lbm_sc_host_alloc's virtual-memory allocation, reached through
// the runtime's driver entry points (no link against the driver library).
struct HostVmm {
    PFN_cuMemGetAllocationGranularity_v10020 granularity = nullptr;
    PFN_cuMemCreate_v10020 create = nullptr;
    PFN_cuMemRelease_v10020 release = nullptr;
    PFN_cuMemAddressReserve_v10020 reserve = nullptr;
    PFN_cuMemAddressFree_v10020 address_free = nullptr;
    PFN_cuMemMap_v10020 map = nullptr;
    PFN_cuMemUnmap_v10020 unmap = nullptr;
    PFN_cuMemSetAccess_v10020 set_access = nullptr;
    bool ok = false;
};

void* driver_entry(const char* name) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return ptr;
}

const HostVmm& host_vmm() {
    static const HostVmm v = [] {
        HostVmm t;
        t.granularity = (PFN_cuMemGetAllocationGranularity_v10020)driver_entry("cuMemGetAllocationGranularity");
        t.create = (PFN_cuMemCreate_v10020)driver_entry("cuMemCreate");
        t.release = (PFN_cuMemRelease_v10020)driver_entry("cuMemRelease");
        t.reserve = (PFN_cuMemAddressReserve_v10020)driver_entry("cuMemAddressReserve");
        t.address_free = (PFN_cuMemAddressFree_v10020)driver_entry("cuMemAddressFree");
        t.map = (PFN_cuMemMap_v10020)driver_entry("cuMemMap");
        t.unmap = (PFN_cuMemUnmap_v10020)driver_entry("cuMemUnmap");
        t.set_access = (PFN_cuMemSetAccess_v10020)driver_entry("cuMemSetAccess");
        t.ok = t.granularity && t.create && t.release && t.reserve && t.address_free && t.map && t.unmap &&
               t.set_access;
        return t;
    }();
    return v;
}

// Pinned host memory on the host NUMA node nearest the current device (node 0
// where the system has no NUMA), and the mapping size of a buffer of `bytes`
// (whole allocation granules).
bool host_prop(CUmemAllocationProp& prop, int& device, size_t bytes, size_t& size) {
    const HostVmm& v = host_vmm();
    if (!v.ok || cudaFree(nullptr) != cudaSuccess || cudaGetDevice(&device) != cudaSuccess) return false;
    int numa = -1;
    if (cudaDeviceGetAttribute(&numa, cudaDevAttrHostNumaId, device) != cudaSuccess || numa < 0) numa = 0;
    memset(&prop, 0, sizeof(prop));
    prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    prop.location.type = CU_MEM_LOCATION_TYPE_HOST_NUMA;
    prop.location.id = numa;
    size_t gran = 0;
    if (v.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || gran == 0) return false;
    if (bytes > SIZE_MAX - gran) return false;
    size = (bytes + gran - 1) / gran * gran;
    return true;
}

}  // namespace

lbm_status lbm_sc_host_alloc(size_t bytes, void** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (bytes == 0) return LBM_ERR_INVALID_ARG;
    CUmemAllocationProp prop;
    int device = 0;
    size_t size = 0;
    if (!host_prop(prop, device, bytes, size)) return LBM_ERR_CUDA;
    const HostVmm& v = host_vmm();
    CUmemGenericAllocationHandle handle;
    const CUresult cr = v.create(&handle, size, &prop, 0);
    if (cr != CUDA_SUCCESS) return cr == CUDA_ERROR_OUT_OF_MEMORY ? LBM_ERR_OUT_OF_MEMORY : LBM_ERR_CUDA;
    CUdeviceptr va = 0;
    if (v.reserve(&va, size, 0, 0, 0) != CUDA_SUCCESS) {
        v.release(handle);
        return LBM_ERR_CUDA;
    }
    const bool mapped = v.map(va, size, 0, handle, 0) == CUDA_SUCCESS;
    v.release(handle);  // the mapping keeps the memory until it is unmapped
    CUmemAccessDesc access[2];
    memset(access, 0, sizeof(access));
    access[0].location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    access[0].location.id = device;
    access[0].flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    access[1].location = prop.location;
    access[1].flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    if (!mapped || v.set_access(va, size, access, 2) != CUDA_SUCCESS) {
        if (mapped) v.unmap(va, size);
        v.address_free(va, size);
        return LBM_ERR_CUDA;
    }
    memset(reinterpret_cast<void*>(va), 0, size);
    *out = reinterpret_cast<void*>(va);
    return LBM_OK;
}

lbm_status lbm_sc_host_free(void* p, size_t bytes) {
    if (!p) return LBM_OK;
    if (bytes == 0) return LBM_ERR_INVALID_ARG;
    CUmemAllocationProp prop;
    int device = 0;
    size_t size = 0;
    if (!host_prop(prop, device, bytes, size)) return LBM_ERR_CUDA;
    const HostVmm& v = host_vmm();
    const CUdeviceptr va = reinterpret_cast<CUdeviceptr>(p);
    const bool unmapped = v.unmap(va, size) == CUDA_SUCCESS;
    const bool freed = v.address_free(va, size) == CUDA_SUCCESS;
    return unmapped && freed ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_sc_run_host(lbm_sc_handle* h, void* d_staging, size_t staging_bytes, const void* h_rhoA,
                           const void* h_rhoB, const void* h_u, int nsteps, void* h_rhoA_out, void* h_rhoB_out,
                           void* h_u_out, void* h_p_out) {
    if (!h || !d_staging || !h_rhoA || !h_rhoB || nsteps < 0) return LBM_ERR_INVALID_ARG;
    if (((uintptr_t)d_staging) % kAlign != 0) return LBM_ERR_INVALID_ARG;
    if (staging_bytes < lbm_sc_host_staging_bytes(&h->params)) return LBM_ERR_OUT_OF_MEMORY;
    if (io_setup(h) != cudaSuccess) return LBM_ERR_CUDA;
    const size_t esz = compute_bytes(h->params.precision);
    const size_t fb = (size_t)h->plan.N * esz;
    const size_t field = align_up(fb);
    const int D = d_of(h->params.lattice);
    const int nz = h->params.nz;
    const size_t plane = (size_t)h->params.nx * h->params.ny * esz;  // bytes of one z plane of a field
    char* s = static_cast<char*>(d_staging);
    char* dA = s;
    char* dB = s + field;
    char* dP = s + 2 * field;
    char* dU = s + 3 * field;  // D consecutive planes of fb bytes
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
    const cudaStream_t ms = h->stream, cs = h->io_stream;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // z slabs: the host copies of one slab overlap the kernels of another.
    // Moments slabs are whole chunks of 32 planes (their own z chunking).
    Plan mp = h->plan;
    if (nz >= 64) mp.zchunk = 32;
    const int chunks = (nz + mp.zchunk - 1) / mp.zchunk;
    const int nslab = nz >= 64 ? (chunks < kIoSlabs ? chunks : kIoSlabs) : 1;  // no empty slab
    int zb[kIoSlabs + 1];
    for (int k = 0; k <= nslab; ++k) zb[k] = (int)((long long)chunks * k / nslab) * mp.zchunk;
    zb[nslab] = nz;
    auto copy_planes = [&](char* dev, const void* host, int z0, int z1, int nfield, cudaMemcpyKind kind) {
        // planes [z0, z1) of nfield consecutive fields of fb bytes each
        for (int f = 0; f < nfield; ++f) {
            const size_t off = (size_t)f * fb + (size_t)z0 * plane, n = (size_t)(z1 - z0) * plane;
            cudaError_t e = kind == h2d ? cudaMemcpyAsync(dev + off, static_cast<const char*>(host) + off, n, kind, cs)
                                        : cudaMemcpyAsync(static_cast<char*>(const_cast<void*>(host)) + off, dev + off,
                                                          n, kind, cs);
            if (e != cudaSuccess) return false;
        }
        return true;
    };
    // inputs: the copy stream starts after the work already on the handle's
    // stream (the staging may still be in use), last plane first (slab 0's
    // periodic neighbour), then slab by slab; the init of slab k starts once
    // slab k + 1 (its z + 1 neighbours) has landed
    if (!ok(cudaEventRecord(h->io_start, ms)) || !ok(cudaStreamWaitEvent(cs, h->io_start, 0))) return LBM_ERR_CUDA;
    if (!copy_planes(dA, h_rhoA, nz - 1, nz, 1, h2d) || !copy_planes(dB, h_rhoB, nz - 1, nz, 1, h2d) ||
        (h_u && !copy_planes(dU, h_u, nz - 1, nz, D, h2d)))
        return LBM_ERR_CUDA;
    for (int k = 0; k < nslab; ++k) {
        if (!copy_planes(dA, h_rhoA, zb[k], zb[k + 1], 1, h2d) || !copy_planes(dB, h_rhoB, zb[k], zb[k + 1], 1, h2d) ||
            (h_u && !copy_planes(dU, h_u, zb[k], zb[k + 1], D, h2d)))
            return LBM_ERR_CUDA;
        if (!ok(cudaEventRecord(h->io_in[k], cs))) return LBM_ERR_CUDA;
    }
    h->cur = 0;
    if (!ok(cudaMemsetAsync(h->plan.err, 0, sizeof(int), ms))) return LBM_ERR_CUDA;
    for (int k = 0; k < nslab; ++k) {
        if (!ok(cudaStreamWaitEvent(ms, h->io_in[k + 1 < nslab ? k + 1 : nslab - 1], 0))) return LBM_ERR_CUDA;
        const cudaError_t e = h->plan.lattice == LBM_D2Q9
                                  ? lbmsc::d2q9_init(h->plan, dA, dB, h_u ? dU : nullptr, h->buf[0], ms, zb[k], zb[k + 1])
                                  : lbmsc::d3q19_init(h->plan, dA, dB, h_u ? dU : nullptr, h->buf[0], ms, zb[k], zb[k + 1]);
        if (e != cudaSuccess) return LBM_ERR_CUDA;
    }
    lbm_status st = lbm_sc_step(h, nsteps);
    if (st != LBM_OK) return st;
    // outputs: the moments of slab k, then its copies on the copy stream while slab k + 1 computes
    for (int k = 0; k < nslab; ++k) {
        lbmsc::MomentsOut o;
        o.rhoA = h_rhoA_out ? dA : nullptr;
        o.rhoB = h_rhoB_out ? dB : nullptr;
        o.u = h_u_out ? dU : nullptr;
        o.p = h_p_out ? dP : nullptr;
        o.partials = nullptr;
        o.win[0] = o.win[1] = o.win[2] = 0.0;
        o.win[3] = -1.0;
        o.win[4] = 1e300;
        o.zlo = zb[k];
        o.zhi = zb[k + 1];
        if (launch_moments(mp, h->buf[h->cur], o, ms) != cudaSuccess) return LBM_ERR_CUDA;
        if (!ok(cudaEventRecord(h->io_out[k], ms)) || !ok(cudaStreamWaitEvent(cs, h->io_out[k], 0))) return LBM_ERR_CUDA;
        if ((h_rhoA_out && !copy_planes(dA, h_rhoA_out, zb[k], zb[k + 1], 1, d2h)) ||
            (h_rhoB_out && !copy_planes(dB, h_rhoB_out, zb[k], zb[k + 1], 1, d2h)) ||
            (h_u_out && !copy_planes(dU, h_u_out, zb[k], zb[k + 1], D, d2h)) ||
            (h_p_out && !copy_planes(dP, h_p_out, zb[k], zb[k + 1], 1, d2h)))
            return LBM_ERR_CUDA;
    }
    if (!ok(cudaEventRecord(h->io_done, cs)) || !ok(cudaStreamWaitEvent(ms, h->io_done, 0))) return LBM_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(ms));
}

lbm_status lbm_sc_layout(const lbm_sc_handle* h, int* elem_bytes, int* q, int* pitch_x, int* pitch_y, int* ghost_x,
                         int* ghost_y, const void** d_populations) {
    if (!h) return LBM_ERR_INVALID_ARG;
    if (elem_bytes) *elem_bytes = (int)store_bytes(h->params.precision);
    if (q) *q = q_of(h->params.lattice);
    if (pitch_x) *pitch_x = h->plan.px;
    if (pitch_y) *pitch_y = h->plan.py;
    if (ghost_x) *ghost_x = h->plan.gxo;
    if (ghost_y) *ghost_y = h->plan.gyo;
    if (d_populations) *d_populations = h->buf[h->cur];
    return LBM_OK;
}

void lbm_sc_destroy(lbm_sc_handle* h) {
    if (!h) return;
    io_release(h);
    free(h);
}

const char* lbm_sc_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_ERR_INVALID_ARG: return "LBM_ERR_INVALID_ARG: invalid parameter, pointer or size";
        case LBM_ERR_OUT_OF_MEMORY: return "LBM_ERR_OUT_OF_MEMORY: workspace too small or host allocation failed";
        case LBM_ERR_CUDA: return "LBM_ERR_CUDA: a CUDA call or kernel launch failed";
        case LBM_ERR_UNSTABLE: return "LBM_ERR_UNSTABLE: non-finite value or non-positive density";
        case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT: bounded device wait expired";
    }
    return "unknown lbm_status";
}

}  // extern "C"

// ---- ragged batch -------------------------------------------------------------
#include <algorithm>
#include <vector>

#include "sc_batch_launch.h"

struct lbm_sc_batch {
    std::vector<lbm_sc_handle*> h;
    std::vector<int> cur0;
    int lattice, precision, tile, zchunk, graph_steps;
    void* d_lats;
    lbmsc::BatchItem* d_items;
    int* d_ctr;  // work-queue counters of the batch kernels
    int nitems;
    int parity;
    int sm_count;
    cudaStream_t stream;
    cudaGraphExec_t graph[2];  // graph_steps launches starting at parity 0 / 1
};

namespace {

bool batch_valid(lbm_sc_handle* const* handles, int n, int tile, int zchunk) {
    if (!handles || n < 1 || tile < 0 || tile >= lbmsc::kNumBatchTiles || zchunk < 0) return false;
    for (int k = 0; k < n; ++k) {
        if (!handles[k]) return false;
        if (handles[k]->params.lattice != handles[0]->params.lattice ||
            handles[k]->params.precision != handles[0]->params.precision)
            return false;
        if (!lbmsc::batch_tile_fits(tile, handles[k]->plan)) return false;
    }
    return true;
}

int batch_zchunk(const lbm_sc_handle* h, int zchunk) {
    if (h->params.lattice == LBM_D2Q9) return 1;
    const int zc = zchunk == 0 ? 32 : zchunk;
    return zc > h->params.nz ? h->params.nz : zc;
}

std::vector<lbmsc::BatchItem> batch_items(lbm_sc_handle* const* handles, int n, int tile, int zchunk) {
    std::vector<lbmsc::BatchItem> items;
    std::vector<int> len;
    for (int k = 0; k < n; ++k) {
        const lbm_sc_params& p = handles[k]->params;
        int tx, ty;
        lbmsc::batch_item_tile(tile, handles[k]->plan, tx, ty);
        const int zc = batch_zchunk(handles[k], zchunk);
        for (int z0 = 0; z0 < p.nz; z0 += zc)
            for (int y0 = 0; y0 < p.ny; y0 += ty)
                for (int x0 = 0; x0 < p.nx; x0 += tx) {
                    items.push_back({k, x0, y0, z0});
                    len.push_back(std::min(zc, p.nz - z0));
                }
    }
    // longest items first, so the walk (counter or block order) ends with the short ones
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return len[a] > len[b]; });
    std::vector<lbmsc::BatchItem> sorted;
    sorted.reserve(items.size());
    for (size_t i : order) sorted.push_back(items[i]);
    return sorted;
}

cudaError_t batch_launch_steps(lbm_sc_batch* b, int nsteps) {
    for (int t = 0; t < nsteps; ++t) {
        const cudaError_t e = lbmsc::batch_step(b->lattice, b->precision, b->tile, b->d_lats, b->d_items, b->nitems,
                                                b->parity, b->sm_count, b->d_ctr, b->stream);
        if (e != cudaSuccess) return e;
        b->parity ^= 1;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t lbm_sc_batch_workspace_bytes(lbm_sc_handle* const* handles, int n, int tile, int zchunk) {
    if (!batch_valid(handles, n, tile, zchunk)) return 0;
    const size_t items = batch_items(handles, n, tile, zchunk).size();
    return align_up(lbmsc::batch_lattice_bytes(handles[0]->params.precision, tile) * (size_t)n) +
           align_up(items * sizeof(lbmsc::BatchItem)) + kAlign /* queue counters */;
}

lbm_status lbm_sc_batch_create(lbm_sc_handle* const* handles, int n, int tile, int zchunk, int graph_steps,
                               void* d_workspace, size_t workspace_bytes, void* cuda_stream, lbm_sc_batch** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!batch_valid(handles, n, tile, zchunk) || !d_workspace || graph_steps < 0 || graph_steps % 2 != 0)
        return LBM_ERR_INVALID_ARG;
    if (((uintptr_t)d_workspace) % kAlign != 0) return LBM_ERR_INVALID_ARG;
    if (workspace_bytes < lbm_sc_batch_workspace_bytes(handles, n, tile, zchunk)) return LBM_ERR_OUT_OF_MEMORY;
    lbm_sc_batch* b = new (std::nothrow) lbm_sc_batch();
    if (!b) return LBM_ERR_OUT_OF_MEMORY;
    b->h.assign(handles, handles + n);
    b->lattice = handles[0]->params.lattice;
    b->precision = handles[0]->params.precision;
    b->tile = tile;
    b->zchunk = zchunk;
    b->graph_steps = graph_steps;
    b->parity = 0;
    b->sm_count = handles[0]->plan.sm_count;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->graph[0] = b->graph[1] = nullptr;
    const size_t lb = lbmsc::batch_lattice_bytes(b->precision, tile);
    std::vector<unsigned char> lats(lb * (size_t)n);
    for (int k = 0; k < n; ++k) {
        b->cur0.push_back(handles[k]->cur);
        if (lbmsc::batch_lattice_fill(handles[k]->plan, handles[k]->buf[0], handles[k]->buf[1], handles[k]->cur,
                                      batch_zchunk(handles[k], zchunk), tile, lats.data() + lb * k) != cudaSuccess) {
            delete b;
            return LBM_ERR_INVALID_ARG;
        }
    }
    const std::vector<lbmsc::BatchItem> items = batch_items(handles, n, tile, zchunk);
    b->nitems = (int)items.size();
    char* ws = static_cast<char*>(d_workspace);
    b->d_lats = ws;
    b->d_items = reinterpret_cast<lbmsc::BatchItem*>(ws + align_up(lb * (size_t)n));
    b->d_ctr = reinterpret_cast<int*>(ws + align_up(lb * (size_t)n) + align_up(items.size() * sizeof(lbmsc::BatchItem)));
    cudaError_t e = cudaMemcpyAsync(b->d_lats, lats.data(), lats.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctr, 0, 2 * sizeof(int), b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(lbmsc::BatchItem),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host staging goes out of scope
    // kernel attributes and occupancy are set up now, outside any later stream capture
    if (e == cudaSuccess)
        e = lbmsc::batch_step(b->lattice, b->precision, tile, b->d_lats, b->d_items, 0, 0, b->sm_count, b->d_ctr,
                              b->stream);
    if (e != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_sc_batch_step(lbm_sc_batch* b, int nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
    for (size_t k = 0; k < b->h.size(); ++k)
        if (b->h[k]->cur != (b->cur0[k] ^ b->parity)) return LBM_ERR_INVALID_ARG;  // stepped outside the batch
    int left = nsteps;
    if (b->graph_steps > 0 && b->stream != nullptr) {
        while (left >= b->graph_steps) {
            const int p = b->parity;
            if (!b->graph[p]) {
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return LBM_ERR_CUDA;
                const cudaError_t le = batch_launch_steps(b, b->graph_steps);
                const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
                b->parity = p;  // capturing did not advance the lattices
                if (le != cudaSuccess || ce != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return LBM_ERR_CUDA;
                }
                const cudaError_t ie = cudaGraphInstantiate(&b->graph[p], g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) {
                    b->graph[p] = nullptr;
                    return LBM_ERR_CUDA;
                }
            }
            if (cudaGraphLaunch(b->graph[p], b->stream) != cudaSuccess) return LBM_ERR_CUDA;
            // graph_steps is even: the parity is back where it started
            left -= b->graph_steps;
        }
    }
    if (batch_launch_steps(b, left) != cudaSuccess) return LBM_ERR_CUDA;
    for (size_t k = 0; k < b->h.size(); ++k) b->h[k]->cur = b->cur0[k] ^ b->parity;
    return LBM_OK;
}

void lbm_sc_batch_destroy(lbm_sc_batch* b) {
    if (!b) return;
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
    delete b;
}

}  // extern "C"

// Host-side launchers of the Shan-Chen kernels, one instantiation per lattice
// (sc_d2q9.cu, sc_d3q19.cu) so the two compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "sc_common.cuh"

namespace lbmsc {

// Everything a launcher needs to know about one lattice.
struct Plan {
    int lattice;    // 0 D2Q9, 1 D3Q19
    int precision;  // lbm_precision (4, 5: rest-offset 16-bit storage)
    int nx, ny, nz;
    long long N;
    int zchunk;     // planes per CTA along z for the moments kernel (D3Q19)
    int step_tile;  // index into kTiles for the step kernel
    int step_zchunk;
    int sm_count;   // multiprocessors of the device (persistent grids)
    double tau_A, tau_B, G, ref_A, ref_B;
    double body_A;         // Kolmogorov forcing amplitude (Eq. kolmo); 0 = none
    int forcing;           // kForcingShift or kForcingGuo
    int model;             // kModelSC or kModelFE
    double kappa, gamma;   // FE: gradient coefficient, Gamma
    int px, py, gxo, gyo;  // ghost-padded storage geometry (see LatticeArgs)
    long long Np;          // values per population plane
    int* err;              // device error word (set by a kernel whose bounded wait expired)
    int wait_probe;        // failure-detection test hook (lbm_sc_set_wait_probe); 0 = off
};

// Bytes of one stored element for a precision (lbm_precision): FP64 8, FP32 4,
// reference-offset 16-bit 2, paired rest-offset 16-bit 4 (both species of one
// direction in one word); 0 for an unknown precision.
inline int storage_elem_bytes(int precision) {
    switch (precision) {
        case 0: return 8;
        case 1: return 4;
        case 2:
        case 3: return 2;
        case 4:
        case 5: return 4;
    }
    return 0;
}
inline bool rest_precision(int precision) { return precision == 4 || precision == 5; }
// Population planes of one buffer: 2 Q (a plane per species and direction), or
// Q paired planes for the rest-offset precisions (which add one plane of float2
// densities after them).
inline int population_planes(int lattice, int precision) {
    const int q = lattice == 0 ? 9 : 19;
    return rest_precision(precision) ? q : 2 * q;
}

// Ghost-padded storage geometry for a lattice.  Node x = 0 sits 128 bytes into
// each row and the row pitch is a multiple of 128 bytes, so every warp's row
// segment of a tile starting at a multiple of 32 nodes is whole cache lines
// (a misaligned store would leave partial sectors shared with the next CTA's
// tile).  The ghost columns x = -2, -1, nx, nx+1 and rows y = -2, -1, ny, ny+1
// hold periodic images; on lattices at least a sector wide the images fill the
// whole 32-byte sector on each side of the row (store_node), and the row has
// room for it, which also keeps 16-byte-aligned TMA boxes of x0 - 16 bytes ..
// x0 + TX + 16 bytes inside the row.
inline void storage_geometry(int nx, int ny, int nz, int elem_bytes, int& px, int& py, int& gxo, int& gyo,
                             long long& Np) {
    const int line = 128 / elem_bytes;  // values per 128 bytes
    // right margin: the 32-byte sector of ghost images beyond column nx - 1
    // (store_node), which also covers the 16-byte pad of the TMA boxes
    const int margin = 32 / elem_bytes;
    gxo = line;
    gyo = 2;
    px = (nx + gxo + margin + line - 1) / line * line;
    py = ny + 2 * gyo;
    Np = (long long)px * py * nz;
}

// Tile of one CTA (threads = TX * TY, one (x, y) column each) for the moments
// kernel, and the tiles the step kernel can be launched with (autotuned).
constexpr int kTX = 32;
constexpr int kTY = 8;
// kind 0: register-pipelined kernel (every lattice and precision);
// kind 3: low-register kernel that re-pulls a plane for its collision, with
//         `stages` = CTAs per SM requested from the register allocator;
// kind 4: register-pipelined kernel with three planes of pulls in registers
//         (D3Q19, 32-bit and 16-bit storage), `stages` = CTAs per SM;
// kind 5: TMA-fed kernel with `stages` shared-memory stages (D3Q19, FP32
//         storage, lattices at least one tile wide in x and y), launched as
//         clusters of cx x cy neighbouring tiles (co-scheduled on one GPC, so
//         the halo lines the tiles share are fetched into one die's L2);
// kind 6: the TMA-fed kernel for 16-bit storage (D3Q19; the rest-offset
//         modes also stage boxes of the FP32 node densities).
// Retired ids (kind kRetired) keep their slot so that the other ids stay
// stable; every call that names one is rejected.  They were measured slower
// than the kinds above at every size and removed: 5-7, a persistent kernel
// copying every pull with cp.async into thread-private stages; 8-10, a
// software-pipelined kernel holding two planes in registers and shared memory;
// 26-29, 64x4 / 32x8 TMA tiles with 128-byte or no L2 promotion (no change
// against the 256-byte promotion every kept tile uses).
constexpr int kRetired = -1;
// promo: L2 promotion of the tensor copies (3: 256 bytes fetched per L2 miss);
// minb: CTAs per SM the register allocation is made for (TMA kinds; two
// CTAs per SM let one CTA's per-plane barrier overlap the other's work).
struct TileShape { int tx, ty, kind, stages, cx = 1, cy = 1, promo = 3, minb = 1; };
constexpr int kNumTiles = 45;
constexpr TileShape kTiles[kNumTiles] = {
    {32, 8, 0, 0},       {32, 16, 0, 0},      {64, 8, 0, 0},       {32, 4, 0, 0},       {64, 4, 0, 0},
    {32, 8, kRetired, 0}, {32, 8, kRetired, 0}, {64, 4, kRetired, 0}, {32, 8, kRetired, 0}, {64, 4, kRetired, 0},
    {32, 4, kRetired, 0}, {32, 4, 3, 6},       {32, 8, 3, 3},       {64, 4, 3, 3},       {32, 4, 3, 4},
    {32, 4, 4, 3},       {32, 8, 4, 1},       {16, 8, 4, 3},       {32, 8, 5, 3},       {64, 4, 5, 3},
    {32, 4, 5, 4},       {32, 4, 5, 2},       {64, 4, 5, 3, 1, 2}, {64, 4, 5, 3, 1, 4}, {64, 4, 5, 3, 2, 2},
    {32, 8, 5, 3, 2, 2}, {64, 4, kRetired, 0}, {64, 4, kRetired, 0}, {32, 8, kRetired, 0},
    {32, 8, kRetired, 0}, {64, 4, 6, 3, 1, 2}, {64, 4, 6, 4, 1, 2}, {32, 8, 6, 3},
    {64, 6, 5, 2, 1, 2}, {64, 6, 5, 2},       {64, 6, 6, 3, 1, 2}, {32, 12, 5, 2, 1, 2}, {32, 12, 5, 2},
    {32, 12, 6, 3, 1, 2}, {64, 8, 6, 2, 1, 2}, {48, 8, 5, 2, 1, 2}, {48, 8, 5, 2},
    {64, 4, 6, 2, 1, 2, 3, 2}, {32, 8, 6, 2, 1, 2, 3, 2}, {64, 4, 6, 2, 1, 1, 3, 2}};

// forcing = kForcingGuo or model = kModelFE: the kernels that choose the
// collision at run time (kinds 0 and 3) and the 64x6 TMA tile (34), which has
// a Guo and an FE instantiation.
inline bool tile_supported(int tile, int lattice, int precision, int forcing = kForcingShift, int model = kModelSC) {
    if (tile < 0 || tile >= kNumTiles) return false;
    if ((forcing == kForcingGuo || model == kModelFE) && kTiles[tile].kind != 0 && kTiles[tile].kind != 3 &&
        tile != 34)
        return false;
    switch (kTiles[tile].kind) {
        case 0: return true;
        case 3: return true;
        case 4: return lattice == 1 && precision >= 1 && precision <= 3;
        case 5: return lattice == 1 && precision == 1;
        case 6: return lattice == 1 && precision >= 2 && precision <= 5;
    }
    return false;
}

// Size rules beyond the lattice kind and precision: the TMA boxes need the
// lattice to span at least one tile in x and y.
inline bool tile_fits(int tile, const Plan& p) {
    if (!tile_supported(tile, p.lattice, p.precision, p.forcing, p.model)) return false;
    const TileShape& t = kTiles[tile];
    if (t.kind == 5 || t.kind == 6) {
        const int tiles_x = (p.nx + t.tx - 1) / t.tx, tiles_y = (p.ny + t.ty - 1) / t.ty;
        return p.nx >= t.tx && p.ny >= t.ty && tiles_x % t.cx == 0 && tiles_y % t.cy == 0;
    }
    return true;
}

struct MomentsOut {
    void* rhoA;
    void* rhoB;
    void* u;
    void* p;
    double* partials;       // per-CTA diagnostics, or null
    double win[5];          // cx, cy, cz, r_in, r_out (r_in < 0: no inner window)
    int zlo = 0, zhi = 0;   // zhi > 0: fields of planes [zlo, zhi) only (D3Q19, no partials)
};

inline dim3 fused_grid(const Plan& p) {
    return dim3((unsigned)((p.nx + kTX - 1) / kTX), (unsigned)((p.ny + kTY - 1) / kTY),
                (unsigned)(p.lattice == 1 ? (p.nz + p.zchunk - 1) / p.zchunk : 1));
}

inline dim3 step_grid(const Plan& p) {
    const TileShape t = kTiles[p.step_tile];
    return dim3((unsigned)((p.nx + t.tx - 1) / t.tx), (unsigned)((p.ny + t.ty - 1) / t.ty),
                (unsigned)(p.lattice == 1 ? (p.nz + p.step_zchunk - 1) / p.step_zchunk : 1));
}

inline long long fused_blocks(const Plan& p) {
    const dim3 g = fused_grid(p);
    return (long long)g.x * g.y * g.z;
}

cudaError_t d2q9_step(const Plan& p, const void* fin, void* fout, cudaStream_t st);
// init of planes [zlo, zhi) (zhi = 0: all planes)
cudaError_t d2q9_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout,
                      cudaStream_t st, int zlo = 0, int zhi = 0);
cudaError_t d2q9_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st);
cudaError_t d3q19_step(const Plan& p, const void* fin, void* fout, cudaStream_t st);
// the step of each storage precision (sc_d3q19_step_*.cu)
cudaError_t d3q19_step_f64(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_step_f32(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_step_bf16(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_step_f16(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_step_bf16_rest(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_step_f16_rest(const Plan& p, const void* fin, void* fout, cudaStream_t st);
cudaError_t d3q19_init(const Plan& p, const void* rA, const void* rB, const void* u, void* fout,
                       cudaStream_t st, int zlo = 0, int zhi = 0);
cudaError_t d3q19_moments(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st);
cudaError_t diag_finish(const double* partials, long long nparts, double* out, cudaStream_t st);

}  // namespace lbmsc

// Declarations shared by the batch launcher TU and the C-ABI TU.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sc_launch.cuh"

namespace lbmsc {

// One work item of a batch: lattice index, tile origin, first plane of the z chunk.
struct BatchItem {
    int lat, x0, y0, z0;
};

// Batch tiles (x by y columns per CTA): 0 = 32x8, 1 = 32x4, 2 = 64x4 (z-marching
// kernel, every lattice and precision); 3 = 32x8, 4 = 64x4 (TMA-fed kernel with
// 3 stages, D3Q19 with FP32 storage, lattices at least one tile wide in x and
// y).  Tiles 0-4 run persistent grids over an atomic work counter; 5 = 32x8
// and 6 = 64x4 TMA-fed, 7 = 32x8 and 8 = 64x4 z-marching launch one CTA per
// work item and leave the order to the hardware's block scheduler; 9 = TMA-fed,
// one CTA per item, with each lattice's own tile: 64x4 for lattices at least
// 64 wide, else 32x8 (kBatchTileX/Y give the narrow one); with 384 threads
// (12 warps per SM, 2 stages): 10 = 32x12 TMA-fed one CTA per item, 11 = the
// mixed form with 64x6 and 32x12; 12 = each lattice in the best of 64x6, 48x8
// and 32x12 for its size (batch_shape3).  13 = the TMA-fed kernel for the
// paired 16-bit rest-offset storages (D3Q19, lattices at least 32 x 8): 32x8
// tiles, 2 stages, two CTAs per SM, one CTA per item (the solo tile 43 shape).
constexpr int kNumBatchTiles = 14;
constexpr int kBatchTileX[kNumBatchTiles] = {32, 32, 64, 32, 64, 32, 64, 32, 64, 32, 32, 32, 32, 32};
constexpr int kBatchTileY[kNumBatchTiles] = {8, 4, 4, 8, 4, 8, 4, 8, 4, 8, 12, 12, 12, 8};
constexpr bool kBatchTileTma[kNumBatchTiles] = {false, false, false, true, true, true, true,
                                                false, false, true, true, true, true, true};
constexpr bool kBatchTileGrid[kNumBatchTiles] = {false, false, false, false, false, true, true,
                                                 true, true, true, true, true, true, true};
constexpr int kBatchTileMixed = 9;
constexpr int kBatchTileMixed384 = 11;
constexpr int kBatchTileShape3 = 12;
constexpr int kBatchTileRest = 13;

// The 384-thread tile shapes of batch tile 12, and the one a lattice takes:
// the shape with the least work per node of the lattice, counting the padding
// of ragged edge tiles ((tiles_x TX)(tiles_y TY) / (nx ny)) times the columns
// its boxes read per tile column ((TX + 8) / TX: the halo rows in y mostly come
// from L2, the extra columns in x do not), among the shapes at most as large
// as the lattice.  Lattices 32 wide get 32x12, 48 and 96 wide 48x8 (no ragged
// tile: a 64-wide tile on 96 columns leaves half of every second tile idle),
// 64 and 128 wide 64x6.  -1: none fits.
constexpr int kShape3X[3] = {32, 64, 48};
constexpr int kShape3Y[3] = {12, 6, 8};
inline int batch_shape3(const Plan& p) {
    int best = -1;
    double best_cost = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int tx = kShape3X[k], ty = kShape3Y[k];
        if (p.nx < tx || p.ny < ty) continue;
        const double pad = (double)((p.nx + tx - 1) / tx * tx) * ((p.ny + ty - 1) / ty * ty) / ((double)p.nx * p.ny);
        const double cost = pad * (tx + 8) / (double)tx;
        if (best < 0 || cost < best_cost - 1e-12) {
            best = k;
            best_cost = cost;
        }
    }
    return best;
}

// The tile of one lattice's items in a batch of this tile kind.
inline void batch_item_tile(int tile, const Plan& p, int& tx, int& ty) {
    if (tile == kBatchTileShape3) {
        const int k = batch_shape3(p);
        tx = kShape3X[k < 0 ? 0 : k];
        ty = kShape3Y[k < 0 ? 0 : k];
        return;
    }
    const bool mixed = tile == kBatchTileMixed || tile == kBatchTileMixed384;
    const bool wide = mixed && p.nx >= 64;
    tx = wide ? 64 : kBatchTileX[tile];
    ty = wide ? (tile == kBatchTileMixed ? 4 : 6) : kBatchTileY[tile];
}

inline bool batch_tile_fits(int tile, const Plan& p) {
    if (tile < 0 || tile >= kNumBatchTiles) return false;
    if (!kBatchTileTma[tile]) return true;  // the z-marching batch kernel chooses the collision at run time
    if (tile == kBatchTileRest)
        return p.lattice == 1 && rest_precision(p.precision) && p.forcing == kForcingShift && p.model == kModelSC &&
               p.nx >= kBatchTileX[tile] && p.ny >= kBatchTileY[tile];
    if (!(p.lattice == 1 && p.precision == 1 && p.forcing == kForcingShift && p.model == kModelSC)) return false;
    if (tile == kBatchTileShape3) return batch_shape3(p) >= 0;
    return p.nx >= kBatchTileX[tile] && p.ny >= kBatchTileY[tile];
}

// Bytes of one lattice's descriptor, and the descriptor itself (both parities;
// parity p reads buffer cur0 ^ p).  err: the lattice's device error word.
size_t batch_lattice_bytes(int precision, int tile);
cudaError_t batch_lattice_fill(const Plan& p, const void* b0, const void* b1, int cur0, int zchunk, int tile,
                               void* dst);
// ctr: two device ints, zero before the first launch (each launch leaves them zero).
cudaError_t batch_step(int lattice, int precision, int tile, const void* lats, const BatchItem* items, int nitems,
                       int parity, int sm_count, int* ctr, cudaStream_t st);

}  // namespace lbmsc

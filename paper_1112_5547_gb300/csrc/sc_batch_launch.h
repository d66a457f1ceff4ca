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
// mixed form with 64x6 and 32x12.
constexpr int kNumBatchTiles = 12;
constexpr int kBatchTileX[kNumBatchTiles] = {32, 32, 64, 32, 64, 32, 64, 32, 64, 32, 32, 32};
constexpr int kBatchTileY[kNumBatchTiles] = {8, 4, 4, 8, 4, 8, 4, 8, 4, 8, 12, 12};
constexpr bool kBatchTileTma[kNumBatchTiles] = {false, false, false, true, true, true, true,
                                                false, false, true, true, true};
constexpr bool kBatchTileGrid[kNumBatchTiles] = {false, false, false, false, false, true, true,
                                                 true, true, true, true, true};
constexpr int kBatchTileMixed = 9;
constexpr int kBatchTileMixed384 = 11;

// The tile of one lattice's items in a batch of this tile kind.
inline void batch_item_tile(int tile, const Plan& p, int& tx, int& ty) {
    const bool mixed = tile == kBatchTileMixed || tile == kBatchTileMixed384;
    const bool wide = mixed && p.nx >= 64;
    tx = wide ? 64 : kBatchTileX[tile];
    ty = wide ? (tile == kBatchTileMixed ? 4 : 6) : kBatchTileY[tile];
}

inline bool batch_tile_fits(int tile, const Plan& p) {
    if (tile < 0 || tile >= kNumBatchTiles) return false;
    if (!kBatchTileTma[tile]) return true;  // the z-marching batch kernel chooses the collision at run time
    return p.lattice == 1 && p.precision == 1 && p.forcing == kForcingShift && p.model == kModelSC &&
           p.nx >= kBatchTileX[tile] && p.ny >= kBatchTileY[tile];
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

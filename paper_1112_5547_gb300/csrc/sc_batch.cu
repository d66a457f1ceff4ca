// Host launchers of the ragged-batch step (sc_batch.cuh).
#include <atomic>
#include <cstring>
#include <type_traits>

#include "sc_batch.cuh"
#include "sc_batch_launch.h"
#include "sc_args.cuh"

namespace lbmsc {

namespace {

// Kernel attributes and occupancy belong to a device: the one-time setup of a
// kernel is kept per device ordinal (the first call on each device does it).
constexpr int kMaxDevices = 64;

int current_device() {
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices ? dev : -1;
}

template <auto Kern> cudaError_t dynamic_smem_once(int bytes) {
    static std::atomic<int> done[kMaxDevices];  // zero-initialised: not yet set
    const int dev = current_device();
    if (dev >= 0 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev >= 0) done[dev].store(1, std::memory_order_release);
    return e;
}

template <auto Kern> cudaError_t blocks_per_sm_once(int threads, int* out) {
    static std::atomic<int> cache[kMaxDevices];  // zero: not yet asked (a kernel always fits once)
    const int dev = current_device();
    if (dev >= 0) {
        const int c = cache[dev].load(std::memory_order_acquire);
        if (c > 0) {
            *out = c;
            return cudaSuccess;
        }
    }
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, Kern, threads, 0);
    if (e != cudaSuccess) return e;
    *out = n > 0 ? n : 1;
    if (dev >= 0) cache[dev].store(*out, std::memory_order_release);
    return cudaSuccess;
}

// grid: one CTA per item (ctr unused), else a persistent grid over the counter.
template <class L, class S, int TX, int TY>
cudaError_t launch_batch(const void* lats, const BatchItem* items, int nitems, int parity, int sm_count, int* ctr,
                         bool grid_mode, cudaStream_t st) {
    using C = typename Codec<S>::C;
    constexpr int kMin = sizeof(C) == 8 ? 1 : (TX * TY <= 128 ? 4 : 2);
    constexpr auto kern = sc_batch_step_kernel<L, S, TX, TY, kMin>;
    int per_sm = 1;  // resident CTAs per SM
    const cudaError_t oe = blocks_per_sm_once<kern>(TX * TY, &per_sm);
    if (oe != cudaSuccess) return oe;
    long long grid = grid_mode ? nitems : (long long)sm_count * per_sm;
    if (grid > nitems) grid = nitems;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, dim3(TX, TY), 0, st>>>(static_cast<const BatchLattice<S>*>(lats), items, nitems, parity,
                                                  grid_mode ? nullptr : ctr);
    return cudaGetLastError();
}

template <int TX, int TY, int ST>
cudaError_t launch_batch_tma(const void* lats, const BatchItem* items, int nitems, int parity, int sm_count, int* ctr,
                             bool grid_mode, cudaStream_t st) {
    using T = TmaTile<TX, TY, ST>;
    constexpr auto kern = sc_batch_tma_kernel<TX, TY, ST>;
    const cudaError_t attr = dynamic_smem_once<kern>((int)T::smem_bytes);
    if (attr != cudaSuccess) return attr;
    // persistent: one CTA per SM (the stages take most of shared memory)
    long long grid = grid_mode ? nitems : sm_count;
    if (grid > nitems) grid = nitems;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, dim3(TX, TY), T::smem_bytes, st>>>(static_cast<const BatchTmaLattice*>(lats), items,
                                                              nitems, parity, grid_mode ? nullptr : ctr);
    return cudaGetLastError();
}

template <int WX, int WY, int NX, int NY, int S>
cudaError_t launch_batch_tma_mixed(const void* lats, const BatchItem* items, int nitems, int parity,
                                   cudaStream_t st) {
    constexpr size_t smem = TmaTile<WX, WY, S>::smem_bytes > TmaTile<NX, NY, S>::smem_bytes
                                ? TmaTile<WX, WY, S>::smem_bytes
                                : TmaTile<NX, NY, S>::smem_bytes;
    constexpr auto kern = sc_batch_tma_mixed_kernel<WX, WY, NX, NY, S>;
    const cudaError_t attr = dynamic_smem_once<kern>((int)smem);
    if (attr != cudaSuccess) return attr;
    if (nitems < 1) return cudaSuccess;
    kern<<<(unsigned)nitems, WX * WY, smem, st>>>(static_cast<const BatchTmaLattice*>(lats), items, nitems, parity);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_batch_tma_shape3(const void* lats, const BatchItem* items, int nitems, int parity, cudaStream_t st) {
    constexpr size_t a = TmaTile<64, 6, S>::smem_bytes, b = TmaTile<48, 8, S>::smem_bytes,
                     c = TmaTile<32, 12, S>::smem_bytes;
    constexpr size_t smem = a > b ? (a > c ? a : c) : (b > c ? b : c);
    constexpr auto kern = sc_batch_tma_shape3_kernel<S>;
    const cudaError_t attr = dynamic_smem_once<kern>((int)smem);
    if (attr != cudaSuccess) return attr;
    if (nitems < 1) return cudaSuccess;
    kern<<<(unsigned)nitems, 384, smem, st>>>(static_cast<const BatchTmaLattice*>(lats), items, nitems, parity);
    return cudaGetLastError();
}

template <class St>
cudaError_t launch_batch_tma_rest(const void* lats, const BatchItem* items, int nitems, int parity, cudaStream_t st) {
    using T = TmaTile<32, 8, 2, St>;
    constexpr auto kern = sc_batch_tma_rest_kernel<St>;
    const cudaError_t attr = dynamic_smem_once<kern>((int)T::smem_bytes);
    if (attr != cudaSuccess) return attr;
    if (nitems < 1) return cudaSuccess;
    kern<<<(unsigned)nitems, 256, T::smem_bytes, st>>>(static_cast<const BatchTmaRestLattice<St>*>(lats), items,
                                                        nitems, parity);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t batch_typed(int tile, const void* lats, const BatchItem* items, int nitems, int parity, int sm_count,
                        int* ctr, cudaStream_t st) {
    static_assert(kNumBatchTiles == 14 && kBatchTileX[6] == 64 && kBatchTileGrid[5] && kBatchTileTma[6] &&
                      !kBatchTileTma[7] && kBatchTileY[8] == 4 && kBatchTileMixed == 9 && kBatchTileY[10] == 12 &&
                      kBatchTileMixed384 == 11 && kBatchTileShape3 == 12 && kBatchTileRest == 13 &&
                      kBatchTileX[13] == 32 && kBatchTileY[13] == 8,
                  "batch tile table and dispatch disagree");
    switch (tile) {
        case 0: return launch_batch<L, S, 32, 8>(lats, items, nitems, parity, sm_count, ctr, false, st);
        case 1: return launch_batch<L, S, 32, 4>(lats, items, nitems, parity, sm_count, ctr, false, st);
        case 2: return launch_batch<L, S, 64, 4>(lats, items, nitems, parity, sm_count, ctr, false, st);
        case 7: return launch_batch<L, S, 32, 8>(lats, items, nitems, parity, sm_count, ctr, true, st);
        case 8: return launch_batch<L, S, 64, 4>(lats, items, nitems, parity, sm_count, ctr, true, st);
    }
    if constexpr (std::is_same<L, D3Q19>::value && std::is_same<S, float>::value) {
        switch (tile) {
            case 3: return launch_batch_tma<32, 8, 3>(lats, items, nitems, parity, sm_count, ctr, false, st);
            case 4: return launch_batch_tma<64, 4, 3>(lats, items, nitems, parity, sm_count, ctr, false, st);
            case 5: return launch_batch_tma<32, 8, 3>(lats, items, nitems, parity, sm_count, ctr, true, st);
            case 6: return launch_batch_tma<64, 4, 3>(lats, items, nitems, parity, sm_count, ctr, true, st);
            case 9: return launch_batch_tma_mixed<64, 4, 32, 8, 3>(lats, items, nitems, parity, st);
            case 10: return launch_batch_tma<32, 12, 2>(lats, items, nitems, parity, sm_count, ctr, true, st);
            case 11: return launch_batch_tma_mixed<64, 6, 32, 12, 2>(lats, items, nitems, parity, st);
            case 12: return launch_batch_tma_shape3<2>(lats, items, nitems, parity, st);
        }
    }
    if constexpr (std::is_same<L, D3Q19>::value && Codec<S>::kRest) {
        if (tile == kBatchTileRest) return launch_batch_tma_rest<S>(lats, items, nitems, parity, st);
    }
    return cudaErrorInvalidValue;
}

template <class L>
cudaError_t batch_lat(int precision, int tile, const void* lats, const BatchItem* items, int nitems, int parity,
                      int sm_count, int* ctr, cudaStream_t st) {
    switch (precision) {
        case 0: return batch_typed<L, double>(tile, lats, items, nitems, parity, sm_count, ctr, st);
        case 1: return batch_typed<L, float>(tile, lats, items, nitems, parity, sm_count, ctr, st);
        case 2: return batch_typed<L, __nv_bfloat16>(tile, lats, items, nitems, parity, sm_count, ctr, st);
        case 3: return batch_typed<L, __half>(tile, lats, items, nitems, parity, sm_count, ctr, st);
        case 4: return batch_typed<L, bf16_rest>(tile, lats, items, nitems, parity, sm_count, ctr, st);
        case 5: return batch_typed<L, f16_rest>(tile, lats, items, nitems, parity, sm_count, ctr, st);
    }
    return cudaErrorInvalidValue;
}

// Descriptor of batch tile 13: both parities' arguments and their population
// and density maps (the boxes of the 32x8 rest-offset tile).
template <class St>
cudaError_t fill_rest(const Plan& p, const void* b0, const void* b1, int cur0, int zchunk, void* dst) {
    using T = TmaTile<32, 8, 2, St>;
    BatchTmaRestLattice<St> bl;
    memset(&bl, 0, sizeof(bl));
    const void* bufs[2] = {b0, b1};
    for (int par = 0; par < 2; ++par) {
        const int src = cur0 ^ par;
        bl.a[par] = make_args<St>(p, bufs[src], const_cast<void*>(bufs[src ^ 1]));
        bl.a[par].zchunk = zchunk;
        cudaError_t e = encode_population_map(p, bl.a[par].fin, T::BX, T::BY, &bl.maps[par].pop, 3, T::E, T::Q2);
        if (e == cudaSuccess)
            e = encode_rho_map(p, rest_rho<D3Q19>(bl.a[par].fin, p.Np), T::RBX, T::RBY, &bl.maps[par].rho, 3);
        if (e != cudaSuccess) return e;
    }
    bl.err = p.err;
    memcpy(dst, &bl, sizeof(bl));
    return cudaSuccess;
}

template <class S> void fill_typed(const Plan& p, const void* b0, const void* b1, int cur0, int zchunk, void* dst) {
    BatchLattice<S> bl;
    const void* bufs[2] = {b0, b1};
    for (int par = 0; par < 2; ++par) {
        const int src = cur0 ^ par;
        bl.a[par] = make_args<S>(p, bufs[src], const_cast<void*>(bufs[src ^ 1]));
        bl.a[par].zchunk = zchunk;
    }
    memcpy(dst, &bl, sizeof(bl));
}

}  // namespace

size_t batch_lattice_bytes(int precision, int tile) {
    if (tile == kBatchTileRest)
        return precision == 4 ? sizeof(BatchTmaRestLattice<bf16_rest>)
                              : (precision == 5 ? sizeof(BatchTmaRestLattice<f16_rest>) : 0);
    if (tile >= 0 && tile < kNumBatchTiles && kBatchTileTma[tile]) return sizeof(BatchTmaLattice);
    switch (precision) {
        case 0: return sizeof(BatchLattice<double>);
        case 1: return sizeof(BatchLattice<float>);
        case 2: return sizeof(BatchLattice<__nv_bfloat16>);
        case 3: return sizeof(BatchLattice<__half>);
        case 4: return sizeof(BatchLattice<bf16_rest>);
        case 5: return sizeof(BatchLattice<f16_rest>);
    }
    return 0;
}

cudaError_t batch_lattice_fill(const Plan& p, const void* b0, const void* b1, int cur0, int zchunk, int tile,
                               void* dst) {
    if (!batch_tile_fits(tile, p)) return cudaErrorInvalidValue;
    if (tile == kBatchTileRest)
        return p.precision == 4 ? fill_rest<bf16_rest>(p, b0, b1, cur0, zchunk, dst)
                                : fill_rest<f16_rest>(p, b0, b1, cur0, zchunk, dst);
    if (kBatchTileTma[tile]) {
        BatchTmaLattice bl;
        memset(&bl, 0, sizeof(bl));
        const void* bufs[2] = {b0, b1};
        for (int par = 0; par < 2; ++par) {
            const int src = cur0 ^ par;
            bl.a[par] = make_args<float>(p, bufs[src], const_cast<void*>(bufs[src ^ 1]));
            bl.a[par].zchunk = zchunk;
            int tx, ty;
            batch_item_tile(tile, p, tx, ty);
            const cudaError_t e =
                encode_population_map(p, static_cast<const float*>(bufs[src]), tx + 8, ty + 2, &bl.map[par]);
            if (e != cudaSuccess) return e;
        }
        bl.err = p.err;
        int tx, ty;
        batch_item_tile(tile, p, tx, ty);
        bl.wide = tile == kBatchTileShape3 ? batch_shape3(p) : (tx == 64 ? 1 : 0);
        memcpy(dst, &bl, sizeof(bl));
        return cudaSuccess;
    }
    switch (p.precision) {
        case 0: fill_typed<double>(p, b0, b1, cur0, zchunk, dst); break;
        case 1: fill_typed<float>(p, b0, b1, cur0, zchunk, dst); break;
        case 2: fill_typed<__nv_bfloat16>(p, b0, b1, cur0, zchunk, dst); break;
        case 3: fill_typed<__half>(p, b0, b1, cur0, zchunk, dst); break;
        case 4: fill_typed<bf16_rest>(p, b0, b1, cur0, zchunk, dst); break;
        case 5: fill_typed<f16_rest>(p, b0, b1, cur0, zchunk, dst); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t batch_step(int lattice, int precision, int tile, const void* lats, const BatchItem* items, int nitems,
                       int parity, int sm_count, int* ctr, cudaStream_t st) {
    return lattice == 0 ? batch_lat<D2Q9>(precision, tile, lats, items, nitems, parity, sm_count, ctr, st)
                        : batch_lat<D3Q19>(precision, tile, lats, items, nitems, parity, sm_count, ctr, st);
}

}  // namespace lbmsc

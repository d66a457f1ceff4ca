// Ragged batch: one launch advances many independent lattices by one step.
//
// The host builds a work list of items (lattice, x tile, y tile, z chunk) for
// every lattice of the batch, longest items first.  Either persistent CTAs take
// items from an atomic counter, or the launch has one CTA per item.  Each item
// runs the per-node code of a solo step (the z-marching body of
// sc_fused_kernel, or tma_item of the TMA-fed kernel) on its own lattice's
// arguments, read from a device descriptor array holding both ping-pong
// parities, so every lattice gets exactly the arithmetic of a solo step:
// batched and solo results are bit-identical.
#pragma once

#include "sc_batch_launch.h"
#include "sc_kernels.cuh"
#include "sc_tma.cuh"

namespace lbmsc {

// Work list order of a batch launch.  With a counter (persistent grids): CTAs
// take items in list order from an atomic counter, so a CTA that finishes
// early takes more; the next index is fetched while the current item runs (the
// TMA-fed kernel fetches it itself, late in the item), and the last CTA to
// find the list empty resets both counters for the next
// launch (no memset between launches; graph replays work).  Without a counter
// (one CTA per item, grid = item count): CTA b runs item b, and the hardware's
// block scheduler starts each item as an earlier one retires, which keeps the
// items in flight at any moment neighbours in the list.
struct BatchQueue {
    int* ctr;   // [0]: next item, [1]: CTAs done; null: static order
    int* slot;  // shared: the fetched index
    int k;      // fetches so far (static order)

    __device__ __forceinline__ void fetch(int tid) {
        if (tid == 0) *slot = ctr ? atomicAdd(&ctr[0], 1) : (int)blockIdx.x + k * (int)gridDim.x;
        ++k;
    }
    __device__ __forceinline__ void retire(int tid) {
        if (ctr && tid == 0) {
            __threadfence();
            if (atomicAdd(&ctr[1], 1) == (int)gridDim.x - 1) {
                ctr[0] = 0;
                ctr[1] = 0;
                __threadfence();
            }
        }
    }
};

// Both parities of one lattice: a[p] reads buffer cur0 ^ p and writes the other.
template <class S> struct BatchLattice {
    LatticeArgs<S> a[2];
};

template <class L, class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB)
    sc_batch_step_kernel(const BatchLattice<S>* __restrict__ lats,
                         const BatchItem* __restrict__ items, int nitems, int parity, int* __restrict__ ctr) {
    using C = typename Codec<S>::C;
    constexpr int Q = L::Q;
    constexpr int FX = TX + 2, FY = TY + 2;
    constexpr int NPL = L::D == 3 ? 3 : 1;
    constexpr int H = 2 * FX + 2 * TY;
    static_assert(H <= TX * TY, "halo ring must fit in the CTA");
    __shared__ C srho[NPL][2][FY][FX];
    __shared__ int s_next;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const bool halo = tid < H;
    int hfx, hfy;
    halo_cell<TX, TY>(tid, hfx, hfy);
    BatchQueue queue{ctr, &s_next, 0};
    queue.fetch(tid);
    __syncthreads();

#pragma unroll 1
    for (;;) {
        const int it = s_next;
        if (it >= nitems) break;
        __syncthreads();  // every thread has read s_next
        queue.fetch(tid);  // the next index, while this item runs
        const BatchItem w = items[it];
        const LatticeArgs<S> a = lats[w.lat].a[parity];
        const int nx = a.nx, ny = a.ny, nz = a.nz;
        const int x0 = w.x0, y0 = w.y0;
        const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
        const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
        const int hgx = (x0 - 1 + hfx + nx) % nx;
        const int hgy = (y0 - 1 + hfy + ny) % ny;

        auto density_plane = [&](int slot, int z, C (&f)[2][Q]) {
            pull_node<L, S>(a, gx, gy, z, f);
            srho[slot][0][ty + 1][tx + 1] = node_density<L, C>(f[0]);
            srho[slot][1][ty + 1][tx + 1] = node_density<L, C>(f[1]);
            if (halo) {
                C h[2][Q];
                pull_node<L, S>(a, hgx, hgy, z, h);
                srho[slot][0][hfy][hfx] = node_density<L, C>(h[0]);
                srho[slot][1][hfy][hfx] = node_density<L, C>(h[1]);
            }
        };
        auto process = [&](C (&f)[2][Q], int sm, int sc, int sp, int z) {
            const C rA = srho[sc][0][ty + 1][tx + 1];
            const C rB = srho[sc][1][ty + 1][tx + 1];
            auto nbr = [&](int s, int i) -> C {
                const int slot = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm);
                return srho[slot][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
            };
            node_update<L, C>(a, gy, nbr, f, rA, rB);
            if (owner) store_node<L, S>(a, gx, gy, z, f, rA, rB);
        };

        C cur[2][Q];
        if (L::D == 2) {
            density_plane(0, 0, cur);
            __syncthreads();
            process(cur, 0, 0, 0, 0);
        } else {
            const int z0 = w.z0;
            const int z1 = min(z0 + a.zchunk, nz);
            {
                C tmp[2][Q];
                density_plane(0, z0 == 0 ? nz - 1 : z0 - 1, tmp);
            }
            density_plane(1, z0, cur);
            int sm = 0, sc = 1, sp = 2;
#pragma unroll 1
            for (int z = z0; z < z1; ++z) {
                C nxt[2][Q];
                density_plane(sp, z + 1 == nz ? 0 : z + 1, nxt);
                __syncthreads();
                process(cur, sm, sc, sp, z);
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int i = 0; i < Q; ++i) cur[s][i] = nxt[s][i];
                const int t = sm;
                sm = sc;
                sc = sp;
                sp = t;
                __syncthreads();
            }
        }
        __syncthreads();  // the next item rewrites the density ring; s_next is visible
    }
    queue.retire(tid);
}

// Both parities of one FP32 D3Q19 lattice for the TMA-fed batch kernel: the
// tensor map of the buffer each parity reads, its arguments, and the lattice's
// error word (raised if a bounded wait expires on one of its items).
struct BatchTmaLattice {  // CUtensorMap brings its own 128-byte alignment
    CUtensorMap map[2];
    LatticeArgs<float> a[2];
    int* err;
    int wide;  // mixed-shape batches: 1 = this lattice's items are the wide tiles, 0 = the narrow ones;
               // batch tile 12: the index of the lattice's shape in kShape3X / kShape3Y
};

// TMA-fed batch step: persistent CTAs run tma_item (sc_tma.cuh) over the work
// list, so each item gets the arithmetic and order of the solo TMA kernel.
template <int TX, int TY, int S>
__global__ void __launch_bounds__(TX* TY, 1)
    sc_batch_tma_kernel(const BatchTmaLattice* __restrict__ lats, const BatchItem* __restrict__ items, int nitems,
                        int parity, int* __restrict__ ctr) {
    static_assert(S <= 3, "every item has at least 3 planes: all S first planes of the next item are pre-issued");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_next;
    TmaSmem<TX, TY, S> sm(smem_raw);
    const int tid = threadIdx.y * TX + threadIdx.x;
    BatchQueue queue{ctr, &s_next, 0};
    queue.fetch(tid);  // the first item
    sm.init_barriers();  // (ends with a CTA barrier)
    unsigned qbase = 0;
    bool preissued = false;
    // The next item is taken from the counter a few planes before the end of
    // the current one, not at its start: items then start in the order earlier
    // ones finish, as with the hardware block scheduler, and neighbouring
    // tiles stay in flight together (taking it a whole item ahead let the CTAs
    // drift apart and lose the halo rows they share in L2).
    int nit = 0;
    BatchItem wn{0, 0, 0, 0};
    TmaNext nxt{nullptr, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (;;) {
        const int it = s_next;
        if (it >= nitems) break;
        __syncthreads();  // every thread has read s_next
        const BatchItem w = items[it];
        const BatchTmaLattice* l = lats + w.lat;
        const LatticeArgs<float> a = l->a[parity];
        if (tid == 0 && !preissued) tma_prefetch_map(&l->map[parity]);
        nxt.nplanes = 0;
        // elected thread, at the start of plane q: take the next index three
        // planes before the pre-issue, read its item two before, its lattice one
        // before (each load has a plane of time to land)
        auto hook = [&](int q, int np) {
            const int pre = np - S;  // plane whose barrier is followed by the first pre-issue
            // (one CTA per item, ctr null: the static order, which ends the loop)
            if (q == max(0, pre - 3)) nit = ctr ? atomicAdd(&ctr[0], 1) : it + (int)gridDim.x;
            if (q == max(0, pre - 2) && nit < nitems) wn = items[nit];
            if (q == max(0, pre - 1)) {
                s_next = nit;  // visible to every thread after the end-of-item barrier
                if (nit < nitems) {
                    const BatchTmaLattice* ln = lats + wn.lat;
                    const LatticeArgs<float>& an = ln->a[parity];
                    nxt.map = &ln->map[parity];
                    tma_prefetch_map(nxt.map);
                    nxt.x0 = wn.x0;
                    nxt.y0 = wn.y0;
                    nxt.z0 = wn.z0;
                    nxt.gxo = an.gxo;
                    nxt.gyo = an.gyo;
                    nxt.nz = an.nz;
                    nxt.nplanes = min(wn.z0 + an.zchunk, an.nz) - wn.z0 + 2;
                    nxt.down = tma_march_down(wn.z0, an.zchunk);
                }
            }
        };
        const int n = tma_item<TX, TY, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, qbase, sm, l->err,
                                          preissued, &nxt, hook, true);
        if (n < 0) break;  // a lost wait: the lattice's error word is raised
        qbase += (unsigned)n;
        // the next item's first planes went out with this one (the elected
        // thread decided; every item has at least S planes, so all did)
        preissued = true;
        __syncthreads();  // the next item rewrites the density ring; s_next is visible
    }
    queue.retire(tid);
}

// Mixed-shape TMA batch step, one CTA per work item: items of lattices at
// least WX wide run as WX x WY tiles (fewer halo rows and boxes re-read per
// node), the others as NX x NY tiles of the same thread count; the shared
// memory holds the larger of the two layouts.
template <int WX, int WY, int NX, int NY, int S>
__global__ void __launch_bounds__(WX* WY, 1)
    sc_batch_tma_mixed_kernel(const BatchTmaLattice* __restrict__ lats, const BatchItem* __restrict__ items,
                              int nitems, int parity) {
    static_assert(WX * WY == NX * NY, "both tile shapes use the same block");
    extern __shared__ unsigned char smem_raw[];
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const BatchItem w = items[it];
    const BatchTmaLattice* l = lats + w.lat;
    const LatticeArgs<float> a = l->a[parity];
    if (threadIdx.x == 0) tma_prefetch_map(&l->map[parity]);
    if (l->wide) {
        TmaSmem<WX, WY, S> sm(smem_raw);
        sm.init_barriers();
        tma_item<WX, WY, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false, nullptr,
                            TmaNoHook(), true);
    } else {
        TmaSmem<NX, NY, S> sm(smem_raw);
        sm.init_barriers();
        tma_item<NX, NY, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false, nullptr,
                            TmaNoHook(), true);
    }
}

// Batch tile 12, one CTA per work item: each lattice's items run in its own
// one of three 384-thread tile shapes (batch_shape3); the shared memory holds
// the largest of their layouts.
template <int S>
__global__ void __launch_bounds__(384, 1)
    sc_batch_tma_shape3_kernel(const BatchTmaLattice* __restrict__ lats, const BatchItem* __restrict__ items,
                               int nitems, int parity) {
    static_assert(kShape3X[0] * kShape3Y[0] == 384 && kShape3X[1] * kShape3Y[1] == 384 &&
                      kShape3X[2] * kShape3Y[2] == 384,
                  "every shape uses the same block");
    extern __shared__ unsigned char smem_raw[];
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const BatchItem w = items[it];
    const BatchTmaLattice* l = lats + w.lat;
    const LatticeArgs<float> a = l->a[parity];
    if (threadIdx.x == 0) tma_prefetch_map(&l->map[parity]);
    if (l->wide == 1) {
        TmaSmem<64, 6, S> sm(smem_raw);
        sm.init_barriers();
        tma_item<64, 6, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false, nullptr,
                           TmaNoHook(), true);
    } else if (l->wide == 2) {
        TmaSmem<48, 8, S> sm(smem_raw);
        sm.init_barriers();
        tma_item<48, 8, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false, nullptr,
                           TmaNoHook(), true);
    } else {
        TmaSmem<32, 12, S> sm(smem_raw);
        sm.init_barriers();
        tma_item<32, 12, S>(&l->map[parity], nullptr, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false, nullptr,
                            TmaNoHook(), true);
    }
}

// Descriptor of one lattice of a rest-offset TMA batch (batch tile 13): the
// population and density maps and the arguments of both parities.
template <class St> struct BatchTmaRestLattice {
    TmaMaps maps[2];
    LatticeArgs<St> a[2];
    int* err;
};

// Batch tile 13, one CTA per work item: the paired 16-bit rest-offset storage
// through the TMA pipeline of the solo kernel's tile 43 (32x8 tiles, 2 stages,
// two CTAs per SM at 128 registers), odd z chunks marching downwards.
template <class St>
__global__ void __launch_bounds__(256, 2)
    sc_batch_tma_rest_kernel(const BatchTmaRestLattice<St>* __restrict__ lats, const BatchItem* __restrict__ items,
                             int nitems, int parity) {
    extern __shared__ unsigned char smem_raw[];
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const BatchItem w = items[it];
    const BatchTmaRestLattice<St>* l = lats + w.lat;
    const LatticeArgs<St> a = l->a[parity];
    if (threadIdx.x == 0) {
        tma_prefetch_map(&l->maps[parity].pop);
        tma_prefetch_map(&l->maps[parity].rho);
    }
    TmaSmem<32, 8, 2, St> sm(smem_raw);
    sm.init_barriers();
    tma_item<32, 8, 2, St>(&l->maps[parity].pop, &l->maps[parity].rho, a, w.x0, w.y0, w.z0, 0u, sm, l->err, false,
                           nullptr, TmaNoHook(), true);
}

}  // namespace lbmsc

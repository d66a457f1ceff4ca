// Persistent, cp.async-pipelined D3Q19 step for 32-bit population storage.
//
// Same arithmetic as sc_fused_kernel (Eq. eq:be with the force of Eq. FORCE,
// paper Sec. 2.1) and the same per-node operation order, so results are
// bit-identical; only the data movement differs:
//
//  * Persistent CTAs walk a list of work items (x tile, y tile, z chunk), x
//    fastest, so the items in flight at one time are neighbours and share
//    their halo lines in L2.
//  * Each thread copies the 38 pulled values of its own column node (and, for
//    84 threads, of one halo-ring node) for plane z+1+LOOK with cp.async into a
//    shared-memory stage, so up to LOOK planes of loads are in flight while the
//    CTA collides plane z.  No registers are held by the copies.
//  * Every stage slot is written and read by the same thread, so stages need
//    no barrier; the only data shared between threads is the density ring
//    (densities of the tile plus a one-node frame).  With four ring slots one
//    __syncthreads per plane is enough: plane q+1's densities go to slot
//    (q+1) % 4 while slower threads may still read slots (q-2..q) % 4.
#pragma once

#include "sc_kernels.cuh"

namespace lbmsc {

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
template <int B> __device__ __forceinline__ void cp_async_bytes(void* smem_dst, const void* gmem_src) {
    static_assert(B == 4 || B == 8 || B == 16, "cp.async copies 4, 8 or 16 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int TX, int TY, int STAGES> struct AsyncTile {
    static constexpr int FX = TX + 2, FY = TY + 2;
    static constexpr int H = 2 * FX + 2 * TY;  // halo ring nodes
    static constexpr int OWN = TX * TY;
    static constexpr int NODES = OWN + H;
    static constexpr int Q2 = 2 * D3Q19::Q;
    static constexpr size_t stage_floats = (size_t)Q2 * NODES;
    static constexpr size_t smem_bytes = (STAGES * stage_floats + 4 * 2 * FY * FX) * sizeof(float);
};

template <int TX, int TY, int STAGES>
__global__ void __launch_bounds__(TX* TY, 1)
    sc_step_async_kernel(const LatticeArgs<float> a, const int tiles_x, const int tiles_y, const int nchunks) {
    using L = D3Q19;
    using T = AsyncTile<TX, TY, STAGES>;
    using C = float;
    constexpr int Q = L::Q;
    constexpr int FX = T::FX, FY = T::FY, H = T::H, OWN = T::OWN, NODES = T::NODES;
    static_assert(H <= OWN, "halo ring must fit in the CTA");
    static_assert(STAGES >= 3, "need a stage to collide, one to reduce and one in flight");
    constexpr int LOOK = STAGES - 2;  // planes of copies in flight while colliding

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* const stage = reinterpret_cast<C*>(smem_raw);
    C(*const ring)[2][FY][FX] = reinterpret_cast<C(*)[2][FY][FX]>(stage + STAGES * T::stage_floats);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t Np = (size_t)a.Np;

    const bool halo = tid < H;
    int hfx, hfy;
    halo_cell<TX, TY>(tid, hfx, hfy);

    const long long total = (long long)tiles_x * tiles_y * nchunks;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int itx = (int)(item % tiles_x);
        const int ity = (int)((item / tiles_x) % tiles_y);
        const int ich = (int)(item / ((long long)tiles_x * tiles_y));
        const int x0 = itx * TX, y0 = ity * TY;
        const int z0 = ich * a.zchunk;
        const int z1 = min(z0 + a.zchunk, nz);
        const int nplanes = z1 - z0 + 2;  // z0-1 .. z1
        const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
        const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
        const int hgx = (x0 - 1 + hfx + nx) % nx;
        const int hgy = (y0 - 1 + hfy + ny) % ny;

        // Copies of plane q (z = z0 - 1 + q) into stage q % STAGES; always commits a
        // group (empty past the last plane) so the wait counts stay uniform.
        auto issue = [&](int q) {
            if (q < nplanes) {
                int z = z0 - 1 + q;
                z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                const int zs[3] = {wrap_inc(z, nz), z, wrap_dec(z, nz)};
                C* st = stage + (size_t)(q % STAGES) * T::stage_floats;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const size_t on = cell(a, gx - L::c(i, 0), gy - L::c(i, 1), zs[L::c(i, 2) + 1]);
                    cp_async4(st + (size_t)i * NODES + tid, a.fin + (size_t)i * Np + on);
                    cp_async4(st + (size_t)(Q + i) * NODES + tid, a.fin + (size_t)(Q + i) * Np + on);
                }
                if (halo) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const size_t hn = cell(a, hgx - L::c(i, 0), hgy - L::c(i, 1), zs[L::c(i, 2) + 1]);
                        cp_async4(st + (size_t)i * NODES + OWN + tid, a.fin + (size_t)i * Np + hn);
                        cp_async4(st + (size_t)(Q + i) * NODES + OWN + tid, a.fin + (size_t)(Q + i) * Np + hn);
                    }
                }
            }
            cp_async_commit();
        };
        // Densities of plane q (own node and halo node of this thread) into ring slot q % 4.
        auto reduce = [&](int q) {
            const C* st = stage + (size_t)(q % STAGES) * T::stage_floats;
            C rA = st[tid], rB = st[(size_t)Q * NODES + tid];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                rA = Ar<C>::add(rA, st[(size_t)i * NODES + tid]);
                rB = Ar<C>::add(rB, st[(size_t)(Q + i) * NODES + tid]);
            }
            ring[q & 3][0][ty + 1][tx + 1] = rA;
            ring[q & 3][1][ty + 1][tx + 1] = rB;
            if (halo) {
                C hA = st[OWN + tid], hB = st[(size_t)Q * NODES + OWN + tid];
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    hA = Ar<C>::add(hA, st[(size_t)i * NODES + OWN + tid]);
                    hB = Ar<C>::add(hB, st[(size_t)(Q + i) * NODES + OWN + tid]);
                }
                ring[q & 3][0][hfy][hfx] = hA;
                ring[q & 3][1][hfy][hfx] = hB;
            }
        };
        // Collide plane q (own node) with densities from ring slots (q-1, q, q+1) % 4.
        auto collide = [&](int q) {
            const C* st = stage + (size_t)(q % STAGES) * T::stage_floats;
            C f[2][Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[0][i] = st[(size_t)i * NODES + tid];
                f[1][i] = st[(size_t)(Q + i) * NODES + tid];
            }
            const int sm = (q - 1) & 3, sc = q & 3, sp = (q + 1) & 3;
            const C rA = ring[sc][0][ty + 1][tx + 1];
            const C rB = ring[sc][1][ty + 1][tx + 1];
            auto nbr = [&](int s, int i) -> C {
                const int slot = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm);
                return ring[slot][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
            };
            C gA[3], gB[3];
            node_force<L, C>(nbr, a.G, gA, gB);
            node_body_force<C>(a.body_A, gy, a.ny, gA, gB);
            node_collide<L, C>(f, rA, rB, gA, gB, a.omega_A, a.omega_B, a.tau_A, a.tau_B);
            if (owner) store_node<L, float>(a, gx, gy, z0 - 1 + q, f);
        };

#pragma unroll 1
        for (int q = 0; q < STAGES - 1; ++q) issue(q);
        cp_async_wait<STAGES - 2>();
        reduce(0);
#pragma unroll 1
        for (int q = 1; q < nplanes; ++q) {
            issue(q + LOOK);  // reuses the stage of plane q - 2, collided last iteration
            cp_async_wait<STAGES - 2>();
            reduce(q);
            __syncthreads();
            if (q >= 2) collide(q - 1);
        }
        cp_async_wait<0>();
        __syncthreads();  // the next item rewrites ring slots 0 and 1
    }
}

}  // namespace lbmsc

// Software-pipelined D3Q19 step: loads of plane z+2 in flight while plane z
// collides.
//
// Same per-node arithmetic and operation order as sc_fused_kernel (Eq. eq:be
// with the force of Eq. FORCE, paper Sec. 2.1), so results are bit-identical;
// only the schedule differs.  Per z plane q of a CTA's chunk:
//
//   1. the own-node pulls of plane q+1, issued one iteration earlier into
//      registers, are summed into the density ring and parked in a
//      thread-private shared-memory slot (double-buffered by plane parity);
//   2. the halo-ring densities of plane q+1 are summed from a thread-private
//      shared-memory stage filled by cp.async one iteration earlier (plain
//      loads for 16-bit storage, whose 2-byte values cp.async cannot copy);
//   3. one __syncthreads (the four-slot ring lets slower threads still read
//      slots q-1..q+1 while plane q+2 fills slot (q+2) % 4 next iteration);
//   4. the pulls of plane q+2 are issued (registers + cp.async) and stay in
//      flight while
//   5. plane q collides from its parked populations and the ring, and stores.
//
// Every shared-memory stage slot is written and read by one thread only, so
// the ring is the only data that needs the barrier.
#pragma once

#include "sc_async.cuh"

namespace lbmsc {

template <class S, int TX, int TY> struct PipeTile {
    using C = typename Codec<S>::C;
    static constexpr int FX = TX + 2, FY = TY + 2;
    static constexpr int H = 2 * FX + 2 * TY;
    static constexpr int OWN = TX * TY;
    static constexpr int Q2 = 2 * D3Q19::Q;
    static constexpr bool kAsyncHalo = sizeof(S) >= 4;  // cp.async copies 4, 8 or 16 bytes
    static constexpr size_t pops_bytes = (size_t)2 * Q2 * OWN * sizeof(C);
    static constexpr size_t halo_bytes = kAsyncHalo ? (size_t)Q2 * H * sizeof(S) : 0;
    static constexpr size_t ring_bytes = (size_t)4 * 2 * FY * FX * sizeof(C);
    static constexpr size_t smem_bytes = pops_bytes + halo_bytes + ring_bytes;
};

template <class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB) sc_step_pipe_kernel(const LatticeArgs<S> a) {
    using L = D3Q19;
    using T = PipeTile<S, TX, TY>;
    using C = typename Codec<S>::C;
    constexpr int Q = L::Q, Q2 = T::Q2;
    constexpr int FX = T::FX, FY = T::FY, H = T::H, OWN = T::OWN;
    static_assert(H <= OWN, "halo ring must fit in the CTA");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* const pops = reinterpret_cast<C*>(smem_raw);                         // [2][Q2][OWN]
    S* const hst = reinterpret_cast<S*>(smem_raw + T::pops_bytes);          // [Q2][H]
    C(*const ring)[2][FY][FX] = reinterpret_cast<C(*)[2][FY][FX]>(smem_raw + T::pops_bytes + T::halo_bytes);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t Np = (size_t)a.Np;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    const int nplanes = z1 - z0 + 2;  // planes z0-1 .. z1
    const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
    const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
    const bool halo = tid < H;
    int hfx, hfy;
    halo_cell<TX, TY>(tid, hfx, hfy);
    const int hgx = (x0 - 1 + hfx + nx) % nx;
    const int hgy = (y0 - 1 + hfy + ny) % ny;

    auto zof = [&](int q) {
        const int z = z0 - 1 + q;
        return z < 0 ? z + nz : (z >= nz ? z - nz : z);
    };
    auto own_density = [&](int q, const C (&R)[2][Q]) {
        ring[q & 3][0][ty + 1][tx + 1] = node_density<L, C>(R[0]);
        ring[q & 3][1][ty + 1][tx + 1] = node_density<L, C>(R[1]);
    };
    auto park = [&](int q, const C (&R)[2][Q]) {
        C* slot = pops + (size_t)(q & 1) * Q2 * OWN;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            slot[(size_t)i * OWN + tid] = R[0][i];
            slot[(size_t)(Q + i) * OWN + tid] = R[1][i];
        }
    };
    auto halo_issue = [&](int q) {
        if constexpr (T::kAsyncHalo) {
            if (halo) {
                const int z = zof(q);
                const int zs[3] = {wrap_inc(z, nz), z, wrap_dec(z, nz)};
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const size_t hn = cell(a, hgx - L::c(i, 0), hgy - L::c(i, 1), zs[L::c(i, 2) + 1]);
                    cp_async_bytes<sizeof(S)>(hst + (size_t)i * H + tid, a.fin + (size_t)i * Np + hn);
                    cp_async_bytes<sizeof(S)>(hst + (size_t)(Q + i) * H + tid, a.fin + (size_t)(Q + i) * Np + hn);
                }
            }
            cp_async_commit();
        }
    };
    auto halo_density = [&](int q) {
        if constexpr (T::kAsyncHalo) {
            cp_async_wait<0>();
            if (halo) {
                C hA = (C)hst[tid], hB = (C)hst[(size_t)Q * H + tid];
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    hA = Ar<C>::add(hA, (C)hst[(size_t)i * H + tid]);
                    hB = Ar<C>::add(hB, (C)hst[(size_t)(Q + i) * H + tid]);
                }
                ring[q & 3][0][hfy][hfx] = hA;
                ring[q & 3][1][hfy][hfx] = hB;
            }
        } else if (halo) {
            C h[2][Q];
            pull_node<L, S>(a, hgx, hgy, zof(q), h);
            ring[q & 3][0][hfy][hfx] = node_density<L, C>(h[0]);
            ring[q & 3][1][hfy][hfx] = node_density<L, C>(h[1]);
        }
    };
    auto collide = [&](int q) {
        const C* slot = pops + (size_t)(q & 1) * Q2 * OWN;
        C f[2][Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[0][i] = slot[(size_t)i * OWN + tid];
            f[1][i] = slot[(size_t)(Q + i) * OWN + tid];
        }
        const int sm = (q - 1) & 3, sc = q & 3, sp = (q + 1) & 3;
        const C rA = ring[sc][0][ty + 1][tx + 1];
        const C rB = ring[sc][1][ty + 1][tx + 1];
        auto nbr = [&](int s, int i) -> C {
            const int sl = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm);
            return ring[sl][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
        };
        C gA[3], gB[3];
        node_force<L, C>(nbr, a.G, gA, gB);
        node_body_force<C>(a.body_A, gy, a.ny, gA, gB);
        node_collide<L, C>(f, rA, rB, gA, gB, a.omega_A, a.omega_B, a.tau_A, a.tau_B);
        if (owner) store_node<L, S>(a, gx, gy, zof(q), f);
    };

    C R[2][Q];
    halo_issue(0);
    pull_node<L, S>(a, gx, gy, zof(0), R);
    own_density(0, R);
    halo_density(0);
    halo_issue(1);
    pull_node<L, S>(a, gx, gy, zof(1), R);
    own_density(1, R);
    park(1, R);
    halo_density(1);
    halo_issue(2);
    pull_node<L, S>(a, gx, gy, zof(2), R);
#pragma unroll 1
    for (int q = 1; q <= nplanes - 2; ++q) {
        own_density(q + 1, R);
        park(q + 1, R);  // slot of plane q-1, collided last iteration by this thread
        halo_density(q + 1);
        __syncthreads();
        if (q + 2 < nplanes) {
            halo_issue(q + 2);
            pull_node<L, S>(a, gx, gy, zof(q + 2), R);
        }
        collide(q);
    }
}

}  // namespace lbmsc

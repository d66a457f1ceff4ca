// Register-pipelined D3Q19 step: each thread keeps three planes of its own
// pulls in registers -- plane q colliding, plane q+1 landed and reduced to
// densities, plane q+2 in flight -- so global loads overlap the collision and
// the stores instead of stalling each plane.  The halo ring's pulls go to a
// thread-private shared-memory stage with cp.async one plane ahead.
//
// Per plane q of the CTA's z chunk (planes are numbered from z0 - 1):
//   reduce(q+1): densities of plane q+1 (own from registers, halo from the
//                cp.async stage) into ring slot (q+1) % 4;
//   __syncthreads (ring complete; four slots let slower threads still read
//                slots q-1..q+1 while slot (q+2) % 4 fills next iteration);
//   issue(q+2):  own pulls of plane q+2 into the third register set, halo
//                pulls into the stage;
//   collide(q):  from the registers of plane q and ring slots q-1..q+1.
// The three register sets rotate through a loop unrolled three times.  Same
// per-node arithmetic and order as the other step kernels (sc_node.cuh), so
// results are bit-identical.  16-bit storage copies the aligned 4-byte word
// that holds each halo value and picks its half.
#pragma once

#include <type_traits>

#include "sc_kernels.cuh"

namespace lbmsc {

// cp.async (Ampere-style asynchronous copies into shared memory) for the halo stage.
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

template <class S, int TX, int TY> struct RegPipeTile {
    static constexpr int FX = TX + 2, FY = TY + 2;
    static constexpr int H = 2 * FX + 2 * TY;
    static constexpr int Q2 = 2 * D3Q19::Q;
    static constexpr int WORD = sizeof(S) >= 4 ? (int)sizeof(S) : 4;  // bytes copied per halo value
};

template <class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB) sc_step_regpipe_kernel(const LatticeArgs<S> a) {
    using L = D3Q19;
    using T = RegPipeTile<S, TX, TY>;
    using C = typename Codec<S>::C;
    using W = typename std::conditional<T::WORD == 8, unsigned long long, unsigned int>::type;
    constexpr int Q = L::Q, Q2 = T::Q2;
    constexpr int FX = T::FX, FY = T::FY, H = T::H;
    static_assert(H <= TX * TY, "halo ring must fit in the CTA");

    __shared__ __align__(16) W hst[Q2][H];
    __shared__ C ring[4][2][FY][FX];

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
    // 16-bit storage: bit j set when staged value j sits in the upper half of its word
    unsigned hsel_lo = 0, hsel_hi = 0;

    auto issue = [&](int q, C (&X)[2][Q]) {
        const int z = zof(q);
        if (halo) {
            const int zs[3] = {wrap_inc(z, nz), z, wrap_dec(z, nz)};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const size_t hn = cell(a, hgx - L::c(i, 0), hgy - L::c(i, 1), zs[L::c(i, 2) + 1]);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int j = s * Q + i;
                    const S* src = a.fin + (size_t)j * Np + hn;
                    if constexpr (sizeof(S) >= 4) {
                        cp_async_bytes<sizeof(S)>(&hst[j][tid], src);
                    } else {
                        const uintptr_t p = reinterpret_cast<uintptr_t>(src);
                        const unsigned up = (unsigned)((p >> 1) & 1u);
                        if (j < 32)
                            hsel_lo = (hsel_lo & ~(1u << j)) | (up << j);
                        else
                            hsel_hi = (hsel_hi & ~(1u << (j - 32))) | (up << (j - 32));
                        cp_async_bytes<4>(&hst[j][tid], reinterpret_cast<const void*>(p & ~(uintptr_t)3));
                    }
                }
            }
        }
        cp_async_commit();
        pull_node<L, S>(a, gx, gy, z, X);
    };
    auto reduce = [&](int q, const C (&X)[2][Q]) {
        ring[q & 3][0][ty + 1][tx + 1] = node_density<L, C>(X[0]);
        ring[q & 3][1][ty + 1][tx + 1] = node_density<L, C>(X[1]);
        cp_async_wait<0>();
        if (halo) {
            C h[2][Q];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int j = s * Q + i;
                    if constexpr (sizeof(S) >= 4) {
                        const W w = hst[j][tid];
                        S v;
                        memcpy(&v, &w, sizeof(S));
                        h[s][i] = (C)v;
                    } else {
                        const unsigned word = hst[j][tid];
                        const unsigned up = j < 32 ? (hsel_lo >> j) & 1u : (hsel_hi >> (j - 32)) & 1u;
                        const unsigned short bits = (unsigned short)(up ? (word >> 16) : (word & 0xffffu));
                        S v;
                        memcpy(&v, &bits, sizeof(S));
                        const C off = (C)__fmul_rn((float)L::w(i), (float)(s == 0 ? a.ref_A : a.ref_B));
                        h[s][i] = Codec<S>::decode(v, off);
                    }
                }
            ring[q & 3][0][hfy][hfx] = node_density<L, C>(h[0]);
            ring[q & 3][1][hfy][hfx] = node_density<L, C>(h[1]);
        }
    };
    auto collide = [&](int q, C (&X)[2][Q]) {
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
        node_collide<L, C>(X, rA, rB, gA, gB, a.omega_A, a.omega_B, a.tau_A, a.tau_B);
        if (owner) store_node<L, S>(a, gx, gy, zof(q), X, rA, rB);
    };
    // one plane of the steady state; false once the chunk is done
    auto body = [&](int q, C (&Xq)[2][Q], C (&Xq1)[2][Q], C (&Xq2)[2][Q]) -> bool {
        if (q > nplanes - 2) return false;
        reduce(q + 1, Xq1);
        __syncthreads();
        if (q + 2 < nplanes) issue(q + 2, Xq2);
        collide(q, Xq);
        return true;
    };

    C R0[2][Q], R1[2][Q], R2[2][Q];
    issue(0, R0);
    reduce(0, R0);
    issue(1, R1);
    reduce(1, R1);
    issue(2, R2);
#pragma unroll 1
    for (int q = 1;; q += 3) {
        if (!body(q, R1, R2, R0)) break;
        if (!body(q + 1, R2, R0, R1)) break;
        if (!body(q + 2, R0, R1, R2)) break;
    }
}

}  // namespace lbmsc

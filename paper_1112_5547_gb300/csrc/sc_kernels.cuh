// Fused two-component Shan-Chen step on sm_103a: register-pipelined kernel,
// moments / diagnostics kernel, initialisation and the diagnostics fold.
//
// One kernel performs a whole time step of Eq. eq:be with the force of
// Eq. FORCE (paper Sec. 2.1): pull-streaming of both species' populations,
// densities and momenta, the neighbour-density force, the common velocity u',
// the velocity-shifted equilibrium and BGK relaxation, and the store.  The
// per-node arithmetic is in sc_node.cuh.
//
// Storage: structure of arrays, plane (s*Q + i) holds f_is for all N nodes,
// node index x + nx*(y + ny*z).  The buffer holds post-collision values at the
// node where they were produced; pulling f_i(x, t) = f*_i(x - c_i, t - 1) is the
// streaming step, so stores are always aligned and coalesced.
//
// Tiling: a CTA owns a TX x TY tile of (x, y) columns and marches along z over
// a chunk of planes.  The force at plane z needs the densities of planes z-1,
// z, z+1 on the tile plus a one-node ring; they live in a ring of shared
// memory.  Each iteration pulls the populations of plane z+1 (kept in
// registers for the next iteration), writes their densities to the ring,
// computes the densities of the ring's halo nodes (extra pulls served mostly
// by L2, since neighbouring tiles read the same lines at about the same time),
// then collides plane z.  The halo costs 2(TX+TY)+4 extra density pulls per
// TX*TY nodes of a plane, in x and y only: marching removes the z halo.
#pragma once

#include "sc_node.cuh"

namespace lbmsc {

enum KernelMode { kModeStep = 0, kModeMoments = 1 };

// Pulled populations of node (x, y, z): f_is = f*_is(x - c_i).
template <class L, class S>
__device__ __forceinline__ void pull_node(const LatticeArgs<S>& a, int x, int y, int z,
                                          typename Codec<S>::C (&f)[2][L::Q]) {
    using C = typename Codec<S>::C;
    const int nz = a.nz;
    int zs[3] = {z, z, z};  // source plane for c_z = -1, 0, +1
    if (L::D == 3) {
        zs[0] = wrap_inc(z, nz);
        zs[2] = wrap_dec(z, nz);
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        // x - c_x and y - c_y lie in [-1, n]: the ghost images make them valid
        const size_t node = cell(a, x - L::c(i, 0), y - L::c(i, 1), zs[L::c(i, 2) + 1]);
        if constexpr (Codec<S>::kRest) {
            const uint32_t v = __ldg(&(a.fin + (size_t)i * (size_t)a.Np + node)->v);
            rest_decode<S>(v, (C)L::w(i), __ldg(rest_rho<L>(a.fin, a.Np) + node), f[0][i], f[1][i]);
        } else {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const C off = Codec<S>::kOffset ? (C)__fmul_rn((float)L::w(i), (float)(s == 0 ? a.ref_A : a.ref_B)) : (C)0;
                f[s][i] = Codec<S>::load(a.fin + (size_t)(s * L::Q + i) * (size_t)a.Np + node, off);
            }
        }
    }
}

// Store the values of one cell.  base: the offset bases of the rest-offset
// storage (the node's densities rho_A, rho_B; any value works as long as the
// stored one is used, and a node's own density keeps the offsets small);
// ignored by the other storage types.
template <class L, class S>
__device__ __forceinline__ void store_cell(const LatticeArgs<S>& a, size_t c,
                                           const typename Codec<S>::C (&f)[2][L::Q], float2 base) {
    using C = typename Codec<S>::C;
    if constexpr (Codec<S>::kRest) {
        // the bases, kept in FP32 for the nodes that pull from this cell
        const float2 r = base;
        __stcs(rest_rho<L>(a.fout, a.Np) + c, r);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            __stcs(&(a.fout + (size_t)i * (size_t)a.Np + c)->v, rest_encode<S>(f[0][i], f[1][i], (C)L::w(i), r));
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const C off = Codec<S>::kOffset ? (C)__fmul_rn((float)L::w(i), (float)(s == 0 ? a.ref_A : a.ref_B)) : (C)0;
                Codec<S>::store(a.fout + (size_t)(s * L::Q + i) * (size_t)a.Np + c, f[s][i], off);
            }
        }
    }
}

// Post-collision populations of node (x, y, z), x in [0, nx), y in [0, ny), and
// of its periodic images in the ghost columns x in {-2, -1, nx, nx + 1} and
// rows y in {-2, -1, ny, ny + 1}.  Two ghost layers let a node of the halo
// ring itself (x = -1 .. nx) pull without wrapping.
// rA, rB: the node's densities (pre-collision, equal to the post-collision
// sums in exact arithmetic), the offset bases of rest-offset storage.
template <class L, class S>
__device__ __forceinline__ void store_node(const LatticeArgs<S>& a, int x, int y, int z,
                                           const typename Codec<S>::C (&f)[2][L::Q], typename Codec<S>::C rA,
                                           typename Codec<S>::C rB) {
    float2 base = make_float2(0.f, 0.f);
    if constexpr (Codec<S>::kRest) base = make_float2(rA, rB);
    store_cell<L, S>(a, cell(a, x, y, z), f, base);
    const int nx = a.nx, ny = a.ny;
    // x images: the two ghost columns the pulls read, widened to a whole 32-byte
    // sector on each side (columns -GX .. -1 and nx .. nx + GX - 1) when the
    // lattice is at least that wide, so the ghost sectors are written whole: a
    // partly written sector costs a read of the sector from HBM besides its
    // write (measured: 20 % more write traffic on 128-wide rows without it)
    constexpr int kSector = 32 / (int)sizeof(S) > 2 ? 32 / (int)sizeof(S) : 2;
    const int GX = nx >= kSector ? kSector : 2;
    if (x < GX || x >= nx - GX || y < 2 || y >= ny - 2) {
#pragma unroll 1
        for (int ix = -2; ix <= 2; ++ix) {
            const int xi = x + ix * nx;
            if (xi < -GX || xi > nx + GX - 1) continue;
#pragma unroll 1
            for (int iy = -2; iy <= 2; ++iy) {
                const int yi = y + iy * ny;
                if ((ix | iy) == 0 || yi < -2 || yi > ny + 1) continue;
                store_cell<L, S>(a, cell(a, xi, yi, z), f, base);
            }
        }
    }
}

// Halo ring cell of thread tid (frame coordinates; frame (1, 1) = tile (0, 0)):
// the top row, the bottom row, the left column, the right column.
template <int TX, int TY> __device__ __forceinline__ void halo_cell(int tid, int& hfx, int& hfy) {
    constexpr int FX = TX + 2, FY = TY + 2;
    if (tid < FX) {
        hfx = tid;
        hfy = 0;
    } else if (tid < 2 * FX) {
        hfx = tid - FX;
        hfy = FY - 1;
    } else if (tid < 2 * FX + TY) {
        hfx = 0;
        hfy = tid - 2 * FX + 1;
    } else {
        hfx = FX - 1;
        hfy = tid - 2 * FX - TY + 1;
    }
}

__device__ __forceinline__ double diag_fold(int k, double a, double b) {
    return (k == kMaxSpeed) ? fmax(a, b) : (k == kMinRhoA || k == kMinRhoB) ? fmin(a, b) : a + b;
}

template <class L, class S, int TX, int TY, int MODE, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB)
    sc_fused_kernel(const LatticeArgs<S> a, const FieldArgs<typename Codec<S>::C> fo) {
    using C = typename Codec<S>::C;
    using A = Ar<C>;
    constexpr int Q = L::Q;
    constexpr int FX = TX + 2, FY = TY + 2;
    constexpr int NPL = L::D == 3 ? 3 : 1;
    constexpr int H = 2 * FX + 2 * TY;
    static_assert(H <= TX * TY, "halo ring must fit in the CTA");
    __shared__ C srho[NPL][2][FY][FX];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
    const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
    const bool halo = tid < H;
    int hfx, hfy;
    halo_cell<TX, TY>(tid, hfx, hfy);
    const int hgx = (x0 - 1 + hfx + nx) % nx;
    const int hgy = (y0 - 1 + hfy + ny) % ny;

    double acc[kNumDiag];
    if (MODE == kModeMoments) {
#pragma unroll
        for (int k = 0; k < kNumDiag; ++k) acc[k] = 0.0;
        acc[kMinRhoA] = 1e300;
        acc[kMinRhoB] = 1e300;
    }

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
        const C r0 = srho[sc][0][ty + 1][tx + 1];
        const C r1 = srho[sc][1][ty + 1][tx + 1];
        auto nbr = [&](int s, int i) -> C {
            const int slot = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm);
            return srho[slot][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
        };
        const size_t node = (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * z);
        if (MODE == kModeStep) {
            node_update<L, C>(a, gy, nbr, f, r0, r1);
            if (owner) store_node<L, S>(a, gx, gy, z, f, r0, r1);
        } else {
            // SC: physical velocity u = (j_A + j_B + (F_A + F_B) / 2) / rho (F dt/2
            // shift, Sec. 2.3).  FE (Sec. 2.2): u = sum_i f_i c_i / rho, and the
            // reported densities are rho_A = (rho + phi)/2, rho_B = (rho - phi)/2.
            const bool fe = a.model == kModelFE;
            C gA[3] = {(C)0, (C)0, (C)0}, gB[3] = {(C)0, (C)0, (C)0};
            if (!fe) {
                node_force<L, C>(nbr, a.G, gA, gB);
                node_body_force<C>(a.body_A, gy, a.ny, gA, gB);
            }
            const C rA = fe ? A::mul((C)0.5, A::add(r0, r1)) : r0;
            const C rB = fe ? A::mul((C)0.5, A::sub(r0, r1)) : r1;
            C jA[3], jB[3] = {(C)0, (C)0, (C)0};
            node_momentum<L, C>(f[0], jA);
            if (!fe) node_momentum<L, C>(f[1], jB);
            const C rho = fe ? r0 : A::add(rA, rB);
            const C inv_rho = A::rcp(rho);
            C u[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const C half_force = A::mul((C)0.5, A::fma(rA, gA[d], A::mul(rB, gB[d])));
                u[d] = A::mul(A::add(A::add(jA[d], jB[d]), half_force), inv_rho);
            }
            const C p = A::mul(A::fma(A::mul(a.G, rA), rB, rho), (C)(1.0 / 3.0));
            if (owner) {
                if (fo.rhoA) fo.rhoA[node] = rA;
                if (fo.rhoB) fo.rhoB[node] = rB;
                if (fo.u)
#pragma unroll
                    for (int d = 0; d < L::D; ++d) fo.u[(size_t)d * (size_t)a.N + node] = u[d];
                if (fo.p) fo.p[node] = p;
                if (fo.partials) {
                    const double dA = (double)rA, dB = (double)rB, drho = dA + dB;
                    double uu = 0.0;
#pragma unroll
                    for (int d = 0; d < 3; ++d) uu += (double)u[d] * (double)u[d];
                    const bool finite = isfinite(dA) && isfinite(dB) && isfinite(uu) && isfinite((double)p);
                    if (finite) {
                        acc[kMassA] += dA;
                        acc[kMassB] += dB;
                        acc[kMomX] += (double)u[0] * drho;
                        acc[kMomY] += (double)u[1] * drho;
                        acc[kMomZ] += (double)u[2] * drho;
                        acc[kKE] += 0.5 * drho * uu;
                        acc[kMaxSpeed] = fmax(acc[kMaxSpeed], sqrt(uu));
                        acc[kMinRhoA] = fmin(acc[kMinRhoA], dA);
                        acc[kMinRhoB] = fmin(acc[kMinRhoB], dB);
                    } else {
                        acc[kNonFinite] += 1.0;
                    }
                    // periodic minimum-image distance from the window centre
                    double dx = fabs((double)gx - fo.win_c[0]);
                    double dy = fabs((double)gy - fo.win_c[1]);
                    double dz = fabs((double)z - fo.win_c[2]);
                    dx = fmin(dx, (double)nx - dx);
                    dy = fmin(dy, (double)ny - dy);
                    dz = fmin(dz, (double)nz - dz);
                    const double r2 = dx * dx + dy * dy + (L::D == 3 ? dz * dz : 0.0);
                    if (r2 < fo.r_in2) {
                        acc[kInCount] += 1.0;
                        acc[kInRhoA] += dA;
                        acc[kInP] += (double)p;
                    }
                    if (r2 > fo.r_out2) {
                        acc[kOutCount] += 1.0;
                        acc[kOutRhoA] += dA;
                        acc[kOutP] += (double)p;
                    }
                    // inside the drop: phi = rho_A - rho_B >= 0, compared in the compute type (Sec. 4.2)
                    if (rA >= rB) acc[kDropNodes] += 1.0;
                }
            }
        }
    };

    C cur[2][Q];
    if (L::D == 2) {
        density_plane(0, 0, cur);
        __syncthreads();
        process(cur, 0, 0, 0, 0);
    } else {
        const int z0 = a.zbase + blockIdx.z * a.zchunk;
        const int z1 = min(z0 + a.zchunk, a.zend);
        {
            C tmp[2][Q];
            density_plane(0, z0 == 0 ? nz - 1 : z0 - 1, tmp);
        }
        density_plane(1, z0, cur);
        int sm = 0, sc = 1, sp = 2;
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

    if (MODE == kModeMoments && fo.partials) {
        // CTA reduction of the diagnostics: warp shuffles, then one warp over the warps.
        constexpr int NW = TX * TY / 32;
        __shared__ double red[NW][kNumDiag];
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int k = 0; k < kNumDiag; ++k) {
            double v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = diag_fold(k, v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (tid < kNumDiag) {
            const int k = tid;
            double v = red[0][k];
            for (int w = 1; w < NW; ++w) v = diag_fold(k, v, red[w][k]);
            const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
            fo.partials[b * kNumDiag + k] = v;
        }
    }
}

// Low-register variant of the step: the populations of plane z are not kept
// in registers while plane z+1 is reduced to densities; they are pulled a
// second time for the collision, one iteration after their first load, when
// they are normally still in L1.  Holding only one plane of pulls lets more
// CTAs share an SM (more loads in flight), and the four-slot density ring
// needs one __syncthreads per plane.  Arithmetic and order as sc_fused_kernel.
template <class L, class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB) sc_step_reload_kernel(const LatticeArgs<S> a) {
    using C = typename Codec<S>::C;
    constexpr int Q = L::Q;
    constexpr int FX = TX + 2, FY = TY + 2;
    constexpr int NPL = L::D == 3 ? 4 : 1;
    constexpr int H = 2 * FX + 2 * TY;
    static_assert(H <= TX * TY, "halo ring must fit in the CTA");
    __shared__ C ring[NPL][2][FY][FX];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
    const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
    const bool halo = tid < H;
    int hfx, hfy;
    halo_cell<TX, TY>(tid, hfx, hfy);
    const int hgx = (x0 - 1 + hfx + nx) % nx;
    const int hgy = (y0 - 1 + hfy + ny) % ny;

    auto density_plane = [&](int slot, int z) {
        C f[2][Q];
        pull_node<L, S>(a, gx, gy, z, f);
        ring[slot][0][ty + 1][tx + 1] = node_density<L, C>(f[0]);
        ring[slot][1][ty + 1][tx + 1] = node_density<L, C>(f[1]);
        if (halo) {
            pull_node<L, S>(a, hgx, hgy, z, f);
            ring[slot][0][hfy][hfx] = node_density<L, C>(f[0]);
            ring[slot][1][hfy][hfx] = node_density<L, C>(f[1]);
        }
    };
    auto collide = [&](int sm, int sc, int sp, int z) {
        C f[2][Q];
        pull_node<L, S>(a, gx, gy, z, f);
        const C rA = ring[sc][0][ty + 1][tx + 1];
        const C rB = ring[sc][1][ty + 1][tx + 1];
        auto nbr = [&](int s, int i) -> C {
            const int sl = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm);
            return ring[sl][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
        };
        node_update<L, C>(a, gy, nbr, f, rA, rB);
        if (owner) store_node<L, S>(a, gx, gy, z, f, rA, rB);
    };

    if (L::D == 2) {
        density_plane(0, 0);
        __syncthreads();
        collide(0, 0, 0, 0);
        return;
    }
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    // ring slot of plane z is (z - z0 + 1) & 3
    density_plane(0, z0 == 0 ? nz - 1 : z0 - 1);
    density_plane(1, z0);
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        const int k = z - z0 + 1;
        density_plane((k + 1) & 3, z + 1 == nz ? 0 : z + 1);
        __syncthreads();
        collide((k - 1) & 3, k & 3, (k + 1) & 3, z);
    }
}

// Second pass of the diagnostics: one CTA folds the per-CTA partials.
template <int NT>
__global__ void __launch_bounds__(NT) sc_diag_finish_kernel(const double* __restrict__ partials,
                                                            long long nparts, double* __restrict__ out) {
    __shared__ double red[NT / 32][kNumDiag];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc[kNumDiag];
#pragma unroll
    for (int k = 0; k < kNumDiag; ++k) acc[k] = 0.0;
    acc[kMinRhoA] = 1e300;
    acc[kMinRhoB] = 1e300;
    for (long long b = tid; b < nparts; b += NT) {
#pragma unroll
        for (int k = 0; k < kNumDiag; ++k) acc[k] = diag_fold(k, acc[k], partials[b * kNumDiag + k]);
    }
#pragma unroll
    for (int k = 0; k < kNumDiag; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = diag_fold(k, v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (tid < kNumDiag) {
        const int k = tid;
        double v = red[0][k];
        for (int w = 1; w < NT / 32; ++w) v = diag_fold(k, v, red[w][k]);
        out[k] = v;
    }
}

// Populations of the rest / moving equilibrium (planes [zlo, zhi)): the buffer slot of direction i
// at node x holds f^eq_i(rho_s(x + c_i), u(x + c_i)), so pulling it at x + c_i
// gives f_i(x + c_i, 0) = f^eq_i of that node.  The ghost columns and rows get
// the values of their periodic images.
template <class L, class S>
__global__ void __launch_bounds__(256)
    sc_init_kernel(const LatticeArgs<S> a, const typename Codec<S>::C* __restrict__ rhoA,
                   const typename Codec<S>::C* __restrict__ rhoB, const typename Codec<S>::C* __restrict__ u, int zlo,
                   int zhi) {
    using C = typename Codec<S>::C;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int ex = nx + 4, ey = ny + 4;  // cells x in [-2, nx + 1], y in [-2, ny + 1]
    // the cells of planes [zlo, zhi); they read the fields of planes zlo - 1 .. zhi (periodic)
    const long long ncells = (long long)ex * ey * zhi;
    for (long long k = (long long)ex * ey * zlo + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ncells;
         k += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(k % ex) - 2;
        const int cy = (int)((k / ex) % ey) - 2;
        const int z = (int)(k / ((long long)ex * ey));
        const size_t n = cell(a, cx, cy, z);
        const int x = ((cx % nx) + nx) % nx, y = ((cy % ny) + ny) % ny;
        C fr[2][L::Q];  // rest-offset storage: the cell's values, stored together
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int sx = (x + L::c(i, 0) + nx) % nx;
            const int sy = (y + L::c(i, 1) + ny) % ny;
            const int sz = L::D == 3 ? (z + L::c(i, 2) + nz) % nz : 0;
            const size_t m = (size_t)sx + (size_t)nx * ((size_t)sy + (size_t)ny * sz);
            C uv[3] = {0, 0, 0};
            if (u)
                for (int d = 0; d < L::D; ++d) uv[d] = u[(size_t)d * (size_t)a.N + m];
            C uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
            C cu = (C)0;
            for (int d = 0; d < L::D; ++d) cu += (C)L::c(i, d) * uv[d];
            const C shape = (C)1 - (C)1.5 * uu + cu * ((C)3 + (C)4.5 * cu);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                // SC: species densities; FE: f from rho = rho_A + rho_B, g from phi = rho_A - rho_B
                const C rho = a.model == kModelFE ? (s == 0 ? rhoA[m] + rhoB[m] : rhoA[m] - rhoB[m])
                                                  : (s == 0 ? rhoA[m] : rhoB[m]);
                const C f = (C)L::w(i) * rho * shape;
                if constexpr (Codec<S>::kRest) {
                    fr[s][i] = f;
                } else {
                    const C off = Codec<S>::kOffset ? (C)__fmul_rn((float)L::w(i), (float)(s == 0 ? a.ref_A : a.ref_B)) : (C)0;
                    Codec<S>::store(a.fout + (size_t)(s * L::Q + i) * (size_t)a.Np + n, f, off);
                }
            }
        }
        if constexpr (Codec<S>::kRest) {
            // rest-offset bases: the sums of the cell's stored values, in a fixed order
            float2 r = make_float2(fr[0][0], fr[1][0]);
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                r.x = __fadd_rn(r.x, fr[0][i]);
                r.y = __fadd_rn(r.y, fr[1][i]);
            }
            store_cell<L, S>(a, n, fr, r);
        }
    }
}

}  // namespace lbmsc

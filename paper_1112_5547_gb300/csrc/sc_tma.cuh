// TMA-fed D3Q19 step (FP32 storage, or 16-bit storage decoded on the pull).
//
// Same per-node arithmetic and order as the other step kernels (sc_node.cuh:
// Eq. eq:be with the force of Eq. FORCE, paper Sec. 2.1), so results are
// bit-identical; only the data movement differs.  Per z plane of the CTA's
// chunk one elected thread issues 38 tensor copies (cp.async.bulk.tensor, one
// per species and direction, completing on an mbarrier), each a box of
// (TX + 8) x (TY + 2) values of the ghost-padded population plane that the
// direction is pulled from:
//     x from x0 - 4 (16-byte aligned, as TMA requires) to x0 + TX + 4,
//     y from y0 - 1 - c_y to y0 + TY - c_y,  z = plane - c_z (periodic).
// The pulled value of frame node (fx, fy) (frame (1, 1) = tile (0, 0)) is then
// box[fy][fx + 3 - c_x]: every pull, for the tile and for its one-node halo
// ring, is a shared-memory load at a constant offset (16-bit storage: boxes
// of TX + 16 values from x0 - 8, same rule with 7 for 3).
//
// Per plane q: wait for plane q's copies; read the own node's 38 pulls into
// registers and write own and halo densities to the four-slot ring; one
// barrier (ring complete, stage q read); the elected thread refills a stage;
// collide plane q - 1 from registers and store.  The refill schedule (which
// stage, before or after the wait) depends on the storage type, see tma_item.
// Every mbarrier wait is bounded: on expiry the CTA raises the error word,
// waits (bounded) for its copies still in flight and leaves (the host reports
// LBM_ERR_TIMEOUT).  tma_item is the per-item pipeline; the solo kernel runs
// one item per CTA, the batch kernel (sc_batch.cuh) a work list of them.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "sc_kernels.cuh"

namespace lbmsc {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
// Bring a tensor map held in global memory into the copy engine's descriptor cache.
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Iterations of mbarrier.try_wait before a wait is declared lost (each try
// waits up to a hardware time slice; this bound is seconds, far beyond any
// plane's copies).
constexpr int kMbarSpinLimit = 1 << 24;

// Geometry of one CTA's stages for storage type St (FP32, 16-bit offsets, or
// paired 16-bit rest offsets).  Population boxes: (TX + 2 PAD) x (TY + 2)
// elements, PAD = 16 bytes of elements on each side in x (TMA copies start on
// 16-byte boundaries); one box per species and direction (Q2 = 2 Q), or one
// per direction for the paired rest-offset words (both species in one 32-bit
// element).  Rest-offset storage also stages, per source plane z - 1, z, z + 1,
// a box of (TX + 4) x (TY + 4) float2 densities (rho_A, rho_B) of the storing
// nodes.
template <int TX, int TY, int S, class St = float> struct TmaTile {
    static constexpr int E = (int)sizeof(St);
    static constexpr int PAD = 16 / E;
    static constexpr int BX = TX + 2 * PAD, BY = TY + 2;
    static constexpr int FX = TX + 2, FY = TY + 2;
    static constexpr int H = 2 * FX + 2 * TY;
    static constexpr bool REST = Codec<St>::kRest;
    static constexpr int Q2 = (REST ? 1 : 2) * D3Q19::Q;  // population boxes per plane
    static constexpr int RBX = TX + 4, RBY = TY + 4;
    static constexpr int NR = REST ? 3 : 0;  // density boxes per plane
    static constexpr unsigned box_bytes = BX * BY * E;
    static constexpr unsigned box_stride = (box_bytes + 127) / 128 * 128;  // TMA destinations 128-byte aligned
    static constexpr unsigned rbox_bytes = RBX * RBY * 8;
    static constexpr unsigned rbox_stride = (rbox_bytes + 127) / 128 * 128;
    static constexpr unsigned stage_bytes = Q2 * box_stride + NR * rbox_stride;
    static constexpr unsigned tx_bytes = Q2 * box_bytes + NR * rbox_bytes;  // bytes landing per plane
    static constexpr size_t ring_bytes = (size_t)4 * 2 * FY * FX * 4;
    // S stage barriers and one barrier nothing arrives on (the wait-probe test hook)
    static constexpr size_t smem_bytes = 128 + (size_t)S * stage_bytes + ring_bytes + (size_t)(S + 1) * 8;
    static_assert((BX * E) % 16 == 0 && (RBX * 8) % 16 == 0, "TMA box rows are whole 16-byte units");
};

// The tensor maps of one population buffer: the population planes and, for
// rest-offset storage, its float2 density plane.
struct TmaMaps {
    CUtensorMap pop;
    CUtensorMap rho;
};

// Shared memory of one CTA: S stages of boxes, the density ring, S mbarriers
// and one mbarrier that nothing ever arrives on (bars[S]: the wait-probe test
// hook waits on it, so that a bounded wait runs out without any fault).
template <int TX, int TY, int S, class St = float> struct TmaSmem {
    using T = TmaTile<TX, TY, S, St>;
    unsigned char* stage;
    float (*ring)[2][T::FY][T::FX];
    uint64_t* bars;

    __device__ __forceinline__ explicit TmaSmem(unsigned char* raw) {
        unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~(uintptr_t)127);
        stage = base;
        ring = reinterpret_cast<float(*)[2][T::FY][T::FX]>(base + (size_t)S * T::stage_bytes);
        bars = reinterpret_cast<uint64_t*>(base + (size_t)S * T::stage_bytes + T::ring_bytes);
    }
    __device__ __forceinline__ void init_barriers() {
        if (threadIdx.x + threadIdx.y * blockDim.x == 0) {
#pragma unroll
            for (int k = 0; k <= S; ++k) mbar_init(&bars[k], 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
};

// The copies of plane z (0 <= z < nz) of a work item (tile x0, y0) into the
// stage of pipeline slot g: 38 population boxes, one per species and
// direction (19 paired boxes and 3 density boxes for rest-offset storage),
// completing on the slot's mbarrier.  Elected thread only.
template <int TX, int TY, int S, class St>
__device__ __forceinline__ void tma_issue_plane(const CUtensorMap* pmap, const CUtensorMap* rmap, int x0, int y0, int z,
                                                int gxo, int gyo, int nz, unsigned g, const TmaSmem<TX, TY, S, St>& sm) {
    using L = D3Q19;
    using T = TmaTile<TX, TY, S, St>;
    const unsigned st = g % S;
    mbar_arrive_expect_tx(&sm.bars[st], T::tx_bytes);
    unsigned char* sb = sm.stage + (size_t)st * T::stage_bytes;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int zs = z - L::c(i, 2);
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        const int cy = y0 + gyo - 1 - L::c(i, 1);
#pragma unroll
        for (int s = 0; s < T::Q2 / L::Q; ++s) {
            const int j = s * L::Q + i;
            tma_load_4d(sb + (size_t)j * T::box_stride, pmap, &sm.bars[st], x0 + gxo - T::PAD, cy, zs, j);
        }
    }
    if constexpr (T::REST) {
        // float2 densities of nodes x0 - 2 .. x0 + TX + 1, y0 - 2 .. y0 + TY + 1
        // (the map counts floats in x: 2 per node)
        unsigned char* rb = sb + (size_t)T::Q2 * T::box_stride;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            int zs = z + dz;
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            tma_load_4d(rb + (size_t)(dz + 1) * T::rbox_stride, rmap, &sm.bars[st], 2 * (x0 + gxo - 2), y0 + gyo - 2,
                        zs, 0);
        }
    }
}

// The pulled value f_is of frame node (fx, fy) (frame (1, 1) = tile node
// (0, 0)) for direction i from a landed stage, decoded to FP32 with the same
// operations as pull_node.
template <int TX, int TY, int S, class St>
__device__ __forceinline__ float tma_pulled(const unsigned char* sb, int s, int i, int fx, int fy, float ref_s) {
    using L = D3Q19;
    using T = TmaTile<TX, TY, S, St>;
    const int j = s * L::Q + i;
    const St* box = reinterpret_cast<const St*>(sb + (size_t)j * T::box_stride);
    const St v = box[fy * T::BX + fx + T::PAD - 1 - L::c(i, 0)];
    if constexpr (std::is_same<St, float>::value) {
        return v;
    } else {
        return Codec<St>::decode(v, __fmul_rn((float)L::w(i), ref_s));
    }
}

// The pulled pair (f_iA, f_iB) of frame node (fx, fy) for direction i from a
// landed stage of paired rest-offset storage, decoded with the density pair
// of the source node x - c_i (the same operations as pull_node).
template <int TX, int TY, int S, class St>
__device__ __forceinline__ void tma_pulled_pair(const unsigned char* sb, int i, int fx, int fy, float& fA, float& fB) {
    using L = D3Q19;
    using T = TmaTile<TX, TY, S, St>;
    const uint32_t* box = reinterpret_cast<const uint32_t*>(sb + (size_t)i * T::box_stride);
    const uint32_t v = box[fy * T::BX + fx + T::PAD - 1 - L::c(i, 0)];
    const float2* rb =
        reinterpret_cast<const float2*>(sb + (size_t)T::Q2 * T::box_stride + (size_t)(1 - L::c(i, 2)) * T::rbox_stride);
    rest_decode<St>(v, (float)L::w(i), rb[(fy + 1 - L::c(i, 1)) * T::RBX + fx + 1 - L::c(i, 0)], fA, fB);
}

// Density rho_s of frame node (fx, fy) for one species s (a run-time value:
// the same instructions read the other species' planes or half-words), with
// the values decoded and summed exactly as node_density sums a node's pulls
// (moving populations in order, the rest population last).
template <int TX, int TY, int S, class St>
__device__ __forceinline__ float tma_density(const unsigned char* sb, int s, int fx, int fy, float ref_s) {
    using L = D3Q19;
    using T = TmaTile<TX, TY, S, St>;
    auto pulled = [&](int i) -> float {
        if constexpr (T::REST) {
            const uint32_t* box = reinterpret_cast<const uint32_t*>(sb + (size_t)i * T::box_stride);
            const uint32_t v = box[fy * T::BX + fx + T::PAD - 1 - L::c(i, 0)];
            const float2* rb = reinterpret_cast<const float2*>(sb + (size_t)T::Q2 * T::box_stride +
                                                               (size_t)(1 - L::c(i, 2)) * T::rbox_stride);
            const float2 r = rb[(fy + 1 - L::c(i, 1)) * T::RBX + fx + 1 - L::c(i, 0)];
            return __fmaf_rn((float)L::w(i), s == 0 ? r.x : r.y, s == 0 ? Codec<St>::lo(v) : Codec<St>::hi(v));
        } else {
            return tma_pulled<TX, TY, S, St>(sb, s, i, fx, fy, ref_s);
        }
    };
    float r = pulled(1);
#pragma unroll
    for (int i = 2; i < L::Q; ++i) r = __fadd_rn(r, pulled(i));
    return __fadd_rn(r, pulled(0));
}

// The item a CTA runs after the current one (batch kernels): the elected
// thread issues its first planes into the stages the current item frees,
// so the pipeline does not drain between items.
struct TmaNext {
    const CUtensorMap* map;
    int x0, y0, z0, gxo, gyo, nz, nplanes;  // nplanes = 0: no next item
    int down;                               // the item marches down (tma_march_down)
};

// In the batch kernels the z chunks of a lattice march in alternating
// directions: chunk k = z0 / zchunk upwards (planes z0 - 1, z0, ..., z1) if k
// is even, downwards (z1, z1 - 1, ..., z0 - 1) if k is odd.  Two neighbouring
// chunks then reach the planes they both read (each one's boundary planes,
// z0 - 1 and z1) at the same time when they run together, at the start of
// both or at the end of both, instead of one at its start and the other at
// its end.  A batch's work list places a lattice's chunks a few dozen items
// apart, so they do run together (ragged 64-lattice set: 12.85 -> 13.05
// GLUPS, 96^3 lattices 12.5 -> 13.0); the solo grid launches the chunks of a
// plane of tiles hundreds of CTAs apart, and there the alternation measured
// 0.2 - 0.9 % slower, so the solo kernel marches every chunk upwards.
__device__ __forceinline__ bool tma_march_down(int z0, int zchunk) { return ((z0 / zchunk) & 1) != 0; }

// Plane of pipeline step q (0 .. nplanes - 1) of an item of planes z0 .. z0 +
// nplanes - 3 (periodic in nz).
__device__ __forceinline__ int tma_plane(int z0, int nplanes, int nz, bool down, int q) {
    const int z = down ? z0 + nplanes - 2 - q : z0 - 1 + q;
    return z < 0 ? z + nz : (z >= nz ? z - nz : z);
}

// Called by the elected thread at the start of every plane of an item (plane
// q of nplanes); the persistent batch kernel uses it to take its next work
// item late in the current one and fill the TmaNext before the pre-issue.
struct TmaNoHook {
    __device__ __forceinline__ void operator()(int, int) const {}
};

// One work item through the plane pipeline: the TX x TY tile at (x0, y0),
// planes z0 .. min(z0 + zchunk, nz) - 1.  qbase counts the planes this CTA
// pushed through its stages before (the mbarrier phases continue from there).
// preissued: the item's first planes were issued by the previous item (as
// its TmaNext; FP32 batch kernel only).  Every thread returns the number of
// planes the item used, or -1 if a wait was lost (the error word is then
// raised, and the copies still in flight have been waited for, again with a
// bound).  The caller must synchronise the CTA between two items.
// alternate: odd chunks march downwards (tma_march_down; batch kernels).
template <int TX, int TY, int S, class St = float, class Hook = TmaNoHook, int FORCING = kForcingShift>
__device__ __forceinline__ int tma_item(const CUtensorMap* pmap, const CUtensorMap* rmap, const LatticeArgs<St>& a,
                                        int x0, int y0, int z0, unsigned qbase, const TmaSmem<TX, TY, S, St>& sm,
                                        int* __restrict__ err, bool preissued = false, const TmaNext* nxt = nullptr,
                                        Hook hook = Hook(), bool alternate = false) {
    using L = D3Q19;
    using T = TmaTile<TX, TY, S, St>;
    using C = float;
    constexpr int Q = L::Q, H = T::H;
    static_assert(H <= TX * TY, "halo ring must fit in the CTA");

    auto ring = sm.ring;
    uint64_t* const bars = sm.bars;
    // linear thread id: the tile shape need not be the block shape (the mixed
    // batch kernels run two tile shapes in blocks of the same thread count)
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int z1 = min(z0 + a.zchunk, nz);
    const int nplanes = z1 - z0 + 2;  // planes z0-1 .. z1
    const bool owner = (x0 + tx) < nx && (y0 + ty) < ny;
    const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
    const C kolmo = kolmogorov_accel<C>(a.body_A, gy, ny);  // the row's forcing, the same on every plane
    // Two issue schedules, measured per storage type at 512^3: FP32 refills a
    // stage right after the barrier that frees it (S planes in flight ahead,
    // 8.34 ms per step against 8.58 for the other schedule); 16-bit storage
    // refills the stage of plane q - 1 before waiting for plane q (S - 1 planes
    // ahead; 9.80 against 10.24 ms for the rest-offset mode), with the halo
    // ring pulled by the last H threads so that warp 0, whose first thread
    // issues the copies, carries no second pull.
    constexpr bool kEarly = Codec<St>::kOffset;
    // Halo densities: where the CTA has twice as many threads as halo cells,
    // two threads share a cell, one species each (the same instructions on
    // another species' planes, no divergence), which halves the extra work the
    // halo threads bring to the per-plane barrier; otherwise one thread pulls
    // both species of a cell.
    constexpr bool kSplit = 2 * H <= TX * TY;
    constexpr int HT = kSplit ? 2 * H : H;  // halo threads
    const int hid = kEarly ? tid - (TX * TY - HT) : tid;  // halo thread index in [0, HT) for halo threads
    const bool halo = hid >= 0 && hid < HT;
    const int hs = kSplit ? (hid & 1) : 0;  // the species of a shared halo cell
    int hfx, hfy;
    halo_cell<TX, TY>(halo ? (kSplit ? hid >> 1 : hid) : 0, hfx, hfy);

    const bool down = alternate && tma_march_down(z0, a.zchunk);
    auto zof = [&](int q) { return tma_plane(z0, nplanes, nz, down, q); };
    // elected thread: the boxes of plane q into its stage.  (Spreading the 38
    // copy instructions over the lanes of a warp measured 1.8x slower.)
    auto issue = [&](int q) {
        fence_proxy_async_smem();  // earlier generic reads of the stage precede the async refill
        tma_issue_plane<TX, TY, S, St>(pmap, rmap, x0, y0, zof(q), a.gxo, a.gyo, nz, qbase + q, sm);
    };
    const bool issuer = tid == 0;
    auto try_plane = [&](int q) {
        const unsigned g = qbase + q;
        int n = 0;
        while (!mbar_try_wait(&bars[g % S], (g / S) & 1))
            if (++n >= kMbarSpinLimit) return false;
        return true;
    };

    // early schedule: planes 0 .. S-2 go out now and body(q) issues plane
    // q + S - 1 into the stage plane q - 1 used (read by every thread before
    // the barrier of body(q - 1)); late schedule: planes 0 .. S-1 now, and
    // body(q) refills plane q's stage with plane q + S after its barrier
    constexpr int kAhead = kEarly ? S - 1 : S;
    if (issuer && !preissued)
        for (int q = 0; q < kAhead && q < nplanes; ++q) issue(q);

    bool lost = false;
    // own pulls of plane q into X; own and halo densities into ring slot q % 4
    auto pull_frame = [&](const unsigned char* sb, int fx, int fy, C (&X)[2][Q]) {
        if constexpr (T::REST) {
#pragma unroll
            for (int i = 0; i < Q; ++i) tma_pulled_pair<TX, TY, S, St>(sb, i, fx, fy, X[0][i], X[1][i]);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int s = 0; s < 2; ++s)
                    X[s][i] = tma_pulled<TX, TY, S, St>(sb, s, i, fx, fy, s == 0 ? a.ref_A : a.ref_B);
        }
    };
    auto take_plane = [&](int q, C (&X)[2][Q]) {
        const unsigned char* sb = sm.stage + (size_t)((qbase + q) % S) * T::stage_bytes;
        pull_frame(sb, tx + 1, ty + 1, X);
        ring[q & 3][0][ty + 1][tx + 1] = node_density<L, C>(X[0]);
        ring[q & 3][1][ty + 1][tx + 1] = node_density<L, C>(X[1]);
        if (halo) {
            if constexpr (kSplit) {
                ring[q & 3][hs][hfy][hfx] = tma_density<TX, TY, S, St>(sb, hs, hfx, hfy, hs == 0 ? a.ref_A : a.ref_B);
            } else {
                C h[2][Q];
                pull_frame(sb, hfx, hfy, h);
                ring[q & 3][0][hfy][hfx] = node_density<L, C>(h[0]);
                ring[q & 3][1][hfy][hfx] = node_density<L, C>(h[1]);
            }
        }
    };
    auto collide = [&](int q, C (&X)[2][Q]) {
        // ring slots of the planes z - 1, z, z + 1 (steps q - 1 and q + 1 swap roles downwards)
        const int sc = q & 3, sm_ = (down ? q + 1 : q - 1) & 3, sp = (down ? q - 1 : q + 1) & 3;
        const C rA = ring[sc][0][ty + 1][tx + 1];
        const C rB = ring[sc][1][ty + 1][tx + 1];
        auto nbr = [&](int s, int i) -> C {
            const int sl = L::c(i, 2) == 0 ? sc : (L::c(i, 2) > 0 ? sp : sm_);
            return ring[sl][s][ty + 1 + L::c(i, 1)][tx + 1 + L::c(i, 0)];
        };
        if constexpr (FORCING == kSchemeFE) {
            C gp[3], lp;
            node_fe_derivs<L, C>(nbr, rB, gp, lp);
            node_collide_fe<L, C>(X, rA, rB, gp, lp, a.omega_A, a.omega_B, a.G, a.kappa, a.gamma);
        } else {
            C gA[3], gB[3];
            node_force<L, C>(nbr, a.G, gA, gB);
            node_add_body<C>(a.body_A, kolmo, gA, gB);
            if constexpr (FORCING == kForcingGuo)
                node_collide_guo<L, C>(X, rA, rB, gA, gB, a.omega_A, a.omega_B);
            else
                node_collide<L, C>(X, rA, rB, gA, gB, a.omega_A, a.omega_B, a.tau_A, a.tau_B);
        }
        if (owner) store_node<L, St>(a, gx, gy, zof(q), X, rA, rB);
    };
    // plane q arrives; plane q - 1 collides.  0: go on; 1: chunk done; -1: a wait was lost.
    auto body = [&](int q, C (&Xc)[2][Q], C (&Xp)[2][Q]) -> int {
        if (q >= nplanes) return 1;
        if (issuer) hook(q, nplanes);
        if (kEarly && issuer) {
            // before the wait: the issuing warp's copy instructions overlap the
            // other warps' halo pulls instead of delaying everyone's collision
            const int r = q + S - 1;
            if (r < nplanes) {
                issue(r);
            } else if (nxt && r - nplanes < nxt->nplanes) {
                fence_proxy_async_smem();
                tma_issue_plane<TX, TY, S, St>(nxt->map, nullptr, nxt->x0, nxt->y0,
                                               tma_plane(nxt->z0, nxt->nplanes, nxt->nz, nxt->down != 0, r - nplanes),
                                               nxt->gxo, nxt->gyo, nxt->nz, qbase + r, sm);
            }
        }
        if (q == 0 && a.wait_probe > 0 && issuer && x0 == 0 && y0 == 0 && z0 == 0) {
            // failure-detection test hook: the first CTA of the lattice waits,
            // a.wait_probe tries long, on the barrier nothing arrives on, so
            // that the bounded wait expires and the error path below runs
            int n = 0;
            while (!mbar_try_wait(&bars[S], 0u))
                if (++n >= a.wait_probe) {
                    lost = true;
                    break;
                }
        }
        if (!try_plane(q)) lost = true;
        take_plane(q, Xc);
        if (__syncthreads_or(lost)) {
            if (tid == 0) {
                // drain: wait (bounded) for the planes issued from q on (the
                // next item's first planes included).  Bit 0 of the error word:
                // a wait expired; bit 1: copies into this CTA's shared memory
                // were still outstanding after the drain's own bound, so the
                // device state is suspect.
                const int last = nxt && nxt->nplanes > 0 ? nplanes + min(kAhead, nxt->nplanes) : nplanes;
                bool drained = true;
                for (int r = q; r < last && r < q + S; ++r) drained = try_plane(r) && drained;
                atomicOr(err, drained ? 1 : 3);
            }
            return -1;
        }
        if (!kEarly && issuer) {
            const int r = q + S;  // into the stage plane q was read from, before the barrier above
            if (r < nplanes) {
                issue(r);
            } else if (nxt && r - nplanes < nxt->nplanes) {
                fence_proxy_async_smem();
                tma_issue_plane<TX, TY, S, St>(nxt->map, nullptr, nxt->x0, nxt->y0,
                                               tma_plane(nxt->z0, nxt->nplanes, nxt->nz, nxt->down != 0, r - nplanes),
                                               nxt->gxo, nxt->gyo, nxt->nz, qbase + r, sm);
            }
        }
        if (q >= 2) collide(q - 1, Xp);
        return 0;
    };

    C R0[2][Q], R1[2][Q];
    int r = 0;
#pragma unroll 1
    for (int q = 0;; q += 2) {
        if ((r = body(q, R0, R1)) != 0) break;
        if ((r = body(q + 1, R1, R0)) != 0) break;
    }
    return r < 0 ? -1 : nplanes;
}

// FORCING: the collision, fixed at compile time: kForcingShift, kForcingGuo or
// kSchemeFE (the FE model); the last two are instantiated for the 64x6 FP32
// tile only.
template <int TX, int TY, int S, class St = float, int FORCING = kForcingShift, int MINB = 1>
__global__ void __launch_bounds__(TX* TY, MINB)
    sc_step_tma_kernel(const __grid_constant__ TmaMaps maps, const LatticeArgs<St> a, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    TmaSmem<TX, TY, S, St> sm(smem_raw);
    sm.init_barriers();
    tma_item<TX, TY, S, St, TmaNoHook, FORCING>(&maps.pop, &maps.rho, a, blockIdx.x * TX, blockIdx.y * TY,
                                                blockIdx.z * a.zchunk, 0u, sm, err);
}

}  // namespace lbmsc

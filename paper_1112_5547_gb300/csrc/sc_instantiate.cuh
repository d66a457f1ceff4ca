// Typed launch helpers shared by the per-lattice translation units.
#pragma once

#include <cstring>

#include "sc_tma.cuh"
#include "sc_kernels.cuh"
#include "sc_regpipe.cuh"
#include "sc_launch.cuh"
#include "sc_args.cuh"

namespace lbmsc {

template <class L, class S, int TX, int TY>
cudaError_t step_tiled(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st) {
    using C = typename Codec<S>::C;
    FieldArgs<C> fo{};
    // register budget: 65536 / (threads * CTAs per SM)
    constexpr int kMin = sizeof(C) == 8 ? 1 : (TX * TY <= 128 ? 4 : (TX * TY <= 256 ? 2 : 1));
    sc_fused_kernel<L, S, TX, TY, kModeStep, kMin><<<step_grid(p), dim3(TX, TY), 0, st>>>(a, fo);
    return cudaGetLastError();
}

template <class L, class S, int TX, int TY, int MINB>
cudaError_t step_reload(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st) {
    using C = typename Codec<S>::C;
    constexpr int kMin = sizeof(C) == 8 ? (MINB > 2 ? MINB / 2 : 1) : MINB;
    sc_step_reload_kernel<L, S, TX, TY, kMin><<<step_grid(p), dim3(TX, TY), 0, st>>>(a);
    return cudaGetLastError();
}

template <class L, class S, int TX, int TY, int ST, int FORCING = kForcingShift, int MINB = 1> struct TmaLaunch {
    static cudaError_t run(const Plan&, const LatticeArgs<S>&, cudaStream_t) { return cudaErrorInvalidValue; }
};
template <class S, int TX, int TY, int ST, int FORCING, int MINB> struct TmaLaunch<D3Q19, S, TX, TY, ST, FORCING, MINB> {
    static cudaError_t run(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st) {
        if constexpr (sizeof(S) == 8) {
            return cudaErrorInvalidValue;
        } else {
            const TileShape& ts = kTiles[p.step_tile];
            using T = TmaTile<TX, TY, ST, S>;
            if (p.nx < TX || p.ny < TY) return cudaErrorInvalidValue;
            TmaMaps maps;
            memset(&maps, 0, sizeof(maps));
            cudaError_t e = encode_population_map(p, a.fin, T::BX, T::BY, &maps.pop, ts.promo, T::E, T::Q2);
            if constexpr (T::REST)
                if (e == cudaSuccess)
                    e = encode_rho_map(p, rest_rho<D3Q19>(a.fin, p.Np), T::RBX, T::RBY, &maps.rho, ts.promo);
            if (e != cudaSuccess) return e;
            auto kern = sc_step_tma_kernel<TX, TY, ST, S, FORCING, MINB>;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem_bytes);
            if (e != cudaSuccess) return e;
            if (ts.cx == 1 && ts.cy == 1) {
                kern<<<step_grid(p), dim3(TX, TY), T::smem_bytes, st>>>(maps, a, p.err);
                return cudaGetLastError();
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = step_grid(p);
            cfg.blockDim = dim3(TX, TY);
            cfg.dynamicSmemBytes = T::smem_bytes;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = ts.cx;
            attr[0].val.clusterDim.y = ts.cy;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, kern, maps, a, p.err);
        }
    }
};

template <class L, class S, int TX, int TY, int MINB> struct RegPipeLaunch {
    static cudaError_t run(const Plan&, const LatticeArgs<S>&, cudaStream_t) { return cudaErrorInvalidValue; }
};
template <class S, int TX, int TY, int MINB> struct RegPipeLaunch<D3Q19, S, TX, TY, MINB> {
    static cudaError_t run(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st) {
        if constexpr (sizeof(S) == 8) {
            return cudaErrorInvalidValue;  // three planes of doubles do not fit in registers
        } else {
            sc_step_regpipe_kernel<S, TX, TY, MINB><<<step_grid(p), dim3(TX, TY), 0, st>>>(a);
            return cudaGetLastError();
        }
    }
};

template <class L, class S> cudaError_t step_typed_other(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st);

template <class L, class S> cudaError_t step_typed(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    if (!tile_supported(p.step_tile, p.lattice, p.precision, p.forcing, p.model)) return cudaErrorInvalidValue;
    LatticeArgs<S> a = make_args<S>(p, fin, fout);
    a.zchunk = p.step_zchunk;
    static_assert(kTiles[0].tx == 32 && kTiles[0].ty == 8 && kTiles[1].ty == 16 && kTiles[2].tx == 64 &&
                      kTiles[3].ty == 4 && kTiles[4].tx == 64 && kTiles[5].kind == kRetired &&
                      kTiles[10].kind == kRetired && kTiles[11].stages == 6 && kTiles[12].ty == 8 && kTiles[13].tx == 64 && kTiles[14].stages == 4 &&
                      kTiles[15].kind == 4 && kTiles[16].ty == 8 && kTiles[17].tx == 16 && kTiles[18].kind == 5 &&
                      kTiles[19].tx == 64 && kTiles[20].stages == 4 && kTiles[21].stages == 2 && kTiles[22].cy == 2 &&
                      kTiles[23].cy == 4 && kTiles[24].cx == 2 && kTiles[25].tx == 32 && kTiles[26].kind == kRetired &&
                      kTiles[29].kind == kRetired && kTiles[30].kind == 6 &&
                      kTiles[31].stages == 4 && kTiles[32].tx == 32 && kTiles[33].ty == 6 && kTiles[34].stages == 2 &&
                      kTiles[35].kind == 6 && kTiles[36].ty == 12 && kTiles[37].cy == 1 && kTiles[38].kind == 6 &&
                      kTiles[39].ty == 8 && kTiles[40].tx == 48 && kTiles[41].cy == 1 && kTiles[42].minb == 2 &&
                      kTiles[43].tx == 32 && kTiles[44].cy == 1 && kNumTiles == 45,
                  "tile table and dispatch disagree");
    if constexpr (Codec<S>::kRest) {
        // rest-offset storage: the kernels that pull through pull_node
        switch (p.step_tile) {
            case 0: return step_tiled<L, S, 32, 8>(p, a, st);
            case 1: return step_tiled<L, S, 32, 16>(p, a, st);
            case 2: return step_tiled<L, S, 64, 8>(p, a, st);
            case 3: return step_tiled<L, S, 32, 4>(p, a, st);
            case 4: return step_tiled<L, S, 64, 4>(p, a, st);
            case 11: return step_reload<L, S, 32, 4, 6>(p, a, st);
            case 12: return step_reload<L, S, 32, 8, 3>(p, a, st);
            case 13: return step_reload<L, S, 64, 4, 3>(p, a, st);
            case 14: return step_reload<L, S, 32, 4, 4>(p, a, st);
            case 30: return TmaLaunch<L, S, 64, 4, 3>::run(p, a, st);
            case 31: return TmaLaunch<L, S, 64, 4, 4>::run(p, a, st);
            case 32: return TmaLaunch<L, S, 32, 8, 3>::run(p, a, st);
            case 35: return TmaLaunch<L, S, 64, 6, 3>::run(p, a, st);
            case 38: return TmaLaunch<L, S, 32, 12, 3>::run(p, a, st);
            case 39: return TmaLaunch<L, S, 64, 8, 2>::run(p, a, st);
            case 42:
            case 44: return TmaLaunch<L, S, 64, 4, 2, kForcingShift, 2>::run(p, a, st);
            case 43: return TmaLaunch<L, S, 32, 8, 2, kForcingShift, 2>::run(p, a, st);
        }
        return cudaErrorInvalidValue;
    } else {
        return step_typed_other<L, S>(p, a, st);
    }
}

template <class L, class S> cudaError_t step_typed_other(const Plan& p, const LatticeArgs<S>& a, cudaStream_t st) {
    switch (p.step_tile) {
        case 0: return step_tiled<L, S, 32, 8>(p, a, st);
        case 1: return step_tiled<L, S, 32, 16>(p, a, st);
        case 2: return step_tiled<L, S, 64, 8>(p, a, st);
        case 3: return step_tiled<L, S, 32, 4>(p, a, st);
        case 4: return step_tiled<L, S, 64, 4>(p, a, st);
        case 11: return step_reload<L, S, 32, 4, 6>(p, a, st);
        case 12: return step_reload<L, S, 32, 8, 3>(p, a, st);
        case 13: return step_reload<L, S, 64, 4, 3>(p, a, st);
        case 14: return step_reload<L, S, 32, 4, 4>(p, a, st);
        case 15: return RegPipeLaunch<L, S, 32, 4, 3>::run(p, a, st);
        case 16: return RegPipeLaunch<L, S, 32, 8, 1>::run(p, a, st);
        case 17: return RegPipeLaunch<L, S, 16, 8, 3>::run(p, a, st);
    }
    if constexpr (std::is_same<S, float>::value) {
        switch (p.step_tile) {
            case 18: return TmaLaunch<L, S, 32, 8, 3>::run(p, a, st);
            case 19: return TmaLaunch<L, S, 64, 4, 3>::run(p, a, st);
            case 20: return TmaLaunch<L, S, 32, 4, 4>::run(p, a, st);
            case 21: return TmaLaunch<L, S, 32, 4, 2>::run(p, a, st);
            case 22:
            case 23:
            case 24: return TmaLaunch<L, S, 64, 4, 3>::run(p, a, st);
            case 25: return TmaLaunch<L, S, 32, 8, 3>::run(p, a, st);
            case 33: return TmaLaunch<L, S, 64, 6, 2>::run(p, a, st);
            case 34:
                if (p.model == kModelFE) return TmaLaunch<L, S, 64, 6, 2, kSchemeFE>::run(p, a, st);
                return p.forcing == kForcingGuo ? TmaLaunch<L, S, 64, 6, 2, kForcingGuo>::run(p, a, st)
                                                : TmaLaunch<L, S, 64, 6, 2>::run(p, a, st);
            case 36:
            case 37: return TmaLaunch<L, S, 32, 12, 2>::run(p, a, st);
            case 40:
            case 41: return TmaLaunch<L, S, 48, 8, 2>::run(p, a, st);
        }
    }
    if constexpr (sizeof(S) == 2) {
        switch (p.step_tile) {
            case 30: return TmaLaunch<L, S, 64, 4, 3>::run(p, a, st);
            case 31: return TmaLaunch<L, S, 64, 4, 4>::run(p, a, st);
            case 32: return TmaLaunch<L, S, 32, 8, 3>::run(p, a, st);
            case 35: return TmaLaunch<L, S, 64, 6, 3>::run(p, a, st);
            case 38: return TmaLaunch<L, S, 32, 12, 3>::run(p, a, st);
            case 39: return TmaLaunch<L, S, 64, 8, 2>::run(p, a, st);
            case 42:
            case 44: return TmaLaunch<L, S, 64, 4, 2, kForcingShift, 2>::run(p, a, st);
            case 43: return TmaLaunch<L, S, 32, 8, 2, kForcingShift, 2>::run(p, a, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <class L, class S>
cudaError_t init_typed(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st,
                       int zlo, int zhi) {
    using C = typename Codec<S>::C;
    const LatticeArgs<S> a = make_args<S>(p, nullptr, fout);
    if (zhi <= 0 || zhi > p.nz) zhi = p.nz;
    if (zlo < 0 || zlo >= zhi) return zlo == zhi ? cudaSuccess : cudaErrorInvalidValue;
    long long blocks = ((long long)p.nx * p.ny * (zhi - zlo) + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    sc_init_kernel<L, S><<<(unsigned)blocks, 256, 0, st>>>(a, static_cast<const C*>(rA), static_cast<const C*>(rB),
                                                          static_cast<const C*>(u), zlo, zhi);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t moments_typed(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    using C = typename Codec<S>::C;
    LatticeArgs<S> a = make_args<S>(p, fin, nullptr);
    FieldArgs<C> fo;
    fo.rhoA = static_cast<C*>(o.rhoA);
    fo.rhoB = static_cast<C*>(o.rhoB);
    fo.u = static_cast<C*>(o.u);
    fo.p = static_cast<C*>(o.p);
    fo.partials = o.partials;
    fo.win_c[0] = o.win[0];
    fo.win_c[1] = o.win[1];
    fo.win_c[2] = o.win[2];
    fo.r_in2 = o.win[3] < 0 ? -1.0 : o.win[3] * o.win[3];
    fo.r_out2 = o.win[4] * o.win[4];
    dim3 grid = fused_grid(p);
    if (o.zhi > 0) {
        // planes [zlo, zhi) only (whole chunks of p.zchunk from zlo; fields only, no partials)
        if (o.partials || o.zlo < 0 || o.zlo >= o.zhi || o.zhi > p.nz) return cudaErrorInvalidValue;
        a.zbase = o.zlo;
        a.zend = o.zhi;
        grid.z = (unsigned)((o.zhi - o.zlo + p.zchunk - 1) / p.zchunk);
    }
    sc_fused_kernel<L, S, kTX, kTY, kModeMoments, 1><<<grid, dim3(kTX, kTY), 0, st>>>(a, fo);
    return cudaGetLastError();
}

template <class L> cudaError_t step_any(const Plan& p, const void* fin, void* fout, cudaStream_t st) {
    switch (p.precision) {
        case 0: return step_typed<L, double>(p, fin, fout, st);
        case 1: return step_typed<L, float>(p, fin, fout, st);
        case 2: return step_typed<L, __nv_bfloat16>(p, fin, fout, st);
        case 3: return step_typed<L, __half>(p, fin, fout, st);
        case 4: return step_typed<L, bf16_rest>(p, fin, fout, st);
        case 5: return step_typed<L, f16_rest>(p, fin, fout, st);
    }
    return cudaErrorInvalidValue;
}

template <class L>
cudaError_t init_any(const Plan& p, const void* rA, const void* rB, const void* u, void* fout, cudaStream_t st,
                     int zlo, int zhi) {
    switch (p.precision) {
        case 0: return init_typed<L, double>(p, rA, rB, u, fout, st, zlo, zhi);
        case 1: return init_typed<L, float>(p, rA, rB, u, fout, st, zlo, zhi);
        case 2: return init_typed<L, __nv_bfloat16>(p, rA, rB, u, fout, st, zlo, zhi);
        case 3: return init_typed<L, __half>(p, rA, rB, u, fout, st, zlo, zhi);
        case 4: return init_typed<L, bf16_rest>(p, rA, rB, u, fout, st, zlo, zhi);
        case 5: return init_typed<L, f16_rest>(p, rA, rB, u, fout, st, zlo, zhi);
    }
    return cudaErrorInvalidValue;
}

template <class L> cudaError_t moments_any(const Plan& p, const void* fin, const MomentsOut& o, cudaStream_t st) {
    switch (p.precision) {
        case 0: return moments_typed<L, double>(p, fin, o, st);
        case 1: return moments_typed<L, float>(p, fin, o, st);
        case 2: return moments_typed<L, __nv_bfloat16>(p, fin, o, st);
        case 3: return moments_typed<L, __half>(p, fin, o, st);
        case 4: return moments_typed<L, bf16_rest>(p, fin, o, st);
        case 5: return moments_typed<L, f16_rest>(p, fin, o, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbmsc

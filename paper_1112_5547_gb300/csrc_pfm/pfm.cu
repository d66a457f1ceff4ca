// Pseudo-spectral phase-field model of Sec. 3 on one GPU (C ABI in pfm.h).
//
// One time step (Sec. 3.1, Eqs. eq10-eq13), all fields periodic:
//   1. prep (spectral, one thread per complex coefficient): phi^, i k phi^ (D
//      components), -|k|^2 phi^ and u^ (D components), scaled by 1/N, into the
//      inverse-transform batch;
//   2. one batched complex-to-real cuFFT call (2 + 2D transforms);
//   3. phys (one thread per node): u.grad phi, the explicit Cahn-Hilliard
//      bracket ln((rho+phi)/(rho-phi))/g_tau - 3 phi, the capillary force
//      mu grad phi / rho and the products u_a u_b, into the forward batch;
//   4. one batched real-to-complex cuFFT call (2 + D + D(D+1)/2 transforms);
//   5. update (spectral): S^ and the projected momentum right-hand side N^,
//      then phi^ and u^ by AB2 (explicit) / Crank-Nicolson (implicit).
// The spectral state (phi^, u^ and the previous explicit terms) stays in the
// caller's workspace between steps; the real fields exist only inside a step.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/pfm.h"

namespace {

constexpr double kCs2 = 1.0 / 3.0;

template <class T> struct Cx;
template <> struct Cx<float> {
    using type = cufftComplex;
};
template <> struct Cx<double> {
    using type = cufftDoubleComplex;
};

struct Geometry {
    int dim, nx, ny, nz, nxh;  // nxh = nx/2 + 1 (the half axis of the real transforms)
    long long nreal, ncplx;
};

// Wavenumbers of complex coefficient c (x the half axis, fastest): the full
// ones (Laplacian) and the first-derivative ones (Nyquist of an even axis
// zeroed), in the solver's precision T (FP32 arithmetic for the FP32 solver:
// FP64 throughput is a small fraction of FP32 on this GPU).
template <class T> struct Wave {
    T k[3], kd[3], k2;
};

template <class T> __device__ __forceinline__ Wave<T> wave_of(const Geometry& g, long long c) {
    Wave<T> w;
    const int ix = (int)(c % g.nxh);
    const int iy = (int)((c / g.nxh) % g.ny);
    const int iz = (int)(c / ((long long)g.nxh * g.ny));
    const int idx[3] = {ix, iy, iz};
    const int n[3] = {g.nx, g.ny, g.nz};
    w.k2 = (T)0;
    for (int a = 0; a < 3; ++a) {
        if (a >= g.dim) {
            w.k[a] = w.kd[a] = (T)0;
            continue;
        }
        const int m = idx[a] <= n[a] / 2 ? idx[a] : idx[a] - n[a];  // signed frequency (x: 0..nx/2)
        // an even axis' Nyquist index is the frequency -n/2 (as numpy's fftfreq)
        const int f = (n[a] % 2 == 0 && idx[a] == n[a] / 2) ? -n[a] / 2 : m;
        w.k[a] = (T)6.283185307179586 * (T)f / (T)n[a];
        w.kd[a] = (n[a] % 2 == 0 && idx[a] == n[a] / 2) ? (T)0 : w.k[a];
        w.k2 += w.k[a] * w.k[a];
    }
    return w;
}

struct Coeffs {
    double rho, g, g_tau, Dc, xi2, nu, dt, inv_n;
    double body_half_n;  // A N / 2: the Fourier coefficient (times -+i) of A sin(2 pi y/ny) at ky = +-1
};

template <class C, class T> __device__ __forceinline__ C cmul_i(C a, T k) {  // (i k) a
    C r;
    r.x = -k * a.y;
    r.y = k * a.x;
    return r;
}
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) {
    C r;
    r.x = s * a.x;
    r.y = s * a.y;
    return r;
}

// 1. the inverse-transform inputs: phi^, i kd_a phi^, -k^2 phi^, u^_a (each / N)
template <class T>
__global__ void pfm_prep_kernel(Geometry g, Coeffs c, const typename Cx<T>::type* __restrict__ phi_h,
                                const typename Cx<T>::type* __restrict__ u_h, typename Cx<T>::type* __restrict__ cin) {
    using C = typename Cx<T>::type;
    const int D = g.dim;
    const T inv_n = (T)c.inv_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.ncplx;
         i += (long long)gridDim.x * blockDim.x) {
        const Wave<T> w = wave_of<T>(g, i);
        const C p = phi_h[i];
        cin[i] = cscale(p, inv_n);
        for (int a = 0; a < D; ++a) cin[(1 + a) * g.ncplx + i] = cscale(cmul_i(p, w.kd[a]), inv_n);
        cin[(1 + D) * g.ncplx + i] = cscale(p, -w.k2 * inv_n);
        for (int a = 0; a < D; ++a) cin[(2 + D + a) * g.ncplx + i] = cscale(u_h[a * g.ncplx + i], inv_n);
    }
}

// 3. nonlinear terms in physical space.  rin: phi, d_a phi (D), lap phi, u_a (D);
// rout: u.grad phi, bracket, F_a = mu d_a phi / rho (D), u_a u_b (a <= b).
template <class T>
__global__ void pfm_phys_kernel(Geometry g, Coeffs c, const T* __restrict__ rin, T* __restrict__ rout) {
    const int D = g.dim;
    const long long N = g.nreal;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const T phi = rin[n];
        T gp[3] = {0, 0, 0}, u[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            gp[a] = rin[(1 + a) * N + n];
            u[a] = rin[(2 + D + a) * N + n];
        }
        const T lap = rin[(1 + D) * N + n];
        const T rho = (T)c.rho;
        const T lnr = log((rho + phi) / (rho - phi));
        T adv = 0;
        for (int a = 0; a < D; ++a) adv += u[a] * gp[a];
        rout[n] = adv;
        rout[N + n] = lnr / (T)c.g_tau - (T)3 * phi;
        const T mu = (T)(0.5 * kCs2) * lnr - (T)(0.5 * c.g * kCs2) * phi - (T)(0.25 * c.g * kCs2 * kCs2) * lap;
        for (int a = 0; a < D; ++a) rout[(2 + a) * N + n] = mu * gp[a] / rho;
        int q = 2 + D;
        for (int a = 0; a < D; ++a)
            for (int b = a; b < D; ++b) rout[(q++) * N + n] = u[a] * u[b];
    }
}

// index of the product u_a u_b (a, b in any order) in the forward batch
__device__ __forceinline__ int uu_slot(int D, int a, int b) {
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    int q = 2 + D;
    for (int i = 0; i < a; ++i) q += D - i;
    return q + (b - a);
}

// 5. S^, N^ (projected; zero mean) and the AB2 / CN update of phi^ and u^.
template <class T>
__global__ void pfm_update_kernel(Geometry g, Coeffs c, int first, const typename Cx<T>::type* __restrict__ cout,
                                  typename Cx<T>::type* __restrict__ phi_h, typename Cx<T>::type* __restrict__ u_h,
                                  typename Cx<T>::type* __restrict__ s_prev, typename Cx<T>::type* __restrict__ n_prev) {
    using C = typename Cx<T>::type;
    const int D = g.dim;
    const long long M = g.ncplx;
    const T Dc = (T)c.Dc, dt = (T)c.dt, nu = (T)c.nu;
    const T bi = (T)(c.Dc * (c.xi2 - c.dt * c.Dc / 2.0));
    const T half = (T)0.5, three = (T)3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const Wave<T> w = wave_of<T>(g, i);
        const T k2 = w.k2, k4 = k2 * k2;
        const C p = phi_h[i];
        const C adv = cout[i], br = cout[M + i];
        const T sx = -adv.x - Dc * k2 * br.x - bi * k4 * p.x;
        const T sy = -adv.y - Dc * k2 * br.y - bi * k4 * p.y;
        const C sp = first ? C{sx, sy} : s_prev[i];
        const T lam = Dc * ((T)2 * k2 + dt * Dc * half * k4);
        const T am = (T)1 - dt * lam * half, inv_ap = (T)1 / ((T)1 + dt * lam * half);
        phi_h[i] = C{(am * p.x + dt * (three * sx - sp.x) * half) * inv_ap,
                     (am * p.y + dt * (three * sy - sp.y) * half) * inv_ap};
        s_prev[i] = C{sx, sy};
        // momentum right-hand side: -i sum_b kd_b (u_a u_b)^ + F_a^
        T nx_[3] = {0, 0, 0}, ny_[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            T re = cout[(2 + a) * M + i].x, im = cout[(2 + a) * M + i].y;
            for (int b = 0; b < D; ++b) {
                const C q = cout[uu_slot(D, a, b) * M + i];
                // -(i kd_b) q = kd_b (q.y - i q.x)
                re += w.kd[b] * q.y;
                im -= w.kd[b] * q.x;
            }
            nx_[a] = re;
            ny_[a] = im;
        }
        // Kolmogorov forcing A sin(2 pi y/ny) e_x: -i A N/2 at ky = +1, +i A N/2 at ky = -1 (kx = kz = 0)
        if (c.body_half_n != 0.0 && g.ny > 2) {
            const int ix = (int)(i % g.nxh), iy = (int)((i / g.nxh) % g.ny), iz = (int)(i / ((long long)g.nxh * g.ny));
            if (ix == 0 && iz == 0 && iy == 1) ny_[0] -= (T)c.body_half_n;
            if (ix == 0 && iz == 0 && iy == g.ny - 1) ny_[0] += (T)c.body_half_n;
        }
        const T kd2 = w.kd[0] * w.kd[0] + w.kd[1] * w.kd[1] + w.kd[2] * w.kd[2];
        T kre = 0, kim = 0;
        for (int a = 0; a < D; ++a) {
            kre += w.kd[a] * nx_[a];
            kim += w.kd[a] * ny_[a];
        }
        const T inv = kd2 > (T)0 ? (T)1 / kd2 : (T)0;
        const bool mean = k2 == (T)0;
        const T vis = nu * k2;
        const T bm = (T)1 - dt * vis * half, inv_bp = (T)1 / ((T)1 + dt * vis * half);
        for (int a = 0; a < D; ++a) {
            const T re = mean ? (T)0 : nx_[a] - w.kd[a] * kre * inv;
            const T im = mean ? (T)0 : ny_[a] - w.kd[a] * kim * inv;
            const C prev = first ? C{re, im} : n_prev[a * M + i];
            const C u = u_h[a * M + i];
            u_h[a * M + i] = C{(bm * u.x + dt * (three * re - prev.x) * half) * inv_bp,
                               (bm * u.y + dt * (three * im - prev.y) * half) * inv_bp};
            n_prev[a * M + i] = C{re, im};
        }
    }
}

constexpr size_t kAlign = 256;
size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

bool valid(const pfm_params* p) {
    if (!p) return false;
    if (p->dim != 2 && p->dim != 3) return false;
    if (p->precision != PFM_F64 && p->precision != PFM_F32) return false;
    if (p->nx < 2 || p->ny < 2 || p->nz < 1) return false;
    if (p->dim == 2 && p->nz != 1) return false;
    if (p->dim == 3 && p->nz < 2) return false;
    if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return false;
    // g > 0: the explicit bracket carries 1/g_tau and the mobility D = M g_tau cs2/2
    if (!(p->rho > 0) || !(p->tau > 0.5) || !(p->dt > 0) || !(p->g > 0) || !(p->g - p->g == 0.0)) return false;
    if (!(p->body_A - p->body_A == 0.0)) return false;
    return true;
}

Geometry geometry(const pfm_params* p) {
    Geometry g;
    g.dim = p->dim;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->dim == 3 ? p->nz : 1;
    g.nxh = p->nx / 2 + 1;
    g.nreal = (long long)g.nx * g.ny * g.nz;
    g.ncplx = (long long)g.nxh * g.ny * g.nz;
    return g;
}

int n_inverse(int D) { return 2 + 2 * D; }
int n_forward(int D) { return 2 + D + D * (D + 1) / 2; }

struct Layout {
    size_t phi_h, u_h, s_prev, n_prev, cin, rin, rphys, cout, total;
};

Layout layout(const Geometry& g, size_t real_bytes) {
    const size_t cb = 2 * real_bytes;
    const int D = g.dim;
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes);
        return at;
    };
    L.phi_h = take(g.ncplx * cb);
    L.u_h = take(D * g.ncplx * cb);
    L.s_prev = take(g.ncplx * cb);
    L.n_prev = take(D * g.ncplx * cb);
    L.cin = take(n_inverse(D) * g.ncplx * cb);
    L.rin = take(n_inverse(D) * g.nreal * real_bytes);
    L.rphys = take(n_forward(D) * g.nreal * real_bytes);
    L.cout = take(n_forward(D) * g.ncplx * cb);
    L.total = o;
    return L;
}

}  // namespace

struct pfm_handle {
    pfm_params params;
    Geometry g;
    Coeffs c;
    Layout L;
    unsigned char* ws;
    cudaStream_t stream;
    cufftHandle inv, fwd;
    int started;  // an explicit term of the previous step exists
};

namespace {

Coeffs coeffs(const pfm_params* p, const Geometry& g) {
    Coeffs c;
    c.rho = p->rho;
    c.g = p->g;
    c.g_tau = p->tau * p->g / (p->tau - 0.5);
    const double M = p->rho * (p->tau - 0.5);
    c.Dc = M * c.g_tau * kCs2 / 2.0;
    c.xi2 = kCs2 / 2.0;
    c.nu = kCs2 * (p->tau - 0.5);
    c.dt = p->dt;
    c.inv_n = 1.0 / (double)g.nreal;
    c.body_half_n = p->body_A * (double)g.nreal / 2.0;
    return c;
}

lbm_status make_plan(const Geometry& g, bool inverse, bool dbl, int batch, cufftHandle* out) {
    int n[3];
    int rank = g.dim;
    if (g.dim == 3) {
        n[0] = g.nz;
        n[1] = g.ny;
        n[2] = g.nx;
    } else {
        n[0] = g.ny;
        n[1] = g.nx;
    }
    const cufftType t = inverse ? (dbl ? CUFFT_Z2D : CUFFT_C2R) : (dbl ? CUFFT_D2Z : CUFFT_R2C);
    if (cufftPlanMany(out, rank, n, nullptr, 1, 0, nullptr, 1, 0, t, batch) != CUFFT_SUCCESS) return LBM_ERR_CUDA;
    return LBM_OK;
}

unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <class T> lbm_status exec(cufftHandle plan, bool inverse, void* in, void* out) {
    cufftResult r;
    if constexpr (sizeof(T) == 8) {
        r = inverse ? cufftExecZ2D(plan, (cufftDoubleComplex*)in, (cufftDoubleReal*)out)
                    : cufftExecD2Z(plan, (cufftDoubleReal*)in, (cufftDoubleComplex*)out);
    } else {
        r = inverse ? cufftExecC2R(plan, (cufftComplex*)in, (cufftReal*)out)
                    : cufftExecR2C(plan, (cufftReal*)in, (cufftComplex*)out);
    }
    return r == CUFFT_SUCCESS ? LBM_OK : LBM_ERR_CUDA;
}

template <class T> lbm_status step_typed(pfm_handle* h) {
    using C = typename Cx<T>::type;
    unsigned char* w = h->ws;
    const Geometry& g = h->g;
    auto P = [&](size_t off) { return (void*)(w + off); };
    pfm_prep_kernel<T><<<grid_for(g.ncplx), 256, 0, h->stream>>>(g, h->c, (const C*)P(h->L.phi_h),
                                                                 (const C*)P(h->L.u_h), (C*)P(h->L.cin));
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    lbm_status s = exec<T>(h->inv, true, P(h->L.cin), P(h->L.rin));
    if (s != LBM_OK) return s;
    pfm_phys_kernel<T><<<grid_for(g.nreal), 256, 0, h->stream>>>(g, h->c, (const T*)P(h->L.rin), (T*)P(h->L.rphys));
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    s = exec<T>(h->fwd, false, P(h->L.rphys), P(h->L.cout));
    if (s != LBM_OK) return s;
    pfm_update_kernel<T><<<grid_for(g.ncplx), 256, 0, h->stream>>>(
        g, h->c, h->started ? 0 : 1, (const C*)P(h->L.cout), (C*)P(h->L.phi_h), (C*)P(h->L.u_h),
        (C*)P(h->L.s_prev), (C*)P(h->L.n_prev));
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    h->started = 1;
    return LBM_OK;
}

size_t real_bytes(const pfm_params* p) { return p->precision == PFM_F64 ? 8 : 4; }

}  // namespace

extern "C" {

LBM_SC_API size_t pfm_workspace_bytes(const pfm_params* p) {
    if (!valid(p)) return 0;
    return layout(geometry(p), real_bytes(p)).total;
}

LBM_SC_API lbm_status pfm_create(const pfm_params* p, void* d_ws, size_t bytes, void* stream, pfm_handle** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid(p) || !d_ws || ((uintptr_t)d_ws % kAlign) != 0) return LBM_ERR_INVALID_ARG;
    const Geometry g = geometry(p);
    const Layout L = layout(g, real_bytes(p));
    if (bytes < L.total) return LBM_ERR_OUT_OF_MEMORY;
    pfm_handle* h = new (std::nothrow) pfm_handle;
    if (!h) return LBM_ERR_OUT_OF_MEMORY;
    h->params = *p;
    h->g = g;
    h->c = coeffs(p, g);
    h->L = L;
    h->ws = static_cast<unsigned char*>(d_ws);
    h->stream = static_cast<cudaStream_t>(stream);
    h->started = 0;
    const bool dbl = p->precision == PFM_F64;
    if (make_plan(g, true, dbl, n_inverse(g.dim), &h->inv) != LBM_OK) {
        delete h;
        return LBM_ERR_CUDA;
    }
    if (make_plan(g, false, dbl, n_forward(g.dim), &h->fwd) != LBM_OK) {
        cufftDestroy(h->inv);
        delete h;
        return LBM_ERR_CUDA;
    }
    if (cufftSetStream(h->inv, h->stream) != CUFFT_SUCCESS || cufftSetStream(h->fwd, h->stream) != CUFFT_SUCCESS) {
        cufftDestroy(h->inv);
        cufftDestroy(h->fwd);
        delete h;
        return LBM_ERR_CUDA;
    }
    *out = h;
    return LBM_OK;
}

LBM_SC_API lbm_status pfm_init(pfm_handle* h, const void* d_phi, const void* d_u) {
    if (!h || !d_phi) return LBM_ERR_INVALID_ARG;
    const Geometry& g = h->g;
    const int D = g.dim;
    const size_t rb = real_bytes(&h->params), cb = 2 * rb;
    unsigned char* w = h->ws;
    // the forward batch's inputs: phi, u_a, the rest zero; transformed together
    if (cudaMemsetAsync(w + h->L.rphys, 0, n_forward(D) * g.nreal * rb, h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(w + h->L.rphys, d_phi, g.nreal * rb, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (d_u && cudaMemcpyAsync(w + h->L.rphys + g.nreal * rb, d_u, D * g.nreal * rb, cudaMemcpyDeviceToDevice,
                               h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    const lbm_status s = h->params.precision == PFM_F64 ? exec<double>(h->fwd, false, w + h->L.rphys, w + h->L.cout)
                                                        : exec<float>(h->fwd, false, w + h->L.rphys, w + h->L.cout);
    if (s != LBM_OK) return s;
    if (cudaMemcpyAsync(w + h->L.phi_h, w + h->L.cout, g.ncplx * cb, cudaMemcpyDeviceToDevice, h->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(w + h->L.u_h, w + h->L.cout + g.ncplx * cb, D * g.ncplx * cb, cudaMemcpyDeviceToDevice,
                        h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    h->started = 0;
    return LBM_OK;
}

LBM_SC_API lbm_status pfm_step(pfm_handle* h, int nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < nsteps; ++i) {
        const lbm_status s = h->params.precision == PFM_F64 ? step_typed<double>(h) : step_typed<float>(h);
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

LBM_SC_API lbm_status pfm_fields(pfm_handle* h, void* d_phi, void* d_u) {
    if (!h) return LBM_ERR_INVALID_ARG;
    const Geometry& g = h->g;
    const int D = g.dim;
    const size_t rb = real_bytes(&h->params);
    unsigned char* w = h->ws;
    lbm_status s;
    if (h->params.precision == PFM_F64) {
        pfm_prep_kernel<double><<<grid_for(g.ncplx), 256, 0, h->stream>>>(
            g, h->c, (const cufftDoubleComplex*)(w + h->L.phi_h), (const cufftDoubleComplex*)(w + h->L.u_h),
            (cufftDoubleComplex*)(w + h->L.cin));
        if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
        s = exec<double>(h->inv, true, w + h->L.cin, w + h->L.rin);
    } else {
        pfm_prep_kernel<float><<<grid_for(g.ncplx), 256, 0, h->stream>>>(
            g, h->c, (const cufftComplex*)(w + h->L.phi_h), (const cufftComplex*)(w + h->L.u_h),
            (cufftComplex*)(w + h->L.cin));
        if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
        s = exec<float>(h->inv, true, w + h->L.cin, w + h->L.rin);
    }
    if (s != LBM_OK) return s;
    if (d_phi && cudaMemcpyAsync(d_phi, w + h->L.rin, g.nreal * rb, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (d_u && cudaMemcpyAsync(d_u, w + h->L.rin + (size_t)(2 + D) * g.nreal * rb, D * g.nreal * rb,
                               cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}

LBM_SC_API void pfm_destroy(pfm_handle* h) {
    if (!h) return;
    cufftDestroy(h->inv);
    cufftDestroy(h->fwd);
    delete h;
}

}  // extern "C"

// Per-node arithmetic of the two-component Shan-Chen step (paper Sec. 2.1),
// shared by every kernel so that all launch shapes give bit-identical results.
//
// For one node with pulled populations f_is (post-streaming, pre-collision):
//   rho_s = sum_i f_is,  j_s = sum_i f_is c_i                      (Sec. 2.1 moments)
//   g_s = F_s / rho_s = -G sum_i w_i rho_s'(x + c_i) c_i           (Eq. FORCE)
//         [+ A sin(2 pi y / ny) e_x: Kolmogorov forcing, Eq. kolmo]
//   u' = (j_A / tau_A + j_B / tau_B) / (rho_A / tau_A + rho_B / tau_B)
//   f_is += (1 / tau_s) (f^eq_i(rho_s, u' + tau_s g_s) - f_is)      (Eq. eq:be)
// with f^eq_i(rho, u) = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u].
//
// All operations go through Ar<C> (explicitly rounded intrinsics) in a fixed
// order.  The force is taken per unit density, so a vanishing rho_s is never
// divided by.  Momentum and force are summed over opposite-direction pairs
// (the GPU velocity order keeps c_{i+1} = -c_i for odd i): the pair difference
// f_i - f_{i+1}, resp. rho(x + c_i) - rho(x - c_i), is formed first, so both
// vanish exactly in a uniform region and their rounding is antisymmetric.
// Accumulating single terms instead (rho(x + c_i) with an FMA, then
// rho(x - c_i)) leaves a force of about one ulp in uniform regions; in FP32
// that random-walks the total momentum and lets a drop drift by about 1e-5
// lattice units per 1000 steps.  The rest population of the equilibrium is closed as
// f^eq_0 = rho - sum_{i>0} f^eq_i (equal to w_0 rho (...) in exact arithmetic;
// the rounded weights float(1/9), float(4/9), float(1/36) all err upwards and
// would otherwise create about 7e-9 of mass per step at tau = 1), and that
// closure is evaluated as f^eq_0 - f_0 = -sum_{i>0} (f^eq_i - f_i), with
// rho = sum_i f_i: the rest population relaxes by minus the sum of the very
// increments the moving ones receive, so the collision conserves mass up to
// the roundings of that short sum of non-equilibrium parts (a few ulp of
// |f^eq - f|, not of rho) and of the final updates.  Summing rho and
// sum_{i>0} f^eq_i separately instead rounds both at the scale of rho; at
// nodes that repeat the same values those roundings do not average out, and a
// 20000-step FP32 drop drifts in mass by several 1e-6.
#pragma once

#include "sc_common.cuh"

namespace lbmsc {

// rho = (f_1 + f_2 + ... + f_{Q-1}) + f_0, the moving populations first and
// the rest population last, in one fixed order.  rho enters the equilibria
// and the velocity; the closure of f^eq_0 below does not round through it.
template <class L, class C> __device__ __forceinline__ C node_density(const C (&f)[L::Q]) {
    C r = f[1];
#pragma unroll
    for (int i = 2; i < L::Q; ++i) r = Ar<C>::add(r, f[i]);
    return Ar<C>::add(r, f[0]);
}

template <class L> __host__ __device__ constexpr bool opposite_pairs() {
    for (int i = 1; i + 1 < L::Q; i += 2)
        for (int d = 0; d < 3; ++d)
            if (L::c(i + 1, d) != -L::c(i, d)) return false;
    return L::Q % 2 == 1;
}

// Signed sums of terms in a fixed order.  The first term is taken as it is
// (or negated) rather than added to zero: 0 + x = x for every x but -0, so
// the values are those of the plain running sum, without its first add.
template <class C> struct SignedSum {
    C v;
    bool empty = true;
    __device__ __forceinline__ void add(C x) {
        v = empty ? x : Ar<C>::add(v, x);
        empty = false;
    }
    __device__ __forceinline__ void sub(C x) {
        v = empty ? -x : Ar<C>::sub(v, x);
        empty = false;
    }
    __device__ __forceinline__ C get() const { return empty ? (C)0 : v; }
};

template <class L, class C> __device__ __forceinline__ void node_momentum(const C (&f)[L::Q], C (&j)[3]) {
    static_assert(opposite_pairs<L>(), "velocity order must pair c_{i+1} = -c_i");
    SignedSum<C> acc[3];
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const C dlt = Ar<C>::sub(f[i], f[i + 1]);
#pragma unroll
        for (int d = 0; d < L::D; ++d) {
            if (L::c(i, d) == 1) acc[d].add(dlt);
            if (L::c(i, d) == -1) acc[d].sub(dlt);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) j[d] = acc[d].get();
}

// g_s = -G sum_i w_i rho_s'(x + c_i) c_i for both species; nbr(s, i) returns
// rho_s(x + c_i).
template <class L, class C, class Nbr>
__device__ __forceinline__ void node_force(const Nbr& nbr, C G, C (&gA)[3], C (&gB)[3]) {
    using A = Ar<C>;
    static_assert(opposite_pairs<L>(), "velocity order must pair c_{i+1} = -c_i");
    gA[0] = gA[1] = gA[2] = gB[0] = gB[1] = gB[2] = (C)0;
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const C w = (C)L::w(i);
        const C dA = A::sub(nbr(0, i), nbr(0, i + 1));  // rho_A(x + c_i) - rho_A(x - c_i)
        const C dB = A::sub(nbr(1, i), nbr(1, i + 1));
#pragma unroll
        for (int d = 0; d < L::D; ++d) {
            if (L::c(i, d) == 1) {
                gA[d] = A::fma(w, dB, gA[d]);
                gB[d] = A::fma(w, dA, gB[d]);
            }
            if (L::c(i, d) == -1) {
                gA[d] = A::fma(-w, dB, gA[d]);
                gB[d] = A::fma(-w, dA, gB[d]);
            }
        }
    }
    const C mG = -G;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        gA[d] = A::mul(gA[d], mG);
        gB[d] = A::mul(gB[d], mG);
    }
}

// sin(2 pi y / ny) of the Kolmogorov forcing, y in [0, ny).
template <class C> __device__ __forceinline__ C kolmogorov_sine(int y, int ny);
template <> __device__ __forceinline__ float kolmogorov_sine<float>(int y, int ny) {
    return sinpif(__fdiv_rn((float)(2 * y), (float)ny));
}
template <> __device__ __forceinline__ double kolmogorov_sine<double>(int y, int ny) {
    return sinpi(__ddiv_rn((double)(2 * y), (double)ny));
}

// The Kolmogorov body force of Eq. kolmo (Sec. 4.2), F_x = rho A sin(2 pi y / ny),
// shared by the species in proportion to their densities (F_s,x = rho_s A sin):
// per unit density both g_A and g_B gain b = A sin(2 pi y / ny) along x, which
// then enters the shifted velocities u' + tau_s g_s and the F/2 shift of u_phys.
// A = 0 leaves g untouched.  b depends on the row only, so a kernel whose
// threads keep their row may form it once (kolmogorov_accel) and add it per
// node (node_add_body); node_body_force does both.
template <class C> __device__ __forceinline__ C kolmogorov_accel(C A, int y, int ny) {
    return A == (C)0 ? (C)0 : Ar<C>::mul(A, kolmogorov_sine<C>(y, ny));
}
template <class C> __device__ __forceinline__ void node_add_body(C A, C b, C (&gA)[3], C (&gB)[3]) {
    if (A == (C)0) return;
    gA[0] = Ar<C>::add(gA[0], b);
    gB[0] = Ar<C>::add(gB[0], b);
}
template <class C>
__device__ __forceinline__ void node_body_force(C A, int y, int ny, C (&gA)[3], C (&gB)[3]) {
    if (A == (C)0) return;
    node_add_body<C>(A, kolmogorov_accel<C>(A, y, ny), gA, gB);
}

// c_i . u as a signed sum of u's components (in the order of d).
template <class L, class C> __device__ __forceinline__ C node_cu(int i, const C (&u)[3]) {
    SignedSum<C> cu;
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
        if (L::c(i, d) == 1) cu.add(u[d]);
        if (L::c(i, d) == -1) cu.sub(u[d]);
    }
    return cu.get();
}

// BGK relaxation of one species towards f^eq(rho, u), each moving population
// relaxed as soon as its equilibrium is formed (fewer live values), the rest
// population last from the closure f^eq_0 = rho - sum_{i>0} f^eq_i, taken as
// f^eq_0 - f_0 = -sum_{i>0} (f^eq_i - f_i).
template <class L, class C> __device__ __forceinline__ void node_relax(C (&f)[L::Q], C rho, const C (&u)[3], C omega) {
    using A = Ar<C>;
    C uu = L::D == 3 ? A::fma(u[0], u[0], A::fma(u[1], u[1], A::mul(u[2], u[2]))) : A::fma(u[0], u[0], A::mul(u[1], u[1]));
    const C base = A::fma((C)-1.5, uu, (C)1);
    SignedSum<C> neq;  // sum_{i>0} (f^eq_i - f_i)
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const C cu = node_cu<L, C>(i, u);
        const C wr = A::mul((C)L::w(i), rho);
        const C feq = A::mul(wr, A::fma(cu, A::fma((C)4.5, cu, (C)3), base));
        const C d = A::sub(feq, f[i]);
        neq.add(d);
        f[i] = A::fma(omega, d, f[i]);
    }
    f[0] = A::fma(omega, -neq.get(), f[0]);  // f^eq_0 - f_0 = -sum_{i>0} (f^eq_i - f_i)
}

// Collision of both species of one node: common velocity shifted by tau_s g_s.
template <class L, class C>
__device__ __forceinline__ void node_collide(C (&f)[2][L::Q], C rA, C rB, const C (&gA)[3], const C (&gB)[3],
                                             C omega_A, C omega_B, C tau_A, C tau_B) {
    using A = Ar<C>;
    C jA[3], jB[3];
    node_momentum<L, C>(f[0], jA);
    node_momentum<L, C>(f[1], jB);
    const C inv_den = A::rcp(A::fma(rA, omega_A, A::mul(rB, omega_B)));
    C uA[3], uB[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const C up = A::mul(A::fma(jA[d], omega_A, A::mul(jB[d], omega_B)), inv_den);
        uA[d] = A::fma(tau_A, gA[d], up);
        uB[d] = A::fma(tau_B, gB[d], up);
    }
    node_relax<L, C>(f[0], rA, uA, omega_A);
    node_relax<L, C>(f[1], rB, uB, omega_B);
}

// Guo forcing, the discrete-forcing cure that Sec. 2.3 names for the
// tau-dependent coupling of the velocity shift (the paper prints no formulas;
// this is the standard form, per species, with F_s = rho_s g_s):
//   u_G = sum_s (j_s + F_s / 2) / tau_s / sum_s rho_s / tau_s
//   f_is += (1 / tau_s) (f^eq_i(rho_s, u_G) - f_is) + (1 - 1 / (2 tau_s)) S_is
//   S_is = w_i [3 (c_i - u_G).F_s + 9 (c_i.u_G) (c_i.F_s)]
// The source's rest component is closed as S_0 = -sum_{i>0} S_i (its sum over
// i vanishes in exact arithmetic), and f^eq_0 as in node_relax.  Opposite directions share
// their terms: with t1 = 9 (c.u)(c.F) - 3 u.F and t2 = 3 c.F (c = c_i),
// S_i = w_i (t1 + t2) and S_{i+1} = w_i (t1 - t2), since c_{i+1} = -c_i.
template <class L, class C>
__device__ __forceinline__ void node_relax_guo(C (&f)[L::Q], C rho, const C (&u)[3], const C (&F)[3], C omega) {
    using A = Ar<C>;
    C uu = L::D == 3 ? A::fma(u[0], u[0], A::fma(u[1], u[1], A::mul(u[2], u[2]))) : A::fma(u[0], u[0], A::mul(u[1], u[1]));
    C uF = L::D == 3 ? A::fma(u[0], F[0], A::fma(u[1], F[1], A::mul(u[2], F[2]))) : A::fma(u[0], F[0], A::mul(u[1], F[1]));
    const C base = A::fma((C)-1.5, uu, (C)1);
    const C keep = A::fma((C)-0.5, omega, (C)1);  // 1 - 1 / (2 tau)
    const C m3uF = A::mul((C)-3, uF);
    static_assert(opposite_pairs<L>(), "velocity order must pair c_{i+1} = -c_i");
    SignedSum<C> neq, sources;
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const C cu = node_cu<L, C>(i, u);  // c_{i+1}.u = -cu exactly (a signed sum of the same terms)
        const C cF = node_cu<L, C>(i, F);
        const C w = (C)L::w(i);
        const C wr = A::mul(w, rho);
        const C feq_p = A::mul(wr, A::fma(cu, A::fma((C)4.5, cu, (C)3), base));
        const C feq_m = A::mul(wr, A::fma(-cu, A::fma((C)4.5, -cu, (C)3), base));
        const C d_p = A::sub(feq_p, f[i]);
        const C d_m = A::sub(feq_m, f[i + 1]);
        neq.add(d_p);
        neq.add(d_m);
        const C t1 = A::fma(A::mul((C)9, cu), cF, m3uF);
        const C t2 = A::mul((C)3, cF);
        const C src_p = A::mul(w, A::add(t1, t2));
        const C src_m = A::mul(w, A::sub(t1, t2));
        sources.add(src_p);
        sources.add(src_m);
        f[i] = A::fma(keep, src_p, A::fma(omega, d_p, f[i]));
        f[i + 1] = A::fma(keep, src_m, A::fma(omega, d_m, f[i + 1]));
    }
    const C src0 = -sources.get();
    f[0] = A::fma(keep, src0, A::fma(omega, -neq.get(), f[0]));
}

template <class L, class C>
__device__ __forceinline__ void node_collide_guo(C (&f)[2][L::Q], C rA, C rB, const C (&gA)[3], const C (&gB)[3],
                                                 C omega_A, C omega_B) {
    using A = Ar<C>;
    C jA[3], jB[3];
    node_momentum<L, C>(f[0], jA);
    node_momentum<L, C>(f[1], jB);
    const C inv_den = A::rcp(A::fma(rA, omega_A, A::mul(rB, omega_B)));
    C FA[3], FB[3], u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        FA[d] = A::mul(rA, gA[d]);
        FB[d] = A::mul(rB, gB[d]);
        const C mA = A::fma((C)0.5, FA[d], jA[d]);
        const C mB = A::fma((C)0.5, FB[d], jB[d]);
        u[d] = A::mul(A::fma(mA, omega_A, A::mul(mB, omega_B)), inv_den);
    }
    node_relax_guo<L, C>(f[0], rA, u, FA, omega_A);
    node_relax_guo<L, C>(f[1], rB, u, FB, omega_B);
}

// ---- Free-energy (FE) two-population model (Sec. 2.2) ----------------------
// The storage's two "species" hold f_i (density and momentum) and g_i (order
// parameter): rho = sum_i f_i, phi = sum_i g_i, u = sum_i f_i c_i / rho.  The
// free energy is the Eq. FEtau functional with coupling g and gradient
// coefficient kappa; its derivatives come from the isotropic lattice stencils
//   grad phi = 3 sum_i w_i c_i phi(x + c_i),  lap phi = 6 sum_i w_i (phi(x + c_i) - phi(x)),
// formed over opposite pairs like the SC force.  nbr(1, i) = phi(x + c_i).
template <class L, class C, class Nbr>
__device__ __forceinline__ void node_fe_derivs(const Nbr& nbr, C phi0, C (&gp)[3], C& lp) {
    using A = Ar<C>;
    static_assert(opposite_pairs<L>(), "velocity order must pair c_{i+1} = -c_i");
    gp[0] = gp[1] = gp[2] = (C)0;
    C lap = (C)0;
    const C two_phi = A::add(phi0, phi0);
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const C w = (C)L::w(i);
        const C p = nbr(1, i), m = nbr(1, i + 1);
        const C d = A::sub(p, m);  // phi(x + c_i) - phi(x - c_i)
#pragma unroll
        for (int k = 0; k < L::D; ++k) {
            if (L::c(i, k) == 1) gp[k] = A::fma(w, d, gp[k]);
            if (L::c(i, k) == -1) gp[k] = A::fma(-w, d, gp[k]);
        }
        lap = A::fma(w, A::sub(A::add(p, m), two_phi), lap);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) gp[k] = A::mul((C)3, gp[k]);
    lp = A::mul((C)6, lap);
}

// ln x for the chemical potential (the library's log, FP32 or FP64).
__device__ __forceinline__ float fe_log(float x) { return logf(x); }
__device__ __forceinline__ double fe_log(double x) { return log(x); }

// The FE collision of one node (Eqs. FE1, FE2) with the second-order Hermite
// equilibria that meet Eqs. EQFE1 and EQFE2:
//   mu  = cs2/2 ln((rho + phi)/(rho - phi)) - g cs2 phi/2 - kappa lap phi
//   p_b = cs2 rho + g cs2 (rho^2 - phi^2)/4,  s = p_b - kappa phi lap - kappa/2 |grad|^2 - cs2 rho
//   f_i^eq = w_i [rho + 3 rho c.u + 9/2 (s (c.c - D cs2) + kappa ((c.grad)^2 - cs2 |grad|^2)
//                 + rho ((c.u)^2 - cs2 u.u))]
//   g_i^eq = w_i [phi + 3 phi c.u + 9/2 ((Gamma mu - cs2 phi)(c.c - D cs2) + phi ((c.u)^2 - cs2 u.u))]
// (the Hermite term (c_a c_b - cs2 d_ab) M_ab / (2 cs2^2) written out for the
// isotropic-plus-dyadic M of each population), rest components closed as
// rho - sum_{i>0} and phi - sum_{i>0} (each taken, as in node_relax, as minus
// the sum of the moving populations' increments f^eq_i - f_i).  omega = 1/tau, omega_g = 1/tau_g.
template <class L, class C>
__device__ __forceinline__ void node_collide_fe(C (&f)[2][L::Q], C rho, C phi, const C (&gp)[3], C lp, C omega,
                                                C omega_g, C g, C kappa, C gamma) {
    using A = Ar<C>;
    constexpr C cs2 = (C)(1.0 / 3.0);
    C j[3];
    node_momentum<L, C>(f[0], j);
    const C inv_rho = A::rcp(rho);
    C u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = A::mul(j[d], inv_rho);
    const C uu = L::D == 3 ? A::fma(u[0], u[0], A::fma(u[1], u[1], A::mul(u[2], u[2])))
                           : A::fma(u[0], u[0], A::mul(u[1], u[1]));
    const C gg = L::D == 3 ? A::fma(gp[0], gp[0], A::fma(gp[1], gp[1], A::mul(gp[2], gp[2])))
                           : A::fma(gp[0], gp[0], A::mul(gp[1], gp[1]));
    const C mu = A::sub(A::sub(A::mul(A::mul((C)0.5, cs2), fe_log(A::mul(A::add(rho, phi), A::rcp(A::sub(rho, phi))))),
                               A::mul(A::mul((C)0.5, A::mul(g, cs2)), phi)),
                        A::mul(kappa, lp));
    const C pb = A::fma(A::mul((C)0.25, A::mul(g, cs2)), A::mul(A::sub(rho, phi), A::add(rho, phi)), A::mul(cs2, rho));
    const C s = A::sub(A::sub(A::sub(pb, A::mul(A::mul(kappa, phi), lp)), A::mul(A::mul((C)0.5, kappa), gg)),
                       A::mul(cs2, rho));
    const C sg = A::sub(A::mul(gamma, mu), A::mul(cs2, phi));
    const C ku = A::mul(cs2, uu), kg = A::mul(cs2, gg);
    SignedSum<C> fneq, gneq;  // sum_{i>0} (f^eq_i - f_i), sum_{i>0} (g^eq_i - g_i)
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const C cu = node_cu<L, C>(i, u);
        const C cg = node_cu<L, C>(i, gp);
        int c2 = 0;
#pragma unroll
        for (int d = 0; d < L::D; ++d) c2 += L::c(i, d) * L::c(i, d);
        const C iso = (C)((double)c2 - (double)L::D / 3.0);  // c.c - D cs2
        const C quad_u = A::sub(A::mul(cu, cu), ku);       // (c.u)^2 - cs2 u.u
        const C quad_g = A::sub(A::mul(cg, cg), kg);
        const C w = (C)L::w(i);
        const C hf = A::fma(s, iso, A::fma(kappa, quad_g, A::mul(rho, quad_u)));
        const C feq = A::mul(w, A::fma((C)4.5, hf, A::fma(A::mul((C)3, rho), cu, rho)));
        const C hg = A::fma(sg, iso, A::mul(phi, quad_u));
        const C geq = A::mul(w, A::fma((C)4.5, hg, A::fma(A::mul((C)3, phi), cu, phi)));
        const C df = A::sub(feq, f[0][i]);
        const C dg = A::sub(geq, f[1][i]);
        fneq.add(df);
        gneq.add(dg);
        f[0][i] = A::fma(omega, df, f[0][i]);
        f[1][i] = A::fma(omega_g, dg, f[1][i]);
    }
    f[0][0] = A::fma(omega, -fneq.get(), f[0][0]);
    f[1][0] = A::fma(omega_g, -gneq.get(), f[1][0]);
}

// The collision of the lattice's forcing scheme, chosen at run time (kernels
// whose launch shapes accept either scheme).
template <class L, class C>
__device__ __forceinline__ void node_collide_any(int forcing, C (&f)[2][L::Q], C rA, C rB, const C (&gA)[3],
                                                 const C (&gB)[3], C omega_A, C omega_B, C tau_A, C tau_B) {
    if (forcing == kForcingGuo)
        node_collide_guo<L, C>(f, rA, rB, gA, gB, omega_A, omega_B);
    else
        node_collide<L, C>(f, rA, rB, gA, gB, omega_A, omega_B, tau_A, tau_B);
}

// The whole node update after the pulls: the SC force (and body force) with
// the lattice's forcing scheme, or the FE derivatives and collision, chosen at
// run time.  r0, r1: the two population sums of the node (rho_A, rho_B for SC;
// rho, phi for FE); nbr(s, i) returns the neighbour's sum s at x + c_i.
template <class L, class C, class Args, class Nbr>
__device__ __forceinline__ void node_update(const Args& a, int y, const Nbr& nbr, C (&f)[2][L::Q], C r0, C r1) {
    if (a.model == kModelFE) {
        C gp[3], lp;
        node_fe_derivs<L, C>(nbr, r1, gp, lp);
        node_collide_fe<L, C>(f, r0, r1, gp, lp, a.omega_A, a.omega_B, a.G, a.kappa, a.gamma);
        return;
    }
    C gA[3], gB[3];
    node_force<L, C>(nbr, a.G, gA, gB);
    node_body_force<C>(a.body_A, y, a.ny, gA, gB);
    node_collide_any<L, C>(a.forcing, f, r0, r1, gA, gB, a.omega_A, a.omega_B, a.tau_A, a.tau_B);
}

}  // namespace lbmsc

/*
 * pfm.h -- C ABI of the pseudo-spectral phase-field model (PFM) of Sec. 3,
 * the continuum counterpart the paper compares the lattice Boltzmann models
 * with (its cost ratio T_PFM / T_SC, Fig. 6), on one GPU.
 *
 * The model, in lattice units (grid spacing 1) on a periodic box, density- and
 * viscosity-matched, incompressible (Sec. 3, Eqs. eq8.1, eq2.2, eq3.2):
 *   div u = 0
 *   d phi/dt + u.grad phi = M lap mu_tau(phi),          M = rho (tau - 1/2)
 *   du/dt + u.grad u = -grad p + nu lap u + mu(phi) grad phi / rho,  nu = cs2 (tau - 1/2)
 *   mu_tau = cs2/2 ln((rho+phi)/(rho-phi)) - g_tau cs2 phi/2 - g_tau cs2^2/4 lap phi  (Eq. eq45)
 *   mu     = the same with the SC coupling g in place of g_tau = tau g/(tau - 1/2) (Eq. eq45.2)
 * (the paper writes the momentum equation per unit mass; its capillary force
 * is taken as mu grad phi / rho).  Time stepping as Sec. 3.1 (Eqs. eq10-eq13):
 * with D = M g_tau cs2/2 and xi^2 = cs2/2 the Cahn-Hilliard right-hand side is
 * split into an explicit part
 *   S = -u.grad phi + D lap[ln((rho+phi)/(rho-phi))/g_tau - 3 phi] - D (xi^2 - dt D/2) lap^2 phi
 * advanced by second-order Adams-Bashforth, and an implicit part
 *   Psi = D (2 lap phi - (dt D/2) lap^2 phi)
 * advanced by Crank-Nicolson; the velocity likewise, with -div(u u) + mu grad phi / rho
 * explicit (projected onto divergence-free fields) and nu lap u implicit.  The
 * first step takes the previous explicit term equal to the current one.
 * Optional Kolmogorov forcing of Eq. kolmo (Sec. 4.2): A sin(2 pi y / ny) along x
 * added to the explicit momentum right-hand side (per unit mass; divergence-free).
 * Spectral derivatives: i k for first derivatives (the Nyquist wavenumber of
 * an even axis zeroed), -|k|^2 for the Laplacian; products in physical space,
 * no dealiasing.  Transforms: cuFFT (real-to-complex and back, batched); the
 * spectral and physical-space steps are this library's kernels.
 *
 * Conventions: fields are arrays of nx*ny*nz values, x fastest, in the
 * precision's type (double for PFM_F64, float for PFM_F32); velocities D
 * planes u_x, u_y (, u_z).  The caller owns the device workspace and the
 * stream; the handle owns its cuFFT plans (cuFFT allocates their work areas).
 * Every call returns an lbm_status (lbm_sc.h) and never aborts.
 */
#ifndef PFM_H
#define PFM_H

#include <stddef.h>
#include <stdint.h>

#include "lbm_sc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { PFM_F64 = 0, PFM_F32 = 1 } pfm_precision;

typedef struct {
    int32_t dim;         /* 2 or 3                                                   */
    int32_t precision;   /* pfm_precision                                            */
    int32_t nx, ny, nz;  /* >= 2 each (nz = 1 for dim 2); nx*ny*nz < 2^31            */
    int32_t reserved;    /* set to 0                                                 */
    double rho;          /* uniform density (> 0)                                    */
    double tau;          /* LBM relaxation time the PFM is matched to (> 1/2)        */
    double g;            /* SC coupling g > 0 (g_tau = tau g / (tau - 1/2))          */
    double dt;           /* time step (> 0)                                          */
    double body_A;       /* Kolmogorov forcing amplitude A (finite); 0 = none        */
} pfm_params;

typedef struct pfm_handle pfm_handle;

/* Bytes of device workspace (spectral state, previous explicit terms and
 * transform scratch), 0 if the parameters are invalid. */
LBM_SC_API size_t pfm_workspace_bytes(const pfm_params* params);

/* Bind a solver to caller-owned device workspace (>= pfm_workspace_bytes,
 * 256-byte aligned) and a CUDA stream; builds the cuFFT plans. */
LBM_SC_API lbm_status pfm_create(const pfm_params* params, void* d_workspace, size_t workspace_bytes,
                                 void* cuda_stream, pfm_handle** out);

/* The state at t = 0 from phi (device, N values) and u (device, D*N values, or
 * NULL for rest; it should be divergence-free, the scheme keeps div u). */
LBM_SC_API lbm_status pfm_init(pfm_handle* h, const void* d_phi, const void* d_u);

/* Advance nsteps (>= 0) time steps of dt. */
LBM_SC_API lbm_status pfm_step(pfm_handle* h, int nsteps);

/* phi and u in physical space into device arrays (either may be NULL). */
LBM_SC_API lbm_status pfm_fields(pfm_handle* h, void* d_phi, void* d_u);

/* Release the handle and its plans (not the workspace). */
LBM_SC_API void pfm_destroy(pfm_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* PFM_H */

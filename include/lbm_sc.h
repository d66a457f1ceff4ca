/*
 * lbm_sc.h -- C ABI of the GB300 two-component Shan-Chen lattice Boltzmann step.
 *
 * The model (Scarbolo et al., Sec. 2.1): two species s in {A, B}, each with
 * BGK populations f_is on a D2Q9 or D3Q19 lattice, dt = 1,
 *
 *   f_is(x + c_i, t + 1) - f_is(x, t) = -(1/tau_s) [f_is - f^eq_is(rho_s, u' + tau_s F_s / rho_s)]
 *                                                                 (Eq. eq:be)
 *   rho_s = sum_i f_is,   u' = sum_s (1/tau_s) sum_i f_is c_i / sum_s rho_s / tau_s
 *   F_s(x) = -G rho_s(x) sum_i w_i rho_s'(x + c_i) c_i             (Eq. FORCE)
 *
 * with the second-order equilibrium f^eq_i = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u]
 * and fully periodic boundaries (Sec. 4).  Options of the same step (see
 * lbm_sc_params): the Kolmogorov body force of Eq. kolmo (Sec. 4.2), Guo forcing
 * in place of the velocity shift (lbm_forcing, Sec. 2.3), and the free-energy
 * two-population model of Sec. 2.2 on the same storage (lbm_model).  The
 * pseudo-spectral phase-field model of Sec. 3 has its own ABI (pfm.h).
 *
 * Conventions for every entry point:
 *   - The caller owns all device memory and the CUDA stream.  The library never
 *     allocates or frees device memory and never synchronises the device, except
 *     where an entry point says it does (lbm_sc_diagnostics, lbm_sc_run_host).
 *     lbm_sc_create allocates only the small host-side handle (malloc);
 *     lbm_sc_host_alloc / lbm_sc_host_free allocate and free pinned HOST memory
 *     through the driver (their mapping calls are synchronous driver calls).
 *   - "Device pointer" arguments must be device (or managed) memory on the
 *     current device; "host pointer" arguments ordinary host memory (pinned
 *     memory makes the copies asynchronous-capable and faster).
 *   - Fields are arrays of nx*ny*nz values, x fastest (index x + nx*(y + ny*z)),
 *     in the COMPUTE type of the precision: double for LBM_F64, float otherwise.
 *     Velocity fields hold D planes (D = 2 for D2Q9, 3 for D3Q19) one after the
 *     other: u_x[N], u_y[N] (, u_z[N]).
 *   - Every call returns an lbm_status and never aborts the process.  Kernel
 *     launches are asynchronous: a device fault surfaces as LBM_ERR_CUDA on a
 *     later call.
 *   - Calls on one handle must not run concurrently from several host threads.
 */
#ifndef LBM_SC_H
#define LBM_SC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_SC_API __attribute__((visibility("default")))
#else
#define LBM_SC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1,    /* bad parameter, pointer or size                        */
    LBM_ERR_OUT_OF_MEMORY = 2,  /* workspace too small, or the host handle malloc failed */
    LBM_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed           */
    LBM_ERR_UNSTABLE = 4,       /* diagnostics saw a non-finite value or rho_s <= 0       */
    LBM_ERR_TIMEOUT = 5         /* a bounded device-side wait expired                    */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Arithmetic is FP64 for LBM_F64 and FP32 otherwise.  LBM_F32_STORE_BF16 and
 * LBM_F32_STORE_F16 store h_is = f_is - w_i rho_ref_s (an offset from the rest
 * equilibrium of a reference density, one per species) in bf16 / fp16 and
 * decode to FP32 on load.  The _REST variants store h_is(n) = f_is(n) -
 * w_i rho_s(n), the offset from the rest equilibrium of the density of the
 * node n the value is stored at, with rho_s(n) itself kept in FP32, the two
 * species' offsets of one direction paired in one 32-bit word (A in the low
 * half, B in the high half) and encoded / decoded with one fused multiply-add
 * each (h = round16(fma(-w_i, rho_s, f)), f = fma(w_i, rho_s, h)): 16-bit
 * populations plus one float2 density plane per buffer (84 instead of 152
 * bytes per D3Q19 node), and an error that no longer grows with
 * |rho_s - rho_ref_s|, which in a two-phase lattice is large in one of the
 * phases whatever rho_ref_s is.  The paper computes in double precision throughout; the
 * 16-bit storage modes are a bandwidth option of this library. */
typedef enum {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F32_STORE_BF16 = 2,
    LBM_F32_STORE_F16 = 3,
    LBM_F32_STORE_BF16_REST = 4,
    LBM_F32_STORE_F16_REST = 5
} lbm_precision;

/* How the forces (Eq. FORCE and the body force) enter the collision.
 * LBM_FORCING_SHIFT is the paper's model (Sec. 2.1): each species relaxes to
 * f^eq(rho_s, u' + tau_s F_s / rho_s).  LBM_FORCING_GUO is the discrete-forcing
 * cure of Guo, Zheng and Shi that Sec. 2.3 names as the way to remove the
 * tau-dependent coupling g_tau = tau g / (tau - 1/2) of the shift; the paper
 * prints no formulas, and the library uses the standard form per species:
 * relaxation to f^eq(rho_s, u_G), u_G = sum_s (j_s + F_s/2)/tau_s /
 * sum_s rho_s/tau_s, plus (1 - 1/(2 tau_s)) w_i [3 (c_i - u_G).F_s +
 * 9 (c_i.u_G)(c_i.F_s)].  The reported velocity u_phys is the same for both. */
typedef enum { LBM_FORCING_SHIFT = 0, LBM_FORCING_GUO = 1 } lbm_forcing;

/* The lattice Boltzmann model.  LBM_MODEL_SC: the two-component Shan-Chen
 * model (Sec. 2.1), everything above.  LBM_MODEL_FE: the free-energy model of
 * Sec. 2.2 (Eqs. FE1, FE2) on the same storage, species 0 holding f_i
 * (rho = sum f_i, u = sum f_i c_i / rho) and species 1 holding g_i
 * (phi = sum g_i); tau_A is tau of f, tau_B is tau_g of g, G is the coupling g
 * of the Eq. FEtau functional
 *   V = cs2 (rho+phi)/2 ln((rho+phi)/2) + cs2 (rho-phi)/2 ln((rho-phi)/2) + g cs2 (rho^2-phi^2)/4,
 * with gradient coefficient kappa (g cs2^2 / 4 in Eq. FEtau) and mobility
 * Gamma (tau_g - 1/2).  mu = dV/dphi - kappa lap(phi) and the pressure tensor
 * P = (p_b - kappa phi lap(phi) - kappa/2 |grad phi|^2) delta + kappa grad(phi) grad(phi),
 * p_b = cs2 rho + g cs2 (rho^2 - phi^2)/4, enter second-order Hermite
 * equilibria that meet Eqs. EQFE1 and EQFE2 (sum f^eq cc = P + rho uu,
 * sum g^eq cc = Gamma mu delta + phi uu); derivatives by the isotropic lattice
 * stencils grad = 3 sum_i w_i c_i phi(x + c_i), lap = 6 sum_i w_i (phi(x + c_i) - phi(x)).
 * lbm_sc_init_fields takes rho_A, rho_B and sets f = w_i rho (rho = rho_A + rho_B),
 * g = w_i phi (phi = rho_A - rho_B) times the usual velocity factor; moments and
 * diagnostics report rho_A = (rho + phi)/2, rho_B = (rho - phi)/2, u and p_b.
 * FE needs LBM_F64 or LBM_F32, forcing 0 and body_A 0; |phi| < rho throughout. */
typedef enum { LBM_MODEL_SC = 0, LBM_MODEL_FE = 1 } lbm_model;

/* Parameters of one periodic lattice (Eq. eq:be, Eq. FORCE, and the optional
 * Kolmogorov forcing of Eq. kolmo). */
typedef struct {
    int32_t lattice;     /* lbm_lattice                                              */
    int32_t precision;   /* lbm_precision                                            */
    int32_t nx, ny, nz;  /* >= 1 each; nz must be 1 for D2Q9; nx*ny*nz < 2^31        */
    int32_t forcing;     /* lbm_forcing (0 = the paper's velocity shift)             */
    double tau_A, tau_B; /* relaxation times tau_s (> 1/2)                           */
    double G;            /* coupling G_AB = G_BA (> 0 repulsive)                     */
    double rho_ref_A;    /* reference densities of the 16-bit storage offsets;      */
    double rho_ref_B;    /* ignored for LBM_F64 / LBM_F32                            */
    double body_A;       /* amplitude A of the Kolmogorov body force of Eq. kolmo   */
                         /* (Sec. 4.2), F_x = rho A sin(2 pi y / ny), y = 0..ny-1,  */
                         /* shared by the species in proportion to their densities */
                         /* (F_s,x = rho_s A sin(2 pi y / ny)); finite; 0 = none    */
    int32_t model;       /* lbm_model (0 = the SC model)                             */
    int32_t reserved;    /* set to 0                                                 */
    double kappa;        /* LBM_MODEL_FE: gradient coefficient kappa (finite); a     */
                         /* negative value selects the Eq. FEtau coefficient        */
                         /* g cs2^2 / 4 = G / 36                                    */
    double gamma;        /* LBM_MODEL_FE: Gamma of Eq. EQFE2 (finite)                */
} lbm_sc_params;

/* Optional spherical windows for the drop diagnostics: nodes whose periodic
 * minimum-image distance r from (cx, cy, cz) satisfies r < r_in form the
 * inner window, r > r_out the outer window (Sec. 4.1, P_i and P_o). */
typedef struct {
    double cx, cy, cz;
    double r_in, r_out;
} lbm_sc_window;

/* FP64 scalars of the current state.  The velocity is the physical one,
 * u_phys = (sum_s j_s + (1/2) sum_s F_s) / (rho_A + rho_B) (Sec. 2.3, momentum
 * shifted by F dt/2; F includes the body force); p = cs2 (rho_A + rho_B) +
 * cs2 G rho_A rho_B (bulk part of the pressure tensor, Sec. 2.1). */
typedef struct {
    double mass_A, mass_B;        /* sum_x rho_A, sum_x rho_B                          */
    double momentum[3];           /* sum_x (j_A + j_B + (F_A + F_B) / 2)               */
    double kinetic_energy;        /* sum_x (rho/2) |u_phys|^2                          */
    double max_speed;             /* max_x |u_phys|                                    */
    double min_rho_A, min_rho_B;  /* minima over the lattice                           */
    double nonfinite;             /* number of nodes with a non-finite moment          */
    double in_count, in_rho_A, in_p;    /* inner window: node count, sum rho_A, sum p */
    double out_count, out_rho_A, out_p; /* outer window: node count, sum rho_A, sum p */
    double droplet_nodes;         /* nodes with phi = rho_A - rho_B >= 0, compared in  */
                                  /* the compute type: M(t) of the mass leakage       */
                                  /* L(t) = M(t) / M_0 (Sec. 4.2)                      */
} lbm_sc_diag;

typedef struct lbm_sc_handle lbm_sc_handle;

/* Launch shape of the step kernel.  tile selects the CTA tile of x by y
 * columns and the kernel: 0 = 32x8, 1 = 32x16, 2 = 64x8, 3 = 32x4, 4 = 64x4
 * (register-pipelined kernel, every lattice and precision); 5 to 10 are
 * retired ids (kernels measured slower at every size and removed; rejected
 * with LBM_ERR_INVALID_ARG); 11 = 32x4, 12 = 32x8, 13 = 64x4, 14 = 32x4 (low-register
 * kernel that pulls a plane a second time for its collision, every lattice and
 * precision; 11 and 14 differ in the register budget); 15 = 32x4, 16 = 32x8,
 * 17 = 16x8 (register-pipelined kernel holding three planes of pulls, D3Q19
 * with 32-bit storage or the reference-offset 16-bit storage); 18 = 32x8 with 3 stages, 19 = 64x4 with 3
 * stages, 20 = 32x4 with 4 stages, 21 = 32x4 with 2 stages, and the cluster
 * launches 22 = 64x4 in clusters of 1x2 tiles, 23 = 64x4 in 1x4, 24 = 64x4 in
 * 2x2, 25 = 32x8 in 2x2 (TMA-fed kernel, D3Q19 with LBM_F32 only, lattices
 * at least one tile wide in x and y whose tile counts divide by the cluster
 * shape); 26 to 29 are retired ids (other L2 fetch granularities of the
 * tensor copies, no faster); 30 = 64x4 in 1x2 clusters
 * with 3 stages, 31 = the same with 4 stages, 32 = 32x8 with 3 stages (the
 * TMA-fed kernel for the four 16-bit storage precisions, same size rules; the
 * rest-offset ones also stage the float2 densities); 33 = 64x6 with 2 stages in
 * 1x2 clusters, 34 = the same without clusters (FP32, 384 threads: 12 warps
 * per SM), 35 = 64x6 with 3 stages in 1x2 clusters (16-bit), 36 = 32x12 with
 * 2 stages in 1x2 clusters, 37 = the same without clusters (FP32), 38 = 32x12
 * with 3 stages in 1x2 clusters (16-bit), 39 = 64x8 with 2 stages in 1x2
 * clusters (16-bit, 512 threads), 40 = 48x8 with 2 stages in 1x2 clusters,
 * 41 = the same without clusters (FP32); 42 = 64x4 with 2 stages in 1x2
 * clusters, 43 = 32x8 with 2 stages in 1x2 clusters, 44 = 64x4 with 2 stages
 * without clusters (16-bit, two CTAs per SM: one CTA's per-plane barrier
 * overlaps the other's work).  With LBM_FORCING_GUO or
 * LBM_MODEL_FE the accepted tiles are those of the register and low-register
 * kernels (0-4, 11-14) and the TMA tile 34.  zchunk is the number
 * of z planes each CTA marches over per work item (D3Q19 only; 0 = automatic).
 * The shape changes only speed: every shape computes bit-identical results. */
typedef struct {
    int32_t tile;
    int32_t zchunk;
} lbm_sc_tuning;

/* Bytes of device workspace one lattice needs: two population buffers
 * (2 species x Q x N values of the storage type each) and the diagnostics
 * scratch.  Returns 0 if the parameters are invalid. */
LBM_SC_API size_t lbm_sc_workspace_bytes(const lbm_sc_params* params);

/* Bind a lattice to caller-owned device workspace (>= lbm_sc_workspace_bytes,
 * 256-byte aligned) and a CUDA stream (cudaStream_t; NULL = legacy default
 * stream).  The populations are undefined until lbm_sc_init_fields.  On
 * success *out receives a host handle that lbm_sc_destroy releases. */
LBM_SC_API lbm_status lbm_sc_create(const lbm_sc_params* params, void* d_workspace, size_t workspace_bytes,
                         void* cuda_stream, lbm_sc_handle** out);

/* Set / read the launch shape of the step kernel (see lbm_sc_tuning).
 * LBM_ERR_INVALID_ARG for an unknown tile, a tile the lattice and precision
 * do not support, or a negative zchunk. */
LBM_SC_API lbm_status lbm_sc_set_tuning(lbm_sc_handle* h, const lbm_sc_tuning* tuning);
LBM_SC_API lbm_status lbm_sc_get_tuning(const lbm_sc_handle* h, lbm_sc_tuning* tuning);

/* Change the stream later calls are enqueued on. */
LBM_SC_API lbm_status lbm_sc_set_stream(lbm_sc_handle* h, void* cuda_stream);

/* Populations at equilibrium of the given fields: f_is = f^eq(rho_s, u) (Sec. 2.1),
 * the state at t = 0.  d_rhoA, d_rhoB: device pointers to N compute-type values;
 * d_u: device pointer to D*N values, or NULL for a fluid at rest. */
LBM_SC_API lbm_status lbm_sc_init_fields(lbm_sc_handle* h, const void* d_rhoA, const void* d_rhoB,
                              const void* d_u);

/* Advance nsteps time steps (Eq. eq:be with Eq. FORCE): one fused kernel per
 * step pulls the populations along -c_i (periodic), forms rho_s and j_s, the
 * force from the neighbours' densities (plus the body force of Eq. kolmo when
 * body_A != 0), the common velocity u', relaxes each species to
 * f^eq(rho_s, u' + tau_s F_s / rho_s) and stores.  nsteps >= 0. */
LBM_SC_API lbm_status lbm_sc_step(lbm_sc_handle* h, int nsteps);

/* Macroscopic fields of the current state (moments of the populations at the
 * current time, before its collision): rho_A, rho_B, u_phys (D planes) and the
 * bulk pressure p.  Device pointers; any may be NULL. */
LBM_SC_API lbm_status lbm_sc_moments(lbm_sc_handle* h, void* d_rhoA, void* d_rhoB, void* d_u, void* d_p);

/* FP64 diagnostics of the current state (window may be NULL: no windows).
 * Synchronises the handle's stream and copies the result to *host_out.
 * Returns LBM_ERR_UNSTABLE (with *host_out filled) if a moment is non-finite or
 * a density is <= 0. */
LBM_SC_API lbm_status lbm_sc_diagnostics(lbm_sc_handle* h, const lbm_sc_window* window, lbm_sc_diag* host_out);

/* The diagnostics of lbm_sc_diagnostics for a caller that cannot allocate
 * device memory -- for example code running inside someone else's CUDA graph
 * capture or custom allocator, or a plugin that is handed device buffers but
 * may not call cudaMalloc itself.  It needs no handle and no workspace: the
 * per-CTA partial sums go to a fixed array of 16384 slots of 17 doubles
 * (2.1 MiB) in the library's static
 * device memory (allocated when the library is loaded, on every GPU that
 * loads it, and kept until the process exits).  The paper has no counterpart;
 * this is an interface convenience.
 *   params        the lattice (same rules as lbm_sc_workspace_bytes)
 *   d_populations device pointer to one population buffer in the layout of
 *                 lbm_sc_layout (for example the pointer it returns; with
 *                 its density planes for the _REST precisions)
 *   window        as for lbm_sc_diagnostics, or NULL
 *   d_out         device pointer to one lbm_sc_diag that receives the result
 *   cuda_stream   stream the work is enqueued on; the call does not synchronise
 * Returns LBM_ERR_INVALID_ARG for invalid parameters or pointers, and also when
 * the lattice needs more than 16384 partial-sum slots (one per 32 x 8 column
 * tile: more than about 4.2 million nodes per z plane), which the static array
 * cannot hold.  Unlike lbm_sc_diagnostics it does not check stability or
 * timeouts: read nonfinite and the minima from d_out.  The first call on each
 * device looks up the array's device address; make that first call before
 * any stream capture.  Every call reuses the same array (its contents are left
 * from the last call; each slot read is first written by the same call), so
 * calls whose execution overlaps on the GPU -- on different streams, or from
 * several threads -- race and must be serialised by the caller. */
LBM_SC_API lbm_status lbm_sc_diagnostics_noalloc(const lbm_sc_params* params, const void* d_populations,
                                                 const lbm_sc_window* window, lbm_sc_diag* d_out,
                                                 void* cuda_stream);

/* Bytes of device staging lbm_sc_run_host needs for its field copies. */
LBM_SC_API size_t lbm_sc_host_staging_bytes(const lbm_sc_params* params);

/* End-to-end run from host memory: copies rho_A, rho_B (and u, if not NULL)
 * from host pointers into d_staging, initialises, advances nsteps, computes the
 * moments and copies each non-NULL output back to host pointers (same layouts as
 * lbm_sc_moments).  d_staging: >= lbm_sc_host_staging_bytes, 256-byte aligned.
 * The copies run on a second stream in slabs of z planes (up to 8 for
 * D3Q19 lattices of 64 planes or more), so that the input copies overlap the
 * initialisation of the slabs already landed and the output copies of one
 * slab overlap the moments of the next; results are those of init_fields,
 * step and moments.  The first call on a handle creates that stream and a
 * few events (no device memory; lbm_sc_destroy releases them); make it
 * outside any stream capture.  Synchronises the handle's stream before
 * returning. */
LBM_SC_API lbm_status lbm_sc_run_host(lbm_sc_handle* h, void* d_staging, size_t staging_bytes,
                           const void* h_rhoA, const void* h_rhoB, const void* h_u, int nsteps,
                           void* h_rhoA_out, void* h_rhoB_out, void* h_u_out, void* h_p_out);

/* Page-locked host memory for the host buffers of lbm_sc_run_host (or any
 * other copy to or from the device): *out receives a buffer of at least bytes
 * bytes, zero-filled, allocated by the CUDA driver as pinned memory on the host
 * NUMA node nearest the current device (cuMemCreate with a host location, in
 * the driver's recommended granules, mapped for the host and the current
 * device).  The driver owns these pages, so the host kernel neither moves nor
 * splits them: measured on a Grace host, a 60-step 512^3 job of
 * lbm_sc_run_host took 0.499 s on every run with such buffers, and 0.50 to
 * 0.93 s with buffers of cudaHostAlloc or of registered user pages (64 KiB
 * base pages; their copies slowed after the link had been idle, and
 * registered huge pages were split by the kernel within seconds).  The caller
 * owns the buffer and releases it with lbm_sc_host_free(p, bytes) (the same
 * bytes, same current device).  Returns LBM_ERR_INVALID_ARG for bytes == 0 or a
 * NULL out, LBM_ERR_OUT_OF_MEMORY if the driver has no memory for it,
 * LBM_ERR_CUDA for any other failure (no device, no driver support); nothing
 * stays allocated and *out is NULL on every error. */
LBM_SC_API lbm_status lbm_sc_host_alloc(size_t bytes, void** out);

/* Release a buffer of lbm_sc_host_alloc (NULL: nothing to do).  bytes: the size
 * it was allocated with (LBM_ERR_INVALID_ARG if 0).  LBM_ERR_CUDA if the driver
 * reports a failure. */
LBM_SC_API lbm_status lbm_sc_host_free(void* p, size_t bytes);

/* Population storage layout (for tools such as checkpointing): bytes of one
 * stored value, number of velocities Q, and the geometry of the current
 * population buffer.  It holds 2 x Q planes (index s*Q + i, GPU velocity order)
 * of pitch_x * pitch_y * nz values each; node (x, y, z) sits at
 * (x + ghost_x) + pitch_x * ((y + ghost_y) + pitch_y * z).  The columns
 * x = -2, -1, nx, nx + 1 and rows y = -2, -1, ny, ny + 1 hold periodic images;
 * other padding is unused.  For the _REST precisions a stored value is one
 * 32-bit word holding both species (elem_bytes = 4): Q planes (index i) of
 * such words, followed by one plane of float2 densities (rho_A, rho_B) with the
 * same pitches, node (x, y, z) at the same index (8 bytes per node).  Any output pointer may be NULL. */
LBM_SC_API lbm_status lbm_sc_layout(const lbm_sc_handle* h, int* elem_bytes, int* q, int* pitch_x, int* pitch_y,
                                    int* ghost_x, int* ghost_y, const void** d_populations);

/* ---- Failure detection -----------------------------------------------------
 * The paper has no counterpart: these two calls test the library's bounded
 * device waits (every mbarrier wait of the TMA-fed kernels, tile kinds 5 and 6,
 * gives up after a fixed number of tries, raises the device error word, waits
 * with the same bound for its own copies still in flight and returns, so the
 * CUDA context stays usable and lbm_sc_diagnostics reports LBM_ERR_TIMEOUT).
 *
 * lbm_sc_set_wait_probe: tries > 0 makes the first CTA of every later step of
 * this handle (tile (0, 0), first z chunk) wait `tries` tries on a barrier
 * that nothing ever arrives on before its first plane, so that wait runs out
 * and the error path runs; that CTA then stores nothing for that step (the
 * handle's state is no longer a solution: re-initialise it).  tries = 0 turns
 * the hook off.  Other tile kinds ignore it.  The error word stays set until
 * lbm_sc_init_fields clears it.  Returns LBM_ERR_INVALID_ARG for tries < 0. */
LBM_SC_API lbm_status lbm_sc_set_wait_probe(lbm_sc_handle* h, int tries);

/* The device error word of the handle, after synchronising its stream: 0 = no
 * wait expired; bit 0 set = a bounded wait expired; bit 1 set as well = a CTA
 * could not confirm, within the same bound, that the copies into its shared
 * memory had landed before it left (the device state is then suspect). */
LBM_SC_API lbm_status lbm_sc_error_word(lbm_sc_handle* h, int* host_out);

/* ---- Ragged batch ---------------------------------------------------------
 * Many independent lattices of different sizes and parameters advanced
 * together, one kernel launch per time step for the whole batch.  Each step
 * is Eq. eq:be with Eq. FORCE on every lattice of the batch, exactly as
 * lbm_sc_step computes it: the results are bit-identical to stepping each
 * lattice alone.  The paper runs one lattice at a time; batching is a
 * throughput device for many small lattices, which alone cannot fill the GPU.
 *
 * The launch covers a work list of (lattice, x tile, y tile, z chunk) items,
 * longest first, either with a persistent grid of CTAs that take items from
 * an atomic counter or with one CTA per item (see tile below); per-lattice
 * arguments come from a descriptor array.  The list, the descriptors and the
 * counter live in the batch workspace (device memory owned by the caller).  When graph_steps > 0 and the stream is not the legacy
 * default stream, whole chunks of graph_steps steps are replayed from a CUDA
 * graph captured on the first use (one per starting parity); the remaining
 * steps are direct launches.
 *
 * All handles of a batch must share the lattice kind and the precision
 * (LBM_ERR_INVALID_ARG otherwise); each must have been initialised
 * (lbm_sc_init_fields) before the first lbm_sc_batch_step.  While the batch
 * exists, advance its lattices only through it: lbm_sc_batch_step reports
 * LBM_ERR_INVALID_ARG if a handle was stepped on its own in between.
 * lbm_sc_moments and lbm_sc_diagnostics on a handle read the state the batch
 * left (enqueue them on the batch's stream, or synchronise it first).
 *   tile    CTA tile (x by y columns) and kernel: 0 = 32x8, 1 = 32x4, 2 = 64x4
 *           (z-marching kernel, every lattice and precision) and 3 = 32x8,
 *           4 = 64x4 (TMA-fed kernel, D3Q19 with LBM_F32, every lattice at
 *           least one tile wide in x and y), all as persistent grids that
 *           take work items from an atomic counter in the batch workspace;
 *           5 = 32x8, 6 = 64x4 (TMA-fed) and 7 = 32x8, 8 = 64x4 (z-marching)
 *           launch one CTA per work item instead; 9 = TMA-fed, one CTA per
 *           item, each lattice with its own tile: 64x4 if it is at least 64
 *           wide, else 32x8 (same requirements as 5); 10 = 32x12 and 11 =
 *           64x6 / 32x12 per lattice, the same with 384-thread CTAs (every
 *           lattice at least 32 x 12); 12 = each lattice in the one of 64x6,
 *           48x8 and 32x12 with the least work per node for its size (384
 *           threads, one CTA per item).  13 = the TMA-fed kernel for
 *           LBM_F32_STORE_BF16_REST / LBM_F32_STORE_F16_REST (D3Q19, every
 *           lattice at least 32 x 8): 32x8 tiles, two CTAs per SM, one CTA
 *           per item.  The TMA-fed tiles (3-6, 9-13) need every lattice on
 *           LBM_MODEL_SC with LBM_FORCING_SHIFT; in the TMA batches odd z
 *           chunks march downwards (results unchanged); the z-marching ones
 *           take lattices of any forcing and model, mixed.
 *   zchunk  z planes per work item (D3Q19; 0 = 32; capped at each nz)
 *   graph_steps  steps per captured graph (even, >= 0; 0 = no graphs) */
typedef struct lbm_sc_batch lbm_sc_batch;

/* Bytes of batch workspace for these handles and shape (0 if invalid). */
LBM_SC_API size_t lbm_sc_batch_workspace_bytes(lbm_sc_handle* const* handles, int n, int tile, int zchunk);

/* Build a batch over n handles (the array is copied; the handles must outlive
 * the batch).  d_workspace: >= lbm_sc_batch_workspace_bytes, 256-byte aligned.
 * Uploads the descriptors and the work list and synchronises cuda_stream once. */
LBM_SC_API lbm_status lbm_sc_batch_create(lbm_sc_handle* const* handles, int n, int tile, int zchunk,
                                          int graph_steps, void* d_workspace, size_t workspace_bytes,
                                          void* cuda_stream, lbm_sc_batch** out);

/* Advance every lattice of the batch by nsteps (>= 0) on the batch's stream;
 * asynchronous like lbm_sc_step. */
LBM_SC_API lbm_status lbm_sc_batch_step(lbm_sc_batch* b, int nsteps);

/* Release the batch (and its graphs).  The handles and workspace stay the caller's. */
LBM_SC_API void lbm_sc_batch_destroy(lbm_sc_batch* b);

/* Release the host handle (and the copy stream and events of lbm_sc_run_host,
 * if it made them).  The workspace stays the caller's. */
LBM_SC_API void lbm_sc_destroy(lbm_sc_handle* h);

/* Static, human-readable name of a status code. */
LBM_SC_API const char* lbm_sc_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_SC_H */

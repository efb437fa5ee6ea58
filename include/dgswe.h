/*
 * dgswe.h -- C-ABI of libdgswe, a GB300 (sm_103a) solver for the rotating
 * shallow water equations on the sphere, discretised by the modal
 * Discontinuous Galerkin method of arxiv 2303.11767 (Sec. 2) and advanced by
 * explicit SSP Runge-Kutta.
 *
 * Problem (paper Sec. 2, Eq. sph3 and the definitions of U, F, G, S after it):
 *   d_t U + d_lambda F(U) + d_theta G(U) = S(U),   U = cos(theta) (h, hu, hv),
 * on the longitude-latitude rectangle lambda in [0, 2 pi], theta in
 * [-pi/2, pi/2], periodic in lambda, zero flux through the pole edges
 * (Sec. 2 and Sec. 4.3).  Element (i, j) covers
 *   lambda in [i dlam, (i+1) dlam],  theta in [-pi/2 + j dth, -pi/2 + (j+1) dth],
 * dlam = 2 pi / nlon, dth = pi / nlat.  The unknowns are the modal
 * coefficients of (h, hu, hv) in the tensor basis phi_m = L_a(xi) L_b(eta) of
 * orthonormal Legendre polynomials L_k = sqrt((2k+1)/2) P_k, m = b (p+1) + a
 * (Eq. basis_expansion); cos(theta) lives in the element mass matrix (Eq. ode
 * and the cos(theta)-weighted M that follows it).
 *
 * State layout, everywhere in this API: double array of
 *   len = nlat * nlon * 3 * (p+1)^2  values, index
 *   ((j * nlon + i) * 3 + f) * (p+1)^2 + m,   f = 0 h, 1 hu, 2 hv.
 *
 * Conventions:
 *   - Every call returns a dg_status and never aborts the process.
 *   - Host pointers are borrowed for the duration of the call only; the
 *     library copies what it keeps.
 *   - The state stays resident on the GPU between calls (paper Sec. 5.2.3:
 *     host-device traffic only at the start).
 *   - Calls on one handle must not run concurrently from several threads.
 *     Separate handles are independent.
 *   - dg_last_error() describes the last failing call of the calling thread.
 *   - An error returned by a CUDA call (DG_ECUDA) may leave the device
 *     context unusable; destroy the handle.
 */
#ifndef DGSWE_H
#define DGSWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx *dg_handle;

typedef enum {
    DG_OK = 0,
    DG_EINVAL = 1,          /* invalid argument (message in dg_last_error) */
    DG_ENOMEM = 2,          /* host or device allocation failed */
    DG_ECUDA = 3,           /* a CUDA runtime call failed */
    DG_ENONFINITE = 4,      /* a NaN or Inf appeared in the state or tendency */
    DG_ENONPHYSICAL = 5,    /* h <= 0 at a quadrature point (u = hu/h undefined) */
    DG_ETIMEOUT = 6,        /* a bounded device-side wait gave up */
    DG_EUNSUPPORTED = 7     /* valid request that the library does not implement */
} dg_status;

typedef enum {
    DG_PREC_FP64 = 0,           /* all stage arithmetic in FP64 */
    DG_PREC_FP32 = 1,           /* stage arithmetic in FP32, FP64 tables and mass sums */
    DG_PREC_FP32_TC_BF16 = 2,   /* FP32 stage; the basis contractions (modes -> Gauss and
                                   edge points, volume integral and lift) as BF16 x BF16
                                   tensor-core GEMMs with FP32 accumulation; C_j^-1, fluxes
                                   and the RK update in FP32 */
    DG_PREC_FP32_TC_FP16 = 3,   /* the same with FP16 operands (momenta scaled by 2^-5
                                   into the FP16 range) */
    DG_PREC_FP32_TC_BF16_SPLIT = 4, /* BF16 tensor cores with split operands: every operand
                                   held as a pair hi + lo of BF16 values (lo = the rounded
                                   residual) and every contraction taken as A_hi B_hi +
                                   A_lo B_hi + A_hi B_lo in the FP32 accumulator, so the
                                   rounding error per term falls from u to ~u^2 */
    DG_PREC_FP32_TC_FP16_SPLIT = 5  /* the same with FP16 pairs (22 of FP32's 24 bits) */
} dg_precision;

typedef enum {
    DG_OPT_PRECISION = 1,        /* dg_precision; default DG_PREC_FP64.  Changing it
                                    converts the resident state. */
    DG_OPT_RK_ORDER = 2,         /* 1..4, the SSP RK schemes of Table "Butcher";
                                    default 3 */
    DG_OPT_CHECK_FINITE = 3,     /* 0/1, default 1: dg_step and dg_rhs report
                                    DG_ENONFINITE / DG_ENONPHYSICAL */
    DG_OPT_ALPHA_MODE = 4,       /* 0: local Rusanov alpha, the larger one-sided
                                    speed of each face point (default); 1: global,
                                    every face uses the maxima of |u| + sqrt(gh)
                                    (lambda faces) and |v| + sqrt(gh) (theta faces)
                                    over all Gauss points of the stage input,
                                    computed by one extra kernel per stage */
    DG_OPT_STREAM = 5,           /* cudaStream_t cast to long long; 0 = the
                                    library's own non-blocking stream */
    DG_OPT_STEPS_PER_GRAPH = 6,  /* time steps captured per CUDA graph, 1..1024,
                                    default 16 */
    DG_OPT_TILE_ROWS = 7,        /* ensemble only: latitude rows per CTA tile, 4 or 8
                                    (default 8; dg_ensemble_autotune picks it) */
    DG_OPT_BLOCKS_PER_SM = 8,    /* ensemble only: persistent CTAs per SM, 1..8 (default 2) */
    DG_OPT_WELL_BALANCED = 9     /* 0 (default) / 1: remove from every tendency that of the
                                    fluid at rest at the reference depth (the mean depth of the
                                    state at dg_set_state), i.e. the quadrature residual of its
                                    constant pressure, so that rest state is exactly steady;
                                    FP64 then also stores h relative to that depth */
} dg_option;

/* Make CUDA device `device` current for the calling thread in this library
 * (the device dg_create allocates on).  DG_EINVAL if it does not exist. */
dg_status dg_set_device(int device);

/* Create a solver for an nlon x nlat element mesh of degree p (0 <= p <= 4;
 * p = 0 is the first-order finite-volume special case).  nlon >= 1, nlat >= 2,
 * radius > 0, g > 0.  Builds the FP64 tables (Gauss-Legendre rules, Legendre
 * tables, per-row cos(theta)-weighted mass matrices C_j and their inverses,
 * Sec. 3.2 "DG solver: precomputation") and allocates the device buffers on
 * the current CUDA device.  *out receives the handle (NULL on failure). */
dg_status dg_create(int nlon, int nlat, int degree, double radius, double g, double omega,
                    dg_handle *out);

/* The paper's planar validation problem (Sec. 4.1, Eq. lin_adv): linear
 * advection du/dt + div(beta u) = 0 of one scalar on the unit square,
 * periodic in both directions, nx x ny elements of degree 0..4, FP64, beta =
 * (bx, by); alpha_speed 1: Rusanov alpha = |beta|, 0: |beta . n| (upwind).
 * State layout [y j][x i][mode m = b*n + a], dg_state_len = nx ny (p+1)^2.
 * The handle supports dg_set_state(_device), dg_get_state(_device), dg_rhs,
 * dg_step (DG_OPT_RK_ORDER 1..4, graphs), DG_OPT_RK_ORDER / STEPS_PER_GRAPH /
 * STREAM / CHECK_FINITE, dg_get_time / dg_set_time and dg_destroy; the
 * sphere-only calls return DG_EUNSUPPORTED. */
dg_status dg_create_plane_advection(int nx, int ny, int degree, double bx, double by, int alpha_speed,
                                    dg_handle *out);

/* Planar shallow water on the f-plane (Sec. 4.3, the geostrophic adjustment
 * set-up, also the workload of the paper's timings): (h, hu, hv) on the
 * square [0, L]^2, periodic in both directions, constant Coriolis parameter
 * f, nx x ny elements of degree 0..4, FP64; F = (hu, hu u + g h^2/2, hu v),
 * G = (hv, hv u, hv v + g h^2/2), S = (0, f hv, -f hu), Rusanov alpha = the
 * larger one-sided |u| + c or |v| + c.  State layout as on the sphere,
 * [y j][x i][field f][mode m]; the same calls as dg_create_plane_advection
 * plus dg_total_mass (int h dx dy). */
dg_status dg_create_plane_swe(int nx, int ny, int degree, double L, double g, double f, dg_handle *out);

/* Free the handle and its device buffers.  NULL is accepted. */
dg_status dg_destroy(dg_handle h);

/* Set an option (see dg_option). */
dg_status dg_set_option(dg_handle h, int key, long long value);

/* Number of doubles in a state array: nlat * nlon * 3 * (degree+1)^2
 * (0 for a NULL handle). */
size_t dg_state_len(dg_handle h);

/* Copy a modal state from host memory into the solver (layout above).
 * len must equal dg_state_len(h).  Resets nothing else; the simulated time is
 * kept (see dg_set_time). */
dg_status dg_set_state(dg_handle h, const double *modal, size_t len);

/* Copy the current modal state into caller-owned host memory; synchronises
 * the solver's stream. */
dg_status dg_get_state(dg_handle h, double *modal, size_t len);

/* Same as dg_set_state / dg_get_state with a device pointer (FP64, same
 * layout), ordered on the solver's stream. */
dg_status dg_set_state_device(dg_handle h, const double *d_modal, size_t len);
dg_status dg_get_state_device(dg_handle h, double *d_modal, size_t len);

/* Tendency d(modal)/dt = M^{-1} h(modal) of Eq. (ode) for the given host
 * state: the volume, source and edge integrals of the weak form (Eq. dg_parts)
 * with the Rusanov flux (Eq. rusanov), then the inverse element mass matrix.
 * Does not touch the resident state.  modal_in and tend_out are host arrays of
 * length len = dg_state_len(h), layout above. */
dg_status dg_rhs(dg_handle h, const double *modal_in, double *tend_out, size_t len);

/* Advance the resident state by n >= 0 steps of size dt > 0 with the SSP
 * Runge-Kutta scheme of order DG_OPT_RK_ORDER (Table "Butcher"), replaying a
 * captured CUDA graph of fused stage kernels.  Adds n*dt to the simulated
 * time.  With DG_OPT_CHECK_FINITE, synchronises and reports DG_ENONFINITE or
 * DG_ENONPHYSICAL if any stage met a non-finite value or h <= 0. */
dg_status dg_step(dg_handle h, int n, double dt);

/* Total mass R^2 sum_k int h cos(theta) dlambda dtheta of the resident state
 * (paper Sec. 2: the single-valued numerical flux conserves it), reduced on
 * the GPU in FP64 with compensated (Neumaier) sums in a fixed order, so the
 * result is reproducible bit for bit. */
dg_status dg_total_mass(dg_handle h, double *mass);

/* Same reduction, enqueued on the solver's stream without waiting: writes the
 * total mass (one double) to the device pointer d_mass when the stream
 * reaches it.  Usable inside CUDA graph capture of the solver's stream. */
dg_status dg_total_mass_device(dg_handle h, double *d_mass);

/* Largest stable step from the Courant number p c dt / H of Sec. 2:
 *   H = min over elements and Gauss points of min(R dth, R cos(theta) dlam),
 *   c = max over Gauss points of sqrt(u^2 + v^2) + sqrt(g h),
 *   dt = cfl * H / (max(p, 1) * c),
 * evaluated on the resident state on the GPU.  Returns DG_ENONPHYSICAL if
 * h <= 0 at a Gauss point. */
dg_status dg_max_dt(dg_handle h, double cfl, double *dt);

/* Coordinates of the projection points: nm = p + 9 Gauss-Legendre points per
 * element and direction.  lam receives nlon * nm values (index i * nm + q),
 * theta nlat * nm values (index j * nm + q). */
dg_status dg_projection_nodes(dg_handle h, double *lam, size_t nlam, double *theta, size_t ntheta);

/* cos(theta)-weighted L^2 projection (mass matrix of Eq. ode) of point values
 * onto the modal basis.  nodal holds the three fields at the projection
 * points of every element, layout [j][i][f][q_theta][q_lambda]
 * (len_nodal = nlat * nlon * 3 * nm * nm); modal_out receives dg_state_len(h)
 * values.  Host computation in FP64; does not touch the resident state. */
dg_status dg_project_nodal(dg_handle h, const double *nodal, size_t len_nodal, double *modal_out,
                           size_t len);

/* Simulated time of the resident state (advanced by dg_step). */
dg_status dg_get_time(dg_handle h, double *t);
dg_status dg_set_time(dg_handle h, double t);

/* ------------------------------------------------------------------------
 * Latitude-band sharding of one mesh.  The paper (Sec. 5.1) names the
 * Rusanov-flux phase as the only one that exchanges data between neighbouring
 * elements: an element needs only its four neighbours' traces (Eq. rusanov),
 * so contiguous latitude bands exchange one boundary row with each
 * neighbouring band per Runge-Kutta stage.  A band
 * handle owns rows [j_begin, j_end) of an nlon x nlat mesh; every state array
 * of the handle also holds one ghost row below (j_begin > 0) and one above
 * (j_end < nlat) the own rows, which receive the neighbour bands' rows.  Its
 * state (dg_set_state, dg_get_state, dg_state_len) covers the own rows only,
 * layout as above with j counted from j_begin.  The stage kernel is the
 * whole mesh's, so a band split reproduces the whole mesh's stages bit for
 * bit when every band uses the same reference depth
 * (dg_band_set_reference_depth, FP32).  Supported: FP64 and FP32 stages, RK
 * orders 1-4, the local Rusanov alpha, the well-balanced option.  dg_step,
 * dg_rhs, dg_restrict_from, dg_attach_mlp, the tensor-core precisions and
 * the global alpha mode return DG_EUNSUPPORTED on a band.  Per stage the
 * driver packs each band's boundary rows, delivers them to the neighbours
 * (any transport: a device copy, NCCL, host memory), unpacks them into the
 * ghost rows, then calls dg_band_stage on every band.
 * ------------------------------------------------------------------------ */

/* Create the band [j_begin, j_end) of the nlon x nlat mesh of degree p
 * (arguments otherwise as dg_create; 0 <= j_begin < j_end <= nlat). */
dg_status dg_create_band(int nlon, int nlat, int j_begin, int j_end, int degree, double radius, double g,
                         double omega, dg_handle *out);

/* Values (of the working precision: double for FP64, float for FP32) of one
 * halo message: a row's stage base followed by its stage increment,
 * 2 * nlon * 3 * (p+1)^2.  0 for a handle that is not a band. */
size_t dg_band_halo_len(dg_handle h);

/* Reference depth of the FP32 storage (h is stored relative to it; FP64 only
 * with the well-balanced option) for the next dg_set_state: give every band
 * the whole mesh's mean element depth, 0.5 * sum_e u_e[h][0] / nel, so the
 * bands hold the same bits as the whole mesh would. */
dg_status dg_band_set_reference_depth(dg_handle h, double href);

/* Copy the input of the next stage on own row 0 (side 0, south) or on the
 * last own row (side 1, north) -- the row's u^n and the stage's increment
 * (zeros for a stage without one) -- into d_out, a caller-owned device buffer
 * of dg_band_halo_len values.  Ordered on the handle's stream. */
dg_status dg_band_pack(dg_handle h, int side, void *d_out);

/* Write a neighbour's packed row into the south (side 0) or north (side 1)
 * ghost row, as the input of this band's next stage.  DG_EINVAL where that
 * side is a pole.  Ordered on the handle's stream. */
dg_status dg_band_unpack(dg_handle h, int side, const void *d_in);

/* Run the next stage of the current time step (stage 1, 2, ... of the RK
 * scheme of DG_OPT_RK_ORDER) with step size dt, which must stay the same
 * within a step (DG_EINVAL otherwise); change DG_OPT_RK_ORDER only between
 * steps.  After a step's last stage the simulated time advances by dt and,
 * with DG_OPT_CHECK_FINITE, the status is read as in dg_step. */
dg_status dg_band_stage(dg_handle h, double dt);

/* The two terms of the CFL step of dg_max_dt over the band's own rows:
 * *H = min over the rows and Gauss points of min(R dth, R cos(theta) dlam)
 * and *c = max over the Gauss points of sqrt(u^2 + v^2) + sqrt(g h).  The
 * whole mesh's step is cfl * min(H) / (max(p, 1) * max(c)) over the bands
 * (the smallest H and the largest c may sit in different bands, so the
 * bands' own steps do not give it).  Works on any sphere handle. */
dg_status dg_band_cfl_terms(dg_handle h, double *H, double *c);

/* The band's mass as the compensated (Neumaier) pair of its fixed-order
 * reduction: the band's mass is R^2 (sum + err); merging the bands' pairs in
 * band order with an error-free two-sum gives the whole mesh's mass. */
dg_status dg_band_mass_pair(dg_handle h, double *sum, double *err);

/* ------------------------------------------------------------------------
 * Learned correction: a per-element multilayer perceptron (n_in -> H -> H ->
 * n_out, GELU (erf form), BF16 weights, FP32 accumulation, FP32 master
 * weights and Adam moments) trained on the GPU by the library's own forward
 * and backward kernels, used as an added modal source term of a degree-1
 * solver.  The paper has no learned component; this is the ML extension of
 * the method built on it (trained on pairs the method itself generates).
 * Batches are row-major FP32 device arrays [batch][features], batch <= 8192.
 * ------------------------------------------------------------------------ */
typedef struct dg_mlp_ctx *dg_mlp;

/* He-uniform weights from `seed`, zero biases, identity normalisation. */
dg_status dg_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed, dg_mlp *out);
dg_status dg_mlp_destroy(dg_mlp m);
/* Number of parameters; layout W1[H][n_in], b1[H], W2[H][H], b2[H],
 * W3[n_out][H], b3[n_out]. */
size_t dg_mlp_num_params(dg_mlp m);
dg_status dg_mlp_get_params(dg_mlp m, float *params, size_t n);   /* host buffer */
dg_status dg_mlp_set_params(dg_mlp m, const float *params, size_t n);
/* Inputs are used as (x - in_mean) / in_std; the network predicts targets as
 * (t - out_mean) / out_std (host arrays of n_in and n_out values, std > 0). */
dg_status dg_mlp_set_normalization(dg_mlp m, const float *in_mean, const float *in_std, const float *out_mean,
                                   const float *out_std);
/* Optional per-latitude-row output statistics for the learned source
 * (dg_attach_mlp): with them the source of an element of row j is
 * y * out_std_rows[j][q] + out_mean_rows[j][q] (host arrays of nlat x n_out
 * values, std > 0) instead of the global out_mean / out_std, so a network
 * trained on row-normalised targets carries the latitude dependence of the
 * coarse mesh's error without a position input.  nlat must equal the
 * attached solver's nlat (else its steps fail with DG_EINVAL); nlat = 0
 * removes them. */
dg_status dg_mlp_set_row_normalization(dg_mlp m, int nlat, const float *out_mean_rows, const float *out_std_rows);
/* Normalised network output of a batch (device arrays). */
dg_status dg_mlp_forward(dg_mlp m, const float *d_x, int batch, float *d_y);
/* Mean squared error on normalised targets and its gradient (host buffer of
 * dg_mlp_num_params values, same layout as the parameters). */
dg_status dg_mlp_gradients(dg_mlp m, const float *d_x, const float *d_t, int batch, float *grads, size_t n,
                           double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch; loss before the step. */
dg_status dg_mlp_train_step(dg_mlp m, const float *d_x, const float *d_t, int batch, double lr, double *loss);
/* Add the network's output as a modal source to every stage of h (degree 1,
 * FP32; inputs: the 3 x 4 modes of the element and of its W, E, S, N
 * neighbours, zeros across a pole; the h mode-0 output is shifted so that the
 * total mass is unchanged).  m = NULL detaches.  The network must outlive the
 * attachment. */
dg_status dg_attach_mlp(dg_handle h, dg_mlp m);
/* Make the coarse solver's state the cos(theta)-weighted L2 projection of
 * the fine solver's state (nested meshes: fine nlon = r coarse nlon and fine
 * nlat = r coarse nlat), computed on the GPU in FP64. */
dg_status dg_restrict_from(dg_handle coarse, dg_handle fine);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent meshes of uneven sizes and degrees (the
 * decoupled copies of the 2-D problem of the paper's vertical-levels
 * experiment, Sec. 5.2.2), advanced together in FP32 by one persistent
 * launch per SSP-RK3 stage (Table "Butcher") inside a captured CUDA graph.
 * Each member has its own state (same layout as above), its own time step
 * and its own reference depth; members never interact.
 * ------------------------------------------------------------------------ */
typedef struct dg_ens *dg_ensemble;

/* members >= 1 meshes; member m has nlon[m] x nlat[m] elements of degree
 * degree[m] (0..4).  Allocates all state arrays on the current device. */
dg_status dg_ensemble_create(int members, const int *nlon, const int *nlat, const int *degree, double radius,
                             double g, double omega, dg_ensemble *out);
dg_status dg_ensemble_destroy(dg_ensemble e);
/* DG_OPT_STREAM, DG_OPT_STEPS_PER_GRAPH, DG_OPT_TILE_ROWS, DG_OPT_BLOCKS_PER_SM. */
dg_status dg_ensemble_set_option(dg_ensemble e, int key, long long value);
/* Values in member m's state (0 for a bad member index). */
size_t dg_ensemble_state_len(dg_ensemble e, int member);
/* Values in one state array of the whole ensemble (the ensemble's DOF). */
size_t dg_ensemble_total_dof(dg_ensemble e);
/* Copy member m's modal state in / out (host buffers, layout above). */
dg_status dg_ensemble_set_state(dg_ensemble e, int member, const double *modal, size_t len);
dg_status dg_ensemble_get_state(dg_ensemble e, int member, double *modal, size_t len);
/* One time step per member (dt[m] > 0), used by every following dg_ensemble_step. */
dg_status dg_ensemble_set_dt(dg_ensemble e, const double *dt, int members);
/* n SSP-RK3 steps of every member; reports DG_ENONFINITE / DG_ENONPHYSICAL. */
dg_status dg_ensemble_step(dg_ensemble e, int n);
/* Total mass and CFL time step of member m, as dg_total_mass / dg_max_dt. */
dg_status dg_ensemble_total_mass(dg_ensemble e, int member, double *mass);
dg_status dg_ensemble_max_dt(dg_ensemble e, int member, double cfl, double *dt);
/* Autotuner: times `trials` steps for every tile height (4, 8 rows per CTA)
 * and persistent grid size (1..4 CTAs per SM) on the ensemble's own state
 * (saved and restored), keeps the fastest and returns it, with the time of
 * one step in ms. */
dg_status dg_ensemble_autotune(dg_ensemble e, int trials, int *tile_rows, int *blocks_per_sm, double *best_ms);
/* Persistent stage launches issued so far (one per RK stage). */
long long dg_ensemble_stage_launches(dg_ensemble e);

/* The paper has no counterpart to this entry point.
 * The time step of dg_max_dt for an FP64 state that the caller already holds
 * in device memory (layout as above, full depth h), for callers that cannot
 * allocate device memory and therefore cannot create a handle: code that runs
 * while a CUDA graph is being captured (cudaMalloc is not permitted there), or
 * an application whose own memory manager owns the device and forbids other
 * cudaMalloc calls.  It allocates nothing: its only scratch is one fixed array
 * of DG_NOALLOC_MAX_NLAT + 1 64-bit words (64 KiB) inside the library, which
 * every GPU that loads the library holds until the process exits.  Meshes with
 * more than DG_NOALLOC_MAX_NLAT latitude rows are rejected with DG_EINVAL.
 * The result, dt = cfl H / (max(p,1) c) as for dg_max_dt, or -1 if at some
 * Gauss point h <= 0, h is NaN, or the wave speed is not finite (a NaN or Inf
 * in hu or hv), is written to the device double *d_dt; the work is enqueued on
 * `stream` (a cudaStream_t, NULL = the default stream) and the call returns
 * without waiting.  The first call on a device sets that device up (finds the
 * scratch array's device address and copies a small basis table to constant
 * memory; host threads making that first call together are serialised), so
 * make it before any stream capture begins.  The set-up is kept for the life
 * of the process: after cudaDeviceReset of a device, do not call this entry
 * point on that device again.  All calls share the one scratch array and each
 * call overwrites it: calls whose work overlaps on the GPU (unordered streams)
 * race and can return wrong values. */
#define DG_NOALLOC_MAX_NLAT 8192
dg_status dg_max_dt_noalloc(const double *d_modal, int nlon, int nlat, int degree, double radius, double g,
                            double cfl, double *d_dt, void *stream);

/* Diagnostic of the tensor-core building block: D = A * B1 for one 128-row
 * operand, where B1 is the library's eval/trace matrix of degree `degree`
 * (rows: the (p+1)^2 Gauss points, padded to 8, then the S, N, W, E edge
 * points) rounded to the operand type `op` (0 BF16, 1 FP16).  d_a is device
 * FP32 [128][k1] row-major (rounded to the operand type on the way in), d_out
 * device FP32 [128][n1] row-major; both are caller-owned.  n1 and k1 (host)
 * receive the padded sizes; with d_a or d_out NULL only the sizes are
 * returned.  Synchronous.  DG_ETIMEOUT if the tensor cores did not answer. */
dg_status dg_tc_check_contraction(int degree, int op, const float *d_a, float *d_out, int *n1, int *k1);

/* Measured FP64 arithmetic peak of the current device in GFLOP/s: the best of
 * `reps` timed launches of a kernel of independent double-precision FMA chains
 * over every SM (2 flops per FMA).  The roof of the FP64 stage, which on GB300
 * is bound by FP64 arithmetic rather than by HBM.  Synchronous. */
dg_status dg_measure_fp64_peak(int reps, double *gflops);

/* Number of fused stage-kernel launches issued by this handle so far. */
long long dg_stage_launches(dg_handle h);

/* Message describing the last failing call made by this thread (h may be
 * NULL, e.g. after a failed dg_create); valid until the thread's next call.
 * Never NULL. */
const char *dg_last_error(dg_handle h);

#ifdef __cplusplus
}
#endif

#endif /* DGSWE_H */

// dg_internal.h -- types shared by the translation units of libdgswe.
#pragma once

#include <cstddef>
#include <cstdint>

#define DG_MAXN 5          // up to degree 4: (p+1) <= 5 modes per direction
#define DG_WARPS 8         // warps per stage-kernel block (= tile rows)

// Basis tables of one n = p+1 (n Gauss-Legendre points xi on [-1, 1]):
//   LV[a][q]  = L_a(xi_q)             SE[a] = L_a(+1)      SW[a] = L_a(-1)
//   WLV[a][q] = w_q L_a(xi_q)         WLD[a][q] = w_q L_a'(xi_q)
template <typename T>
struct BasisTab {
    T LV[DG_MAXN][DG_MAXN];
    T WLV[DG_MAXN][DG_MAXN];
    T WLD[DG_MAXN][DG_MAXN];
    T SE[DG_MAXN];
    T SW[DG_MAXN];
};

// Per latitude row j (the element mass matrix depends only on the row):
//   cosn/sinn: cos, sin of theta at the n Gauss points of the row
//   ce_s/ce_n: cos(theta) at the south / north edge (0 at a pole edge)
//   Ci:  inverse of C_j[b][b'] = int L_b L_b' cos(theta(eta)) deta
//   Q:   Ci * WLV, i.e. Q[b][q] = sum_b' Ci[b][b'] w_q L_b'(eta_q)
//   QT, PT: the transposes [q][b] of Q and of Ci * WLD (the beta-pass with
//        the inverse mass matrix folded in, read one Gauss point at a time)
//   CSE, CSW: Ci * L(+1), Ci * L(-1) (north / south lift)
//   rho: hv tendency of the (a = 0, b) modes produced by a unit constant
//        pressure flux (the rest state with g h^2 / 2 = 1), n-point rules
template <typename T>
struct RowTab {
    T cosn[DG_MAXN];
    T sinn[DG_MAXN];
    T ce_s, ce_n;
    T Ci[DG_MAXN][DG_MAXN];
    T Q[DG_MAXN][DG_MAXN];
    T QT[DG_MAXN][DG_MAXN];
    T PT[DG_MAXN][DG_MAXN];
    T CSE[DG_MAXN];
    T CSW[DG_MAXN];
    T rho[DG_MAXN];
};

// Host-side FP64 tables of one mesh.
struct HostTables {
    int n = 0, nm = 0, nlon = 0, nlat = 0;
    double dlam = 0, dth = 0, R = 0;
    double xg[DG_MAXN], wg[DG_MAXN];
    double xm[32], wm[32];
    BasisTab<double> basis;
    RowTab<double> *rows = nullptr;   // nlat entries
    double *C = nullptr;              // nlat * n * n: C_j itself (mass and projection)
};

// dg_tables.cpp
void dg_gauss_legendre(int n, double *x, double *w);
double dg_legendre(int k, double x);
double dg_legendre_deriv(int k, double x);
int dg_build_tables(HostTables &t, int nlon, int nlat, int p, double R, double g);
void dg_free_tables(HostTables &t);

// Stage-kernel launch description.  The time integration is written in
// increment form: the state u^n is held as (base, lo) -- lo carries the bits
// that do not fit into base (FP32 path; null in FP64) -- and every stage
// state is u^n + inc.  One fused kernel computes k = M^{-1} h(u_stage),
// u_stage = base + inc (inc may be null), and then, as requested:
//   out_rhs  = k                                              (tendency only)
//   inc_out  = ci * inc + cc * dt * k                         (next increment)
//   acc_out  = acc_in + ca * dt * k                           (RK4 accumulator)
//   (out_base, out_lo) = (base, lo) + ci * inc + cd * acc_in + cc * dt * k
//                         (final stage, error-free two-sum update of u^n)
template <typename T>
struct StageArgs {
    const T *base;
    const T *inc;
    const T *lo;
    const T *acc_in;
    T *out_rhs;
    T *inc_out;
    T *acc_out;
    T *out_base;
    T *out_lo;
    const T *src;    // optional modal source added to k (learned correction)
    const T *galpha; // global Rusanov mode: [max |u| + c, max |v| + c] of the stage input; null = local
    const RowTab<T> *rows;
    unsigned int *status;
    int nlon, nlat;
    // latitude-band sharding: 1 when the row south of row 0 (halo_s) or north
    // of row nlat - 1 (halo_n) is a neighbour band's row, held in the state
    // arrays just before / after the band's own rows, instead of a pole
    int halo_s, halo_n;
    T href;          // reference depth: h = href + stored h
    T P0;            // g href^2 / 2 (pressure carried by the rho table)
    T g, cF, cG, invR, twoOmega;
    T ci, ca, cc, cd, dt;
};

// Batched ensemble: the members' states are concatenated in every state
// array; one persistent launch per stage walks a work list of tiles.
template <typename T>
struct EnsMember {
    long long off;   // offset of the member's first value in the state arrays
    int rows;        // index of the member's first row table
    int nlon, nlat, n;
    T href, P0, cF, cG, dt;
};

struct EnsItem {
    int member, tx, ty, cost;
};

template <typename T>
struct EnsArgs {
    const T *base, *inc, *lo, *acc_in;
    T *out_rhs, *inc_out, *acc_out, *out_base, *out_lo;
    const RowTab<T> *rows;
    const EnsMember<T> *members;
    const EnsItem *items;
    int nitems;
    unsigned int *status;
    T g, invR, twoOmega;
    T ci, ca, cc, cd;
};

// tile rows (warps per CTA) the ensemble kernel is built for
#define DG_ENS_TILE_ROWS_A 4
#define DG_ENS_TILE_ROWS_B 8

template <typename T>
int dg_launch_ensemble_stage(int tile_rows, int grid, const EnsArgs<T> &a, void *stream);
int dg_ensemble_tile_width(int n);   // elements per warp for degree n - 1

// status bits written by device code
#define DG_STATUS_NONPHYSICAL 1u
#define DG_STATUS_NONFINITE 2u
#define DG_STATUS_TIMEOUT 4u      // a bounded wait on the tensor cores gave up

template <typename T>
int dg_launch_stage(int n, const StageArgs<T> &a, void *stream);
template <typename T>
int dg_upload_basis(const BasisTab<double> *all);   // all[n-1] for n = 1..DG_MAXN

// dg_tc.cu: the stage with the basis contractions on the tensor cores
// (tcgen05; op 0 = BF16, 1 = FP16 operands, FP32 accumulation).  The state
// arrays are in the lane-contiguous layout [lat][field][mode][lon].
int dg_launch_stage_tc(int n, int op, const StageArgs<float> &a, void *stream);
// Upload the tensor-core tables of (n, op) and set the kernel's shared-memory
// opt-in on the current device (outside any stream capture); 0 on success.
int dg_prepare_stage_tc(int n, int op);
// [lat][lon][field][mode] <-> [lat][field][mode][lon] (to_lanes = 1: first to second)
int dg_launch_permute(const float *src, float *dst, int nlat, int nlon, int el, int to_lanes, void *stream);
// tensor-core contraction check: D = A * B1 for a 128-row operand A
// (row-major [128][K1]) with the degree's eval/trace matrix; d is [128][N1]
// row-major in FP32, and n1 / k1 receive the padded sizes.
int dg_tc_gemm_check(int n, int op, const float *a, float *d, int *n1, int *k1, void *stream);

// dg_aux.cu
// FP64 API layout <-> internal (base, lo) with h stored relative to href; lo
// may be null (FP64 path).
template <typename T>
int dg_launch_to_internal(const double *src, T *dst, T *lo, size_t nel, int nphi, double href, void *stream);
template <typename T>
int dg_launch_to_api(const T *src, const T *lo, double *dst, size_t nel, int nphi, double href, void *stream);
// result (may be null): scale * (sum + correction); pair (may be null): the
// unscaled compensated pair (sum, correction) itself.
template <typename T>
int dg_launch_mass(const T *u, const T *lo, const double *c0, int nlon, int nlat, int n, double href,
                   double dlam, double dth, double scale, double *partials, int nblocks, double *result,
                   double *pair, void *stream);
// Global Rusanov speeds of the stage state base + inc (inc may be null): the
// maxima of |u| + sqrt(g h) and |v| + sqrt(g h) over all Gauss points, as the
// bits of T atomically maxed into out[0], out[1] (zero them first).  lanes:
// the state is [lat][field][mode][lon] instead of [lat][lon][field][mode].
template <typename T>
int dg_launch_global_speeds(int n, const T *base, const T *inc, int nlon, int nlat, int lanes, T href, T g, T *out,
                            void *stream);
template <typename T>
int dg_launch_max_speed(const T *u, int nlon, int nlat, int n, double href, double g,
                        unsigned long long *maxbits, unsigned int *status, void *stream);
int dg_mass_blocks(size_t nel);

// dg_restrict.cu: nested fine -> coarse projection
struct RestrictTab {
    double x[8], w[8];            // 8-point Gauss rule on [-1, 1]
    double LVf[DG_MAXN][8];       // fine basis L_a at the points
    double jf;                    // fine element Jacobian (dlam_f / 2)(dth_f / 2)
    double dthc;                  // coarse dtheta
    double inv_jc;                // 4 / (dlam_c dth_c)
};
int dg_launch_restrict(const double *fine, int fnlon, int fn, double *coarse, int cnlon, int cnlat, int cn, int r,
                       const RowTab<double> *crows, const RestrictTab &tab, void *stream);

// dg_mlp.cu: the learned source term of a degree-1 solver
struct dg_mlp_ctx;
int dg_mlp_launch_source(const dg_mlp_ctx *m, const float *base, const float *inc, float href, int nlon, int nlat,
                         const double *c0, float *src, void *stream);
bool dg_mlp_shape_is(const dg_mlp_ctx *m, int nin, int h, int nout);

// dg_plane.cu: planar linear advection (one scalar, periodic unit square)
// and planar shallow water on the f-plane (h, hu, hv; periodic square).
// k = M^{-1} h(u) with the FP64 stage semantics of StageArgs (href, rows, lo
// unused); cx = 2 / dx, cy = 2 / dy; alpha_speed 1: Rusanov alpha = |beta|,
// 0: |beta . n|.
struct PlaneArgs {
    StageArgs<double> s;
    BasisTab<double> basis;
    double bx, by, cx, cy;
    int nx, ny, alpha_speed;
    int swe;          // 1: shallow water on the f-plane (3 fields) instead of advection
    double g, fcor;   // gravity and the constant Coriolis parameter (swe)
};
int dg_launch_stage_plane(int n, const PlaneArgs &p, void *stream);

// dg_probe.cu: measured FP64 FMA rate of the current device (GFLOP/s).
int dg_probe_fp64_gflops(int reps, double *gflops);

// dg_api.cpp: set the calling thread's message returned by dg_last_error().
void dg_set_last_error(const char *msg);
// dg_api.cpp: make sure the constant basis tables are on device `device`
// (0 on success).
int dg_ensure_basis(int device);

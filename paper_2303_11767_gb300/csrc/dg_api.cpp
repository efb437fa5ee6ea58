// dg_api.cpp -- the C-ABI of libdgswe (declared in include/dgswe.h).
//
// The handle owns the FP64 host tables, the device buffers of the resident
// state, the stream and the captured CUDA graphs of the Runge-Kutta steps.
// Every time step is a fixed sequence of fused stage kernels (one per RK
// stage, Table "Butcher" of the paper), captured once per (steps, dt, order,
// precision) and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.h"
#include "../../include/dgswe.h"

namespace {

thread_local std::string g_err;

dg_status fail(dg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(call)                                                                                       \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return fail(DG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int steps = 0, order = 0, prec = 0, cur_in = 0, cur_out = 0;
    double dt = 0;
    cudaStream_t stream = nullptr;
};

unsigned long long g_basis_uploaded = 0;   // per-device bit: constant tables present

}  // namespace

struct dg_ctx {
    int physics = 0;   // 0: shallow water on the sphere; 1: planar linear advection; 2: planar shallow water
    int nlon = 0, nlat = 0, p = 0, n = 0, nphi = 0;
    size_t nel = 0, len = 0;
    double R = 0, g = 0, omega = 0;
    int device = 0;
    HostTables tab;
    // options
    int prec = DG_PREC_FP64, rk = 3, check = 1, alpha_mode = 0, spg = 16;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    // device buffers of the active precision (increment-form time stepping)
    void *B[2] = {nullptr, nullptr};   // u^n, ping-pong: the last stage writes the other one
    void *L[2] = {nullptr, nullptr};   // low parts of u^n (FP32 path only)
    void *I[2] = {nullptr, nullptr};   // stage increments u_s - u^n
    void *D = nullptr;                 // RK4 accumulator
    // tensor-core precisions: u^n in the lane-contiguous layout while stepping
    void *SB[2] = {nullptr, nullptr};
    void *SL[2] = {nullptr, nullptr};
    int cur = 0;                       // index of B / L holding u^n
    double *stage64 = nullptr;                            // FP64 staging of one state
    RowTab<double> *rows64 = nullptr;
    RowTab<float> *rows32 = nullptr;
    double *c0 = nullptr;                                 // mass table: C_j[0][b], then row areas
    double *partials = nullptr;                           // per-block compensated mass sums
    int nblocks = 0;
    double *d_result = nullptr;
    unsigned *d_status = nullptr;
    unsigned long long *d_maxbits = nullptr;
    void *galpha = nullptr;   // global Rusanov mode: the stage's two speeds (2 values of T)
    double href = 0;      // reference depth of the resident state (FP32 path, or well balanced); else 0
    int wb = 0;           // well-balanced option: the rest state at href is exactly steady
    double t = 0;
    bool have_state = false;
    long long launches = 0;       // fused stage kernels
    long long aux_launches = 0;   // conversion, mass and wave-speed kernels
    dg_mlp_ctx *mlp = nullptr;    // learned source term (degree 1, FP32)
    float *src = nullptr;         // its per-stage modal output
    std::vector<GraphEntry> graphs;
    double bx = 0, by = 0;       // planar advection velocity
    double plen = 1.0, fcor = 0; // planar domain side and f-plane Coriolis parameter
    int alpha_speed = 0;         // planar: Rusanov alpha = |beta| (1) or |beta . n| (0)
    BasisTab<double> pbasis{};   // planar: basis tables of degree p
    // latitude band of a larger mesh (dg_create_band): the own rows are rows
    // [j0, j0 + nlat) of a mesh of nlat_g rows; every state array holds, when
    // gs / gn, one ghost row (a neighbour band's row) just before / after them
    int band = 0, j0 = 0, nlat_g = 0, gs = 0, gn = 0;
    size_t ghost_bytes = 0;    // byte offset of own row 0 in each state allocation
    int band_stage = 0;        // the next stage of the current step
    double band_dt = 0;        // step size of the current step
    int href_fixed = 0;        // reference depth given by dg_band_set_reference_depth
    double href_given = 0;
    size_t row_len() const { return (size_t)nlon * 3 * nphi; }
    bool f32() const { return prec != DG_PREC_FP64; }                 // FP32 storage
    bool tc() const { return prec >= DG_PREC_FP32_TC_BF16 && prec <= DG_PREC_FP32_TC_FP16_SPLIT; }
};

namespace {

size_t elem_size(int prec) { return prec == DG_PREC_FP64 ? sizeof(double) : sizeof(float); }

void drop_graphs(dg_ctx *h)
{
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

void free_state_buffers(dg_ctx *h)
{
    void **all[] = {&h->B[0], &h->B[1], &h->L[0], &h->L[1], &h->I[0], &h->I[1], &h->D,
                    &h->SB[0], &h->SB[1], &h->SL[0], &h->SL[1]};
    for (void **u : all) {
        if (*u) cudaFree(static_cast<char *>(*u) - h->ghost_bytes);
        *u = nullptr;
    }
}

dg_status alloc_state_buffers(dg_ctx *h)
{
    // a band's arrays carry its ghost rows around the own rows; the pointers
    // kept point at own row 0.  The length is rounded up to 16 bytes: the
    // stage kernel copies halo elements in whole 16-byte blocks.
    const size_t es = elem_size(h->prec);
    const size_t bytes = ((h->len + (size_t)(h->gs + h->gn) * h->row_len()) * es + 15) / 16 * 16;
    h->ghost_bytes = (size_t)h->gs * h->row_len() * es;
    std::vector<void **> want = {&h->B[0], &h->B[1], &h->I[0], &h->I[1], &h->D};
    if (h->f32()) {
        want.push_back(&h->L[0]);
        want.push_back(&h->L[1]);
    }
    if (h->tc()) {
        for (int k = 0; k < 2; ++k) {
            want.push_back(&h->SB[k]);
            want.push_back(&h->SL[k]);
        }
    }
    for (void **u : want) {
        if (cudaMalloc(u, bytes) != cudaSuccess) {
            *u = nullptr;
            free_state_buffers(h);
            return fail(DG_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
        if (h->band && cudaMemset(*u, 0, bytes) != cudaSuccess) {   // ghost rows start at zero
            cudaFree(*u);
            *u = nullptr;
            free_state_buffers(h);
            return fail(DG_ECUDA, "cudaMemset failed");
        }
        *u = static_cast<char *>(*u) + h->ghost_bytes;
    }
    return DG_OK;
}

// Stage launch in the active precision.
template <typename T>
StageArgs<T> base_args(dg_ctx *h, const RowTab<T> *rows, double href)
{
    StageArgs<T> a;
    std::memset(&a, 0, sizeof a);
    a.rows = rows;
    a.status = h->d_status;
    a.nlon = h->nlon;
    a.nlat = h->nlat;
    a.halo_s = h->gs;
    a.halo_n = h->gn;
    a.href = (T)href;
    // the pressure of the rest state at href enters through the per-row
    // vector rho; the well-balanced option drops it (that state is steady)
    a.P0 = h->wb ? T(0) : (T)(0.5 * h->g * href * href);
    a.g = (T)h->g;
    a.cF = (T)(2.0 / (h->R * h->tab.dlam));
    a.cG = (T)(2.0 / (h->R * h->tab.dth));
    a.invR = (T)(1.0 / h->R);
    a.twoOmega = (T)(2.0 * h->omega);
    return a;
}

// One stage of the increment-form RK step.  inc_in / inc_out index I[],
// -1 = none; acc_in / acc_out use D; fin = last stage (updates u^n into the
// other base buffer).
struct StagePlan {
    int inc_in, inc_out, acc_in, acc_out, fin;
    double ci, ca, cc, cd;
};

// The explicit RK schemes of Table "Butcher" in increment form: every stage
// state is u^n + inc, and the last stage adds
//   u^{n+1} - u^n = sum_s b_s dt k_s
// to u^n once, with a two-sum.  SSP RK3: inc1 = dt k1, inc2 = (inc1 + dt k2)/4,
// u^{n+1} = u^n + 2/3 (inc2 + dt k3) (the Shu-Osher stages minus u^n).
int rk_plan(int order, StagePlan *pl)
{
    switch (order) {
    case 1:
        pl[0] = {-1, -1, -1, -1, 1, 0, 0, 1, 0};
        return 1;
    case 2:
        pl[0] = {-1, 0, -1, -1, 0, 0, 0, 1, 0};
        pl[1] = {0, -1, -1, -1, 1, 0.5, 0, 0.5, 0};
        return 2;
    case 3:
        pl[0] = {-1, 0, -1, -1, 0, 0, 0, 1, 0};
        pl[1] = {0, 1, -1, -1, 0, 0.25, 0, 0.25, 0};
        pl[2] = {1, -1, -1, -1, 1, 2.0 / 3.0, 0, 2.0 / 3.0, 0};
        return 3;
    case 4:   // classical tableau: stages u + dt k1/2, u + dt k2/2, u + dt k3
        pl[0] = {-1, 0, -1, 1, 0, 0, 1.0 / 6.0, 0.5, 0};
        pl[1] = {0, 1, 1, 1, 0, 0, 1.0 / 3.0, 0.5, 0};
        pl[2] = {1, 0, 1, 1, 0, 0, 1.0 / 3.0, 1.0, 0};
        pl[3] = {0, -1, 1, -1, 1, 0, 0, 1.0 / 6.0, 1.0};
        return 4;
    default:
        return 0;
    }
}

// Planar advection stage with the FP64 stage semantics of `a`.
int launch_plane(dg_ctx *h, const StageArgs<double> &a)
{
    PlaneArgs pa;
    pa.s = a;
    pa.basis = h->pbasis;
    pa.bx = h->bx;
    pa.by = h->by;
    pa.cx = 2.0 * h->nlon / h->plen;   // 2 / dx on the square of side plen
    pa.cy = 2.0 * h->nlat / h->plen;
    pa.nx = h->nlon;
    pa.ny = h->nlat;
    pa.alpha_speed = h->alpha_speed;
    pa.swe = h->physics == 2;
    pa.g = h->g;
    pa.fcor = h->fcor;
    return dg_launch_stage_plane(h->n, pa, h->stream);
}

dg_status planar_unsupported(dg_ctx *h, const char *what)
{
    (void)h;
    return fail(DG_EUNSUPPORTED, "%s is not available for the planar problems", what);
}

// Global Rusanov mode: the stage input's two speeds into h->galpha, then the
// stage reads them (a.galpha).
template <typename T>
dg_status enqueue_global_speeds(dg_ctx *h, StageArgs<T> &a)
{
    if (!h->alpha_mode) return DG_OK;
    if (cudaMemsetAsync(h->galpha, 0, 2 * sizeof(T), h->stream) != cudaSuccess ||
        dg_launch_global_speeds<T>(h->n, a.base, a.inc, h->nlon, h->nlat, h->tc() ? 1 : 0, a.href, a.g,
                                   static_cast<T *>(h->galpha), h->stream))
        return fail(DG_ECUDA, "global speed kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    a.galpha = static_cast<const T *>(h->galpha);
    h->aux_launches += 1;
    return DG_OK;
}

// Stage s of one RK step from u^n in base buffer `cur`.
template <typename T>
dg_status launch_stage_t(dg_ctx *h, double dt, int cur, const RowTab<T> *rows, int s)
{
    StagePlan pl[4];
    rk_plan(h->rk, pl);
    auto I = [&](int i) -> T * { return i < 0 ? nullptr : static_cast<T *>(h->I[i]); };
    {
        StageArgs<T> a = base_args<T>(h, rows, h->href);
        a.inc = I(pl[s].inc_in);
        a.inc_out = I(pl[s].inc_out);
        a.acc_in = pl[s].acc_in >= 0 ? static_cast<const T *>(h->D) : nullptr;
        a.acc_out = pl[s].acc_out >= 0 ? static_cast<T *>(h->D) : nullptr;
        void *const *Bv = h->tc() ? h->SB : h->B;
        void *const *Lv = h->tc() ? h->SL : h->L;
        a.base = static_cast<const T *>(Bv[cur]);
        if (pl[s].fin) {
            a.lo = static_cast<const T *>(Lv[cur]);
            a.out_base = static_cast<T *>(Bv[cur ^ 1]);
            a.out_lo = static_cast<T *>(Lv[cur ^ 1]);
        }
        a.ci = (T)pl[s].ci;
        a.ca = (T)pl[s].ca;
        a.cc = (T)pl[s].cc;
        a.cd = (T)pl[s].cd;
        a.dt = (T)dt;
        if constexpr (sizeof(T) == sizeof(float)) {
            if (h->mlp) {
                const int ms = dg_mlp_launch_source(h->mlp, reinterpret_cast<const float *>(a.base),
                                                    reinterpret_cast<const float *>(a.inc), (float)h->href, h->nlon,
                                                    h->nlat, h->c0, h->src, h->stream);
                if (ms == 2) return fail(DG_EINVAL, "the network's row statistics belong to another mesh");
                if (ms)
                    return fail(DG_ECUDA, "learned source launch failed: %s", cudaGetErrorString(cudaGetLastError()));
                a.src = reinterpret_cast<const T *>(h->src);
                h->aux_launches += 2;
            }
        }
        if (dg_status gs = enqueue_global_speeds<T>(h, a)) return gs;
        int r;
        if constexpr (sizeof(T) == sizeof(float)) {
            r = h->tc() ? dg_launch_stage_tc(h->n, h->prec - DG_PREC_FP32_TC_BF16, a, h->stream)
                        : dg_launch_stage<T>(h->n, a, h->stream);
        } else {
            r = h->physics != 0 ? launch_plane(h, a) : dg_launch_stage<T>(h->n, a, h->stream);
        }
        if (r) return fail(DG_ECUDA, "stage kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        h->launches++;
    }
    return DG_OK;
}

template <typename T>
dg_status launch_step_t(dg_ctx *h, double dt, int cur, const RowTab<T> *rows)
{
    StagePlan pl[4];
    const int ns = rk_plan(h->rk, pl);
    for (int s = 0; s < ns; ++s)
        if (dg_status st = launch_stage_t<T>(h, dt, cur, rows, s)) return st;
    return DG_OK;
}

// Tensor-core precisions: u^n (base and low parts) between the element-major
// layout of the API-side kernels and the lane-contiguous one of the stage.
dg_status permute_state(dg_ctx *h, int idx, int to_lanes)
{
    const int el = 3 * h->nphi;
    float *B = static_cast<float *>(h->B[idx]), *L = static_cast<float *>(h->L[idx]);
    float *SB = static_cast<float *>(h->SB[idx]), *SL = static_cast<float *>(h->SL[idx]);
    int r = to_lanes ? (dg_launch_permute(B, SB, h->nlat, h->nlon, el, 1, h->stream) ||
                        dg_launch_permute(L, SL, h->nlat, h->nlon, el, 1, h->stream))
                     : (dg_launch_permute(SB, B, h->nlat, h->nlon, el, 0, h->stream) ||
                        dg_launch_permute(SL, L, h->nlat, h->nlon, el, 0, h->stream));
    if (r) return fail(DG_ECUDA, "layout permutation failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->aux_launches += 2;
    return DG_OK;
}

dg_status launch_steps(dg_ctx *h, int nsteps, double dt, int *cur)
{
    for (int s = 0; s < nsteps; ++s) {
        dg_status st = h->prec == DG_PREC_FP64 ? launch_step_t<double>(h, dt, *cur, h->rows64)
                                               : launch_step_t<float>(h, dt, *cur, h->rows32);
        if (st) return st;
        *cur ^= 1;   // u^{n+1} lives in the other base buffer
    }
    return DG_OK;
}

dg_status read_status(dg_ctx *h)
{
    unsigned st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (st) {
        CUDA_TRY(cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
        if (st & DG_STATUS_TIMEOUT) return fail(DG_ETIMEOUT, "a bounded wait for the tensor cores gave up");
        if (st & DG_STATUS_NONPHYSICAL) return fail(DG_ENONPHYSICAL, "h <= 0 at a quadrature point");
        return fail(DG_ENONFINITE, "non-finite value in the state");
    }
    return DG_OK;
}

dg_status check(dg_ctx *h)
{
    if (!h) return fail(DG_EINVAL, "NULL handle");
    return DG_OK;
}

template <typename T>
dg_status upload_rows(dg_ctx *h, RowTab<T> **dst)
{
    std::vector<RowTab<T>> r(h->nlat);
    for (int j = 0; j < h->nlat; ++j) {
        const RowTab<double> &s = h->tab.rows[j];
        RowTab<T> &d = r[j];
        std::memset(&d, 0, sizeof d);
        for (int a = 0; a < DG_MAXN; ++a) {
            d.cosn[a] = (T)s.cosn[a];
            d.sinn[a] = (T)s.sinn[a];
            d.rho[a] = (T)s.rho[a];
            d.CSE[a] = (T)s.CSE[a];
            d.CSW[a] = (T)s.CSW[a];
            for (int b = 0; b < DG_MAXN; ++b) {
                d.Ci[a][b] = (T)s.Ci[a][b];
                d.Q[a][b] = (T)s.Q[a][b];
                d.QT[a][b] = (T)s.QT[a][b];
                d.PT[a][b] = (T)s.PT[a][b];
            }
        }
        d.ce_s = (T)s.ce_s;
        d.ce_n = (T)s.ce_n;
    }
    const size_t bytes = sizeof(RowTab<T>) * h->nlat;
    if (cudaMalloc(reinterpret_cast<void **>(dst), bytes) != cudaSuccess)
        return fail(DG_ENOMEM, "cudaMalloc of row tables failed");
    CUDA_TRY(cudaMemcpy(*dst, r.data(), bytes, cudaMemcpyHostToDevice));
    return DG_OK;
}

dg_status upload_basis_once(int dev)
{
    if (g_basis_uploaded >> dev & 1ull) return DG_OK;
    BasisTab<double> all[DG_MAXN];
    for (int n = 1; n <= DG_MAXN; ++n) {
        HostTables t;
        if (dg_build_tables(t, 1, 2, n - 1, 1.0, 1.0)) {
            dg_free_tables(t);
            return fail(DG_EINVAL, "basis table construction failed");
        }
        all[n - 1] = t.basis;
        dg_free_tables(t);
    }
    if (dg_upload_basis<float>(all) || dg_upload_basis<double>(all))
        return fail(DG_ECUDA, "upload of the basis tables failed: %s", cudaGetErrorString(cudaGetLastError()));
    g_basis_uploaded |= 1ull << dev;
    return DG_OK;
}

double mean_depth(const double *modal, size_t nel, int nphi)
{
    double s = 0.0;
    for (size_t e = 0; e < nel; ++e) s += modal[e * 3 * nphi];
    return 0.5 * s / (double)nel;   // mode 0 of h times phi_0 = 1/2
}

dg_status to_internal(dg_ctx *h, const double *d_src, void *dst, void *lo, double href)
{
    int r = h->prec == DG_PREC_FP64
                ? dg_launch_to_internal<double>(d_src, static_cast<double *>(dst), static_cast<double *>(lo), h->nel,
                                                h->nphi, href, h->stream)
                : dg_launch_to_internal<float>(d_src, static_cast<float *>(dst), static_cast<float *>(lo), h->nel,
                                               h->nphi, href, h->stream);
    if (r) return fail(DG_ECUDA, "conversion kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
}

dg_status to_api(dg_ctx *h, const void *src, const void *lo, double *d_dst, double href)
{
    int r = h->prec == DG_PREC_FP64
                ? dg_launch_to_api<double>(static_cast<const double *>(src), static_cast<const double *>(lo), d_dst,
                                           h->nel, h->nphi, href, h->stream)
                : dg_launch_to_api<float>(static_cast<const float *>(src), static_cast<const float *>(lo), d_dst,
                                          h->nel, h->nphi, href, h->stream);
    if (r) return fail(DG_ECUDA, "conversion kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_set_device(int device)
{
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) return fail(DG_ECUDA, "no CUDA device");
    if (device < 0 || device >= count) return fail(DG_EINVAL, "device %d of %d", device, count);
    CUDA_TRY(cudaSetDevice(device));
    return DG_OK;
}

}  // extern "C"

namespace {

// A solver for rows [jb, je) of an nlon x nlat_g sphere mesh: the whole mesh
// (dg_create) or one latitude band of it (dg_create_band).
dg_status create_sphere(int nlon, int nlat_g, int jb, int je, int degree, double radius, double g, double omega,
                        dg_handle *out)
{
    if (!out) return fail(DG_EINVAL, "out is NULL");
    *out = nullptr;
    if (nlon < 1 || nlat_g < 2) return fail(DG_EINVAL, "need nlon >= 1 and nlat >= 2 (got %d, %d)", nlon, nlat_g);
    if (jb < 0 || je > nlat_g || je <= jb) return fail(DG_EINVAL, "band rows [%d, %d) outside [0, %d)", jb, je, nlat_g);
    if (degree < 0 || degree > DG_MAXN - 1) return fail(DG_EINVAL, "degree must be in [0, %d]", DG_MAXN - 1);
    if (!(radius > 0) || !(g > 0) || !std::isfinite(omega))
        return fail(DG_EINVAL, "radius and g must be positive, omega finite");
    if ((double)nlon * nlat_g > 2.0e9) return fail(DG_EINVAL, "mesh too large");
    dg_ctx *h = new (std::nothrow) dg_ctx;
    if (!h) return fail(DG_ENOMEM, "host allocation failed");
    const int nlat = je - jb;
    h->band = (jb > 0 || je < nlat_g) ? 1 : 0;
    h->j0 = jb;
    h->nlat_g = nlat_g;
    h->gs = jb > 0 ? 1 : 0;
    h->gn = je < nlat_g ? 1 : 0;
    h->nlon = nlon;
    h->nlat = nlat;
    h->p = degree;
    h->n = degree + 1;
    h->nphi = h->n * h->n;
    h->nel = (size_t)nlon * nlat;
    h->len = h->nel * 3 * h->nphi;
    h->R = radius;
    h->g = g;
    h->omega = omega;
    dg_status st = DG_OK;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(DG_ECUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (dg_build_tables(h->tab, nlon, nlat_g, degree, radius, g)) {
        dg_free_tables(h->tab);
        delete h;
        return fail(DG_EINVAL, "table construction failed");
    }
    if (h->band) {   // keep the own rows' tables (built for the whole mesh), first at index 0
        std::memmove(h->tab.rows, h->tab.rows + jb, sizeof(RowTab<double>) * nlat);
        std::memmove(h->tab.C, h->tab.C + (size_t)jb * h->nphi, sizeof(double) * (size_t)nlat * h->nphi);
        h->tab.nlat = nlat;
    }
#define CREATE_TRY(x)                 \
    do {                              \
        st = (x);                     \
        if (st) {                     \
            dg_destroy(h);            \
            return st;                \
        }                             \
    } while (0)
    CREATE_TRY(upload_basis_once(h->device));
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ECUDA, "stream creation failed");
    }
    h->stream = h->own_stream;
    CREATE_TRY(alloc_state_buffers(h));
    if (cudaMalloc(&h->stage64, h->len * sizeof(double)) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ENOMEM, "cudaMalloc of the staging buffer failed");
    }
    CREATE_TRY(upload_rows<double>(h, &h->rows64));
    CREATE_TRY(upload_rows<float>(h, &h->rows32));
    {
        std::vector<double> c0((size_t)nlat * h->n + nlat);
        for (int j = 0; j < nlat; ++j) {
            for (int b = 0; b < h->n; ++b) c0[(size_t)j * h->n + b] = h->tab.C[(size_t)j * h->nphi + b];
            const double tb = -0.5 * M_PI + (h->j0 + j) * h->tab.dth;
            c0[(size_t)nlat * h->n + j] = std::sin(tb + h->tab.dth) - std::sin(tb);
        }
        if (cudaMalloc(&h->c0, c0.size() * sizeof(double)) != cudaSuccess) {
            dg_destroy(h);
            return fail(DG_ENOMEM, "cudaMalloc failed");
        }
        if (cudaMemcpy(h->c0, c0.data(), c0.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            dg_destroy(h);
            return fail(DG_ECUDA, "copy of the mass table failed");
        }
    }
    h->nblocks = dg_mass_blocks(h->nel);
    if (cudaMalloc(&h->partials, 2 * sizeof(double) * (h->nblocks + 1)) != cudaSuccess ||   // + the pair
        cudaMalloc(&h->d_result, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&h->d_maxbits, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&h->galpha, 2 * sizeof(double)) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ENOMEM, "cudaMalloc failed");
    }
    if (cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ECUDA, "cudaMemset failed");
    }
#undef CREATE_TRY
    *out = h;
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_create(int nlon, int nlat, int degree, double radius, double g, double omega, dg_handle *out)
{
    return create_sphere(nlon, nlat, 0, nlat, degree, radius, g, omega, out);
}

dg_status dg_create_band(int nlon, int nlat, int j_begin, int j_end, int degree, double radius, double g,
                         double omega, dg_handle *out)
{
    return create_sphere(nlon, nlat, j_begin, j_end, degree, radius, g, omega, out);
}

dg_status dg_create_plane_swe(int nx, int ny, int degree, double L, double g, double f, dg_handle *out)
{
    if (!(L > 0) || !(g > 0) || !std::isfinite(f) || !std::isfinite(L))
        return fail(DG_EINVAL, "need L > 0, g > 0 and a finite f");
    dg_status st = dg_create_plane_advection(nx, ny, degree, 0.0, 0.0, 0, out);
    if (st) return st;
    dg_ctx *h = *out;
    DeviceGuard dg(h->device);
    // three fields: re-size the state buffers
    free_state_buffers(h);
    h->physics = 2;
    h->len = h->nel * 3 * h->nphi;
    h->plen = L;
    h->g = g;
    h->fcor = f;
    if ((st = alloc_state_buffers(h)) != DG_OK) {
        dg_destroy(h);
        *out = nullptr;
        return st;
    }
    return DG_OK;
}

dg_status dg_create_plane_advection(int nx, int ny, int degree, double bx, double by, int alpha_speed,
                                    dg_handle *out)
{
    if (!out) return fail(DG_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1) return fail(DG_EINVAL, "need nx, ny >= 1 (got %d, %d)", nx, ny);
    if (degree < 0 || degree > DG_MAXN - 1) return fail(DG_EINVAL, "degree must be in [0, %d]", DG_MAXN - 1);
    if (!std::isfinite(bx) || !std::isfinite(by)) return fail(DG_EINVAL, "beta must be finite");
    if (alpha_speed != 0 && alpha_speed != 1) return fail(DG_EINVAL, "alpha_speed must be 0 or 1");
    if ((double)nx * ny > 2.0e9) return fail(DG_EINVAL, "mesh too large");
    dg_ctx *h = new (std::nothrow) dg_ctx;
    if (!h) return fail(DG_ENOMEM, "host allocation failed");
    h->physics = 1;
    h->nlon = nx;
    h->nlat = ny;
    h->p = degree;
    h->n = degree + 1;
    h->nphi = h->n * h->n;
    h->nel = (size_t)nx * ny;
    h->len = h->nel * h->nphi;
    h->R = 1.0;
    h->bx = bx;
    h->by = by;
    h->alpha_speed = alpha_speed;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(DG_ECUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
    }
    {
        HostTables t;
        if (dg_build_tables(t, 1, 2, degree, 1.0, 1.0)) {
            dg_free_tables(t);
            delete h;
            return fail(DG_EINVAL, "basis table construction failed");
        }
        h->pbasis = t.basis;
        dg_free_tables(t);
        h->tab.n = h->n;
        h->tab.nm = degree + 9;
        dg_gauss_legendre(h->tab.nm, h->tab.xm, h->tab.wm);
    }
    dg_status st = DG_OK;
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ECUDA, "stream creation failed");
    }
    h->stream = h->own_stream;
    if ((st = alloc_state_buffers(h)) != DG_OK) {
        dg_destroy(h);
        return st;
    }
    if (cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        dg_destroy(h);
        return fail(DG_ENOMEM, "cudaMalloc failed");
    }
    *out = h;
    return DG_OK;
}

dg_status dg_destroy(dg_handle h)
{
    if (!h) return DG_OK;
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    free_state_buffers(h);
    cudaFree(h->stage64);
    cudaFree(h->rows64);
    cudaFree(h->rows32);
    cudaFree(h->c0);
    cudaFree(h->partials);
    cudaFree(h->d_result);
    cudaFree(h->d_status);
    cudaFree(h->d_maxbits);
    cudaFree(h->galpha);
    cudaFree(h->src);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    dg_free_tables(h->tab);
    delete h;
    return DG_OK;
}

size_t dg_state_len(dg_handle h) { return h ? h->len : 0; }

long long dg_stage_launches(dg_handle h) { return h ? h->launches : 0; }

const char *dg_last_error(dg_handle) { return g_err.c_str(); }

dg_status dg_set_option(dg_handle h, int key, long long value)
{
    if (dg_status s = check(h)) return s;
    DeviceGuard dg(h->device);
    if (h->physics != 0 && ((key == DG_OPT_PRECISION && value != DG_PREC_FP64) || (key == DG_OPT_ALPHA_MODE && value) ||
                            (key == DG_OPT_WELL_BALANCED && value)))
        return planar_unsupported(h, key == DG_OPT_PRECISION ? "a precision other than FP64"
                                     : key == DG_OPT_ALPHA_MODE ? "the global alpha mode"
                                                                : "the well-balanced option");
    if (h->band && ((key == DG_OPT_PRECISION && value >= DG_PREC_FP32_TC_BF16) ||
                    (key == DG_OPT_ALPHA_MODE && value)))
        return fail(DG_EUNSUPPORTED, "a latitude band supports the FP64 and FP32 stages with the local Rusanov alpha");
    switch (key) {
    case DG_OPT_PRECISION: {
        if (value < DG_PREC_FP64 || value > DG_PREC_FP32_TC_FP16_SPLIT)
            return fail(DG_EINVAL, "unknown precision %lld", value);
        if (value >= DG_PREC_FP32_TC_BF16 && dg_prepare_stage_tc(h->n, (int)(value - DG_PREC_FP32_TC_BF16)))
            return fail(DG_ECUDA, "tensor-core tables: %s", cudaGetErrorString(cudaGetLastError()));
        if (value == h->prec) return DG_OK;
        if (h->mlp) return fail(DG_EINVAL, "detach the learned source (dg_attach_mlp(h, NULL)) first");
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        // carry the resident state over through the FP64 staging buffer
        if (h->have_state) {
            if (dg_status s = to_api(h, h->B[h->cur], h->L[h->cur], h->stage64, h->href)) return s;
            CUDA_TRY(cudaStreamSynchronize(h->stream));
        }
        drop_graphs(h);
        free_state_buffers(h);
        h->prec = (int)value;
        if (dg_status s = alloc_state_buffers(h)) return s;
        h->cur = 0;
        if (h->have_state) {
            if (h->f32() || h->wb) {
                // reference depth: mean of the element mean depths
                std::vector<double> m0(h->nel);
                CUDA_TRY(cudaMemcpy2D(m0.data(), sizeof(double), h->stage64, sizeof(double) * 3 * h->nphi,
                                      sizeof(double), h->nel, cudaMemcpyDeviceToHost));
                double s = 0;
                for (double v : m0) s += v;
                h->href = h->href_fixed ? h->href_given : 0.5 * s / (double)h->nel;
            } else {
                h->href = 0.0;
            }
            if (dg_status s = to_internal(h, h->stage64, h->B[0], h->L[0], h->href)) return s;
            CUDA_TRY(cudaStreamSynchronize(h->stream));
        }
        return DG_OK;
    }
    case DG_OPT_WELL_BALANCED: {
        if (value != 0 && value != 1) return fail(DG_EINVAL, "well-balanced option must be 0 or 1");
        if (value == h->wb) return DG_OK;
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        // the reference depth of the FP64 path changes: re-encode the state
        if (h->have_state)
            if (dg_status s = to_api(h, h->B[h->cur], h->L[h->cur], h->stage64, h->href)) return s;
        h->wb = (int)value;
        if (h->have_state) {
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            h->href = 0.0;
            if (h->f32() || h->wb) {
                std::vector<double> m0(h->nel);
                CUDA_TRY(cudaMemcpy2D(m0.data(), sizeof(double), h->stage64, sizeof(double) * 3 * h->nphi,
                                      sizeof(double), h->nel, cudaMemcpyDeviceToHost));
                double sum = 0;
                for (double v : m0) sum += v;
                h->href = h->href_fixed ? h->href_given : 0.5 * sum / (double)h->nel;
            }
            h->cur = 0;
            if (dg_status s = to_internal(h, h->stage64, h->B[0], h->L[0], h->href)) return s;
            CUDA_TRY(cudaStreamSynchronize(h->stream));
        }
        return DG_OK;
    }
    case DG_OPT_RK_ORDER:
        if (value < 1 || value > 4) return fail(DG_EINVAL, "RK order must be 1..4");
        h->rk = (int)value;
        return DG_OK;
    case DG_OPT_CHECK_FINITE:
        h->check = value ? 1 : 0;
        return DG_OK;
    case DG_OPT_ALPHA_MODE:
        if (value != 0 && value != 1) return fail(DG_EINVAL, "unknown alpha mode %lld", value);
        if (value != h->alpha_mode) {
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            drop_graphs(h);
            h->alpha_mode = (int)value;
        }
        return DG_OK;
    case DG_OPT_STREAM:
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->stream = value ? reinterpret_cast<cudaStream_t>(value) : h->own_stream;
        drop_graphs(h);
        return DG_OK;
    case DG_OPT_STEPS_PER_GRAPH:
        if (value < 1 || value > 1024) return fail(DG_EINVAL, "steps per graph must be 1..1024");
        h->spg = (int)value;
        return DG_OK;
    default:
        return fail(DG_EINVAL, "unknown option %d", key);
    }
}

dg_status dg_set_state_device(dg_handle h, const double *d_modal, size_t len)
{
    if (dg_status s = check(h)) return s;
    if (!d_modal || len != h->len) return fail(DG_EINVAL, "state length %zu, expected %zu", len, h->len);
    DeviceGuard dg(h->device);
    if (h->physics != 0) {
        CUDA_TRY(cudaMemcpyAsync(h->B[0], d_modal, len * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->cur = 0;
        h->href = 0.0;
        h->have_state = true;
        return DG_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(h->stage64, d_modal, len * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->href = 0.0;
    if (h->f32() || h->wb) {
        std::vector<double> m0(h->nel);
        CUDA_TRY(cudaMemcpy2DAsync(m0.data(), sizeof(double), h->stage64, sizeof(double) * 3 * h->nphi,
                                   sizeof(double), h->nel, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        double s = 0;
        for (double v : m0) s += v;
        h->href = h->href_fixed ? h->href_given : 0.5 * s / (double)h->nel;
    }
    h->cur = 0;
    if (dg_status s = to_internal(h, h->stage64, h->B[0], h->L[0], h->href)) return s;
    h->have_state = true;
    return DG_OK;
}

dg_status dg_set_state(dg_handle h, const double *modal, size_t len)
{
    if (dg_status s = check(h)) return s;
    if (!modal || len != h->len) return fail(DG_EINVAL, "state length %zu, expected %zu", len, h->len);
    DeviceGuard dg(h->device);
    if (h->physics != 0) {
        CUDA_TRY(cudaMemcpyAsync(h->B[0], modal, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->cur = 0;
        h->href = 0.0;
        h->have_state = true;
        return DG_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(h->stage64, modal, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->href = (h->f32() || h->wb) ? (h->href_fixed ? h->href_given : mean_depth(modal, h->nel, h->nphi)) : 0.0;
    h->cur = 0;
    if (dg_status s = to_internal(h, h->stage64, h->B[0], h->L[0], h->href)) return s;
    CUDA_TRY(cudaStreamSynchronize(h->stream));   // the host buffer is only borrowed
    h->have_state = true;
    return DG_OK;
}

dg_status dg_get_state_device(dg_handle h, double *d_modal, size_t len)
{
    if (dg_status s = check(h)) return s;
    if (!d_modal || len != h->len) return fail(DG_EINVAL, "state length %zu, expected %zu", len, h->len);
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    if (h->physics != 0) {
        CUDA_TRY(cudaMemcpyAsync(d_modal, h->B[h->cur], len * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        return DG_OK;
    }
    return to_api(h, h->B[h->cur], h->L[h->cur], d_modal, h->href);
}

dg_status dg_get_state(dg_handle h, double *modal, size_t len)
{
    if (dg_status s = check(h)) return s;
    if (!modal || len != h->len) return fail(DG_EINVAL, "state length %zu, expected %zu", len, h->len);
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    if (h->physics != 0) {
        CUDA_TRY(cudaMemcpyAsync(modal, h->B[h->cur], len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        return DG_OK;
    }
    if (dg_status s = to_api(h, h->B[h->cur], h->L[h->cur], h->stage64, h->href)) return s;
    CUDA_TRY(cudaMemcpyAsync(modal, h->stage64, len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DG_OK;
}

dg_status dg_rhs(dg_handle h, const double *modal_in, double *tend_out, size_t len)
{
    if (dg_status s = check(h)) return s;
    if (!modal_in || !tend_out || len != h->len) return fail(DG_EINVAL, "state length %zu, expected %zu", len, h->len);
    if (h->band) return fail(DG_EUNSUPPORTED, "dg_rhs needs a whole mesh (a band's ghost rows are not inputs)");
    DeviceGuard dg(h->device);
    // scratch: the increment buffers are free between steps
    void *in = h->I[0], *outb = h->I[1];
    if (h->physics != 0) {
        CUDA_TRY(cudaMemcpyAsync(in, modal_in, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        StageArgs<double> a;
        std::memset(&a, 0, sizeof a);
        a.status = h->d_status;
        a.base = static_cast<double *>(in);
        a.out_rhs = static_cast<double *>(outb);
        if (launch_plane(h, a))
            return fail(DG_ECUDA, "planar stage launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        h->launches++;
        CUDA_TRY(cudaMemcpyAsync(tend_out, outb, len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (h->check) return read_status(h);
        return DG_OK;
    }
    const double href = (h->f32() || h->wb) ? mean_depth(modal_in, h->nel, h->nphi) : 0.0;
    CUDA_TRY(cudaMemcpyAsync(h->stage64, modal_in, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (dg_status s = to_internal(h, h->stage64, in, nullptr, href)) return s;
    int r;
    if (h->prec == DG_PREC_FP64) {
        StageArgs<double> a = base_args<double>(h, h->rows64, href);
        a.base = static_cast<double *>(in);
        a.out_rhs = static_cast<double *>(outb);
        if (dg_status gs = enqueue_global_speeds<double>(h, a)) return gs;
        r = dg_launch_stage<double>(h->n, a, h->stream);
    } else if (h->tc()) {
        // stage in the lane-contiguous layout: input through SB[0], tendency in SB[1]
        const int el = 3 * h->nphi;
        if (dg_launch_permute(static_cast<float *>(in), static_cast<float *>(h->SB[0]), h->nlat, h->nlon, el, 1,
                              h->stream))
            return fail(DG_ECUDA, "layout permutation failed: %s", cudaGetErrorString(cudaGetLastError()));
        StageArgs<float> a = base_args<float>(h, h->rows32, href);
        a.base = static_cast<float *>(h->SB[0]);
        a.out_rhs = static_cast<float *>(h->SB[1]);
        if (dg_status gs = enqueue_global_speeds<float>(h, a)) return gs;
        r = dg_launch_stage_tc(h->n, h->prec - DG_PREC_FP32_TC_BF16, a, h->stream);
        if (!r) r = dg_launch_permute(static_cast<float *>(h->SB[1]), static_cast<float *>(outb), h->nlat, h->nlon,
                                      el, 0, h->stream);
        h->aux_launches += 2;
    } else {
        StageArgs<float> a = base_args<float>(h, h->rows32, href);
        a.base = static_cast<float *>(in);
        a.out_rhs = static_cast<float *>(outb);
        if (h->mlp) {   // the attached learned source is part of the tendency
            const int ms = dg_mlp_launch_source(h->mlp, a.base, nullptr, (float)href, h->nlon, h->nlat, h->c0, h->src,
                                                h->stream);
            if (ms == 2) return fail(DG_EINVAL, "the network's row statistics belong to another mesh");
            if (ms) return fail(DG_ECUDA, "learned source launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            a.src = h->src;
        }
        if (dg_status gs = enqueue_global_speeds<float>(h, a)) return gs;
        r = dg_launch_stage<float>(h->n, a, h->stream);
    }
    if (r) return fail(DG_ECUDA, "stage kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->launches++;
    if (dg_status s = to_api(h, outb, nullptr, h->stage64, 0.0)) return s;   // tendencies carry no reference depth
    CUDA_TRY(cudaMemcpyAsync(tend_out, h->stage64, len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->check) return read_status(h);
    return DG_OK;
}

dg_status dg_step(dg_handle h, int n, double dt)
{
    if (dg_status s = check(h)) return s;
    if (n < 0) return fail(DG_EINVAL, "n must be >= 0");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(DG_EINVAL, "dt must be positive and finite");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    if (h->band)
        return fail(DG_EUNSUPPORTED, "a latitude band advances one stage at a time (dg_band_stage), after its "
                                     "ghost rows have received the neighbours' rows");
    if (n == 0) return DG_OK;
    DeviceGuard dg(h->device);
    if (h->tc())
        if (dg_status s = permute_state(h, h->cur, 1)) return s;
    int K = std::min(h->spg, n);
    if ((K & 1) && K > 1) K -= 1;   // even graphs return u^n to the same base buffer
    int full = n / K, rest = n - full * K;
    if (full > 0) {
        GraphEntry *ge = nullptr;
        for (auto &g : h->graphs)
            if (g.steps == K && g.dt == dt && g.order == h->rk && g.prec == h->prec && g.cur_in == h->cur &&
                g.stream == h->stream)
                ge = &g;
        if (!ge) {
            GraphEntry g;
            g.steps = K;
            g.dt = dt;
            g.order = h->rk;
            g.prec = h->prec;
            g.cur_in = h->cur;
            g.stream = h->stream;
            int cur = h->cur;
            long long before = h->launches;
            CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            dg_status st = launch_steps(h, K, dt, &cur);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
            h->launches = before;   // capture only records; replays are counted below
            if (st) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return fail(DG_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(DG_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
            g.cur_out = cur;
            if (h->graphs.size() >= 8) {
                cudaGraphExecDestroy(h->graphs.front().exec);
                h->graphs.erase(h->graphs.begin());
            }
            h->graphs.push_back(g);
            ge = &h->graphs.back();
        }
        StagePlan pl[4];
        const int ns = rk_plan(h->rk, pl);
        for (int r = 0; r < full; ++r) {
            CUDA_TRY(cudaGraphLaunch(ge->exec, h->stream));
            h->launches += (long long)K * ns;
            h->cur = ge->cur_out;
        }
    }
    if (rest > 0) {
        int cur = h->cur;
        if (dg_status st = launch_steps(h, rest, dt, &cur)) return st;
        h->cur = cur;
    }
    if (h->tc())
        if (dg_status s = permute_state(h, h->cur, 0)) return s;
    h->t += n * dt;
    if (h->check) return read_status(h);
    return DG_OK;
}

}  // extern "C"

namespace {
dg_status enqueue_mass(dg_ctx *h, double *d_out, double *d_pair = nullptr)
{
    int r = h->prec == DG_PREC_FP64
                ? dg_launch_mass<double>(static_cast<const double *>(h->B[h->cur]),
                                         static_cast<const double *>(h->L[h->cur]), h->c0, h->nlon, h->nlat, h->n,
                                         h->href, h->tab.dlam, h->tab.dth, h->R * h->R, h->partials, h->nblocks,
                                         d_out, d_pair, h->stream)
                : dg_launch_mass<float>(static_cast<const float *>(h->B[h->cur]),
                                        static_cast<const float *>(h->L[h->cur]), h->c0, h->nlon, h->nlat, h->n,
                                        h->href, h->tab.dlam, h->tab.dth, h->R * h->R, h->partials, h->nblocks,
                                        d_out, d_pair, h->stream);
    if (r) return fail(DG_ECUDA, "mass kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->aux_launches += 2;
    return DG_OK;
}
}  // namespace

extern "C" {

dg_status dg_total_mass(dg_handle h, double *mass)
{
    if (dg_status s = check(h)) return s;
    if (h->physics == 1) return planar_unsupported(h, "dg_total_mass");
    if (h->physics == 2) {   // planar shallow water: R^0 sum_k (dx dy / 2) h_00, compensated, on the host
        if (!h->have_state) return fail(DG_EINVAL, "no state set");
        DeviceGuard dg(h->device);
        std::vector<double> u(h->len);
        CUDA_TRY(cudaMemcpyAsync(u.data(), h->B[h->cur], h->len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        const double w = 0.5 * (h->plen / h->nlon) * (h->plen / h->nlat);   // int L0(xi) L0(eta) = 2, jac dx dy / 4
        double sum = 0.0, comp = 0.0;
        for (size_t e = 0; e < h->nel; ++e) {
            const double x = w * u[e * 3 * h->nphi];
            const double t = sum + x;
            comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
            sum = t;
        }
        *mass = sum + comp;
        return DG_OK;
    }
    if (!mass) return fail(DG_EINVAL, "mass is NULL");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    if (dg_status s = enqueue_mass(h, h->d_result)) return s;
    double m = 0;
    CUDA_TRY(cudaMemcpyAsync(&m, h->d_result, sizeof m, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *mass = m;
    return DG_OK;
}

dg_status dg_total_mass_device(dg_handle h, double *d_mass)
{
    if (dg_status s = check(h)) return s;
    if (h->physics != 0) return planar_unsupported(h, "dg_total_mass_device");
    if (!d_mass) return fail(DG_EINVAL, "d_mass is NULL");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    return enqueue_mass(h, d_mass);
}

}  // extern "C"

namespace {
// The two terms of the CFL step of the resident state: H = min over the
// rows and Gauss points of min(R dth, R cos(theta) dlam), c = max over the
// Gauss points of sqrt(u^2 + v^2) + sqrt(g h).
dg_status cfl_terms(dg_ctx *h, double *H_out, double *c_out)
{
    CUDA_TRY(cudaMemsetAsync(h->d_maxbits, 0, sizeof(unsigned long long), h->stream));
    int r = h->prec == DG_PREC_FP64
                ? dg_launch_max_speed<double>(static_cast<const double *>(h->B[h->cur]), h->nlon, h->nlat, h->n,
                                              h->href, h->g, h->d_maxbits, h->d_status, h->stream)
                : dg_launch_max_speed<float>(static_cast<const float *>(h->B[h->cur]), h->nlon, h->nlat, h->n,
                                             h->href, h->g, h->d_maxbits, h->d_status, h->stream);
    if (r) return fail(DG_ECUDA, "wave-speed kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    unsigned long long bits = 0;
    CUDA_TRY(cudaMemcpyAsync(&bits, h->d_maxbits, sizeof bits, cudaMemcpyDeviceToHost, h->stream));
    if (dg_status s = read_status(h)) return s;
    double c;
    std::memcpy(&c, &bits, sizeof c);
    if (!(c > 0)) return fail(DG_ENONPHYSICAL, "no positive wave speed");
    double H = INFINITY;
    for (int j = 0; j < h->nlat; ++j)
        for (int q = 0; q < h->n; ++q)
            H = std::min(H, std::min(h->R * h->tab.dth, h->R * h->tab.rows[j].cosn[q] * h->tab.dlam));
    *H_out = H;
    *c_out = c;
    return DG_OK;
}
}  // namespace

extern "C" {

dg_status dg_max_dt(dg_handle h, double cfl, double *dt)
{
    if (dg_status s = check(h)) return s;
    if (h->physics != 0) return planar_unsupported(h, "dg_max_dt");
    if (!dt || !(cfl > 0)) return fail(DG_EINVAL, "need cfl > 0 and dt != NULL");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    double H, c;
    if (dg_status s = cfl_terms(h, &H, &c)) return s;
    *dt = cfl * H / (std::max(h->p, 1) * c);
    return DG_OK;
}

dg_status dg_band_cfl_terms(dg_handle h, double *H, double *c)
{
    if (dg_status s = check(h)) return s;
    if (h->physics != 0) return planar_unsupported(h, "dg_band_cfl_terms");
    if (!H || !c) return fail(DG_EINVAL, "H and c must not be NULL");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    return cfl_terms(h, H, c);
}

dg_status dg_projection_nodes(dg_handle h, double *lam, size_t nlam, double *theta, size_t ntheta)
{
    if (dg_status s = check(h)) return s;
    const int nm = h->tab.nm;
    if (h->physics != 0) {   // planar: x_i = (i + (1 + x_q) / 2) dx, y likewise, on [0, plen]^2
        if (!lam || !theta || nlam != (size_t)h->nlon * nm || ntheta != (size_t)h->nlat * nm)
            return fail(DG_EINVAL, "need nx*nm = %zu and ny*nm = %zu values", (size_t)h->nlon * nm,
                        (size_t)h->nlat * nm);
        const double dx = h->plen / h->nlon, dy = h->plen / h->nlat;
        for (int i = 0; i < h->nlon; ++i)
            for (int q = 0; q < nm; ++q) lam[(size_t)i * nm + q] = (i + 0.5 * (1.0 + h->tab.xm[q])) * dx;
        for (int j = 0; j < h->nlat; ++j)
            for (int q = 0; q < nm; ++q) theta[(size_t)j * nm + q] = (j + 0.5 * (1.0 + h->tab.xm[q])) * dy;
        return DG_OK;
    }
    if (!lam || !theta || nlam != (size_t)h->nlon * nm || ntheta != (size_t)h->nlat * nm)
        return fail(DG_EINVAL, "need nlon*nm = %zu and nlat*nm = %zu values", (size_t)h->nlon * nm,
                    (size_t)h->nlat * nm);
    for (int i = 0; i < h->nlon; ++i)
        for (int q = 0; q < nm; ++q) lam[(size_t)i * nm + q] = (i + 0.5 * (1.0 + h->tab.xm[q])) * h->tab.dlam;
    for (int j = 0; j < h->nlat; ++j)
        for (int q = 0; q < nm; ++q)
            theta[(size_t)j * nm + q] = -0.5 * M_PI + (h->j0 + j + 0.5 * (1.0 + h->tab.xm[q])) * h->tab.dth;
    return DG_OK;
}

dg_status dg_project_nodal(dg_handle h, const double *nodal, size_t len_nodal, double *modal_out, size_t len)
{
    if (dg_status s = check(h)) return s;
    const int n = h->n, nm = h->tab.nm;
    if (h->physics != 0) {   // planar: the mass matrix is (dx dy / 4) I, so u_m = sum_q w w f L_a L_b
        const int nf = h->physics == 2 ? 3 : 1;
        if (!nodal || !modal_out || len != h->len || len_nodal != h->nel * nf * nm * nm)
            return fail(DG_EINVAL, "bad lengths");
        std::vector<double> PL((size_t)n * nm);
        for (int a = 0; a < n; ++a)
            for (int q = 0; q < nm; ++q) PL[(size_t)a * nm + q] = h->tab.wm[q] * dg_legendre(a, h->tab.xm[q]);
        for (size_t el = 0; el < h->nel; ++el)
            for (int f = 0; f < nf; ++f) {
                const double *v = nodal + (el * nf + f) * nm * nm;
                double *o = modal_out + (el * nf + f) * h->nphi;
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        double acc = 0.0;
                        for (int qy = 0; qy < nm; ++qy) {
                            double t = 0.0;
                            for (int qx = 0; qx < nm; ++qx) t += PL[(size_t)a * nm + qx] * v[qy * nm + qx];
                            acc += PL[(size_t)b * nm + qy] * t;
                        }
                        o[b * n + a] = acc;
                    }
            }
        return DG_OK;
    }
    if (!nodal || !modal_out || len != h->len || len_nodal != h->nel * 3 * nm * nm)
        return fail(DG_EINVAL, "bad lengths");
    // separable projection: sum over the lambda points, then the theta points
    // weighted by cos(theta), then the inverse of C_j (the dlam dth / 4 of the
    // mass matrix cancels against the same factor of the right-hand side)
    std::vector<double> PL((size_t)n * nm), PC((size_t)n * nm), s((size_t)nm * n), r((size_t)n * n);
    for (int a = 0; a < n; ++a)
        for (int q = 0; q < nm; ++q) PL[(size_t)a * nm + q] = h->tab.wm[q] * dg_legendre(a, h->tab.xm[q]);
    for (int j = 0; j < h->nlat; ++j) {
        const double tb = -0.5 * M_PI + (h->j0 + j) * h->tab.dth;
        for (int b = 0; b < n; ++b)
            for (int q = 0; q < nm; ++q)
                PC[(size_t)b * nm + q] =
                    PL[(size_t)b * nm + q] * std::cos(tb + 0.5 * (1.0 + h->tab.xm[q]) * h->tab.dth);
        const RowTab<double> &rt = h->tab.rows[j];
        for (int i = 0; i < h->nlon; ++i)
            for (int f = 0; f < 3; ++f) {
                const size_t el = (size_t)j * h->nlon + i;
                const double *v = nodal + (el * 3 + f) * nm * nm;
                for (int qy = 0; qy < nm; ++qy)
                    for (int a = 0; a < n; ++a) {
                        double acc = 0;
                        for (int qx = 0; qx < nm; ++qx) acc += PL[(size_t)a * nm + qx] * v[qy * nm + qx];
                        s[(size_t)qy * n + a] = acc;
                    }
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        double acc = 0;
                        for (int qy = 0; qy < nm; ++qy) acc += PC[(size_t)b * nm + qy] * s[(size_t)qy * n + a];
                        r[(size_t)b * n + a] = acc;
                    }
                double *o = modal_out + (el * 3 + f) * h->nphi;
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        double acc = 0;
                        for (int c = 0; c < n; ++c) acc += rt.Ci[b][c] * r[(size_t)c * n + a];
                        o[b * n + a] = acc;
                    }
            }
    }
    return DG_OK;
}

dg_status dg_attach_mlp(dg_handle h, dg_mlp m)
{
    if (dg_status s = check(h)) return s;
    if (h->band && m) return fail(DG_EUNSUPPORTED, "the learned source needs a whole mesh");
    DeviceGuard dg(h->device);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    if (!m) {
        h->mlp = nullptr;
        return DG_OK;
    }
    if (h->physics != 0 || h->p != 1 || h->prec != DG_PREC_FP32)
        return fail(DG_EUNSUPPORTED, "the learned source needs a degree-1 FP32 sphere solver");
    if (!dg_mlp_shape_is(m, 60, 128, 12)) return fail(DG_EINVAL, "the learned source needs a 60-128-128-12 network");
    if (!h->src && cudaMalloc(&h->src, sizeof(float) * h->len) != cudaSuccess)
        return fail(DG_ENOMEM, "cudaMalloc of the source buffer failed");
    h->mlp = m;
    return DG_OK;
}

dg_status dg_restrict_from(dg_handle coarse, dg_handle fine)
{
    if (dg_status s = check(coarse)) return s;
    if (dg_status s = check(fine)) return s;
    if (coarse->physics != 0 || fine->physics != 0) return planar_unsupported(coarse, "dg_restrict_from");
    if (coarse->band || fine->band) return fail(DG_EUNSUPPORTED, "dg_restrict_from needs whole meshes");
    if (!fine->have_state) return fail(DG_EINVAL, "the fine solver has no state");
    if (coarse->device != fine->device) return fail(DG_EINVAL, "the solvers live on different devices");
    const int r = fine->nlon / coarse->nlon;
    if (r < 1 || fine->nlon != r * coarse->nlon || fine->nlat != r * coarse->nlat)
        return fail(DG_EINVAL, "the fine mesh must refine every coarse element into r x r elements");
    if (fine->R != coarse->R) return fail(DG_EINVAL, "different sphere radii");
    DeviceGuard dg(coarse->device);
    if (dg_status s = to_api(fine, fine->B[fine->cur], fine->L[fine->cur], fine->stage64, fine->href)) return s;
    CUDA_TRY(cudaStreamSynchronize(fine->stream));
    RestrictTab tab;
    std::memset(&tab, 0, sizeof tab);
    dg_gauss_legendre(8, tab.x, tab.w);
    for (int a = 0; a < fine->n; ++a)
        for (int q = 0; q < 8; ++q) tab.LVf[a][q] = dg_legendre(a, tab.x[q]);
    tab.jf = 0.25 * fine->tab.dlam * fine->tab.dth;
    tab.dthc = coarse->tab.dth;
    tab.inv_jc = 4.0 / (coarse->tab.dlam * coarse->tab.dth);
    if (dg_launch_restrict(fine->stage64, fine->nlon, fine->n, coarse->stage64, coarse->nlon, coarse->nlat, coarse->n, r,
                           coarse->rows64, tab, coarse->stream))
        return fail(DG_ECUDA, "restriction kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
    coarse->href = 0.0;
    if (coarse->f32() || coarse->wb) {
        std::vector<double> m0(coarse->nel);
        CUDA_TRY(cudaMemcpy2DAsync(m0.data(), sizeof(double), coarse->stage64, sizeof(double) * 3 * coarse->nphi,
                                   sizeof(double), coarse->nel, cudaMemcpyDeviceToHost, coarse->stream));
        CUDA_TRY(cudaStreamSynchronize(coarse->stream));
        double s = 0;
        for (double v : m0) s += v;
        coarse->href = 0.5 * s / (double)coarse->nel;
    }
    coarse->cur = 0;
    if (dg_status s = to_internal(coarse, coarse->stage64, coarse->B[0], coarse->L[0], coarse->href)) return s;
    CUDA_TRY(cudaStreamSynchronize(coarse->stream));
    coarse->have_state = true;
    return DG_OK;
}

dg_status dg_tc_check_contraction(int degree, int op, const float *d_a, float *d_out, int *n1, int *k1)
{
    if (degree < 0 || degree > DG_MAXN - 1 || (op != 0 && op != 1) || !n1 || !k1)
        return fail(DG_EINVAL, "need 0 <= degree <= %d, op 0 or 1, n1 and k1", DG_MAXN - 1);
    cudaStream_t s = nullptr;
    if (d_a && d_out && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(DG_ECUDA, "stream creation failed");
    int r = dg_tc_gemm_check(degree + 1, op, d_a, d_out, n1, k1, s);
    if (s) cudaStreamDestroy(s);
    if (r == 2) return fail(DG_ETIMEOUT, "the tensor cores did not complete the contraction");
    if (r) return fail(DG_ECUDA, "contraction check failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
}

dg_status dg_measure_fp64_peak(int reps, double *gflops)
{
    if (!gflops || reps < 1) return fail(DG_EINVAL, "need reps >= 1 and gflops");
    if (dg_probe_fp64_gflops(reps, gflops))
        return fail(DG_ECUDA, "FP64 probe failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
}

// ------------------------------------------------------ latitude bands --

size_t dg_band_halo_len(dg_handle h) { return h && h->band ? 2 * h->row_len() : 0; }

dg_status dg_band_set_reference_depth(dg_handle h, double href)
{
    if (dg_status s = check(h)) return s;
    if (!h->band) return fail(DG_EINVAL, "not a band handle");
    if (!(href > 0) || !std::isfinite(href)) return fail(DG_EINVAL, "the reference depth must be positive");
    h->href_fixed = 1;
    h->href_given = href;
    return DG_OK;
}

namespace {
// The current stage's input: u^n in B[cur] and the increment the stage reads
// (null for a stage without one).
void band_stage_inputs(dg_ctx *h, char **base, char **inc)
{
    StagePlan pl[4];
    rk_plan(h->rk, pl);
    const int ii = pl[h->band_stage].inc_in;
    *base = static_cast<char *>(h->B[h->cur]);
    *inc = ii >= 0 ? static_cast<char *>(h->I[ii]) : nullptr;
}
}  // namespace

dg_status dg_band_pack(dg_handle h, int side, void *d_out)
{
    if (dg_status s = check(h)) return s;
    if (!h->band) return fail(DG_EINVAL, "not a band handle");
    if (!d_out || (side != 0 && side != 1)) return fail(DG_EINVAL, "need side 0 (south) or 1 (north) and d_out");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    const size_t rb = h->row_len() * elem_size(h->prec);
    char *base, *inc;
    band_stage_inputs(h, &base, &inc);
    const size_t off = side == 0 ? 0 : (size_t)(h->nlat - 1) * rb;
    char *o = static_cast<char *>(d_out);
    CUDA_TRY(cudaMemcpyAsync(o, base + off, rb, cudaMemcpyDeviceToDevice, h->stream));
    if (inc) CUDA_TRY(cudaMemcpyAsync(o + rb, inc + off, rb, cudaMemcpyDeviceToDevice, h->stream));
    else CUDA_TRY(cudaMemsetAsync(o + rb, 0, rb, h->stream));
    return DG_OK;
}

dg_status dg_band_unpack(dg_handle h, int side, const void *d_in)
{
    if (dg_status s = check(h)) return s;
    if (!h->band) return fail(DG_EINVAL, "not a band handle");
    if (!d_in || (side != 0 && side != 1)) return fail(DG_EINVAL, "need side 0 (south) or 1 (north) and d_in");
    if ((side == 0 && !h->gs) || (side == 1 && !h->gn)) return fail(DG_EINVAL, "no ghost row on that side (a pole)");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    const size_t rb = h->row_len() * elem_size(h->prec);
    char *base, *inc;
    band_stage_inputs(h, &base, &inc);
    // the south ghost row sits just before own row 0, the north one just after the last own row
    const ptrdiff_t off = side == 0 ? -(ptrdiff_t)rb : (ptrdiff_t)h->nlat * (ptrdiff_t)rb;
    const char *in = static_cast<const char *>(d_in);
    CUDA_TRY(cudaMemcpyAsync(base + off, in, rb, cudaMemcpyDeviceToDevice, h->stream));
    if (inc) CUDA_TRY(cudaMemcpyAsync(inc + off, in + rb, rb, cudaMemcpyDeviceToDevice, h->stream));
    return DG_OK;
}

dg_status dg_band_stage(dg_handle h, double dt)
{
    if (dg_status s = check(h)) return s;
    if (!h->band) return fail(DG_EINVAL, "not a band handle");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(DG_EINVAL, "dt must be positive and finite");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    StagePlan pl[4];
    const int ns = rk_plan(h->rk, pl);
    if (h->band_stage >= ns) h->band_stage = 0;   // the RK order changed between steps
    if (h->band_stage == 0) h->band_dt = dt;
    else if (dt != h->band_dt) return fail(DG_EINVAL, "dt changed within a step");
    DeviceGuard dg(h->device);
    const int s = h->band_stage;
    dg_status st = h->prec == DG_PREC_FP64 ? launch_stage_t<double>(h, dt, h->cur, h->rows64, s)
                                           : launch_stage_t<float>(h, dt, h->cur, h->rows32, s);
    if (st) return st;
    if (pl[s].fin) {
        h->cur ^= 1;
        h->band_stage = 0;
        h->t += dt;
        if (h->check) return read_status(h);
    } else {
        h->band_stage = s + 1;
    }
    return DG_OK;
}

dg_status dg_band_mass_pair(dg_handle h, double *sum, double *err)
{
    if (dg_status s = check(h)) return s;
    if (h->physics != 0) return planar_unsupported(h, "dg_band_mass_pair");
    if (!sum || !err) return fail(DG_EINVAL, "sum and err must not be NULL");
    if (!h->have_state) return fail(DG_EINVAL, "no state set");
    DeviceGuard dg(h->device);
    if (dg_status s = enqueue_mass(h, nullptr, h->partials + 2 * h->nblocks)) return s;
    double pair[2];
    CUDA_TRY(cudaMemcpyAsync(pair, h->partials + 2 * h->nblocks, sizeof pair, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *sum = pair[0];
    *err = pair[1];
    return DG_OK;
}

dg_status dg_get_time(dg_handle h, double *t)
{
    if (dg_status s = check(h)) return s;
    if (!t) return fail(DG_EINVAL, "t is NULL");
    *t = h->t;
    return DG_OK;
}

dg_status dg_set_time(dg_handle h, double t)
{
    if (dg_status s = check(h)) return s;
    if (!std::isfinite(t)) return fail(DG_EINVAL, "t must be finite");
    h->t = t;
    return DG_OK;
}

}  // extern "C"

void dg_set_last_error(const char *msg) { g_err = msg ? msg : ""; }

int dg_ensure_basis(int device) { return upload_basis_once(device) == DG_OK ? 0 : 1; }

int dg_mass_blocks(size_t nel)
{
    size_t b = (nel + 1023) / 1024;
    return (int)std::max<size_t>(1, std::min<size_t>(b, 1024));
}

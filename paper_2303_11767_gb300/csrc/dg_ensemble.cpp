// dg_ensemble.cpp -- batched ensemble of independent meshes (uneven sizes and
// degrees) advanced together: one persistent FP32 launch per SSP-RK stage
// over all members, captured in a CUDA graph, with a tile-shape / grid-size
// autotuner.  The members are the decoupled copies of the 2-D problem of the
// paper's vertical-levels experiment (Sec. 5.2.2), here each with its own
// mesh, degree and initial field.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dg_internal.h"
#include "../../include/dgswe.h"

namespace {

dg_status efail(dg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    dg_set_last_error(buf);
    return s;
}

#define ECUDA(call)                                                                                      \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return efail(DG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

}  // namespace

struct dg_ens {
    int nm = 0;
    std::vector<int> nlon, nlat, deg;
    std::vector<size_t> off, nel;   // value offset and element count per member
    size_t total = 0;               // values in one state array
    double R = 0, g = 0, omega = 0;
    int device = 0, sms = 0;
    std::vector<HostTables> tabs;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    float *B[2] = {nullptr, nullptr}, *L[2] = {nullptr, nullptr}, *I[2] = {nullptr, nullptr};
    int cur = 0;
    double *stage64 = nullptr;      // FP64 staging for one member
    RowTab<float> *rows = nullptr;
    std::vector<EnsMember<float>> hm;
    EnsMember<float> *dm = nullptr;
    EnsItem *items[2] = {nullptr, nullptr};   // work lists for the two tile heights
    int nitems[2] = {0, 0};
    double *c0 = nullptr, *partials = nullptr, *d_result = nullptr;
    std::vector<size_t> c0_off;
    int nblocks = 0;
    unsigned *d_status = nullptr;
    unsigned long long *d_maxbits = nullptr;
    std::vector<double> href, dt;
    std::vector<char> have;
    int tile_rows = DG_ENS_TILE_ROWS_B, bps = 2, spg = 16;
    bool members_dirty = true;
    long long launches = 0;
    struct Graph {
        cudaGraphExec_t exec;
        int steps, cur_in, cur_out, tile_rows, bps;
        cudaStream_t stream;
    };
    std::vector<Graph> graphs;
};

namespace {

void drop_graphs(dg_ens *e)
{
    for (auto &g : e->graphs) cudaGraphExecDestroy(g.exec);
    e->graphs.clear();
}

int tile_index(int tile_rows) { return tile_rows == DG_ENS_TILE_ROWS_A ? 0 : 1; }

dg_status upload_members(dg_ens *e)
{
    if (!e->members_dirty) return DG_OK;
    for (int m = 0; m < e->nm; ++m) {
        EnsMember<float> &x = e->hm[m];
        x.href = (float)e->href[m];
        x.P0 = (float)(0.5 * e->g * e->href[m] * e->href[m]);
        x.dt = (float)e->dt[m];
    }
    ECUDA(cudaMemcpyAsync(e->dm, e->hm.data(), sizeof(EnsMember<float>) * e->nm, cudaMemcpyHostToDevice, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    e->members_dirty = false;   // the graphs read the table through its pointer: they stay valid
    return DG_OK;
}

struct EPlan {
    int inc_in, inc_out, fin;
    double ci, cc;
};

// SSP-RK3 (Table "Butcher") in increment form, as in the single-mesh solver
const EPlan kPlan[3] = {{-1, 0, 0, 0, 1}, {0, 1, 0, 0.25, 0.25}, {1, -1, 1, 2.0 / 3.0, 2.0 / 3.0}};

dg_status launch_step(dg_ens *e, int cur)
{
    const int ti = tile_index(e->tile_rows);
    for (int s = 0; s < 3; ++s) {
        EnsArgs<float> a;
        std::memset(&a, 0, sizeof a);
        a.base = e->B[cur];
        a.inc = kPlan[s].inc_in >= 0 ? e->I[kPlan[s].inc_in] : nullptr;
        a.inc_out = kPlan[s].inc_out >= 0 ? e->I[kPlan[s].inc_out] : nullptr;
        if (kPlan[s].fin) {
            a.lo = e->L[cur];
            a.out_base = e->B[cur ^ 1];
            a.out_lo = e->L[cur ^ 1];
        }
        a.rows = e->rows;
        a.members = e->dm;
        a.items = e->items[ti];
        a.nitems = e->nitems[ti];
        a.status = e->d_status;
        a.g = (float)e->g;
        a.invR = (float)(1.0 / e->R);
        a.twoOmega = (float)(2.0 * e->omega);
        a.ci = (float)kPlan[s].ci;
        a.cc = (float)kPlan[s].cc;
        const int grid = std::max(1, std::min(e->nitems[ti], e->sms * e->bps));
        if (dg_launch_ensemble_stage<float>(e->tile_rows, grid, a, e->stream))
            return efail(DG_ECUDA, "ensemble stage launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        e->launches++;
    }
    return DG_OK;
}

dg_status build_items(dg_ens *e)
{
    for (int ti = 0; ti < 2; ++ti) {
        const int W = ti == 0 ? DG_ENS_TILE_ROWS_A : DG_ENS_TILE_ROWS_B;
        std::vector<EnsItem> it;
        for (int m = 0; m < e->nm; ++m) {
            const int n = e->deg[m] + 1, G = dg_ensemble_tile_width(n);
            const int tx = (e->nlon[m] + G - 1) / G, ty = (e->nlat[m] + W - 1) / W;
            for (int y = 0; y < ty; ++y)
                for (int x = 0; x < tx; ++x) it.push_back({m, x, y, n * n * n * 16});   // cost ~ n^3 per element
        }
        // largest cost first, then member and position: CTAs that walk the list
        // round-robin end up with nearly equal work
        std::stable_sort(it.begin(), it.end(), [](const EnsItem &a, const EnsItem &b) { return a.cost > b.cost; });
        if (cudaMalloc(&e->items[ti], sizeof(EnsItem) * it.size()) != cudaSuccess)
            return efail(DG_ENOMEM, "cudaMalloc of the work list failed");
        ECUDA(cudaMemcpy(e->items[ti], it.data(), sizeof(EnsItem) * it.size(), cudaMemcpyHostToDevice));
        e->nitems[ti] = (int)it.size();
    }
    return DG_OK;
}

dg_status check_member(dg_ens *e, int m)
{
    if (!e) return efail(DG_EINVAL, "NULL ensemble");
    if (m < 0 || m >= e->nm) return efail(DG_EINVAL, "member %d of %d", m, e ? e->nm : 0);
    return DG_OK;
}

}  // namespace

int dg_ensemble_tile_width(int n) { return 32 / n; }

extern "C" {

dg_status dg_ensemble_create(int members, const int *nlon, const int *nlat, const int *degree, double radius,
                             double g, double omega, dg_ensemble *out)
{
    if (!out) return efail(DG_EINVAL, "out is NULL");
    *out = nullptr;
    if (members < 1 || !nlon || !nlat || !degree) return efail(DG_EINVAL, "need members >= 1 and the size arrays");
    if (!(radius > 0) || !(g > 0) || !std::isfinite(omega)) return efail(DG_EINVAL, "radius and g must be positive");
    for (int m = 0; m < members; ++m)
        if (nlon[m] < 1 || nlat[m] < 2 || degree[m] < 0 || degree[m] > DG_MAXN - 1)
            return efail(DG_EINVAL, "member %d: bad mesh %d x %d degree %d", m, nlon[m], nlat[m], degree[m]);
    dg_ens *e = new (std::nothrow) dg_ens;
    if (!e) return efail(DG_ENOMEM, "host allocation failed");
    e->nm = members;
    e->R = radius;
    e->g = g;
    e->omega = omega;
    e->nlon.assign(nlon, nlon + members);
    e->nlat.assign(nlat, nlat + members);
    e->deg.assign(degree, degree + members);
    e->href.assign(members, 0.0);
    e->dt.assign(members, 0.0);
    e->have.assign(members, 0);
    dg_status st = DG_OK;
#define ETRY(x)                    \
    do {                           \
        st = (x);                  \
        if (st) {                  \
            dg_ensemble_destroy(e); \
            return st;             \
        }                          \
    } while (0)
    if (cudaGetDevice(&e->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device) != cudaSuccess) {
        delete e;
        return efail(DG_ECUDA, "no CUDA device");
    }
    if (dg_ensure_basis(e->device)) {
        delete e;
        return efail(DG_ECUDA, "upload of the basis tables failed");
    }
    e->tabs.resize(members);
    size_t max_len = 0, rows_total = 0;
    for (int m = 0; m < members; ++m) {
        if (dg_build_tables(e->tabs[m], nlon[m], nlat[m], degree[m], radius, g)) ETRY(efail(DG_EINVAL, "tables"));
        const int n = degree[m] + 1;
        e->nel.push_back((size_t)nlon[m] * nlat[m]);
        e->off.push_back(e->total);
        // every member starts on a 128-byte boundary: the stage kernel loads
        // element rows as float2 / float4 vectors
        e->total += (e->nel[m] * 3 * n * n + 31) / 32 * 32;
        max_len = std::max(max_len, e->nel[m] * 3 * n * n);
        rows_total += nlat[m];
    }
    if (cudaStreamCreateWithFlags(&e->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        ETRY(efail(DG_ECUDA, "stream creation failed"));
    e->stream = e->own_stream;
    float **bufs[] = {&e->B[0], &e->B[1], &e->L[0], &e->L[1], &e->I[0], &e->I[1]};
    for (float **b : bufs)
        if (cudaMalloc(b, sizeof(float) * e->total) != cudaSuccess)
            ETRY(efail(DG_ENOMEM, "cudaMalloc of %zu floats failed", e->total));
    if (cudaMalloc(&e->stage64, sizeof(double) * max_len) != cudaSuccess) ETRY(efail(DG_ENOMEM, "cudaMalloc failed"));
    // concatenated FP32 row tables, member table, mass tables
    {
        std::vector<RowTab<float>> rt;
        rt.reserve(rows_total);
        std::vector<double> c0;
        e->hm.resize(members);
        for (int m = 0; m < members; ++m) {
            const int n = degree[m] + 1;
            EnsMember<float> &x = e->hm[m];
            std::memset(&x, 0, sizeof x);
            x.off = (long long)e->off[m];
            x.rows = (int)rt.size();
            x.nlon = nlon[m];
            x.nlat = nlat[m];
            x.n = n;
            x.cF = (float)(2.0 / (radius * e->tabs[m].dlam));
            x.cG = (float)(2.0 / (radius * e->tabs[m].dth));
            for (int j = 0; j < nlat[m]; ++j) {
                const RowTab<double> &s = e->tabs[m].rows[j];
                RowTab<float> d;
                std::memset(&d, 0, sizeof d);
                for (int a = 0; a < DG_MAXN; ++a) {
                    d.cosn[a] = (float)s.cosn[a];
                    d.sinn[a] = (float)s.sinn[a];
                    d.rho[a] = (float)s.rho[a];
                    d.CSE[a] = (float)s.CSE[a];
                    d.CSW[a] = (float)s.CSW[a];
                    for (int b = 0; b < DG_MAXN; ++b) {
                        d.Ci[a][b] = (float)s.Ci[a][b];
                        d.Q[a][b] = (float)s.Q[a][b];
                        d.QT[a][b] = (float)s.QT[a][b];
                        d.PT[a][b] = (float)s.PT[a][b];
                    }
                }
                d.ce_s = (float)s.ce_s;
                d.ce_n = (float)s.ce_n;
                rt.push_back(d);
            }
            e->c0_off.push_back(c0.size());
            for (int j = 0; j < nlat[m]; ++j)
                for (int b = 0; b < n; ++b) c0.push_back(e->tabs[m].C[(size_t)j * n * n + b]);
            for (int j = 0; j < nlat[m]; ++j) {
                const double tb = -0.5 * M_PI + j * e->tabs[m].dth;
                c0.push_back(std::sin(tb + e->tabs[m].dth) - std::sin(tb));
            }
        }
        if (cudaMalloc(&e->rows, sizeof(RowTab<float>) * rt.size()) != cudaSuccess ||
            cudaMalloc(&e->dm, sizeof(EnsMember<float>) * members) != cudaSuccess ||
            cudaMalloc(&e->c0, sizeof(double) * c0.size()) != cudaSuccess)
            ETRY(efail(DG_ENOMEM, "cudaMalloc of the tables failed"));
        if (cudaMemcpy(e->rows, rt.data(), sizeof(RowTab<float>) * rt.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(e->c0, c0.data(), sizeof(double) * c0.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            ETRY(efail(DG_ECUDA, "table upload failed"));
    }
    ETRY(build_items(e));
    size_t max_nel = *std::max_element(e->nel.begin(), e->nel.end());
    e->nblocks = dg_mass_blocks(max_nel);
    if (cudaMalloc(&e->partials, 2 * sizeof(double) * e->nblocks) != cudaSuccess ||
        cudaMalloc(&e->d_result, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&e->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&e->d_maxbits, sizeof(unsigned long long)) != cudaSuccess)
        ETRY(efail(DG_ENOMEM, "cudaMalloc failed"));
    if (cudaMemset(e->d_status, 0, sizeof(unsigned)) != cudaSuccess) ETRY(efail(DG_ECUDA, "cudaMemset failed"));
    // the device table must exist before the first launch
    ETRY(upload_members(e));
#undef ETRY
    *out = e;
    return DG_OK;
}

dg_status dg_ensemble_destroy(dg_ensemble e)
{
    if (!e) return DG_OK;
    if (e->stream) cudaStreamSynchronize(e->stream);
    drop_graphs(e);
    for (float *b : {e->B[0], e->B[1], e->L[0], e->L[1], e->I[0], e->I[1]}) cudaFree(b);
    cudaFree(e->stage64);
    cudaFree(e->rows);
    cudaFree(e->dm);
    cudaFree(e->items[0]);
    cudaFree(e->items[1]);
    cudaFree(e->c0);
    cudaFree(e->partials);
    cudaFree(e->d_result);
    cudaFree(e->d_status);
    cudaFree(e->d_maxbits);
    if (e->own_stream) cudaStreamDestroy(e->own_stream);
    for (auto &t : e->tabs) dg_free_tables(t);
    delete e;
    return DG_OK;
}

size_t dg_ensemble_state_len(dg_ensemble e, int member)
{
    if (!e || member < 0 || member >= e->nm) return 0;
    const int n = e->deg[member] + 1;
    return e->nel[member] * 3 * n * n;
}

size_t dg_ensemble_total_dof(dg_ensemble e)
{
    if (!e) return 0;
    size_t d = 0;
    for (int m = 0; m < e->nm; ++m) d += dg_ensemble_state_len(e, m);
    return d;
}

long long dg_ensemble_stage_launches(dg_ensemble e) { return e ? e->launches : 0; }

dg_status dg_ensemble_set_option(dg_ensemble e, int key, long long value)
{
    if (!e) return efail(DG_EINVAL, "NULL ensemble");
    switch (key) {
    case DG_OPT_STREAM:
        ECUDA(cudaStreamSynchronize(e->stream));
        e->stream = value ? reinterpret_cast<cudaStream_t>(value) : e->own_stream;
        drop_graphs(e);
        return DG_OK;
    case DG_OPT_STEPS_PER_GRAPH:
        if (value < 1 || value > 1024) return efail(DG_EINVAL, "steps per graph must be 1..1024");
        e->spg = (int)value;
        return DG_OK;
    case DG_OPT_TILE_ROWS:
        if (value != DG_ENS_TILE_ROWS_A && value != DG_ENS_TILE_ROWS_B)
            return efail(DG_EINVAL, "tile rows must be %d or %d", DG_ENS_TILE_ROWS_A, DG_ENS_TILE_ROWS_B);
        e->tile_rows = (int)value;
        drop_graphs(e);
        return DG_OK;
    case DG_OPT_BLOCKS_PER_SM:
        if (value < 1 || value > 8) return efail(DG_EINVAL, "blocks per SM must be 1..8");
        e->bps = (int)value;
        drop_graphs(e);
        return DG_OK;
    default:
        return efail(DG_EINVAL, "option %d does not apply to an ensemble", key);
    }
}

dg_status dg_ensemble_set_state(dg_ensemble e, int member, const double *modal, size_t len)
{
    if (dg_status s = check_member(e, member)) return s;
    if (!modal || len != dg_ensemble_state_len(e, member)) return efail(DG_EINVAL, "bad state length");
    const int n = e->deg[member] + 1;
    double s = 0.0;
    for (size_t k = 0; k < e->nel[member]; ++k) s += modal[k * 3 * n * n];
    e->href[member] = 0.5 * s / (double)e->nel[member];
    e->members_dirty = true;
    ECUDA(cudaMemcpyAsync(e->stage64, modal, len * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    if (dg_launch_to_internal<float>(e->stage64, e->B[e->cur] + e->off[member], e->L[e->cur] + e->off[member],
                                     e->nel[member], n * n, e->href[member], e->stream))
        return efail(DG_ECUDA, "conversion failed");
    ECUDA(cudaStreamSynchronize(e->stream));
    e->have[member] = 1;
    return DG_OK;
}

dg_status dg_ensemble_get_state(dg_ensemble e, int member, double *modal, size_t len)
{
    if (dg_status s = check_member(e, member)) return s;
    if (!modal || len != dg_ensemble_state_len(e, member)) return efail(DG_EINVAL, "bad state length");
    const int n = e->deg[member] + 1;
    if (dg_launch_to_api<float>(e->B[e->cur] + e->off[member], e->L[e->cur] + e->off[member], e->stage64,
                                e->nel[member], n * n, e->href[member], e->stream))
        return efail(DG_ECUDA, "conversion failed");
    ECUDA(cudaMemcpyAsync(modal, e->stage64, len * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    return DG_OK;
}

dg_status dg_ensemble_set_dt(dg_ensemble e, const double *dt, int members)
{
    if (!e) return efail(DG_EINVAL, "NULL ensemble");
    if (!dt || members != e->nm) return efail(DG_EINVAL, "need one time step per member");
    for (int m = 0; m < members; ++m)
        if (!(dt[m] > 0) || !std::isfinite(dt[m])) return efail(DG_EINVAL, "member %d: dt must be positive", m);
    e->dt.assign(dt, dt + members);
    e->members_dirty = true;
    return DG_OK;
}

dg_status dg_ensemble_step(dg_ensemble e, int n)
{
    if (!e) return efail(DG_EINVAL, "NULL ensemble");
    if (n < 0) return efail(DG_EINVAL, "n must be >= 0");
    for (int m = 0; m < e->nm; ++m) {
        if (!e->have[m]) return efail(DG_EINVAL, "member %d has no state", m);
        if (!(e->dt[m] > 0)) return efail(DG_EINVAL, "member %d has no time step (dg_ensemble_set_dt)", m);
    }
    if (n == 0) return DG_OK;
    if (dg_status s = upload_members(e)) return s;
    int K = std::min(e->spg, n);
    if ((K & 1) && K > 1) K -= 1;
    const int full = n / K, rest = n - full * K;
    if (full > 0) {
        dg_ens::Graph *ge = nullptr;
        for (auto &g : e->graphs)
            if (g.steps == K && g.cur_in == e->cur && g.tile_rows == e->tile_rows && g.bps == e->bps &&
                g.stream == e->stream)
                ge = &g;
        if (!ge) {
            dg_ens::Graph g;
            g.steps = K;
            g.cur_in = e->cur;
            g.tile_rows = e->tile_rows;
            g.bps = e->bps;
            g.stream = e->stream;
            int cur = e->cur;
            const long long before = e->launches;
            ECUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
            dg_status st = DG_OK;
            for (int k = 0; k < K && !st; ++k) {
                st = launch_step(e, cur);
                cur ^= 1;
            }
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
            e->launches = before;
            if (st) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ce != cudaSuccess) return efail(DG_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return efail(DG_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
            g.cur_out = cur;
            e->graphs.push_back(g);
            ge = &e->graphs.back();
        }
        for (int r = 0; r < full; ++r) {
            ECUDA(cudaGraphLaunch(ge->exec, e->stream));
            e->launches += 3LL * K;
            e->cur = ge->cur_out;
        }
    }
    for (int k = 0; k < rest; ++k) {
        if (dg_status st = launch_step(e, e->cur)) return st;
        e->cur ^= 1;
    }
    unsigned st = 0;
    ECUDA(cudaMemcpyAsync(&st, e->d_status, sizeof st, cudaMemcpyDeviceToHost, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    if (st) {
        ECUDA(cudaMemset(e->d_status, 0, sizeof(unsigned)));
        if (st & DG_STATUS_NONPHYSICAL) return efail(DG_ENONPHYSICAL, "h <= 0 at a quadrature point");
        return efail(DG_ENONFINITE, "non-finite value in the state");
    }
    return DG_OK;
}

dg_status dg_ensemble_total_mass(dg_ensemble e, int member, double *mass)
{
    if (dg_status s = check_member(e, member)) return s;
    if (!mass) return efail(DG_EINVAL, "mass is NULL");
    const int n = e->deg[member] + 1;
    const HostTables &t = e->tabs[member];
    if (dg_launch_mass<float>(e->B[e->cur] + e->off[member], e->L[e->cur] + e->off[member], e->c0 + e->c0_off[member],
                              e->nlon[member], e->nlat[member], n, e->href[member], t.dlam, t.dth, e->R * e->R,
                              e->partials, e->nblocks, e->d_result, nullptr, e->stream))
        return efail(DG_ECUDA, "mass kernel failed");
    ECUDA(cudaMemcpyAsync(mass, e->d_result, sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    return DG_OK;
}

dg_status dg_ensemble_max_dt(dg_ensemble e, int member, double cfl, double *dt)
{
    if (dg_status s = check_member(e, member)) return s;
    if (!dt || !(cfl > 0)) return efail(DG_EINVAL, "need cfl > 0 and dt != NULL");
    const int n = e->deg[member] + 1;
    ECUDA(cudaMemsetAsync(e->d_maxbits, 0, sizeof(unsigned long long), e->stream));
    if (dg_launch_max_speed<float>(e->B[e->cur] + e->off[member], e->nlon[member], e->nlat[member], n,
                                   e->href[member], e->g, e->d_maxbits, e->d_status, e->stream))
        return efail(DG_ECUDA, "wave-speed kernel failed");
    unsigned long long bits = 0;
    ECUDA(cudaMemcpyAsync(&bits, e->d_maxbits, sizeof bits, cudaMemcpyDeviceToHost, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    double c;
    std::memcpy(&c, &bits, sizeof c);
    if (!(c > 0)) return efail(DG_ENONPHYSICAL, "no positive wave speed");
    const HostTables &t = e->tabs[member];
    double H = INFINITY;
    for (int j = 0; j < e->nlat[member]; ++j)
        for (int q = 0; q < n; ++q) H = std::min(H, std::min(e->R * t.dth, e->R * t.rows[j].cosn[q] * t.dlam));
    *dt = cfl * H / (std::max(e->deg[member], 1) * c);
    return DG_OK;
}

// Time `trials` steps for every (tile rows, blocks per SM) candidate on the
// ensemble's own state (saved and restored around the trials) and keep the
// fastest.  Returns the choice in *tile_rows and *blocks_per_sm.
dg_status dg_ensemble_autotune(dg_ensemble e, int trials, int *tile_rows, int *blocks_per_sm, double *best_ms)
{
    if (!e) return efail(DG_EINVAL, "NULL ensemble");
    if (trials < 1) return efail(DG_EINVAL, "trials must be >= 1");
    for (int m = 0; m < e->nm; ++m)
        if (!e->have[m] || !(e->dt[m] > 0)) return efail(DG_EINVAL, "member %d needs a state and a time step", m);
    // save u^n (the trials advance it)
    float *saveB = nullptr, *saveL = nullptr;
    if (cudaMalloc(&saveB, sizeof(float) * e->total) != cudaSuccess ||
        cudaMalloc(&saveL, sizeof(float) * e->total) != cudaSuccess) {
        cudaFree(saveB);
        return efail(DG_ENOMEM, "cudaMalloc for the autotuner failed");
    }
    const int cur0 = e->cur;
    ECUDA(cudaMemcpyAsync(saveB, e->B[cur0], sizeof(float) * e->total, cudaMemcpyDeviceToDevice, e->stream));
    ECUDA(cudaMemcpyAsync(saveL, e->L[cur0], sizeof(float) * e->total, cudaMemcpyDeviceToDevice, e->stream));
    cudaEvent_t a, b;
    ECUDA(cudaEventCreate(&a));
    ECUDA(cudaEventCreate(&b));
    const int rows_opts[2] = {DG_ENS_TILE_ROWS_A, DG_ENS_TILE_ROWS_B};
    double best = INFINITY;
    int best_w = e->tile_rows, best_b = e->bps;
    dg_status st = DG_OK;
    for (int w : rows_opts) {
        for (int bpsm = 1; bpsm <= 4 && !st; ++bpsm) {
            e->tile_rows = w;
            e->bps = bpsm;
            drop_graphs(e);
            st = dg_ensemble_step(e, 2);   // capture + warm-up
            if (st) break;
            cudaEventRecord(a, e->stream);
            st = dg_ensemble_step(e, trials);
            cudaEventRecord(b, e->stream);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (!st && ms < best) {
                best = ms;
                best_w = w;
                best_b = bpsm;
            }
        }
    }
    e->tile_rows = best_w;
    e->bps = best_b;
    drop_graphs(e);
    e->cur = cur0;
    cudaMemcpyAsync(e->B[cur0], saveB, sizeof(float) * e->total, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(e->L[cur0], saveL, sizeof(float) * e->total, cudaMemcpyDeviceToDevice, e->stream);
    cudaStreamSynchronize(e->stream);
    cudaFree(saveB);
    cudaFree(saveL);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    if (tile_rows) *tile_rows = best_w;
    if (blocks_per_sm) *blocks_per_sm = best_b;
    if (best_ms) *best_ms = best / trials;
    return DG_OK;
}

}  // extern "C"

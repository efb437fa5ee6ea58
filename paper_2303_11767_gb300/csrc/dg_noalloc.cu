// dg_noalloc.cu -- dg_max_dt_noalloc: the CFL time step of a device-resident
// FP64 state without any device allocation.
//
// Callers that cannot allocate device memory -- code running while a CUDA
// graph is being captured (cudaMalloc is not allowed there), or a host
// application whose memory manager owns the whole device and forbids foreign
// cudaMalloc calls -- cannot create a dg_handle, because dg_create allocates
// the solver's buffers.  This entry point gives them the time step of a state
// they already hold on the device.  Its only scratch is the fixed array below,
// which lives in the library image: every GPU that loads the library holds it
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "dg_internal.h"
#include "../../include/dgswe.h"

// Scratch: one slot per latitude row for the row maximum of the wave speed
// (bit pattern of a positive double), plus one status word at the end.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[DG_NOALLOC_MAX_NLAT + 1];

// L_a at the n Gauss points, for n = 1..DG_MAXN (this file's own copy).
__constant__ double c_na_LV[DG_MAXN][DG_MAXN][DG_MAXN];

namespace {

// One block per latitude row: largest sqrt(u^2 + v^2) + sqrt(g h) over the
// Gauss points of the row's elements, written to the row's slot (every slot
// of the rows in use is overwritten, so nothing there needs clearing).
template <int N>
__global__ void noalloc_row_speed(const double *__restrict__ u, int nlon, double g,
                                  unsigned long long *__restrict__ scratch, int status_slot)
{
    const int j = blockIdx.x;
    const double(&LV)[DG_MAXN][DG_MAXN] = c_na_LV[N - 1];
    double best = 0.0;
    unsigned bad = 0;
    for (int i = threadIdx.x; i < nlon; i += blockDim.x) {
        const double *ue = u + ((size_t)j * nlon + i) * 3 * N * N;
        for (int q = 0; q < N; ++q)
            for (int r = 0; r < N; ++r) {
                double qv[3];
                for (int f = 0; f < 3; ++f) {
                    double s = 0.0;
                    for (int b = 0; b < N; ++b) {
                        double t = 0.0;
                        for (int a = 0; a < N; ++a) t += LV[a][r] * ue[f * N * N + b * N + a];
                        s += LV[b][q] * t;
                    }
                    qv[f] = s;
                }
                const double h = qv[0];
                if (!(h > 0.0)) { bad = 1; continue; }
                const double uu = qv[1] / h, vv = qv[2] / h;
                const double sp = sqrt(uu * uu + vv * vv) + sqrt(g * h);
                // a NaN or Inf in hu or hv makes the speed non-finite, and
                // fmax would silently drop it
                if (!isfinite(sp)) { bad = 1; continue; }
                best = fmax(best, sp);
            }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmax(m, red[w]);
        scratch[j] = (unsigned long long)__double_as_longlong(m);
    }
    if (bad) atomicOr(&scratch[status_slot], 1ull);
}

// Single block: maximum over the rows, then dt = cfl H / (max(p,1) c);
// writes -1 when some Gauss point had h <= 0, a NaN depth or a non-finite
// wave speed (a NaN or Inf in hu or hv).
__global__ void noalloc_finish(const unsigned long long *__restrict__ scratch, int nlat, int status_slot,
                               double cfl_H_over_p, double *__restrict__ dt_out)
{
    __shared__ double red[32];
    double m = 0.0;
    for (int j = threadIdx.x; j < nlat; j += blockDim.x) m = fmax(m, __longlong_as_double((long long)scratch[j]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) c = fmax(c, red[w]);
        const bool bad = scratch[status_slot] != 0ull || !(c > 0.0);
        *dt_out = bad ? -1.0 : cfl_H_over_p / c;
    }
}

// Per-device set-up: the device address of the scratch array and the basis
// table, done once per device on the first call (with that device current).
// Host threads that make their first call on the same device at the same
// time are serialised by g_setup_mu, so none of them can see the device
// marked done before its scratch address is stored.  The cached address
// belongs to the device's primary context: after cudaDeviceReset on that
// device the module is loaded again and the address (and the constant basis
// table) must be set up anew, which this file does not detect; a process
// that resets a device must not call dg_max_dt_noalloc on it afterwards.
struct DeviceSetup {
    bool done = false;
    unsigned long long *scratch = nullptr;
};
DeviceSetup g_setup[64];
std::mutex g_setup_mu;

dg_status setup_device(int dev, unsigned long long **scratch, const char **why)
{
    if (dev < 0 || dev >= 64) {
        *why = "device index outside the 64 devices this entry point supports";
        return DG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *why = cudaGetErrorString(e);
            return DG_ECUDA;
        }
        double lv[DG_MAXN][DG_MAXN][DG_MAXN];
        std::memset(lv, 0, sizeof lv);
        for (int n = 1; n <= DG_MAXN; ++n) {
            double x[DG_MAXN], w[DG_MAXN];
            dg_gauss_legendre(n, x, w);
            for (int a = 0; a < n; ++a)
                for (int q = 0; q < n; ++q) lv[n - 1][a][q] = dg_legendre(a, x[q]);
        }
        e = cudaMemcpyToSymbol(c_na_LV, lv, sizeof lv);
        if (e != cudaSuccess) {
            *why = cudaGetErrorString(e);
            return DG_ECUDA;
        }
        s.scratch = static_cast<unsigned long long *>(ptr);
        s.done = true;
    }
    *scratch = s.scratch;
    return DG_OK;
}

dg_status noalloc_fail(dg_status st, const char *what)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "dg_max_dt_noalloc: %s", what);
    dg_set_last_error(buf);
    return st;
}

}  // namespace

extern "C" dg_status dg_max_dt_noalloc(const double *d_modal, int nlon, int nlat, int degree, double radius,
                                       double g, double cfl, double *d_dt, void *stream)
{
    if (!d_modal || !d_dt || nlon < 1 || nlat < 2 || degree < 0 || degree > DG_MAXN - 1 || !(radius > 0) ||
        !(g > 0) || !(cfl > 0))
        return noalloc_fail(DG_EINVAL, "invalid argument (null pointer, mesh, degree, radius, g or cfl)");
    if (nlat > DG_NOALLOC_MAX_NLAT) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "nlat = %d exceeds the scratch limit of %d rows", nlat, DG_NOALLOC_MAX_NLAT);
        return noalloc_fail(DG_EINVAL, buf);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(DG_ECUDA, "no CUDA device");
    unsigned long long *scratch = nullptr;
    const char *why = "";
    if (dg_status st = setup_device(dev, &scratch, &why)) return noalloc_fail(st, why);
    // H = min over rows and Gauss points of min(R dth, R cos(theta) dlam)
    const int n = degree + 1;
    double x[DG_MAXN], w[DG_MAXN];
    dg_gauss_legendre(n, x, w);
    const double dlam = 2.0 * M_PI / nlon, dth = M_PI / nlat;
    double H = radius * dth;
    for (int j = 0; j < nlat; ++j)
        for (int q = 0; q < n; ++q)
            H = std::fmin(H, radius * std::cos(-0.5 * M_PI + (j + 0.5 * (1.0 + x[q])) * dth) * dlam);
    const double num = cfl * H / (degree > 1 ? degree : 1);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int status_slot = DG_NOALLOC_MAX_NLAT;
    if (cudaMemsetAsync(scratch + status_slot, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return noalloc_fail(DG_ECUDA, cudaGetErrorString(cudaGetLastError()));
    switch (n) {
    case 1: noalloc_row_speed<1><<<nlat, 128, 0, s>>>(d_modal, nlon, g, scratch, status_slot); break;
    case 2: noalloc_row_speed<2><<<nlat, 128, 0, s>>>(d_modal, nlon, g, scratch, status_slot); break;
    case 3: noalloc_row_speed<3><<<nlat, 128, 0, s>>>(d_modal, nlon, g, scratch, status_slot); break;
    case 4: noalloc_row_speed<4><<<nlat, 128, 0, s>>>(d_modal, nlon, g, scratch, status_slot); break;
    default: noalloc_row_speed<5><<<nlat, 128, 0, s>>>(d_modal, nlon, g, scratch, status_slot); break;
    }
    noalloc_finish<<<1, 256, 0, s>>>(scratch, nlat, status_slot, num, d_dt);
    if (cudaPeekAtLastError() != cudaSuccess) return noalloc_fail(DG_ECUDA, cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
}

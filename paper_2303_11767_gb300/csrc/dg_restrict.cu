// dg_restrict.cu -- cos(theta)-weighted L2 projection of a fine-mesh modal
// state onto a nested coarse mesh (each coarse element made of r x r fine
// elements), in FP64 on the GPU: the coarse modes solve
//   M_c u_c = int u_fine phi_c cos(theta) dlambda dtheta
// over the coarse element, the integral taken element by element of the fine
// mesh with a Gauss rule that is exact for the polynomial part.
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace {

constexpr int RQ = 8;          // Gauss points per direction and fine element
constexpr int RTHREADS = 128;

__device__ __forceinline__ void coarse_basis(int n, double x, double *L)
{
    // orthonormal Legendre by the recurrence of the library's tables
    L[0] = 0.70710678118654752440;
    double prev = 0.0, a_prev = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        const double a = sqrt((2.0 * k + 1.0) * (2.0 * k + 3.0)) / (k + 1.0);
        const double r = k > 0 ? a / a_prev : 0.0;
        const double next = a * x * L[k] - r * prev;
        prev = L[k];
        L[k + 1] = next;
        a_prev = a;
    }
}

__global__ void __launch_bounds__(RTHREADS) restrict_kernel(const double *__restrict__ fine, int fnlon, int fn,
                                                            double *__restrict__ coarse, int cnlon, int cn, int r,
                                                            const RowTab<double> *__restrict__ crows,
                                                            RestrictTab tab)
{
    __shared__ double red[RTHREADS];
    const int ce = blockIdx.x;
    const int J = ce / cnlon, I = ce - J * cnlon;
    const int fnp = fn * fn, cnp = cn * cn;
    double mom[3 * DG_MAXN * DG_MAXN];
    for (int t = 0; t < 3 * cnp; ++t) mom[t] = 0.0;
    const int items = r * r * RQ * RQ;
    for (int it = threadIdx.x; it < items; it += RTHREADS) {
        const int sub = it / (RQ * RQ), q = it - sub * (RQ * RQ);
        const int sj = sub / r, si = sub - sj * r, qy = q / RQ, qx = q - qy * RQ;
        const int fj = J * r + sj, fi = I * r + si;
        const double *u = fine + ((size_t)fj * fnlon + fi) * 3 * fnp;
        double val[3];
        for (int f = 0; f < 3; ++f) {
            double s = 0.0;
            for (int b = 0; b < fn; ++b) {
                double t = 0.0;
                for (int a = 0; a < fn; ++a) t += u[f * fnp + b * fn + a] * tab.LVf[a][qx];
                s += t * tab.LVf[b][qy];
            }
            val[f] = s;
        }
        const double xc = -1.0 + (2.0 * si + 1.0 + tab.x[qx]) / r;
        const double yc = -1.0 + (2.0 * sj + 1.0 + tab.x[qy]) / r;
        double Lx[DG_MAXN], Ly[DG_MAXN];
        coarse_basis(cn, xc, Lx);
        coarse_basis(cn, yc, Ly);
        const double theta = -0.5 * M_PI + (J + 0.5 * (1.0 + yc)) * tab.dthc;
        const double w = tab.w[qx] * tab.w[qy] * tab.jf * cos(theta);
        for (int f = 0; f < 3; ++f)
            for (int b = 0; b < cn; ++b)
                for (int a = 0; a < cn; ++a) mom[(f * cn + b) * cn + a] += w * val[f] * Lx[a] * Ly[b];
    }
    // fixed-order block reduction of every moment, then the coarse mass matrix
    double total[3 * DG_MAXN * DG_MAXN];
    for (int t = 0; t < 3 * cnp; ++t) {
        red[threadIdx.x] = mom[t];
        __syncthreads();
        for (int s = RTHREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        total[t] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const RowTab<double> &rt = crows[J];
        double *out = coarse + (size_t)ce * 3 * cnp;
        for (int f = 0; f < 3; ++f)
            for (int b = 0; b < cn; ++b)
                for (int a = 0; a < cn; ++a) {
                    double s = 0.0;
                    for (int c = 0; c < cn; ++c) s += rt.Ci[b][c] * total[(f * cn + c) * cn + a];
                    out[(f * cn + b) * cn + a] = tab.inv_jc * s;
                }
    }
}

}  // namespace

int dg_launch_restrict(const double *fine, int fnlon, int fn, double *coarse, int cnlon, int cnlat, int cn, int r,
                       const RowTab<double> *crows, const RestrictTab &tab, void *stream)
{
    restrict_kernel<<<cnlon * cnlat, RTHREADS, 0, static_cast<cudaStream_t>(stream)>>>(fine, fnlon, fn, coarse, cnlon,
                                                                                       cn, r, crows, tab);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

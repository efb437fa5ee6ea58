// dg_plane.cu -- the paper's planar validation problem (Sec. 4.1, Eq.
// lin_adv): linear advection du/dt + div(beta u) = 0 of one scalar on the unit
// square, periodic in both directions, with the same modal DG discretisation
// as the sphere (orthonormal Legendre basis, n = p + 1 Gauss points per
// direction, Rusanov flux, lift) and the same increment-form RK stages.
// FP64, one thread per element: it exists to pin the DG machinery against
// the convergence tables the paper prints, not for speed.
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace {

template <int N>
__global__ void __launch_bounds__(128) plane_stage_kernel(const PlaneArgs P)
{
    constexpr int NP = N * N;
    const StageArgs<double> &A = P.s;
    const BasisTab<double> &B = P.basis;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.nx * P.ny) return;
    const int j = e / P.nx, i = e - j * P.nx;
    auto load = [&](int jj, int ii, double *u) {
        const size_t o = ((size_t)jj * P.nx + ii) * NP;
#pragma unroll
        for (int m = 0; m < NP; ++m) u[m] = A.base[o + m] + (A.inc ? A.inc[o + m] : 0.0);
    };
    double u[NP], nb[NP];
    load(j, i, u);

    // values at the Gauss points q[beta][alpha]
    double q[N][N];
#pragma unroll
    for (int be = 0; be < N; ++be)
#pragma unroll
        for (int al = 0; al < N; ++al) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < N; ++b) {
                double t = 0.0;
#pragma unroll
                for (int a = 0; a < N; ++a) t += B.LV[a][al] * u[b * N + a];
                s += B.LV[b][be] * t;
            }
            q[be][al] = s;
        }
    // volume term with the inverse mass matrix (4 / (dx dy)) I folded in:
    //   k[b][a] = sum_q q (bx cx w L_a' w L_b + by cy w L_a w L_b')
    double k[NP];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int a = 0; a < N; ++a) {
            double s = 0.0;
#pragma unroll
            for (int be = 0; be < N; ++be)
#pragma unroll
                for (int al = 0; al < N; ++al)
                    s += q[be][al] * (P.bx * P.cx * B.WLD[a][al] * B.WLV[b][be] +
                                      P.by * P.cy * B.WLV[a][al] * B.WLD[b][be]);
            k[b * N + a] = s;
        }

    // Rusanov flux f* . n at the n points of each edge (own state o, neighbour
    // state v across the edge, outward normal component bn = beta . n):
    //   f* . n = bn (o + v) / 2 - alpha / 2 (v - o)
    const double speed = sqrt(P.bx * P.bx + P.by * P.by);
    auto rusanov = [&](double o, double v, double bn) {
        const double alpha = P.alpha_speed ? speed : fabs(bn);
        return 0.5 * bn * (o + v) - 0.5 * alpha * (v - o);
    };
    // lambda (x) edges: W at xi = -1 against the west neighbour's xi = +1
    // trace, E at +1 against the east neighbour's -1 trace; lift c_x w_k L_b(eta_k) L_a(+-1)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int ii = side == 0 ? (i - 1 + P.nx) % P.nx : (i + 1) % P.nx;
        load(j, ii, nb);
        const double bn = side == 0 ? -P.bx : P.bx;
#pragma unroll
        for (int kk = 0; kk < N; ++kk) {
            double o = 0.0, v = 0.0;
#pragma unroll
            for (int b = 0; b < N; ++b) {
                double so = 0.0, sv = 0.0;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    so += (side == 0 ? B.SW[a] : B.SE[a]) * u[b * N + a];
                    sv += (side == 0 ? B.SE[a] : B.SW[a]) * nb[b * N + a];
                }
                o += B.LV[b][kk] * so;
                v += B.LV[b][kk] * sv;
            }
            const double fs = rusanov(o, v, bn);
#pragma unroll
            for (int b = 0; b < N; ++b)
#pragma unroll
                for (int a = 0; a < N; ++a)
                    k[b * N + a] -= P.cx * B.WLV[b][kk] * (side == 0 ? B.SW[a] : B.SE[a]) * fs;
        }
    }
    // theta (y) edges: S at eta = -1, N at eta = +1, periodic
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int jj = side == 0 ? (j - 1 + P.ny) % P.ny : (j + 1) % P.ny;
        load(jj, i, nb);
        const double bn = side == 0 ? -P.by : P.by;
#pragma unroll
        for (int kk = 0; kk < N; ++kk) {
            double o = 0.0, v = 0.0;
#pragma unroll
            for (int b = 0; b < N; ++b) {
                double so = 0.0, sv = 0.0;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    so += B.LV[a][kk] * u[b * N + a];
                    sv += B.LV[a][kk] * nb[b * N + a];
                }
                o += (side == 0 ? B.SW[b] : B.SE[b]) * so;
                v += (side == 0 ? B.SE[b] : B.SW[b]) * sv;
            }
            const double fs = rusanov(o, v, bn);
#pragma unroll
            for (int b = 0; b < N; ++b)
#pragma unroll
                for (int a = 0; a < N; ++a)
                    k[b * N + a] -= P.cy * B.WLV[a][kk] * (side == 0 ? B.SW[b] : B.SE[b]) * fs;
        }
    }

    // the increment-form RK combination of the sphere stage (FP64: no low part)
    unsigned st = 0;
    const size_t o0 = (size_t)e * NP;
    const double cdt = A.cc * A.dt, adt = A.ca * A.dt;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const size_t o = o0 + m;
        const double kv = k[m];
        if (!isfinite(kv)) st |= DG_STATUS_NONFINITE;
        if (A.out_rhs) A.out_rhs[o] = kv;
        const double inc = A.inc ? A.inc[o] : 0.0;
        if (A.inc_out) A.inc_out[o] = fma(cdt, kv, A.ci * inc);
        const double acc = A.acc_in ? A.acc_in[o] : 0.0;
        if (A.acc_out) A.acc_out[o] = fma(adt, kv, acc);
        if (A.out_base) {
            const double hi = A.base[o] + fma(cdt, kv, fma(A.cd, acc, A.ci * inc));
            A.out_base[o] = hi;
            if (!isfinite(hi)) st |= DG_STATUS_NONFINITE;
        }
    }
    if (st) atomicOr(A.status, st);
}

}  // namespace

int dg_launch_stage_plane(int n, const PlaneArgs &p, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nel = p.nx * p.ny, threads = 128, blocks = (nel + threads - 1) / threads;
    switch (n) {
    case 1: plane_stage_kernel<1><<<blocks, threads, 0, s>>>(p); break;
    case 2: plane_stage_kernel<2><<<blocks, threads, 0, s>>>(p); break;
    case 3: plane_stage_kernel<3><<<blocks, threads, 0, s>>>(p); break;
    case 4: plane_stage_kernel<4><<<blocks, threads, 0, s>>>(p); break;
    case 5: plane_stage_kernel<5><<<blocks, threads, 0, s>>>(p); break;
    default: return 1;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

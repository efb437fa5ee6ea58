// dg_plane.cu -- the paper's planar problems on a doubly periodic square,
// with the same modal DG discretisation as the sphere (orthonormal Legendre
// basis, n = p + 1 Gauss points per direction, Rusanov flux, lift, planar
// mass matrix (dx dy / 4) I) and the same increment-form RK stages:
//   * linear advection du/dt + div(beta u) = 0 of one scalar (Sec. 4.1, Eq.
//     lin_adv), the validation problem whose convergence tables the paper
//     prints;
//   * shallow water (h, hu, hv) on the f-plane (Sec. 4.3, the geostrophic
//     adjustment set-up, which is also the workload of the paper's timings).
// FP64, one thread per element: these pin the DG machinery, they are not the
// performance path.
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

// Shallow water on the f-plane: F = (hu, hu u + g h^2/2, hu v),
// G = (hv, hv u, hv v + g h^2/2), S = (0, f hv, -f hu); Rusanov alpha = the
// larger one-sided |u| + c (x faces) or |v| + c (y faces).
template <int N>
__global__ void __launch_bounds__(128) plane_swe_stage_kernel(const PlaneArgs P)
{
    constexpr int NP = N * N, EL = 3 * NP;
    const StageArgs<double> &A = P.s;
    const BasisTab<double> &B = P.basis;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.nx * P.ny) return;
    const int j = e / P.nx, i = e - j * P.nx;
    unsigned st = 0;
    auto at = [&](int jj, int ii, int c) {
        const size_t o = ((size_t)jj * P.nx + ii) * EL + c;
        return A.base[o] + (A.inc ? A.inc[o] : 0.0);
    };
    auto flux = [&](const double *q, double *F, double *G, double &su, double &sv) {
        const double h = q[0];
        if (!(h > 0.0)) st |= (h != h) ? DG_STATUS_NONFINITE : DG_STATUS_NONPHYSICAL;
        const double u = q[1] / h, v = q[2] / h, pr = 0.5 * P.g * h * h, c = sqrt(P.g * h);
        F[0] = q[1];
        F[1] = q[1] * u + pr;
        F[2] = q[1] * v;
        G[0] = q[2];
        G[1] = q[2] * u;
        G[2] = q[2] * v + pr;
        su = fabs(u) + c;
        sv = fabs(v) + c;
    };
    double u[EL], k[EL];
#pragma unroll
    for (int c = 0; c < EL; ++c) {
        u[c] = at(j, i, c);
        k[c] = 0.0;
    }
    // volume and source terms at the Gauss points (M^{-1} folded in)
#pragma unroll
    for (int be = 0; be < N; ++be)
#pragma unroll
        for (int al = 0; al < N; ++al) {
            double q[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                double s = 0.0;
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    double t = 0.0;
#pragma unroll
                    for (int a = 0; a < N; ++a) t += B.LV[a][al] * u[f * NP + b * N + a];
                    s += B.LV[b][be] * t;
                }
                q[f] = s;
            }
            double F[3], G[3], su, sv;
            flux(q, F, G, su, sv);
            const double S[3] = {0.0, P.fcor * q[2], -P.fcor * q[1]};
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int b = 0; b < N; ++b)
#pragma unroll
                    for (int a = 0; a < N; ++a)
                        k[f * NP + b * N + a] += F[f] * P.cx * B.WLD[a][al] * B.WLV[b][be] +
                                                 G[f] * P.cy * B.WLV[a][al] * B.WLD[b][be] +
                                                 S[f] * B.WLV[a][al] * B.WLV[b][be];
        }
    // faces: own trace against the neighbour's opposite trace, periodic
#pragma unroll
    for (int face = 0; face < 4; ++face) {   // 0 W, 1 E, 2 S, 3 N
        const bool xf = face < 2, plus = face & 1;
        const int ii = face == 0 ? (i - 1 + P.nx) % P.nx : face == 1 ? (i + 1) % P.nx : i;
        const int jj = face == 2 ? (j - 1 + P.ny) % P.ny : face == 3 ? (j + 1) % P.ny : j;
        const double sgn = plus ? 1.0 : -1.0;
#pragma unroll
        for (int kk = 0; kk < N; ++kk) {
            double qo[3], qb[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                double so = 0.0, sb = 0.0;
#pragma unroll
                for (int b = 0; b < N; ++b)
#pragma unroll
                    for (int a = 0; a < N; ++a) {
                        // own side: xi = +-1 (x faces) or eta = +-1 (y faces); the
                        // neighbour is evaluated at the opposite side of its element
                        const double wo = xf ? (plus ? B.SE[a] : B.SW[a]) * B.LV[b][kk]
                                             : B.LV[a][kk] * (plus ? B.SE[b] : B.SW[b]);
                        const double wb = xf ? (plus ? B.SW[a] : B.SE[a]) * B.LV[b][kk]
                                             : B.LV[a][kk] * (plus ? B.SW[b] : B.SE[b]);
                        so += wo * u[f * NP + b * N + a];
                        sb += wb * at(jj, ii, f * NP + b * N + a);
                    }
                qo[f] = so;
                qb[f] = sb;
            }
            double Fo[3], Go[3], Fb[3], Gb[3], suo, svo, sub, svb;
            flux(qo, Fo, Go, suo, svo);
            flux(qb, Fb, Gb, sub, svb);
            const double alpha = xf ? fmax(suo, sub) : fmax(svo, svb);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const double fo = sgn * (xf ? Fo[f] : Go[f]), fb = sgn * (xf ? Fb[f] : Gb[f]);
                const double fs = 0.5 * (fo + fb) - 0.5 * alpha * (qb[f] - qo[f]);
#pragma unroll
                for (int b = 0; b < N; ++b)
#pragma unroll
                    for (int a = 0; a < N; ++a)
                        k[f * NP + b * N + a] -= xf ? P.cx * B.WLV[b][kk] * (plus ? B.SE[a] : B.SW[a]) * fs
                                                    : P.cy * B.WLV[a][kk] * (plus ? B.SE[b] : B.SW[b]) * fs;
            }
        }
    }
    // the increment-form RK combination (FP64: no low part)
    const size_t o0 = (size_t)e * EL;
    const double cdt = A.cc * A.dt, adt = A.ca * A.dt;
#pragma unroll
    for (int m = 0; m < EL; ++m) {
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
    // one element per thread is FP64-throughput bound per SM: small meshes
    // (the paper's 50x50) spread over more SMs with one warp per block
    const int nel = p.nx * p.ny, threads = nel <= 32 * 4 * 152 ? 32 : 128, blocks = (nel + threads - 1) / threads;
#define DG_PL(NN)                                                                          \
    (p.swe ? (plane_swe_stage_kernel<NN><<<blocks, threads, 0, s>>>(p), 0)                \
           : (plane_stage_kernel<NN><<<blocks, threads, 0, s>>>(p), 0))
    switch (n) {
    case 1: DG_PL(1); break;
    case 2: DG_PL(2); break;
    case 3: DG_PL(3); break;
    case 4: DG_PL(4); break;
    case 5: DG_PL(5); break;
    default: return 1;
    }
#undef DG_PL
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

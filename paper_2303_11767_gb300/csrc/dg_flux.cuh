// dg_flux.cuh -- pointwise physics shared by the stage kernels: the fluxes
// of the shallow water system on the sphere (paper Eq. sph3) and the Rusanov
// flux (Eq. rusanov), with h stored relative to a reference depth.
#pragma once

#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dgk {

// Programmatic dependent launch: a stage kernel lets the next kernel of the
// stream start its prologue as soon as all of its own CTAs are running, and
// waits for the previous kernel's results before its first dependent read.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on `s` with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T>
__device__ __forceinline__ T rcp(T x);
template <>
__device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }
// FP32: the SFU reciprocal (<= 2 ulp), far inside the FP32 tolerance
template <>
__device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

template <typename T>
__device__ __forceinline__ T wave_sqrt(T x);
template <>
__device__ __forceinline__ double wave_sqrt<double>(double x) { return sqrt(x); }
// FP32: x * rsqrt(x) on the SFU; only feeds the Rusanov dissipation speed
template <>
__device__ __forceinline__ float wave_sqrt<float>(float x) { return x * rsqrtf(x); }

// Finiteness of many values with one test at the end: chk = fma(x, 0, chk)
// for each x stays 0 while every x is finite and becomes NaN (for good) at
// the first Inf or NaN (Inf * 0 = NaN); one FMA per value instead of a
// compare and a predicated OR.  The rounding intrinsics keep the compiler
// from dropping the product.
__device__ __forceinline__ float nf_acc(float x, float chk) { return __fmaf_rn(x, 0.0f, chk); }
__device__ __forceinline__ double nf_acc(double x, double chk) { return __fma_rn(x, 0.0, chk); }

// h <= 0 makes u = hu/h meaningless; a NaN depth is reported as non-finite.
template <typename T>
__device__ __forceinline__ void check_depth(T h, unsigned &st)
{
    if (!(h > T(0))) st |= (h != h) ? DG_STATUS_NONFINITE : DG_STATUS_NONPHYSICAL;
}

// Every multiply-add below is an explicit fma: these functions are inlined at
// several call sites (an edge's flux is evaluated by whichever tile or band
// owns it), and left to the compiler's contraction the same edge could round
// differently at two sites.

// Physical lambda-flux (hu, hu u + P, hu v) of a state q = (h', hu, hv) with
// h = href + h' and the pressure P = g h' (href + h'/2) (the constant part
// g href^2/2 is carried by the rho table), and the wave speed |u| + sqrt(g h).
template <typename T>
__device__ __forceinline__ void lam_flux(const T *q, T href, T g, T *f, T &speed, unsigned &st)
{
    const T h = href + q[0];
    check_depth(h, st);
    const T u = q[1] * rcp(h);
    const T P = (q[0] * g) * fma(T(0.5), q[0], href);
    f[0] = q[1];
    f[1] = fma(q[1], u, P);
    f[2] = q[2] * u;
    speed = fabs(u) + wave_sqrt(g * h);
}

template <typename T>
__device__ __forceinline__ void th_flux(const T *q, T href, T g, T *f, T &speed, unsigned &st)
{
    const T h = href + q[0];
    check_depth(h, st);
    const T v = q[2] * rcp(h);
    const T P = (q[0] * g) * fma(T(0.5), q[0], href);
    f[0] = q[2];
    f[1] = q[1] * v;
    f[2] = fma(q[2], v, P);
    speed = fabs(v) + wave_sqrt(g * h);
}

// Rusanov flux through a lambda-face, left state L (west), right state R
// (east): F* = (F(L) + F(R))/2 - alpha/2 (R - L) with alpha the larger
// one-sided |u| + c; the cos(theta) of U = cos(theta) q cancels against the
// 1/cos(theta) of the eigenvalue of dF/dU.  Scaled by cF = 2/(R dlambda).
template <typename T>
__device__ __forceinline__ void rusanov_lam(const T *L, const T *R, T href, T g, T cF, T *out, unsigned &st,
                                            T aglob = T(0))
{
    T fl[3], fr[3], al, ar;
    lam_flux(L, href, g, fl, al, st);
    lam_flux(R, href, g, fr, ar, st);
    const T ha = T(0.5) * (aglob > T(0) ? aglob : fmax(al, ar));   // global mode: the stage's largest |u| + c
#pragma unroll
    for (int f = 0; f < 3; ++f) out[f] = cF * fma(-ha, R[f] - L[f], T(0.5) * (fl[f] + fr[f]));
}

// Rusanov flux through a theta-face, lower state S, upper state N, times the
// edge cos(theta) ce (flux and jump of U both carry it); scaled by cG.
template <typename T>
__device__ __forceinline__ void rusanov_th(const T *S, const T *Nq, T href, T g, T cGce, T *out, unsigned &st,
                                           T aglob = T(0))
{
    T fs[3], fn[3], as, an;
    th_flux(S, href, g, fs, as, st);
    th_flux(Nq, href, g, fn, an, st);
    const T ha = T(0.5) * (aglob > T(0) ? aglob : fmax(as, an));   // global mode: the stage's largest |v| + c
#pragma unroll
    for (int f = 0; f < 3; ++f) out[f] = cGce * fma(-ha, Nq[f] - S[f], T(0.5) * (fs[f] + fn[f]));
}

}  // namespace dgk

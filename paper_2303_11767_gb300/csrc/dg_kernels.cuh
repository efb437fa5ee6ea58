// dg_kernels.cuh -- device code of libdgswe, included once per precision by
// dg_kernels_f32.cu / dg_kernels_f64.cu with DG_REAL defined to the element
// type.  Each translation unit owns its constant basis tables.
//
// The fused stage kernel evaluates, for every element, the tendency
//   k = M^{-1} h(u)   (paper Eq. ode)
// of the weak form Eq. (dg_parts) for the shallow water system of Eq. (sph3):
//   S1  modal -> Gauss-point values, sum-factorised (a-pass, then b-pass)
//   S2  pointwise fluxes F, G and sources S with cos/sin(theta) row tables
//   S3  volume integral, sum-factorised (beta-pass, then alpha-pass)
//   S4  edge traces of the element; the modes of the tile's halo ring are
//       copied into shared memory (asynchronous copies issued at the start
//       of the tile) and the ring's traces computed from them, so no second
//       pass over memory is made
//   S5  Rusanov flux (Eq. rusanov) at every edge point, zero at pole edges
//   S6  lift of the edge fluxes
//   S7  inverse of the per-row cos(theta)-weighted mass matrix
//   S8  Runge-Kutta combination and store
// and all of it happens in one kernel launch per stage.
//
// Thread mapping: one warp owns G = 32 / N consecutive elements of one
// latitude row; N lanes per element.  Lane k first owns row b = k of the modal
// coefficients, then column alpha = k of the Gauss points (after a transpose
// through shared memory), then row b = k again for the output.  A block of
// DG_WARPS warps covers G x DG_WARPS elements.  Up to p = 3 there is one
// kernel per stage kind (increment or not, final stage or not) and the FP32
// contractions run on paired FP32 instructions.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "dg_internal.h"
#include "dg_flux.cuh"

#ifndef DG_REAL
#error "define DG_REAL before including dg_kernels.cuh"
#endif

__constant__ BasisTab<DG_REAL> c_basis[DG_MAXN];

namespace dgk {

// Smallest slot stride S >= base for which lanes (g, k), g < G, k < N, that
// access word g*S + k of a slotted array hit 32 different banks.
constexpr int bank_free_stride(int base, int N, int G)
{
    for (int S = base; S < base + 64; ++S) {
        bool used[32] = {};
        bool ok = true;
        for (int g = 0; g < G && ok; ++g)
            for (int k = 0; k < N && ok; ++k) {
                const int b = (g * S + k) % 32;
                if (used[b]) ok = false;
                used[b] = true;
            }
        if (ok) return S;
    }
    return base;
}

template <int N, int W>
struct Geo {
    static constexpr int G = 32 / N;            // elements per warp
    static constexpr int NP = N * N;            // modes per field
    static constexpr int EL = 3 * NP;           // values per element
    static constexpr int SA = N + 1;            // padded stride of transposed rows
    static constexpr int T1_OFF = 0;            // [f][alpha][SA]
    static constexpr int EW_OFF = 3 * N * SA;   // [f][2][N]
    static constexpr int X_OFF = 0;             // [f][2][alpha][SA]   (reuses T1/EW)
    static constexpr int WB_MIN = 6 * N * SA;
    // element stride in the warp buffer, padded to spread groups over banks:
    // congruent to N modulo 32, or at degree 4 to -N (the same bank pattern,
    // 10 words shorter, which leaves room for the aligned halo ring)
    static constexpr int WB = N == 5 ? WB_MIN + ((-N - (WB_MIN % 32)) % 32 + 64) % 32
                                     : WB_MIN + ((N - (WB_MIN % 32)) % 32 + 32) % 32;
    static constexpr int TW = G + 2;            // padded tile width (halo columns)
    static constexpr int TH = W + 2;            // padded tile height (halo rows)
    // slot strides padded so that the N lanes of the G elements of a warp
    // touch distinct banks
    static constexpr int TRC = bank_free_stride(12 * N, N, 32 / N);   // traces W,E,S,N x 3 x N
    static constexpr int EFC = bank_free_stride(6 * N, N, 32 / N);    // edge fluxes W,S x 3 x N
    static constexpr int HALO_MAX = 2 * W * N + 2 * G * N;
    static_assert(HALO_MAX <= 32 * W, "halo items exceed the block");
    static_assert(W * N + G * N <= 32 * W, "boundary flux items exceed the block");
};

// Shared-memory map of one tile, in elements of T: the warp buffers, the
// trace slots, then the edge-flux region.  The edge-flux region is dead until
// the Rusanov phase, so the halo ring's modes (stage base, then increment)
// are staged there first; it starts on a 16-byte boundary for the
// asynchronous copies and is as long as the larger of the two uses.
//
// The ring is always copied in 16-byte pieces.  Where an element's modes are
// a multiple of 16 bytes (degrees 1 and 3), the elements are 16-byte aligned
// in global memory and sit back to back in the ring.  Otherwise (degrees 0, 2
// and 4) each ring element gets a slot of RS values starting on a 16-byte
// boundary and lands at offset s = (its global address / sizeof(T)) mod VA in
// it, so that source and destination agree modulo 16 bytes: the copy covers
// the aligned 16-byte blocks that hold the element, a few values of the
// neighbouring elements included (the state arrays start on a 16-byte
// boundary and are padded to a multiple of 16 bytes, so every block read
// lies inside the array).
template <typename T, int N, int W>
struct SmemMap {
    using GE = Geo<N, W>;
    static constexpr int VA = 16 / (int)sizeof(T);
    static constexpr bool PACKED = (GE::EL * (int)sizeof(T)) % 16 == 0;
    // ring slot: room for the element at any offset in its first block, and
    // an odd number of 16-byte blocks, so that the slots the lanes of a warp
    // read in the halo-trace phase start in different banks
    static constexpr int RS0 = (GE::EL + 2 * (VA - 1)) / VA * VA;
    static constexpr int RS = PACKED ? GE::EL : (RS0 / VA) % 2 ? RS0 : RS0 + VA;
    static constexpr int PPS = RS / VA;                // 16-byte pieces per ring slot
    // values of one copy of the halo ring (at most 2 W + 2 G elements)
    static constexpr int HALO_CAP = (2 * W + 2 * GE::G) * RS;
    static constexpr int TRC_OFF = W * GE::G * GE::WB;
    static constexpr int EF_OFF = (TRC_OFF + GE::TW * GE::TH * GE::TRC + VA - 1) / VA * VA;
    static constexpr int EF_LEN = GE::TW * GE::TH * GE::EFC > 2 * HALO_CAP ? GE::TW * GE::TH * GE::EFC : 2 * HALO_CAP;
    static constexpr size_t BYTES = sizeof(T) * (size_t)(EF_OFF + EF_LEN);
    static_assert(RS % VA == 0 && RS >= GE::EL + (PACKED ? 0 : VA - 1), "ring slot too short");
};

// Asynchronous global -> shared copy of 16 bytes (both addresses 16-byte
// aligned); it completes at cp_async_wait_all, and a block barrier then
// publishes it.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const size_t g = __cvta_generic_to_global(src);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The FP32 stage at p <= 3 runs its contractions and its Runge-Kutta update
// on the paired FP32 instructions of sm_100+ (two independent FMAs or adds
// per instruction, each rounded exactly as the scalar one, so the results are
// unchanged); at p = 4 the pairs' extra registers would cost a resident CTA
// per SM and the scalar form is kept.
template <typename T, int N>
__host__ __device__ constexpr bool use_f2()
{
    return std::is_same<T, float>::value && N <= 4;
}
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// number of leading entries of an N-vector handled in pairs
template <typename T, int N>
__host__ __device__ constexpr int pair_len()
{
    return use_f2<T, N>() ? N - (N & 1) : 0;
}

// y[q] = sum_a M[a][q] x[a] for q < N, accumulated in a = 0..N-1 order
template <typename T, int N>
__device__ __forceinline__ void colsum(const T (&M)[DG_MAXN][DG_MAXN], const T *x, T *y)
{
    constexpr int PL = pair_len<T, N>();
    if constexpr (PL > 0) {
#pragma unroll
        for (int q = 0; q < PL; q += 2) {
            float2 s = bc2(0.f);
#pragma unroll
            for (int a = 0; a < N; ++a) s = __ffma2_rn(f2(M[a][q], M[a][q + 1]), bc2(x[a]), s);
            y[q] = s.x;
            y[q + 1] = s.y;
        }
    }
#pragma unroll
    for (int q = PL; q < N; ++q) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) s = fma(M[a][q], x[a], s);
        y[q] = s;
    }
}

template <typename T, int N>
__device__ __forceinline__ void load_row(const T *__restrict__ p, T *o)
{
#pragma unroll
    for (int a = 0; a < N; ++a) o[a] = __ldg(p + a);
}

template <>
__device__ __forceinline__ void load_row<float, 4>(const float *__restrict__ p, float *o)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

template <>
__device__ __forceinline__ void load_row<float, 2>(const float *__restrict__ p, float *o)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = v.x; o[1] = v.y;
}

template <>
__device__ __forceinline__ void load_row<double, 2>(const double *__restrict__ p, double *o)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = v.x; o[1] = v.y;
}

template <>
__device__ __forceinline__ void load_row<double, 4>(const double *__restrict__ p, double *o)
{
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

template <typename T, int N>
__device__ __forceinline__ void store_row(T *p, const T *o)
{
#pragma unroll
    for (int a = 0; a < N; ++a) p[a] = o[a];
}

template <>
__device__ __forceinline__ void store_row<float, 4>(float *p, const float *o)
{
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}

template <>
__device__ __forceinline__ void store_row<float, 2>(float *p, const float *o)
{
    *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
}

template <>
__device__ __forceinline__ void store_row<double, 2>(double *p, const double *o)
{
    *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
}

template <>
__device__ __forceinline__ void store_row<double, 4>(double *p, const double *o)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
}

// Row of the stage state u_stage = base + inc (inc may be null).
template <typename T, int N>
__device__ __forceinline__ void load_stage_row(const T *__restrict__ base, const T *__restrict__ inc, bool has_inc,
                                               size_t off, T *o)
{
    load_row<T, N>(base + off, o);
    if (has_inc) {
        T d[N];
        load_row<T, N>(inc + off, d);
#pragma unroll
        for (int a = 0; a < N; ++a) o[a] += d[a];
    }
}

// One tile of G x W elements (tile column bx, tile row by) of one mesh.  The
// modes of the tile's halo ring reach shared memory through asynchronous
// contiguous copies issued at the start of the tile, so that their latency
// overlaps the tile's own S1 / S4 work.
// INC / FIN fix at compile time whether the stage has an increment (A.inc)
// and whether it is a step's final stage (A.out_base): 1 yes, 0 no, -1 read
// from the arguments.
template <typename T, int N, int W, int INC = -1, int FIN = -1>
__device__ __forceinline__ void stage_tile(const StageArgs<T> &A, int bx, int by, unsigned char *smem_raw)
{
    const T *const incp = INC == 0 ? nullptr : A.inc;
    const bool has_inc = INC == 0 ? false : INC == 1 ? true : (A.inc != nullptr);
    T *const outb = FIN == 0 ? nullptr : A.out_base;
    const bool fin = FIN == 0 ? false : FIN == 1 ? true : (A.out_base != nullptr);
    using GE = Geo<N, W>;
    constexpr int G = GE::G, NP = GE::NP, EL = GE::EL, SA = GE::SA, WB = GE::WB;
    constexpr int TW = GE::TW, TRC = GE::TRC;
    const BasisTab<T> &B = c_basis[N - 1];

    using SM = SmemMap<T, N, W>;
    T *wbuf = reinterpret_cast<T *>(smem_raw);
    T *trc = wbuf + SM::TRC_OFF;             // [slot][W,E,S,N][f][N] traces
    T *ef = wbuf + SM::EF_OFF;               // [slot][W,S][f][N] edge fluxes

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane / N, k = lane - (lane / N) * N;
    const bool lane_ok = g < G;
    const int i0 = bx * G, j0 = by * W;
    const int Gv = min(G, A.nlon - i0);
    const int Wv = min(W, A.nlat - j0);
    const int i = i0 + g, j = j0 + warp;
    const bool valid = lane_ok && g < Gv && warp < Wv;
    const size_t e = valid ? (size_t)j * A.nlon + i : 0;
    const int own = (warp + 1) * TW + (lane_ok ? g + 1 : 1);   // own slot of the padded tile
    const T href = A.href, gg = A.g;
    unsigned st = 0;

    T *wb = wbuf + (warp * G + (lane_ok ? g : 0)) * WB;

    const RowTab<T> *RT = A.rows + (valid ? j : 0);
    const T ga_l = A.galpha ? A.galpha[0] : T(0), ga_t = A.galpha ? A.galpha[1] : T(0);

    // ---- S0: own modal row b = k of the stage state
    T uh[3][N];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        if (valid) load_stage_row<T, N>(A.base, incp, has_inc, e * EL + f * NP + k * N, uh[f]);
        else {
#pragma unroll
            for (int a = 0; a < N; ++a) uh[f][a] = T(0);
        }
    }

    // ---- S0 halo: the modes of the ring of neighbour elements facing the tile
    //      (W / E columns, S / N rows; periodic in lambda, none across a pole),
    //      copied asynchronously by all threads, the base to ef[0, HALO_CAP)
    //      and the increment to ef[HALO_CAP, 2 HALO_CAP)
    const bool hasS = j0 > 0 || A.halo_s, hasN = j0 + Wv < A.nlat || A.halo_n;
    const int nSe = hasS ? Gv : 0, nNe = hasN ? Gv : 0;
    const int nH = 2 * Wv + nSe + nNe;
    const int iW = i0 > 0 ? i0 - 1 : A.nlon - 1, iE = i0 + Gv < A.nlon ? i0 + Gv : 0;   // i0 + Gv <= nlon
    // value offset of ring element h: W column, E column, S row, N row (hj =
    // -1 is a neighbour band's row held just before row 0)
    auto ring_off = [&](int h) -> long long {
        int hj, hi;
        if (h < 2 * Wv) {
            const bool east = h >= Wv;
            hj = j0 + (east ? h - Wv : h);
            hi = east ? iE : iW;
        } else {
            const int r = h - 2 * Wv;
            const bool north = r >= nSe;
            hj = north ? j0 + Wv : j0 - 1;
            hi = i0 + (north ? r - nSe : r);
        }
        return ((long long)hj * A.nlon + hi) * EL;
    };
    // position of a value within its 16-byte block
    auto lead = [](const T *p) -> int {
        return (int)((reinterpret_cast<uintptr_t>(p) / sizeof(T)) & (SM::VA - 1));
    };
    if constexpr (SM::PACKED) {
        // the W / E columns found in the loop (one or two pieces per thread:
        // measured faster than finding them once at degree 3)
        constexpr int CPE = EL / SM::VA;
        for (int v = tid; v < nH * CPE; v += 32 * W) {
            const int h = v / CPE, c = (v - h * CPE) * SM::VA;
            int hj, hi;
            if (h < 2 * Wv) {
                const bool east = h >= Wv;
                hj = j0 + (east ? h - Wv : h);
                hi = east ? (i0 + Gv) % A.nlon : (i0 - 1 + A.nlon) % A.nlon;
            } else {
                const int r = h - 2 * Wv;
                const bool north = r >= nSe;
                hj = north ? j0 + Wv : j0 - 1;
                hi = i0 + (north ? r - nSe : r);
            }
            const long long o = ((long long)hj * A.nlon + hi) * EL + c;
            cp_async16(ef + h * EL + c, A.base + o);
            if (has_inc) cp_async16(ef + SM::HALO_CAP + h * EL + c, incp + o);
        }
    } else {
        // piece c of ring slot h: the c-th 16-byte block from the one that
        // holds the element's first value, while it still holds some of them
        for (int v = tid; v < nH * SM::PPS; v += 32 * W) {
            const int h = v / SM::PPS, c = v - h * SM::PPS;
            const long long o = ring_off(h);
            const T *sb = A.base + o;
            const int lb = lead(sb);
            if (c * SM::VA < lb + EL) cp_async16(ef + h * SM::RS + c * SM::VA, sb - lb + c * SM::VA);
            if (has_inc) {
                const T *si = incp + o;
                const int li = lead(si);
                if (c * SM::VA < li + EL)
                    cp_async16(ef + SM::HALO_CAP + h * SM::RS + c * SM::VA, si - li + c * SM::VA);
            }
        }
    }
    // where ring element h's modes start in shared memory (base, increment)
    auto ring_at = [&](int h, const T *&rb, const T *&ri) {
        if constexpr (SM::PACKED) {
            rb = ef + h * EL;
            ri = rb + SM::HALO_CAP;
        } else {
            const long long o = ring_off(h);
            rb = ef + h * SM::RS + lead(A.base + o);
            ri = ef + SM::HALO_CAP + h * SM::RS + (has_inc ? lead(incp + o) : 0);
        }
    };

    // rows the epilogue will read: start moving them towards L1 now
    if (valid) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const size_t off = e * EL + f * NP + k * N;
            if (fin) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.base + off));
            if (A.lo) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.lo + off));
            if (A.acc_in) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.acc_in + off));
        }
    }

    // ---- S1 a-pass (row b = k): t1[alpha] = sum_a L_a(xi_alpha) u[b][a], and
    //      the lambda-edge partial sums sum_a L_a(+-1) u[b][a]
    if (lane_ok) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T t1[N];
            colsum<T, N>(B.LV, uh[f], t1);
#pragma unroll
            for (int q = 0; q < N; ++q) wb[GE::T1_OFF + (f * N + q) * SA + k] = t1[q];
            T se = T(0), sw = T(0);
#pragma unroll
            for (int a = 0; a < N; ++a) {
                se = fma(B.SE[a], uh[f][a], se);
                sw = fma(B.SW[a], uh[f][a], sw);
            }
            wb[GE::EW_OFF + (f * 2 + 0) * N + k] = se;
            wb[GE::EW_OFF + (f * 2 + 1) * N + k] = sw;
        }
    }
    __syncwarp();

    // ---- S1 b-pass (column alpha = k) and S4 own traces
    T qn[3][N];      // Gauss-point values at (alpha = k, beta)
    T tr[4][3];      // traces at own point k: W, E (at eta_k), S, N (at xi_k)
    {
        T LVk[N];
#pragma unroll
        for (int b = 0; b < N; ++b) LVk[b] = B.LV[b][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T c[N], ee[N], ew[N];
#pragma unroll
            for (int b = 0; b < N; ++b) {
                c[b] = wb[GE::T1_OFF + (f * N + k) * SA + b];
                ee[b] = wb[GE::EW_OFF + (f * 2 + 0) * N + b];
                ew[b] = wb[GE::EW_OFF + (f * 2 + 1) * N + b];
            }
            colsum<T, N>(B.LV, c, qn[f]);
            T ts = T(0), tn = T(0), tw = T(0), te = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) {
                ts = fma(B.SW[b], c[b], ts);
                tn = fma(B.SE[b], c[b], tn);
                tw = fma(LVk[b], ew[b], tw);
                te = fma(LVk[b], ee[b], te);
            }
            tr[0][f] = tw; tr[1][f] = te; tr[2][f] = ts; tr[3][f] = tn;
        }
    }
    if (valid) {
        T *slot = trc + own * TRC;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int f = 0; f < 3; ++f) slot[(s * 3 + f) * N + k] = tr[s][f];
    }

    // ---- S4 halo: traces of the ring of neighbour elements facing the tile
    cp_async_wait_all();   // the ring's modes are in shared memory
    __syncthreads();
    if constexpr (N >= 5) {
        // degree 4: one item per (ring element, field), its N traces on the
        // side that faces the tile, each mode row read once (a third of the
        // instructions of one item per trace point; measured +9 % at 1440x720
        // and 360x180, while up to degree 3 the shorter per-point items keep
        // more threads busy on the one-wave 180x90 mesh).  The sums run in
        // the order the owning tile uses for the element's own traces (lambda
        // edge: sum_b L_b(eta_k) (sum_a L_a(+-1) u[b][a]); theta edge:
        // sum_b L_b(+-1) (sum_a L_a(xi_k) u[b][a])), so both tiles of a tile
        // boundary evaluate that edge's flux from the same bits and the
        // single-valued flux keeps mass to roundoff.
        // whole warps take halo items (no divergence inside a warp)
        for (int it = tid; it < 3 * nH; it += 32 * W) {
            const int r = it / 3, f = it - 3 * r;
            int side, sl, hh;
            if (r < 2 * Wv) {                   // west / east halo columns
                const bool east = r >= Wv;
                const int w = east ? r - Wv : r;
                side = east ? 0 : 1;            // east halo needs its W trace
                sl = (w + 1) * TW + (east ? Gv + 1 : 0);
                hh = east ? Wv + w : w;
            } else {                            // south / north halo rows
                const int r0 = r - 2 * Wv;
                const bool north = r0 >= nSe;
                const int c = north ? r0 - nSe : r0;
                side = north ? 2 : 3;           // north halo needs its S trace
                sl = (north ? Wv + 1 : 0) * TW + c + 1;
                hh = 2 * Wv + (north ? nSe + c : c);
            }
            const T *hb, *hbi;
            ring_at(hh, hb, hbi);
            hb += f * NP;
            hbi += f * NP;
            T acc[N];
#pragma unroll
            for (int kk = 0; kk < N; ++kk) acc[kk] = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) {
                T row[N];                       // row b of the halo element's stage state
#pragma unroll
                for (int a = 0; a < N; ++a) row[a] = hb[b * N + a];
                if (has_inc) {
#pragma unroll
                    for (int a = 0; a < N; ++a) row[a] += hbi[b * N + a];
                }
                if (side <= 1) {
                    T sb = T(0);
#pragma unroll
                    for (int a = 0; a < N; ++a) sb = fma(side == 1 ? B.SE[a] : B.SW[a], row[a], sb);
#pragma unroll
                    for (int kk = 0; kk < N; ++kk) acc[kk] = fma(B.LV[b][kk], sb, acc[kk]);
                } else {
                    const T cb = side == 3 ? B.SE[b] : B.SW[b];
#pragma unroll
                    for (int kk = 0; kk < N; ++kk) {
                        T s = T(0);
#pragma unroll
                        for (int a = 0; a < N; ++a) s = fma(B.LV[a][kk], row[a], s);
                        acc[kk] = fma(cb, s, acc[kk]);
                    }
                }
            }
            T *slot = trc + sl * TRC + (side * 3 + f) * N;
#pragma unroll
            for (int kk = 0; kk < N; ++kk) slot[kk] = acc[kk];
        }
    } else {
        // up to degree 3: one item per trace point (ring element, side, k),
        // the same sums in the same order
        const int nWE = Wv * N;
        const int nS = hasS ? Gv * N : 0, nN = hasN ? Gv * N : 0;
        const int it = tid;   // whole warps take halo items (no divergence inside a warp)
        if (it < 2 * nWE + nS + nN) {
            int side, kk, sl, hh;
            if (it < 2 * nWE) {                 // west / east halo columns
                const bool east = it >= nWE;
                const int r = east ? it - nWE : it;
                const int w = r / N;
                kk = r - w * N;
                side = east ? 0 : 1;            // east halo needs its W trace
                sl = (w + 1) * TW + (east ? Gv + 1 : 0);
                hh = east ? Wv + w : w;
            } else {                            // south / north halo rows
                const int r0 = it - 2 * nWE;
                const bool north = r0 >= nS;
                const int r = north ? r0 - nS : r0;
                const int c = r / N;
                kk = r - c * N;
                side = north ? 2 : 3;           // north halo needs its S trace
                sl = (north ? Wv + 1 : 0) * TW + c + 1;
                hh = 2 * Wv + (north ? nSe + c : c);
            }
            const T *rb, *ri;
            ring_at(hh, rb, ri);
            // row b of field f of the halo element's stage state
            auto halo_row = [&](int f, int b, T *row) {
                const T *hb = rb + f * NP + b * N, *hbi = ri + f * NP + b * N;
#pragma unroll
                for (int a = 0; a < N; ++a) row[a] = hb[a];
                if (has_inc) {
#pragma unroll
                    for (int a = 0; a < N; ++a) row[a] += hbi[a];
                }
            };
            T *slot = trc + sl * TRC;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                T acc = T(0);
                if (side <= 1) {                // lambda edge: sum_b L_b(eta_kk) sum_a L_a(+-1) u[b][a]
#pragma unroll
                    for (int b = 0; b < N; ++b) {
                        T row[N];
                        halo_row(f, b, row);
                        T s = T(0);
#pragma unroll
                        for (int a = 0; a < N; ++a) s = fma(side == 1 ? B.SE[a] : B.SW[a], row[a], s);
                        acc = fma(B.LV[b][kk], s, acc);
                    }
                } else {                        // theta edge: sum_b L_b(+-1) sum_a L_a(xi_kk) u[b][a]
#pragma unroll
                    for (int b = 0; b < N; ++b) {
                        T row[N];
                        halo_row(f, b, row);
                        T s = T(0);
#pragma unroll
                        for (int a = 0; a < N; ++a) s = fma(B.LV[a][kk], row[a], s);
                        acc = fma(side == 3 ? B.SE[b] : B.SW[b], s, acc);
                    }
                }
                slot[(side * 3 + f) * N + kk] = acc;
            }
        }
    }
    __syncthreads();

    // ---- S5 Rusanov fluxes, each edge once: every element evaluates its W
    //      edge (at eta_k) and S edge (at xi_k); the tile's east column and top
    //      row borrow the W / S edges of the east and north halo slots
    {
        T nb[3], fx[3];
        if (valid) {
            const T *tW = trc + (own - 1) * TRC;
#pragma unroll
            for (int f = 0; f < 3; ++f) nb[f] = tW[(1 * 3 + f) * N + k];       // W neighbour's E trace
            rusanov_lam(nb, tr[0], href, gg, A.cF, fx, st, ga_l);
#pragma unroll
            for (int f = 0; f < 3; ++f) ef[(own * 2 + 0) * 3 * N + f * N + k] = fx[f];
            if (j > 0 || A.halo_s) {
                const T *tS = trc + (own - TW) * TRC;
#pragma unroll
                for (int f = 0; f < 3; ++f) nb[f] = tS[(3 * 3 + f) * N + k];   // S neighbour's N trace
                rusanov_th(nb, tr[2], href, gg, A.cG * __ldg(&RT->ce_s), fx, st, ga_t);
            } else {
#pragma unroll
                for (int f = 0; f < 3; ++f) fx[f] = T(0);                       // pole edge: zero flux
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) ef[(own * 2 + 1) * 3 * N + f * N + k] = fx[f];
        }
        const int nE = Wv * N, nN = hasN ? Gv * N : 0;
        const int it = 32 * W - 1 - tid;   // the last warps, which have no halo items
        if (it < nE + nN) {
            T L[3], R[3];
            if (it < nE) {                      // E edge of the last valid column
                const int w = it / N, kk = it - (it / N) * N;
                const int sl = (w + 1) * TW + Gv, sr = sl + 1;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    L[f] = trc[sl * TRC + (1 * 3 + f) * N + kk];
                    R[f] = trc[sr * TRC + (0 * 3 + f) * N + kk];
                }
                rusanov_lam(L, R, href, gg, A.cF, fx, st, ga_l);
#pragma unroll
                for (int f = 0; f < 3; ++f) ef[(sr * 2 + 0) * 3 * N + f * N + kk] = fx[f];
            } else {                            // N edge of the top valid row
                const int r = it - nE, c = r / N, kk = r - (r / N) * N;
                const int sl = Wv * TW + c + 1, su = sl + TW;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    L[f] = trc[sl * TRC + (3 * 3 + f) * N + kk];
                    R[f] = trc[su * TRC + (2 * 3 + f) * N + kk];
                }
                rusanov_th(L, R, href, gg, A.cG * __ldg(&A.rows[j0 + Wv - 1].ce_n), fx, st, ga_t);
#pragma unroll
                for (int f = 0; f < 3; ++f) ef[(su * 2 + 1) * 3 * N + f * N + kk] = fx[f];
            }
        }
    }
    __syncthreads();

    // ---- S2 pointwise fluxes at (alpha = k, beta), S3 beta-pass with the
    //      inverse mass matrix folded in (per-row QT = (Ci W L)^T, PT = (Ci W L')^T)
    //      and the N/S lift through Ci L(+-1)
    {
        T GsS[3], GsN[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            GsS[f] = ef[(own * 2 + 1) * 3 * N + f * N + k];
            GsN[f] = (valid && (j < A.nlat - 1 || A.halo_n)) ? ef[((own + TW) * 2 + 1) * 3 * N + f * N + k] : T(0);
        }
        T X1[3][N], X2[3][N];
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                X2[f][b] = __ldg(&RT->CSW[b]) * GsS[f] - __ldg(&RT->CSE[b]) * GsN[f];
                X1[f][b] = T(0);
            }
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const T hp = qn[0][q], hu = qn[1][q], hv = qn[2][q];
            const T h = href + hp;
            check_depth(h, st);
            const T rh = rcp(h);
            const T u = hu * rh, v = hv * rh;
            const T P = hp * gg * (href + T(0.5) * hp);
            const T c = __ldg(&RT->cosn[q]), s = __ldg(&RT->sinn[q]);
            const T F0 = A.cF * hu, F1 = A.cF * fma(hu, u, P), F2 = A.cF * (hu * v);
            const T cGc = A.cG * c;
            const T G0 = cGc * hv, G1 = cGc * (hv * u), G2 = cGc * fma(hv, v, P);
            const T K = s * fma(A.twoOmega, c, u * A.invR);
            const T S1 = K * hv, S2 = -(P * s * A.invR) - K * hu;
            constexpr int PL = pair_len<T, N>();
            if constexpr (PL > 0) {
#pragma unroll
                for (int b = 0; b < PL; b += 2) {
                    const float2 wl = f2(__ldg(&RT->QT[q][b]), __ldg(&RT->QT[q][b + 1]));
                    const float2 wd = f2(__ldg(&RT->PT[q][b]), __ldg(&RT->PT[q][b + 1]));
                    float2 x;
                    x = __ffma2_rn(wl, bc2(F0), f2(X1[0][b], X1[0][b + 1]));
                    X1[0][b] = x.x, X1[0][b + 1] = x.y;
                    x = __ffma2_rn(wl, bc2(F1), f2(X1[1][b], X1[1][b + 1]));
                    X1[1][b] = x.x, X1[1][b + 1] = x.y;
                    x = __ffma2_rn(wl, bc2(F2), f2(X1[2][b], X1[2][b + 1]));
                    X1[2][b] = x.x, X1[2][b + 1] = x.y;
                    x = __ffma2_rn(wd, bc2(G0), f2(X2[0][b], X2[0][b + 1]));
                    X2[0][b] = x.x, X2[0][b + 1] = x.y;
                    x = __ffma2_rn(wd, bc2(G1), __ffma2_rn(wl, bc2(S1), f2(X2[1][b], X2[1][b + 1])));
                    X2[1][b] = x.x, X2[1][b + 1] = x.y;
                    x = __ffma2_rn(wd, bc2(G2), __ffma2_rn(wl, bc2(S2), f2(X2[2][b], X2[2][b + 1])));
                    X2[2][b] = x.x, X2[2][b + 1] = x.y;
                }
            }
#pragma unroll
            for (int b = PL; b < N; ++b) {
                const T wl = __ldg(&RT->QT[q][b]), wd = __ldg(&RT->PT[q][b]);
                X1[0][b] = fma(wl, F0, X1[0][b]);
                X1[1][b] = fma(wl, F1, X1[1][b]);
                X1[2][b] = fma(wl, F2, X1[2][b]);
                X2[0][b] = fma(wd, G0, X2[0][b]);
                X2[1][b] = fma(wd, G1, fma(wl, S1, X2[1][b]));
                X2[2][b] = fma(wd, G2, fma(wl, S2, X2[2][b]));
            }
        }
        if (lane_ok) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    wb[GE::X_OFF + ((f * 2 + 0) * N + k) * SA + b] = X1[f][b];
                    wb[GE::X_OFF + ((f * 2 + 1) * N + k) * SA + b] = X2[f][b];
                }
        }
    }
    __syncwarp();

    // ---- S3 alpha-pass and S6 E/W lift (row b = k), S8 combine and store
    {
        T Qk[N];
#pragma unroll
        for (int q = 0; q < N; ++q) Qk[q] = __ldg(&RT->Q[k][q]);
        const T rhok = __ldg(&RT->rho[k]);
        const T *efW = ef + (own * 2 + 0) * 3 * N;          // W edge fluxes of this element
        const T *efE = ef + ((own + 1) * 2 + 0) * 3 * N;    // = W edge fluxes of the E neighbour
        T kk[3][N];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T y1[N], y2[N];
            T ye = T(0), yw = T(0);
#pragma unroll
            for (int q = 0; q < N; ++q) {
                y1[q] = wb[GE::X_OFF + ((f * 2 + 0) * N + q) * SA + k];
                y2[q] = wb[GE::X_OFF + ((f * 2 + 1) * N + q) * SA + k];
                ye = fma(Qk[q], efE[f * N + q], ye);
                yw = fma(Qk[q], efW[f * N + q], yw);
            }
            constexpr int PL = pair_len<T, N>();
            if constexpr (PL > 0) {
#pragma unroll
                for (int a = 0; a < PL; a += 2) {
                    float2 s = bc2(0.f);
#pragma unroll
                    for (int q = 0; q < N; ++q)
                        s = __ffma2_rn(f2(B.WLD[a][q], B.WLD[a + 1][q]), bc2(y1[q]),
                                       __ffma2_rn(f2(B.WLV[a][q], B.WLV[a + 1][q]), bc2(y2[q]), s));
                    kk[f][a] = s.x - (B.SE[a] * ye - B.SW[a] * yw);
                    kk[f][a + 1] = s.y - (B.SE[a + 1] * ye - B.SW[a + 1] * yw);
                }
            }
#pragma unroll
            for (int a = PL; a < N; ++a) {
                T s = T(0);
#pragma unroll
                for (int q = 0; q < N; ++q) s = fma(B.WLD[a][q], y1[q], fma(B.WLV[a][q], y2[q], s));
                kk[f][a] = s - (B.SE[a] * ye - B.SW[a] * yw);
            }
        }
        kk[2][0] = fma(A.P0, rhok, kk[2][0]);
        if (A.src && valid) {   // learned modal source, same layout as the state
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                T sv[N];
                load_row<T, N>(A.src + e * EL + f * NP + k * N, sv);
#pragma unroll
                for (int a = 0; a < N; ++a) kk[f][a] += sv[a];
            }
        }

        if (valid) {
            const T cdt = A.cc * A.dt, adt = A.ca * A.dt;
            T chk = T(0);   // non-finite tendency or state: NaN (nf_acc)
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const size_t off = e * EL + f * NP + k * N;
#pragma unroll
                for (int a = 0; a < N; ++a) chk = nf_acc(kk[f][a], chk);
                if (A.out_rhs) store_row<T, N>(A.out_rhs + off, kk[f]);
                T inc[N];
                if (has_inc) load_row<T, N>(incp + off, inc);
                else {
#pragma unroll
                    for (int a = 0; a < N; ++a) inc[a] = T(0);
                }
                if (A.inc_out) {
                    T o[N];
#pragma unroll
                    for (int a = 0; a < N; ++a) o[a] = fma(cdt, kk[f][a], A.ci * inc[a]);
                    store_row<T, N>(A.inc_out + off, o);
                }
                T acc[N];
                if (A.acc_in) load_row<T, N>(A.acc_in + off, acc);
                else {
#pragma unroll
                    for (int a = 0; a < N; ++a) acc[a] = T(0);
                }
                if (A.acc_out) {
                    T o[N];
#pragma unroll
                    for (int a = 0; a < N; ++a) o[a] = fma(adt, kk[f][a], acc[a]);
                    store_row<T, N>(A.acc_out + off, o);
                }
                if (fin) {
                    // u^{n+1} = (base + lo) + delta with an error-free two-sum,
                    // so increments far below one ulp of the state survive
                    T bs[N], lo[N], ob[N], ol[N];
                    load_row<T, N>(A.base + off, bs);
                    if (A.lo) load_row<T, N>(A.lo + off, lo);
                    else {
#pragma unroll
                        for (int a = 0; a < N; ++a) lo[a] = T(0);
                    }
                    constexpr int PL = pair_len<T, N>();
                    if constexpr (PL > 0) {
#pragma unroll
                        for (int a = 0; a < PL; a += 2) {
                            const float2 bs2 = f2(bs[a], bs[a + 1]);
                            const float2 delta = __ffma2_rn(bc2(cdt), f2(kk[f][a], kk[f][a + 1]),
                                                            __ffma2_rn(bc2(A.cd), f2(acc[a], acc[a + 1]),
                                                                       __fmul2_rn(bc2(A.ci), f2(inc[a], inc[a + 1]))));
                            const float2 s1 = __fadd2_rn(bs2, delta);
                            const float2 bp = __fadd2_rn(s1, neg2(bs2));
                            const float2 err = __fadd2_rn(__fadd2_rn(bs2, neg2(__fadd2_rn(s1, neg2(bp)))),
                                                          __fadd2_rn(delta, neg2(bp)));
                            const float2 l1 = __fadd2_rn(f2(lo[a], lo[a + 1]), err);
                            const float2 hi = __fadd2_rn(s1, l1);
                            const float2 ol2 = __fadd2_rn(l1, neg2(__fadd2_rn(hi, neg2(s1))));
                            ob[a] = hi.x, ob[a + 1] = hi.y;
                            ol[a] = ol2.x, ol[a + 1] = ol2.y;
                            chk = nf_acc(hi.y, nf_acc(hi.x, chk));
                        }
                    }
#pragma unroll
                    for (int a = PL; a < N; ++a) {
                        const T delta = fma(cdt, kk[f][a], fma(A.cd, acc[a], A.ci * inc[a]));
                        const T s1 = bs[a] + delta;
                        const T bp = s1 - bs[a];
                        const T err = (bs[a] - (s1 - bp)) + (delta - bp);
                        const T l1 = lo[a] + err;
                        const T hi = s1 + l1;
                        ob[a] = hi;
                        ol[a] = l1 - (hi - s1);
                        chk = nf_acc(hi, chk);
                    }
                    store_row<T, N>(outb + off, ob);
                    if (A.out_lo) store_row<T, N>(A.out_lo + off, ol);
                }
            }
            if (!isfinite(chk)) st |= DG_STATUS_NONFINITE;
        }
    }
    if (st && valid) atomicOr(A.status, st);
}

template <typename T, int N, int W, int INC, int FIN>
__global__ void __launch_bounds__(32 * W) stage_kernel(const StageArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    stage_tile<T, N, W, INC, FIN>(A, blockIdx.x, blockIdx.y, smem_raw);
    pdl_launch_dependents();
}

template <typename T, int N, int W>
constexpr size_t stage_smem_bytes()
{
    return SmemMap<T, N, W>::BYTES;
}

template <typename T, int N>
int launch_stage_n(const StageArgs<T> &a, cudaStream_t s)
{
    constexpr int W = DG_WARPS;
    using GE = Geo<N, W>;
    const size_t smem = stage_smem_bytes<T, N, W>();
    // One kernel per stage kind (increment present or not, final stage or
    // not) up to p = 3, where the specialised kernels measured faster
    // (180x90: 6.28 -> 5.98 us per stage); one kernel reading the kind from
    // its arguments at p = 4, where they did not (360x180: 43.2 -> 44.2 us).
    using K = void (*)(const StageArgs<T>);
    K k00, k01, k10, k11;
    if constexpr (N <= 4) {
        k00 = stage_kernel<T, N, W, 0, 0>;
        k01 = stage_kernel<T, N, W, 0, 1>;
        k10 = stage_kernel<T, N, W, 1, 0>;
        k11 = stage_kernel<T, N, W, 1, 1>;
    } else {
        k00 = k01 = k10 = k11 = stage_kernel<T, N, W, -1, -1>;
    }
    // the shared-memory opt-in is a per-device function attribute
    static std::atomic<unsigned long long> attr_set{0};   // handles on other host threads may launch too
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!(attr_set.load(std::memory_order_acquire) >> dev & 1ull)) {
        for (K k : {k00, k01, k10, k11})
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return 1;
        attr_set.fetch_or(1ull << dev, std::memory_order_release);   // setting it twice is harmless
    }
    dim3 grid((a.nlon + GE::G - 1) / GE::G, (a.nlat + W - 1) / W);
    const K k = a.inc ? (a.out_base ? k11 : k10) : (a.out_base ? k01 : k00);
    if (launch_pdl(k, grid, dim3(32 * W), smem, s, a) != cudaSuccess) return 1;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

// ---------------------------------------------------------------- ensemble --

// One persistent launch per RK stage for a batch of meshes of different sizes
// and degrees: every CTA walks the work list (member, tile column, tile row)
// and runs the tile with the member's degree.  Items are ordered by cost,
// largest first, so the round-robin walk balances the CTAs.
template <typename T, int W>
__global__ void __launch_bounds__(32 * W, 24 / W) ensemble_kernel(const EnsArgs<T> E)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < E.nitems; it += gridDim.x) {
        const EnsItem item = E.items[it];
        const EnsMember<T> m = E.members[item.member];
        StageArgs<T> A;
        A.base = E.base + m.off;
        A.inc = E.inc ? E.inc + m.off : nullptr;
        A.lo = E.lo ? E.lo + m.off : nullptr;
        A.acc_in = E.acc_in ? E.acc_in + m.off : nullptr;
        A.out_rhs = E.out_rhs ? E.out_rhs + m.off : nullptr;
        A.inc_out = E.inc_out ? E.inc_out + m.off : nullptr;
        A.acc_out = E.acc_out ? E.acc_out + m.off : nullptr;
        A.out_base = E.out_base ? E.out_base + m.off : nullptr;
        A.out_lo = E.out_lo ? E.out_lo + m.off : nullptr;
        A.rows = E.rows + m.rows;
        A.src = nullptr;
        A.galpha = nullptr;
        A.status = E.status;
        A.nlon = m.nlon;
        A.nlat = m.nlat;
        A.halo_s = A.halo_n = 0;
        A.href = m.href;
        A.P0 = m.P0;
        A.g = E.g;
        A.cF = m.cF;
        A.cG = m.cG;
        A.invR = E.invR;
        A.twoOmega = E.twoOmega;
        A.ci = E.ci;
        A.ca = E.ca;
        A.cc = E.cc;
        A.cd = E.cd;
        A.dt = m.dt;
        switch (m.n) {
        case 1: stage_tile<T, 1, W>(A, item.tx, item.ty, smem_raw); break;
        case 2: stage_tile<T, 2, W>(A, item.tx, item.ty, smem_raw); break;
        case 3: stage_tile<T, 3, W>(A, item.tx, item.ty, smem_raw); break;
        case 4: stage_tile<T, 4, W>(A, item.tx, item.ty, smem_raw); break;
        default: stage_tile<T, 5, W>(A, item.tx, item.ty, smem_raw); break;
        }
        __syncthreads();   // the next item reuses the shared memory
    }
}

template <typename T, int W>
constexpr size_t ensemble_smem_bytes()
{
    size_t m = stage_smem_bytes<T, 1, W>();
    m = m > stage_smem_bytes<T, 2, W>() ? m : stage_smem_bytes<T, 2, W>();
    m = m > stage_smem_bytes<T, 3, W>() ? m : stage_smem_bytes<T, 3, W>();
    m = m > stage_smem_bytes<T, 4, W>() ? m : stage_smem_bytes<T, 4, W>();
    m = m > stage_smem_bytes<T, 5, W>() ? m : stage_smem_bytes<T, 5, W>();
    return m;
}

template <typename T, int W>
int launch_ensemble_w(int grid, const EnsArgs<T> &a, cudaStream_t s)
{
    const size_t smem = ensemble_smem_bytes<T, W>();
    static std::atomic<unsigned long long> attr_set{0};   // handles on other host threads may launch too
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!(attr_set.load(std::memory_order_acquire) >> dev & 1ull)) {
        if (cudaFuncSetAttribute(ensemble_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 1;
        attr_set.fetch_or(1ull << dev, std::memory_order_release);   // setting it twice is harmless
    }
    ensemble_kernel<T, W><<<grid, 32 * W, smem, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------- auxiliary --

// API layout (FP64, full h) <-> internal (base, lo) layout with h stored
// relative to href.  lo receives what base (T) cannot hold; may be null.
template <typename T>
__global__ void to_internal_kernel(const double *__restrict__ src, T *__restrict__ dst, T *__restrict__ lo,
                                   size_t nval, int per_el, double href)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nval; t += (size_t)gridDim.x * blockDim.x) {
        double v = src[t];
        if (t % per_el == 0) v -= 2.0 * href;   // mode 0 of h: phi_0 = 1/2
        const T hi = (T)v;
        dst[t] = hi;
        if (lo) lo[t] = (T)(v - (double)hi);
    }
}

template <typename T>
__global__ void to_api_kernel(const T *__restrict__ src, const T *__restrict__ lo, double *__restrict__ dst,
                              size_t nval, int per_el, double href)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nval; t += (size_t)gridDim.x * blockDim.x) {
        double v = (double)src[t];
        if (lo) v += (double)lo[t];
        if (t % per_el == 0) v += 2.0 * href;
        dst[t] = v;
    }
}

// Neumaier-compensated pair (sum, correction); combining two pairs uses the
// error-free TwoSum of the sums, so the fixed reduction tree below gives the
// same bits on every run.
struct CSum {
    double s, c;
};

__device__ __forceinline__ CSum csum_add(CSum a, double x)
{
    const double t = a.s + x;
    const double bp = t - a.s;
    const double err = (a.s - (t - bp)) + (x - bp);
    return CSum{t, a.c + err};
}

__device__ __forceinline__ CSum csum_merge(CSum a, CSum b)
{
    CSum r = csum_add(a, b.s);
    r.c += b.c;
    return r;
}

constexpr int MASS_THREADS = 256;

// Per element: int h cos(theta) dlambda dtheta
//   = (dlam dth / 2) sum_b C_j[0][b] h'_{a=0,b} + href dlam (sin t - sin b).
// c0: nlat * n values C_j[0][b]; area row j in c0[nlat*n + j].
template <typename T>
__global__ void __launch_bounds__(MASS_THREADS) mass_partial_kernel(const T *__restrict__ u,
                                                                    const T *__restrict__ ulo,
                                                                    const double *__restrict__ c0, int nlon,
                                                                    int nlat, int n, double href, double half_dd,
                                                                    double dlam, size_t chunk,
                                                                    double *__restrict__ partials)
{
    __shared__ CSum red[MASS_THREADS];
    const size_t nel = (size_t)nlon * nlat;
    const size_t b0 = blockIdx.x * chunk, b1 = min(nel, b0 + chunk);
    const int per = 3 * n * n;
    CSum acc{0.0, 0.0};
    for (size_t e = b0 + threadIdx.x; e < b1; e += MASS_THREADS) {
        const int j = (int)(e / nlon);
        const T *ue = u + e * per;
        double m = 0.0;
        for (int b = 0; b < n; ++b) {
            double hb = (double)ue[b * n];
            if (ulo) hb += (double)ulo[e * per + b * n];
            m += c0[j * n + b] * hb;
        }
        acc = csum_add(acc, half_dd * m + href * dlam * c0[nlat * n + j]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = MASS_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = csum_merge(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = red[0].s;
        partials[2 * blockIdx.x + 1] = red[0].c;
    }
}

static __global__ void __launch_bounds__(MASS_THREADS) mass_final_kernel(const double *__restrict__ partials, int nblocks,
                                                                  double scale, double *__restrict__ result,
                                                                  double *__restrict__ pair)
{
    __shared__ CSum red[MASS_THREADS];
    CSum acc{0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += MASS_THREADS)
        acc = csum_merge(acc, CSum{partials[2 * b], partials[2 * b + 1]});
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = MASS_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = csum_merge(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (result) *result = scale * (red[0].s + red[0].c);
        if (pair) {
            pair[0] = red[0].s;
            pair[1] = red[0].c;
        }
    }
}

// Largest sqrt(u^2 + v^2) + sqrt(g h) over the n x n Gauss points; one thread
// per element.  Positive doubles order like their bit patterns, so an atomic
// max on the bits is exact and order independent.
template <typename T, int N>
__global__ void max_speed_kernel(const T *__restrict__ u, int nel, double href, double g,
                                 unsigned long long *maxbits, unsigned *status)
{
    const BasisTab<T> &B = c_basis[N - 1];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double best = 0.0;
    unsigned st = 0;
    if (e < nel) {
        const T *ue = u + (size_t)e * 3 * N * N;
        for (int q = 0; q < N; ++q)
            for (int r = 0; r < N; ++r) {
                double qv[3];
                for (int f = 0; f < 3; ++f) {
                    double s = 0.0;
                    for (int b = 0; b < N; ++b) {
                        double t = 0.0;
                        for (int a = 0; a < N; ++a) t += (double)B.LV[a][r] * (double)ue[f * N * N + b * N + a];
                        s += (double)B.LV[b][q] * t;
                    }
                    qv[f] = s;
                }
                const double h = href + qv[0];
                if (!(h > 0.0)) { st |= DG_STATUS_NONPHYSICAL; continue; }
                const double uu = qv[1] / h, vv = qv[2] / h;
                best = fmax(best, sqrt(uu * uu + vv * vv) + sqrt(g * h));
            }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > 0.0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(best));
    if (st) atomicOr(status, st);
}

__device__ __forceinline__ void atomic_max_pos(float *a, float v)
{
    atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_pos(double *a, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(a), (unsigned long long)__double_as_longlong(v));
}

// Global Rusanov speeds of the stage state base + inc: the maxima of
// |u| + sqrt(g h) and |v| + sqrt(g h) over every Gauss point (one thread per
// element; non-physical points are left to the stage kernel to report).
// Positive floating-point values order like their bit patterns, so the
// atomic maxima on the bits are exact and order independent.
template <typename T, int N>
__global__ void global_speeds_kernel(const T *__restrict__ base, const T *__restrict__ inc, int nlon, int nel,
                                     int lanes, T href, T g, T *out)
{
    constexpr int NP = N * N, EL = 3 * NP;
    const BasisTab<T> &B = c_basis[N - 1];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    T su = T(0), sv = T(0);
    if (e < nel) {
        const int j = e / nlon, i = e - j * nlon;
        const size_t o0 = lanes ? (size_t)j * EL * nlon + i : (size_t)e * EL;
        const size_t ms = lanes ? (size_t)nlon : 1;
        T u[EL];
#pragma unroll
        for (int c = 0; c < EL; ++c) {
            u[c] = __ldg(base + o0 + c * ms);
            if (inc) u[c] += __ldg(inc + o0 + c * ms);
        }
#pragma unroll
        for (int be = 0; be < N; ++be)
#pragma unroll
            for (int al = 0; al < N; ++al) {
                T qv[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    T s = T(0);
#pragma unroll
                    for (int b = 0; b < N; ++b) {
                        T t = T(0);
#pragma unroll
                        for (int a = 0; a < N; ++a) t = fma(B.LV[a][al], u[f * NP + b * N + a], t);
                        s = fma(B.LV[b][be], t, s);
                    }
                    qv[f] = s;
                }
                const T h = href + qv[0];
                if (!(h > T(0))) continue;
                const T c = sqrt(g * h);
                su = fmax(su, fabs(qv[1] / h) + c);
                sv = fmax(sv, fabs(qv[2] / h) + c);
            }
    }
    for (int o = 16; o > 0; o >>= 1) {
        su = fmax(su, __shfl_xor_sync(0xffffffffu, su, o));
        sv = fmax(sv, __shfl_xor_sync(0xffffffffu, sv, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (su > T(0)) atomic_max_pos(out, su);
        if (sv > T(0)) atomic_max_pos(out + 1, sv);
    }
}

}  // namespace dgk

// ------------------------------------------------------ host-side launchers --

template <>
int dg_launch_global_speeds<DG_REAL>(int n, const DG_REAL *base, const DG_REAL *inc, int nlon, int nlat, int lanes,
                                     DG_REAL href, DG_REAL g, DG_REAL *out, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nel = nlon * nlat;
    const int threads = 128;
    const int blocks = (nel + threads - 1) / threads;
#define DG_GS(NN) dgk::global_speeds_kernel<DG_REAL, NN><<<blocks, threads, 0, s>>>(base, inc, nlon, nel, lanes, href, g, out)
    switch (n) {
    case 1: DG_GS(1); break;
    case 2: DG_GS(2); break;
    case 3: DG_GS(3); break;
    case 4: DG_GS(4); break;
    case 5: DG_GS(5); break;
    default: return 1;
    }
#undef DG_GS
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

template <>
int dg_upload_basis<DG_REAL>(const BasisTab<double> *all)
{
    BasisTab<DG_REAL> t[DG_MAXN];
    for (int n = 0; n < DG_MAXN; ++n) {
        for (int a = 0; a < DG_MAXN; ++a) {
            t[n].SE[a] = (DG_REAL)all[n].SE[a];
            t[n].SW[a] = (DG_REAL)all[n].SW[a];
            for (int q = 0; q < DG_MAXN; ++q) {
                t[n].LV[a][q] = (DG_REAL)all[n].LV[a][q];
                t[n].WLV[a][q] = (DG_REAL)all[n].WLV[a][q];
                t[n].WLD[a][q] = (DG_REAL)all[n].WLD[a][q];
            }
        }
    }
    return cudaMemcpyToSymbol(c_basis, t, sizeof(t)) == cudaSuccess ? 0 : 1;
}

template <>
int dg_launch_stage<DG_REAL>(int n, const StageArgs<DG_REAL> &a, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (n) {
    case 1: return dgk::launch_stage_n<DG_REAL, 1>(a, s);
    case 2: return dgk::launch_stage_n<DG_REAL, 2>(a, s);
    case 3: return dgk::launch_stage_n<DG_REAL, 3>(a, s);
    case 4: return dgk::launch_stage_n<DG_REAL, 4>(a, s);
    case 5: return dgk::launch_stage_n<DG_REAL, 5>(a, s);
    default: return 1;
    }
}

#ifdef DG_REAL_IS_F32   // the ensemble runs in FP32 only
template <>
int dg_launch_ensemble_stage<DG_REAL>(int tile_rows, int grid, const EnsArgs<DG_REAL> &a, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (tile_rows == DG_ENS_TILE_ROWS_A) return dgk::launch_ensemble_w<DG_REAL, DG_ENS_TILE_ROWS_A>(grid, a, s);
    if (tile_rows == DG_ENS_TILE_ROWS_B) return dgk::launch_ensemble_w<DG_REAL, DG_ENS_TILE_ROWS_B>(grid, a, s);
    return 1;
}
#endif

template <>
int dg_launch_to_internal<DG_REAL>(const double *src, DG_REAL *dst, DG_REAL *lo, size_t nel, int nphi, double href,
                                   void *stream)
{
    const size_t nval = nel * 3 * nphi;
    const int threads = 256;
    const size_t blocks = (nval + threads - 1) / threads;
    dgk::to_internal_kernel<DG_REAL><<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0,
                                       static_cast<cudaStream_t>(stream)>>>(src, dst, lo, nval, 3 * nphi, href);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

template <>
int dg_launch_to_api<DG_REAL>(const DG_REAL *src, const DG_REAL *lo, double *dst, size_t nel, int nphi, double href,
                              void *stream)
{
    const size_t nval = nel * 3 * nphi;
    const int threads = 256;
    const size_t blocks = (nval + threads - 1) / threads;
    dgk::to_api_kernel<DG_REAL><<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0,
                                  static_cast<cudaStream_t>(stream)>>>(src, lo, dst, nval, 3 * nphi, href);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

template <>
int dg_launch_mass<DG_REAL>(const DG_REAL *u, const DG_REAL *lo, const double *c0, int nlon, int nlat, int n,
                            double href, double dlam, double dth, double scale, double *partials, int nblocks,
                            double *result, double *pair, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nel = (size_t)nlon * nlat;
    const size_t chunk = (nel + nblocks - 1) / nblocks;
    dgk::mass_partial_kernel<DG_REAL><<<nblocks, dgk::MASS_THREADS, 0, s>>>(u, lo, c0, nlon, nlat, n, href,
                                                                            0.5 * dlam * dth, dlam, chunk, partials);
    dgk::mass_final_kernel<<<1, dgk::MASS_THREADS, 0, s>>>(partials, nblocks, scale, result, pair);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

template <>
int dg_launch_max_speed<DG_REAL>(const DG_REAL *u, int nlon, int nlat, int n, double href, double g,
                                 unsigned long long *maxbits, unsigned int *status, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nel = nlon * nlat;
    const int threads = 128;
    const int blocks = (nel + threads - 1) / threads;
    switch (n) {
    case 1: dgk::max_speed_kernel<DG_REAL, 1><<<blocks, threads, 0, s>>>(u, nel, href, g, maxbits, status); break;
    case 2: dgk::max_speed_kernel<DG_REAL, 2><<<blocks, threads, 0, s>>>(u, nel, href, g, maxbits, status); break;
    case 3: dgk::max_speed_kernel<DG_REAL, 3><<<blocks, threads, 0, s>>>(u, nel, href, g, maxbits, status); break;
    case 4: dgk::max_speed_kernel<DG_REAL, 4><<<blocks, threads, 0, s>>>(u, nel, href, g, maxbits, status); break;
    case 5: dgk::max_speed_kernel<DG_REAL, 5><<<blocks, threads, 0, s>>>(u, nel, href, g, maxbits, status); break;
    default: return 1;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

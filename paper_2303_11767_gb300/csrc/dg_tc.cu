// dg_tc.cu -- the fused RK stage with the basis contractions on the tensor
// cores of sm_103a: tcgen05.mma with BF16 or FP16 operands staged in shared
// memory and FP32 accumulators in tensor memory (TMEM).
//
// The element operator of paper Eq. (dg_parts) with the orthonormal Legendre
// basis is written as dense per-element maps:
//   GEMM1  modes -> values at the n x n Gauss points and at the 4n edge
//          points (S, N, W, E), one MMA per field over 128 elements;
//   GEMM2  [F | G | S | edge fluxes] -> the modal residual before the inverse
//          mass matrix, one MMA per field;
// the pointwise fluxes and sources (Eq. sph3), the Rusanov flux (Eq.
// rusanov, zero at the poles), the inverse of the per-row mass matrix C_j
// (Eq. ode) and the Runge-Kutta combination (Table Butcher) run on the CUDA
// cores in FP32.
//
// Thread mapping: thread = element.  A warp is one latitude row of the tile:
// lane 0 holds the element west of the tile, lanes 1..30 the interior, the
// lane after the last interior one the element east of it.  An MMA row is a
// TMEM lane, so every thread reads the accumulators of its own element.  The
// rows south and north of the tile go through a third MMA that produces only
// their edge traces.  The state arrays are lane-contiguous,
// [lat][field][mode][lon], so every global load and store of a warp is one
// contiguous segment.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "dg_internal.h"
#include "dg_flux.cuh"

namespace {

constexpr int TC_TW = 30;            // interior elements of a warp row
constexpr uint32_t CH = 2048;        // bytes of one 8-wide K chunk of a 128-row operand
constexpr uint32_t TMEM_COLS = 256;  // tensor-memory columns of one CTA (two CTAs per SM)
constexpr int WAIT_LIMIT = 1 << 22;  // bounded wait for the tensor cores

// Padded sizes of the per-element maps for n = p + 1 points per direction.
//   GEMM1: K1 modes (NP, padded to 16) -> N1 columns: NC node columns (NP
//          padded to 8), then the 4n traces S, N, W, E (n each)
//   GEMM2: K2 = 8 * KC2 inputs: chunks [0, CN) F, [CN, 2CN) G, [2CN, 3CN) S,
//          then CE chunks of edge fluxes (W, E, S, N, EW slots each)
//          -> N2 output modes (NP padded to 16)
template <int N>
struct TcGeo {
    static constexpr int NP = N * N;
    static constexpr int CN = (NP + 7) / 8;
    static constexpr int NC = 8 * CN;
    static constexpr int K1 = 16 * ((NP + 15) / 16);
    static constexpr int K1C = K1 / 8;
    static constexpr int N1 = 16 * ((NC + (4 * N > 16 ? 4 * N : 16) + 15) / 16);
    static constexpr int N2 = 16 * ((NP + 15) / 16);
    static constexpr int EW = N <= 4 ? 4 : 8;
    static constexpr int CE = 4 * EW / 8;
    static constexpr int KC2 = ((3 * CN + CE + 1) / 2) * 2;
    static constexpr int K2 = 8 * KC2;
    static constexpr int TRC = (4 * N + 7) / 8 * 8;   // trace columns read back
};

// Threads per element: warps w and w + 4 share TMEM lane quarter w & 3 (the
// same 32 elements) and split the element's work, which doubles the warps
// that hide latency and halves each thread's serial chain.
constexpr int TC_TPE = 2;

// Shared-memory plan (bytes) of one 4-row tile.  A1 / A1h (GEMM1 operands
// of the tile and of the halo rows) are dead once GEMM1 has completed, so
// GEMM2's operand A2 reuses the region.  Field h has no source term: its S
// chunks of A2 are never written and GEMM2 skips them (whole K steps, so CN
// must be even).  The 16-bit row exchange of the theta faces (XN: N traces,
// XS: S-face fluxes) lives there when it fits, else in its own region.
//
// SPLIT: every operand is held as a pair (hi, lo) of 16-bit values, x ~ hi +
// lo with lo the rounded residual x - hi, and every product A B is taken as
// A_hi B_hi + A_lo B_hi + A_hi B_lo (three MMAs per K step into the same FP32
// accumulator), which leaves an error of order u^2 instead of u per term.
// The lo operands follow the hi ones (B1L, B2L; A lo = A hi + LO1 for GEMM1,
// + LO2 for GEMM2).  The theta-face exchange carries FP32 values: XN in its
// own region, XS (read as fluxes into the A2 pairs) in field h's unused S
// chunks of the hi (rows 0, 1) and lo (rows 2, 3) operands when they fit.
// At degree 4 the split plan needs 223 KB: one CTA per SM.
template <int N, bool SPLIT = false>
struct TcSmem {
    using GE = TcGeo<N>;
    static constexpr int NB = SPLIT ? 2 : 1;   // copies of each operand (hi, lo)
    static constexpr uint32_t B1 = 0;
    static constexpr uint32_t SZ_B1 = GE::N1 * GE::K1 * 2;
    static constexpr uint32_t B1L = B1 + SZ_B1;
    static constexpr uint32_t B2 = (NB * SZ_B1 + 127) / 128 * 128;
    static constexpr uint32_t SZ_B2 = GE::N2 * GE::K2 * 2;
    static constexpr uint32_t B2L = B2 + SZ_B2;
    static constexpr uint32_t A = (B2 + NB * SZ_B2 + 1023) / 1024 * 1024;
    static constexpr uint32_t SZ_A1 = 3 * GE::K1C * CH;
    static constexpr uint32_t SZ_A1H = 3 * GE::K1C * CH;
    static constexpr uint32_t SZ_A2 = 3 * GE::KC2 * CH;
    static constexpr uint32_t LO1 = SZ_A1 + SZ_A1H;   // GEMM1 lo operands after the hi ones
    static constexpr uint32_t LO2 = SZ_A2;            // GEMM2 lo operand after the hi one
    static constexpr uint32_t SZ_A = NB * (SZ_A1 + SZ_A1H > SZ_A2 ? SZ_A1 + SZ_A1H : SZ_A2);
    static constexpr bool SKIP_S0 = GE::CN % 2 == 0;
    // 16-bit exchange (one array) / FP32 exchange (one array, or half of one)
    static constexpr uint32_t SZ_X = SPLIT ? 4 * 32 * 3 * N * 4 : 4 * 32 * 3 * N * 2;
    static constexpr bool X_IN_S0 = SKIP_S0 && (SPLIT ? SZ_X / 2 : 2 * SZ_X) <= GE::CN * CH;
    // non-split: XN and XS together in the S chunks of field h, else after A;
    // split: XN after A, XS halves in the S chunks of field h (hi and lo) or after XN
    static constexpr uint32_t S0 = A + 2 * GE::CN * CH;
    static constexpr uint32_t XN = SPLIT ? A + SZ_A : X_IN_S0 ? S0 : A + SZ_A;
    static constexpr uint32_t XS = SPLIT ? (X_IN_S0 ? S0 : XN + SZ_X) : XN + SZ_X;
    static constexpr uint32_t XS_HI = SPLIT && X_IN_S0 ? S0 + LO2 : XS + SZ_X / 2;   // rows 2, 3
    static constexpr uint32_t BYTES =
        A + SZ_A + (SPLIT ? (X_IN_S0 ? SZ_X : 2 * SZ_X) : (X_IN_S0 ? 0 : 2 * SZ_X));
    static constexpr int CTAS = BYTES <= 113 * 1024 ? 2 : 1;   // CTAs per SM
    static_assert(3 * GE::N1 + 48 <= (int)TMEM_COLS, "tensor-memory columns");
    static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
    static_assert(SPLIT || CTAS == 2, "two CTAs per SM");
};

template <typename OpT>
struct Op;
template <>
struct Op<__nv_bfloat16> {
    static constexpr bool bf16 = true;
    static constexpr float mom_scale = 1.0f;
    __device__ static uint32_t pack(float a, float b)
    {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&v);
    }
    __device__ static uint16_t to16(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    __device__ static float from16(uint16_t u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
    static uint16_t host_bits(float x)
    {
        __nv_bfloat16 v = __float2bfloat16_rn(x);
        uint16_t u;
        std::memcpy(&u, &v, 2);
        return u;
    }
    static float host_value(uint16_t u)
    {
        __nv_bfloat16 v;
        std::memcpy(&v, &u, 2);
        return __bfloat162float(v);
    }
};
template <>
struct Op<__half> {
    static constexpr bool bf16 = false;
    // momenta of up to 2^21 m^2/s stay inside the FP16 range; a power of two,
    // so the scaling itself is exact
    static constexpr float mom_scale = 1.0f / 32.0f;
    __device__ static uint32_t pack(float a, float b)
    {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&v);
    }
    __device__ static uint16_t to16(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ static float from16(uint16_t u) { return __half2float(__ushort_as_half(u)); }
    static uint16_t host_bits(float x)
    {
        __half v = __float2half_rn(x);
        uint16_t u;
        std::memcpy(&u, &v, 2);
        return u;
    }
    static float host_value(uint16_t u)
    {
        __half v;
        std::memcpy(&v, &u, 2);
        return __half2float(v);
    }
};

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8
// rows x 16 bytes; lbo = byte distance of K-adjacent core matrices, sbo = of
// row-adjacent (M or N) ones.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B of the same
// 16-bit type, both K-major, M x N.
template <bool BF16>
__host__ __device__ constexpr uint32_t idesc(int M, int N)
{
    return (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for phase `parity` of the barrier, giving up after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

// Barrier among the 4 warps of one part of the CTA (id 1; id 0 is __syncthreads).
__device__ __forceinline__ void part_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive accumulator columns of the thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Ties 8 registers to the point after tmem_wait(): no use of them can be
// scheduled before the loads have landed.
__device__ __forceinline__ void reg_fence8(float *v)
{
    asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]));
}

template <typename OpT>
__device__ __forceinline__ void put_chunk(unsigned char *p, const float *v)
{
    uint4 u;
    u.x = Op<OpT>::pack(v[0], v[1]);
    u.y = Op<OpT>::pack(v[2], v[3]);
    u.z = Op<OpT>::pack(v[4], v[5]);
    u.w = Op<OpT>::pack(v[6], v[7]);
    *reinterpret_cast<uint4 *>(p) = u;
}

// The pair (hi, lo) of 8 values: hi = the rounded value, lo = the rounded
// residual v - hi; written to p and p + lo_off.
template <typename OpT>
__device__ __forceinline__ void put_chunk_split(unsigned char *p, uint32_t lo_off, const float *v)
{
    float hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        hi[k] = Op<OpT>::from16(Op<OpT>::to16(v[k]));
        lo[k] = v[k] - hi[k];
    }
    put_chunk<OpT>(p, hi);
    put_chunk<OpT>(p + lo_off, lo);
}

// ------------------------------------------------------------ stage kernel --

template <int N, typename OpT, bool SPLIT>
__global__ void __launch_bounds__(128 * TC_TPE, TcSmem<N, SPLIT>::CTAS) tc_stage_kernel(const StageArgs<float> A,
                                                                   const uint4 *__restrict__ gB1,
                                                                   const uint4 *__restrict__ gB2)
{
    using GE = TcGeo<N>;
    using SM = TcSmem<N, SPLIT>;
    constexpr int NP = GE::NP, CN = GE::CN, NC = GE::NC, K1C = GE::K1C, N1 = GE::N1, N2 = GE::N2, EW = GE::EW,
                  KC2 = GE::KC2, TRC = GE::TRC;
    constexpr int NT = 128 * TC_TPE;
    constexpr int PE = 0, PN = 1 % TC_TPE;   // parts doing the lambda / theta faces
    constexpr float MS = Op<OpT>::mom_scale, IMS = 1.0f / Op<OpT>::mom_scale;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;

    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int q4 = w & 3, part = w >> 2;   // tile row (= TMEM lane quarter) and share of the element's work
    const int i0 = blockIdx.x * TC_TW, j0 = blockIdx.y * 4;
    const int Gv = min(TC_TW, A.nlon - i0), Wv = min(4, A.nlat - j0);
    const bool row_ok = q4 < Wv;
    const int j = row_ok ? j0 + q4 : j0;   // rows past the mesh borrow the first row's tables
    const bool lane_ok = l <= Gv + 1;
    const bool interior = row_ok && l >= 1 && l <= Gv;
    // longitude of lane l (lanes 0 and Gv + 1 are the W / E halo columns,
    // periodic in lambda; lanes past Gv + 1 load nothing)
    const int il = i0 + l - 1;
    const int i = !lane_ok ? 0 : il < 0 ? il + A.nlon : il >= A.nlon ? il - A.nlon : il;
    const size_t rowlen = (size_t)3 * NP * A.nlon;
    const float href = A.href, gg = A.g;
    unsigned st = 0, st_int = 0;   // status of any thread / of interior elements only
    const uint32_t rowoff = (uint32_t)(32 * q4 + l) * 16;
    unsigned char *const opA = sm + SM::A;
    const RowTab<float> *const RT = A.rows + j;
    float ga_l = 0.0f, ga_t = 0.0f;   // global Rusanov speeds (0 = local mode), read after the dependency wait

    // prologue (independent of the previous kernel's results): tensor
    // memory, the completion barrier, the two basis operands
    if (w == 0) tmem_alloc(smem_u32(&tslot));
    if (tid == 0) mbar_init(smem_u32(&mbar));
    // (hi, then lo in SPLIT mode)
    for (int c = tid; c < (int)(SM::NB * SM::SZ_B1 / 16); c += NT)
        reinterpret_cast<uint4 *>(sm + SM::B1)[c] = __ldg(gB1 + c);
    for (int c = tid; c < (int)(SM::NB * SM::SZ_B2 / 16); c += NT)
        reinterpret_cast<uint4 *>(sm + SM::B2)[c] = __ldg(gB2 + c);
    dgk::pdl_wait();
    if (A.galpha) {
        ga_l = __ldg(A.galpha);
        ga_t = __ldg(A.galpha + 1);
    }

    // operand rows: one 16-bit value, or the (hi, lo) pair in SPLIT mode
    auto put_a1 = [&](unsigned char *dst, const float *v) {
        if constexpr (SPLIT) put_chunk_split<OpT>(dst, SM::LO1, v);
        else put_chunk<OpT>(dst, v);
    };
    auto put_a2 = [&](unsigned char *dst, const float *v) {
        if constexpr (SPLIT) put_chunk_split<OpT>(dst, SM::LO2, v);
        else put_chunk<OpT>(dst, v);
    };

    // ---- S0: 8 modes (chunk c) of one field of the stage state u = base + inc
    //      of one element -> its row of a GEMM1 operand (zeros where missing)
    auto stage_chunk = [&](int jj, bool ok, int f, int c, unsigned char *dst) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0f;
        if (ok) {
            const float s = f == 0 ? 1.0f : MS;
            const size_t o0 = (size_t)jj * rowlen + (size_t)(f * NP + 8 * c) * A.nlon + i;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (8 * c + k < NP) v[k] = __ldg(A.base + o0 + (size_t)k * A.nlon);
            if (A.inc) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (8 * c + k < NP) v[k] += __ldg(A.inc + o0 + (size_t)k * A.nlon);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] *= s;
        }
        put_a1(dst + c * CH, v);
    };
    // the low parts and the RK4 accumulator are read only by the epilogue:
    // start moving this thread's share of them into L2 now
    if (interior && (A.lo || A.acc_in)) {
        const float *pl = A.lo ? A.lo : A.acc_in;
        const size_t o0 = (size_t)j * rowlen + i;
        for (int m = part; m < 3 * NP; m += TC_TPE)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + o0 + (size_t)m * A.nlon));
    }
    // the tile rows: part p stages the chunks c = p, p + TPE, ... (all of its
    // loads in flight before the first conversion)
#pragma unroll
    for (int fc = 0; fc < 3 * K1C; fc += TC_TPE) {
        if (fc + part < 3 * K1C) {
            const int f = (fc + part) / K1C, c = (fc + part) - f * K1C;
            stage_chunk(j0 + q4, row_ok && lane_ok, f, c, opA + (uint32_t)(f * K1C) * CH + rowoff);
        }
    }
    // halo rows: job = (side * 3 + f) * K1C + c; side 0 = the row south of
    // the tile (TMEM quarter 0), side 1 = the row north of it (quarter 3)
#pragma unroll
    for (int job0 = 0; job0 < 6 * K1C; job0 += 4 * TC_TPE) {
        const int job = job0 + w;
        if (job >= 6 * K1C) break;
        const int sf = job / K1C, c = job - sf * K1C;
        const int side = sf / 3, f = sf - 3 * side;
        const int jj = side ? j0 + 4 : j0 - 1;
        const bool ok = lane_ok && (side ? jj < A.nlat : jj >= 0);
        stage_chunk(ok ? jj : 0, ok, f, c, opA + SM::SZ_A1 + (uint32_t)(f * K1C) * CH + (uint32_t)((side ? 96 : 0) + l) * 16);
    }

    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot;
    const uint32_t mb = smem_u32(&mbar);
    const uint32_t a0 = smem_u32(opA);

    // ---- S1 + S4 on the tensor cores: values at the Gauss and edge points
    if (tid == 0) {
        const uint32_t b1 = smem_u32(sm + SM::B1);
        constexpr uint32_t LB1 = N1 * 16;
        constexpr uint32_t id1 = idesc<Op<OpT>::bf16>(128, N1), idh = idesc<Op<OpT>::bf16>(128, 16);
        // A B, or A_hi B_hi + A_lo B_hi + A_hi B_lo in SPLIT mode
        auto mma3 = [&](uint32_t d, uint32_t a, uint32_t lo_a, uint32_t b, uint32_t lo_b, uint32_t lbo_b,
                        uint32_t id, uint32_t acc) {
            mma(d, sdesc(a, CH, 128), sdesc(b, lbo_b, 128), id, acc);
            if constexpr (SPLIT) {
                mma(d, sdesc(a + lo_a, CH, 128), sdesc(b, lbo_b, 128), id, 1);
                mma(d, sdesc(a, CH, 128), sdesc(b + lo_b, lbo_b, 128), id, 1);
            }
        };
        constexpr uint32_t LOB1 = SM::B1L - SM::B1;
        for (int f = 0; f < 3; ++f)
            for (int s = 0; s < K1C / 2; ++s)
                mma3(tbase + (uint32_t)(f * N1), a0 + (uint32_t)(f * K1C + 2 * s) * CH, SM::LO1,
                     b1 + 2 * s * LB1, LOB1, LB1, id1, s > 0);
        for (int f = 0; f < 3; ++f)
            for (int s = 0; s < K1C / 2; ++s)
                mma3(tbase + (uint32_t)(3 * N1 + 16 * f), a0 + SM::SZ_A1 + (uint32_t)(f * K1C + 2 * s) * CH, SM::LO1,
                     b1 + NC * 16 + 2 * s * LB1, LOB1, LB1, idh, s > 0);
        mma_commit(mb);
    }
    if (!mbar_wait(mb, 0)) st |= DG_STATUS_TIMEOUT;
    tc_fence_after();
    __syncwarp();

    const uint32_t tl = tbase + ((uint32_t)(32 * q4) << 16);
    unsigned char *const a2row = opA + rowoff;
    auto a2 = [&](int f, int c) { return a2row + (uint32_t)(f * KC2 + c) * CH; };
    // theta-face row exchange: N traces (XN) and S-face fluxes (XS) of tile
    // row q, field f, point k, lane l; 16-bit values (unscaled, as the
    // operands), or FP32 in SPLIT mode (XS rows 2, 3 in a second half)
    uint16_t *XN = reinterpret_cast<uint16_t *>(sm + SM::XN);
    uint16_t *XS = reinterpret_cast<uint16_t *>(sm + SM::XS);
    auto xn_put = [&](int q, int f, int k, float v) {
        if constexpr (SPLIT) reinterpret_cast<float *>(sm + SM::XN)[((q * 3 + f) * N + k) * 32 + l] = v;
        else XN[((q * 3 + f) * N + k) * 32 + l] = Op<OpT>::to16(v * (f == 0 ? 1.0f : MS));
    };
    auto xn_get = [&](int q, int f, int k) -> float {
        if constexpr (SPLIT) return reinterpret_cast<const float *>(sm + SM::XN)[((q * 3 + f) * N + k) * 32 + l];
        else return Op<OpT>::from16(XN[((q * 3 + f) * N + k) * 32 + l]) * (f == 0 ? 1.0f : IMS);
    };
    auto xs_slot = [&](int q, int f, int k) -> float * {
        return reinterpret_cast<float *>(sm + (q < 2 ? SM::XS : SM::XS_HI)) + (((q & 1) * 3 + f) * N + k) * 32 + l;
    };
    auto xs_put = [&](int q, int f, int k, float v) {
        if constexpr (SPLIT) *xs_slot(q, f, k) = v;
        else XS[((q * 3 + f) * N + k) * 32 + l] = Op<OpT>::to16(v);
    };
    auto xs_get = [&](int q, int f, int k) -> float {
        if constexpr (SPLIT) return *xs_slot(q, f, k);
        else return Op<OpT>::from16(XS[((q * 3 + f) * N + k) * 32 + l]);
    };

    // own traces of 3 fields, columns [NC + c0, NC + c0 + 2N): (S, N) for
    // c0 = 0, (W, E) for c0 = 2N; unscaled
    auto load_traces = [&](int c0, float (*t)[2 * N]) {
        constexpr int C8 = (2 * N + 7) / 8 + 1;   // 8-column loads covering [c0, c0 + 2N) from an aligned start
        float raw[3][8 * C8];
        const int base = (NC + c0) & ~7, sh = (NC + c0) & 7;
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int c = 0; c < C8; ++c) tmem_ld8(tl + (uint32_t)(f * N1 + base + 8 * c), &raw[f][8 * c]);
        tmem_wait();
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int c = 0; c < C8; ++c) reg_fence8(&raw[f][8 * c]);
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int k = 0; k < 2 * N; ++k) t[f][k] = (sh ? raw[f][sh + k] : raw[f][k]) * (f == 0 ? 1.0f : IMS);
    };
    (void)TRC;

    // ---- S5 lambda faces (part PE): lanes 1..Gv+1 evaluate their W edge (the
    //      last one is the tile's east boundary); the E edge is the next
    //      lane's W edge
    if (part == PE) {
        float twe[3][2 * N];   // [0, N) W, [N, 2N) E
        load_traces(2 * N, twe);
        float efW[3][N], efE[3][N];
        unsigned sw = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            float L[3], R[3], o[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                L[f] = __shfl_up_sync(0xffffffffu, twe[f][N + k], 1);
                R[f] = twe[f][k];
            }
            dgk::rusanov_lam(L, R, href, gg, A.cF, o, sw, ga_l);
#pragma unroll
            for (int f = 0; f < 3; ++f) efW[f][k] = o[f];
        }
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int k = 0; k < N; ++k) efE[f][k] = __shfl_down_sync(0xffffffffu, efW[f][k], 1);
        if (row_ok && l >= 1 && l <= Gv + 1) st_int |= sw;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            float c0[8], c1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) c0[k] = c1[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                c0[k] = efW[f][k];
                if (EW == 4) c0[4 + k] = efE[f][k];
                else c1[k] = efE[f][k];
            }
            put_a2(a2(f, 3 * CN), c0);
            if (EW == 8) put_a2(a2(f, 3 * CN + 1), c1);
#pragma unroll
            for (int c = 3 * CN + GE::CE; c < KC2; ++c) {   // zero K padding
                float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                put_a2(a2(f, c), z);
            }
        }
    }

    // ---- S5 theta faces (part PN) through the 16-bit row exchange (the
    //      faces' fluxes are rounded to the operand type in A2 anyway; the
    //      neighbour's trace carries one rounding of the operand type; FP32
    //      in SPLIT mode, where A2 holds the fluxes to ~u^2): every
    //      element evaluates its S edge; its N edge is the S edge of the
    //      element above (for the top row of a full tile: evaluated against
    //      the halo).  Only part PN's warps meet at these barriers; the other
    //      part goes on to the Gauss-point fluxes.
    float tsn[3][2 * N];   // [0, N) S, [N, 2N) N
    float halo[3][N];      // row 0: N trace of the row south; row 3: S trace of the row north
    if (part == PN) {
        load_traces(0, tsn);
        if (q4 == 0 || q4 == 3) {
            float hv[3][16];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                tmem_ld8(tl + (uint32_t)(3 * N1 + 16 * f), hv[f]);
                tmem_ld8(tl + (uint32_t)(3 * N1 + 16 * f + 8), hv[f] + 8);
            }
            tmem_wait();
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                reg_fence8(hv[f]);
                reg_fence8(hv[f] + 8);
            }
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int k = 0; k < N; ++k) halo[f][k] = (q4 == 0 ? hv[f][N + k] : hv[f][k]) * (f == 0 ? 1.0f : IMS);
        }
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int k = 0; k < N; ++k)
                xn_put(q4, f, k, tsn[f][N + k]);
        part_barrier();
    }
    float efS[3][N];
    if (part == PN) {
        const float cgs = A.cG * __ldg(&RT->ce_s);
        unsigned ss = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            float Sq[3], Nq[3], o[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                Sq[f] = q4 > 0 ? xn_get(q4 - 1, f, k) : halo[f][k];
                Nq[f] = tsn[f][k];
            }
            dgk::rusanov_th(Sq, Nq, href, gg, cgs, o, ss, ga_t);
#pragma unroll
            for (int f = 0; f < 3; ++f) efS[f][k] = j0 + q4 > 0 ? o[f] : 0.0f;   // pole edge: zero flux
        }
        if (interior && j0 + q4 > 0) st_int |= ss;
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int k = 0; k < N; ++k) xs_put(q4, f, k, efS[f][k]);
        part_barrier();
    }
    float efN[3][N];
    if (part == PN) {
        if (q4 + 1 < Wv) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int k = 0; k < N; ++k) efN[f][k] = xs_get(q4 + 1, f, k);
        } else if (j0 + q4 + 1 >= A.nlat) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int k = 0; k < N; ++k) efN[f][k] = 0.0f;   // pole edge (or a row past the mesh)
        } else {   // the top row of a full tile: its N neighbours are the halo row
            const float cgn = A.cG * __ldg(&RT->ce_n);
            unsigned sn = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                float Sq[3], Nq[3], o[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    Sq[f] = tsn[f][N + k];
                    Nq[f] = halo[f][k];
                }
                dgk::rusanov_th(Sq, Nq, href, gg, cgn, o, sn, ga_t);
#pragma unroll
                for (int f = 0; f < 3; ++f) efN[f][k] = o[f];
            }
            if (interior) st_int |= sn;
        }
    }
    if (part == PN) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            float c0[8], c1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) c0[k] = c1[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                c0[k] = efS[f][k];
                if (EW == 4) c0[4 + k] = efN[f][k];
                else c1[k] = efN[f][k];
            }
            if (EW == 4) put_a2(a2(f, 3 * CN + 1), c0);
            else {
                put_a2(a2(f, 3 * CN + 2), c0);
                put_a2(a2(f, 3 * CN + 3), c1);
            }
        }
    }

    // ---- S2 pointwise fluxes and sources at the Gauss points, 8 at a time;
    //      part p takes the chunks g = p, p + TPE, ...
    {
        unsigned sq = 0;
#pragma unroll 1
        for (int g = part; g < CN; g += TC_TPE) {
            float x[3][8];
#pragma unroll
            for (int f = 0; f < 3; ++f) tmem_ld8(tl + (uint32_t)(f * N1 + 8 * g), x[f]);
            tmem_wait();
#pragma unroll
            for (int f = 0; f < 3; ++f) reg_fence8(x[f]);
            float Fv[3][8], Gq[3][8], Sv[3][8];
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                const int q = 8 * g + qq;
                if (q < NP) {
                    const int be = q / N;
                    const float hp = x[0][qq], hu = x[1][qq] * IMS, hv = x[2][qq] * IMS;
                    const float h = href + hp;
                    dgk::check_depth(h, sq);
                    const float rh = dgk::rcp(h);
                    const float u = hu * rh, v = hv * rh;
                    const float P = hp * gg * fmaf(0.5f, hp, href);
                    const float c = __ldg(&RT->cosn[be]), sn = __ldg(&RT->sinn[be]);
                    Fv[0][qq] = A.cF * hu;
                    Fv[1][qq] = A.cF * fmaf(hu, u, P);
                    Fv[2][qq] = A.cF * (hu * v);
                    const float cGc = A.cG * c;
                    Gq[0][qq] = cGc * hv;
                    Gq[1][qq] = cGc * (hv * u);
                    Gq[2][qq] = cGc * fmaf(hv, v, P);
                    const float K = sn * fmaf(A.twoOmega, c, u * A.invR);
                    Sv[0][qq] = 0.0f;
                    Sv[1][qq] = K * hv;
                    Sv[2][qq] = -(P * sn * A.invR) - K * hu;
                } else {
#pragma unroll
                    for (int f = 0; f < 3; ++f) Fv[f][qq] = Gq[f][qq] = Sv[f][qq] = 0.0f;
                }
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                put_a2(a2(f, g), Fv[f]);
                put_a2(a2(f, CN + g), Gq[f]);
                if (f > 0 || !SM::SKIP_S0) put_a2(a2(f, 2 * CN + g), Sv[f]);
            }
        }
        if (interior) st_int |= sq;
    }

    // ---- S3 + S6 on the tensor cores: volume integral and lift
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        const uint32_t b2 = smem_u32(sm + SM::B2);
        constexpr uint32_t LB2 = N2 * 16;
        constexpr uint32_t id2 = idesc<Op<OpT>::bf16>(128, N2);
        constexpr uint32_t LOB2 = SM::B2L - SM::B2;
        for (int f = 0; f < 3; ++f)
            for (int s = 0; s < KC2 / 2; ++s) {
                if (f == 0 && SM::SKIP_S0 && 2 * s >= 2 * CN && 2 * s < 3 * CN) continue;   // S_h = 0
                const uint32_t d = tbase + (uint32_t)(f * N1), a = a0 + (uint32_t)(f * KC2 + 2 * s) * CH;
                const uint32_t b = b2 + 2 * s * LB2;
                mma(d, sdesc(a, CH, 128), sdesc(b, LB2, 128), id2, s > 0);
                if constexpr (SPLIT) {
                    mma(d, sdesc(a + SM::LO2, CH, 128), sdesc(b, LB2, 128), id2, 1);
                    mma(d, sdesc(a, CH, 128), sdesc(b + LOB2, LB2, 128), id2, 1);
                }
            }
        mma_commit(mb);
    }
    if (!mbar_wait(mb, 1)) st |= DG_STATUS_TIMEOUT;
    tc_fence_after();
    __syncwarp();

    // ---- S7 inverse mass matrix (FP32 on the CUDA cores), S8 combine, store.
    //      Part p owns the mode rows b of field f with (f N + b) mod TPE = p;
    //      per field, all of its global inputs are requested before the first
    //      is used.
    {
        constexpr int RPF = (N + TC_TPE - 1) / TC_TPE;   // rows per field and part, at most
        const size_t e0 = (size_t)j * rowlen + i;
        const float cdt = A.cc * A.dt, adt = A.ca * A.dt;
        const bool fin = A.out_base != nullptr;
        float chk = 0.0f;   // non-finite tendency or state of an interior element: NaN (nf_acc)
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            const int b0 = ((part - f * N) % TC_TPE + TC_TPE) % TC_TPE;
            float vinc[RPF][N], vacc[RPF][N], vbase[RPF][N], vlo[RPF][N];
#pragma unroll
            for (int rr = 0; rr < RPF; ++rr) {
                const int b = b0 + rr * TC_TPE;
                const bool ok = interior && b < N;
                const size_t ob = e0 + (size_t)(f * NP + b * N) * A.nlon;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    const size_t o = ob + (size_t)(a * A.nlon);
                    vinc[rr][a] = ok && A.inc ? __ldg(A.inc + o) : 0.0f;
                    vacc[rr][a] = ok && A.acc_in ? __ldg(A.acc_in + o) : 0.0f;
                    vbase[rr][a] = ok && fin ? __ldg(A.base + o) : 0.0f;
                    vlo[rr][a] = ok && fin && A.lo ? __ldg(A.lo + o) : 0.0f;
                }
            }
            float r[8 * CN];
#pragma unroll
            for (int c = 0; c < CN; ++c) tmem_ld8(tl + (uint32_t)(f * N1 + 8 * c), r + 8 * c);
            tmem_wait();
#pragma unroll
            for (int c = 0; c < CN; ++c) reg_fence8(r + 8 * c);
#pragma unroll
            for (int rr = 0; rr < RPF; ++rr) {
                const int b = b0 + rr * TC_TPE;
                if (b >= N) break;
                float kk[N];
#pragma unroll
                for (int a = 0; a < N; ++a) kk[a] = 0.0f;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    const float cic = __ldg(&RT->Ci[b][c]);
#pragma unroll
                    for (int a = 0; a < N; ++a) kk[a] = fmaf(cic, r[c * N + a], kk[a]);
                }
                if (f == 2) kk[0] = fmaf(A.P0, __ldg(&RT->rho[b]), kk[0]);
                if (interior) {
                    const size_t ob = e0 + (size_t)(f * NP + b * N) * A.nlon;
#pragma unroll
                    for (int a = 0; a < N; ++a) {
                        const size_t o = ob + (size_t)(a * A.nlon);
                        const float kv = kk[a], inc = vinc[rr][a], acc = vacc[rr][a];
                        chk = dgk::nf_acc(kv, chk);
                        if (A.out_rhs) A.out_rhs[o] = kv;
                        if (A.inc_out) A.inc_out[o] = fmaf(cdt, kv, A.ci * inc);
                        if (A.acc_out) A.acc_out[o] = fmaf(adt, kv, acc);
                        if (fin) {
                            // u^{n+1} = (base + lo) + delta with an error-free two-sum
                            const float bs = vbase[rr][a], lo = vlo[rr][a];
                            const float delta = fmaf(cdt, kv, fmaf(A.cd, acc, A.ci * inc));
                            const float s1 = bs + delta;
                            const float bp = s1 - bs;
                            const float err = (bs - (s1 - bp)) + (delta - bp);
                            const float l1 = lo + err;
                            const float hi = s1 + l1;
                            A.out_base[o] = hi;
                            if (A.out_lo) A.out_lo[o] = l1 - (hi - s1);
                            chk = dgk::nf_acc(hi, chk);
                        }
                    }
                }
            }
        }
        if (!isfinite(chk)) st_int |= DG_STATUS_NONFINITE;
    }

    dgk::pdl_launch_dependents();
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(tbase);
    if (interior) st |= st_int;
    if (st) atomicOr(A.status, st);
}

// --------------------------------------------------- contraction check ------

// One GEMM1 of the degree's eval/trace matrix on a 128-row operand, read
// back from TMEM: the tensor-core building block in isolation.
template <int N, typename OpT>
__global__ void __launch_bounds__(128) tc_gemm_check_kernel(const float *__restrict__ a, float *__restrict__ d,
                                                            const uint4 *__restrict__ gB1, unsigned *status)
{
    using GE = TcGeo<N>;
    constexpr int K1 = GE::K1, K1C = GE::K1C, N1 = GE::N1;
    constexpr uint32_t SZ_B1 = N1 * K1 * 2, OFF_A = (SZ_B1 + 1023) / 1024 * 1024;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, w = tid >> 5;
    if (w == 0) tmem_alloc(smem_u32(&tslot));
    if (tid == 0) mbar_init(smem_u32(&mbar));
    for (int c = tid; c < (int)(SZ_B1 / 16); c += 128) reinterpret_cast<uint4 *>(sm)[c] = __ldg(gB1 + c);
    float v[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) v[k] = a[tid * K1 + k];
#pragma unroll
    for (int c = 0; c < K1C; ++c) put_chunk<OpT>(sm + OFF_A + c * CH + tid * 16, v + 8 * c);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot, mb = smem_u32(&mbar);
    if (tid == 0) {
        constexpr uint32_t LB1 = N1 * 16;
        for (int s = 0; s < K1C / 2; ++s)
            mma(tbase, sdesc(smem_u32(sm + OFF_A) + 2 * s * CH, CH, 128), sdesc(smem_u32(sm) + 2 * s * LB1, LB1, 128),
                idesc<Op<OpT>::bf16>(128, N1), s > 0);
        mma_commit(mb);
    }
    const bool ok = mbar_wait(mb, 0);
    tc_fence_after();
    __syncwarp();
    const uint32_t tl = tbase + ((uint32_t)(32 * w) << 16);
#pragma unroll
    for (int c = 0; c < N1 / 8; ++c) {
        float r[8];
        tmem_ld8(tl + 8 * c, r);
        tmem_wait();
        reg_fence8(r);
#pragma unroll
        for (int k = 0; k < 8; ++k) d[tid * N1 + 8 * c + k] = r[k];
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(tbase);
    if (!ok) atomicOr(status, DG_STATUS_TIMEOUT);
}

// ------------------------------------------------------------ permutation --

// [lat][lon][el] <-> [lat][el][lon], 32 x 32 tiles through shared memory.
__global__ void permute_kernel(const float *__restrict__ src, float *__restrict__ dst, int nlon, int el,
                               int to_lanes)
{
    __shared__ float t[32][33];
    const int j = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;   // r: lon, c: el (in the [lon][el] view)
    const size_t base = (size_t)j * nlon * el;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        if (to_lanes) {
            const int r = r0 + y, c = c0 + threadIdx.x;
            if (r < nlon && c < el) t[y][threadIdx.x] = src[base + (size_t)r * el + c];
        } else {
            const int c = c0 + y, r = r0 + threadIdx.x;
            if (r < nlon && c < el) t[threadIdx.x][y] = src[base + (size_t)c * nlon + r];
        }
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        if (to_lanes) {
            const int c = c0 + y, r = r0 + threadIdx.x;
            if (r < nlon && c < el) dst[base + (size_t)c * nlon + r] = t[threadIdx.x][y];
        } else {
            const int r = r0 + y, c = c0 + threadIdx.x;
            if (r < nlon && c < el) dst[base + (size_t)r * el + c] = t[y][threadIdx.x];
        }
    }
}

// ------------------------------------------------------------- host side ----

// Operand B of both GEMMs in the canonical K-major layout: element (r, k) of
// an R-row operand at byte (k / 8) * R * 16 + r * 16 + (k % 8) * 2.
// SPLIT: each table is followed by its lo part, the rounded residual of the
// FP32 value after the hi rounding.
template <int N, typename OpT>
void build_tables(std::vector<uint16_t> &b1, std::vector<uint16_t> &b2, bool split)
{
    using GE = TcGeo<N>;
    constexpr int NP = GE::NP, NC = GE::NC, K1 = GE::K1, N1 = GE::N1, N2 = GE::N2, K2 = GE::K2, EW = GE::EW,
                  CN = GE::CN;
    double x[DG_MAXN], wq[DG_MAXN];
    dg_gauss_legendre(N, x, wq);
    double LV[DG_MAXN][DG_MAXN], LD[DG_MAXN][DG_MAXN], Lm[DG_MAXN], Lp[DG_MAXN];
    for (int a = 0; a < N; ++a) {
        for (int q = 0; q < N; ++q) {
            LV[a][q] = dg_legendre(a, x[q]);
            LD[a][q] = dg_legendre_deriv(a, x[q]);
        }
        Lm[a] = dg_legendre(a, -1.0);
        Lp[a] = dg_legendre(a, 1.0);
    }
    std::vector<double> m1((size_t)N1 * K1, 0.0), m2((size_t)N2 * K2, 0.0);
    auto B1 = [&](int r, int k) -> double & { return m1[(size_t)r * K1 + k]; };
    auto B2 = [&](int r, int k) -> double & { return m2[(size_t)r * K2 + k]; };
    for (int m = 0; m < NP; ++m) {
        const int a = m % N, b = m / N;
        for (int q = 0; q < NP; ++q) B1(q, m) = LV[a][q % N] * LV[b][q / N];
        for (int k = 0; k < N; ++k) {
            B1(NC + 0 * N + k, m) = LV[a][k] * Lm[b];   // S edge at xi_k
            B1(NC + 1 * N + k, m) = LV[a][k] * Lp[b];   // N edge
            B1(NC + 2 * N + k, m) = Lm[a] * LV[b][k];   // W edge at eta_k
            B1(NC + 3 * N + k, m) = Lp[a] * LV[b][k];   // E edge
        }
    }
    // residual mode m' = (b', a) before C_j^{-1}: volume terms of F, G, S at
    // the Gauss points, lift of the W, E, S, N edge fluxes
    for (int r = 0; r < NP; ++r) {
        const int a = r % N, bp = r / N;
        for (int q = 0; q < NP; ++q) {
            const int al = q % N, be = q / N;
            const double wl_a = wq[al] * LV[a][al], wd_a = wq[al] * LD[a][al];
            const double wl_b = wq[be] * LV[bp][be], wd_b = wq[be] * LD[bp][be];
            B2(r, q) = wd_a * wl_b;
            B2(r, NC + q) = wl_a * wd_b;
            B2(r, 2 * NC + q) = wl_a * wl_b;
        }
        const int E0 = 3 * NC;
        for (int k = 0; k < N; ++k) {
            B2(r, E0 + 0 * EW + k) = wq[k] * LV[bp][k] * Lm[a];
            B2(r, E0 + 1 * EW + k) = -wq[k] * LV[bp][k] * Lp[a];
            B2(r, E0 + 2 * EW + k) = wq[k] * LV[a][k] * Lm[bp];
            B2(r, E0 + 3 * EW + k) = -wq[k] * LV[a][k] * Lp[bp];
        }
    }
    (void)CN;
    auto canon = [split](const std::vector<double> &m, int R, int K, std::vector<uint16_t> &out) {
        const size_t sz = (size_t)R * K;
        out.assign(split ? 2 * sz : sz, 0);
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < K; ++k) {
                const size_t o = (size_t)(k / 8) * R * 8 + (size_t)r * 8 + (k % 8);
                const float v = (float)m[(size_t)r * K + k];
                out[o] = Op<OpT>::host_bits(v);
                if (split) out[sz + o] = Op<OpT>::host_bits(v - Op<OpT>::host_value(out[o]));
            }
    };
    canon(m1, N1, K1, b1);
    canon(m2, N2, K2, b2);
}

struct TabSet {
    uint4 *b1 = nullptr, *b2 = nullptr;
};
// per device, degree and operand type: the basis operands and whether the
// shared-memory opt-in is set; handles on several host threads share them,
// so every access holds g_tc_mu
std::mutex g_tc_mu;
// op: 0 BF16, 1 FP16, 2 BF16 split, 3 FP16 split
TabSet g_tabs[64][DG_MAXN][4];
unsigned long long g_attr[DG_MAXN][4];
unsigned long long g_check_attr[DG_MAXN][2];

template <int N, typename OpT>
int tables_for(int dev, int op, TabSet &out)   // caller holds g_tc_mu
{
    TabSet &t = g_tabs[dev][N - 1][op];
    if (!t.b1) {
        std::vector<uint16_t> b1, b2;
        build_tables<N, OpT>(b1, b2, op >= 2);
        uint4 *d1 = nullptr, *d2 = nullptr;
        if (cudaMalloc(&d1, b1.size() * 2) != cudaSuccess) return 1;
        if (cudaMalloc(&d2, b2.size() * 2) != cudaSuccess) {
            cudaFree(d1);
            return 1;
        }
        if (cudaMemcpy(d1, b1.data(), b1.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d2, b2.data(), b2.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d1);
            cudaFree(d2);
            return 1;
        }
        t.b1 = d1;
        t.b2 = d2;
    }
    out = t;
    return 0;
}

// Tables and the shared-memory opt-in of one (degree, operand type) on the
// current device; allocates and copies, so it must run outside stream capture.
template <int N, typename OpT, bool SPLIT>
int prepare_tc(int op, TabSet &t)
{
    using SM = TcSmem<N, SPLIT>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(g_tc_mu);
    if (tables_for<N, OpT>(dev, op, t)) return 1;
    if (!(g_attr[N - 1][op] >> dev & 1ull)) {
        if (cudaFuncSetAttribute(tc_stage_kernel<N, OpT, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SM::BYTES) != cudaSuccess)
            return 1;
        g_attr[N - 1][op] |= 1ull << dev;
    }
    return 0;
}

template <int N, typename OpT, bool SPLIT>
int launch_tc(int op, const StageArgs<float> &a, cudaStream_t s)
{
    using SM = TcSmem<N, SPLIT>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    TabSet t;
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        t = g_tabs[dev][N - 1][op];
        if (!t.b1 || !(g_attr[N - 1][op] >> dev & 1ull)) return 1;   // dg_prepare_stage_tc was not called
    }
    dim3 grid((a.nlon + TC_TW - 1) / TC_TW, (a.nlat + 3) / 4);
    if (dgk::launch_pdl(tc_stage_kernel<N, OpT, SPLIT>, grid, dim3(128 * TC_TPE), SM::BYTES, s, a,
                        (const uint4 *)t.b1, (const uint4 *)t.b2) != cudaSuccess)
        return 1;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

template <int N, typename OpT>
int check_tc(int op, const float *a, float *d, int *n1, int *k1, cudaStream_t s)
{
    using GE = TcGeo<N>;
    *n1 = GE::N1;
    *k1 = GE::K1;
    if (!a || !d) return 0;   // sizes only
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    TabSet t;
    constexpr uint32_t bytes = (GE::N1 * GE::K1 * 2 + 1023) / 1024 * 1024 + GE::K1C * CH;
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        if (tables_for<N, OpT>(dev, op, t)) return 1;
        if (!(g_check_attr[N - 1][op] >> dev & 1ull)) {
            if (cudaFuncSetAttribute(tc_gemm_check_kernel<N, OpT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bytes) != cudaSuccess)
                return 1;
            g_check_attr[N - 1][op] |= 1ull << dev;
        }
    }
    unsigned *st = nullptr;
    if (cudaMallocAsync(&st, sizeof(unsigned), s) != cudaSuccess) return 1;
    cudaMemsetAsync(st, 0, sizeof(unsigned), s);
    tc_gemm_check_kernel<N, OpT><<<1, 128, bytes, s>>>(a, d, t.b1, st);
    unsigned h = 0;
    cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
    return h ? 2 : 0;
}

}  // namespace

namespace {
// (degree, operand mode) -> the instantiation: op 0 BF16, 1 FP16, 2 BF16
// split, 3 FP16 split
template <template <int, typename, bool> class F, typename... Args>
int dispatch_tc(int n, int op, Args... args)
{
#define DG_TC_CASES(OPT, SPL)                                         \
    switch (n) {                                                      \
    case 1: return F<1, OPT, SPL>::run(op, args...);                  \
    case 2: return F<2, OPT, SPL>::run(op, args...);                  \
    case 3: return F<3, OPT, SPL>::run(op, args...);                  \
    case 4: return F<4, OPT, SPL>::run(op, args...);                  \
    case 5: return F<5, OPT, SPL>::run(op, args...);                  \
    default: return 1;                                                \
    }
    switch (op) {
    case 0: DG_TC_CASES(__nv_bfloat16, false)
    case 1: DG_TC_CASES(__half, false)
    case 2: DG_TC_CASES(__nv_bfloat16, true)
    case 3: DG_TC_CASES(__half, true)
    default: return 1;
    }
#undef DG_TC_CASES
}

template <int N, typename OpT, bool SPLIT>
struct PrepareTc {
    static int run(int op)
    {
        TabSet t;
        return prepare_tc<N, OpT, SPLIT>(op, t);
    }
};

template <int N, typename OpT, bool SPLIT>
struct LaunchTc {
    static int run(int op, const StageArgs<float> *a, cudaStream_t s) { return launch_tc<N, OpT, SPLIT>(op, *a, s); }
};
}  // namespace

int dg_prepare_stage_tc(int n, int op) { return dispatch_tc<PrepareTc>(n, op); }

int dg_launch_stage_tc(int n, int op, const StageArgs<float> &a, void *stream)
{
    return dispatch_tc<LaunchTc>(n, op, &a, static_cast<cudaStream_t>(stream));
}

int dg_tc_gemm_check(int n, int op, const float *a, float *d, int *n1, int *k1, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op == 0) {
        switch (n) {
        case 1: return check_tc<1, __nv_bfloat16>(0, a, d, n1, k1, s);
        case 2: return check_tc<2, __nv_bfloat16>(0, a, d, n1, k1, s);
        case 3: return check_tc<3, __nv_bfloat16>(0, a, d, n1, k1, s);
        case 4: return check_tc<4, __nv_bfloat16>(0, a, d, n1, k1, s);
        case 5: return check_tc<5, __nv_bfloat16>(0, a, d, n1, k1, s);
        default: return 1;
        }
    }
    switch (n) {
    case 1: return check_tc<1, __half>(1, a, d, n1, k1, s);
    case 2: return check_tc<2, __half>(1, a, d, n1, k1, s);
    case 3: return check_tc<3, __half>(1, a, d, n1, k1, s);
    case 4: return check_tc<4, __half>(1, a, d, n1, k1, s);
    case 5: return check_tc<5, __half>(1, a, d, n1, k1, s);
    default: return 1;
    }
}

int dg_launch_permute(const float *src, float *dst, int nlat, int nlon, int el, int to_lanes, void *stream)
{
    dim3 grid((el + 31) / 32, (nlon + 31) / 32, nlat), block(32, 8);
    permute_kernel<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(src, dst, nlon, el, to_lanes);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

// dg_mlp.cu -- a small per-element multilayer perceptron (n_in -> H -> H ->
// n_out, GELU, BF16 weights, FP32 accumulation) trained on the GPU by the
// kernels below (forward, backward, Adam), and its inference as a learned
// modal source term of a degree-1 solver.
//
// Layout: a batch of samples is row-major [batch][features] in FP32.
// Parameters (FP32 master copy, and a BF16 copy used by every product):
//   W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out].
// Inputs are normalised by per-feature (mean, std) and the network predicts
// targets normalised by their own (mean, std); both are part of the model.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dg_internal.h"
#include "../../include/dgswe.h"

namespace {

dg_status mfail(dg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    dg_set_last_error(buf);
    return s;
}

#define MCUDA(call)                                                                                      \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return mfail(DG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

constexpr int TB = 64;     // output tile of a GEMM block (TB x TB)
constexpr int TK = 16;     // reduction slice staged in shared memory
constexpr int MAXB = 8192; // largest batch of one call
constexpr int CHUNK = 256; // batch rows per partial weight gradient

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) for an M x N output, reduction
// length K.  The operands are addressed through accessors so that the same
// tiled kernel serves X W^T, dZ W and dZ^T X.  16 x 16 threads, 4 x 4 outputs
// each, TK-wide slices of A and B in shared memory, FP32 accumulation.
template <class AccA, class AccB>
__global__ void __launch_bounds__(256) gemm_kernel(AccA A, AccB Bm, int M, int N, int K, float *__restrict__ C,
                                                    int ldc, const float *__restrict__ bias)
{
    __shared__ float As[TK][TB + 1];
    __shared__ float Bs[TK][TB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * TB, n0 = blockIdx.x * TB;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int t = threadIdx.x; t < TK * TB; t += 256) {
            const int kk = t / TB, r = t % TB;
            As[kk][r] = (m0 + r < M && k0 + kk < K) ? A(m0 + r, k0 + kk) : 0.0f;
            Bs[kk][r] = (n0 + r < N && k0 + kk < K) ? Bm(k0 + kk, n0 + r) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Bs[kk][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) C[(size_t)m * ldc + n] = acc[i][j] + (bias ? bias[n] : 0.0f);
        }
}

// accessors
struct RowF32 {   // a row-major FP32 matrix read as (row, col)
    const float *p;
    int ld;
    __device__ float operator()(int r, int c) const { return p[(size_t)r * ld + c]; }
};
struct ColF32 {   // a row-major FP32 matrix read transposed: (r, c) -> p[c][r]
    const float *p;
    int ld;
    __device__ float operator()(int r, int c) const { return p[(size_t)c * ld + r]; }
};
struct RowBF16 {
    const __nv_bfloat16 *p;
    int ld;
    __device__ float operator()(int r, int c) const { return __bfloat162float(p[(size_t)r * ld + c]); }
};
struct ColBF16 {
    const __nv_bfloat16 *p;
    int ld;
    __device__ float operator()(int r, int c) const { return __bfloat162float(p[(size_t)c * ld + r]); }
};
struct NormIn {   // normalised network input (x - mean) / std
    const float *x;
    const float *mean, *stdv;
    int ld;
    __device__ float operator()(int r, int c) const { return (x[(size_t)r * ld + c] - mean[c]) / stdv[c]; }
};
struct NormInT {  // the same, transposed
    const float *x;
    const float *mean, *stdv;
    int ld;
    __device__ float operator()(int r, int c) const { return (x[(size_t)c * ld + r] - mean[r]) / stdv[r]; }
};

template <class AccA, class AccB>
void gemm(AccA a, AccB b, int M, int N, int K, float *C, int ldc, const float *bias, cudaStream_t s)
{
    dim3 grid((N + TB - 1) / TB, (M + TB - 1) / TB);
    gemm_kernel<<<grid, 256, 0, s>>>(a, b, M, N, K, C, ldc, bias);
}

__global__ void gelu_kernel(const float *__restrict__ z, float *__restrict__ a, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        a[t] = gelu(z[t]);
}

__global__ void gelu_back_kernel(const float *__restrict__ z, float *__restrict__ d, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] *= gelu_grad(z[t]);
}

// dY = 2 (Y - T_norm) / (batch n_out); per-block partial losses (fixed order)
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ mean,
                           const float *__restrict__ stdv, int batch, int nout, float *__restrict__ dy,
                           double *__restrict__ partial)
{
    __shared__ double red[256];
    double acc = 0.0;
    const size_t n = (size_t)batch * nout;
    const float scale = 2.0f / (float)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % nout);
        const float d = y[i] - (t[i] - mean[c]) / stdv[c];
        dy[i] = scale * d;
        acc += (double)d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Sum of the per-chunk partial weight gradients in a fixed order, and the
// bias gradient (sum of dZ over the batch, also in a fixed order).
__global__ void reduce_chunks_kernel(const float *__restrict__ part, int chunks, size_t size, float *__restrict__ out)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < size; t += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < chunks; ++c) s += part[(size_t)c * size + t];
        out[t] = s;
    }
}

__global__ void bias_grad_kernel(const float *__restrict__ dz, int batch, int n, float *__restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float s = 0.0f;
    for (int b = 0; b < batch; ++b) s += dz[(size_t)b * n + c];
    db[c] = s;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; refresh the BF16 copy.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[t];
        const float mi = b1 * m[t] + (1.0f - b1) * gi;
        const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
        m[t] = mi;
        v[t] = vi;
        const float wi = w[t] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[t] = wi;
        wb[t] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        wb[t] = __float2bfloat16_rn(w[t]);
}

unsigned grid_for(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 4096); }

}  // namespace

struct dg_mlp_ctx {
    int nin = 0, H = 0, nout = 0;
    size_t np = 0;            // parameters
    size_t oW1, ob1, oW2, ob2, oW3, ob3;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    float *norm = nullptr;    // in_mean[nin], in_std[nin], out_mean[nout], out_std[nout]
    float *rownorm = nullptr; // optional per latitude row: out_mean[nlat][nout], out_std[nlat][nout]
    int rownorm_nlat = 0;
    float *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *Y = nullptr, *dY = nullptr, *dA = nullptr,
          *dA2 = nullptr, *part = nullptr;
    double *lpart = nullptr;
    long long step = 0;
    cudaStream_t stream = nullptr;
};

namespace {

void free_mlp(dg_mlp_ctx *c)
{
    for (float *p : {c->w, c->g, c->m, c->v, c->norm, c->rownorm, c->Z1, c->A1, c->Z2, c->A2, c->Y, c->dY, c->dA, c->dA2,
                     c->part})
        cudaFree(p);
    cudaFree(c->wb);
    cudaFree(c->lpart);
    delete c;
}

// forward of a batch: Z1 = Xn W1^T + b1, A1 = gelu(Z1), Z2 = A1 W2^T + b2,
// A2 = gelu(Z2), Y = A2 W3^T + b3 (normalised output)
void forward(dg_mlp_ctx *c, const float *x, int batch, cudaStream_t s)
{
    const float *nm = c->norm, *ns = c->norm + c->nin;
    gemm(NormIn{x, nm, ns, c->nin}, ColBF16{c->wb + c->oW1, c->nin}, batch, c->H, c->nin, c->Z1, c->H, c->w + c->ob1, s);
    gelu_kernel<<<grid_for((size_t)batch * c->H), 256, 0, s>>>(c->Z1, c->A1, (size_t)batch * c->H);
    gemm(RowF32{c->A1, c->H}, ColBF16{c->wb + c->oW2, c->H}, batch, c->H, c->H, c->Z2, c->H, c->w + c->ob2, s);
    gelu_kernel<<<grid_for((size_t)batch * c->H), 256, 0, s>>>(c->Z2, c->A2, (size_t)batch * c->H);
    gemm(RowF32{c->A2, c->H}, ColBF16{c->wb + c->oW3, c->H}, batch, c->nout, c->H, c->Y, c->nout, c->w + c->ob3, s);
}

// dW = dZ^T X over the batch, in chunks of CHUNK rows reduced in a fixed order
template <class AccX>
void weight_grad(dg_mlp_ctx *c, const float *dz, int nrows_out, AccX xT, int ncols, int batch, float *dw,
                 cudaStream_t s)
{
    const int chunks = (batch + CHUNK - 1) / CHUNK;
    const size_t size = (size_t)nrows_out * ncols;
    for (int ch = 0; ch < chunks; ++ch) {
        const int r0 = ch * CHUNK, rows = std::min(CHUNK, batch - r0);
        // [nrows_out x ncols] = sum over rows: dz[row][o] * x[row][i]
        gemm(ColF32{dz + (size_t)r0 * nrows_out, nrows_out}, xT.offset(r0), nrows_out, ncols, rows,
             c->part + (size_t)ch * size, ncols, nullptr, s);
    }
    reduce_chunks_kernel<<<grid_for(size), 256, 0, s>>>(c->part, chunks, size, dw);
}

// row-offset views of the B operand of the weight gradient: (k = batch row, n = feature)
struct XRows {
    const float *p;
    int ld;
    __device__ float operator()(int r, int c) const { return p[(size_t)r * ld + c]; }
    XRows offset(int r0) const { return XRows{p + (size_t)r0 * ld, ld}; }
};
struct XRowsNorm {
    const float *p;
    const float *mean, *stdv;
    int ld;
    __device__ float operator()(int r, int c) const { return (p[(size_t)r * ld + c] - mean[c]) / stdv[c]; }
    XRowsNorm offset(int r0) const { return XRowsNorm{p + (size_t)r0 * ld, mean, stdv, ld}; }
};

// full backward of a batch after forward(); the MSE gradient is in dY
void backward(dg_mlp_ctx *c, const float *x, int batch, cudaStream_t s)
{
    float *g = c->g;
    // layer 3
    weight_grad(c, c->dY, c->nout, XRows{c->A2, c->H}, c->H, batch, g + c->oW3, s);
    bias_grad_kernel<<<(c->nout + 127) / 128, 128, 0, s>>>(c->dY, batch, c->nout, g + c->ob3);
    gemm(RowF32{c->dY, c->nout}, RowBF16{c->wb + c->oW3, c->H}, batch, c->H, c->nout, c->dA2, c->H, nullptr, s);
    gelu_back_kernel<<<grid_for((size_t)batch * c->H), 256, 0, s>>>(c->Z2, c->dA2, (size_t)batch * c->H);
    // layer 2
    weight_grad(c, c->dA2, c->H, XRows{c->A1, c->H}, c->H, batch, g + c->oW2, s);
    bias_grad_kernel<<<(c->H + 127) / 128, 128, 0, s>>>(c->dA2, batch, c->H, g + c->ob2);
    gemm(RowF32{c->dA2, c->H}, RowBF16{c->wb + c->oW2, c->H}, batch, c->H, c->H, c->dA, c->H, nullptr, s);
    gelu_back_kernel<<<grid_for((size_t)batch * c->H), 256, 0, s>>>(c->Z1, c->dA, (size_t)batch * c->H);
    // layer 1
    weight_grad(c, c->dA, c->H, XRowsNorm{x, c->norm, c->norm + c->nin, c->nin}, c->nin, batch, g + c->oW1, s);
    bias_grad_kernel<<<(c->H + 127) / 128, 128, 0, s>>>(c->dA, batch, c->H, g + c->ob1);
}

dg_status loss_and_grad(dg_mlp_ctx *c, const float *x, const float *t, int batch, double *loss)
{
    cudaStream_t s = c->stream;
    forward(c, x, batch, s);
    const int nb = 64;
    mse_kernel<<<nb, 256, 0, s>>>(c->Y, t, c->norm + 2 * c->nin, c->norm + 2 * c->nin + c->nout, batch, c->nout, c->dY,
                                  c->lpart);
    backward(c, x, batch, s);
    double part[64];
    MCUDA(cudaMemcpyAsync(part, c->lpart, sizeof part, cudaMemcpyDeviceToHost, s));
    MCUDA(cudaStreamSynchronize(s));
    double l = 0.0;
    for (double p : part) l += p;
    *loss = l / ((double)batch * c->nout);
    MCUDA(cudaPeekAtLastError());
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed, dg_mlp *out)
{
    if (!out) return mfail(DG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 1024 || n_hidden > 1024 || n_out > 1024)
        return mfail(DG_EINVAL, "layer sizes must be 1..1024");
    dg_mlp_ctx *c = new (std::nothrow) dg_mlp_ctx;
    if (!c) return mfail(DG_ENOMEM, "host allocation failed");
    c->nin = n_in;
    c->H = n_hidden;
    c->nout = n_out;
    c->oW1 = 0;
    c->ob1 = c->oW1 + (size_t)n_hidden * n_in;
    c->oW2 = c->ob1 + n_hidden;
    c->ob2 = c->oW2 + (size_t)n_hidden * n_hidden;
    c->oW3 = c->ob2 + n_hidden;
    c->ob3 = c->oW3 + (size_t)n_out * n_hidden;
    c->np = c->ob3 + n_out;
    const int chunks = (MAXB + CHUNK - 1) / CHUNK;
    const size_t maxw = std::max((size_t)n_hidden * n_hidden, std::max((size_t)n_hidden * n_in, (size_t)n_out * n_hidden));
    bool ok = cudaMalloc(&c->w, sizeof(float) * c->np) == cudaSuccess &&
              cudaMalloc(&c->g, sizeof(float) * c->np) == cudaSuccess &&
              cudaMalloc(&c->m, sizeof(float) * c->np) == cudaSuccess &&
              cudaMalloc(&c->v, sizeof(float) * c->np) == cudaSuccess &&
              cudaMalloc(&c->wb, sizeof(__nv_bfloat16) * c->np) == cudaSuccess &&
              cudaMalloc(&c->norm, sizeof(float) * 2 * (n_in + n_out)) == cudaSuccess &&
              cudaMalloc(&c->Z1, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->A1, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->Z2, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->A2, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->Y, sizeof(float) * MAXB * n_out) == cudaSuccess &&
              cudaMalloc(&c->dY, sizeof(float) * MAXB * n_out) == cudaSuccess &&
              cudaMalloc(&c->dA, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->dA2, sizeof(float) * MAXB * n_hidden) == cudaSuccess &&
              cudaMalloc(&c->part, sizeof(float) * chunks * maxw) == cudaSuccess &&
              cudaMalloc(&c->lpart, sizeof(double) * 64) == cudaSuccess;
    if (!ok) {
        free_mlp(c);
        return mfail(DG_ENOMEM, "cudaMalloc failed");
    }
    // He-uniform weights from splitmix64, zero biases, unit normalisation
    std::vector<float> w(c->np, 0.0f);
    unsigned long long st = seed;
    auto next = [&st]() {
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto fill = [&](size_t off, int rows, int cols) {
        const double a = std::sqrt(6.0 / cols);
        for (size_t t = 0; t < (size_t)rows * cols; ++t)
            w[off + t] = (float)(a * (2.0 * ((next() >> 11) * 0x1.0p-53) - 1.0));
    };
    fill(c->oW1, n_hidden, n_in);
    fill(c->oW2, n_hidden, n_hidden);
    fill(c->oW3, n_out, n_hidden);
    std::vector<float> norm(2 * (n_in + n_out), 0.0f);
    for (int i = 0; i < n_in; ++i) norm[n_in + i] = 1.0f;
    for (int i = 0; i < n_out; ++i) norm[2 * n_in + n_out + i] = 1.0f;
    c->stream = nullptr;
    if (cudaMemcpy(c->w, w.data(), sizeof(float) * c->np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->norm, norm.data(), sizeof(float) * norm.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->m, 0, sizeof(float) * c->np) != cudaSuccess ||
        cudaMemset(c->v, 0, sizeof(float) * c->np) != cudaSuccess) {
        free_mlp(c);
        return mfail(DG_ECUDA, "initial copy failed");
    }
    to_bf16_kernel<<<grid_for(c->np), 256>>>(c->w, c->wb, c->np);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_mlp(c);
        return mfail(DG_ECUDA, "initialisation failed");
    }
    *out = c;
    return DG_OK;
}

dg_status dg_mlp_destroy(dg_mlp m)
{
    if (!m) return DG_OK;
    cudaDeviceSynchronize();
    free_mlp(m);
    return DG_OK;
}

size_t dg_mlp_num_params(dg_mlp m) { return m ? m->np : 0; }

dg_status dg_mlp_get_params(dg_mlp m, float *params, size_t n)
{
    if (!m || !params || n != m->np) return mfail(DG_EINVAL, "need %zu parameters", m ? m->np : 0);
    MCUDA(cudaMemcpy(params, m->w, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return DG_OK;
}

dg_status dg_mlp_set_params(dg_mlp m, const float *params, size_t n)
{
    if (!m || !params || n != m->np) return mfail(DG_EINVAL, "need %zu parameters", m ? m->np : 0);
    MCUDA(cudaMemcpy(m->w, params, sizeof(float) * n, cudaMemcpyHostToDevice));
    to_bf16_kernel<<<grid_for(m->np), 256>>>(m->w, m->wb, m->np);
    MCUDA(cudaDeviceSynchronize());
    return DG_OK;
}

dg_status dg_mlp_set_normalization(dg_mlp m, const float *in_mean, const float *in_std, const float *out_mean,
                                   const float *out_std)
{
    if (!m || !in_mean || !in_std || !out_mean || !out_std) return mfail(DG_EINVAL, "NULL argument");
    for (int i = 0; i < m->nin; ++i)
        if (!(in_std[i] > 0)) return mfail(DG_EINVAL, "input std %d must be positive", i);
    for (int i = 0; i < m->nout; ++i)
        if (!(out_std[i] > 0)) return mfail(DG_EINVAL, "output std %d must be positive", i);
    std::vector<float> n(2 * (m->nin + m->nout));
    std::memcpy(n.data(), in_mean, sizeof(float) * m->nin);
    std::memcpy(n.data() + m->nin, in_std, sizeof(float) * m->nin);
    std::memcpy(n.data() + 2 * m->nin, out_mean, sizeof(float) * m->nout);
    std::memcpy(n.data() + 2 * m->nin + m->nout, out_std, sizeof(float) * m->nout);
    MCUDA(cudaMemcpy(m->norm, n.data(), sizeof(float) * n.size(), cudaMemcpyHostToDevice));
    return DG_OK;
}

dg_status dg_mlp_set_row_normalization(dg_mlp m, int nlat, const float *out_mean_rows, const float *out_std_rows)
{
    if (!m) return mfail(DG_EINVAL, "NULL network");
    if (nlat == 0) {
        cudaFree(m->rownorm);
        m->rownorm = nullptr;
        m->rownorm_nlat = 0;
        return DG_OK;
    }
    if (nlat < 0 || !out_mean_rows || !out_std_rows) return mfail(DG_EINVAL, "need nlat > 0 and both arrays");
    const size_t k = (size_t)nlat * m->nout;
    for (size_t i = 0; i < k; ++i)
        if (!(out_std_rows[i] > 0)) return mfail(DG_EINVAL, "row std %zu must be positive", i);
    std::vector<float> n(2 * k);
    std::memcpy(n.data(), out_mean_rows, sizeof(float) * k);
    std::memcpy(n.data() + k, out_std_rows, sizeof(float) * k);
    cudaFree(m->rownorm);
    m->rownorm = nullptr;
    MCUDA(cudaMalloc(&m->rownorm, sizeof(float) * n.size()));
    MCUDA(cudaMemcpy(m->rownorm, n.data(), sizeof(float) * n.size(), cudaMemcpyHostToDevice));
    m->rownorm_nlat = nlat;
    return DG_OK;
}

dg_status dg_mlp_forward(dg_mlp m, const float *d_x, int batch, float *d_y)
{
    if (!m || !d_x || !d_y || batch < 1 || batch > MAXB) return mfail(DG_EINVAL, "batch must be 1..%d", MAXB);
    forward(m, d_x, batch, m->stream);
    MCUDA(cudaMemcpyAsync(d_y, m->Y, sizeof(float) * batch * m->nout, cudaMemcpyDeviceToDevice, m->stream));
    MCUDA(cudaStreamSynchronize(m->stream));
    return DG_OK;
}

dg_status dg_mlp_gradients(dg_mlp m, const float *d_x, const float *d_t, int batch, float *grads, size_t n,
                           double *loss)
{
    if (!m || !d_x || !d_t || !grads || n != m->np || batch < 1 || batch > MAXB)
        return mfail(DG_EINVAL, "bad arguments (batch 1..%d, %zu gradients)", MAXB, m ? m->np : 0);
    double l = 0;
    if (dg_status s = loss_and_grad(m, d_x, d_t, batch, &l)) return s;
    MCUDA(cudaMemcpy(grads, m->g, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (loss) *loss = l;
    return DG_OK;
}

dg_status dg_mlp_train_step(dg_mlp m, const float *d_x, const float *d_t, int batch, double lr, double *loss)
{
    if (!m || !d_x || !d_t || batch < 1 || batch > MAXB || !(lr > 0))
        return mfail(DG_EINVAL, "bad arguments (batch 1..%d, lr > 0)", MAXB);
    double l = 0;
    if (dg_status s = loss_and_grad(m, d_x, d_t, batch, &l)) return s;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
    adam_kernel<<<grid_for(m->np), 256, 0, m->stream>>>(m->w, m->g, m->m, m->v, m->wb, m->np, (float)lr, b1, b2,
                                                       1e-8f, c1, c2);
    MCUDA(cudaPeekAtLastError());
    if (loss) *loss = l;
    return DG_OK;
}

}  // extern "C"

// ------------------------------------------------ inference as a source term --

namespace {

// One CTA of 128 threads (one per hidden unit) evaluates the network for
// SRC_EPC consecutive coarse elements of a degree-1 mesh: gather each
// element's and its four neighbours' modes (zeros across a pole), normalise
// them into shared memory, then every thread forms its hidden unit of the
// first and of the second layer for all the CTA's elements (BF16 weights,
// FP32 accumulation), and the outputs (element, q) are spread over the
// threads.  Every sum starts at its bias and runs over inputs / units in
// index order, exactly as an evaluation of one element at a time.  The
// state is u_stage = base + inc with h stored relative to href (mode 0 of h
// carries 2 href).
constexpr int SRC_EPC = 8;

__global__ void __launch_bounds__(128) mlp_source_kernel(
    const float *__restrict__ base, const float *__restrict__ inc, float href, int nlon, int nlat,
    const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ wf, size_t ob1, size_t oW2, size_t ob2,
    size_t oW3, size_t ob3, const float *__restrict__ norm, const float *__restrict__ rownorm,
    float *__restrict__ src)
{
    constexpr int NIN = 60, H = 128, NOUT = 12, PER = 12, EPC = SRC_EPC;
    static_assert(EPC * NOUT <= H, "one output per thread");
    __shared__ float xs[EPC][NIN];
    __shared__ float hs[EPC][H];
    const int nel = nlon * nlat;
    const int e0 = blockIdx.x * EPC;
    const int t = threadIdx.x;
    for (int v = t; v < EPC * NIN; v += H) {
        const int el = v / NIN, c = v - el * NIN;
        const int e = e0 + el;
        float xv = 0.0f;
        if (e < nel) {
            const int j = e / nlon, i = e - j * nlon;
            const int s = c / PER, q = c - s * PER;
            const int nb = s == 0   ? e
                           : s == 1 ? j * nlon + (i + nlon - 1) % nlon
                           : s == 2 ? j * nlon + (i + 1) % nlon
                           : s == 3 ? (j > 0 ? e - nlon : -1)
                                    : (j < nlat - 1 ? e + nlon : -1);
            float val = 0.0f;
            if (nb >= 0) {
                const size_t o = (size_t)nb * PER + q;
                val = base[o] + (inc ? inc[o] : 0.0f) + (q == 0 ? 2.0f * href : 0.0f);
            }
            xv = (val - norm[c]) / norm[NIN + c];
        }
        xs[el][c] = xv;
    }
    __syncthreads();
    {   // first hidden layer, unit t
        float z[EPC];
        const float b = wf[ob1 + t];
#pragma unroll
        for (int el = 0; el < EPC; ++el) z[el] = b;
        for (int c = 0; c < NIN; ++c) {
            const float w = __bfloat162float(wb[(size_t)t * NIN + c]);
#pragma unroll
            for (int el = 0; el < EPC; ++el) z[el] = fmaf(w, xs[el][c], z[el]);
        }
#pragma unroll
        for (int el = 0; el < EPC; ++el) hs[el][t] = gelu(z[el]);
    }
    __syncthreads();
    float a2[EPC];
    {   // second hidden layer, unit t
        const float b = wf[ob2 + t];
#pragma unroll
        for (int el = 0; el < EPC; ++el) a2[el] = b;
        for (int c = 0; c < H; ++c) {
            const float w = __bfloat162float(wb[oW2 + (size_t)t * H + c]);
#pragma unroll
            for (int el = 0; el < EPC; ++el) a2[el] = fmaf(w, hs[el][c], a2[el]);
        }
#pragma unroll
        for (int el = 0; el < EPC; ++el) a2[el] = gelu(a2[el]);
    }
    __syncthreads();   // every thread has read the first layer's activations
#pragma unroll
    for (int el = 0; el < EPC; ++el) hs[el][t] = a2[el];
    __syncthreads();
    if (t < EPC * NOUT) {   // output q of element el
        const int el = t / NOUT, q = t - el * NOUT;
        const int e = e0 + el;
        if (e < nel) {
            float y = wf[ob3 + q];
            for (int c = 0; c < H; ++c) y = fmaf(__bfloat162float(wb[oW3 + (size_t)q * H + c]), hs[el][c], y);
            // denormalise: per latitude row if row statistics are set, else globally
            const int j = e / nlon;
            const float om = rownorm ? rownorm[(size_t)j * NOUT + q] : norm[2 * NIN + q];
            const float os = rownorm ? rownorm[(size_t)(nlat + j) * NOUT + q] : norm[2 * NIN + NOUT + q];
            src[(size_t)e * PER + q] = y * os + om;
        }
    }
}

// Keep the total mass: remove from mode (a=0, b=0) of h the mass the learned
// source would add, sum_e sum_b w_j[b] s_e(h, a=0, b) with w_j[b] the mass
// weights C_j[0][b] of the element's row, spread over the area sum_e w_j[0].
__global__ void mlp_massfix_kernel(float *__restrict__ src, const double *__restrict__ c0, int nlon, int nlat)
{
    __shared__ double red[2][256];
    double m = 0.0, area = 0.0;
    const int nel = nlon * nlat;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const int j = e / nlon;
        m += c0[j * 2 + 0] * (double)src[(size_t)e * 12 + 0] + c0[j * 2 + 1] * (double)src[(size_t)e * 12 + 2];
        area += c0[j * 2 + 0];
    }
    red[0][threadIdx.x] = m;
    red[1][threadIdx.x] = area;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    const float shift = (float)(red[0][0] / red[1][0]);
    for (int e = threadIdx.x; e < nel; e += blockDim.x) src[(size_t)e * 12] -= shift;
}

}  // namespace

int dg_mlp_launch_source(const dg_mlp_ctx *m, const float *base, const float *inc, float href, int nlon, int nlat,
                         const double *c0, float *src, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nel = nlon * nlat;
    if (m->rownorm && m->rownorm_nlat != nlat) return 2;   // row statistics of another mesh
    mlp_source_kernel<<<(nel + SRC_EPC - 1) / SRC_EPC, 128, 0, s>>>(base, inc, href, nlon, nlat, m->wb, m->w, m->ob1, m->oW2, m->ob2,
                                                     m->oW3, m->ob3, m->norm, m->rownorm, src);
    mlp_massfix_kernel<<<1, 256, 0, s>>>(src, c0, nlon, nlat);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}

bool dg_mlp_shape_is(const dg_mlp_ctx *m, int nin, int h, int nout)
{
    return m && m->nin == nin && m->H == h && m->nout == nout;
}

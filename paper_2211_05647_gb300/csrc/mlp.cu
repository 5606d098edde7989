// mlp.cu -- training and stand-alone inference kernels of the closure network
// (17 -> 128 -> 128 -> 1, GELU), and their C ABI.
//
// Forward: the tensor-core tile of mlp.cuh (BF16 operands, FP32 accumulate),
// which can also record z1, h1, z2, h2 for the backward pass.
// Backward of L = mean_b (y_b - t_b)^2, straight through the BF16 roundings
// (the recorded h1 is the rounded value the forward used):
//   dy = 2 (y - t) / B;  dW3 = h2^T dy;  db3 = sum dy
//   dz2 = (dy W3^T) * GELU'(z2);  dW2 = h1^T dz2;  db2 = colsum dz2
//   dz1 = (dz2 W2^T) * GELU'(z1); dW1 = x^T dz1;   db1 = colsum dz1
// in FP32 on the CUDA cores (the weight-gradient reductions are split over
// row chunks and combined with atomics).  Adam (Kingma & Ba) updates the FP32
// master parameters in place.
#include <cstdio>

#include "mlp_tc.cuh"

namespace fp {

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ P, const float *__restrict__ X,
                                                     int64_t B, float *__restrict__ Y, MlpTrace tr, int use_trace)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(smem_raw);
    mlp_load_weights(s, P);
    const int64_t ntiles = (B + kMlpRows - 1) / kMlpRows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kMlpRows;
        for (int i = threadIdx.x; i < kMlpRows * kMlpK1; i += blockDim.x) {
            const int r = i / kMlpK1, k = i % kMlpK1;
            const int64_t row = row0 + r;
            s.x[r][k] = __float2bfloat16_rn((k < kMlpIn && row < B) ? X[row * kMlpIn + k] : 0.0f);
        }
        __syncthreads();
        MlpTrace t = tr;
        t.row0 = row0;
        t.nrows = B;
        mlp_tile_forward(s, use_trace ? &t : nullptr);
        __syncthreads();
        for (int r = threadIdx.x; r < kMlpRows; r += blockDim.x)
            if (row0 + r < B) Y[row0 + r] = s.y[r];
        __syncthreads();
    }
}

// per row: dy, loss, dz2 (in place over z2), partial dW3 / db3
__global__ void __launch_bounds__(128) k_mlp_out_grad(const float *__restrict__ P, const float *__restrict__ y,
                                                      const float *__restrict__ target, int64_t B,
                                                      float *__restrict__ z2, const float *__restrict__ h2,
                                                      float *__restrict__ dy_out, float *__restrict__ grad,
                                                      float *__restrict__ loss)
{
    const int n = threadIdx.x;   // hidden unit
    const float w3 = P[kOffW3 + n];
    float gw3 = 0.0f, gb3 = 0.0f, ls = 0.0f;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const float r = y[b] - target[b];
        const float dy = 2.0f * r / (float)B;
        const int64_t o = b * kMlpH + n;
        gw3 += h2[o] * dy;
        z2[o] = dy * w3 * gelu_grad_f(z2[o]);
        if (n == 0) {
            gb3 += dy;
            ls += r * r;
            dy_out[b] = dy;
        }
    }
    atomicAdd(grad + kOffW3 + n, gw3);
    if (n == 0) {
        atomicAdd(grad + kOffB3, gb3);
        atomicAdd(loss, ls / (float)B);
    }
}

// dz1 = (dz2 W2^T) * GELU'(z1), in place over z1; W2 as the forward used it (BF16-rounded)
__global__ void __launch_bounds__(128) k_mlp_hidden_grad(const float *__restrict__ P, int64_t B,
                                                         const float *__restrict__ dz2, float *__restrict__ z1)
{
    __shared__ float w2[kMlpH][kMlpH + 1];
    __shared__ float row[kMlpH];
    const int k = threadIdx.x;
    for (int i = 0; i < kMlpH; ++i)
        w2[i][k] = __bfloat162float(__float2bfloat16_rn(P[kOffW2 + i * kMlpH + k]));   // w2[k'][n] = W2[k'][n]
    __syncthreads();
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        row[k] = dz2[b * kMlpH + k];
        __syncthreads();
        float acc = 0.0f;
#pragma unroll 8
        for (int n = 0; n < kMlpH; ++n) acc += row[n] * w2[k][n];
        const int64_t o = b * kMlpH + k;
        z1[o] = acc * gelu_grad_f(z1[o]);
        __syncthreads();
    }
}

// C[m][n] += sum_b A[b][m] * D[b][n] over a chunk of rows per block (m < M <= 128,
// n < 128); A's row pitch lda.  Bias sums use M = 1 with a == nullptr (A = 1).
__global__ void __launch_bounds__(256) k_mlp_atb(const float *__restrict__ A, int lda, int M, const float *__restrict__ D,
                                                 int64_t B, int64_t chunk, float *__restrict__ C, int bf16_a)
{
    __shared__ float sa[32][129];
    __shared__ float sd[32][129];
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(b0 + chunk, B);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, each 8 m x 8 n
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int64_t bb = b0; bb < b1; bb += 32) {
        for (int i = threadIdx.x; i < 32 * 128; i += blockDim.x) {
            const int r = i / 128, c = i % 128;
            const int64_t b = bb + r;
            float av = 0.0f;
            if (b < b1 && c < M) {
                av = A ? A[b * lda + c] : 1.0f;
                if (bf16_a) av = __bfloat162float(__float2bfloat16_rn(av));
            }
            sa[r][c] = av;
            sd[r][c] = b < b1 ? D[b * kMlpH + c] : 0.0f;
        }
        __syncthreads();
        for (int r = 0; r < 32; ++r) {
            float av[8], dv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) av[i] = sa[r][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) dv[j] = sd[r][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * dv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(C + m * kMlpH + tx + 16 * j, acc[i][j]);
    }
}

__global__ void k_mlp_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t mlp_smem_bytes() { return sizeof(MlpSmem); }

// tcgen05 forward: one warpgroup per CTA, grid-stride over 128-row tiles.
// A wait that gives up sets *err and the tile's outputs to NaN.
__global__ void __launch_bounds__(128) k_mlp_forward_tc(const float *__restrict__ P, const float *__restrict__ X,
                                                        int64_t B, float *__restrict__ Y, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTcSmem &s = *reinterpret_cast<MlpTcSmem *>(smem_raw);
    mlp_tc_load_weights(s, P);
    mlp_tc_setup(s);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (B + kMlpRows - 1) / kMlpRows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row = tile * kMlpRows + threadIdx.x;
        float x[kMlpK1];
#pragma unroll
        for (int k = 0; k < kMlpK1; ++k) x[k] = (k < kMlpIn && row < B) ? X[row * kMlpIn + k] : 0.0f;
        mlp_tc_put_row(s, threadIdx.x, x);
        const float y = mlp_tc_tile(s, &phase, &ok);
        ok = __syncthreads_and(ok);           // CTA-uniform decision
        if (row < B) Y[row] = ok ? y : __int_as_float(0x7fc00000);
        if (!ok) break;
    }
    if (!ok) atomicExch(err, 1);
    mlp_tc_teardown(s);
}

// Self-test of the bounded mbarrier wait the tcgen05 kernels use: one CTA
// waits on a barrier that nothing arrives at; the wait gives up after max_iter
// tries and the kernel records that it did, instead of hanging.
__global__ void k_wait_selftest(uint32_t max_iter, int *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool done = mbar_wait(&bar, 0u, max_iter);
    if (threadIdx.x == 0) *gave_up = done ? 0 : 1;
}

// Self-test of the wall-clock-bounded wait the TMA stencil kernels use (the
// thread sleeps in the barrier between polls): gives up after limit_ns.
__global__ void k_timed_wait_selftest(uint64_t limit_ns, int *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool done = mbar_wait_timed(&bar, 0u, limit_ns);
    if (threadIdx.x == 0) *gave_up = done ? 0 : 1;
}

}  // namespace fp

using namespace fp;

namespace {

int mlp_num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

cudaError_t launch_forward(const float *P, const float *X, int64_t B, float *Y, MlpTrace tr, int use_trace,
                           cudaStream_t st)
{
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (B + kMlpRows - 1) / kMlpRows;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)mlp_num_sms() * 2);
    k_mlp_forward<<<(unsigned)std::max<int64_t>(grid, 1), 256, smem, st>>>(P, X, B, Y, tr, use_trace);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t fdtd_mlp_workspace_bytes(int64_t batch)
{
    if (batch < 1) return 0;
    return (size_t)(4 * batch * kMlpH + 2 * batch) * sizeof(float) + 256;
}

int fdtd_mlp_forward(const float *params, const float *x, int64_t batch, float *y, void *stream)
{
    if (!params || !x || !y || batch < 1) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_forward: bad argument");
    cudaError_t e = launch_forward(params, x, batch, y, MlpTrace{}, 0, (cudaStream_t)stream);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_mlp_forward_tc(const float *params, const float *x, int64_t batch, float *y, int *err, void *stream)
{
    if (!params || !x || !y || !err || batch < 1)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_forward_tc: bad argument");
    const size_t smem = sizeof(MlpTcSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    const int64_t tiles = (batch + kMlpRows - 1) / kMlpRows;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)mlp_num_sms() * 2);
    k_mlp_forward_tc<<<(unsigned)std::max<int64_t>(grid, 1), 128, smem, (cudaStream_t)stream>>>(params, x, batch, y,
                                                                                              err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_mlp_loss_grad(const float *params, const float *x, const float *target, int64_t batch, float *grad,
                       float *loss, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!params || !x || !target || !grad || !loss || !workspace || batch < 1)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_loss_grad: bad argument");
    if (workspace_bytes < fdtd_mlp_workspace_bytes(batch))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_loss_grad: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    float *ws = reinterpret_cast<float *>(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    const int64_t BH = batch * kMlpH;
    MlpTrace tr{ws, ws + BH, ws + 2 * BH, ws + 3 * BH, 0, batch};
    float *y = ws + 4 * BH, *dy = y + batch;
    cudaError_t e = cudaMemsetAsync(grad, 0, kMlpNParams * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = launch_forward(params, x, batch, y, tr, 1, st);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    const int sms = mlp_num_sms();
    const unsigned rows_grid = (unsigned)std::min<int64_t>(batch, (int64_t)sms * 8);
    k_mlp_out_grad<<<rows_grid, kMlpH, 0, st>>>(params, y, target, batch, tr.z2, tr.h2, dy, grad, loss);
    k_mlp_hidden_grad<<<(unsigned)std::min<int64_t>(batch, (int64_t)sms * 2), kMlpH, 0, st>>>(params, batch, tr.z2,
                                                                                             tr.z1);
    const int64_t chunk = 512;
    const unsigned cg = (unsigned)((batch + chunk - 1) / chunk);
    // dW2 = h1^T dz2, db2 = colsum dz2, dW1 = x^T dz1 (x rounded as the forward used it), db1 = colsum dz1
    k_mlp_atb<<<cg, 256, 0, st>>>(tr.h1, kMlpH, kMlpH, tr.z2, batch, chunk, grad + kOffW2, 0);
    k_mlp_atb<<<cg, 256, 0, st>>>(nullptr, 0, 1, tr.z2, batch, chunk, grad + kOffB2, 0);
    k_mlp_atb<<<cg, 256, 0, st>>>(x, kMlpIn, kMlpIn, tr.z1, batch, chunk, grad + kOffW1, 1);
    k_mlp_atb<<<cg, 256, 0, st>>>(nullptr, 0, 1, tr.z1, batch, chunk, grad + kOffB1, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t n, int64_t t, double lr, double beta1,
                  double beta2, double eps, void *stream)
{
    if (!params || !grad || !m || !v || n < 1 || t < 1)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_adam: bad argument");
    const float c1 = (float)(1.0 - std::pow(beta1, (double)t)), c2 = (float)(1.0 - std::pow(beta2, (double)t));
    k_mlp_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, (float)lr,
                                                                            (float)beta1, (float)beta2, (float)eps,
                                                                            c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_selftest_wait_timeout(uint32_t max_iter, int32_t *gave_up)
{
    if (!gave_up || max_iter == 0 || max_iter > (1u << 20))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_selftest_wait_timeout: gave_up NULL or max_iter not in 1..2^20");
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return fp_set_global_error(FDTD_ERR_NOMEM, "cudaMalloc failed");
    int h = -1;
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(max_iter, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    *gave_up = h;
    return FDTD_OK;
}

int fdtd_selftest_timed_wait(uint32_t limit_us, int32_t *gave_up)
{
    if (!gave_up || limit_us == 0 || limit_us > 1000000u)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_selftest_timed_wait: gave_up NULL or limit_us not in 1..10^6");
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return fp_set_global_error(FDTD_ERR_NOMEM, "cudaMalloc failed");
    int h = -1;
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        k_timed_wait_selftest<<<1, 32>>>((uint64_t)limit_us * 1000u, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    *gave_up = h;
    return FDTD_OK;
}

}  // extern "C"

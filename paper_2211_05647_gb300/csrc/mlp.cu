// mlp.cu -- stand-alone inference, Adam and the bounded-wait self-tests of the
// closure network (17 -> 128 -> 128 -> 1, GELU), and their C ABI.  The loss and
// gradient kernels are in mlp_train.cu.
//
// Forward: the tensor-core tile of mlp.cuh (BF16 operands, FP32 accumulate).
// Adam (Kingma & Ba) updates the FP32 master parameters in place.
#include <cstdio>

#include "mlp_tc.cuh"

namespace fp {

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ P, const float *__restrict__ X,
                                                     int64_t B, float *__restrict__ Y)
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
        mlp_tile_forward(s);
        __syncthreads();
        for (int r = threadIdx.x; r < kMlpRows; r += blockDim.x)
            if (row0 + r < B) Y[row0 + r] = s.y[r];
        __syncthreads();
    }
}

__global__ void k_mlp_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    adam_update(p, m, v, i, g[i], lr, b1, b2, eps, c1, c2);
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

cudaError_t launch_forward(const float *P, const float *X, int64_t B, float *Y, cudaStream_t st)
{
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (B + kMlpRows - 1) / kMlpRows;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)mlp_num_sms() * 2);
    k_mlp_forward<<<(unsigned)std::max<int64_t>(grid, 1), 256, smem, st>>>(P, X, B, Y);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int fdtd_mlp_forward(const float *params, const float *x, int64_t batch, float *y, void *stream)
{
    if (!params || !x || !y || batch < 1) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_forward: bad argument");
    cudaError_t e = launch_forward(params, x, batch, y, (cudaStream_t)stream);
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

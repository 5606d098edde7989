// closure_train.cu -- the learned closure's training pipeline on the GPU: the
// normalisation and Drude part from recorded samples, the network's inputs and
// residual targets, the initial weights and shuffled minibatches (the training
// epoch itself is in mlp_train.cu).
//
// A recorded sample is 19 floats [E^{n-15} .. E^n, n, J^{n+1/2}, J^{n-1/2}].
// The closure keeps the Crank-Nicolson update of a Drude plasma with the mean
// collision frequency nu (the Sec. 5.2 f_1x update and Jx sum with nu(v) = nu,
// for which the velocity-space solve reduces to it) and learns the rest:
//     rho  = (2 - dt nu) / (2 + dt nu),   beta = 2 dt (e^2/m) / (2 + dt nu)
//     r    = J^{n+1/2} - rho J^{n-1/2} - beta n E^n            (the kinetic correction)
//     x    = [E^{n-15..n} / E_s, n / n_c],  target = r / J_s
// with E_s the RMS of the recorded E values, n_c = eps0 m w0^2 / e^2 the
// critical density at the carrier frequency w0 and J_s the RMS of r (targets
// of unit variance).  The direct form (increment = 0) has rho = beta = 0.
// Sums are FP64 (per-thread, then per block, then over blocks).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "mlp.cuh"
#include "shuffle.cuh"

namespace fp {

constexpr int kSumBlocks = 1024;
constexpr int kSampleW = 19;

// per block: [sum of E^2 over the 16 history values, sum of r^2]
__global__ void __launch_bounds__(256) k_closure_sums(const float *__restrict__ s, int64_t n, double rho, double beta,
                                                      double *__restrict__ partials)
{
    __shared__ double red[2][8];
    double se = 0.0, sr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *q = s + i * kSampleW;
#pragma unroll
        for (int k = 0; k < 16; ++k) se += (double)q[k] * (double)q[k];
        const double r = (double)q[17] - rho * (double)q[18] - beta * (double)q[16] * (double)q[15];
        sr += r * r;
    }
    for (int o = 16; o; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = se;
        red[1][w] = sr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += red[0][q];
            b += red[1][q];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_closure_sums_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += 32) {
        a += partials[2 * q];
        b += partials[2 * q + 1];
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// x[i] = [E^{n-15..n} / E_s, n / n_c] and t[i] = r / J_s, in FP64, rounded once to FP32
__global__ void k_closure_dataset(const float *__restrict__ s, int64_t n, double inv_es, double inv_ns, double inv_js,
                                  double rho, double beta, float *__restrict__ x, float *__restrict__ t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *q = s + i * kSampleW;
    float *xo = x + i * kMlpIn;
#pragma unroll
    for (int k = 0; k < 16; ++k) xo[k] = (float)((double)q[k] * inv_es);
    xo[16] = (float)((double)q[16] * inv_ns);
    const double r = (double)q[17] - rho * (double)q[18] - beta * (double)q[16] * (double)q[15];
    t[i] = (float)(r * inv_js);
}

// He-style initial weights: W1 ~ N(0, 2/17), W2 ~ N(0, 2/128), W3 ~ N(0, 1/128),
// biases 0.  Normal draws by the Box-Muller transform of two uniforms from
// Philox4x32-7 counted by the parameter index.
__global__ void k_mlp_init(float *__restrict__ P, uint64_t seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpNParams) return;
    double sd = 0.0;
    if (i < kOffB1) sd = sqrt(2.0 / kMlpIn);
    else if (i >= kOffW2 && i < kOffB2) sd = sqrt(2.0 / kMlpH);
    else if (i >= kOffW3 && i < kOffB3) sd = sqrt(1.0 / kMlpH);
    float v = 0.0f;
    if (sd > 0.0) {
        const uint4 r = philox4x32_7(make_uint4((uint32_t)i, 0x5eed1u, 0u, 0u),
                                     make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const double u1 = ((double)r.x + 1.0) * 2.3283064365386963e-10;   // (0, 1]
        const double u2 = (double)r.y * 2.3283064365386963e-10;           // [0, 1)
        v = (float)(sd * sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2));
    }
    P[i] = v;
}

// rows first .. first + batch - 1 of the epoch's permuted order
__global__ void k_mlp_gather(const float *__restrict__ x, const float *__restrict__ t, Perm p, int64_t first,
                             int64_t batch, float *__restrict__ xb, float *__restrict__ tb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const uint64_t src = perm_index((uint64_t)(first + i), p);
    const float *xs = x + src * kMlpIn;
    float *xd = xb + i * kMlpIn;
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xd[k] = xs[k];
    tb[i] = t[src];
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace fp

using namespace fp;

extern "C" {

size_t fdtd_closure_workspace_bytes(void) { return align256((2 * kSumBlocks + 2) * sizeof(double)) + 256; }

int fdtd_closure_scales(const float *samples, int64_t n, double omega0, double dt, double nu_mean, int increment,
                        fdtd_closure_scales_t *out, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!samples || n < 1 || !out || !workspace || !(omega0 > 0) || !(dt > 0) || !(nu_mean >= 0) ||
        !std::isfinite(omega0) || !std::isfinite(dt) || !std::isfinite(nu_mean))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_closure_scales: bad argument");
    if (workspace_bytes < fdtd_closure_workspace_bytes())
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_closure_scales: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    double *ws = reinterpret_cast<double *>(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    double *res = ws + 2 * kSumBlocks;
    // Crank-Nicolson Drude update of a plasma with collision frequency nu_mean
    const double rho = increment ? (2.0 - dt * nu_mean) / (2.0 + dt * nu_mean) : 0.0;
    const double beta = increment ? 2.0 * dt * (kQe * kQe / kMe) / (2.0 + dt * nu_mean) : 0.0;
    const double n_c = kEps0 * kMe * omega0 * omega0 / (kQe * kQe);
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)std::min<int64_t>(want, kSumBlocks);
    k_closure_sums<<<blocks, 256, 0, st>>>(samples, n, rho, beta, ws);
    k_closure_sums_final<<<1, 32, 0, st>>>(ws, blocks, res);
    double h[2] = {0.0, 0.0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    const double e_s = std::sqrt(h[0] / (16.0 * (double)n));
    double j_s = std::sqrt(h[1] / (double)n);
    if (!(e_s > 0) || !std::isfinite(e_s) || !std::isfinite(j_s))
        return fp_set_global_error(FDTD_ERR_NONFINITE, "fdtd_closure_scales: E samples all zero or not finite");
    if (!(j_s > 0)) j_s = kEps0 * omega0 * e_s;   // no correction to learn: the Drude current scale
    out->e_scale = e_s;
    out->j_scale = j_s;
    out->n_scale = n_c;
    out->rho = rho;
    out->beta = beta;
    return FDTD_OK;
}

int fdtd_closure_dataset(const float *samples, int64_t n, const fdtd_closure_scales_t *sc, float *x, float *t,
                         void *stream)
{
    if (!samples || n < 1 || !sc || !x || !t || !(sc->e_scale > 0) || !(sc->j_scale > 0) || !(sc->n_scale > 0))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_closure_dataset: bad argument");
    k_closure_dataset<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        samples, n, 1.0 / sc->e_scale, 1.0 / sc->n_scale, 1.0 / sc->j_scale, sc->rho, sc->beta, x, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_mlp_init(float *params, uint64_t seed, void *stream)
{
    if (!params) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_init: params NULL");
    k_mlp_init<<<(kMlpNParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, seed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_mlp_gather(const float *x, const float *t, int64_t n, uint64_t seed, int64_t epoch, int64_t first,
                    int64_t batch, float *xb, float *tb, void *stream)
{
    if (!x || !t || !xb || !tb || n < 1 || n > (int64_t)1 << 40 || batch < 1 || first < 0 || first + batch > n ||
        epoch < 0)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_gather: bad argument (need 0 <= first, first + batch <= n)");
    k_mlp_gather<<<(unsigned)((batch + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, t, make_perm(n, seed, epoch),
                                                                                 first, batch, xb, tb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

}  // extern "C"

// mlp_train.cu -- loss and gradient of the closure network on the tensor
// cores: one CTA (8 warps, 16 rows each) per 128-row tile of the batch runs
// the forward pass and the whole backward pass of its tile on mma.sync BF16
// tiles with FP32 accumulation, and writes the tile's gradient; a second
// kernel sums the tiles' gradients in a fixed order.
//
// Loss L = mean_b (y_b - t_b)^2.  Backward, straight through the forward's BF16
// roundings (h1 and W2 as the forward's MMAs used them):
//   dy_b = 2 (y_b - t_b) / B                      (rows past the batch: 0)
//   dW3 = h2^T dy, db3 = sum dy                    (column sums, FP32)
//   dz2 = (dy w3^T) * GELU'(z2), db2 = colsum dz2
//   dW2 = h1^T dz2                                 MMA, M = K = N = 128 (K over the tile's rows)
//   dh1 = dz2 W2^T, dz1 = dh1 * GELU'(z1)          MMA per warp (its 16 rows), K = 128
//   dW1 = x^T dz1, db1 = colsum dz1                MMA, M = 32 (17 used), K over the rows
// dz2 and dz1 enter the MMAs rounded to BF16; z1, z2 and the column sums stay
// FP32.  The transposed operands (h1^T, x^T as A; dz2, dz1 as B over rows)
// are read with ldmatrix .trans from the row-major tiles.  In training the
// tile kernel takes its rows straight from the sample arrays through the
// epoch's permutation, and one kernel sums the tiles' gradients and applies
// Adam: two launches a minibatch.
#include <algorithm>
#include <cmath>

#include "mlp_tc.cuh"
#include "shuffle.cuh"

namespace fp {

constexpr int kTrainStride = kMlpNParams + 1;   // per tile: the packed gradient, then the tile's loss sum

struct MlpTrainSmem {
    __nv_bfloat16 w1t[kMlpH][kLd1];    // w1t[n][k] = W1[k][n] (k >= 17 zero): B of layer 1
    __nv_bfloat16 w2t[kMlpH][kLd2];    // w2t[n][k] = W2[k][n]: B of layer 2
    __nv_bfloat16 w2n[kMlpH][kLd2];    // w2n[k][n] = W2[k][n]: B of dh1 = dz2 W2^T
    __nv_bfloat16 x[kMlpRows][kLd1];   // the tile's inputs (cols >= 17 zero)
    __nv_bfloat16 h1[kMlpRows][kLd2];  // h1, later dz1 (after dW2 is formed)
    __nv_bfloat16 dz2[kMlpRows][kLd2];
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float colsum[3][8][kMlpH];         // per warp: dW3, db2, db1 partial column sums
    float loss[8], dyb[8];
    int64_t src[kMlpRows];             // sample index of each row (-1: past the batch)
    float b3;
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const __nv_bfloat16 *row)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(row)));
}

// Sum of the two rows a thread holds for fragment column pair (c0, c1), then
// over the 8 row groups of the warp (lanes with equal t); lanes 0..3 store.
__device__ __forceinline__ void warp_colsum(float *dst, int col, float v0, float v1, int lane)
{
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, off);
        v1 += __shfl_xor_sync(0xffffffffu, v1, off);
    }
    if (lane < 4) {
        dst[col] = v0;
        dst[col + 1] = v1;
    }
}

// One 128-row tile per CTA (256 threads) of a batch of B rows; writes ws[tile][0 .. kMlpNParams)
// = the tile's gradient contribution and ws[tile][kMlpNParams] = its sum of squared residuals / B.
// Row r of the batch is sample r of X / T, or with use_perm sample perm(first + r).
__global__ void __launch_bounds__(256, 1) k_mlp_train_tile(const float *__restrict__ P, const float *__restrict__ X,
                                                           const float *__restrict__ T, int64_t B,
                                                           float *__restrict__ ws, Perm perm, int64_t first,
                                                           int use_perm)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTrainSmem &s = *reinterpret_cast<MlpTrainSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int r0 = warp * 16;
    const int64_t row0 = (int64_t)blockIdx.x * kMlpRows;
    float *out = ws + (int64_t)blockIdx.x * kTrainStride;

    // ---- weights (BF16 operands as the forward uses them) and the input tile
    for (int i = tid; i < kMlpH * kLd1; i += blockDim.x) {
        const int n = i / kLd1, k = i % kLd1;
        s.w1t[n][k] = __float2bfloat16_rn(k < kMlpIn ? P[kOffW1 + k * kMlpH + n] : 0.0f);
    }
    for (int i = tid; i < kMlpH * kMlpH; i += blockDim.x) {
        const int k = i / kMlpH, n = i % kMlpH;
        const __nv_bfloat16 w = __float2bfloat16_rn(P[kOffW2 + i]);
        s.w2t[n][k] = w;
        s.w2n[k][n] = w;
    }
    for (int i = tid; i < kMlpH; i += blockDim.x) {
        s.b1[i] = P[kOffB1 + i];
        s.b2[i] = P[kOffB2 + i];
        s.w3[i] = P[kOffW3 + i];
    }
    if (tid == 0) s.b3 = P[kOffB3];
    if (tid < kMlpRows) {
        const int64_t row = row0 + tid;
        s.src[tid] = row < B ? (use_perm ? (int64_t)perm_index((uint64_t)(first + row), perm) : row) : -1;
    }
    __syncthreads();
    for (int i = tid; i < kMlpRows * kLd1; i += blockDim.x) {
        const int r = i / kLd1, k = i % kLd1;
        const int64_t src = s.src[r];
        s.x[r][k] = __float2bfloat16_rn((k < kMlpIn && src >= 0) ? X[src * kMlpIn + k] : 0.0f);
    }
    __syncthreads();

    // ---- forward, layer 1: h1 = gelu(z1) -> shared (BF16); z1 is formed again, bit for bit, where
    //      GELU'(z1) is needed (two MMAs per column tile), rather than kept in registers
    uint32_t xa[2][4];   // the warp's rows of x as A fragments (K = 32: two k steps)
#pragma unroll
    for (int ks = 0; ks < kMlpK1 / 16; ++ks) {
        xa[ks][0] = ld_b32(&s.x[r0 + g][ks * 16 + 2 * t]);
        xa[ks][1] = ld_b32(&s.x[r0 + g + 8][ks * 16 + 2 * t]);
        xa[ks][2] = ld_b32(&s.x[r0 + g][ks * 16 + 2 * t + 8]);
        xa[ks][3] = ld_b32(&s.x[r0 + g + 8][ks * 16 + 2 * t + 8]);
    }
    auto z1_tile = [&](int nt, float (&z)[4]) {
        z[0] = z[1] = z[2] = z[3] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < kMlpK1 / 16; ++ks)
            mma_bf16_16816(z, xa[ks], ld_b32(&s.w1t[nt * 8 + g][ks * 16 + 2 * t]),
                           ld_b32(&s.w1t[nt * 8 + g][ks * 16 + 2 * t + 8]));
        const int col = nt * 8 + 2 * t;
        z[0] += s.b1[col];
        z[1] += s.b1[col + 1];
        z[2] += s.b1[col];
        z[3] += s.b1[col + 1];
    };
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        float z[4];
        z1_tile(nt, z);
        const int col = nt * 8 + 2 * t;
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g][col]) = pack_bf16(gelu_f(z[0]), gelu_f(z[1]));
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g + 8][col]) = pack_bf16(gelu_f(z[2]), gelu_f(z[3]));
    }
    __syncwarp();

    // ---- forward, layer 2 (the warp's own rows of h1) and the output y
    float z2[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) z2[nt][0] = z2[nt][1] = z2[nt][2] = z2[nt][3] = 0.0f;
#pragma unroll 2
    for (int ks = 0; ks < kMlpH / 16; ++ks) {
        uint32_t a[4];
        a[0] = ld_b32(&s.h1[r0 + g][ks * 16 + 2 * t]);
        a[1] = ld_b32(&s.h1[r0 + g + 8][ks * 16 + 2 * t]);
        a[2] = ld_b32(&s.h1[r0 + g][ks * 16 + 2 * t + 8]);
        a[3] = ld_b32(&s.h1[r0 + g + 8][ks * 16 + 2 * t + 8]);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
            mma_bf16_16816(z2[nt], a, ld_b32(&s.w2t[nt * 8 + g][ks * 16 + 2 * t]),
                           ld_b32(&s.w2t[nt * 8 + g][ks * 16 + 2 * t + 8]));
    }
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        z2[nt][0] += s.b2[col];
        z2[nt][1] += s.b2[col + 1];
        z2[nt][2] += s.b2[col];
        z2[nt][3] += s.b2[col + 1];
        y0 += gelu_f(z2[nt][0]) * s.w3[col] + gelu_f(z2[nt][1]) * s.w3[col + 1];
        y1 += gelu_f(z2[nt][2]) * s.w3[col] + gelu_f(z2[nt][3]) * s.w3[col + 1];
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    const int64_t sa = s.src[r0 + g], sb = s.src[r0 + g + 8];
    const float e0 = sa >= 0 ? y0 + s.b3 - T[sa] : 0.0f;
    const float e1 = sb >= 0 ? y1 + s.b3 - T[sb] : 0.0f;
    const float dy0 = 2.0f * e0 / (float)B, dy1 = 2.0f * e1 / (float)B;

    // ---- dW3 = h2^T dy, dz2 = dy w3 GELU'(z2) (-> shared, BF16), db2 = colsum dz2
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        warp_colsum(s.colsum[0][warp], col, gelu_f(z2[nt][0]) * dy0 + gelu_f(z2[nt][2]) * dy1,
                    gelu_f(z2[nt][1]) * dy0 + gelu_f(z2[nt][3]) * dy1, lane);
        const float d00 = dy0 * s.w3[col] * gelu_grad_f(z2[nt][0]);
        const float d01 = dy0 * s.w3[col + 1] * gelu_grad_f(z2[nt][1]);
        const float d10 = dy1 * s.w3[col] * gelu_grad_f(z2[nt][2]);
        const float d11 = dy1 * s.w3[col + 1] * gelu_grad_f(z2[nt][3]);
        warp_colsum(s.colsum[1][warp], col, d00 + d10, d01 + d11, lane);
        *reinterpret_cast<uint32_t *>(&s.dz2[r0 + g][col]) = pack_bf16(d00, d01);
        *reinterpret_cast<uint32_t *>(&s.dz2[r0 + g + 8][col]) = pack_bf16(d10, d11);
    }
    {
        float l = e0 * e0 + e1 * e1, d = dy0 + dy1;
        if (t != 0) l = d = 0.0f;   // every lane of a quad holds the same two rows
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, off);
            d += __shfl_xor_sync(0xffffffffu, d, off);
        }
        if (lane == 0) {
            s.loss[warp] = l / (float)B;
            s.dyb[warp] = d;
        }
    }
    __syncthreads();

    // ---- dW2[k][n] = sum_b h1[b][k] dz2[b][n]: warp w forms rows k in [16 w, 16 w + 16)
    {
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
        const int q = lane >> 3, rr = lane & 7;
#pragma unroll 2
        for (int ks = 0; ks < kMlpRows / 16; ++ks) {
            const int b0 = ks * 16;
            uint32_t a[4];   // A(k, b) = h1[b][k]: blocks (b lo/hi) x (k lo/hi) in the a0..a3 order
            ldsm_x4_trans(a, &s.h1[b0 + ((q >> 1) << 3) + rr][r0 + ((q & 1) << 3)]);
#pragma unroll
            for (int nt = 0; nt < 16; nt += 2) {
                uint32_t bq[4];   // B(b, n) = dz2[b][n]: (nt, b lo), (nt, b hi), (nt + 1, b lo), (nt + 1, b hi)
                ldsm_x4_trans(bq, &s.dz2[b0 + ((q & 1) << 3) + rr][(nt + (q >> 1)) * 8]);
                mma_bf16_16816(acc[nt], a, bq[0], bq[1]);
                mma_bf16_16816(acc[nt + 1], a, bq[2], bq[3]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int col = nt * 8 + 2 * t;
            float *o = out + kOffW2 + (r0 + g) * kMlpH + col;
            *reinterpret_cast<float2 *>(o) = make_float2(acc[nt][0], acc[nt][1]);
            *reinterpret_cast<float2 *>(o + 8 * kMlpH) = make_float2(acc[nt][2], acc[nt][3]);
        }
    }

    // ---- dh1 = dz2 W2^T for the warp's own rows, dz1 = dh1 GELU'(z1)
    float dh[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) dh[nt][0] = dh[nt][1] = dh[nt][2] = dh[nt][3] = 0.0f;
#pragma unroll 2
    for (int ks = 0; ks < kMlpH / 16; ++ks) {
        uint32_t a[4];
        a[0] = ld_b32(&s.dz2[r0 + g][ks * 16 + 2 * t]);
        a[1] = ld_b32(&s.dz2[r0 + g + 8][ks * 16 + 2 * t]);
        a[2] = ld_b32(&s.dz2[r0 + g][ks * 16 + 2 * t + 8]);
        a[3] = ld_b32(&s.dz2[r0 + g + 8][ks * 16 + 2 * t + 8]);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
            mma_bf16_16816(dh[nt], a, ld_b32(&s.w2n[nt * 8 + g][ks * 16 + 2 * t]),
                           ld_b32(&s.w2n[nt * 8 + g][ks * 16 + 2 * t + 8]));
    }
    __syncthreads();   // every warp has read h1 (dW2) before dz1 takes its place
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        float z[4];
        z1_tile(nt, z);
        const float d00 = dh[nt][0] * gelu_grad_f(z[0]), d01 = dh[nt][1] * gelu_grad_f(z[1]);
        const float d10 = dh[nt][2] * gelu_grad_f(z[2]), d11 = dh[nt][3] * gelu_grad_f(z[3]);
        warp_colsum(s.colsum[2][warp], col, d00 + d10, d01 + d11, lane);
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g][col]) = pack_bf16(d00, d01);
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g + 8][col]) = pack_bf16(d10, d11);
    }
    __syncthreads();

    // ---- dW1[k][n] = sum_b x[b][k] dz1[b][n] (k < 17): warp w forms the 16-row block
    //      k in [16 (w & 1), +16) for the n tiles [4 (w >> 1), +4)
    {
        const int mt = warp & 1, n0 = (warp >> 1) * 4;
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
        const int q = lane >> 3, rr = lane & 7;
#pragma unroll 2
        for (int ks = 0; ks < kMlpRows / 16; ++ks) {
            const int b0 = ks * 16;
            uint32_t a[4];
            ldsm_x4_trans(a, &s.x[b0 + ((q >> 1) << 3) + rr][mt * 16 + ((q & 1) << 3)]);
#pragma unroll
            for (int j = 0; j < 4; j += 2) {
                uint32_t bq[4];
                ldsm_x4_trans(bq, &s.h1[b0 + ((q & 1) << 3) + rr][(n0 + j + (q >> 1)) * 8]);
                mma_bf16_16816(acc[j], a, bq[0], bq[1]);
                mma_bf16_16816(acc[j + 1], a, bq[2], bq[3]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = (n0 + j) * 8 + 2 * t;
            const int k_lo = mt * 16 + g, k_hi = k_lo + 8;
            if (k_lo < kMlpIn)
                *reinterpret_cast<float2 *>(out + kOffW1 + k_lo * kMlpH + col) = make_float2(acc[j][0], acc[j][1]);
            if (k_hi < kMlpIn)
                *reinterpret_cast<float2 *>(out + kOffW1 + k_hi * kMlpH + col) = make_float2(acc[j][2], acc[j][3]);
        }
    }

    // ---- column sums over the warps: dW3, db2, db1; db3 and the loss
    if (tid < kMlpH) {
        float a = 0.0f, b = 0.0f, c = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            a += s.colsum[0][w][tid];
            b += s.colsum[1][w][tid];
            c += s.colsum[2][w][tid];
        }
        out[kOffW3 + tid] = a;
        out[kOffB2 + tid] = b;
        out[kOffB1 + tid] = c;
    }
    if (tid == 0) {
        float l = 0.0f, d = 0.0f;
        for (int w = 0; w < 8; ++w) {
            l += s.loss[w];
            d += s.dyb[w];
        }
        out[kOffB3] = d;
        out[kMlpNParams] = l;
    }
}

// grad[i] = sum over tiles (in tile order) of ws[tile][i]; loss = sum of ws[tile][kMlpNParams]
__global__ void k_mlp_train_reduce(const float *__restrict__ ws, int ntiles, float *__restrict__ grad,
                                   float *__restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kMlpNParams) return;
    float a = 0.0f;
    for (int q = 0; q < ntiles; ++q) a += ws[(int64_t)q * kTrainStride + i];
    if (i < kMlpNParams) grad[i] = a;
    else *loss = a;
}

// the same sum per parameter followed by its Adam step (step count t: c1, c2), and the minibatch's loss
// added to *loss_acc times loss_scale
__global__ void k_mlp_train_reduce_adam(const float *__restrict__ ws, int ntiles, float *__restrict__ P,
                                        float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                                        float eps, float c1, float c2, double *__restrict__ loss_acc,
                                        double loss_scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kMlpNParams) return;
    float a = 0.0f;
    for (int q = 0; q < ntiles; ++q) a += ws[(int64_t)q * kTrainStride + i];
    if (i < kMlpNParams) adam_update(P, m, v, i, a, lr, b1, b2, eps, c1, c2);
    else *loss_acc += (double)a * loss_scale;
}

size_t train_smem_bytes() { return sizeof(MlpTrainSmem); }

cudaError_t launch_train_tile(cudaStream_t st, const float *P, const float *X, const float *T, int64_t B, float *ws,
                              const Perm *perm, int64_t first)
{
    const size_t smem = sizeof(MlpTrainSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (B + kMlpRows - 1) / kMlpRows;
    k_mlp_train_tile<<<(unsigned)tiles, 256, smem, st>>>(P, X, T, B, ws, perm ? *perm : Perm{}, first, perm ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace fp

using namespace fp;

extern "C" {

size_t fdtd_mlp_workspace_bytes(int64_t batch)
{
    if (batch < 1) return 0;
    const int64_t tiles = (batch + kMlpRows - 1) / kMlpRows;
    return (size_t)tiles * kTrainStride * sizeof(float) + 256;
}

int fdtd_mlp_loss_grad(const float *params, const float *x, const float *target, int64_t batch, float *grad,
                       float *loss, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!params || !x || !target || !grad || !loss || !workspace || batch < 1)
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_loss_grad: bad argument");
    if (workspace_bytes < fdtd_mlp_workspace_bytes(batch))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_loss_grad: workspace too small");
    const int64_t tiles = (batch + kMlpRows - 1) / kMlpRows;
    if (tiles > (1 << 24)) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_loss_grad: batch too large");
    cudaStream_t st = (cudaStream_t)stream;
    float *ws = reinterpret_cast<float *>(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    cudaError_t e = launch_train_tile(st, params, x, target, batch, ws, nullptr, 0);
    if (e == cudaSuccess) {
        k_mlp_train_reduce<<<(kMlpNParams + 1 + 255) / 256, 256, 0, st>>>(ws, (int)tiles, grad, loss);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

size_t fdtd_mlp_train_workspace_bytes(int64_t batch) { return fdtd_mlp_workspace_bytes(batch); }

int fdtd_mlp_train_epoch(float *params, float *grad, float *m, float *v, const float *x, const float *t, int64_t n,
                         int64_t batch, uint64_t seed, int64_t epoch, int64_t iter0, int64_t total_iters, double lr,
                         double beta1, double beta2, double eps, double *loss_mean, void *workspace,
                         size_t workspace_bytes, void *stream)
{
    (void)grad;   // the fused reduction applies each tile-summed gradient directly
    if (!params || !m || !v || !x || !t || !loss_mean || !workspace || batch < 1 || n < batch ||
        n > (int64_t)1 << 40 || epoch < 0 || iter0 < 0 || total_iters < 1 || !(lr > 0) || !std::isfinite(lr))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_train_epoch: bad argument (need n >= batch >= 1)");
    if (workspace_bytes < fdtd_mlp_train_workspace_bytes(batch))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_train_epoch: workspace too small");
    const int64_t tiles = (batch + kMlpRows - 1) / kMlpRows;
    if (tiles > (1 << 24)) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_mlp_train_epoch: batch too large");
    cudaStream_t st = (cudaStream_t)stream;
    float *ws = reinterpret_cast<float *>(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    cudaError_t e = cudaMemsetAsync(loss_mean, 0, sizeof(double), st);
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    const int64_t nb = n / batch;   // the ragged tail of the permuted order is left out this epoch
    const Perm p = make_perm(n, seed, epoch);
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
        e = launch_train_tile(st, params, x, t, batch, ws, &p, b * batch);
        if (e != cudaSuccess) break;
        const int64_t it = iter0 + b;
        const double lr_t = lr * 0.5 * (1.0 + std::cos(kPi * (double)std::min(it, total_iters) / (double)total_iters));
        const double c1 = 1.0 - std::pow(beta1, (double)(it + 1)), c2 = 1.0 - std::pow(beta2, (double)(it + 1));
        k_mlp_train_reduce_adam<<<(kMlpNParams + 1 + 255) / 256, 256, 0, st>>>(
            ws, (int)tiles, params, m, v, (float)lr_t, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2,
            loss_mean, 1.0 / (double)nb);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

}  // extern "C"

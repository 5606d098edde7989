// mlp.cuh -- the closure network's forward tile on the tensor cores.
//
// Network: x[17] -> 128 -> 128 -> 1, GELU (tanh form, see gelu_f below) after both hidden
// layers.  Parameters are FP32 "master" values packed as
//   W1[17][128] b1[128] W2[128][128] b2[128] W3[128] b3[1]   (18945 floats);
// the tile converts the weights to BF16 once per CTA and keeps them in shared
// memory, transposed so every B fragment is one 32-bit shared load.
// A tile is 128 rows (samples / plasma cells), 8 warps x 16 rows.  The two
// dense layers are mma.sync m16n8k16 BF16 x BF16 -> FP32; the output layer is
// a per-row dot product reduced across the quad of lanes holding a row.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace fp {

constexpr int kMlpIn = 17, kMlpK1 = 32, kMlpH = 128, kMlpRows = 128;
constexpr int kMlpNParams = kMlpIn * kMlpH + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;   // 18945
constexpr int kLd1 = kMlpK1 + 8;    // padded row pitch (bf16) of 32-wide tiles: conflict-free fragments
constexpr int kLd2 = kMlpH + 8;     // padded row pitch of 128-wide tiles
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpIn * kMlpH, kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH, kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpH;

struct MlpSmem {
    __nv_bfloat16 w1t[kMlpH][kLd1];   // w1t[n][k] = W1[k][n], k >= 17 zero
    __nv_bfloat16 w2t[kMlpH][kLd2];   // w2t[n][k] = W2[k][n]
    __nv_bfloat16 x[kMlpRows][kLd1];  // input tile (bf16), columns >= 17 zero
    __nv_bfloat16 h1[kMlpRows][kLd2]; // first hidden activations (bf16)
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float y[kMlpRows];
    float b3;
};

// Activation: the tanh form of GELU (Hendrycks & Gimpel 2016),
//   gelu(z) = 0.5 z (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3),
// with the hardware tanh (tanh.approx.f32, about 2^-11 relative): a handful of
// FMA-pipe operations and one special-function operation per activation, well
// inside the BF16 rounding the activations get next.
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2/pi)
constexpr float kGeluA = 0.044715f;
__device__ __forceinline__ float gelu_f(float z)
{
    const float t = tanh_fast(kGeluC * z * fmaf(kGeluA, z * z, 1.0f));
    const float hz = 0.5f * z;
    return fmaf(hz, t, hz);
}
// 2 gelu(z) = z + z tanh(u), u = z (sqrt(2/pi) + sqrt(2/pi) 0.044715 z^2): four FP32 operations and one tanh
constexpr float kGeluCA = kGeluC * kGeluA;
__device__ __forceinline__ float gelu2_f(float z)
{
    const float t = tanh_fast(z * fmaf(kGeluCA, z * z, kGeluC));
    return fmaf(z, t, z);
}
// d gelu / dz = 0.5 (1 + t) + 0.5 z (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2)
__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float t = tanh_fast(kGeluC * z * fmaf(kGeluA, z * z, 1.0f));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluC * fmaf(3.0f * kGeluA, z * z, 1.0f);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// One Adam step (Kingma & Ba) of parameter i: first / second moments m, v, bias
// corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__device__ __forceinline__ void adam_update(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                            int64_t i, float gi, float lr, float b1, float b2, float eps, float c1,
                                            float c2)
{
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// all threads of the CTA: FP32 packed parameters -> BF16 transposed shared tiles
__device__ __forceinline__ void mlp_load_weights(MlpSmem &s, const float *__restrict__ P)
{
    for (int i = threadIdx.x; i < kMlpH * kLd1; i += blockDim.x) {
        const int n = i / kLd1, k = i % kLd1;
        s.w1t[n][k] = __float2bfloat16_rn(k < kMlpIn ? P[kOffW1 + k * kMlpH + n] : 0.0f);
    }
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x) {
        const int k = i / kMlpH, n = i % kMlpH;   // coalesced read of W2[k][n]
        s.w2t[n][k] = __float2bfloat16_rn(P[kOffW2 + i]);
    }
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        s.b1[i] = P[kOffB1 + i];
        s.b2[i] = P[kOffB2 + i];
        s.w3[i] = P[kOffW3 + i];
    }
    if (threadIdx.x == 0) s.b3 = P[kOffB3];
}

// Forward pass of the 128-row tile in s.x; y[row] lands in s.y.  Requires a
// __syncthreads() between writing s.x and the call and before reading s.y.
__device__ __forceinline__ void mlp_tile_forward(MlpSmem &s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int r0 = warp * 16;
    float acc[16][4];
    // ---- layer 1: [16 x 32] x [32 x 128]
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < kMlpK1 / 16; ++ks) {
        uint32_t a[4];
        a[0] = ld_b32(&s.x[r0 + g][ks * 16 + 2 * t]);
        a[1] = ld_b32(&s.x[r0 + g + 8][ks * 16 + 2 * t]);
        a[2] = ld_b32(&s.x[r0 + g][ks * 16 + 2 * t + 8]);
        a[3] = ld_b32(&s.x[r0 + g + 8][ks * 16 + 2 * t + 8]);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
            mma_bf16_16816(acc[nt], a, ld_b32(&s.w1t[nt * 8 + g][ks * 16 + 2 * t]),
                           ld_b32(&s.w1t[nt * 8 + g][ks * 16 + 2 * t + 8]));
    }
    // bias + GELU -> h1 (bf16, shared)
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float z00 = acc[nt][0] + s.b1[col], z01 = acc[nt][1] + s.b1[col + 1];
        const float z10 = acc[nt][2] + s.b1[col], z11 = acc[nt][3] + s.b1[col + 1];
        const uint32_t p0 = pack_bf16(gelu_f(z00), gelu_f(z01)), p1 = pack_bf16(gelu_f(z10), gelu_f(z11));
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g][col]) = p0;
        *reinterpret_cast<uint32_t *>(&s.h1[r0 + g + 8][col]) = p1;
    }
    __syncwarp();
    // ---- layer 2: [16 x 128] x [128 x 128]; a warp reads only its own h1 rows
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll 2
    for (int ks = 0; ks < kMlpH / 16; ++ks) {
        uint32_t a[4];
        a[0] = ld_b32(&s.h1[r0 + g][ks * 16 + 2 * t]);
        a[1] = ld_b32(&s.h1[r0 + g + 8][ks * 16 + 2 * t]);
        a[2] = ld_b32(&s.h1[r0 + g][ks * 16 + 2 * t + 8]);
        a[3] = ld_b32(&s.h1[r0 + g + 8][ks * 16 + 2 * t + 8]);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
            mma_bf16_16816(acc[nt], a, ld_b32(&s.w2t[nt * 8 + g][ks * 16 + 2 * t]),
                           ld_b32(&s.w2t[nt * 8 + g][ks * 16 + 2 * t + 8]));
    }
    // bias + GELU, then the output layer: y = h2 . W3 + b3
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float z00 = acc[nt][0] + s.b2[col], z01 = acc[nt][1] + s.b2[col + 1];
        const float z10 = acc[nt][2] + s.b2[col], z11 = acc[nt][3] + s.b2[col + 1];
        const float h00 = gelu_f(z00), h01 = gelu_f(z01), h10 = gelu_f(z10), h11 = gelu_f(z11);
        y0 += h00 * s.w3[col] + h01 * s.w3[col + 1];
        y1 += h10 * s.w3[col] + h11 * s.w3[col + 1];
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t == 0) {
        s.y[r0 + g] = y0 + s.b3;
        s.y[r0 + g + 8] = y1 + s.b3;
    }
}

}  // namespace fp

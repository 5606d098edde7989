// mlp_tc.cuh -- the closure network's forward tile on the 5th-generation
// tensor cores (tcgen05): operands in shared memory, the FP32 accumulator in
// tensor memory (TMEM).
//
// One CTA = one warpgroup (128 threads); a tile is 128 rows.  Per layer one
// elected thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
// M = 128, N = 128, K = 16 per instruction) and commits to an mbarrier; every
// thread then reads its own row of the accumulator with tcgen05.ld
// (32x32b shape: warp w owns TMEM lanes 32w..32w+31 = rows), applies bias +
// GELU and writes the next layer's A operand back to shared memory.  The
// output layer is a per-row dot product (each thread holds a whole row).
//
// Shared-memory operand layout: "no swizzle, K-major" core matrices of
// 8 rows x 16 bytes (8 bf16), stored 128 contiguous bytes each; the core
// matrix of row group g and K chunk c sits at (g * (K/8) + c) * 128 bytes, so
// the descriptor's leading byte offset (next core matrix along K) is 128 and
// its stride byte offset (next 8-row group) is K/8 * 128.
#pragma once

#include "async.cuh"
#include "mlp.cuh"

namespace fp {

struct MlpTcSmem {
    __align__(128) __nv_bfloat16 w1[kMlpH * kMlpK1];   // B of layer 1: N=128 x K=32, core layout
    __align__(128) __nv_bfloat16 w2[kMlpH * kMlpH];    // B of layer 2: N=128 x K=128
    __align__(128) __nv_bfloat16 x[kMlpRows * kMlpK1]; // A of layer 1: M=128 x K=32
    __align__(128) __nv_bfloat16 a2[kMlpRows * kMlpH]; // A of layer 2: M=128 x K=128
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float b3;
    __align__(8) uint64_t mbar;
    uint32_t tmem;
};

// byte offset of element (row, k) in a core-matrix K-major tile with K columns
__device__ __forceinline__ uint32_t core_off(int row, int k, int K)
{
    return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores; no swizzle
    return d;
}

// kind::f16 instruction descriptor: D f32, A = B = bf16, both K-major, N = 128, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 columns of the thread's TMEM lane without waiting for them; tc_wait_ld16 waits for every load the
// thread has in flight and ties these registers to the wait, so no use of them moves above it.  With two
// register sets a warp reads the next 16 columns while it works on the last ones.
__device__ __forceinline__ void tc_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

// weights (FP32 packed) -> BF16 core-matrix tiles; biases -> shared
__device__ __forceinline__ void mlp_tc_load_weights(MlpTcSmem &s, const float *__restrict__ P)
{
    unsigned char *w1 = reinterpret_cast<unsigned char *>(s.w1), *w2 = reinterpret_cast<unsigned char *>(s.w2);
    for (int i = threadIdx.x; i < kMlpH * kMlpK1; i += blockDim.x) {
        const int n = i / kMlpK1, k = i % kMlpK1;
        *reinterpret_cast<__nv_bfloat16 *>(w1 + core_off(n, k, kMlpK1)) =
            __float2bfloat16_rn(k < kMlpIn ? P[kOffW1 + k * kMlpH + n] : 0.0f);
    }
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x) {
        const int k = i / kMlpH, n = i % kMlpH;   // W2[k][n] read coalesced; B(n, k) = W2[k][n]
        *reinterpret_cast<__nv_bfloat16 *>(w2 + core_off(n, k, kMlpH)) = __float2bfloat16_rn(P[kOffW2 + i]);
    }
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        s.b1[i] = P[kOffB1 + i];
        s.b2[i] = P[kOffB2 + i];
        s.w3[i] = P[kOffW3 + i];
    }
    if (threadIdx.x == 0) s.b3 = P[kOffB3];
}

// One-time set-up of a CTA (128 threads): mbarrier and 128 TMEM columns.
__device__ __forceinline__ void mlp_tc_setup(MlpTcSmem &s)
{
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s.tmem)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) mbar_init(&s.mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void mlp_tc_teardown(MlpTcSmem &s)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(128u) : "memory");
}

// Thread r writes row r of the layer-1 input (17 values, zero padded to 32).
__device__ __forceinline__ void mlp_tc_put_row(MlpTcSmem &s, int r, const float *x)
{
    unsigned char *xb = reinterpret_cast<unsigned char *>(s.x);
#pragma unroll
    for (int c = 0; c < kMlpK1 / 8; ++c) {
        uint4 v;
        v.x = pack_bf16(x[8 * c + 0], x[8 * c + 1]);
        v.y = pack_bf16(x[8 * c + 2], x[8 * c + 3]);
        v.z = pack_bf16(x[8 * c + 4], x[8 * c + 5]);
        v.w = pack_bf16(x[8 * c + 6], x[8 * c + 7]);
        *reinterpret_cast<uint4 *>(xb + core_off(r, 8 * c, kMlpK1)) = v;
    }
}

// Forward of the tile whose input rows are in s.x; returns row threadIdx.x's
// output.  *phase tracks the mbarrier parity; *ok is cleared if a wait gave up.
__device__ __forceinline__ float mlp_tc_tile(MlpTcSmem &s, uint32_t *phase, bool *ok)
{
    const int r = threadIdx.x, warp = r >> 5;
    const uint32_t tmem = s.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t kWait = 1u << 22;
    // ---- layer 1
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (r == 0) {
        const uint32_t xa = smem_addr(s.x), wa = smem_addr(s.w1);
#pragma unroll
        for (int kk = 0; kk < kMlpK1 / 16; ++kk)
            tc_mma(tmem, tc_desc(xa + kk * 256, 128, (kMlpK1 / 8) * 128), tc_desc(wa + kk * 256, 128, (kMlpK1 / 8) * 128),
                   kTcIdesc, kk > 0);
        tc_commit(&s.mbar);
    }
    if (!mbar_wait(&s.mbar, *phase, kWait)) *ok = false;
    *phase ^= 1u;
    tc_fence_after();
    unsigned char *a2 = reinterpret_cast<unsigned char *>(s.a2);
#pragma unroll
    for (int c = 0; c < kMlpH / 32; ++c) {
        float v[32];
        tc_ld32(tmem + lane_base + c * 32, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k0 = c * 32 + q * 8;
            uint4 pk;
            pk.x = pack_bf16(gelu_f(v[q * 8 + 0] + s.b1[k0 + 0]), gelu_f(v[q * 8 + 1] + s.b1[k0 + 1]));
            pk.y = pack_bf16(gelu_f(v[q * 8 + 2] + s.b1[k0 + 2]), gelu_f(v[q * 8 + 3] + s.b1[k0 + 3]));
            pk.z = pack_bf16(gelu_f(v[q * 8 + 4] + s.b1[k0 + 4]), gelu_f(v[q * 8 + 5] + s.b1[k0 + 5]));
            pk.w = pack_bf16(gelu_f(v[q * 8 + 6] + s.b1[k0 + 6]), gelu_f(v[q * 8 + 7] + s.b1[k0 + 7]));
            *reinterpret_cast<uint4 *>(a2 + core_off(r, k0, kMlpH)) = pk;
        }
    }
    // ---- layer 2
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (r == 0) {
        const uint32_t aa = smem_addr(s.a2), wa = smem_addr(s.w2);
#pragma unroll
        for (int kk = 0; kk < kMlpH / 16; ++kk)
            tc_mma(tmem, tc_desc(aa + kk * 256, 128, (kMlpH / 8) * 128), tc_desc(wa + kk * 256, 128, (kMlpH / 8) * 128),
                   kTcIdesc, kk > 0);
        tc_commit(&s.mbar);
    }
    if (!mbar_wait(&s.mbar, *phase, kWait)) *ok = false;
    *phase ^= 1u;
    tc_fence_after();
    float y = s.b3;
#pragma unroll
    for (int c = 0; c < kMlpH / 32; ++c) {
        float v[32];
        tc_ld32(tmem + lane_base + c * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) y += gelu_f(v[i] + s.b2[c * 32 + i]) * s.w3[c * 32 + i];
    }
    tc_fence_before();   // TMEM reads done before the next tile's MMA overwrites the accumulator
    return y;
}

// ------------------------------------------------------------------------
// Four independent warpgroup pipelines per CTA (512 threads), one copy of the
// weights.  Warpgroup g owns TMEM columns [128 g, 128 g + 128), its own input
// and hidden tiles and mbarrier, and synchronises on named barrier 1 + g, so
// while one warpgroup waits for its MMAs the others run their epilogues.

constexpr int kTcGroups = 4;

struct MlpTcWeights {
    __align__(128) __nv_bfloat16 w1[kMlpH * kMlpK1];   // K rows 17 / 18: b1 as a BF16 high and low part
    __align__(128) __nv_bfloat16 w2[kMlpH * kMlpH];
    __align__(16) float b2[kMlpH];
    __align__(16) float w3[kMlpH];   // half scale (see mlp_tc4_load_weights)
    float b3;
    uint32_t tmem;
};

struct MlpTcGroup {
    __align__(128) __nv_bfloat16 x[kMlpRows * kMlpK1];
    __align__(128) __nv_bfloat16 a2[kMlpRows * kMlpH];
    __align__(8) uint64_t mbar;
    int flag;
};

struct MlpTcSmem4 {
    MlpTcWeights w;
    MlpTcGroup g[kTcGroups];
};

__device__ __forceinline__ void wg_bar(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

// gelu2_f on two activations, lane by lane the same roundings: z z, the polynomial, u = z p, tanh, z t + z
__device__ __forceinline__ float2 gelu2_f2(uint64_t z)
{
    const uint64_t u = f2_mul(z, f2_fma(f2(kGeluCA, kGeluCA), f2_mul(z, z), f2(kGeluC, kGeluC)));
    const float2 uu = f2_split(u);
    return f2_split(f2_fma(z, f2(tanh_fast(uu.x), tanh_fast(uu.y)), z));
}

// The epilogues form 2 gelu(z) = z + z tanh(u) (one multiply fewer than gelu); W2 and w3 are stored at
// half scale to compensate.  Both scalings are by a power of two, so the BF16 operands and every product
// equal those of the unscaled form exactly.
// ring >= 0: the first 16 inputs arrive in history-ring slot order (slot j holds E^{n-15+k} with
// k = (j - ring - 1) mod 16, the oldest first in the network's order), so W1's rows are stored in that
// order: the same products, the ring never rotated per cell.
// Layer 1's bias rides in the MMA: input columns 17 and 18 are 1 (mlp_tc4_put_row_ring) and W1's rows 17
// and 18 hold b1 split into a BF16 high part and the BF16 rounding of the rest, so the FP32 accumulator
// adds b1 to within 2^-17 of it and the epilogue adds no bias.  (Layer 2's K has no spare columns; a
// 16-column extension for b2 cost more than the bias adds it saves.)
__device__ __forceinline__ void mlp_tc4_load_weights(MlpTcWeights &s, const float *__restrict__ P, int ring = -1)
{
    unsigned char *w1 = reinterpret_cast<unsigned char *>(s.w1), *w2 = reinterpret_cast<unsigned char *>(s.w2);
    for (int i = threadIdx.x; i < kMlpH * kMlpK1; i += blockDim.x) {
        const int n = i / kMlpK1, k = i % kMlpK1;
        const int kk = (ring >= 0 && k < 16) ? ((k - ring - 1) & 15) : k;
        __nv_bfloat16 v = __float2bfloat16_rn(k < kMlpIn ? P[kOffW1 + kk * kMlpH + n] : 0.0f);
        if (k == kMlpIn || k == kMlpIn + 1) {
            const float b = P[kOffB1 + n];
            const __nv_bfloat16 hi = __float2bfloat16_rn(b);
            v = k == kMlpIn ? hi : __float2bfloat16_rn(b - __bfloat162float(hi));
        }
        *reinterpret_cast<__nv_bfloat16 *>(w1 + core_off(n, k, kMlpK1)) = v;
    }
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x) {
        const int k = i / kMlpH, n = i % kMlpH;
        *reinterpret_cast<__nv_bfloat16 *>(w2 + core_off(n, k, kMlpH)) = __float2bfloat16_rn(0.5f * P[kOffW2 + i]);
    }
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        s.b2[i] = P[kOffB2 + i];
        s.w3[i] = 0.5f * P[kOffW3 + i];
    }
    if (threadIdx.x == 0) s.b3 = P[kOffB3];
}

// all 512 threads: TMEM (4 x 128 columns), one mbarrier per warpgroup
__device__ __forceinline__ void mlp_tc4_setup(MlpTcSmem4 &s)
{
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s.w.tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x < kTcGroups) {
        mbar_init(&s.g[threadIdx.x].mbar, 1);
        s.g[threadIdx.x].flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void mlp_tc4_teardown(MlpTcSmem4 &s)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.w.tmem), "r"(512u) : "memory");
}

// Thread r writes row r of the layer-1 input from its history ring (16 BF16 values in slot order, two
// 16-byte vectors), its scaled density and the two ones that carry layer 1's bias; columns 19..31 are zero.
__device__ __forceinline__ void mlp_tc4_put_row_ring(MlpTcGroup &g, int r, uint4 h0, uint4 h1, float dn)
{
    unsigned char *xb = reinterpret_cast<unsigned char *>(g.x);
    *reinterpret_cast<uint4 *>(xb + core_off(r, 0, kMlpK1)) = h0;
    *reinterpret_cast<uint4 *>(xb + core_off(r, 8, kMlpK1)) = h1;
    *reinterpret_cast<uint4 *>(xb + core_off(r, 16, kMlpK1)) =
        make_uint4(pack_bf16(dn, 1.0f), pack_bf16(1.0f, 0.0f), 0u, 0u);
    *reinterpret_cast<uint4 *>(xb + core_off(r, 24, kMlpK1)) = make_uint4(0u, 0u, 0u, 0u);
}

// forward of warpgroup gi's tile (rows in g.x); thread r (0..127 inside the
// warpgroup) gets row r's output.  Returns false in every thread of the
// warpgroup if one of its bounded waits gave up.
struct MlpNoMid {
    __device__ void operator()() const {}
};

// mid() runs in every thread between the first epilogue and the second MMA (the caller's hook for work
// that should overlap the tile, e.g. issuing the next tile's loads)
template <typename Mid = MlpNoMid>
__device__ __forceinline__ float mlp_tc4_tile(MlpTcWeights &w, MlpTcGroup &g, int gi, int r, uint32_t *phase,
                                              bool *ok_out, Mid mid = Mid())
{
    const int warp = r >> 5;
    const uint32_t tmem = w.tmem + (uint32_t)(gi * 128);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint64_t kWaitNs = 1000000000ull;   // the waiting warps sleep in the barrier, not poll it
    bool ok = true;
    fence_proxy_async_smem();
    tc_fence_before();
    wg_bar(gi);
    tc_fence_after();
    if (r == 0) {
        const uint32_t xa = smem_addr(g.x), wa = smem_addr(w.w1);
#pragma unroll
        for (int kk = 0; kk < kMlpK1 / 16; ++kk)
            tc_mma(tmem, tc_desc(xa + kk * 256, 128, (kMlpK1 / 8) * 128), tc_desc(wa + kk * 256, 128, (kMlpK1 / 8) * 128),
                   kTcIdesc, kk > 0);
        tc_commit(&g.mbar);
    }
    if (!mbar_wait_timed(&g.mbar, *phase, kWaitNs)) ok = false;
    *phase ^= 1u;
    tc_fence_after();
    unsigned char *a2 = reinterpret_cast<unsigned char *>(g.a2);
    // 16 columns at a time, the next 16 in flight from TMEM while these are activated
    uint32_t ra[16], rb[16];
    tc_ld16_async(tmem + lane_base, ra);
    tc_wait_ld16(ra);
#pragma unroll
    for (int c = 0; c < kMlpH / 16; ++c) {
        uint32_t(&cur)[16] = (c & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
        if (c + 1 < kMlpH / 16) tc_ld16_async(tmem + lane_base + (c + 1) * 16, nxt);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k0 = c * 16 + q * 8;   // the accumulator already holds the bias (rows 17, 18 of W1)
            auto v = [&](int i) { return __uint_as_float(cur[q * 8 + i]); };
            const float2 g0 = gelu2_f2(f2(v(0), v(1)));
            const float2 g1 = gelu2_f2(f2(v(2), v(3)));
            const float2 g2 = gelu2_f2(f2(v(4), v(5)));
            const float2 g3 = gelu2_f2(f2(v(6), v(7)));
            uint4 pk;
            pk.x = pack_bf16(g0.x, g0.y);
            pk.y = pack_bf16(g1.x, g1.y);
            pk.z = pack_bf16(g2.x, g2.y);
            pk.w = pack_bf16(g3.x, g3.y);
            *reinterpret_cast<uint4 *>(a2 + core_off(r, k0, kMlpH)) = pk;
        }
        if (c + 1 < kMlpH / 16) tc_wait_ld16(nxt);
    }
    mid();
    fence_proxy_async_smem();
    tc_fence_before();
    wg_bar(gi);
    tc_fence_after();
    if (r == 0) {
        const uint32_t aa = smem_addr(g.a2), wa = smem_addr(w.w2);
#pragma unroll
        for (int kk = 0; kk < kMlpH / 16; ++kk)
            tc_mma(tmem, tc_desc(aa + kk * 256, 128, (kMlpH / 8) * 128), tc_desc(wa + kk * 256, 128, (kMlpH / 8) * 128),
                   kTcIdesc, kk > 0);
        tc_commit(&g.mbar);
    }
    if (!mbar_wait_timed(&g.mbar, *phase, kWaitNs)) ok = false;
    *phase ^= 1u;
    tc_fence_after();
    float y = w.b3;
    tc_ld16_async(tmem + lane_base, ra);
    tc_wait_ld16(ra);
#pragma unroll
    for (int c = 0; c < kMlpH / 16; ++c) {
        uint32_t(&cur)[16] = (c & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
        if (c + 1 < kMlpH / 16) tc_ld16_async(tmem + lane_base + (c + 1) * 16, nxt);
        auto v = [&](int i) { return __uint_as_float(cur[i]); };
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            const float4 b = *reinterpret_cast<const float4 *>(&w.b2[c * 16 + i]);
            const float4 o = *reinterpret_cast<const float4 *>(&w.w3[c * 16 + i]);
            const float2 g0 = gelu2_f2(f2_add(f2(v(i + 0), v(i + 1)), f2(b.x, b.y)));
            const float2 g1 = gelu2_f2(f2_add(f2(v(i + 2), v(i + 3)), f2(b.z, b.w)));
            y = fmaf(g0.x, o.x, y);
            y = fmaf(g0.y, o.y, y);
            y = fmaf(g1.x, o.z, y);
            y = fmaf(g1.y, o.w, y);
        }
        if (c + 1 < kMlpH / 16) tc_wait_ld16(nxt);
    }
    tc_fence_before();
    // warpgroup-uniform verdict
    if (!ok) g.flag = 1;
    wg_bar(gi);
    *ok_out = g.flag == 0;
    return y;
}

}  // namespace fp

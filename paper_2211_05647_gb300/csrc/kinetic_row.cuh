// kinetic_row.cuh -- per-row pieces of the Sec. 5.2 kinetic update shared by
// the plasma-row kernel (kinetic.cu) and the batched 1-D kernel (batch1d.cu):
// 16-byte storage vectors, FP32/FP64/BF16 unpacking, shared-memory table
// loads and the streaming / stochastically rounded stores.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace fp {

template <typename TS>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
};
template <>
struct Vec<__nv_bfloat16> {
    using type = uint4;
    static constexpr int n = 8;
};

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename TA>
__device__ __forceinline__ TA shfl_xor(TA v, int off)
{
    return __shfl_xor_sync(0xffffffffu, v, off);
}

// unpack a 16-byte storage vector into compute values
__device__ __forceinline__ void unpack(const float4 &v, float *x)
{
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void unpack(const double2 &v, double *x)
{
    x[0] = v.x; x[1] = v.y;
}
__device__ __forceinline__ void unpack(const uint4 &v, float *x)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x[2 * q] = __uint_as_float(w[q] << 16);
        x[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
}

// load VEC consecutive compute values from shared memory (16-byte aligned)
template <int VEC>
__device__ __forceinline__ void lds(const float *p, float *x)
{
#pragma unroll
    for (int q = 0; q < VEC / 4; ++q) {
        float4 t = reinterpret_cast<const float4 *>(p)[q];
        x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
    }
}
template <int VEC>
__device__ __forceinline__ void lds(const double *p, double *x)
{
#pragma unroll
    for (int q = 0; q < VEC / 2; ++q) {
        double2 t = reinterpret_cast<const double2 *>(p)[q];
        x[2 * q] = t.x; x[2 * q + 1] = t.y;
    }
}

template <typename TS>
struct Store;
template <>
struct Store<float> {
    static __device__ __forceinline__ void st(float4 *p, const float *x, uint4, uint2)
    {
        __stcs(p, make_float4(x[0], x[1], x[2], x[3]));
    }
};
template <>
struct Store<double> {
    static __device__ __forceinline__ void st(double2 *p, const double *x, uint4, uint2)
    {
        __stcs(p, make_double2(x[0], x[1]));
    }
};
// BF16 storage: one Philox4x32-7 call per 8 nodes (16 bits a node).  A vector
// whose 8 values sum to a finite number holds no infinity or NaN, so each value
// takes the plain rule (add the draw, keep the high half; two halves packed by
// one byte permute); otherwise (or if the sum overflows) every value goes
// through f32_to_bf16_sr, which keeps infinities and NaNs.
template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ void st(uint4 *p, const float *x, uint4 ctr, uint2 key)
    {
        const uint4 r = philox4x32_7(ctr, key);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        uint32_t w[4];
        const float2 h = f2_split(f2_add(f2_add(f2(x[0], x[1]), f2(x[2], x[3])), f2_add(f2(x[4], x[5]), f2(x[6], x[7]))));
        if (fabsf(h.x + h.y) < INFINITY) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                w[q] = __byte_perm(__float_as_uint(x[2 * q]) + (rr[q] & 0xffffu),
                                   __float_as_uint(x[2 * q + 1]) + (rr[q] >> 16), 0x7632);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t lo = f32_to_bf16_sr(x[2 * q], rr[q] & 0xffffu);
                const uint32_t hi = f32_to_bf16_sr(x[2 * q + 1], rr[q] >> 16);
                w[q] = lo | (hi << 16);
            }
        }
        __stcs(p, make_uint4(w[0], w[1], w[2], w[3]));
    }
};

// One lane's share of a delta-f row: VPL vectors at indices q*L + l.  Updates
// df <- alpha df + beta nE in place (store through Store<TS>) and returns the
// lane's partial sum of w' df in (s, c): compensated (TwoSum) for FP32 / FP64
// rows; for BF16 rows a plain FP32 accumulation, whose rounding (~1e-6 of the
// sum for a row of <= 1024 nodes) is far below the 2^-8 storage rounding of the
// terms, and which takes a fifth of the row's instructions.  BF16 rows run on
// the two-lane FP32 instructions: node pairs (2t, 2t+1) get alpha df + (beta nE)
// with the roundings of the scalar fma, and the sum is kept as two partial sums
// (even and odd nodes) added at the end.
template <typename TS, typename TA, int VPL, int L>
__device__ __forceinline__ void row_update(typename Vec<TS>::type *rp, const typename Vec<TS>::type *v,
                                           const TA *al_tab, const TA *be_tab, const TA *w_tab, TA nE, int l,
                                           uint32_t row_id, int64_t step, uint2 key, TA &s, TA &c)
{
    constexpr int VEC = Vec<TS>::n;
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
        uint64_t s2 = f2(0.0f, 0.0f);
        const uint64_t ne2 = f2(nE, nE);
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            const int vi = q * L + l;
            float x[VEC], al[VEC], be[VEC], w[VEC];
            unpack(v[q], x);
            lds<VEC>(al_tab + vi * VEC, al);
            lds<VEC>(be_tab + vi * VEC, be);
            lds<VEC>(w_tab + vi * VEC, w);
#pragma unroll
            for (int t = 0; t < VEC; t += 2) {
                const uint64_t xn = f2_fma(f2(al[t], al[t + 1]), f2(x[t], x[t + 1]), f2_mul(f2(be[t], be[t + 1]), ne2));
                s2 = f2_fma(f2(w[t], w[t + 1]), xn, s2);
                const float2 xs = f2_split(xn);
                x[t] = xs.x;
                x[t + 1] = xs.y;
            }
            const uint4 ctr = make_uint4(row_id, (uint32_t)vi, (uint32_t)step, (uint32_t)(step >> 32));
            Store<TS>::st(rp + vi, x, ctr, key);
        }
        const float2 ss = f2_split(s2);
        s += ss.x + ss.y;
    } else {
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            const int vi = q * L + l;
            TA x[VEC], al[VEC], be[VEC], w[VEC];
            unpack(v[q], x);
            lds<VEC>(al_tab + vi * VEC, al);
            lds<VEC>(be_tab + vi * VEC, be);
            lds<VEC>(w_tab + vi * VEC, w);
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
                x[t] = al[t] * x[t] + be[t] * nE;
                TA hi, lo;
                two_sum(s, mul_rn(w[t], x[t]), hi, lo);
                s = hi;
                c += lo;
            }
            Store<TS>::st(rp + vi, x, uint4{}, uint2{});
        }
    }
}

// TwoSum tree over the L lanes sharing a row (xor offsets < L stay inside the group)
template <typename TA, int L>
__device__ __forceinline__ TA row_reduce(TA s, TA c)
{
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) {
        const TA so = __shfl_xor_sync(0xffffffffu, s, off), co = __shfl_xor_sync(0xffffffffu, c, off);
        TA hi, lo;
        two_sum(s, so, hi, lo);
        s = hi;
        c = c + co + lo;
    }
    return s + c;
}

}  // namespace fp

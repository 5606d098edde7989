// kinetic.cu -- the phase-space kernel: per plasma cell ("slot") the
// Crank-Nicolson update of the anisotropic distribution (Sec. 5.2, Eq. 22,
// the printed f_1x update)
//     df_j^{n+1/2} = alpha_j df_j^{n-1/2} + beta_j (n E^n)
// on every velocity node j, the current moment (Eq. 24, the Jx sum)
//     J^{n+1/2} = sum_j w'_j df_j^{n+1/2},   w'_j = -e w_j
// reduced with compensated (TwoSum) arithmetic, and the Ampere source term
// applied to the cell's own E in place: E^n <- E^n - (dt/eps0) J^{n+1/2}
// (the curl is added afterwards by the E stencil kernel; the E update is
// linear, so the order of the two additions only changes rounding).
//
// Layout: rows of `pitch` elements, [slot][node], pitch = a power-of-two
// number of 16-byte vectors >= nnode (padding nodes have alpha = beta = w = 0
// and stay 0).  L lanes share a row, each lane holding VPL >= 4 vectors when
// the row has that many; a warp covers 32/L rows.  The whole row is loaded
// before any arithmetic so each lane has VPL 16-byte loads in flight, the
// loads/stores use the streaming (evict-first) cache hint because delta f is
// far larger than L2, and the per-node tables sit in shared memory.
// BF16 storage: FP32 arithmetic, stochastic rounding on store with 16 random
// bits per node from Philox4x32-10 keyed by the seed and counted by
// (slot, vector, step).
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
template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ void st(uint4 *p, const float *x, uint4 ctr, uint2 key)
    {
        const uint4 r = philox4x32_10(ctr, key);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t lo = f32_to_bf16_sr(x[2 * q], rr[q] & 0xffffu);
            uint32_t hi = f32_to_bf16_sr(x[2 * q + 1], rr[q] >> 16);
            w[q] = lo | (hi << 16);
        }
        __stcs(p, make_uint4(w[0], w[1], w[2], w[3]));
    }
};

template <typename TS, typename TA, int VPL, int L>
__global__ void __launch_bounds__(256) k_kinetic(KinArgs<TA> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA *s_tab = reinterpret_cast<TA *>(smem_raw);
    for (int t = threadIdx.x; t < 3 * a.pitch; t += blockDim.x) s_tab[t] = a.tab[t];
    __syncthreads();
    const TA *s_al = s_tab, *s_be = s_tab + a.pitch, *s_w = s_tab + 2 * a.pitch;

    using V = typename Vec<TS>::type;
    constexpr int VEC = Vec<TS>::n;
    constexpr int R = 32 / L;   // rows per warp
    const int lane = threadIdx.x & 31;
    const int sub = lane / L, l = lane % L;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = *a.d_step + a.kstep;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));

    // the slot -> cell index of the next row group is fetched one iteration
    // ahead, so the E gather of a row issues together with its delta-f loads
    int64_t row = wg * R + sub;
    int32_t cell_next = row < a.nslots ? __ldg(a.slot_cell + row) : 0;
    for (int64_t base = wg * R; base < a.nslots; base += nw * R) {
        row = base + sub;
        const bool valid = row < a.nslots;
        const int32_t cell = cell_next;
        V v[VPL];
        TA E = TA(0), nE = TA(0);
        V *rp = reinterpret_cast<V *>(a.df) + (valid ? row : 0) * (a.pitch / VEC);
        if (valid) {
#pragma unroll
            for (int q = 0; q < VPL; ++q) v[q] = __ldcs(rp + q * L + l);
            E = a.E[cell];
            nE = __ldg(a.dens + row) * E;
        }
        const int64_t row_next = row + nw * R;
        cell_next = row_next < a.nslots ? __ldg(a.slot_cell + row_next) : 0;
        TA s = TA(0), c = TA(0);
        if (valid) {
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                const int vi = q * L + l;
                TA x[VEC], al[VEC], be[VEC], w[VEC];
                unpack(v[q], x);
                lds<VEC>(s_al + vi * VEC, al);
                lds<VEC>(s_be + vi * VEC, be);
                lds<VEC>(s_w + vi * VEC, w);
#pragma unroll
                for (int t = 0; t < VEC; ++t) {
                    x[t] = al[t] * x[t] + be[t] * nE;
                    TA hi, lo;
                    two_sum(s, mul_rn(w[t], x[t]), hi, lo);
                    s = hi;
                    c += lo;
                }
                const uint4 ctr = make_uint4((uint32_t)row, (uint32_t)vi, (uint32_t)step, (uint32_t)(step >> 32));
                Store<TS>::st(rp + vi, x, ctr, key);
            }
        }
        // TwoSum tree over the L lanes of the row (xor offsets < L stay inside the group)
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            const TA so = shfl_xor(s, off), co = shfl_xor(c, off);
            TA hi, lo;
            two_sum(s, so, hi, lo);
            s = hi;
            c = c + co + lo;
        }
        if (valid && l == 0) {
            const TA J = s + c;
            a.jslot[row] = J;
            a.E[cell] = E - a.cj * J;
        }
    }
}

int kinetic_pitch(int nnode, int f_dtype)
{
    const int vec = f_dtype == FDTD_DF_BF16 ? 8 : (f_dtype == FDTD_DF_F64 ? 2 : 4);
    int nv = (nnode + vec - 1) / vec;
    int p2 = 1;
    while (p2 < nv) p2 <<= 1;
    return p2 * vec;
}

template <typename TS, typename TA, int VPL, int L>
static cudaError_t run(cudaStream_t st, const KinArgs<TA> &a, int num_sms)
{
    auto kern = k_kinetic<TS, TA, VPL, L>;
    const size_t smem = 3 * (size_t)a.pitch * sizeof(TA);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t rows_per_block = (256 / 32) * (32 / L);
    int64_t blocks = (a.nslots + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename TS, typename TA>
static cudaError_t dispatch(cudaStream_t st, const KinArgs<TA> &a, int num_sms)
{
    // vectors per row (a power of two): lanes per row L chosen so that every
    // lane keeps at least 4 sixteen-byte loads in flight (fewer only for rows
    // shorter than 4 vectors), at most 32 lanes
    const int V = a.pitch / Vec<TS>::n;
    switch (V) {
    case 1: return run<TS, TA, 1, 1>(st, a, num_sms);
    case 2: return run<TS, TA, 2, 1>(st, a, num_sms);
    case 4: return run<TS, TA, 4, 1>(st, a, num_sms);
    case 8: return run<TS, TA, 4, 2>(st, a, num_sms);
    case 16: return run<TS, TA, 4, 4>(st, a, num_sms);
    case 32: return run<TS, TA, 4, 8>(st, a, num_sms);
    case 64: return run<TS, TA, 4, 16>(st, a, num_sms);
    case 128: return run<TS, TA, 4, 32>(st, a, num_sms);
    case 256: return run<TS, TA, 8, 32>(st, a, num_sms);
    case 512: return run<TS, TA, 16, 32>(st, a, num_sms);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_kinetic<float>(cudaStream_t st, const KinArgs<float> &a, int f_dtype, int num_sms)
{
    if (a.nslots == 0) return cudaSuccess;
    if (f_dtype == FDTD_DF_F32) return dispatch<float, float>(st, a, num_sms);
    if (f_dtype == FDTD_DF_BF16) return dispatch<__nv_bfloat16, float>(st, a, num_sms);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_kinetic<double>(cudaStream_t st, const KinArgs<double> &a, int f_dtype, int num_sms)
{
    if (a.nslots == 0) return cudaSuccess;
    if (f_dtype == FDTD_DF_F64) return dispatch<double, double>(st, a, num_sms);
    return cudaErrorInvalidValue;
}

}  // namespace fp

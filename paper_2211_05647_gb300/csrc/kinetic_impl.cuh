// kinetic_impl.cuh -- the plasma-row kernel template and its launch for one
// (lanes per row, vectors per lane) shape; instantiated per storage type in
// kinetic.cu (FP32), kinetic_bf16.cu and kinetic_f64.cu.
#pragma once

#include "kinetic_row.cuh"

namespace fp {

template <typename TS, typename TA, int VPL, int L>
__global__ void __launch_bounds__(256) k_kinetic(KinArgs<TA> a)
{
    pdl_enter();
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
        if (valid) row_update<TS, TA, VPL, L>(rp, v, s_al, s_be, s_w, nE, l, (uint32_t)(row + a.slot_base), step, key, s, c);
        const TA J = row_reduce<TA, L>(s, c);
        if (valid && l == 0) {
            if (a.store_j) a.jslot[row] = J;
            a.E[cell] = E - a.cj * J;
        }
    }
}

template <typename TS, typename TA, int VPL, int L>
cudaError_t run_kinetic(cudaStream_t st, const KinArgs<TA> &a, int num_sms, int blocks_per_sm)
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
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    const int64_t rows_per_block = (256 / 32) * (32 / L);
    int64_t blocks = (a.nslots + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    launch_pdl(kern, dim3((unsigned)blocks), dim3(256), smem, st, a);
    return cudaGetLastError();
}

// Shape candidates (VPL, L) for V vectors per row; the first is the default
// (every lane keeps >= 4 sixteen-byte loads in flight when the row allows it).
inline int kinetic_shape_candidates(int V, int (*out)[2])
{
    static const int tab[][2] = {{1, 1},
                                 {2, 1}, {1, 2},
                                 {4, 1}, {2, 2}, {1, 4},
                                 {4, 2}, {8, 1}, {2, 4}, {1, 8},
                                 {4, 4}, {8, 2}, {2, 8}, {1, 16},
                                 {4, 8}, {8, 4}, {2, 16}, {1, 32},
                                 {4, 16}, {8, 8}, {2, 32},
                                 {4, 32}, {8, 16}, {16, 8},
                                 {8, 32}, {16, 16},
                                 {16, 32}};
    int n = 0;
    for (const auto &p : tab)
        if (p[0] * p[1] == V) { out[n][0] = p[0]; out[n][1] = p[1]; ++n; }
    return n;
}

template <typename TS, typename TA>
cudaError_t dispatch_kinetic(cudaStream_t st, const KinArgs<TA> &a, int num_sms, int vpl, int l, int bps)
{
    switch (vpl * 64 + l) {
#define FP_KCASE(V_, L_) \
    case V_ * 64 + L_: return run_kinetic<TS, TA, V_, L_>(st, a, num_sms, bps);
    FP_KCASE(1, 1) FP_KCASE(2, 1) FP_KCASE(1, 2) FP_KCASE(4, 1) FP_KCASE(2, 2) FP_KCASE(1, 4)
    FP_KCASE(4, 2) FP_KCASE(8, 1) FP_KCASE(2, 4) FP_KCASE(1, 8) FP_KCASE(4, 4) FP_KCASE(8, 2) FP_KCASE(2, 8)
    FP_KCASE(1, 16) FP_KCASE(4, 8) FP_KCASE(8, 4) FP_KCASE(2, 16) FP_KCASE(1, 32) FP_KCASE(4, 16) FP_KCASE(8, 8)
    FP_KCASE(2, 32) FP_KCASE(4, 32) FP_KCASE(8, 16) FP_KCASE(16, 8) FP_KCASE(8, 32) FP_KCASE(16, 16)
    FP_KCASE(16, 32)
#undef FP_KCASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fp

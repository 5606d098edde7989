// kinetic_ring.cu -- the plasma-row kernel of kinetic.cu (Sec. 5.2, Eq. 22:
// df_j <- alpha_j df_j + beta_j n E on every node; Eq. 24: J = sum_j w'_j df_j;
// E <- E - dt/eps0 J) with delta f streamed through shared memory.
//
// One producer warp copies chunks of consecutive rows, together with their
// cell indices and densities, from global memory into a ring of
// shared-memory stages (cp.async.bulk, completion counted in bytes on one
// mbarrier per stage); eight consumer warps update the rows from shared
// memory and store them back with streaming stores, then release the stage.
// The bytes in flight per SM are the ring's (several chunks per CTA), not what
// the consumer threads' registers can hold.  The consumers gather E for the
// next chunk while they update the current one (each cell has one row, so
// those E values are not written by this launch before they are read).
// On GB300 this wins on long FP32 rows (2-D 4096^2, 1024 nodes: 16 rows x
// 4 KB a chunk, three stages, at the measured copy bandwidth); short BF16 rows
// (64-128 bytes) are bound by their stochastic-rounding arithmetic at the
// occupancy they get, and the register kernel stays faster there (the
// autotuner times both).
//
// A chunk is one pass of the consumer threads: 256 / L rows, each row's
// VPL * L vectors held VPL per lane, exactly as in the register kernel, and
// the arithmetic, the stochastic-rounding counters and the J reduction are
// the register kernel's (kinetic_row.cuh): for the same (VPL, L) the stored
// rows, J and E are identical bit for bit.
//
// Every wait is bounded (wall clock): a wait that gives up sets *err, the
// consumers stop, and the producer waits (bounded) for the copies it has in
// flight before the CTA ends.  The index and density copies are rounded up
// to 16 bytes; their arrays are allocated in multiples of four entries.
#include "async.cuh"
#include "kinetic_row.cuh"

namespace fp {

constexpr int kRingConsumerWarps = 8;
constexpr int kRingConsumers = 32 * kRingConsumerWarps;
constexpr int kRingThreads = kRingConsumers + 32;
constexpr uint64_t kRingWaitNs = 1000000000ull;
constexpr size_t kRingMaxSmem = 232448;   // 227 KB, the opt-in limit per CTA

struct RingGeom {
    int rp;            // rows per chunk
    int rowb;          // bytes per row
    int tab_bytes;     // alpha | beta | w' tables (FP32), rounded up to 128 bytes
    int df_bytes;      // rows of a stage
    int stage_bytes;   // rows + cell indices + densities, rounded up to 128 bytes
};

__host__ __device__ inline RingGeom ring_geom(int pitch, int esz, int L)
{
    RingGeom g;
    g.rp = kRingConsumers / L;
    g.rowb = pitch * esz;
    g.tab_bytes = (3 * pitch * 4 + 127) & ~127;
    g.df_bytes = g.rp * g.rowb;
    g.stage_bytes = (g.df_bytes + g.rp * 8 + 127) & ~127;
    return g;
}

inline size_t ring_smem(const RingGeom &g, int stages)
{
    return (size_t)g.tab_bytes + (size_t)stages * g.stage_bytes + 16 * (size_t)stages;   // + full / empty barriers
}

template <typename TS, int VPL, int L>
__global__ void __launch_bounds__(kRingThreads) k_kinetic_ring(KinArgs<float> a, int stages)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using V = typename Vec<TS>::type;
    constexpr int VEC = Vec<TS>::n;
    constexpr int RP = kRingConsumers / L;
    const RingGeom g = ring_geom(a.pitch, (int)sizeof(TS), L);
    float *s_tab = reinterpret_cast<float *>(smem_raw);
    unsigned char *ring = smem_raw + g.tab_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (size_t)stages * g.stage_bytes);
    uint64_t *empty = full + stages;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < 3 * a.pitch; t += blockDim.x) s_tab[t] = a.tab[t];
    if (tid == 0)
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kRingConsumerWarps);
        }
    __syncthreads();
    const int64_t nchunks = (a.nslots + RP - 1) / RP;

    if (warp == kRingConsumerWarps) {
        // producer: one lane issues the copies of this CTA's chunks (blockIdx.x, + gridDim.x, ...)
        if (lane != 0) return;
        bool ok = true;
        int64_t k = 0;
        for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x, ++k) {
            const int s = (int)(k % stages);
            if (k >= stages && !mbar_wait_timed(&empty[s], (uint32_t)((k / stages - 1) & 1), kRingWaitNs)) {
                ok = false;
                break;
            }
            const int64_t r0 = q * RP;
            const int rows = (int)min((int64_t)RP, a.nslots - r0);
            unsigned char *sp = ring + (size_t)s * g.stage_bytes;
            const uint32_t db = (uint32_t)rows * (uint32_t)g.rowb, ib = ((uint32_t)rows * 4u + 15u) & ~15u;
            mbar_arrive_expect_tx(&full[s], db + 2 * ib);
            bulk_load(sp, reinterpret_cast<const unsigned char *>(a.df) + r0 * g.rowb, db, &full[s], true);
            bulk_load(sp + g.df_bytes, a.slot_cell + r0, ib, &full[s], false);
            bulk_load(sp + g.df_bytes + RP * 4, a.dens + r0, ib, &full[s], false);
        }
        // the copies of the last issue on each stage land before the CTA ends
        for (int64_t j = k > stages ? k - stages : 0; j < k; ++j)
            if (!mbar_wait_timed(&full[j % stages], (uint32_t)((j / stages) & 1), kRingWaitNs)) ok = false;
        if (!ok) atomicExch(a.err, 1);
        return;
    }

    // consumers: thread tid holds lane l of row `sub` of every chunk
    const int sub = tid / L, l = tid % L;
    const int64_t step = *a.d_step + a.kstep;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const float *s_al = s_tab, *s_be = s_tab + a.pitch, *s_w = s_tab + 2 * a.pitch;
    auto cells_of = [&](int s) { return reinterpret_cast<const int32_t *>(ring + (size_t)s * g.stage_bytes + g.df_bytes); };
    auto dens_of = [&](int s) {
        return reinterpret_cast<const float *>(ring + (size_t)s * g.stage_bytes + g.df_bytes + RP * 4);
    };
    bool ok = true;
    int32_t cell = 0;
    float E = 0.0f;
    int64_t q = blockIdx.x, k = 0;
    if (q < nchunks) {
        ok = __all_sync(0xffffffffu, mbar_wait_timed(&full[0], 0u, kRingWaitNs));
        if (ok && sub < min((int64_t)RP, a.nslots - q * RP)) {
            cell = cells_of(0)[sub];
            E = a.E[cell];
        }
    }
    for (; ok && q < nchunks; q += gridDim.x, ++k) {
        const int s = (int)(k % stages);
        const int64_t r0 = q * RP;
        const bool valid = sub < min((int64_t)RP, a.nslots - r0);
        // the next chunk's cell and E, gathered while this chunk is updated
        const int64_t qn = q + gridDim.x;
        int32_t cell_n = 0;
        float E_n = 0.0f;
        if (qn < nchunks) {
            const int sn = (int)((k + 1) % stages);
            ok = __all_sync(0xffffffffu, mbar_wait_timed(&full[sn], (uint32_t)(((k + 1) / stages) & 1), kRingWaitNs));
            if (ok && sub < min((int64_t)RP, a.nslots - qn * RP)) {
                cell_n = cells_of(sn)[sub];
                E_n = a.E[cell_n];
            }
        }
        V v[VPL];
        float nE = 0.0f;
        if (valid) {
            const V *rs = reinterpret_cast<const V *>(ring + (size_t)s * g.stage_bytes + (size_t)sub * g.rowb);
#pragma unroll
            for (int p = 0; p < VPL; ++p) v[p] = rs[p * L + l];
            nE = dens_of(s)[sub] * E;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);   // the stage is in registers: the producer may refill it
        float su = 0.0f, c = 0.0f;
        V *rp = reinterpret_cast<V *>(a.df) + (valid ? r0 + sub : 0) * (int64_t)(a.pitch / VEC);
        if (valid)
            row_update<TS, float, VPL, L>(rp, v, s_al, s_be, s_w, nE, l, (uint32_t)(r0 + sub + a.slot_base), step, key,
                                          su, c);
        const float J = row_reduce<float, L>(su, c);
        if (valid && l == 0) {
            if (a.store_j) a.jslot[r0 + sub] = J;
            a.E[cell] = E - a.cj * J;
        }
        cell = cell_n;
        E = E_n;
    }
    if (!ok && lane == 0) atomicExch(a.err, 1);
}

size_t kinetic_ring_smem(int pitch, int f_dtype, int l, int stages)
{
    const int esz = f_dtype == FDTD_DF_BF16 ? 2 : 4;
    return ring_smem(ring_geom(pitch, esz, l), stages);
}

bool kinetic_ring_fits(int pitch, int f_dtype, int l, int stages)
{
    return stages >= 2 && (f_dtype == FDTD_DF_F32 || f_dtype == FDTD_DF_BF16) && l > 0 &&
           kinetic_ring_smem(pitch, f_dtype, l, stages) <= kRingMaxSmem;
}

template <typename TS, int VPL, int L>
cudaError_t run_ring(cudaStream_t st, const KinArgs<float> &a, int num_sms, int bps, int stages)
{
    const RingGeom g = ring_geom(a.pitch, (int)sizeof(TS), L);
    const size_t smem = ring_smem(g, stages);
    if (stages < 2 || smem > kRingMaxSmem || a.err == nullptr) return cudaErrorInvalidValue;
    auto kern = k_kinetic_ring<TS, VPL, L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRingThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidValue;
    if (bps > 0 && bps < per_sm) per_sm = bps;
    const int64_t chunks = (a.nslots + g.rp - 1) / g.rp;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)num_sms * per_sm));
    e = launch_plain(kern, dim3((unsigned)blocks), dim3(kRingThreads), smem, st, a, stages);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename TS>
cudaError_t dispatch_ring(cudaStream_t st, const KinArgs<float> &a, int num_sms, int vpl, int l, int bps, int stages)
{
    switch (vpl * 64 + l) {
#define FP_RCASE(V_, L_) \
    case V_ * 64 + L_: return run_ring<TS, V_, L_>(st, a, num_sms, bps, stages);
    FP_RCASE(1, 1) FP_RCASE(2, 1) FP_RCASE(1, 2) FP_RCASE(4, 1) FP_RCASE(2, 2) FP_RCASE(1, 4)
    FP_RCASE(4, 2) FP_RCASE(8, 1) FP_RCASE(2, 4) FP_RCASE(1, 8) FP_RCASE(4, 4) FP_RCASE(8, 2) FP_RCASE(2, 8)
    FP_RCASE(1, 16) FP_RCASE(4, 8) FP_RCASE(8, 4) FP_RCASE(2, 16) FP_RCASE(1, 32) FP_RCASE(4, 16) FP_RCASE(8, 8)
    FP_RCASE(2, 32) FP_RCASE(4, 32) FP_RCASE(8, 16) FP_RCASE(16, 8) FP_RCASE(8, 32) FP_RCASE(16, 16)
    FP_RCASE(16, 32)
#undef FP_RCASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_kinetic_ring(cudaStream_t st, const KinArgs<float> &a, int f_dtype, int num_sms, int vpl, int l,
                                int bps, int stages)
{
    if (a.nslots == 0) return cudaSuccess;
    if (f_dtype == FDTD_DF_F32) return dispatch_ring<float>(st, a, num_sms, vpl, l, bps, stages);
    if (f_dtype == FDTD_DF_BF16) return dispatch_ring<__nv_bfloat16>(st, a, num_sms, vpl, l, bps, stages);
    return cudaErrorInvalidValue;
}

}  // namespace fp

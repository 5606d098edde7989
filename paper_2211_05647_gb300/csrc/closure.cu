// closure.cu -- the learned J closure inside the time step, and the recorder
// that harvests its training data from kinetic runs.
//
// The closure stands in for the Sec. 5.2 velocity-space update of a plasma
// cell: from the cell's last 16 values of E (a ring buffer, E^{n-15..n}) and
// its density it predicts
//     J^{n+1/2} = rho J^{n-1/2} + beta n E^n + J_s y,   y = MLP(E^{n-15..n} / E_s, n / n_s)
// where rho J^{n-1/2} + beta n E^n is the Crank-Nicolson Drude update of a
// plasma with the mean collision frequency, so the network carries only the
// kinetic correction (rho = beta = 0 gives the direct form J = J_s y), then
// applies the Ampere source
// term E <- E - dt/eps0 J^{n+1/2} like the kinetic kernel.  Cells denser than
// the training range keep the kinetic update (they are separate slots).
//
// Recording (kinetic runs): before the kinetic kernel every plasma cell pushes
// E^n into its ring; after it, a seeded counter-based draw selects about
// `rate` of the (cell, step) pairs, and each selected pair appends one sample
//     [E^{n-15} .. E^n, n, J^{n+1/2}, J^{n-1/2}]   (19 floats)
// to the caller's buffer.
#include "cp_async.cuh"
#include "mlp_tc.cuh"

namespace fp {


__global__ void __launch_bounds__(256) k_closure(ClosureArgs a)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(smem_raw);
    __shared__ int32_t s_cell[kMlpRows];
    __shared__ float s_e[kMlpRows];
    mlp_load_weights(s, a.P);
    const int64_t step = *a.d_step + a.kstep;
    const int ring = (int)(step & 15);
    const int64_t ntiles = (a.n + kMlpRows - 1) / kMlpRows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kMlpRows;
        const int r = threadIdx.x;
        if (r < kMlpRows) {
            const int64_t slot = row0 + r;
            float x[kMlpK1];
#pragma unroll
            for (int k = 0; k < kMlpK1; ++k) x[k] = 0.0f;
            if (slot < a.n) {
                const int32_t c = a.cell[slot];
                const float e = a.E[c];
                float *h = a.hist + slot * 16;
                h[ring] = e;
                float hv[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = reinterpret_cast<const float4 *>(h)[q];
                    hv[4 * q] = v.x; hv[4 * q + 1] = v.y; hv[4 * q + 2] = v.z; hv[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) x[k] = hv[(ring + 1 + k) & 15] * a.inv_es;   // oldest first
                x[16] = a.dens[slot] * a.inv_ns;
                s_cell[r] = c;
                s_e[r] = e;
            }
#pragma unroll
            for (int k = 0; k < kMlpK1; k += 2)
                *reinterpret_cast<uint32_t *>(&s.x[r][k]) = pack_bf16(x[k], x[k + 1]);
        }
        __syncthreads();
        mlp_tile_forward(s);
        __syncthreads();
        if (r < kMlpRows) {
            const int64_t slot = row0 + r;
            if (slot < a.n) {
                const float J = a.rho * a.jprev[slot] + a.beta * a.dens[slot] * s_e[r] + a.js * s.y[r];
                a.jprev[slot] = J;
                if (a.store_j) a.jslot[slot] = J;
                a.E[s_cell[r]] = s_e[r] - a.cj * J;
            }
        }
        __syncthreads();
    }
}

__global__ void k_hist_push(const int32_t *__restrict__ cell, int64_t n, const float *__restrict__ E,
                            float *__restrict__ hist, const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int ring = (int)((*d_step + kstep) & 15);
    hist[s * 16 + ring] = E[cell[s]];
}

__global__ void k_record(int64_t n, const float *__restrict__ hist, const float *__restrict__ dens,
                         const float *__restrict__ jslot, float *__restrict__ jprev, float *__restrict__ out,
                         int64_t capacity, unsigned long long *__restrict__ count, uint32_t threshold, uint64_t seed,
                         const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t step = *d_step + kstep;
    const float J = jslot[s], Jp = jprev[s];
    const uint4 r = philox4x32_7(make_uint4((uint32_t)s, (uint32_t)(s >> 32), (uint32_t)step, (uint32_t)(step >> 32)),
                                 make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    if (r.x < threshold) {
        const unsigned long long idx = atomicAdd(count, 1ull);
        if ((int64_t)idx < capacity) {
            const int ring = (int)(step & 15);
            float *o = out + (int64_t)idx * 19;
#pragma unroll
            for (int k = 0; k < 16; ++k) o[k] = hist[s * 16 + ((ring + 1 + k) & 15)];
            o[16] = dens[s];
            o[17] = J;
            o[18] = Jp;
        }
    }
    jprev[s] = J;
}

// The same closure step on the tcgen05 tile: one 512-thread CTA per SM with
// four independent warpgroup pipelines (each its own TMEM accumulator and
// tiles, one shared copy of the weights); thread r of a warpgroup owns row r
// of its tile (history push, input row, J and E update).  Its history ring
// holds the network inputs themselves, E / E_s rounded to BF16 (the rounding
// the input gets anyway), 32 bytes a cell in slot order: W1's rows are stored
// in the ring's slot order of the step, so a row is copied, never rotated.  If
// a bounded MMA-completion wait gives up, *err is set and the warpgroup stops.
// A warpgroup's copy of its next tile's row data: each thread copies its own row (history ring, cell
// index, density and the previous J while the current tile's first MMA runs, then the E value the cell
// index points at, between the two layers) and reads back only that row, so no barrier is needed.
struct ClosureNext {
    __align__(16) uint4 h[kMlpRows][2];
    int32_t cell[kMlpRows];
    float dens[kMlpRows];
    float e[kMlpRows];
    float jp[kMlpRows];
};
struct ClosureTcSmem {
    MlpTcSmem4 m;
    ClosureNext next[kTcGroups];
};

__global__ void __launch_bounds__(512, 1) k_closure_tc(ClosureArgs a)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ClosureTcSmem &cs = *reinterpret_cast<ClosureTcSmem *>(smem_raw);
    MlpTcSmem4 &s = cs.m;
    const int64_t step = *a.d_step + a.kstep;
    const int ring = (int)(step & 15);
    mlp_tc4_load_weights(s.w, a.P, ring);
    mlp_tc4_setup(s);
    const int gi = threadIdx.x >> 7, r = threadIdx.x & 127;
    MlpTcGroup &g = s.g[gi];
    ClosureNext &nx = cs.next[gi];
    uint32_t phase = 0;
    bool ok = true;
    __nv_bfloat16 *hist = reinterpret_cast<__nv_bfloat16 *>(a.hist);
    const int64_t ntiles = (a.n + kMlpRows - 1) / kMlpRows;
    const int64_t stride = (int64_t)gridDim.x * kTcGroups;
    bool staged = false;   // this tile's row is in nx (copied during the previous tile)
    for (int64_t tile = (int64_t)blockIdx.x * kTcGroups + gi; tile < ntiles; tile += stride) {
        const int64_t slot = tile * kMlpRows + r;
        const bool valid = slot < a.n;
        uint4 h0 = make_uint4(0u, 0u, 0u, 0u), h1 = h0;
        float dn = 0.0f, dens = 0.0f;
        int32_t c = 0;
        float e = 0.0f, jp = 0.0f;
        if (valid) {
            if (staged) {
                cpa_wait_all();
                c = nx.cell[r];
                h0 = nx.h[r][0];
                h1 = nx.h[r][1];
                dens = nx.dens[r];
                e = nx.e[r];
                jp = nx.jp[r];
            } else {
                c = a.cell[slot];
                const uint4 *hp = reinterpret_cast<const uint4 *>(hist + slot * 16);
                h0 = hp[0];
                h1 = hp[1];
                dens = a.dens[slot];
                e = a.E[c];
                jp = a.jprev[slot];
            }
            const __nv_bfloat16 eb = __float2bfloat16_rn(e * a.inv_es);
            hist[slot * 16 + ring] = eb;
            // this step's value into the loaded copy of the ring (slot `ring`: word ring / 2, half ring % 2)
            const uint32_t bits = (uint32_t)__bfloat16_as_ushort(eb);
            const uint32_t keep = (ring & 1) ? 0x0000ffffu : 0xffff0000u, put = (ring & 1) ? bits << 16 : bits;
            const int wi = ring >> 1;
            h0.x = wi == 0 ? (h0.x & keep) | put : h0.x;
            h0.y = wi == 1 ? (h0.y & keep) | put : h0.y;
            h0.z = wi == 2 ? (h0.z & keep) | put : h0.z;
            h0.w = wi == 3 ? (h0.w & keep) | put : h0.w;
            h1.x = wi == 4 ? (h1.x & keep) | put : h1.x;
            h1.y = wi == 5 ? (h1.y & keep) | put : h1.y;
            h1.z = wi == 6 ? (h1.z & keep) | put : h1.z;
            h1.w = wi == 7 ? (h1.w & keep) | put : h1.w;
            dn = dens * a.inv_ns;
        }
        mlp_tc4_put_row_ring(g, r, h0, h1, dn);
        // the next tile's row (its E gather waits for the cell index: between the layers); the cells of
        // different slots differ, so no E value read ahead is one this launch writes later
        const int64_t nslot = slot + stride * kMlpRows;
        const bool nvalid = nslot < a.n;
        if (nvalid) {
            cpa16(&nx.h[r][0], hist + nslot * 16);
            cpa16(&nx.h[r][1], hist + nslot * 16 + 8);
            cpa4(&nx.cell[r], a.cell + nslot);
            cpa4(&nx.dens[r], a.dens + nslot);
            cpa4(&nx.jp[r], a.jprev + nslot);
            cpa_commit();
        }
        const float y = mlp_tc4_tile(s.w, g, gi, r, &phase, &ok, [&] {
            if (nvalid) {
                cpa_wait_all();
                cpa4(&nx.e[r], a.E + nx.cell[r]);
                cpa_commit();
            }
        });
        staged = true;
        if (!ok) break;
        if (valid) {
            const float J = a.rho * jp + a.beta * dens * e + a.js * y;
            a.jprev[slot] = J;
            if (a.store_j) a.jslot[slot] = J;
            a.E[c] = e - a.cj * J;
        }
    }
    cpa_wait_all();   // no copy into shared memory outlives the loop
    if (!ok && r == 0) atomicExch(a.err, 1);
    mlp_tc4_teardown(s);
}

size_t closure_smem_bytes() { return sizeof(MlpSmem); }

cudaError_t launch_closure(cudaStream_t st, const ClosureArgs &a, int num_sms)
{
    if (a.n == 0) return cudaSuccess;
    if (a.engine == 1) {
        const size_t smem = sizeof(ClosureTcSmem);
        cudaError_t e = cudaFuncSetAttribute(k_closure_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // one CTA per SM: it allocates all 512 TMEM columns
        const int64_t tiles = (a.n + kMlpRows - 1) / kMlpRows;
        const int64_t grid = std::min<int64_t>((tiles + kTcGroups - 1) / kTcGroups, (int64_t)num_sms);
        launch_pdl(k_closure_tc, dim3((unsigned)std::max<int64_t>(grid, 1)), dim3(512), smem, st, a);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_closure, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_closure, 256, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.n + kMlpRows - 1) / kMlpRows;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)num_sms * std::max(per_sm, 1));
    launch_pdl(k_closure, dim3((unsigned)grid), dim3(256), smem, st, a);
    return cudaGetLastError();
}

void launch_hist_push(cudaStream_t st, const int32_t *cell, int64_t n, const float *E, float *hist,
                      const int64_t *d_step, int kstep)
{
    if (n) launch_pdl(k_hist_push, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, cell, n, E, hist, d_step, kstep);
}

void launch_record(cudaStream_t st, int64_t n, const float *hist, const float *dens, const float *jslot, float *jprev,
                   float *out, int64_t capacity, unsigned long long *count, uint32_t threshold, uint64_t seed,
                   const int64_t *d_step, int kstep)
{
    if (n)
        launch_pdl(k_record, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, n, hist, dens, jslot, jprev, out, capacity, count,
                                                              threshold, seed, d_step, kstep);
}

}  // namespace fp

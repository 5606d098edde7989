// batch1d.cu -- many independent 1-D FDTD + kinetic runs of uneven size in
// one persistent launch (the step of Sec. 2 / Sec. 5.2 for each run: H, the
// f_1 update and J moment, E with the Ampere source term, soft source, Mur
// ends), captured in a CUDA graph.
//
// Mapping: runs are bin-packed (longest processing time first) onto
// thread-block clusters of C CTAs (C in {8, 4, 2, 1}, the one whose packing
// has the smallest largest per-CTA load among the clusters that fit on the
// GPU at once); inside a cluster the runs'
// nodes are laid end to end and cut into one contiguous, equal-cost range per
// CTA.  Per step a CTA updates H on its range, the cluster synchronises
// (hardware barrier: neighbouring ranges exchange their edge values through
// global memory / L2), the CTA updates the delta-f rows of its plasma nodes
// (E <- E - dt/eps0 J in place; the run's per-node tables are staged in shared
// memory, the next row is loaded while the current one is updated), then E,
// the source and the Mur ends on its range, and the cluster synchronises again.  The H and E
// loops move 4-node quads (16-byte copies and stores: run arrays are aligned and
// padded, CTA ranges start on a multiple of 4 nodes), staged in shared memory by
// cp.async in three buffers, so two rounds' loads are in flight while a round is
// computed; the +-1 neighbour is the staged buffer's next or previous value;
// partial quads, the source node and the Mur ends are stored node by node.
// Clusters never wait for each other.  Cuts never separate node 0 from node 1 or node nz-1 from node nz,
// so the thread that advances E_1 (E_{nz-1}) also applies the Mur update to
// E_0 (E_nz) with values it owns.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "async.cuh"
#include "kinetic_row.cuh"

namespace cg = cooperative_groups;

namespace fp {

constexpr int kBatchThreads = 256;

struct BRun {
    int64_t e_off, h_off, row_off;    // offsets into E_all, H_all and the slot arrays
    int32_t nz, src_k;                // src_k < 0: no source
    int32_t mur, src_kind;
    double mur_m;                     // (c dt - dz) / (c dt + dz)
    double amp, fc, tau, t0;
};

struct BSeg {
    int32_t run, k0, k1;              // E nodes [k0, k1) of the run
    int32_t s0, s1;                   // the run's plasma slots whose node is in [k0, k1)
};

template <typename T>
struct BatchArgs {
    T *E, *H, *mur;
    void *df;
    T *jslot;
    const T *dens;
    const int32_t *slot_node;         // run-local E node of every (global) slot
    const T *tab;                     // per run: alpha[pitch] beta[pitch]
    const T *tab_w;                   // w' = -e w, shared by all runs
    const BRun *runs;
    const BSeg *segs;
    const int32_t *cta_seg0;          // segments of CTA g: [cta_seg0[g], cta_seg0[g+1])
    int pitch;
    T ch, ce, cj;
    double dt;
    uint64_t seed;
    const int64_t *d_step;
    int nsteps;
};

__device__ __forceinline__ double batch_source(const BRun &r, double t)
{
    const double u = (t - r.t0) / r.tau;
    if (r.src_kind == FDTD_SRC_GAUSS_SINE) return r.amp * sin(6.283185307179586 * r.fc * (t - r.t0)) * exp(-u * u);
    if (r.src_kind == FDTD_SRC_GAUSS) return r.amp * exp(-u * u);
    return 0.0;
}

// four consecutive field nodes moved as 16-byte units (the run arrays start on 16-byte boundaries)
template <typename T>
struct Quad {
    T v[4];
};

template <typename T>
__device__ __forceinline__ Quad<T> ld_quad(const T *p)
{
    Quad<T> q;
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        q.v[0] = x.x; q.v[1] = x.y; q.v[2] = x.z; q.v[3] = x.w;
    } else {
        const double2 x = reinterpret_cast<const double2 *>(p)[0], y = reinterpret_cast<const double2 *>(p)[1];
        q.v[0] = x.x; q.v[1] = x.y; q.v[2] = y.x; q.v[3] = y.y;
    }
    return q;
}

template <typename T>
__device__ __forceinline__ void st_quad(T *p, const Quad<T> &q)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(q.v[0], q.v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(q.v[2], q.v[3]);
    }
}

// The field phases stage their quads in shared memory, kBatchBufs rounds deep: a round's E and H quads are
// copied by cp.async (16-byte copies through L2, so values other CTAs of the cluster stored before the last
// cluster barrier are the ones read) while the rounds before it are computed, so a thread's loads no longer
// wait one memory latency per round.  Each buffer holds RN nodes of a round at index 4.. and a quad of halo
// on either side.
constexpr int kBatchU = 2;                                    // quads per thread per round
constexpr int kBatchRoundNodes = 4 * kBatchU * kBatchThreads; // RN
constexpr int kBatchStage = kBatchRoundNodes + 8;             // one buffer, in values
constexpr int kBatchBufs = 3;                                 // buffers per field (two rounds in flight)

template <typename T>
__device__ __forceinline__ void cp_quad(T *dst, const T *src)
{
#pragma unroll
    for (int b = 0; b < (int)(4 * sizeof(T)) / 16; ++b)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst + b * 16 / (int)sizeof(T))),
                     "l"(src + b * 16 / (int)sizeof(T))
                     : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n (0..2) of this thread's newest copy groups are pending
__device__ __forceinline__ void cp_wait(int n)
{
    if (n >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// dynamic shared memory of the kernel: w' and the segment's alpha / beta tables, then the field stages
template <typename T>
__host__ __device__ constexpr size_t batch_tab_bytes(int pitch)
{
    return ((3 * (size_t)pitch * sizeof(T)) + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ constexpr size_t batch_smem_bytes(int pitch)
{
    return batch_tab_bytes<T>(pitch) + 2 * kBatchBufs * (size_t)kBatchStage * sizeof(T);
}

// CTAs per SM the registers are budgeted for: three with FP32 rows (80 registers, no spill: 0.316 -> 0.288 ms a
// step on the 256-run workload), two otherwise (BF16 rows lost at three: 0.189 -> 0.213 ms, the packing then
// taking clusters of eight)
template <typename TS>
constexpr int batch_min_blocks()
{
    return std::is_same<TS, float>::value ? 3 : 2;
}

template <typename TS, typename T, int VPL, int L>
__global__ void __launch_bounds__(kBatchThreads, batch_min_blocks<TS>()) k_batch1d(BatchArgs<T> a)
{
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_w = reinterpret_cast<T *>(smem_raw);    // w' (shared by all runs), then alpha, beta tables
    T *s_tabs = s_w + a.pitch;
    using V = typename Vec<TS>::type;
    constexpr int VEC = Vec<TS>::n;
    constexpr int R = 32 / L;
    constexpr int U = kBatchU;                   // H / E quads (4 nodes each) per thread per round
    // field stages: E buffers [kBatchBufs], then H buffers [kBatchBufs]
    T *stage_base = reinterpret_cast<T *>(smem_raw + batch_tab_bytes<T>(a.pitch));
    auto fe = [&](int b) { return stage_base + b * kBatchStage; };
    auto fh = [&](int b) { return stage_base + (kBatchBufs + b) * kBatchStage; };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / L, l = lane % L;
    const int nwarps = blockDim.x >> 5;
    const int seg0 = a.cta_seg0[blockIdx.x], seg1 = a.cta_seg0[blockIdx.x + 1];
    const int64_t step0 = *a.d_step;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    for (int t = threadIdx.x; t < a.pitch; t += blockDim.x) s_w[t] = a.tab_w[t];

    for (int s = 0; s < a.nsteps; ++s) {
        const int64_t step = step0 + s;
        // ---- H^{n+1/2} on this CTA's nodes; save E_1^n, E_{nz-1}^n for Mur
        for (int q = seg0; q < seg1; ++q) {
            const BSeg sg = a.segs[q];
            const BRun r = a.runs[sg.run];
            const T *E = a.E + r.e_off;
            T *H = a.H + r.h_off;
            const int kend = min(sg.k1, r.nz);
            const int nq = (kend - sg.k0 + 3) / 4;   // quads of H nodes [k0, kend); k0 is a multiple of 4
            const int rq = U * (int)blockDim.x;       // quads per round (block-uniform rounds)
            const int nr = (nq + rq - 1) / rq;
            // round ri into buffer b: H quads starting below kend, E quads starting at or below kend (E at
            // kend is the last node's upper neighbour), and the E quad just past the round
            auto stage = [&](int ri, int b) {
                const int kr = sg.k0 + 4 * rq * ri;
                T *se = fe(b) + 4, *sh = fh(b) + 4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = 4 * (u * (int)blockDim.x + (int)threadIdx.x);
                    if (kr + j <= kend) cp_quad(se + j, E + kr + j);
                    if (kr + j < kend) cp_quad(sh + j, H + kr + j);
                }
                if (threadIdx.x == 0 && kr + 4 * rq <= kend) cp_quad(se + 4 * rq, E + kr + 4 * rq);
                cp_commit();
            };
            for (int ri = 0; ri < kBatchBufs - 1 && ri < nr; ++ri) stage(ri, ri);
            for (int ri = 0; ri < nr; ++ri) {
                if (ri + kBatchBufs - 1 < nr) stage(ri + kBatchBufs - 1, (ri + kBatchBufs - 1) % kBatchBufs);
                cp_wait(min(kBatchBufs - 1, nr - 1 - ri));   // the copies of quad batch ri have landed
                __syncthreads();
                const int kr = sg.k0 + 4 * rq * ri;
                const T *se = fe(ri % kBatchBufs) + 4, *sh = fh(ri % kBatchBufs) + 4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = 4 * (u * (int)blockDim.x + (int)threadIdx.x);
                    const int kq = kr + j;
                    if (kq >= kend) continue;
                    Quad<T> o;
#pragma unroll
                    for (int c = 0; c < 4; ++c) o.v[c] = sh[j + c] - a.ch * (se[j + c + 1] - se[j + c]);
                    if (kq + 4 <= kend) {
                        st_quad(H + kq, o);
                    } else {
                        for (int c = 0; kq + c < kend; ++c) H[kq + c] = o.v[c];
                    }
                }
                __syncthreads();   // buffer ri % kBatchBufs is staged again kBatchBufs - 1 rounds on
            }
            if (r.mur && threadIdx.x == 0) {
                if (sg.k0 <= 1 && 1 < sg.k1) a.mur[2 * sg.run] = E[1];
                if (sg.k0 <= r.nz - 1 && r.nz - 1 < sg.k1) a.mur[2 * sg.run + 1] = E[r.nz - 1];
            }
        }
        cluster.sync();
        // ---- delta-f rows of this CTA's plasma nodes; E <- E - dt/eps0 J
        for (int q = seg0; q < seg1; ++q) {
            const BSeg sg = a.segs[q];
            if (sg.s1 <= sg.s0) continue;
            const BRun r = a.runs[sg.run];
            T *E = a.E + r.e_off;
            const T *al = a.tab + (int64_t)sg.run * 2 * a.pitch;
            __syncthreads();                           // previous segment's tables no longer in use
            for (int t = threadIdx.x; t < 2 * a.pitch; t += blockDim.x) s_tabs[t] = al[t];
            __syncthreads();
            const T *s_al = s_tabs, *s_be = s_tabs + a.pitch;
            // software pipeline: the next row's node index, delta-f vectors, E and
            // density are loaded before the current row is updated, so a lane
            // keeps two rows of loads in flight (128 registers a thread, two
            // 256-thread CTAs per SM).  Rows of a segment have distinct nodes, so
            // reading the next row's E ahead of this row's E store is safe.
            const int stride = nwarps * R;
            struct RowIn {
                V v[VPL];
                T e, dn;
                int node;
                int64_t grow;
                bool valid;
            };
            auto fetch_row = [&](int row, RowIn &in) {
                in.valid = row < sg.s1;
                in.grow = r.row_off + (in.valid ? row : sg.s0);
                in.e = T(0);
                in.dn = T(0);
                in.node = 0;
                if (in.valid) {
                    const V *rp = reinterpret_cast<const V *>(a.df) + in.grow * (a.pitch / VEC);
#pragma unroll
                    for (int qq = 0; qq < VPL; ++qq) in.v[qq] = __ldcs(rp + qq * L + l);
                    in.node = __ldg(a.slot_node + in.grow);
                    in.e = E[in.node];
                    in.dn = __ldg(a.dens + in.grow);
                }
            };
            RowIn cur, nxt;
            fetch_row(sg.s0 + warp * R + sub, cur);
            for (int base = sg.s0 + warp * R; base < sg.s1; base += stride) {
                fetch_row(base + stride + sub, nxt);
                V *rp = reinterpret_cast<V *>(a.df) + cur.grow * (a.pitch / VEC);
                T sm = T(0), cm = T(0);
                if (cur.valid)
                    row_update<TS, T, VPL, L>(rp, cur.v, s_al, s_be, s_w, cur.dn * cur.e, l, (uint32_t)cur.grow, step,
                                              key, sm, cm);
                const T J = row_reduce<T, L>(sm, cm);
                if (cur.valid && l == 0) {
                    if (s == a.nsteps - 1) a.jslot[cur.grow] = J;   // J is read between launches only
                    E[cur.node] = cur.e - a.cj * J;
                }
                cur = nxt;
            }
        }
        __syncthreads();
        // ---- E^{n+1} on this CTA's interior nodes, soft source, Mur ends
        for (int q = seg0; q < seg1; ++q) {
            const BSeg sg = a.segs[q];
            const BRun r = a.runs[sg.run];
            T *E = a.E + r.e_off;
            const T *H = a.H + r.h_off;
            const int kbeg = max(sg.k0, 1), kend = min(sg.k1, r.nz);   // E nodes updated: [kbeg, kend)
            const int nq = (kend - sg.k0 + 3) / 4;
            const int rq = U * (int)blockDim.x;
            const int nr = (nq + rq - 1) / rq;
            // round ri into buffer b: E and H quads starting below kend, and the H quad just before the
            // round (zero before node 0)
            auto stage = [&](int ri, int b) {
                const int kr = sg.k0 + 4 * rq * ri;
                T *se = fe(b) + 4, *sh = fh(b) + 4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = 4 * (u * (int)blockDim.x + (int)threadIdx.x);
                    if (kr + j < kend) {
                        cp_quad(se + j, E + kr + j);
                        cp_quad(sh + j, H + kr + j);
                    }
                }
                if (threadIdx.x == 0) {
                    if (kr > 0) cp_quad(sh - 4, H + kr - 4);
                    else sh[-1] = T(0);
                }
                cp_commit();
            };
            for (int ri = 0; ri < kBatchBufs - 1 && ri < nr; ++ri) stage(ri, ri);
            for (int ri = 0; ri < nr; ++ri) {
                if (ri + kBatchBufs - 1 < nr) stage(ri + kBatchBufs - 1, (ri + kBatchBufs - 1) % kBatchBufs);
                cp_wait(min(kBatchBufs - 1, nr - 1 - ri));   // the copies of quad batch ri have landed
                __syncthreads();
                const int kr = sg.k0 + 4 * rq * ri;
                const T *se = fe(ri % kBatchBufs) + 4, *sh = fh(ri % kBatchBufs) + 4;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = 4 * (u * (int)blockDim.x + (int)threadIdx.x);
                    const int kq = kr + j;
                    if (kq >= kend) continue;
                    Quad<T> o;
#pragma unroll
                    for (int c = 0; c < 4; ++c) o.v[c] = se[j + c] - a.ce * (sh[j + c] - sh[j + c - 1]);
                    const bool special = kq < kbeg || kq + 4 > kend || (r.src_k >= kq && r.src_k < kq + 4) ||
                                         (r.mur && (kq <= 1 || kq + 4 > r.nz - 1));
                    if (!special) {
                        st_quad(E + kq, o);
                        continue;
                    }
                    for (int c = 0; c < 4; ++c) {
                        const int k = kq + c;
                        if (k < kbeg || k >= kend) continue;
                        T v = o.v[c];
                        if (k == r.src_k) v += (T)batch_source(r, (double)(step + 1) * a.dt);
                        E[k] = v;
                        if (r.mur) {
                            if (k == 1) E[0] = a.mur[2 * sg.run] + (T)r.mur_m * (v - E[0]);
                            if (k == r.nz - 1) E[r.nz] = a.mur[2 * sg.run + 1] + (T)r.mur_m * (v - E[r.nz]);
                        }
                    }
                }
                __syncthreads();   // buffer ri % kBatchBufs is staged again kBatchBufs - 1 rounds on
            }
        }
        cluster.sync();
    }
}

__global__ void k_batch_advance(int64_t *d_step, int64_t by) { *d_step += by; }

}  // namespace fp

// ================================================================= host side

using namespace fp;

namespace {

thread_local std::string g_batch_create_error;

}  // namespace

struct fdtd_batch {
    fdtd_runtime_desc rt;
    cudaStream_t stream, cap;
    int precision, f_dtype, nruns, pitch, nnode, nclusters, cluster_ctas;
    uint64_t seed;
    size_t esz, df_esz;
    double dt, dx;
    std::vector<int64_t> nz, e_off, h_off, row_off, nslot;
    int64_t ncell_e, ncell_h, nrows;
    void *E, *H, *mur, *df, *jslot, *dens, *slot_node, *tab, *runs, *segs, *cta_seg0;
    int64_t *d_step;
    int64_t steps_done;
    std::map<int64_t, cudaGraphExec_t> graphs;
    std::string err;
    cudaError_t (*launch)(fdtd_batch *, cudaStream_t, int);
    // row-shape candidates (vectors per lane, lanes per row) for this row length; [0] is the default
    struct Shape {
        int vpl, l;
        cudaError_t (*launch)(fdtd_batch *, cudaStream_t, int);
    };
    std::vector<Shape> shapes;
    int shape;
};

namespace {

int bfail(fdtd_batch *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf; else g_batch_create_error = buf;
    return code;
}

void *balloc(fdtd_batch *b, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (b->rt.alloc) p = b->rt.alloc(bytes, b->rt.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
    return p;
}

void bfree(fdtd_batch *b, void *p)
{
    if (!p) return;
    if (b->rt.free) b->rt.free(p, b->rt.alloc_ctx);
    else cudaFree(p);
}

template <typename TS, typename T, int VPL, int L>
cudaError_t launch_t(fdtd_batch *b, cudaStream_t st, int nsteps)
{
    BatchArgs<T> a{};
    a.E = (T *)b->E; a.H = (T *)b->H; a.mur = (T *)b->mur;
    a.df = b->df; a.jslot = (T *)b->jslot; a.dens = (const T *)b->dens; a.slot_node = (const int32_t *)b->slot_node;
    a.tab = (const T *)b->tab + b->pitch;   // per-run tables follow the shared w'
    a.tab_w = (const T *)b->tab;
    a.runs = (const BRun *)b->runs; a.segs = (const BSeg *)b->segs; a.cta_seg0 = (const int32_t *)b->cta_seg0;
    a.pitch = b->pitch;
    const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
    a.ch = (T)(b->dt / (mu0 * b->dx));
    a.ce = (T)(b->dt / (kEps0 * b->dx));
    a.cj = (T)(b->dt / kEps0);
    a.dt = b->dt;
    a.seed = b->seed;
    a.d_step = b->d_step;
    a.nsteps = nsteps;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->nclusters * b->cluster_ctas);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = batch_smem_bytes<T>(b->pitch);
    if (cfg.dynamicSmemBytes > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_batch1d<TS, T, VPL, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
    }
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = b->cluster_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch1d<TS, T, VPL, L>, a);
    if (e != cudaSuccess) return e;
    k_batch_advance<<<1, 1, 0, st>>>(b->d_step, nsteps);
    return cudaGetLastError();
}

// clusters of `ctas` CTAs that can be resident at once (0: none fits)
template <typename TS, typename T, int VPL, int L>
int max_clusters(int ctas)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kBatchThreads);
    // tables of the largest row (128 vectors of 16 bytes) and the field stages
    cfg.dynamicSmemBytes = 3 * 128 * 16 + 2 * kBatchBufs * (size_t)kBatchStage * sizeof(T);
    if (cfg.dynamicSmemBytes > 48 * 1024 &&
        cudaFuncSetAttribute(k_batch1d<TS, T, VPL, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cfg.dynamicSmemBytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_batch1d<TS, T, VPL, L>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n;
}

// Row-shape candidates (storage, precision, vectors per row): the first is the built-in choice and
// fixes the cluster packing; fdtd_batch_autotune may switch to another (two vectors a lane, twice the
// lanes: eight vectors a lane spill at the kernel's 128 registers).  The FP64 validation instantiation
// keeps the built-in shape only.
template <typename TS, typename T, int VPL, int L>
fdtd_batch::Shape shape_of()
{
    return fdtd_batch::Shape{VPL, L, launch_t<TS, T, VPL, L>};
}

template <typename TS, typename T>
bool pick(int V, std::vector<fdtd_batch::Shape> &sh, int (**maxc)(int))
{
    sh.clear();
    constexpr bool more = !std::is_same<T, double>::value;
    switch (V) {
    case 1: sh = {shape_of<TS, T, 1, 1>()}; *maxc = max_clusters<TS, T, 1, 1>; break;
    case 2:
        sh = {shape_of<TS, T, 2, 1>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 1, 2>());
        *maxc = max_clusters<TS, T, 2, 1>;
        break;
    case 4:
        sh = {shape_of<TS, T, 4, 1>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 2, 2>());
        *maxc = max_clusters<TS, T, 4, 1>;
        break;
    case 8:
        sh = {shape_of<TS, T, 4, 2>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 2, 4>());
        *maxc = max_clusters<TS, T, 4, 2>;
        break;
    case 16:
        sh = {shape_of<TS, T, 4, 4>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 2, 8>());
        *maxc = max_clusters<TS, T, 4, 4>;
        break;
    case 32:
        sh = {shape_of<TS, T, 4, 8>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 2, 16>());
        *maxc = max_clusters<TS, T, 4, 8>;
        break;
    case 64:
        sh = {shape_of<TS, T, 4, 16>()};
        if constexpr (more) sh.push_back(shape_of<TS, T, 2, 32>());
        *maxc = max_clusters<TS, T, 4, 16>;
        break;
    case 128:
        sh = {shape_of<TS, T, 4, 32>()};
        *maxc = max_clusters<TS, T, 4, 32>;
        break;
    default: return false;
    }
    return true;
}

void destroy_batch(fdtd_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    void *ps[] = {b->E, b->H, b->mur, b->df, b->jslot, b->dens, b->slot_node, b->tab, b->runs, b->segs, b->cta_seg0,
                  b->d_step};
    for (void *p : ps) bfree(b, p);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // namespace

extern "C" {

int fdtd_batch_create(const fdtd_run_desc *runs, int32_t nruns, const fdtd_runtime_desc *rt, fdtd_batch_t *out)
{
    if (!out) return bfail(nullptr, FDTD_ERR_INVAL, "out is NULL");
    *out = nullptr;
    if (!runs || nruns < 1) return bfail(nullptr, FDTD_ERR_INVAL, "need at least one run");
    const fdtd_grid_desc &g0 = runs[0].grid;
    const fdtd_plasma_desc &p0 = runs[0].plasma;
    for (int r = 0; r < nruns; ++r) {
        const fdtd_grid_desc &g = runs[r].grid;
        const fdtd_plasma_desc &p = runs[r].plasma;
        if (g.ndim != 1) return bfail(nullptr, FDTD_ERR_INVAL, "run %d: batches are 1-D", r);
        if (g.dx != g0.dx || g.courant != g0.courant || g.precision != g0.precision)
            return bfail(nullptr, FDTD_ERR_INVAL, "run %d: dx, courant and precision must match run 0", r);
        if (g.nz < 3 || g.nz > (1 << 30)) return bfail(nullptr, FDTD_ERR_INVAL, "run %d: nz out of range", r);
        if (g.cpml_cells) return bfail(nullptr, FDTD_ERR_INVAL, "run %d: 1-D runs use Mur or PEC ends", r);
        if (p.vgrid != p0.vgrid || p.nv != p0.nv || p.nv_perp != p0.nv_perp || p.te_ev != p0.te_ev ||
            p.vmax_vth != p0.vmax_vth || p.nu_model != p0.nu_model || p.f_dtype != p0.f_dtype ||
            p.f0_model != p0.f0_model)
            return bfail(nullptr, FDTD_ERR_INVAL,
                         "run %d: velocity grid, te, F0 and nu models and f_dtype must match run 0", r);
        if (const char *why = check_velocity_model(p)) return bfail(nullptr, FDTD_ERR_INVAL, "run %d: %s", r, why);
        if (p.nu_model == FDTD_NU_TABLE &&
            (p.s_n != p0.s_n || !std::equal(p.s_speed, p.s_speed + p.s_n, p0.s_speed) ||
             !std::equal(p.s_sigma, p.s_sigma + p.s_n, p0.s_sigma)))
            return bfail(nullptr, FDTD_ERR_INVAL, "run %d: the s(v) table must match run 0", r);
        if (p.nonlinear || p.evolve_f0)
            return bfail(nullptr, FDTD_ERR_INVAL, "run %d: nonlinear / evolving-F0 modes not available in batches", r);
        if (!(p.nu0 >= 0) || !std::isfinite(p.nu0)) return bfail(nullptr, FDTD_ERR_INVAL, "run %d: nu0", r);
        const fdtd_source_desc &s = runs[r].source;
        if (s.kind && (s.k < 1 || s.k > g.nz - 1 || !(s.tau > 0)))
            return bfail(nullptr, FDTD_ERR_INVAL, "run %d: source node must be in [1, nz-1] and tau > 0", r);
    }
    if (!(g0.dx > 0) || !(g0.courant > 0) || g0.courant >= 1.0)
        return bfail(nullptr, FDTD_ERR_UNSTABLE, "courant must be in (0, 1) in 1-D");
    const bool f64 = g0.precision == FDTD_F64;
    if (f64 ? p0.f_dtype != FDTD_DF_F64 : (p0.f_dtype != FDTD_DF_F32 && p0.f_dtype != FDTD_DF_BF16))
        return bfail(nullptr, FDTD_ERR_INVAL, "f_dtype does not match the field precision");

    fdtd_batch *b = new (std::nothrow) fdtd_batch();
    if (!b) return bfail(nullptr, FDTD_ERR_NOMEM, "host allocation failed");
    if (rt) b->rt = *rt;
    b->stream = (cudaStream_t)b->rt.stream;
    auto bail = [&](int code, const char *msg) {
        g_batch_create_error = msg;
        destroy_batch(b);
        return code;
    };
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(FDTD_ERR_CUDA, "stream creation failed");
    b->precision = g0.precision;
    b->seed = p0.seed;
    b->f_dtype = p0.f_dtype;
    b->nruns = nruns;
    b->esz = f64 ? 8 : 4;
    b->df_esz = p0.f_dtype == FDTD_DF_BF16 ? 2 : (p0.f_dtype == FDTD_DF_F64 ? 8 : 4);
    b->dx = g0.dx;
    b->dt = g0.courant * g0.dx / kC0;
    const int nnode = p0.vgrid == FDTD_VGRID_CART2D ? p0.nv * p0.nv_perp : p0.nv;
    b->nnode = nnode;
    b->pitch = kinetic_pitch(nnode, p0.f_dtype);
    const int vec = p0.f_dtype == FDTD_DF_BF16 ? 8 : (p0.f_dtype == FDTD_DF_F64 ? 2 : 4);
    const int V = b->pitch / vec;
    int (*maxc_of)(int) = nullptr;
    bool ok = p0.f_dtype == FDTD_DF_F32    ? pick<float, float>(V, b->shapes, &maxc_of)
              : p0.f_dtype == FDTD_DF_BF16 ? pick<__nv_bfloat16, float>(V, b->shapes, &maxc_of)
                                           : pick<double, double>(V, b->shapes, &maxc_of);
    if (!ok) return bail(FDTD_ERR_INVAL, "too many velocity nodes for the batched kernel (at most 128 vectors)");
    b->shape = 0;
    b->launch = b->shapes[0].launch;
    int maxc_c[4];
    const int csizes[4] = {8, 4, 2, 1};
    bool any = false;
    for (int i = 0; i < 4; ++i) {
        maxc_c[i] = maxc_of(csizes[i]);
        any = any || maxc_c[i] > 0;
    }
    if (!any) return bail(FDTD_ERR_CUDA, "no cluster of the batched kernel fits on this device");

    // ---- velocity tables (shared node weights; per-run alpha, beta from nu0_r)
    VTab vt;
    if (!velocity_tables(p0, vt)) return bail(FDTD_ERR_INVAL, "bad velocity grid");
    const std::vector<double> &w = vt.w, &f0p = vt.f0p;
    const int P = b->pitch;
    std::vector<double> tab((size_t)P * (1 + 2 * (size_t)nruns), 0.0);
    for (int j = 0; j < nnode; ++j) tab[j] = -kQe * w[j];
    double wpmax = 0;
    // ---- per-run layout and slots
    std::vector<BRun> hr(nruns);
    std::vector<int32_t> slot_node;
    std::vector<double> dens_slot;
    b->nz.resize(nruns); b->e_off.resize(nruns); b->h_off.resize(nruns); b->row_off.resize(nruns); b->nslot.resize(nruns);
    int64_t eo = 0, ho = 0, ro = 0;
    std::vector<std::vector<double>> dens_run(nruns);
    for (int r = 0; r < nruns; ++r) {
        const fdtd_grid_desc &g = runs[r].grid;
        const fdtd_plasma_desc &p = runs[r].plasma;
        const int64_t nz = g.nz;
        b->nz[r] = nz; b->e_off[r] = eo; b->h_off[r] = ho; b->row_off[r] = ro;
        std::vector<double> d(nz + 1, 0.0);
        if (p.density) {
            if (p.density_on_device) {
                if (cudaMemcpy(d.data(), p.density, (nz + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return bail(FDTD_ERR_CUDA, "density copy failed");
            } else {
                std::memcpy(d.data(), p.density, (nz + 1) * 8);
            }
        }
        int64_t ns = 0;
        for (int64_t k = 0; k <= nz; ++k) {
            if (!std::isfinite(d[k]) || d[k] < 0) return bail(FDTD_ERR_NONFINITE, "density must be finite and >= 0");
            if (d[k] > 0 && k >= 1 && k <= nz - 1) {
                slot_node.push_back((int32_t)k);
                dens_slot.push_back(d[k]);
                wpmax = std::max(wpmax, d[k]);
                ++ns;
            }
        }
        b->nslot[r] = ns;
        const double nu0 = p.nu0;
        for (int j = 0; j < nnode; ++j) {
            const double nu = node_nu(p, vt, (size_t)j, nu0);
            tab[(size_t)P * (1 + 2 * r) + j] = (2 - b->dt * nu) / (2 + b->dt * nu);
            tab[(size_t)P * (2 + 2 * r) + j] = 2 * b->dt * (kQe / kMe) * f0p[j] / (2 + b->dt * nu);
        }
        BRun &br = hr[r];
        br.e_off = eo; br.h_off = ho; br.row_off = ro;
        br.nz = (int32_t)nz;
        br.mur = g.mur ? 1 : 0;
        br.mur_m = (kC0 * b->dt - g.dx) / (kC0 * b->dt + g.dx);
        const fdtd_source_desc &s = runs[r].source;
        br.src_kind = s.kind;
        br.src_k = s.kind ? (int32_t)s.k : -1;
        br.amp = s.amp; br.fc = s.fc; br.tau = s.kind ? s.tau : 1.0; br.t0 = s.t0;
        // 16-byte aligned run arrays, padded so a 4-node quad read never leaves the run's extent
        eo += (nz + 1 + 3) / 4 * 4 + 4;
        ho += (nz + 3) / 4 * 4 + 4;
        ro += ns;
    }
    b->ncell_e = eo; b->ncell_h = ho; b->nrows = ro;
    const double wp = std::sqrt(wpmax * kQe * kQe / (kEps0 * kMe));
    if (std::pow(wp * b->dt / 2, 2) + g0.courant * g0.courant >= 1.0)
        return bail(FDTD_ERR_UNSTABLE, "plasma frequency too high for dt");

    // ---- bin packing: runs -> clusters (LPT), then equal-cost CTA ranges.  Every cluster size
    // that fits is packed; the one with the smallest largest per-CTA load (bin load / cluster
    // size) is kept, larger clusters winning ties.
    const double cell_cost = 4.0 * b->esz, node_cost = 2.0 * nnode * b->df_esz + 20.0;
    std::vector<double> cost(nruns);
    for (int r = 0; r < nruns; ++r) cost[r] = cell_cost * (b->nz[r] + 1) + node_cost * b->nslot[r];
    std::vector<int> order(nruns);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    auto pack = [&](int nb, std::vector<std::vector<int>> &bins, std::vector<double> &load) {
        bins.assign(nb, {});
        load.assign(nb, 0.0);
        for (int r : order) {
            int bi = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            bins[bi].push_back(r);
            load[bi] += cost[r];
        }
        return *std::max_element(load.begin(), load.end());
    };
    std::vector<std::vector<int>> bins;
    std::vector<double> load;
    double best = 0.0;
    int nb = 0, csize = 0;
    for (int i = 0; i < 4; ++i) {
        if (maxc_c[i] < 1) continue;
        const int n = std::max(1, std::min(maxc_c[i], nruns));
        std::vector<std::vector<int>> bb;
        std::vector<double> ll;
        const double span = pack(n, bb, ll) / csizes[i];
        if (csize == 0 || span < best * (1.0 - 1e-9)) {
            best = span;
            nb = n;
            csize = csizes[i];
            bins.swap(bb);
            load.swap(ll);
        }
    }
    b->nclusters = nb;
    b->cluster_ctas = csize;
    std::vector<BSeg> segs;
    std::vector<int32_t> cta_seg0;
    // slot index (run-local) of the first slot at node >= k
    std::vector<std::vector<int32_t>> slot_at(nruns);
    for (int r = 0; r < nruns; ++r) {
        slot_at[r].assign(b->nz[r] + 2, 0);
        const int32_t *nodes = slot_node.data() + b->row_off[r];
        int64_t si = 0;
        for (int64_t k = 0; k <= b->nz[r] + 1; ++k) {
            while (si < b->nslot[r] && nodes[si] < k) ++si;
            slot_at[r][k] = (int32_t)si;
        }
    }
    for (int bi = 0; bi < nb; ++bi) {
        // per-node cost along the bin's concatenated nodes, cut into csize ranges
        const double total = load[bi];
        double acc = 0;
        int cta = 0;
        cta_seg0.push_back((int32_t)segs.size());
        for (int r : bins[bi]) {
            const int64_t nz = b->nz[r];
            int64_t k0 = 0;
            const int32_t *nodes = slot_node.data() + b->row_off[r];
            int64_t si = 0;
            for (int64_t k = 0; k <= nz; ++k) {
                while (si < b->nslot[r] && nodes[si] < k) ++si;
                const bool plasma = si < b->nslot[r] && nodes[si] == k;
                acc += cell_cost + (plasma ? node_cost : 0.0);
                const double target = total * (cta + 1) / csize;
                // a cut after node k (range [k0, k+1)) at a multiple of 4 nodes (ranges start on a quad);
                // never between 0|1 or nz-1|nz
                const int64_t cut = k + 1;
                if (acc >= target && cta < csize - 1 && cut % 4 == 0 && cut != nz && cut <= nz) {
                    segs.push_back(BSeg{r, (int32_t)k0, (int32_t)cut, slot_at[r][k0], slot_at[r][cut]});
                    k0 = cut;
                    ++cta;
                    cta_seg0.push_back((int32_t)segs.size());
                }
            }
            if (k0 <= nz) segs.push_back(BSeg{r, (int32_t)k0, (int32_t)(nz + 1), slot_at[r][k0], slot_at[r][nz + 1]});
        }
        while (cta < csize - 1) {   // CTAs left without nodes
            ++cta;
            cta_seg0.push_back((int32_t)segs.size());
        }
    }
    cta_seg0.push_back((int32_t)segs.size());

    // ---- device buffers
    const int64_t nrow = std::max<int64_t>(b->nrows, 1);
    b->E = balloc(b, eo * b->esz);
    b->H = balloc(b, ho * b->esz);
    b->mur = balloc(b, 2 * (size_t)nruns * b->esz);
    b->df = balloc(b, (size_t)nrow * P * b->df_esz);
    b->jslot = balloc(b, (size_t)nrow * b->esz);
    b->dens = balloc(b, (size_t)nrow * b->esz);
    b->slot_node = balloc(b, (size_t)nrow * 4);
    b->tab = balloc(b, tab.size() * b->esz);
    b->runs = balloc(b, hr.size() * sizeof(BRun));
    b->segs = balloc(b, std::max<size_t>(segs.size(), 1) * sizeof(BSeg));
    b->cta_seg0 = balloc(b, cta_seg0.size() * 4);
    b->d_step = (int64_t *)balloc(b, 256);
    if (!b->E || !b->H || !b->mur || !b->df || !b->jslot || !b->dens || !b->slot_node || !b->tab || !b->runs ||
        !b->segs || !b->cta_seg0 || !b->d_step)
        return bail(FDTD_ERR_NOMEM, "batch allocation failed");
    bool up = true;
    auto H2D = [&](void *dst, const void *src, size_t n) {
        if (n && cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) != cudaSuccess) up = false;
    };
    if (b->esz == 8) {
        H2D(b->tab, tab.data(), tab.size() * 8);
        H2D(b->dens, dens_slot.data(), dens_slot.size() * 8);
    } else {
        std::vector<float> t32(tab.begin(), tab.end()), d32(dens_slot.begin(), dens_slot.end());
        H2D(b->tab, t32.data(), t32.size() * 4);
        H2D(b->dens, d32.data(), d32.size() * 4);
    }
    H2D(b->slot_node, slot_node.data(), slot_node.size() * 4);
    H2D(b->runs, hr.data(), hr.size() * sizeof(BRun));
    H2D(b->segs, segs.data(), segs.size() * sizeof(BSeg));
    H2D(b->cta_seg0, cta_seg0.data(), cta_seg0.size() * 4);
    if (!up) return bail(FDTD_ERR_CUDA, "batch upload failed");
    if (cudaMemset(b->E, 0, eo * b->esz) != cudaSuccess || cudaMemset(b->H, 0, ho * b->esz) != cudaSuccess ||
        cudaMemset(b->mur, 0, 2 * (size_t)nruns * b->esz) != cudaSuccess ||
        cudaMemset(b->df, 0, (size_t)nrow * P * b->df_esz) != cudaSuccess ||
        cudaMemset(b->jslot, 0, (size_t)nrow * b->esz) != cudaSuccess || cudaMemset(b->d_step, 0, 8) != cudaSuccess)
        return bail(FDTD_ERR_CUDA, "batch clear failed");
    *out = b;
    return FDTD_OK;
}

int fdtd_batch_step(fdtd_batch_t b, int64_t nsteps)
{
    if (!b) return FDTD_ERR_INVAL;
    if (nsteps < 0) return bfail(b, FDTD_ERR_INVAL, "nsteps < 0");
    int64_t left = nsteps;
    while (left > 0) {
        const int64_t n = std::min<int64_t>(left, 1 << 20);
        auto it = b->graphs.find(n);
        if (it == b->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
            if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
            cudaError_t el = b->launch(b, b->cap, (int)n);
            e = cudaStreamEndCapture(b->cap, &graph);
            if (el != cudaSuccess || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return bfail(b, FDTD_ERR_CUDA, "capturing the batched launch: %s",
                             cudaGetErrorString(el != cudaSuccess ? el : e));
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
            it = b->graphs.emplace(n, exec).first;
        }
        cudaError_t e = cudaGraphLaunch(it->second, b->stream);
        if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
        left -= n;
    }
    b->steps_done += nsteps;
    return FDTD_OK;
}

size_t fdtd_batch_quantity_bytes(fdtd_batch_t b, int32_t run, int which)
{
    if (!b || run < 0 || run >= b->nruns) return 0;
    switch (which) {
    case FDTD_EX: return (size_t)(b->nz[run] + 1) * b->esz;
    case FDTD_HY: return (size_t)b->nz[run] * b->esz;
    case FDTD_J: return (size_t)b->nslot[run] * b->esz;
    case FDTD_DF: return (size_t)b->nslot[run] * b->nnode * b->df_esz;
    default: return 0;
    }
}

int fdtd_batch_read(fdtd_batch_t b, int32_t run, int which, void *dst, size_t bytes, int dst_is_device)
{
    if (!b || !dst) return FDTD_ERR_INVAL;
    const size_t need = fdtd_batch_quantity_bytes(b, run, which);
    if (need == 0) return bfail(b, FDTD_ERR_INVAL, "quantity %d of run %d is absent", which, run);
    if (bytes != need) return bfail(b, FDTD_ERR_INVAL, "needs %zu bytes, got %zu", need, bytes);
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e;
    if (which == FDTD_DF) {
        const size_t row = (size_t)b->nnode * b->df_esz, dp = (size_t)b->pitch * b->df_esz;
        e = cudaMemcpy2DAsync(dst, row, (char *)b->df + b->row_off[run] * dp, dp, row, b->nslot[run], kind,
                              b->stream);
    } else {
        const char *src = which == FDTD_EX   ? (char *)b->E + b->e_off[run] * b->esz
                          : which == FDTD_HY ? (char *)b->H + b->h_off[run] * b->esz
                                             : (char *)b->jslot + b->row_off[run] * b->esz;
        e = cudaMemcpyAsync(dst, src, bytes, kind, b->stream);
    }
    if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "read: %s", cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_batch_write(fdtd_batch_t b, int32_t run, int which, const void *src, size_t bytes, int src_is_device)
{
    if (!b || !src) return FDTD_ERR_INVAL;
    if (which != FDTD_EX && which != FDTD_HY) return bfail(b, FDTD_ERR_INVAL, "only FDTD_EX and FDTD_HY are writable");
    const size_t need = fdtd_batch_quantity_bytes(b, run, which);
    if (need == 0) return bfail(b, FDTD_ERR_INVAL, "quantity %d of run %d is absent", which, run);
    if (bytes != need) return bfail(b, FDTD_ERR_INVAL, "needs %zu bytes, got %zu", need, bytes);
    char *dst = which == FDTD_EX ? (char *)b->E + b->e_off[run] * b->esz : (char *)b->H + b->h_off[run] * b->esz;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess && !src_is_device) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "write: %s", cudaGetErrorString(e));
    return FDTD_OK;
}

int fdtd_batch_autotune(fdtd_batch_t b, int32_t *vpl, int32_t *lanes, double *ms_per_step)
{
    if (!b) return FDTD_ERR_INVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "autotune: stream");
    // save the state the timed steps change, restore it afterwards
    const int64_t nrow = std::max<int64_t>(b->nrows, 1);
    const size_t nE = b->ncell_e * b->esz, nH = b->ncell_h * b->esz, nM = 2 * (size_t)b->nruns * b->esz;
    const size_t nD = (size_t)nrow * b->pitch * b->df_esz, nJ = (size_t)nrow * b->esz, nS = 16;
    const size_t sizes[6] = {nE, nH, nM, nD, nJ, nS};
    void *live[6] = {b->E, b->H, b->mur, b->df, b->jslot, b->d_step};
    void *saved[6] = {};
    bool ok = true;
    for (int i = 0; i < 6 && ok; ++i) ok = (saved[i] = balloc(b, sizes[i])) != nullptr;
    auto release = [&]() {
        for (int i = 0; i < 6; ++i) bfree(b, saved[i]);
    };
    if (!ok) {
        release();
        return bfail(b, FDTD_ERR_NOMEM, "autotune: no room for a copy of the state");
    }
    for (int i = 0; i < 6 && ok; ++i)
        ok = cudaMemcpyAsync(saved[i], live[i], sizes[i], cudaMemcpyDeviceToDevice, b->stream) == cudaSuccess;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    constexpr int kSteps = 20;
    double best = 1e30;
    int best_i = b->shape;
    for (int c = 0; c < (int)b->shapes.size() && ok; ++c) {
        auto fn = b->shapes[c].launch;
        ok = fn(b, b->stream, 2) == cudaSuccess;   // warm-up
        ok = ok && cudaEventRecord(e0, b->stream) == cudaSuccess && fn(b, b->stream, kSteps) == cudaSuccess &&
             cudaEventRecord(e1, b->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0;
        if (ok) cudaEventElapsedTime(&ms, e0, e1);
        // a later candidate replaces the best only when more than 1 % faster
        if (ok && ms / kSteps < best * 0.99) {
            best = ms / kSteps;
            best_i = c;
        }
    }
    for (int i = 0; i < 6 && ok; ++i)
        ok = cudaMemcpyAsync(live[i], saved[i], sizes[i], cudaMemcpyDeviceToDevice, b->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(b->stream) == cudaSuccess;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    release();
    if (!ok) return bfail(b, FDTD_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
    if (best_i != b->shape) {
        for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
        b->graphs.clear();
        b->shape = best_i;
        b->launch = b->shapes[best_i].launch;
    }
    if (vpl) *vpl = b->shapes[b->shape].vpl;
    if (lanes) *lanes = b->shapes[b->shape].l;
    if (ms_per_step) *ms_per_step = best;
    return FDTD_OK;
}

int fdtd_batch_info(fdtd_batch_t b, double *dt, int64_t *steps, int64_t *cells, int64_t *nodes, int32_t *nclusters,
                    int32_t *cluster_ctas)
{
    if (!b) return FDTD_ERR_INVAL;
    if (dt) *dt = b->dt;
    if (steps) *steps = b->steps_done;
    if (cells) {
        int64_t c = 0;
        for (int64_t n : b->nz) c += n;
        *cells = c;
    }
    if (nodes) *nodes = b->nrows * b->nnode;
    if (nclusters) *nclusters = b->nclusters;
    if (cluster_ctas) *cluster_ctas = b->cluster_ctas;
    return FDTD_OK;
}

const char *fdtd_batch_last_error(fdtd_batch_t b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void fdtd_batch_destroy(fdtd_batch_t b) { destroy_batch(b); }

}  // extern "C"

// stencil_tma.cu -- FP32 curl stencils (Sec. 2, Eq. 1-6; CPML Eq. 7-12) fed by
// the tensor memory accelerator: 3-D column kernels and 2-D strip kernels.
//
// A block owns a 32 x 8 column of cells and walks `tz` planes of it along z.
// Per plane one thread issues six tiled TMA loads into a ring of shared-memory
// stages: the three components the curl differentiates, as a 36 x 9 box that
// carries the one-cell x / y neighbours (x is widened to 36 so every box row
// is a whole number of 16-byte units), and the three components being
// updated, as the 32 x 8 tile.  The z neighbour is the previous plane's value
// of the same thread, kept in registers: the H update needs E^{k+1} and walks
// z downwards, the E update needs H^{k-1} and walks upwards.  Ghost nodes past
// the grid read as zero (the TMA fill value), as in the one-cell kernels; the
// low-side differences of the E update at i, j, k = 0 are set to zero
// explicitly, like there.  Stage s of the ring holds plane s, s + S, ...; per
// plane, warp 0 waits on the stage's mbarrier while the other warps sleep in
// the one block barrier of the plane, which also frees the stage of the
// previous plane for the next load: with S = 4 stages three planes (21 KB)
// per block, six blocks per SM, are in flight while one is computed.
//
// These kernels are launched without programmatic dependent launch (see
// launch_plain) and do not let their successors start early.
//
// Every mbarrier wait is bounded: a block whose wait gives up stops storing,
// waits (again bounded) for the loads it issued, sets bit 2 of the device
// error word and returns; blocks that start after that return at once.
#include <cuda.h>

#include "async.cuh"
#include "stencil_common.cuh"

namespace fp {

namespace {

constexpr int kTX = 32, kTY = 8, kTT = kTX * kTY;   // tile; one thread per column cell
constexpr int kBX = kTX + 4, kBY = kTY + 1;          // neighbour box
constexpr int kBoxPitch = 352;                       // floats per box in shared memory (324 rounded to 128 B)
constexpr int kStageFloats = 3 * kBoxPitch + 3 * kTT;
constexpr int kStages = 4;
// 6 resident blocks per SM (40 registers a thread): on GB300 occupancy, not the
// ring depth, sets how many bytes are in flight (3 to 5 stages time the same)
constexpr int kMinBlocks = 6;
constexpr uint32_t kStageBytes = 3 * kBX * kBY * 4 + 3 * kTT * 4;   // what one plane's six loads deliver
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s: a plane load takes microseconds
constexpr size_t kSmemBytes = (size_t)kStages * kStageFloats * 4;

struct Boxes {
    CUtensorMap nb[3];     // neighbour boxes (36 x 9 x 1) of the differentiated components
    CUtensorMap tile[3];   // tiles (32 x 8 x 1) of the updated components
};

template <int S>
struct TmaSmemN {
    __align__(8) uint64_t full[S];
    int quit;
};
using TmaSmem = TmaSmemN<kStages>;

// block-uniform: whether a wait of an earlier block gave up in this launch sequence
__device__ __forceinline__ bool quit_early(const int *err, int *quit)
{
    if (threadIdx.x == 0) *quit = *(const volatile int *)err & 2;
    __syncthreads();
    return *quit != 0;
}

// issue plane p of the block's walk into stage p % S (one thread)
__device__ __forceinline__ void issue_plane(const Boxes &bx, float *ring, uint64_t *full, int p, int xn, int yn, int xt,
                                            int yt, int z)
{
    float *st = ring + (p % kStages) * kStageFloats;
    uint64_t *m = &full[p % kStages];
    mbar_arrive_expect_tx(m, kStageBytes);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_3d(st + c * kBoxPitch, &bx.nb[c], m, xn, yn, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_3d(st + 3 * kBoxPitch + c * kTT, &bx.tile[c], m, xt, yt, z);
}

// Plane q of the walk is in its stage: warp 0 waits on the stage's barrier
// while the other warps sleep in the block barrier (which also tells that
// every warp is done with the previous iteration, so the caller can refill
// the stage that iteration read last).
// If the wait gave up, every thread waits (bounded) for the loads still in
// flight, planes q .. issued - 1, so the block's shared memory is quiet when
// it ends; bit 2 of the error word is set and false returned (block-uniform).
// `lag`: the caller refills the stage of plane q - lag after this barrier, so
// planes up to q - lag - 1 + S have been issued when it runs.
template <int S = kStages>
__device__ __forceinline__ bool plane_ready(uint64_t *full, int q, int np, int warp, int *err, int lag = 1)
{
    bool ok = true;
    if (warp == 0) ok = mbar_wait_timed(&full[q % S], (uint32_t)((q / S) & 1), kWaitNs);
    if (!__syncthreads_or(!ok)) return true;
    const int issued = min(np, S + max(q - lag, 0));
    for (int p = q; p < issued; ++p) mbar_wait_timed(&full[p % S], (uint32_t)((p / S) & 1), kWaitNs);
    if (threadIdx.x == 0) atomicOr(err, 2);
    return false;
}

// whether a cell of column (i, j) lies in an x or y CPML slab (constant along the walk)
__device__ __forceinline__ bool column_in_slab(const Cpml<float> &cp, int64_t i, int64_t j, int nx, int ny)
{
    return cp.L > 0 && (in_slab<float>(i, nx, cp.L) || in_slab<float>(j, ny, cp.L));
}

// H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n; neighbour boxes: Ex, Ey, Ez at
// (x0 .. x0+35, y0 .. y0+8); tiles: Hx, Hy, Hz.  Walks z from the top plane down.
__global__ void __launch_bounds__(kTT, kMinBlocks) k_h3d_tma(const __grid_constant__ Boxes bx, const float *__restrict__ ex,
                                                 const float *__restrict__ ey, float *__restrict__ hx,
                                                 float *__restrict__ hy, float *__restrict__ hz, int nx, int ny, int nz,
                                                 int tz, float ch, float cph, Cpml<float> cp, Source src,
                                                 const int64_t *__restrict__ d_step, int kstep, int *err)
{
    extern __shared__ __align__(128) float ring[];
    __shared__ TmaSmem s;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * tz;
    const int z1 = min(z0 + tz, nz), np = z1 - z0;
    const int64_t i = x0 + tx, j = y0 + ty;
    const bool own = i < nx && j < ny;
    if (quit_early(err, &s.quit)) return;   // an earlier block's wait gave up: the step is void
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) write_source(src, d_step, kstep);
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&s.full[q], 1);
        fence_proxy_async_smem();
        for (int p = 0; p < min(kStages, np); ++p) issue_plane(bx, ring, s.full, p, x0, y0, x0, y0, z1 - 1 - p);
    }
    const int64_t sxy = (int64_t)nx * ny;
    // E^{k+1} of this thread's cell above the top plane (a PEC ghost past nz)
    float exn = 0.f, eyn = 0.f;
    if (own && z1 < nz) {
        const int64_t c = (int64_t)z1 * sxy + j * nx + i;
        exn = ex[c];
        eyn = ey[c];
    }
    __syncthreads();
    const int hc = ty * kBX + tx;
    const bool col_slab = column_in_slab(cp, i, j, nx, ny);
    int64_t c = (int64_t)(z1 - 1) * sxy + j * nx + i;   // this thread's cell in plane k
    for (int q = 0; q < np; ++q, c -= sxy) {
        const int k = z1 - 1 - q;
        if (!plane_ready(s.full, q, np, ty, err)) return;
        if (tid == 0 && q >= 1 && q - 1 + kStages < np)
            issue_plane(bx, ring, s.full, q - 1 + kStages, x0, y0, x0, y0, z1 - (q + kStages));
        const float *st = ring + (q % kStages) * kStageFloats;
        const float *Ex = st, *Ey = st + kBoxPitch, *Ez = st + 2 * kBoxPitch, *Ht = st + 3 * kBoxPitch;
        const float exc = Ex[hc], eyc = Ey[hc], ezc = Ez[hc];
        const float dEz_y = Ez[hc + kBX] - ezc;
        const float dEy_z = eyn - eyc;
        const float dEx_z = exn - exc;
        const float dEz_x = Ez[hc + 1] - ezc;
        const float dEy_x = Ey[hc + 1] - eyc;
        const float dEx_y = Ex[hc + kBX] - exc;
        float hxv = Ht[tid], hyv = Ht[kTT + tid], hzv = Ht[2 * kTT + tid];
        exn = exc;
        eyn = eyc;
        if (own) {
            if (!col_slab && !(cp.L > 0 && in_slab<float>(k, nz, cp.L))) {
                hxv -= ch * (dEz_y - dEy_z);
                hyv -= ch * (dEx_z - dEz_x);
                hzv -= ch * (dEy_x - dEx_y);
            } else {
                h3d_pml<float>(cp, nx, ny, nz, i, j, k, ch, cph, dEz_y, dEy_z, dEx_z, dEz_x, dEy_x, dEx_y, hxv, hyv,
                               hzv);
            }
            hx[c] = hxv;
            hy[c] = hyv;
            hz[c] = hzv;
        }
    }
}

// E^{n+1} = E^n + dt/eps0 curl H^{n+1/2} (J already applied to E); neighbour
// boxes: Hx, Hy, Hz at (x0-4 .. x0+31, y0-1 .. y0+7); tiles: Ex, Ey, Ez.
// Walks z upwards.
__global__ void __launch_bounds__(kTT, kMinBlocks) k_e3d_tma(const __grid_constant__ Boxes bx, const float *__restrict__ hx,
                                                 const float *__restrict__ hy, float *__restrict__ ex,
                                                 float *__restrict__ ey, float *__restrict__ ez, int nx, int ny, int nz,
                                                 int tz, float ce, float cpe, Cpml<float> cp, Source src, int *err)
{
    extern __shared__ __align__(128) float ring[];
    __shared__ TmaSmem s;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * tz;
    const int z1 = min(z0 + tz, nz), np = z1 - z0;
    const int64_t i = x0 + tx, j = y0 + ty;
    const bool own = i < nx && j < ny;
    if (quit_early(err, &s.quit)) return;
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&s.full[q], 1);
        fence_proxy_async_smem();
        for (int p = 0; p < min(kStages, np); ++p) issue_plane(bx, ring, s.full, p, x0 - 4, y0 - 1, x0, y0, z0 + p);
    }
    const int64_t sxy = (int64_t)nx * ny;
    // H^{k-1} of this thread's cell below the first plane (unused at k = 0)
    float hxp = 0.f, hyp = 0.f;
    if (own && z0 > 0) {
        const int64_t c = (int64_t)(z0 - 1) * sxy + j * nx + i;
        hxp = hx[c];
        hyp = hy[c];
    }
    const float g = src.kind ? (float)*src.val : 0.f;
    // whether the source covers this column (then it hits the cell of plane src.k)
    const bool src_col = src.kind && (src.loc == FDTD_LOC_SHEET
                                          ? (i >= src.i0 && i < src.i1 && j >= src.j0 && j < src.j1)
                                          : (i == src.i && j == src.j));
    __syncthreads();
    const int hc = (ty + 1) * kBX + tx + 4;
    const bool col_slab = column_in_slab(cp, i, j, nx, ny);
    int64_t c = (int64_t)z0 * sxy + j * nx + i;   // this thread's cell in plane k
    for (int q = 0; q < np; ++q, c += sxy) {
        const int k = z0 + q;
        if (!plane_ready(s.full, q, np, ty, err)) return;
        if (tid == 0 && q >= 1 && q - 1 + kStages < np)
            issue_plane(bx, ring, s.full, q - 1 + kStages, x0 - 4, y0 - 1, x0, y0, z0 + q - 1 + kStages);
        const float *st = ring + (q % kStages) * kStageFloats;
        const float *Hx = st, *Hy = st + kBoxPitch, *Hz = st + 2 * kBoxPitch, *Et = st + 3 * kBoxPitch;
        const float hxc = Hx[hc], hyc = Hy[hc], hzc = Hz[hc];
        const float exc = Et[tid], eyc = Et[kTT + tid], ezc = Et[2 * kTT + tid];
        const float dHz_y = j > 0 ? hzc - Hz[hc - kBX] : 0.f;
        const float dHy_z = k > 0 ? hyc - hyp : 0.f;
        const float dHx_z = k > 0 ? hxc - hxp : 0.f;
        const float dHz_x = i > 0 ? hzc - Hz[hc - 1] : 0.f;
        const float dHy_x = i > 0 ? hyc - Hy[hc - 1] : 0.f;
        const float dHx_y = j > 0 ? hxc - Hx[hc - kBX] : 0.f;
        hxp = hxc;
        hyp = hyc;
        if (own) {
            float ux, uy, uz;
            if (!col_slab && !(cp.L > 0 && in_slab<float>(k, nz, cp.L))) {
                ux = ce * (dHz_y - dHy_z);
                uy = ce * (dHx_z - dHz_x);
                uz = ce * (dHy_x - dHx_y);
            } else {
                e3d_pml<float>(cp, nx, ny, nz, i, j, k, ce, cpe, dHz_y, dHy_z, dHx_z, dHz_x, dHy_x, dHx_y, ux, uy, uz);
            }
            if (j > 0 && k > 0) {
                float v = exc + ux;
                if (src_col && k == src.k) v += g;
                ex[c] = v;
            }
            if (i > 0 && k > 0) ey[c] = eyc + uy;
            if (i > 0 && j > 0) ez[c] = ezc + uz;
        }
    }
}

// ---------------------------------------------------------------------------
// Fused E^{n+1} + H^{n+3/2} (the opt-in fused step sequence) on TMA-staged
// planes.  Reads field set A (E' = E^n after the plasma current, H^{n+1/2},
// psi) and writes set B, so no block reads what another writes.  A block owns
// a 32 x 8 column and walks up z: per plane z the stage holds the H^{n+1/2}
// box x0-4 .. x0+35, y0-1 .. y0+8 (40 x 10) and the E' box x0 .. x0+35,
// y0 .. y0+8 (36 x 9); E^{n+1}(z) is formed on the tile and its +x / +y halo
// (33 x 9 cells, the halo recomputed by the neighbouring block too) into one
// of two shared buffers, the tile stored; then H^{n+3/2}(z-1) is formed on
// the tile from E^{n+1} of planes z-1 and z.  The walk covers planes
// z0-1 (H only, for dH/dz) .. z1 (E only, for dE/dz of H^{n+3/2}(z1-1)); at
// the top of the grid E^{n+1}(nz) is the PEC ghost 0.  Two block barriers a
// plane; the stage of plane z-2 is refilled after the first.  Every field is
// read once and written once from DRAM: 48 B a cell against 72 B for the two
// separate passes.

constexpr int kFHX = 40, kFHY = 10, kFHPitch = 416;   // H box; 400 floats rounded to 128 B
constexpr int kFEX = 36, kFEY = 9, kFEPitch = 352;    // E' box; 324 floats rounded to 128 B
constexpr int kFStage = 3 * kFHPitch + 3 * kFEPitch;
constexpr uint32_t kFStageBytes = 3 * kFHX * kFHY * 4 + 3 * kFEX * kFEY * 4;
constexpr int kFBX = kTX + 1, kFBY = kTY + 1, kFBuf = kFBX * kFBY;   // E^{n+1} on tile + halo
constexpr int kFStages = 4;
constexpr size_t kFSmemBytes = (size_t)(kFStages * kFStage + 2 * 3 * kFBuf) * 4;
constexpr int kFMinBlocks = 4;

struct FusedBoxes {
    CUtensorMap h[3];   // 40 x 10 x 1 boxes of Hx, Hy, Hz
    CUtensorMap e[3];   // 36 x 9 x 1 boxes of Ex, Ey, Ez
};

struct FusedOut {
    float *f[6];
    float *psi[12];
};

__device__ __forceinline__ void issue_fused_plane(const FusedBoxes &bx, float *ring, uint64_t *full, int p, int x0,
                                                  int y0, int z)
{
    float *st = ring + (p % kFStages) * kFStage;
    uint64_t *m = &full[p % kFStages];
    mbar_arrive_expect_tx(m, kFStageBytes);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_3d(st + c * kFHPitch, &bx.h[c], m, x0 - 4, y0 - 1, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_3d(st + 3 * kFHPitch + c * kFEPitch, &bx.e[c], m, x0, y0, z);
}

__device__ __forceinline__ bool source_column(const Source &src, int64_t i, int64_t j)
{
    return src.kind && (src.loc == FDTD_LOC_SHEET ? (i >= src.i0 && i < src.i1 && j >= src.j0 && j < src.j1)
                                                  : (i == src.i && j == src.j));
}

__global__ void __launch_bounds__(kTT, kFMinBlocks) k_eh3d_tma(const __grid_constant__ FusedBoxes bx, FusedOut out,
                                                              int nx, int ny, int nz, int tz, float ce, float cpe,
                                                              float ch, float cph, Cpml<float> cin, Source src,
                                                              const int64_t *__restrict__ d_step, int kstep, int *err)
{
    extern __shared__ __align__(128) float ring[];
    float *ebuf = ring + kFStages * kFStage;   // [2][3][kFBuf]: E^{n+1} of planes of even / odd z
    __shared__ TmaSmemN<kFStages> s;
    __shared__ float s_g;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * tz;
    const int z1 = min(z0 + tz, nz);
    const int zs = z0 > 0 ? z0 - 1 : 0, ze = z1 < nz ? z1 : z1 - 1, np = ze - zs + 1;
    if (quit_early(err, &s.quit)) return;
    if (tid == 0) {
        const int64_t n1 = *d_step + kstep + 1;   // E^{n+1} is at t^{n+1}
        s_g = src.kind && src.k >= zs && src.k <= ze ? (float)source_value(src, (double)n1 * src.dt) : 0.f;
        if (src.kind && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            *src.val = source_value(src, (double)(n1 + 1) * src.dt);   // for an unfused E update that follows
        for (int q = 0; q < kFStages; ++q) mbar_init(&s.full[q], 1);
        fence_proxy_async_smem();
        for (int p = 0; p < min(kFStages, np); ++p) issue_fused_plane(bx, ring, s.full, p, x0, y0, zs + p);
    }
    __syncthreads();
    const int64_t sxy = (int64_t)nx * ny;
    const int L = cin.L;
    // E^{n+1}(z) of local cell (lx, ly) of the tile + halo; stores the tile's cells (and their psi) to set B
    auto e_cell = [&](const float *cur, const float *prv, int lx, int ly, int z, float *eb) {
        const int64_t i = x0 + lx, j = y0 + ly;
        float exn = 0.f, eyn = 0.f, ezn = 0.f;
        if (i < nx && j < ny) {
            const int hb = (ly + 1) * kFHX + lx + 4, eb_ = ly * kFEX + lx;
            const float *Hx = cur, *Hy = cur + kFHPitch, *Hz = cur + 2 * kFHPitch, *Ep = cur + 3 * kFHPitch;
            const float hxc = Hx[hb], hyc = Hy[hb], hzc = Hz[hb];
            const float dHz_y = j > 0 ? hzc - Hz[hb - kFHX] : 0.f;
            const float dHy_z = z > 0 ? hyc - prv[kFHPitch + hb] : 0.f;
            const float dHx_z = z > 0 ? hxc - prv[hb] : 0.f;
            const float dHz_x = i > 0 ? hzc - Hz[hb - 1] : 0.f;
            const float dHy_x = i > 0 ? hyc - Hy[hb - 1] : 0.f;
            const float dHx_y = j > 0 ? hxc - Hx[hb - kFHX] : 0.f;
            const float exc = Ep[eb_], eyc = Ep[kFEPitch + eb_], ezc = Ep[2 * kFEPitch + eb_];
            const bool own = lx < kTX && ly < kTY && z < z1;
            float ux, uy, uz;
            if (!(L > 0 && (in_slab<float>(i, nx, L) || in_slab<float>(j, ny, L) || in_slab<float>(z, nz, L)))) {
                ux = ce * (dHz_y - dHy_z);
                uy = ce * (dHx_z - dHz_x);
                uz = ce * (dHy_x - dHx_y);
            } else {
                e3d_pml_io<float>(cin, out.psi, own, nx, ny, nz, i, j, z, ce, cpe, dHz_y, dHy_z, dHx_z, dHz_x, dHy_x,
                                  dHx_y, ux, uy, uz);
            }
            exn = exc;
            eyn = eyc;
            ezn = ezc;
            if (j > 0 && z > 0) {
                exn = exc + ux;
                if (z == src.k && source_column(src, i, j)) exn += s_g;
            }
            if (i > 0 && z > 0) eyn = eyc + uy;
            if (i > 0 && j > 0) ezn = ezc + uz;
            if (own) {
                const int64_t c = (int64_t)z * sxy + j * nx + i;
                out.f[FDTD_EX][c] = exn;
                out.f[FDTD_EY][c] = eyn;
                out.f[FDTD_EZ][c] = ezn;
            }
        }
        const int e = ly * kFBX + lx;
        eb[e] = exn;
        eb[kFBuf + e] = eyn;
        eb[2 * kFBuf + e] = ezn;
    };
    // H^{n+3/2}(k) of this thread's cell: H^{n+1/2}(k) from stage hs, E^{n+1}(k) from ek, E^{n+1}(k+1) from ek1
    // (nullptr: the ghost plane above the grid)
    auto h_cell = [&](const float *hs, const float *ek, const float *ek1, int k) {
        const int64_t i = x0 + tx, j = y0 + ty;
        if (i >= nx || j >= ny) return;
        const int hb = (ty + 1) * kFHX + tx + 4, e = ty * kFBX + tx;
        float hxv = hs[hb], hyv = hs[kFHPitch + hb], hzv = hs[2 * kFHPitch + hb];
        const float exc = ek[e], eyc = ek[kFBuf + e], ezc = ek[2 * kFBuf + e];
        const float dEz_y = ek[2 * kFBuf + e + kFBX] - ezc;
        const float dEy_z = (ek1 ? ek1[kFBuf + e] : 0.f) - eyc;
        const float dEx_z = (ek1 ? ek1[e] : 0.f) - exc;
        const float dEz_x = ek[2 * kFBuf + e + 1] - ezc;
        const float dEy_x = ek[kFBuf + e + 1] - eyc;
        const float dEx_y = ek[e + kFBX] - exc;
        if (!(L > 0 && (in_slab<float>(i, nx, L) || in_slab<float>(j, ny, L) || in_slab<float>(k, nz, L)))) {
            hxv -= ch * (dEz_y - dEy_z);
            hyv -= ch * (dEx_z - dEz_x);
            hzv -= ch * (dEy_x - dEx_y);
        } else {
            h3d_pml_io<float>(cin, out.psi, true, nx, ny, nz, i, j, k, ch, cph, dEz_y, dEy_z, dEx_z, dEz_x, dEy_x,
                              dEx_y, hxv, hyv, hzv);
        }
        const int64_t c = (int64_t)k * sxy + j * nx + i;
        out.f[FDTD_HX][c] = hxv;
        out.f[FDTD_HY][c] = hyv;
        out.f[FDTD_HZ][c] = hzv;
    };
    for (int p = 0; p < np; ++p) {
        const int z = zs + p;
        if (!plane_ready<kFStages>(s.full, p, np, ty, err, 2)) return;
        if (tid == 0 && p >= 2 && p - 2 + kFStages < np)
            issue_fused_plane(bx, ring, s.full, p - 2 + kFStages, x0, y0, zs + p - 2 + kFStages);
        if (z < z0) continue;   // plane z0-1: its H^{n+1/2} serves dH/dz of E^{n+1}(z0)
        const float *cur = ring + (p % kFStages) * kFStage;
        const float *prv = ring + ((p + kFStages - 1) % kFStages) * kFStage;
        float *eb = ebuf + (z & 1) * 3 * kFBuf;
        e_cell(cur, prv, tx, ty, z, eb);
        if (tid < kFBuf - kTT) {   // the +x column (9 cells) and the +y row (32 cells)
            const int hx_ = tid < kFBY ? kTX : tid - kFBY, hy_ = tid < kFBY ? tid : kTY;
            e_cell(cur, prv, hx_, hy_, z, eb);
        }
        __syncthreads();
        if (z - 1 >= z0) h_cell(prv, ebuf + ((z - 1) & 1) * 3 * kFBuf, eb, z - 1);
    }
    if (z1 == nz) {   // H^{n+3/2} of the top plane: E^{n+1} above it is the PEC ghost
        const int p = np - 1;
        h_cell(ring + (p % kFStages) * kFStage, ebuf + ((nz - 1) & 1) * 3 * kFBuf, nullptr, nz - 1);
    }
}

// ---------------------------------------------------------------------------
// 2-D TMz strips.  A block of 32 x 8 threads owns a 32-cell strip of x and walks
// `rows` rows of it in chunks of kC2 = 8 * kR2 rows (each thread takes rows ty,
// ty + 8, ...); per chunk one thread issues the tiled 2-D loads of the
// differentiated component(s) as 36 x (kC2 + 1) boxes (the one-cell x / y
// neighbours, zero-filled past the grid) and of the updated component(s) as
// 32 x kC2 tiles into a stage of the same 4-stage ring; one waiting warp and one
// block barrier per chunk.  The cell formulas are those of k_h2d / k_e2d.

constexpr int kR2 = 2;                              // rows per thread and chunk
constexpr int kS2Stages = 4;                        // stages of the 2-D ring
constexpr int kC2 = kTY * kR2;                      // rows per chunk
constexpr int kB2Y = kC2 + 1;
constexpr int kB2Pitch = (kBX * kB2Y + 31) / 32 * 32;   // floats per box, a multiple of 128 bytes
constexpr int kT2 = kTX * kC2;                      // floats per tile
constexpr int kS2H = kB2Pitch + 2 * kT2;            // H update stage: Ez box, Hx and Hy tiles
constexpr int kS2E = 2 * kB2Pitch + kT2;            // E update stage: Hx and Hy boxes, Ez tile
constexpr uint32_t kS2HBytes = kBX * kB2Y * 4 + 2 * kT2 * 4;
constexpr uint32_t kS2EBytes = 2 * kBX * kB2Y * 4 + kT2 * 4;
constexpr size_t kSmem2H = (size_t)kS2Stages * kS2H * 4, kSmem2E = (size_t)kS2Stages * kS2E * 4;

struct Boxes2 {
    CUtensorMap ez_nb, hx_nb, hy_nb;   // 36 x (kC2 + 1) boxes
    CUtensorMap ez_t, hx_t, hy_t;      // 32 x kC2 tiles
};

__global__ void __launch_bounds__(kTT, kMinBlocks) k_h2d_tma(const __grid_constant__ Boxes2 bx, float *__restrict__ hx,
                                                            float *__restrict__ hy, int nx, int ny, int rows, float ch,
                                                            float cph, Cpml<float> cp, Source src,
                                                            const int64_t *__restrict__ d_step, int kstep, int *err)
{
    extern __shared__ __align__(128) float ring[];
    __shared__ TmaSmemN<kS2Stages> s;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * rows;
    const int np = (min(rows, ny - y0) + kC2 - 1) / kC2;   // chunks
    const int64_t i = x0 + tx;
    if (quit_early(err, &s.quit)) return;
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) write_source(src, d_step, kstep);
    auto issue = [&](int p) {
        float *st = ring + (p % kS2Stages) * kS2H;
        uint64_t *m = &s.full[p % kS2Stages];
        const int y = y0 + p * kC2;
        mbar_arrive_expect_tx(m, kS2HBytes);
        tma_load_2d(st, &bx.ez_nb, m, x0, y);
        tma_load_2d(st + kB2Pitch, &bx.hx_t, m, x0, y);
        tma_load_2d(st + kB2Pitch + kT2, &bx.hy_t, m, x0, y);
    };
    if (tid == 0) {
        for (int q = 0; q < kS2Stages; ++q) mbar_init(&s.full[q], 1);
        fence_proxy_async_smem();
        for (int p = 0; p < min(kS2Stages, np); ++p) issue(p);
    }
    __syncthreads();
    for (int q = 0; q < np; ++q) {
        if (!plane_ready<kS2Stages>(s.full, q, np, ty, err)) return;
        if (tid == 0 && q >= 1 && q - 1 + kS2Stages < np) issue(q - 1 + kS2Stages);
        const float *st = ring + (q % kS2Stages) * kS2H;
        const float *Ez = st, *Hx = st + kB2Pitch, *Hy = Hx + kT2;
#pragma unroll
        for (int r = 0; r < kR2; ++r) {
            const int ly = ty + r * kTY;
            const int64_t j = y0 + q * kC2 + ly;
            if (i >= nx || j >= ny) continue;
            const int hc = ly * kBX + tx, tc = ly * kTX + tx;
            const float e = Ez[hc];
            const float dEy = Ez[hc + kBX] - e;   // dEz along y (0 past the last row: TMA fill)
            const float dEx = Ez[hc + 1] - e;     // dEz along x
            float hxv = Hx[tc], hyv = Hy[tc];
            if (cp.L == 0 || !(in_slab<float>(i, nx, cp.L) || in_slab<float>(j, ny, cp.L))) {
                hxv = hx_plain(hxv, ch, dEy);
                hyv = hy_plain(hyv, ch, dEx);
            } else {
                h2d_pml<float>(cp, nx, ny, i, j, ch, cph, dEy, dEx, hxv, hyv);
            }
            const int64_t c = j * nx + i;
            hx[c] = hxv;
            hy[c] = hyv;
        }
    }
}

__global__ void __launch_bounds__(kTT, kMinBlocks) k_e2d_tma(const __grid_constant__ Boxes2 bx, float *__restrict__ ez,
                                                            int nx, int ny, int rows, float ce, float cpe, Cpml<float> cp,
                                                            Source src, int *err)
{
    extern __shared__ __align__(128) float ring[];
    __shared__ TmaSmemN<kS2Stages> s;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * rows;
    const int np = (min(rows, ny - y0) + kC2 - 1) / kC2;
    const int64_t i = x0 + tx;
    if (quit_early(err, &s.quit)) return;
    auto issue = [&](int p) {
        float *st = ring + (p % kS2Stages) * kS2E;
        uint64_t *m = &s.full[p % kS2Stages];
        const int y = y0 + p * kC2;
        mbar_arrive_expect_tx(m, kS2EBytes);
        tma_load_2d(st, &bx.hx_nb, m, x0 - 4, y - 1);
        tma_load_2d(st + kB2Pitch, &bx.hy_nb, m, x0 - 4, y - 1);
        tma_load_2d(st + 2 * kB2Pitch, &bx.ez_t, m, x0, y);
    };
    if (tid == 0) {
        for (int q = 0; q < kS2Stages; ++q) mbar_init(&s.full[q], 1);
        fence_proxy_async_smem();
        for (int p = 0; p < min(kS2Stages, np); ++p) issue(p);
    }
    const float g = src.kind ? (float)*src.val : 0.f;
    __syncthreads();
    for (int q = 0; q < np; ++q) {
        if (!plane_ready<kS2Stages>(s.full, q, np, ty, err)) return;
        if (tid == 0 && q >= 1 && q - 1 + kS2Stages < np) issue(q - 1 + kS2Stages);
        const float *st = ring + (q % kS2Stages) * kS2E;
        const float *Hx = st, *Hy = st + kB2Pitch, *Ezt = st + 2 * kB2Pitch;
#pragma unroll
        for (int r = 0; r < kR2; ++r) {
            const int ly = ty + r * kTY;
            const int64_t j = y0 + q * kC2 + ly;
            if (i < 1 || j < 1 || i >= nx || j >= ny) continue;   // PEC nodes are not updated
            const int hc = (ly + 1) * kBX + tx + 4;
            const float dHx = Hy[hc] - Hy[hc - 1];     // dHy along x
            const float dHy = Hx[hc] - Hx[hc - kBX];   // dHx along y
            const float upd = cp.L == 0 || !(in_slab<float>(i, nx, cp.L) || in_slab<float>(j, ny, cp.L))
                                  ? e2d_term(ce, dHx, dHy)
                                  : e2d_pml<float>(cp, nx, ny, i, j, ce, cpe, dHx, dHy);
            float v = rn_add(Ezt[ly * kTX + tx], upd);
            if (src.kind && i == src.i && j == src.j) v = rn_add(v, g);
            ez[j * nx + i] = v;
        }
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

bool encode(CUtensorMap *m, float *base, int64_t nx, int64_t ny, int64_t nz, uint32_t box_x, uint32_t box_y)
{
    const EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny) * 4};
    const cuuint32_t box[3] = {box_x, box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode2(CUtensorMap *m, float *base, int64_t nx, int64_t ny, uint32_t box_x, uint32_t box_y)
{
    const EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    const cuuint32_t box[2] = {box_x, box_y};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct TmaMaps {
    Boxes h;   // for the H update: neighbour boxes of Ex, Ey, Ez; tiles of Hx, Hy, Hz
    Boxes e;   // for the E update: neighbour boxes of Hx, Hy, Hz; tiles of Ex, Ey, Ez
    const void *f[6];
    int64_t nx, ny, nz;
    // fused E + H pass: boxes of field sets 0 and 1 (made when both sets exist)
    bool fused_ready;
    FusedBoxes fused[2];
    const void *fset[2][6];
    int ndim;
    Boxes2 b2;   // 2-D strips
};

bool tma_stencil_eligible(int64_t nx, int64_t ny, int64_t nz)
{
    // 16-byte row and plane strides; coordinates and plane counts fit int
    return nx % 4 == 0 && nx <= (1 << 24) && ny <= (1 << 24) && nz <= (1 << 24) && nx * ny * nz < (int64_t)1 << 40;
}

TmaMaps *tma_maps_create(float *const f[6], int64_t nx, int64_t ny, int64_t nz)
{
    if (!tma_stencil_eligible(nx, ny, nz)) return nullptr;
    if (nz == 1) {   // 2-D TMz: Ez, Hx, Hy
        for (int q : {FDTD_EZ, FDTD_HX, FDTD_HY})
            if (!f[q] || reinterpret_cast<uintptr_t>(f[q]) % 16) return nullptr;
        TmaMaps *t = new TmaMaps{};
        t->ndim = 2;
        const bool ok2 = encode2(&t->b2.ez_nb, f[FDTD_EZ], nx, ny, kBX, kB2Y) &&
                         encode2(&t->b2.hx_nb, f[FDTD_HX], nx, ny, kBX, kB2Y) &&
                         encode2(&t->b2.hy_nb, f[FDTD_HY], nx, ny, kBX, kB2Y) &&
                         encode2(&t->b2.ez_t, f[FDTD_EZ], nx, ny, kTX, kC2) &&
                         encode2(&t->b2.hx_t, f[FDTD_HX], nx, ny, kTX, kC2) &&
                         encode2(&t->b2.hy_t, f[FDTD_HY], nx, ny, kTX, kC2);
        for (int q = 0; q < 6; ++q) t->f[q] = f[q];
        t->nx = nx;
        t->ny = ny;
        t->nz = 1;
        if (!ok2) {
            delete t;
            return nullptr;
        }
        return t;
    }
    for (int q = 0; q < 6; ++q)
        if (!f[q] || reinterpret_cast<uintptr_t>(f[q]) % 16) return nullptr;
    TmaMaps *t = new TmaMaps{};
    t->ndim = 3;
    bool ok = true;
    for (int c = 0; c < 3 && ok; ++c) {
        ok = encode(&t->h.nb[c], f[FDTD_EX + c], nx, ny, nz, kBX, kBY) &&
             encode(&t->h.tile[c], f[FDTD_HX + c], nx, ny, nz, kTX, kTY) &&
             encode(&t->e.nb[c], f[FDTD_HX + c], nx, ny, nz, kBX, kBY) &&
             encode(&t->e.tile[c], f[FDTD_EX + c], nx, ny, nz, kTX, kTY);
    }
    for (int q = 0; q < 6; ++q) t->f[q] = f[q];
    t->nx = nx;
    t->ny = ny;
    t->nz = nz;
    if (!ok) {
        delete t;
        return nullptr;
    }
    return t;
}

void tma_maps_free(TmaMaps *t) { delete t; }

bool tma_fused_prepare(TmaMaps *t, float *const f0[6], float *const f1[6])
{
    if (!t) return false;
    float *const *sets[2] = {f0, f1};
    bool same = t->fused_ready;
    for (int b = 0; b < 2 && same; ++b)
        for (int q = 0; q < 6; ++q) same = same && t->fset[b][q] == sets[b][q];
    if (same) return true;
    t->fused_ready = false;
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < 6; ++q)
            if (!sets[b][q] || reinterpret_cast<uintptr_t>(sets[b][q]) % 16) return false;
    for (int b = 0; b < 2; ++b) {
        for (int c = 0; c < 3; ++c)
            if (!encode(&t->fused[b].h[c], sets[b][FDTD_HX + c], t->nx, t->ny, t->nz, kFHX, kFHY) ||
                !encode(&t->fused[b].e[c], sets[b][FDTD_EX + c], t->nx, t->ny, t->nz, kFEX, kFEY))
                return false;
        for (int q = 0; q < 6; ++q) t->fset[b][q] = sets[b][q];
    }
    t->fused_ready = true;
    return true;
}

void tma_fused_forget(TmaMaps *t)
{
    if (t) t->fused_ready = false;
}

static inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

bool tma_maps_match(const TmaMaps *t, float *const f[6])
{
    if (!t) return false;
    for (int q = 0; q < 6; ++q)
        if (t->f[q] != f[q]) return false;
    return true;
}

void launch_h2d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, float ch, float cph,
                    Cpml<float> cp, Source src, const int64_t *d_step, int kstep, int rows, int *err)
{
    rows = (rows + kC2 - 1) / kC2 * kC2;
    const dim3 g(cdivu(nx, kTX), cdivu(ny, rows));
    launch_plain(k_h2d_tma, g, dim3(kTT), kSmem2H, st, t->b2, f[FDTD_HX], f[FDTD_HY], (int)nx, (int)ny, rows, ch, cph,
               cp, src, d_step, kstep, err);
}

void launch_e2d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, float ce, float cpe,
                    Cpml<float> cp, Source src, int rows, int *err)
{
    rows = (rows + kC2 - 1) / kC2 * kC2;
    const dim3 g(cdivu(nx, kTX), cdivu(ny, rows));
    launch_plain(k_e2d_tma, g, dim3(kTT), kSmem2E, st, t->b2, f[FDTD_EZ], (int)nx, (int)ny, rows, ce, cpe, cp, src, err);
}


void launch_h3d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, int64_t nz,
                    float ch, float cph, Cpml<float> cp, Source src, const int64_t *d_step, int kstep, int tz, int *err)
{
    const dim3 g(cdivu(nx, kTX), cdivu(ny, kTY), cdivu(nz, tz));
    launch_plain(k_h3d_tma, dim3(g), dim3(kTT), kSmemBytes, st, t->h, f[FDTD_EX], f[FDTD_EY], f[FDTD_HX], f[FDTD_HY], f[FDTD_HZ], (int)nx,
                                          (int)ny, (int)nz, tz, ch, cph, cp, src, d_step, kstep, err);
}

bool launch_eh3d_tma(cudaStream_t st, const TmaMaps *t, float *const fin[6], float *const fout[6],
                     float *const psi_out[12], float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                     const int64_t *d_step, int kstep, int tz, int *err)
{
    if (!t || !t->fused_ready) return false;
    int b = -1;
    for (int q = 0; q < 2 && b < 0; ++q)
        if (t->fset[q][0] == fin[0] && t->fset[q][5] == fin[5]) b = q;
    if (b < 0) return false;
    FusedOut o{};
    for (int q = 0; q < 6; ++q) o.f[q] = fout[q];
    for (int q = 0; q < 12; ++q) o.psi[q] = psi_out[q];
    static const bool attr = cudaFuncSetAttribute(k_eh3d_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kFSmemBytes) == cudaSuccess;
    if (!attr) return false;
    const dim3 g(cdivu(t->nx, kTX), cdivu(t->ny, kTY), cdivu(t->nz, tz));
    launch_plain(k_eh3d_tma, dim3(g), dim3(kTT), kFSmemBytes, st, t->fused[b], o, (int)t->nx, (int)t->ny, (int)t->nz, tz, ce, cpe, ch, cph,
                                            cin, src, d_step, kstep, err);
    return true;
}

void launch_e3d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, int64_t nz,
                    float ce, float cpe, Cpml<float> cp, Source src, int tz, int *err)
{
    const dim3 g(cdivu(nx, kTX), cdivu(ny, kTY), cdivu(nz, tz));
    launch_plain(k_e3d_tma, dim3(g), dim3(kTT), kSmemBytes, st, t->e, f[FDTD_HX], f[FDTD_HY], f[FDTD_EX], f[FDTD_EY], f[FDTD_EZ], (int)nx,
                                          (int)ny, (int)nz, tz, ce, cpe, cp, src, err);
}

}  // namespace fp

// diag.cu -- FP64 diagnostics of the current state: the discrete Yee
// energy invariant, the plain field energy, the particle-number perturbation
// sum_j df_j dV_j (total, max per cell, absolute) and a finiteness flag.
//
// Pass 1: grid-stride blocks accumulate FP64 partials (one row of 6 per block)
// into a scratch buffer; pass 2: one block reduces the rows.  The fields are
// read once; delta f rows are read one warp per row.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "internal.cuh"

namespace fp {

template <typename T>
__device__ __forceinline__ double ld(const void *p, int64_t i)
{
    return (double)reinterpret_cast<const T *>(p)[i];
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ void field_terms(const DiagArgs &a, int64_t c, double &we, double &wh, double &wh2, int &fin)
{
    if (a.ndim == 1) {
        const int64_t nz = a.nz;
        if (c <= nz) {
            double e = ld<T>(a.f[0], c);
            we += e * e;
            fin &= isfinite(e);
        }
        if (c < nz) {
            double h = ld<T>(a.f[4], c);
            double hn = h - a.ch * (ld<T>(a.f[0], c + 1) - ld<T>(a.f[0], c));
            wh += h * hn;
            wh2 += h * h;
            fin &= isfinite(h);
        }
    } else if (a.ndim == 2) {
        const int64_t nx = a.nx, ny = a.ny;
        const int64_t i = c % nx, j = c / nx;
        double e = ld<T>(a.f[2], c);
        double dEy = (j + 1 < ny ? ld<T>(a.f[2], c + nx) : 0.0) - e;
        double dEx = (i + 1 < nx ? ld<T>(a.f[2], c + 1) : 0.0) - e;
        double hx = ld<T>(a.f[3], c), hy = ld<T>(a.f[4], c);
        we += e * e;
        wh += hx * (hx - a.ch * dEy) + hy * (hy + a.ch * dEx);
        wh2 += hx * hx + hy * hy;
        fin &= isfinite(e) && isfinite(hx) && isfinite(hy);
    } else {
        const int64_t nx = a.nx, ny = a.ny, nz = a.nz, sxy = nx * ny;
        const int64_t i = c % nx, j = (c / nx) % ny, k = c / sxy;
        double ex = ld<T>(a.f[0], c), ey = ld<T>(a.f[1], c), ez = ld<T>(a.f[2], c);
        double hx = ld<T>(a.f[3], c), hy = ld<T>(a.f[4], c), hz = ld<T>(a.f[5], c);
        double ez_y = j + 1 < ny ? ld<T>(a.f[2], c + nx) : 0.0, ey_z = k + 1 < nz ? ld<T>(a.f[1], c + sxy) : 0.0;
        double ex_z = k + 1 < nz ? ld<T>(a.f[0], c + sxy) : 0.0, ez_x = i + 1 < nx ? ld<T>(a.f[2], c + 1) : 0.0;
        double ey_x = i + 1 < nx ? ld<T>(a.f[1], c + 1) : 0.0, ex_y = j + 1 < ny ? ld<T>(a.f[0], c + nx) : 0.0;
        double hxn = hx - a.ch * ((ez_y - ez) - (ey_z - ey));
        double hyn = hy - a.ch * ((ex_z - ex) - (ez_x - ez));
        double hzn = hz - a.ch * ((ey_x - ey) - (ex_y - ex));
        we += ex * ex + ey * ey + ez * ez;
        wh += hx * hxn + hy * hyn + hz * hzn;
        wh2 += hx * hx + hy * hy + hz * hz;
        fin &= isfinite(ex) && isfinite(ey) && isfinite(ez) && isfinite(hx) && isfinite(hy) && isfinite(hz);
    }
}

template <typename T>
__device__ __forceinline__ double df_val(const DiagArgs &a, int64_t row, int64_t j)
{
    const int64_t idx = row * a.pitch + j;
    if (a.f_dtype == FDTD_DF_BF16) {
        const uint16_t b = reinterpret_cast<const uint16_t *>(a.df)[idx];
        return (double)__uint_as_float((uint32_t)b << 16);
    }
    if (a.f_dtype == FDTD_DF_F64) return reinterpret_cast<const double *>(a.df)[idx];
    return (double)reinterpret_cast<const float *>(a.df)[idx];
}

template <typename T>
__global__ void __launch_bounds__(256) k_diag_partial(DiagArgs a, double *partials)
{
    __shared__ double red[6][8];
    double we = 0, wh = 0, wh2 = 0, num = 0, nmax = 0, nabs = 0;
    int fin = 1;
    const int64_t ncells = a.ndim == 1 ? a.nz + 1 : a.nx * a.ny * a.nz;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = tid; c < ncells; c += nth) field_terms<T>(a, c, we, wh, wh2, fin);
    // one warp per delta-f row
    const int lane = threadIdx.x & 31;
    const int64_t wg = tid >> 5, nw = nth >> 5;
    for (int64_t r = wg; r < a.nslots; r += nw) {
        double sr = 0, sa = 0;
        for (int64_t j = lane; j < a.nnode; j += 32) {
            double v = df_val<T>(a, r, j);
            sr += v * a.dV[j];
            sa += fabs(v) * a.dV[j];
            fin &= isfinite(v);
        }
        sr = warp_sum(sr);
        sa = warp_sum(sa);
        if (lane == 0) {
            num += sr;
            nabs += sa;
            nmax = fmax(nmax, fabs(sr));
        }
    }
    // block reduction
    we = warp_sum(we); wh = warp_sum(wh); wh2 = warp_sum(wh2);
    num = warp_sum(num); nabs = warp_sum(nabs); nmax = warp_max(nmax);
    fin = __all_sync(0xffffffffu, fin);
    const int w = threadIdx.x >> 5;
    __shared__ int sfin[8];
    if (lane == 0) {
        red[0][w] = we; red[1][w] = wh; red[2][w] = wh2; red[3][w] = num; red[4][w] = nabs; red[5][w] = nmax;
        sfin[w] = fin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double o[6] = {0, 0, 0, 0, 0, 0};
        int f = 1;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            for (int t = 0; t < 5; ++t) o[t] += red[t][q];
            o[5] = fmax(o[5], red[5][q]);
            f &= sfin[q];
        }
        double *p = partials + (int64_t)blockIdx.x * 7;
        for (int t = 0; t < 6; ++t) p[t] = o[t];
        p[6] = f ? 1.0 : 0.0;
    }
}

__global__ void k_diag_final(const double *partials, int nblocks, double eps_half_dv, double mu_half_dv, double *out)
{
    if (threadIdx.x != 0) return;
    double o[6] = {0, 0, 0, 0, 0, 0};
    double fin = 1.0;
    for (int b = 0; b < nblocks; ++b) {
        const double *p = partials + (int64_t)b * 7;
        for (int t = 0; t < 5; ++t) o[t] += p[t];
        o[5] = fmax(o[5], p[5]);
        fin = fmin(fin, p[6]);
    }
    out[0] = eps_half_dv * o[0] + mu_half_dv * o[1];   // invariant energy
    out[1] = eps_half_dv * o[0] + mu_half_dv * o[2];   // plain energy
    out[2] = o[3];                                      // number
    out[3] = o[5];                                      // max per cell
    out[4] = o[4];                                      // abs
    out[5] = fin;
}

cudaError_t launch_diag(cudaStream_t st, const DiagArgs &a, double *partials, int max_blocks, double *out)
{
    int blocks = max_blocks;
    if (a.precision == FDTD_F64)
        k_diag_partial<double><<<blocks, 256, 0, st>>>(a, partials);
    else
        k_diag_partial<float><<<blocks, 256, 0, st>>>(a, partials);
    k_diag_final<<<1, 32, 0, st>>>(partials, blocks, a.eps0_half_dv, a.mu0_half_dv, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ Poynting flux
// S = E x H through the six faces of an axis-aligned box at step n: E^n on
// the face's E-node plane; H time-centred, (H^{n-1/2} + H^{n+1/2}) / 2 with
// the vacuum curl of E^n, then averaged onto the plane from the H nodes on
// either side (nodes off the grid read 0).  All face points of all faces are
// one flat index space; each block keeps one FP64 sum per face.

template <typename T>
struct PoyntingView {
    const DiagArgs &a;
    __device__ double e(int q, int64_t i, int64_t j, int64_t k) const   // E_q at node (i,j,k), 0 off the grid
    {
        if (i < 0 || j < 0 || k < 0 || i >= a.nx || j >= a.ny || k >= a.nz) return 0.0;
        return ld<T>(a.f[q], (k * a.ny + j) * a.nx + i);
    }
    __device__ bool on(int64_t i, int64_t j, int64_t k) const
    {
        return i >= 0 && j >= 0 && k >= 0 && i < a.nx && j < a.ny && k < a.nz;
    }
    // time-centred H components at their own Yee positions (index of the node)
    __device__ double hx(int64_t i, int64_t j, int64_t k) const
    {
        if (!on(i, j, k)) return 0.0;
        const double curl = a.ndim == 2 ? e(2, i, j + 1, k) - e(2, i, j, k)
                                        : (e(2, i, j + 1, k) - e(2, i, j, k)) - (e(1, i, j, k + 1) - e(1, i, j, k));
        return ld<T>(a.f[3], (k * a.ny + j) * a.nx + i) - 0.5 * a.ch * curl;
    }
    __device__ double hy(int64_t i, int64_t j, int64_t k) const
    {
        if (!on(i, j, k)) return 0.0;
        const double curl = a.ndim == 2 ? -(e(2, i + 1, j, k) - e(2, i, j, k))
                                        : (e(0, i, j, k + 1) - e(0, i, j, k)) - (e(2, i + 1, j, k) - e(2, i, j, k));
        return ld<T>(a.f[4], (k * a.ny + j) * a.nx + i) - 0.5 * a.ch * curl;
    }
    __device__ double hz(int64_t i, int64_t j, int64_t k) const
    {
        if (!on(i, j, k)) return 0.0;
        const double curl = (e(1, i + 1, j, k) - e(1, i, j, k)) - (e(0, i, j + 1, k) - e(0, i, j, k));
        return ld<T>(a.f[5], (k * a.ny + j) * a.nx + i) - 0.5 * a.ch * curl;
    }
};

// Normal component of E x H at face point t of face f (before the area factor).
template <typename T>
__device__ double face_flux(const DiagArgs &a, const PoyntingBox &b, int f, int64_t t)
{
    const int ax = f >> 1;
    const int64_t p = b.plane[f];
    if (a.ndim == 1) {   // Ex(k) Hy averaged from k - 1/2 and k + 1/2
        const int64_t k = p;
        double hb = 0.0;
        for (int64_t kk = k - 1; kk <= k; ++kk) {
            if (kk < 0 || kk >= a.nz) continue;
            const double h = ld<T>(a.f[4], kk) - 0.5 * a.ch * (ld<T>(a.f[0], kk + 1) - ld<T>(a.f[0], kk));
            hb += 0.5 * h;
        }
        return k <= a.nz ? ld<T>(a.f[0], k) * hb : 0.0;
    }
    PoyntingView<T> v{a};
    // the two in-plane axes, lower-numbered first
    const int u = ax == 0 ? 1 : 0, w = ax == 2 ? 1 : 2;
    const int64_t nu = b.hi[u] - b.lo[u];
    int64_t c[3];
    c[ax] = p;
    c[u] = b.lo[u] + t % nu;
    c[w] = a.ndim == 2 ? 0 : b.lo[w] + t / nu;
    const int64_t i = c[0], j = c[1], k = c[2];
    if (a.ndim == 2) {
        const double ez = v.e(2, i, j, 0);
        if (ax == 0) return -ez * 0.5 * (v.hy(i - 1, j, 0) + v.hy(i, j, 0));   // S_x = -Ez Hy
        return ez * 0.5 * (v.hx(i, j - 1, 0) + v.hx(i, j, 0));                 // S_y =  Ez Hx
    }
    if (ax == 0)   // S_x = Ey Hz - Ez Hy
        return v.e(1, i, j, k) * 0.5 * (v.hz(i - 1, j, k) + v.hz(i, j, k)) -
               v.e(2, i, j, k) * 0.5 * (v.hy(i - 1, j, k) + v.hy(i, j, k));
    if (ax == 1)   // S_y = Ez Hx - Ex Hz
        return v.e(2, i, j, k) * 0.5 * (v.hx(i, j - 1, k) + v.hx(i, j, k)) -
               v.e(0, i, j, k) * 0.5 * (v.hz(i, j - 1, k) + v.hz(i, j, k));
    return v.e(0, i, j, k) * 0.5 * (v.hy(i, j, k - 1) + v.hy(i, j, k)) -   // S_z = Ex Hy - Ey Hx
           v.e(1, i, j, k) * 0.5 * (v.hx(i, j, k - 1) + v.hx(i, j, k));
}

template <typename T>
__global__ void __launch_bounds__(256) k_poynting_partial(DiagArgs a, PoyntingBox b, double *partials)
{
    __shared__ double red[6][8];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = tid; g < b.off[6]; g += nth) {
        int f = 0;
        while (g >= b.off[f + 1]) ++f;
        acc[f] += face_flux<T>(a, b, f, g - b.off[f]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int f = 0; f < 6; ++f) {
        const double s = warp_sum(acc[f]);
        if (lane == 0) red[f][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
        partials[(int64_t)blockIdx.x * 7 + threadIdx.x] = s;
    }
}

__global__ void k_poynting_final(const double *partials, int nblocks, double dA, double *out)
{
    if (threadIdx.x != 0) return;
    double o[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int f = 0; f < 6; ++f) o[f] += partials[(int64_t)b * 7 + f];
    for (int f = 0; f < 6; ++f) out[f] = o[f] * dA;
    out[6] = (o[1] - o[0] + o[3] - o[2] + o[5] - o[4]) * dA;
}

cudaError_t launch_poynting(cudaStream_t st, const DiagArgs &a, const PoyntingBox &b, double dA, double *partials,
                            int max_blocks, double *out)
{
    int blocks = (int)std::min<int64_t>(max_blocks, std::max<int64_t>(1, (b.off[6] + 255) / 256));
    if (a.precision == FDTD_F64)
        k_poynting_partial<double><<<blocks, 256, 0, st>>>(a, b, partials);
    else
        k_poynting_partial<float><<<blocks, 256, 0, st>>>(a, b, partials);
    k_poynting_final<<<1, 32, 0, st>>>(partials, blocks, dA, out);
    return cudaGetLastError();
}

}  // namespace fp

// ===================================================================
// Allocation-free variant of the diagnostics reduction.
//
// fdtd_diagnostics_noalloc() serves callers that cannot allocate device
// memory at the moment they need a diagnostic: monitoring or watchdog code
// that must not take the allocator's locks or trigger cudaMalloc's implicit
// device synchronisation, frameworks that route every device allocation
// through their own pool and forbid direct cudaMalloc, and code running close
// to the device's memory limit.  The caller passes the device arrays (inputs)
// and the result location (output); the per-tile partial sums live in the
// file-scope array below, which every GPU that loads this library keeps
// (kNoAllocMaxTiles * 7 + 8 doubles, about 459 KB) until the process exits.
//
// Work is split into fixed tiles (65536 field nodes or 16384 plasma slots
// each), one block per tile, so a call needs ceil(nodes / 65536) +
// ceil(slots / 16384) <= 8192 tiles; larger problems are rejected with
// FDTD_ERR_INVAL.  Every scratch entry a call reads is written earlier by
// the same call, so nothing has to be cleared between calls; calls share the
// array, and calls that overlap on the GPU (e.g. on two streams) race.
// Every call looks the array's device address up again (cudaGetSymbolAddress
// allocates nothing), so the address stays right after a cudaDeviceReset or a
// new primary context.
// ===================================================================

namespace fp {

constexpr int kNoAllocMaxTiles = 8192;
constexpr int64_t kNoAllocCellsPerTile = 65536;
constexpr int64_t kNoAllocSlotsPerTile = 16384;

// per-tile partial rows (7 doubles each, the layout k_diag_final reads) + the
// 6-double result area used when the caller wants the result on the host
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxTiles * 7 + 8];

template <typename T>
__global__ void __launch_bounds__(256) k_diag_tiles(DiagArgs a, int64_t field_tiles, double *partials)
{
    __shared__ double red[6][8];
    __shared__ int sfin[8];
    double we = 0, wh = 0, wh2 = 0, num = 0, nmax = 0, nabs = 0;
    int fin = 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t tile = blockIdx.x;
    if (tile < field_tiles) {
        const int64_t ncells = a.ndim == 1 ? a.nz + 1 : a.nx * a.ny * a.nz;
        const int64_t c0 = tile * kNoAllocCellsPerTile;
        const int64_t c1 = min(c0 + kNoAllocCellsPerTile, ncells);
        for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) field_terms<T>(a, c, we, wh, wh2, fin);
    } else {
        const int64_t s0 = (tile - field_tiles) * kNoAllocSlotsPerTile;
        const int64_t s1 = min(s0 + kNoAllocSlotsPerTile, a.nslots);
        for (int64_t r = s0 + w; r < s1; r += blockDim.x >> 5) {
            double sr = 0, sa = 0;
            for (int64_t j = lane; j < a.nnode; j += 32) {
                double v = df_val<T>(a, r, j);
                sr += v * a.dV[j];
                sa += fabs(v) * a.dV[j];
                fin &= isfinite(v);
            }
            sr = warp_sum(sr);
            sa = warp_sum(sa);
            if (lane == 0) {
                num += sr;
                nabs += sa;
                nmax = fmax(nmax, fabs(sr));
            }
        }
    }
    we = warp_sum(we); wh = warp_sum(wh); wh2 = warp_sum(wh2);
    num = warp_sum(num); nabs = warp_sum(nabs); nmax = warp_max(nmax);
    fin = __all_sync(0xffffffffu, fin);
    if (lane == 0) {
        red[0][w] = we; red[1][w] = wh; red[2][w] = wh2; red[3][w] = num; red[4][w] = nabs; red[5][w] = nmax;
        sfin[w] = fin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double o[6] = {0, 0, 0, 0, 0, 0};
        int f = 1;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            for (int t = 0; t < 5; ++t) o[t] += red[t][q];
            o[5] = fmax(o[5], red[5][q]);
            f &= sfin[q];
        }
        double *p = partials + tile * 7;
        for (int t = 0; t < 6; ++t) p[t] = o[t];
        p[6] = f ? 1.0 : 0.0;
    }
}

}  // namespace fp

extern "C" int fdtd_diagnostics_noalloc(const fdtd_diag_arrays *in, double *out, int out_is_device, void *stream)
{
    using namespace fp;
    if (!in || !out) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_diagnostics_noalloc: NULL argument");
    if (in->ndim < 1 || in->ndim > 3 || (in->precision != FDTD_F32 && in->precision != FDTD_F64) ||
        !(in->dx > 0) || !(in->courant > 0))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_diagnostics_noalloc: bad ndim, precision, dx or courant");
    const int64_t nx = in->ndim >= 2 ? in->nx : 1, ny = in->ndim >= 2 ? in->ny : 1;
    const int64_t nz = in->ndim == 2 ? 1 : in->nz;
    if (nx < 1 || ny < 1 || nz < 1) return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_diagnostics_noalloc: bad sizes");
    static const int need1[6] = {1, 0, 0, 0, 1, 0}, need2[6] = {0, 0, 1, 1, 1, 0};
    for (int q = 0; q < 6; ++q) {
        const bool need = in->ndim == 3 || (in->ndim == 1 ? need1[q] : need2[q]);
        if (need && !in->fields[q])
            return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_diagnostics_noalloc: a field array is NULL");
    }
    if (in->nslots < 0 || (in->nslots > 0 && (!in->df || !in->dV || in->nnode < 1)) ||
        (in->nslots > 0 && in->f_dtype != FDTD_DF_F32 && in->f_dtype != FDTD_DF_BF16 && in->f_dtype != FDTD_DF_F64))
        return fp_set_global_error(FDTD_ERR_INVAL, "fdtd_diagnostics_noalloc: bad delta-f description");
    const int64_t ncells = in->ndim == 1 ? nz + 1 : nx * ny * nz;
    const int64_t field_tiles = (ncells + kNoAllocCellsPerTile - 1) / kNoAllocCellsPerTile;
    const int64_t slot_tiles = (in->nslots + kNoAllocSlotsPerTile - 1) / kNoAllocSlotsPerTile;
    const int64_t ntiles = field_tiles + slot_tiles;
    if (ntiles > kNoAllocMaxTiles) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "fdtd_diagnostics_noalloc: problem needs %lld tiles of scratch, the fixed maximum is %d "
                 "(%lld field nodes / 65536 + %lld slots / 16384); use fdtd_plasma_diagnostics",
                 (long long)ntiles, kNoAllocMaxTiles, (long long)ncells, (long long)in->nslots);
        return fp_set_global_error(FDTD_ERR_INVAL, msg);
    }
    // the device address of the file-scope scratch array on the current device
    // (looked up on every call: it allocates nothing and survives device resets)
    double *scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&scratch, g_noalloc_scratch);
    if (e != cudaSuccess || !scratch)
        return fp_set_global_error(FDTD_ERR_CUDA, "fdtd_diagnostics_noalloc: cudaGetSymbolAddress failed");
    const double c0 = 299792458.0, eps0 = 8.8541878128e-12, mu0 = 1.0 / (eps0 * c0 * c0);
    const double dt = in->courant * in->dx / c0;
    const double dvol = std::pow(in->dx, in->ndim);
    DiagArgs a{};
    a.ndim = in->ndim;
    a.nx = nx; a.ny = ny; a.nz = nz;
    for (int q = 0; q < 6; ++q) a.f[q] = in->fields[q];
    a.precision = in->precision;
    a.ch = dt / (mu0 * in->dx);
    a.eps0_half_dv = 0.5 * eps0 * dvol;
    a.mu0_half_dv = 0.5 * mu0 * dvol;
    a.df = in->df;
    a.nslots = in->nslots;
    a.nnode = in->nnode;
    a.pitch = (int)in->nnode;    // caller rows are packed
    a.f_dtype = in->f_dtype;
    a.dV = in->dV;
    cudaStream_t st = (cudaStream_t)stream;
    double *res = out_is_device ? out : scratch + (int64_t)kNoAllocMaxTiles * 7;
    if (in->precision == FDTD_F64)
        k_diag_tiles<double><<<(unsigned)ntiles, 256, 0, st>>>(a, field_tiles, scratch);
    else
        k_diag_tiles<float><<<(unsigned)ntiles, 256, 0, st>>>(a, field_tiles, scratch);
    k_diag_final<<<1, 32, 0, st>>>(scratch, (int)ntiles, a.eps0_half_dv, a.mu0_half_dv, res);
    e = cudaGetLastError();
    if (e == cudaSuccess && !out_is_device) {
        e = cudaMemcpyAsync(out, res, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return fp_set_global_error(FDTD_ERR_CUDA, cudaGetErrorString(e));
    return FDTD_OK;
}

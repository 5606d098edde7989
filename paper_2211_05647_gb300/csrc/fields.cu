// fields.cu -- Yee curl-stencil kernels (Sec. 2, Eq. 1-6) with the CPML
// auxiliary recursion psi <- b psi + a dF and the 1/kappa-scaled curl (Eq. 7-12),
// the soft source and the first-order Mur ends.
//
// One thread per Yee cell, x fastest across the warp so every field access is
// a coalesced 128-byte row segment (the block shape is chosen at launch, by
// default 32 x 8 in 2-D and 32 x 4 x 2 in 3-D, or by the autotuner); the +-1 neighbours along y / z are the
// rows the neighbouring warps load anyway (served by L1/L2).  PEC walls are
// the nodes the kernels never write; high-side neighbours past the last
// stored node read as 0 (PEC ghosts).  The plasma current has already been
// subtracted from E in place by the kinetic kernel, so the E kernels only add
// the curl.
#include <type_traits>

#include "cp_async.cuh"
#include "stencil_common.cuh"

namespace fp {


// ------------------------------------------------------------------- 1-D

template <typename T>
__global__ void k_h1d(const T *__restrict__ ex, T *__restrict__ hy, T *__restrict__ mur, int64_t nz, T ch, Source src,
                      const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) write_source(src, d_step, kstep);
    if (k < nz) hy[k] -= ch * (ex[k + 1] - ex[k]);   // mu0 dHy/dt = -dEx/dz
    if (mur) {                                       // E_1^n and E_{nz-1}^n for the Mur ends
        if (k == 1) mur[0] = ex[1];
        if (k == nz - 1) mur[1] = ex[nz - 1];
    }
}

// E update of the interior nodes; with Mur ends (mur != nullptr) the thread that
// advances E_1 (E_{nz-1}) also sets E_0^{n+1} = E_1^n + m (E_1^{n+1} - E_0^n)
// (and the mirror image at nz), so a step needs no separate boundary launch.
template <typename T>
__global__ void k_e1d(T *__restrict__ ex, const T *__restrict__ hy, int64_t nz, T ce, Source src,
                      const int64_t *__restrict__ d_step, int kstep, const T *__restrict__ mur, T m)
{
    pdl_enter();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 1 || k >= nz) return;
    T v = ex[k] - ce * (hy[k] - hy[k - 1]);           // eps0 dEx/dt = -dHy/dz - Jx
    if (src.kind && k == src.k) v += (T)*src.val;
    ex[k] = v;
    if (mur) {
        if (k == 1) ex[0] = mur[0] + m * (v - ex[0]);
        if (k == nz - 1) ex[nz] = mur[1] + m * (v - ex[nz]);
    }
}

// ------------------------------------------------------------------- 2-D TMz

// (2-D CPML cell updates h2d_pml / e2d_pml: stencil_common.cuh)

template <typename T>
__global__ void __launch_bounds__(256) k_h2d(const T *__restrict__ ez, T *__restrict__ hx, T *__restrict__ hy,
                                             int64_t nx, int64_t ny, T ch, T cph, Cpml<T> cp, Source src,
                                             const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i == 0 && j == 0) write_source(src, d_step, kstep);
    if (i >= nx || j >= ny) return;
    const int64_t c = j * nx + i;
    const T e = ez[c];
    const T dEy = (j + 1 < ny ? ez[c + nx] : T(0)) - e;   // dEz along y at (i, j+1/2)
    const T dEx = (i + 1 < nx ? ez[c + 1] : T(0)) - e;    // dEz along x at (i+1/2, j)
    T hxv = hx[c], hyv = hy[c];
    if (cp.L == 0) {
        hxv = hx_plain(hxv, ch, dEy);                     // mu0 dHx/dt = -dEz/dy
        hyv = hy_plain(hyv, ch, dEx);                     // mu0 dHy/dt = +dEz/dx
    } else {
        h2d_pml<T>(cp, nx, ny, i, j, ch, cph, dEy, dEx, hxv, hyv);
    }
    hx[c] = hxv;
    hy[c] = hyv;
}

template <typename T>
__global__ void __launch_bounds__(256) k_e2d(T *__restrict__ ez, const T *__restrict__ hx, const T *__restrict__ hy,
                                             int64_t nx, int64_t ny, T ce, T cpe, Cpml<T> cp, Source src,
                                             const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i < 1 || j < 1 || i >= nx || j >= ny) return;
    const int64_t c = j * nx + i;
    // E^n is read before any psi store: the compiler cannot prove the psi
    // slabs and Ez apart, so a later load would be a second round trip.
    const T ezc = ez[c];
    const T dHx = hy[c] - hy[c - 1];     // dHy along x
    const T dHy = hx[c] - hx[c - nx];    // dHx along y
    // eps0 dEz/dt = dHy/dx - dHx/dy - Jz
    const T upd = cp.L == 0 ? e2d_term(ce, dHx, dHy) : e2d_pml<T>(cp, nx, ny, i, j, ce, cpe, dHx, dHy);
    T v = rn_add(ezc, upd);
    if (src.kind && i == src.i && j == src.j) v = rn_add(v, (T)*src.val);
    ez[c] = v;
}

// ------------------------------------------------------------------- 3-D
// (psi slots and slab layouts: stencil_common.cuh)


template <typename T>
__global__ void __launch_bounds__(256) k_h3d(const T *__restrict__ ex, const T *__restrict__ ey,
                                             const T *__restrict__ ez, T *__restrict__ hx, T *__restrict__ hy,
                                             T *__restrict__ hz, int64_t nx, int64_t ny, int64_t nz, T ch, T cph,
                                             Cpml<T> cp, Source src, const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t k = (int64_t)blockIdx.z * blockDim.z + threadIdx.z;
    if (i == 0 && j == 0 && k == 0) write_source(src, d_step, kstep);
    if (i >= nx || j >= ny || k >= nz) return;
    const int64_t sxy = nx * ny;
    const int64_t c = k * sxy + j * nx + i;
    const T exc = ex[c], eyc = ey[c], ezc = ez[c];
    const T dEz_y = (j + 1 < ny ? ez[c + nx] : T(0)) - ezc;
    const T dEy_z = (k + 1 < nz ? ey[c + sxy] : T(0)) - eyc;
    const T dEx_z = (k + 1 < nz ? ex[c + sxy] : T(0)) - exc;
    const T dEz_x = (i + 1 < nx ? ez[c + 1] : T(0)) - ezc;
    const T dEy_x = (i + 1 < nx ? ey[c + 1] : T(0)) - eyc;
    const T dEx_y = (j + 1 < ny ? ex[c + nx] : T(0)) - exc;
    T hxv = hx[c], hyv = hy[c], hzv = hz[c];
    if (cp.L == 0) {
        // mu0 dH/dt = -curl E
        hxv -= ch * (dEz_y - dEy_z);
        hyv -= ch * (dEx_z - dEz_x);
        hzv -= ch * (dEy_x - dEx_y);
    } else {
        h3d_pml<T>(cp, nx, ny, nz, i, j, k, ch, cph, dEz_y, dEy_z, dEx_z, dEz_x, dEy_x, dEx_y, hxv, hyv, hzv);
    }
    hx[c] = hxv;
    hy[c] = hyv;
    hz[c] = hzv;
}


template <typename T>
__global__ void __launch_bounds__(256) k_e3d(T *__restrict__ ex, T *__restrict__ ey, T *__restrict__ ez,
                                             const T *__restrict__ hx, const T *__restrict__ hy,
                                             const T *__restrict__ hz, int64_t nx, int64_t ny, int64_t nz, T ce,
                                             T cpe, Cpml<T> cp, Source src, const int64_t *__restrict__ d_step,
                                             int kstep)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t k = (int64_t)blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const int64_t sxy = nx * ny;
    const int64_t c = k * sxy + j * nx + i;
    const T hxc = hx[c], hyc = hy[c], hzc = hz[c];
    // E^n is read up front, before any psi store (see k_e2d).
    const T exc = ex[c], eyc = ey[c], ezc = ez[c];
    const T dHz_y = j > 0 ? hzc - hz[c - nx] : T(0);
    const T dHy_z = k > 0 ? hyc - hy[c - sxy] : T(0);
    const T dHx_z = k > 0 ? hxc - hx[c - sxy] : T(0);
    const T dHz_x = i > 0 ? hzc - hz[c - 1] : T(0);
    const T dHy_x = i > 0 ? hyc - hy[c - 1] : T(0);
    const T dHx_y = j > 0 ? hxc - hx[c - nx] : T(0);
    T ux, uy, uz;
    if (cp.L == 0) {
        // eps0 dE/dt = curl H (- J, already applied to Ex)
        ux = ce * (dHz_y - dHy_z);
        uy = ce * (dHx_z - dHz_x);
        uz = ce * (dHy_x - dHx_y);
    } else {
        e3d_pml<T>(cp, nx, ny, nz, i, j, k, ce, cpe, dHz_y, dHy_z, dHx_z, dHz_x, dHy_x, dHx_y, ux, uy, uz);
    }
    if (j > 0 && k > 0) {
        T v = exc + ux;
        if (src.kind && source_hits_3d(src, i, j, k)) v += (T)*src.val;
        ex[c] = v;
    }
    if (i > 0 && k > 0) ey[c] = eyc + uy;
    if (i > 0 && j > 0) ez[c] = ezc + uz;
}

// ------------------------------------------------- FP32, four cells per thread
// Rows of a multiple of 4 cells: each thread owns 4 consecutive x cells and
// moves them with 16-byte loads and stores, so a warp covers a 512-byte row
// segment per field and a quarter of the instructions per cell.  The x
// neighbour one past the quad (x + 1 for H, x - 1 for E) comes from the
// adjacent lane by a shuffle; a lane whose neighbour quad sits in another
// warp or row loads that one value directly.  Cells inside a CPML slab take
// the same per-cell code as the scalar kernels.  Block sizes are a multiple
// of 32 threads (the launcher checks), so every shuffle has all lanes.

struct Q4 {
    float v[4];
};
__device__ __forceinline__ Q4 ld4(const float *p)
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    return Q4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st4(float *p, const Q4 &q)
{
    *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ Q4 ld4_if(bool ok, const float *p) { return ok ? ld4(p) : Q4{{0.f, 0.f, 0.f, 0.f}}; }
__device__ __forceinline__ unsigned lane_id()
{
    return (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) & 31u;
}

__global__ void __launch_bounds__(256) k_h2d_v4(const float *__restrict__ ez, float *__restrict__ hx,
                                                float *__restrict__ hy, int64_t nx, int64_t ny, float ch, float cph,
                                                Cpml<float> cp, Source src, const int64_t *__restrict__ d_step,
                                                int kstep)
{
    pdl_enter();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (q == 0 && j == 0) write_source(src, d_step, kstep);
    const int64_t i0 = 4 * q;
    const bool live = i0 < nx && j < ny;
    const int64_t c = live ? j * nx + i0 : 0;
    // the lane at the end of a warp row loads its x neighbour with the others,
    // not after the shuffle (that would be a second round trip for the warp)
    const bool edge = threadIdx.x + 1 >= blockDim.x || lane_id() == 31;
    const float eh = edge && live && i0 + 4 < nx ? ez[c + 4] : 0.f;
    const Q4 E = ld4_if(live, ez + c);
    const Q4 Ey = ld4_if(live && j + 1 < ny, ez + c + nx);
    Q4 Hx = ld4_if(live, hx + c), Hy = ld4_if(live, hy + c);   // every load before the shuffle
    float er = __shfl_down_sync(0xffffffffu, E.v[0], 1);
    if (edge) er = eh;
    if (!live) return;
    const int L = cp.L;
    const bool pml = L > 0 && (in_slab<float>(j, ny, L) || i0 < L || i0 + 3 >= nx - L);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float dEy = Ey.v[e] - E.v[e];
        const float dEx = (e < 3 ? E.v[e + 1] : er) - E.v[e];
        if (!pml) {
            Hx.v[e] = hx_plain(Hx.v[e], ch, dEy);
            Hy.v[e] = hy_plain(Hy.v[e], ch, dEx);
        } else {
            h2d_pml<float>(cp, nx, ny, i0 + e, j, ch, cph, dEy, dEx, Hx.v[e], Hy.v[e]);
        }
    }
    st4(hx + c, Hx);
    st4(hy + c, Hy);
}

__global__ void __launch_bounds__(256) k_e2d_v4(float *__restrict__ ez, const float *__restrict__ hx,
                                                const float *__restrict__ hy, int64_t nx, int64_t ny, float ce,
                                                float cpe, Cpml<float> cp, Source src,
                                                const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t i0 = 4 * q;
    const bool live = i0 < nx && j < ny;
    const int64_t c = live ? j * nx + i0 : 0;
    const bool edge = threadIdx.x == 0 || lane_id() == 0;
    const float hh = edge && live && i0 > 0 ? hy[c - 1] : 0.f;
    const Q4 Hy = ld4_if(live, hy + c);
    const bool row = live && j >= 1;   // row 0 is the PEC wall
    const Q4 Hx = ld4_if(row, hx + c), Hxm = ld4_if(row, hx + c - nx);
    Q4 E = ld4_if(row, ez + c);        // every load before the shuffle
    float hl = __shfl_up_sync(0xffffffffu, Hy.v[3], 1);
    if (edge) hl = hh;
    if (!row) return;
    const int L = cp.L;
    const bool pml = L > 0 && (in_slab<float>(j, ny, L) || i0 < L || i0 + 3 >= nx - L);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = i0 + e;
        if (i < 1) continue;      // column 0 is the PEC wall
        const float dHx = Hy.v[e] - (e > 0 ? Hy.v[e - 1] : hl);
        const float dHy = Hx.v[e] - Hxm.v[e];
        E.v[e] = rn_add(E.v[e], pml ? e2d_pml<float>(cp, nx, ny, i, j, ce, cpe, dHx, dHy) : e2d_term(ce, dHx, dHy));
        if (src.kind && i == src.i && j == src.j) E.v[e] = rn_add(E.v[e], (float)*src.val);
    }
    st4(ez + c, E);
}

// 3-D CPML with four cells per thread: a row lies wholly inside or outside a
// y or z slab, so those psi recursions run for the whole quad with 16-byte
// psi accesses and no divergence within the warp.  The x slab cuts rows, and
// is applied per cell as a correction to the update with kappa_x = 1 and no
// x psi: (kappa_x^-1 - 1) times the x difference, plus the x psi term.

__global__ void __launch_bounds__(256) k_h3d_v4(const float *__restrict__ ex, const float *__restrict__ ey,
                                                const float *__restrict__ ez, float *__restrict__ hx,
                                                float *__restrict__ hy, float *__restrict__ hz, int64_t nx,
                                                int64_t ny, int64_t nz, float ch, float cph, Cpml<float> cp,
                                                Source src, const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t k = (int64_t)blockIdx.z * blockDim.z + threadIdx.z;
    if (q == 0 && j == 0 && k == 0) write_source(src, d_step, kstep);
    const int64_t i0 = 4 * q, sxy = nx * ny;
    const bool live = i0 < nx && j < ny && k < nz;
    const int64_t c = live ? k * sxy + j * nx + i0 : 0;
    const bool edge = threadIdx.x + 1 >= blockDim.x || lane_id() == 31;
    const bool hin = edge && live && i0 + 4 < nx;
    const float ezh = hin ? ez[c + 4] : 0.f, eyh = hin ? ey[c + 4] : 0.f;
    const Q4 Ex = ld4_if(live, ex + c), Ey = ld4_if(live, ey + c), Ez = ld4_if(live, ez + c);
    const Q4 Ezy = ld4_if(live && j + 1 < ny, ez + c + nx), Exy = ld4_if(live && j + 1 < ny, ex + c + nx);
    const Q4 Eyz = ld4_if(live && k + 1 < nz, ey + c + sxy), Exz = ld4_if(live && k + 1 < nz, ex + c + sxy);
    Q4 Hx = ld4_if(live, hx + c), Hy = ld4_if(live, hy + c), Hz = ld4_if(live, hz + c);   // all loads first
    float ezr = __shfl_down_sync(0xffffffffu, Ez.v[0], 1);
    float eyr = __shfl_down_sync(0xffffffffu, Ey.v[0], 1);
    if (edge) {
        ezr = ezh;
        eyr = eyh;
    }
    if (!live) return;
    float dEz_y[4], dEy_z[4], dEx_z[4], dEz_x[4], dEy_x[4], dEx_y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        dEz_y[e] = Ezy.v[e] - Ez.v[e];
        dEy_z[e] = Eyz.v[e] - Ey.v[e];
        dEx_z[e] = Exz.v[e] - Ex.v[e];
        dEz_x[e] = (e < 3 ? Ez.v[e + 1] : ezr) - Ez.v[e];
        dEy_x[e] = (e < 3 ? Ey.v[e + 1] : eyr) - Ey.v[e];
        dEx_y[e] = Exy.v[e] - Ex.v[e];
    }
    const int L = cp.L;
    if (L == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {   // mu0 dH/dt = -curl E
            Hx.v[e] -= ch * (dEz_y[e] - dEy_z[e]);
            Hy.v[e] -= ch * (dEx_z[e] - dEz_x[e]);
            Hz.v[e] -= ch * (dEy_x[e] - dEx_y[e]);
        }
    } else {
        float ky = 1.f, kz = 1.f;
        Q4 p6{}, p7{}, p9{}, p11{};
        if (in_slab<float>(j, ny, L)) {   // slots 6 (Hx, dEz/dy) and 11 (Hz, dEx/dy)
            const int64_t o = (k * (2 * L) + slab_slot<float>(j, ny, L)) * nx + i0;
            const float bb = cp.bh[1][j], aa = cp.ah[1][j];
            ky = cp.ikh[1][j];
            const Q4 s6 = ld4(cp.psi[6] + o), s11 = ld4(cp.psi[11] + o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                p6.v[e] = bb * s6.v[e] + aa * dEz_y[e];
                p11.v[e] = bb * s11.v[e] + aa * dEx_y[e];
            }
            st4(cp.psi[6] + o, p6);
            st4(cp.psi[11] + o, p11);
        }
        if (in_slab<float>(k, nz, L)) {   // slots 7 (Hx, dEy/dz) and 9 (Hy, dEx/dz)
            const int64_t o = ((int64_t)slab_slot<float>(k, nz, L) * ny + j) * nx + i0;
            const float bb = cp.bh[2][k], aa = cp.ah[2][k];
            kz = cp.ikh[2][k];
            const Q4 s7 = ld4(cp.psi[7] + o), s9 = ld4(cp.psi[9] + o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                p7.v[e] = bb * s7.v[e] + aa * dEy_z[e];
                p9.v[e] = bb * s9.v[e] + aa * dEx_z[e];
            }
            st4(cp.psi[7] + o, p7);
            st4(cp.psi[9] + o, p9);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            Hx.v[e] -= ch * (dEz_y[e] * ky - dEy_z[e] * kz) + cph * (p6.v[e] - p7.v[e]);
            Hy.v[e] -= ch * (dEx_z[e] * kz - dEz_x[e]) + cph * p9.v[e];
            Hz.v[e] -= ch * (dEy_x[e] - dEx_y[e] * ky) - cph * p11.v[e];
        }
        if (i0 < L || i0 + 3 >= nx - L) {   // slots 8 (Hy, dEz/dx) and 10 (Hz, dEy/dx)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t i = i0 + e;
                if (!in_slab<float>(i, nx, L)) continue;
                const float bb = cp.bh[0][i], aa = cp.ah[0][i], kx1 = cp.ikh[0][i] - 1.f;
                const int64_t o = (k * ny + j) * (2 * L) + slab_slot<float>(i, nx, L);
                const float p8 = bb * cp.psi[8][o] + aa * dEz_x[e];
                const float p10 = bb * cp.psi[10][o] + aa * dEy_x[e];
                cp.psi[8][o] = p8;
                cp.psi[10][o] = p10;
                Hy.v[e] += ch * dEz_x[e] * kx1 + cph * p8;
                Hz.v[e] -= ch * dEy_x[e] * kx1 + cph * p10;
            }
        }
    }
    st4(hx + c, Hx);
    st4(hy + c, Hy);
    st4(hz + c, Hz);
}

__global__ void __launch_bounds__(256) k_e3d_v4(float *__restrict__ ex, float *__restrict__ ey,
                                                float *__restrict__ ez, const float *__restrict__ hx,
                                                const float *__restrict__ hy, const float *__restrict__ hz,
                                                int64_t nx, int64_t ny, int64_t nz, float ce, float cpe,
                                                Cpml<float> cp, Source src, const int64_t *__restrict__ d_step,
                                                int kstep)
{
    pdl_enter();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t k = (int64_t)blockIdx.z * blockDim.z + threadIdx.z;
    const int64_t i0 = 4 * q, sxy = nx * ny;
    const bool live = i0 < nx && j < ny && k < nz;
    const int64_t c = live ? k * sxy + j * nx + i0 : 0;
    const bool edge = threadIdx.x == 0 || lane_id() == 0;
    const bool hin = edge && live && i0 > 0;
    const float hzh = hin ? hz[c - 1] : 0.f, hyh = hin ? hy[c - 1] : 0.f;
    const Q4 Hx = ld4_if(live, hx + c), Hy = ld4_if(live, hy + c), Hz = ld4_if(live, hz + c);
    const Q4 Hzy = ld4_if(live && j > 0, hz + c - nx), Hxy = ld4_if(live && j > 0, hx + c - nx);
    const Q4 Hyz = ld4_if(live && k > 0, hy + c - sxy), Hxz = ld4_if(live && k > 0, hx + c - sxy);
    // E^n too, before the shuffles and any psi store (see k_e2d)
    Q4 Ex = ld4_if(live, ex + c), Ey = ld4_if(live, ey + c), Ez = ld4_if(live, ez + c);
    float hzl = __shfl_up_sync(0xffffffffu, Hz.v[3], 1);
    float hyl = __shfl_up_sync(0xffffffffu, Hy.v[3], 1);
    if (edge) {
        hzl = hzh;
        hyl = hyh;
    }
    if (!live) return;
    float dHz_y[4], dHy_z[4], dHx_z[4], dHz_x[4], dHy_x[4], dHx_y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool xi = i0 + e > 0;
        dHz_y[e] = j > 0 ? Hz.v[e] - Hzy.v[e] : 0.f;
        dHy_z[e] = k > 0 ? Hy.v[e] - Hyz.v[e] : 0.f;
        dHx_z[e] = k > 0 ? Hx.v[e] - Hxz.v[e] : 0.f;
        dHz_x[e] = xi ? Hz.v[e] - (e > 0 ? Hz.v[e - 1] : hzl) : 0.f;
        dHy_x[e] = xi ? Hy.v[e] - (e > 0 ? Hy.v[e - 1] : hyl) : 0.f;
        dHx_y[e] = j > 0 ? Hx.v[e] - Hxy.v[e] : 0.f;
    }
    float ux[4], uy[4], uz[4];
    const int L = cp.L;
    if (L == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {   // eps0 dE/dt = curl H (- J, already applied to Ex)
            ux[e] = ce * (dHz_y[e] - dHy_z[e]);
            uy[e] = ce * (dHx_z[e] - dHz_x[e]);
            uz[e] = ce * (dHy_x[e] - dHx_y[e]);
        }
    } else {
        float ky = 1.f, kz = 1.f;
        Q4 p0{}, p1{}, p3{}, p5{};
        if (in_slab<float>(j, ny, L)) {   // slots 0 (Ex, dHz/dy) and 5 (Ez, dHx/dy)
            const int64_t o = (k * (2 * L) + slab_slot<float>(j, ny, L)) * nx + i0;
            const float bb = cp.be[1][j], aa = cp.ae[1][j];
            ky = cp.ike[1][j];
            const Q4 s0 = ld4(cp.psi[0] + o), s5 = ld4(cp.psi[5] + o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                p0.v[e] = bb * s0.v[e] + aa * dHz_y[e];
                p5.v[e] = bb * s5.v[e] + aa * dHx_y[e];
            }
            st4(cp.psi[0] + o, p0);
            st4(cp.psi[5] + o, p5);
        }
        if (in_slab<float>(k, nz, L)) {   // slots 1 (Ex, dHy/dz) and 3 (Ey, dHx/dz)
            const int64_t o = ((int64_t)slab_slot<float>(k, nz, L) * ny + j) * nx + i0;
            const float bb = cp.be[2][k], aa = cp.ae[2][k];
            kz = cp.ike[2][k];
            const Q4 s1 = ld4(cp.psi[1] + o), s3 = ld4(cp.psi[3] + o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                p1.v[e] = bb * s1.v[e] + aa * dHy_z[e];
                p3.v[e] = bb * s3.v[e] + aa * dHx_z[e];
            }
            st4(cp.psi[1] + o, p1);
            st4(cp.psi[3] + o, p3);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ux[e] = ce * (dHz_y[e] * ky - dHy_z[e] * kz) + cpe * (p0.v[e] - p1.v[e]);
            uy[e] = ce * (dHx_z[e] * kz - dHz_x[e]) + cpe * p3.v[e];
            uz[e] = ce * (dHy_x[e] - dHx_y[e] * ky) - cpe * p5.v[e];
        }
        if (i0 < L || i0 + 3 >= nx - L) {   // slots 2 (Ey, dHz/dx) and 4 (Ez, dHy/dx)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t i = i0 + e;
                if (!in_slab<float>(i, nx, L)) continue;
                const float bb = cp.be[0][i], aa = cp.ae[0][i], kx1 = cp.ike[0][i] - 1.f;
                const int64_t o = (k * ny + j) * (2 * L) + slab_slot<float>(i, nx, L);
                const float p2 = bb * cp.psi[2][o] + aa * dHz_x[e];
                const float p4 = bb * cp.psi[4][o] + aa * dHy_x[e];
                cp.psi[2][o] = p2;
                cp.psi[4][o] = p4;
                uy[e] -= ce * dHz_x[e] * kx1 + cpe * p2;
                uz[e] += ce * dHy_x[e] * kx1 + cpe * p4;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = i0 + e;
        if (j > 0 && k > 0) {
            Ex.v[e] += ux[e];
            if (src.kind && source_hits_3d(src, i, j, k)) Ex.v[e] += (float)*src.val;
        }
        if (i > 0 && k > 0) Ey.v[e] += uy[e];
        if (i > 0 && j > 0) Ez.v[e] += uz[e];
    }
    st4(ex + c, Ex);
    st4(ey + c, Ey);
    st4(ez + c, Ez);
}

// ------------------------------------------ 3-D fused E^{n+1} + H^{n+3/2} (FP32)
// The E update of step n and the H update of step n+1 in one pass: a block owns
// a 32 x 8 column tile and marches up its z range; per plane it stages H^{n+1/2}
// (with the -x / -y halo), E' (E^n after the current density term, with the
// +x / +y halo) in shared memory, forms E^{n+1} on the tile and its +x / +y halo
// (the halo values are recomputed, not exchanged), stores the tile's E^{n+1},
// then forms H^{n+3/2} of the plane below from the two staged E^{n+1} planes.
// Everything is read from field / psi set `in` and written to set `out`, so no
// block reads what another block writes in the same launch.  The source term
// of E^{n+1} is evaluated per block; block (0,0,0) also stores g(t^{n+2}) for a
// following unfused E update.  DRAM: fields read once and written once per step
// (12 x 4 B per cell) instead of twice read and once written per half step.

constexpr int kEhX = 32, kEhY = 8;

struct FieldPtrs {
    const float *ex, *ey, *ez, *hx, *hy, *hz;
};
struct FieldOut {
    float *ex, *ey, *ez, *hx, *hy, *hz;
};
struct PsiOut {
    float *psi[12];
};

__global__ void __launch_bounds__(kEhX * kEhY, 3) k_eh3d(FieldPtrs in, FieldOut out, int64_t nx, int64_t ny, int64_t nz,
                                                     int tz, float ce, float cpe, float ch, float cph, Cpml<float> cin,
                                                     PsiOut pout, Source src, const int64_t *__restrict__ d_step,
                                                     int kstep)
{
    pdl_enter();
    __shared__ float sH[2][3][kEhY + 2][kEhX + 2];   // H^{n+1/2}: x0-1..x0+32, y0-1..y0+8
    __shared__ float sEp[3][kEhY + 1][kEhX + 1];     // E': x0..x0+32, y0..y0+8
    __shared__ float sE[2][3][kEhY + 1][kEhX + 1];   // E^{n+1}: x0..x0+32, y0..y0+8
    __shared__ float s_g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kEhX + tx;
    const int64_t x0 = (int64_t)blockIdx.x * kEhX, y0 = (int64_t)blockIdx.y * kEhY, z0 = (int64_t)blockIdx.z * tz;
    const int64_t z1 = min(z0 + (int64_t)tz, nz);
    const int64_t n1 = *d_step + kstep + 1;   // E^{n+1} is at t^{n+1}
    if (tid == 0) {
        s_g = src.kind && src.k >= z0 && src.k <= z1 ? (float)source_value(src, (double)n1 * src.dt) : 0.f;
        if (src.kind && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            *src.val = source_value(src, (double)(n1 + 1) * src.dt);
    }
    const int64_t sxy = nx * ny;
    // Staging of one plane: each thread fetches its share of the plane's H (with the -x / -y halo) and E'
    // (with the +x / +y halo) into registers, and later commits them to shared memory, so the global loads
    // of plane k+2 are in flight while plane k+1 is computed.
    constexpr int NH = ((kEhY + 2) * (kEhX + 2) + kEhX * kEhY - 1) / (kEhX * kEhY);
    constexpr int NE = ((kEhY + 1) * (kEhX + 1) + kEhX * kEhY - 1) / (kEhX * kEhY);
    float rh[NH][3], re[NE][3];
    auto fetch = [&](int64_t k) {
#pragma unroll
        for (int q = 0; q < NH; ++q) {
            const int r = tid + q * kEhX * kEhY;
            const int rx = r % (kEhX + 2), ry = r / (kEhX + 2);
            const int64_t i = x0 - 1 + rx, j = y0 - 1 + ry;
            const bool ok = r < (kEhY + 2) * (kEhX + 2) && k >= 0 && k < nz && i >= 0 && i < nx && j >= 0 && j < ny;
            const int64_t c = ok ? k * sxy + j * nx + i : 0;
            rh[q][0] = ok ? in.hx[c] : 0.f;
            rh[q][1] = ok ? in.hy[c] : 0.f;
            rh[q][2] = ok ? in.hz[c] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            const int r = tid + q * kEhX * kEhY;
            const int rx = r % (kEhX + 1), ry = r / (kEhX + 1);
            const int64_t i = x0 + rx, j = y0 + ry;
            const bool ok = r < (kEhY + 1) * (kEhX + 1) && k >= 0 && k < nz && i < nx && j < ny;
            const int64_t c = ok ? k * sxy + j * nx + i : 0;
            re[q][0] = ok ? in.ex[c] : 0.f;
            re[q][1] = ok ? in.ey[c] : 0.f;
            re[q][2] = ok ? in.ez[c] : 0.f;
        }
    };
    auto commit = [&](int b) {   // H into sH[b], E' into sEp
#pragma unroll
        for (int q = 0; q < NH; ++q) {
            const int r = tid + q * kEhX * kEhY;
            if (r < (kEhY + 2) * (kEhX + 2)) {
                const int rx = r % (kEhX + 2), ry = r / (kEhX + 2);
                sH[b][0][ry][rx] = rh[q][0];
                sH[b][1][ry][rx] = rh[q][1];
                sH[b][2][ry][rx] = rh[q][2];
            }
        }
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            const int r = tid + q * kEhX * kEhY;
            if (r < (kEhY + 1) * (kEhX + 1)) {
                const int rx = r % (kEhX + 1), ry = r / (kEhX + 1);
                sEp[0][ry][rx] = re[q][0];
                sEp[1][ry][rx] = re[q][1];
                sEp[2][ry][rx] = re[q][2];
            }
        }
    };
    // whether the block's columns (with their halo) meet an x / y CPML slab; per plane add the z slabs
    const int L = cin.L;
    const bool xy_pml = L > 0 && (x0 < L || x0 + kEhX >= nx - L || y0 < L || y0 + kEhY >= ny - L);
    auto pml_plane = [&](int64_t k) { return xy_pml || (L > 0 && (k < L || k >= nz - L)); };
    // E^{n+1} of plane k over the tile and its +x / +y halo into sE[b]; bk / bm: sH buffers of planes k, k-1
    auto compE = [&](int b, int bk, int bm, int64_t k) {
        const bool pml = pml_plane(k);
        for (int r = tid; r < (kEhY + 1) * (kEhX + 1); r += kEhX * kEhY) {
            const int rx = r % (kEhX + 1), ry = r / (kEhX + 1);
            const int64_t i = x0 + rx, j = y0 + ry;
            float exn = 0.f, eyn = 0.f, ezn = 0.f;
            if (k < nz && i < nx && j < ny) {
                const int hx_ = rx + 1, hy_ = ry + 1;
                const float hxc = sH[bk][0][hy_][hx_], hyc = sH[bk][1][hy_][hx_], hzc = sH[bk][2][hy_][hx_];
                const float dHz_y = j > 0 ? hzc - sH[bk][2][hy_ - 1][hx_] : 0.f;
                const float dHy_z = k > 0 ? hyc - sH[bm][1][hy_][hx_] : 0.f;
                const float dHx_z = k > 0 ? hxc - sH[bm][0][hy_][hx_] : 0.f;
                const float dHz_x = i > 0 ? hzc - sH[bk][2][hy_][hx_ - 1] : 0.f;
                const float dHy_x = i > 0 ? hyc - sH[bk][1][hy_][hx_ - 1] : 0.f;
                const float dHx_y = j > 0 ? hxc - sH[bk][0][hy_ - 1][hx_] : 0.f;
                const float exc = sEp[0][ry][rx], eyc = sEp[1][ry][rx], ezc = sEp[2][ry][rx];
                const bool own = rx < kEhX && ry < kEhY && k < z1;
                float ux, uy, uz;
                if (!pml) {   // no CPML cell in this block's plane: psi untouched
                    ux = ce * (dHz_y - dHy_z);
                    uy = ce * (dHx_z - dHz_x);
                    uz = ce * (dHy_x - dHx_y);
                } else {
                    e3d_pml_io<float>(cin, pout.psi, own, nx, ny, nz, i, j, k, ce, cpe, dHz_y, dHy_z, dHx_z, dHz_x,
                                      dHy_x, dHx_y, ux, uy, uz);
                }
                exn = exc; eyn = eyc; ezn = ezc;
                if (j > 0 && k > 0) {
                    exn = exc + ux;
                    if (src.kind && source_hits_3d(src, i, j, k)) exn += s_g;
                }
                if (i > 0 && k > 0) eyn = eyc + uy;
                if (i > 0 && j > 0) ezn = ezc + uz;
                if (own) {
                    const int64_t c = k * sxy + j * nx + i;
                    out.ex[c] = exn;
                    out.ey[c] = eyn;
                    out.ez[c] = ezn;
                }
            }
            sE[b][0][ry][rx] = exn;
            sE[b][1][ry][rx] = eyn;
            sE[b][2][ry][rx] = ezn;
        }
    };
    // H^{n+3/2} of plane k on the tile; bk: sH buffer of plane k, ek / ek1: sE buffers of planes k, k+1
    auto compH = [&](int bk, int ek, int ek1, int64_t k) {
        const bool pml = pml_plane(k);
        const int64_t i = x0 + tx, j = y0 + ty;
        if (k >= nz || i >= nx || j >= ny) return;
        float hxv = sH[bk][0][ty + 1][tx + 1], hyv = sH[bk][1][ty + 1][tx + 1], hzv = sH[bk][2][ty + 1][tx + 1];
        const float exc = sE[ek][0][ty][tx], eyc = sE[ek][1][ty][tx], ezc = sE[ek][2][ty][tx];
        const float dEz_y = sE[ek][2][ty + 1][tx] - ezc;
        const float dEy_z = sE[ek1][1][ty][tx] - eyc;
        const float dEx_z = sE[ek1][0][ty][tx] - exc;
        const float dEz_x = sE[ek][2][ty][tx + 1] - ezc;
        const float dEy_x = sE[ek][1][ty][tx + 1] - eyc;
        const float dEx_y = sE[ek][0][ty + 1][tx] - exc;
        if (!pml) {
            hxv -= ch * (dEz_y - dEy_z);
            hyv -= ch * (dEx_z - dEz_x);
            hzv -= ch * (dEy_x - dEx_y);
        } else {
            h3d_pml_io<float>(cin, pout.psi, true, nx, ny, nz, i, j, k, ch, cph, dEz_y, dEy_z, dEx_z, dEz_x, dEy_x,
                              dEx_y, hxv, hyv, hzv);
        }
        const int64_t c = k * sxy + j * nx + i;
        out.hx[c] = hxv;
        out.hy[c] = hyv;
        out.hz[c] = hzv;
    };
    // prologue: H of plane z0-1 (for dH/dz of E^{n+1}(z0)) into sH[1], plane z0 into sH[0], E'(z0)
    fetch(z0 - 1);
    commit(1);
    fetch(z0);
    commit(0);
    __syncthreads();
    fetch(z0 + 1);                     // in flight during E^{n+1}(z0)
    compE(0, 0, 1, z0);
    __syncthreads();
    int cur = 0;
    for (int64_t k = z0; k < z1; ++k) {
        const int nxt = cur ^ 1;
        commit(nxt);                   // plane k+1 (the buffer held plane k-1, no longer needed)
        __syncthreads();
        if (k + 1 < z1) fetch(k + 2);  // plane k+2 in flight during this iteration's compute
        compE(nxt, nxt, cur, k + 1);
        __syncthreads();
        compH(cur, cur, nxt, k);
        __syncthreads();               // plane k's buffers are overwritten next iteration
        cur = nxt;
    }
}

// ------------------------------------------- 2-D fused E^{n+1} + H^{n+3/2} (FP32)
// A block owns a 64 x 16 tile: it stages H^{n+1/2} (with the -x / -y halo) and
// E' (E^n after the density term, with the +x / +y halo) in shared memory,
// forms E^{n+1} on the tile and its +x / +y halo, stores the tile's E^{n+1},
// then forms H^{n+3/2} on the tile.  Reads set `in`, writes set `out` (fields
// and psi), so no block reads what another writes; two barriers per tile.
constexpr int kF2X = 64, kF2Y = 16, kF2T = 256;

__global__ void __launch_bounds__(kF2T) k_eh2d(const float *__restrict__ ez_in, const float *__restrict__ hx_in,
                                               const float *__restrict__ hy_in, float *__restrict__ ez_out,
                                               float *__restrict__ hx_out, float *__restrict__ hy_out, int64_t nx,
                                               int64_t ny, float ce, float cpe, float ch, float cph, Cpml<float> cin,
                                               PsiOut pout, Source src, const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    __shared__ float sHx[kF2Y + 2][kF2X + 2], sHy[kF2Y + 2][kF2X + 2];   // x0-1..x0+64, y0-1..y0+16
    __shared__ float sEp[kF2Y + 1][kF2X + 1];                           // E': x0..x0+64, y0..y0+16
    __shared__ float sE[kF2Y + 1][kF2X + 1];                            // E^{n+1}
    __shared__ float s_g;
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * kF2X, y0 = (int64_t)blockIdx.y * kF2Y;
    const int64_t n1 = *d_step + kstep + 1;
    if (tid == 0) {
        const bool near = src.kind && src.i >= x0 && src.i <= x0 + kF2X && src.j >= y0 && src.j <= y0 + kF2Y;
        s_g = near ? (float)source_value(src, (double)n1 * src.dt) : 0.f;
        if (src.kind && blockIdx.x == 0 && blockIdx.y == 0) *src.val = source_value(src, (double)(n1 + 1) * src.dt);
    }
    for (int r = tid; r < (kF2Y + 2) * (kF2X + 2); r += kF2T) {
        const int rx = r % (kF2X + 2), ry = r / (kF2X + 2);
        const int64_t i = x0 - 1 + rx, j = y0 - 1 + ry;
        const bool ok = i >= 0 && i < nx && j >= 0 && j < ny;
        const int64_t c = ok ? j * nx + i : 0;
        sHx[ry][rx] = ok ? hx_in[c] : 0.f;
        sHy[ry][rx] = ok ? hy_in[c] : 0.f;
    }
    for (int r = tid; r < (kF2Y + 1) * (kF2X + 1); r += kF2T) {
        const int rx = r % (kF2X + 1), ry = r / (kF2X + 1);
        const int64_t i = x0 + rx, j = y0 + ry;
        const bool ok = i < nx && j < ny;
        sEp[ry][rx] = ok ? ez_in[j * nx + i] : 0.f;
    }
    __syncthreads();
    const int L = cin.L;
    const bool pml = L > 0 && (x0 < L || x0 + kF2X >= nx - L || y0 < L || y0 + kF2Y >= ny - L);
    // E^{n+1} on the tile and its +x / +y halo (PEC rows and columns keep E')
    for (int r = tid; r < (kF2Y + 1) * (kF2X + 1); r += kF2T) {
        const int rx = r % (kF2X + 1), ry = r / (kF2X + 1);
        const int64_t i = x0 + rx, j = y0 + ry;
        float e = 0.f;
        if (i < nx && j < ny) {
            e = sEp[ry][rx];
            if (i >= 1 && j >= 1) {
                const float dHx = sHy[ry + 1][rx + 1] - sHy[ry + 1][rx];   // dHy along x
                const float dHy = sHx[ry + 1][rx + 1] - sHx[ry][rx + 1];   // dHx along y
                const bool own = rx < kF2X && ry < kF2Y;
                e = rn_add(e, pml ? e2d_pml_io<float>(cin, pout.psi, own, nx, ny, i, j, ce, cpe, dHx, dHy)
                                  : e2d_term(ce, dHx, dHy));
                if (src.kind && i == src.i && j == src.j) e = rn_add(e, s_g);
            } else if (pml && rx < kF2X && ry < kF2Y) {
                e2d_psi_carry<float>(cin, pout.psi, nx, ny, i, j);   // PEC wall: psi unchanged
            }
            if (rx < kF2X && ry < kF2Y) ez_out[j * nx + i] = e;
        }
        sE[ry][rx] = e;
    }
    __syncthreads();
    // H^{n+3/2} on the tile
    for (int r = tid; r < kF2Y * kF2X; r += kF2T) {
        const int rx = r % kF2X, ry = r / kF2X;
        const int64_t i = x0 + rx, j = y0 + ry;
        if (i >= nx || j >= ny) continue;
        const float e = sE[ry][rx];
        const float dEy = sE[ry + 1][rx] - e;   // dEz along y (0 past the last row)
        const float dEx = sE[ry][rx + 1] - e;   // dEz along x
        float hxv = sHx[ry + 1][rx + 1], hyv = sHy[ry + 1][rx + 1];
        if (!pml) {
            hxv = hx_plain(hxv, ch, dEy);
            hyv = hy_plain(hyv, ch, dEx);
        } else {
            h2d_pml_io<float>(cin, pout.psi, nx, ny, i, j, ch, cph, dEy, dEx, hxv, hyv);
        }
        const int64_t c = j * nx + i;
        hx_out[c] = hxv;
        hy_out[c] = hyv;
    }
}

// ------------------------------ 2-D fused E^{n+1} + H^{n+3/2}, column march (FP32)
// A warp owns a strip of 128 columns (four a lane) and marches up a segment of
// rows.  At row j it forms E^{n+1}(j) from the H^{n+1/2} rows j and j - 1 (the
// latter kept in registers from the previous row), then H^{n+3/2}(j - 1) from
// the E^{n+1} rows j - 1 and j.  x neighbours come from the adjacent lanes; the
// strip's edge lanes load the one column beyond it (lane 0: H_y at x - 1;
// lane 31: E', H_x and H_y at x + 128, whose E^{n+1} it forms as well).  A
// segment re-reads H_x of the row below it and forms, without storing it,
// E^{n+1} of the row above it.  No barrier: each lane's inputs come through its
// own cp.async ring in shared memory.  Reads set `in` (fields and psi), writes
// set `out`.  Per cell the arithmetic is that of every 2-D kernel (the
// fixed-rounding helpers of stencil_common.cuh), so the fused and separate
// sequences agree bit for bit.
constexpr int kEh2W = 1;   // warps (128-column strips) per block: a block's slot frees as soon as its strip ends
constexpr int kEh2D = 4;   // rows in each lane's copy ring

// g(t^{n1}) in FP32, as the separate E kernel reads it; out of line because
// only the thread at the source node calls it
__device__ __noinline__ float source_f32(int kind, double amp, double fc, double tau, double t0, double dt, int64_t n1)
{
    Source s{};
    s.kind = kind;
    s.amp = amp;
    s.fc = fc;
    s.tau = tau;
    s.t0 = t0;
    s.dt = dt;
    return (float)source_value(s, (double)n1 * dt);
}

__global__ void __launch_bounds__(32 * kEh2W, 22)
    k_eh2d_v4(const float *__restrict__ ez_in, const float *__restrict__ hx_in, const float *__restrict__ hy_in,
              float *__restrict__ ez_out, float *__restrict__ hx_out, float *__restrict__ hy_out, int64_t nx,
              int64_t ny, int rows, int ktop, float ce, float cpe, float ch, float cph, Cpml<float> cin, PsiOut pout,
              Source src, const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    const int lane = (int)(threadIdx.x & 31u), w = (int)(threadIdx.x >> 5);
    const int64_t xs = ((int64_t)blockIdx.x * kEh2W + w) * 128;   // the warp's strip
    const int64_t i0 = xs + 4 * lane;
    // rows in 32 bits (the launcher checks ny < 2^31); cell offsets in 64.  The ktop segments at the top
    // (the slower CPML rows of the upper y slab) are launched first, with those of the lower slab, so
    // they do not trail the grid's last wave.
    const int nyi = (int)ny;
    const int seg = (int)blockIdx.y < ktop ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y - ktop;
    const int j0 = seg * rows;
    const int j1 = j0 + rows < nyi ? j0 + rows : nyi;   // owned rows [j0, j1)
    const int jl = j1 < nyi ? j1 : nyi - 1;             // last row whose E^{n+1} is formed
    const int64_t n1 = *d_step + kstep + 1;
    if (src.kind && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        *src.val = source_value(src, (double)(n1 + 1) * src.dt);   // g(t^{n+2}) for a following unfused E
    if (xs >= nx) return;   // the whole warp is past the grid
    const bool live = i0 < nx;
    const int64_t xr = xs + 128;   // the column beyond the strip (lane 31's quad + 4)
    const bool left = lane == 0 && xs > 0, right = lane == 31 && xr < nx;
    const int L = cin.L;
    const int ylo = L, yhi = nyi - L;   // rows outside [ylo, yhi) are in a y slab
    const unsigned full = 0xffffffffu;
    // per-column parts of the CPML selection and of the source test (the row parts are per row)
    const bool pml_cols = L > 0 && (i0 < L || i0 + 3 >= nx - L);
    const bool pml_cols_r = L > 0 && (xr < L || xr + 3 >= nx - L);
    const int src_e = src.kind && src.i >= i0 && src.i < i0 + 4 ? (int)(src.i - i0) : -1;
    const bool src_r = src.kind && src.i == xr;
    const int srcj = src.kind && src.j >= 0 && src.j < ny ? (int)src.j : -1;
    const bool wall = i0 == 0;   // the quad holds column 0 (PEC)

    // Each lane streams its own inputs through a ring of kEh2D rows in shared
    // memory (cp.async; lane 0 and lane 31 add the columns beyond the strip),
    // so a warp keeps kEh2D - 1 rows of loads in flight while it computes one;
    // a lane reads back only what it copied itself, so no barrier is needed.
    __shared__ float4 ring[kEh2W][kEh2D][3][32];
    __shared__ float halo[kEh2W][kEh2D][4];
    int ji = j0;                              // the next row to copy
    int64_t ci = (int64_t)j0 * nx + i0;       // and its quad's offset
    auto issue = [&](int sl) {                // that row into slot sl, one copy group (empty past the last row)
        if (ji <= jl) {
            if (live) {
                cpa16(&ring[w][sl][0][lane], ez_in + ci);
                cpa16(&ring[w][sl][1][lane], hx_in + ci);
                cpa16(&ring[w][sl][2][lane], hy_in + ci);
            }
            if (left) cpa4(&halo[w][sl][0], hy_in + ci - 1);
            if (right) {
                cpa4(&halo[w][sl][1], ez_in + ci + 4);
                cpa4(&halo[w][sl][2], hx_in + ci + 4);
                cpa4(&halo[w][sl][3], hy_in + ci + 4);
            }
        }
        cpa_commit();
        ++ji;
        ci += nx;
    };
    auto q4 = [](const float4 &t) { return Q4{{t.x, t.y, t.z, t.w}}; };

    int64_t c = (int64_t)j0 * nx + i0;   // the current row's quad
    Q4 hxp = ld4_if(live && j0 >= 1, hx_in + c - nx);   // H_x^{n+1/2} of the row below
    float hxrp = right && j0 >= 1 ? hx_in[c - nx + 4] : 0.f;
    Q4 hyp{}, enp{};         // the previous row's H_y^{n+1/2} and E^{n+1}
    float erp = 0.f;         // and E^{n+1} right of the quad
    bool slab_p = false;     // and whether it lies in a y slab
    // a lane past the grid reads zeros from slots it never fills (its E^{n+1}
    // stays 0: the last live lane takes it as the node beyond the grid)
    if (!live) {
#pragma unroll
        for (int d = 0; d < kEh2D; ++d)
#pragma unroll
            for (int a = 0; a < 3; ++a) ring[w][d][a][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int d = 0; d < kEh2D - 1; ++d) issue(d);
    // The CPML updates read psi from the row they work on: a lane in an x slab
    // (and every lane in a y-slab row, with the row's y profile) asks for that
    // psi kEh2D - 1 rows ahead, as its ring does for the fields, so those
    // reads hit L1 instead of waiting on DRAM in the row loop.
    const int xslot = pml_cols && live ? slab_slot<float>(i0 < L ? i0 : i0 + 3, nx, L) : 0;
    auto prefetch_psi = [&](int jj) {
        if (jj > jl || !live) return;
        if (pml_cols) {
            prefetch_l1(cin.psi[0] + (int64_t)jj * (2 * L) + xslot);
            prefetch_l1(cin.psi[3] + (int64_t)jj * (2 * L) + xslot);
        }
        if (L > 0 && (jj < ylo || jj >= yhi)) {
            const int64_t o = (int64_t)slab_slot<float>(jj, ny, L) * nx + i0;
            prefetch_l1(cin.psi[1] + o);
            prefetch_l1(cin.psi[2] + o);
            if (lane == 0) {   // the row's y profile (one line each, shared by the warp)
                prefetch_l1(cin.be[1] + jj);
                prefetch_l1(cin.ae[1] + jj);
                prefetch_l1(cin.ike[1] + jj);
                prefetch_l1(cin.bh[1] + jj);
                prefetch_l1(cin.ah[1] + jj);
                prefetch_l1(cin.ikh[1] + jj);
            }
        }
    };
#pragma unroll
    for (int d = 0; d < kEh2D - 1; ++d) prefetch_psi(j0 + d);
    int sl = 0;   // the slot of row j (rows j0 + kEh2D m + sl use slot sl)
    for (int j = j0; j <= jl; ++j, c += nx) {
        issue(sl == 0 ? kEh2D - 1 : sl - 1);   // refills the slot row j - 1 was read from
        prefetch_psi(j + kEh2D - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(kEh2D - 1) : "memory");   // row j has landed
        const Q4 ep = q4(ring[w][sl][0][lane]), hx = q4(ring[w][sl][1][lane]), hy = q4(ring[w][sl][2][lane]);
        float hl = __shfl_up_sync(full, hy.v[3], 1);
        if (lane == 0) hl = left ? halo[w][sl][0] : 0.f;
        const bool own = j < j1;
        const bool slab = L > 0 && (j < ylo || j >= yhi);
        const bool pml = pml_cols || slab;
        const bool srow = j == srcj;
        // E^{n+1}(j) on the quad (row 0 and column 0 are the PEC wall)
        Q4 en = ep;
        if (live && !pml && j >= 1 && !wall && !(srow && src_e >= 0)) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float dHx = hy.v[e] - (e > 0 ? hy.v[e - 1] : hl);
                const float dHy = hx.v[e] - hxp.v[e];
                en.v[e] = rn_add(en.v[e], e2d_term(ce, dHx, dHy));
            }
        } else if (live) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t i = i0 + e;
                if (j >= 1 && i >= 1) {
                    const float dHx = hy.v[e] - (e > 0 ? hy.v[e - 1] : hl);
                    const float dHy = hx.v[e] - hxp.v[e];
                    en.v[e] = rn_add(en.v[e], pml ? e2d_pml_io<float>(cin, pout.psi, own, nx, ny, i, j, ce, cpe, dHx, dHy)
                                                  : e2d_term(ce, dHx, dHy));
                    if (srow && e == src_e)
                        en.v[e] = rn_add(en.v[e], source_f32(src.kind, src.amp, src.fc, src.tau, src.t0, src.dt, n1));
                } else if (pml && own) {
                    e2d_psi_carry<float>(cin, pout.psi, nx, ny, i, j);
                }
            }
        }
        // E^{n+1}(j) of the column beyond the strip, as the next strip's lane 0 forms it
        float enr = 0.f, hxr = 0.f;
        if (right) {
            enr = halo[w][sl][1];
            hxr = halo[w][sl][2];
            if (j >= 1) {
                const float dHx = halo[w][sl][3] - hy.v[3], dHy = hxr - hxrp;
                enr = rn_add(enr, pml_cols_r || slab ? e2d_pml_io<float>(cin, pout.psi, false, nx, ny, xr, j, ce, cpe,
                                                                         dHx, dHy)
                                                     : e2d_term(ce, dHx, dHy));
                if (srow && src_r)
                    enr = rn_add(enr, source_f32(src.kind, src.amp, src.fc, src.tau, src.t0, src.dt, n1));
            }
        }
        float er = __shfl_down_sync(full, en.v[0], 1);
        if (lane == 31) er = enr;
        if (live && own) st4(ez_out + c, en);
        // H^{n+3/2}(j - 1)
        if (live && j > j0) {
            Q4 hxo = hxp, hyo = hyp;
            if (!(pml_cols || slab_p)) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    hxo.v[e] = hx_plain(hxo.v[e], ch, en.v[e] - enp.v[e]);
                    hyo.v[e] = hy_plain(hyo.v[e], ch, (e < 3 ? enp.v[e + 1] : erp) - enp.v[e]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float dEy = en.v[e] - enp.v[e];
                    const float dEx = (e < 3 ? enp.v[e + 1] : erp) - enp.v[e];
                    h2d_pml_io<float>(cin, pout.psi, nx, ny, i0 + e, j - 1, ch, cph, dEy, dEx, hxo.v[e], hyo.v[e]);
                }
            }
            st4(hx_out + c - nx, hxo);
            st4(hy_out + c - nx, hyo);
        }
        hxp = hx;
        hyp = hy;
        enp = en;
        erp = er;
        hxrp = hxr;
        slab_p = slab;
        sl = sl + 1 == kEh2D ? 0 : sl + 1;
    }
    // the top row: E^{n+1} above it is 0 (c is one row past it)
    if (live && j1 == nyi) {
        const int j = nyi - 1;
        Q4 hxo = hxp, hyo = hyp;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float dEy = 0.f - enp.v[e];
            const float dEx = (e < 3 ? enp.v[e + 1] : erp) - enp.v[e];
            if (!(pml_cols || slab_p)) {
                hxo.v[e] = hx_plain(hxo.v[e], ch, dEy);
                hyo.v[e] = hy_plain(hyo.v[e], ch, dEx);
            } else {
                h2d_pml_io<float>(cin, pout.psi, nx, ny, i0 + e, j, ch, cph, dEy, dEx, hxo.v[e], hyo.v[e]);
            }
        }
        st4(hx_out + c - nx, hxo);
        st4(hy_out + c - nx, hyo);
    }
}

__global__ void k_advance(int64_t *d_step, int64_t by)
{
    pdl_enter();
    *d_step += by;
}

// ------------------------------------------------------------------ launchers

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

void launch_eh2d(cudaStream_t st, float *const fin[6], float *const fout[6], float *const psi_out[12], int64_t nx,
                 int64_t ny, float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                 const int64_t *d_step, int kstep, int rows)
{
    PsiOut po{};
    for (int q = 0; q < 12; ++q) po.psi[q] = psi_out[q];
    if (rows > 0 && nx % 4 == 0 && ny < (int64_t(1) << 31)) {   // the column march (16-byte rows, 32-bit row index)
        const unsigned nseg = cdiv(ny, rows);
        const int ktop = cin.L > 0 ? (int)std::min<int64_t>(nseg, cdiv(cin.L, rows) + 1) : 0;
        dim3 g(cdiv(nx, 128 * kEh2W), nseg);
        launch_pdl(k_eh2d_v4, g, dim3(32 * kEh2W), 0, st, fin[FDTD_EZ], fin[FDTD_HX], fin[FDTD_HY], fout[FDTD_EZ],
                   fout[FDTD_HX], fout[FDTD_HY], nx, ny, rows, ktop, ce, cpe, ch, cph, cin, po, src, d_step, kstep);
        return;
    }
    dim3 g(cdiv(nx, kF2X), cdiv(ny, kF2Y));
    launch_pdl(k_eh2d, dim3(g), dim3(kF2T), 0, st, fin[FDTD_EZ], fin[FDTD_HX], fin[FDTD_HY], fout[FDTD_EZ], fout[FDTD_HX], fout[FDTD_HY],
                               nx, ny, ce, cpe, ch, cph, cin, po, src, d_step, kstep);
}

void launch_eh3d(cudaStream_t st, float *const fin[6], float *const fout[6], float *const psi_out[12], int64_t nx,
                 int64_t ny, int64_t nz, float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                 const int64_t *d_step, int kstep)
{
    const int tz = 32;
    dim3 g(cdiv(nx, kEhX), cdiv(ny, kEhY), cdiv(nz, tz));
    FieldPtrs a{fin[0], fin[1], fin[2], fin[3], fin[4], fin[5]};
    FieldOut o{fout[0], fout[1], fout[2], fout[3], fout[4], fout[5]};
    PsiOut po{};
    for (int q = 0; q < 12; ++q) po.psi[q] = psi_out[q];
    launch_pdl(k_eh3d, dim3(g), dim3(dim3(kEhX, kEhY)), 0, st, a, o, nx, ny, nz, tz, ce, cpe, ch, cph, cin, po, src, d_step, kstep);
}


template <typename T>
void launch_h1d(cudaStream_t st, const T *ex, T *hy, T *mur_state, int64_t nz, T ch, Source src,
                const int64_t *d_step, int kstep)
{
    launch_pdl(k_h1d<T>, dim3(cdiv(nz + 1, 256)), dim3(256), 0, st, ex, hy, mur_state, nz, ch, src, d_step, kstep);
}
template <typename T>
void launch_e1d(cudaStream_t st, T *ex, const T *hy, int64_t nz, T ce, Source src, const int64_t *d_step, int kstep,
                const T *mur_state, T m)
{
    launch_pdl(k_e1d<T>, dim3(cdiv(nz, 256)), dim3(256), 0, st, ex, hy, nz, ce, src, d_step, kstep, mur_state, m);
}
template <typename T>
bool use_v4(int64_t nx, dim3 b, int cpt)
{
    return cpt == 4 && std::is_same<T, float>::value && nx % 4 == 0 && (b.x * b.y * b.z) % 32 == 0;
}

template <typename T>
void launch_h2d(cudaStream_t st, const T *ez, T *hx, T *hy, int64_t nx, int64_t ny, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b, int cpt)
{
    if constexpr (std::is_same<T, float>::value) {
        if (use_v4<T>(nx, b, cpt)) {
            dim3 g(cdiv(nx / 4, b.x), cdiv(ny, b.y));
            launch_pdl(k_h2d_v4, dim3(g), dim3(b), 0, st, ez, hx, hy, nx, ny, ch, cph, cp, src, d_step, kstep);
            return;
        }
    }
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y));
    launch_pdl(k_h2d<T>, dim3(g), dim3(b), 0, st, ez, hx, hy, nx, ny, ch, cph, cp, src, d_step, kstep);
}
template <typename T>
void launch_e2d(cudaStream_t st, T *ez, const T *hx, const T *hy, int64_t nx, int64_t ny, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b, int cpt)
{
    if constexpr (std::is_same<T, float>::value) {
        if (use_v4<T>(nx, b, cpt)) {
            dim3 g(cdiv(nx / 4, b.x), cdiv(ny, b.y));
            launch_pdl(k_e2d_v4, dim3(g), dim3(b), 0, st, ez, hx, hy, nx, ny, ce, cpe, cp, src, d_step, kstep);
            return;
        }
    }
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y));
    launch_pdl(k_e2d<T>, dim3(g), dim3(b), 0, st, ez, hx, hy, nx, ny, ce, cpe, cp, src, d_step, kstep);
}
template <typename T>
void launch_h3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b, int cpt)
{
    if constexpr (std::is_same<T, float>::value) {
        if (use_v4<T>(nx, b, cpt)) {
            dim3 g(cdiv(nx / 4, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
            launch_pdl(k_h3d_v4, dim3(g), dim3(b), 0, st, f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ch, cph, cp, src, d_step,
                                      kstep);
            return;
        }
    }
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
    launch_pdl(k_h3d<T>, dim3(g), dim3(b), 0, st, f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ch, cph, cp, src, d_step, kstep);
}
template <typename T>
void launch_e3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b, int cpt)
{
    if constexpr (std::is_same<T, float>::value) {
        if (use_v4<T>(nx, b, cpt)) {
            dim3 g(cdiv(nx / 4, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
            launch_pdl(k_e3d_v4, dim3(g), dim3(b), 0, st, f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ce, cpe, cp, src, d_step,
                                      kstep);
            return;
        }
    }
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
    launch_pdl(k_e3d<T>, dim3(g), dim3(b), 0, st, f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ce, cpe, cp, src, d_step, kstep);
}
void launch_advance(cudaStream_t st, int64_t *d_step, int64_t by) { launch_pdl(k_advance, dim3(1), dim3(1), 0, st, d_step, by); }

#define FP_INST(T)                                                                                            \
    template void launch_h1d<T>(cudaStream_t, const T *, T *, T *, int64_t, T, Source, const int64_t *, int);  \
    template void launch_e1d<T>(cudaStream_t, T *, const T *, int64_t, T, Source, const int64_t *, int, const T *, \
                                T);                                                                          \
    template void launch_h2d<T>(cudaStream_t, const T *, T *, T *, int64_t, int64_t, T, T, Cpml<T>, Source,   \
                                const int64_t *, int, dim3, int);                                                  \
    template void launch_e2d<T>(cudaStream_t, T *, const T *, const T *, int64_t, int64_t, T, T, Cpml<T>,     \
                                Source, const int64_t *, int, dim3, int);                                          \
    template void launch_h3d<T>(cudaStream_t, T *const[6], int64_t, int64_t, int64_t, T, T, Cpml<T>, Source,  \
                                const int64_t *, int, dim3, int);                                                  \
    template void launch_e3d<T>(cudaStream_t, T *const[6], int64_t, int64_t, int64_t, T, T, Cpml<T>, Source,  \
                                const int64_t *, int, dim3, int);
FP_INST(float)
FP_INST(double)

}  // namespace fp

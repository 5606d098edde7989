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
#include "internal.cuh"

namespace fp {

template <typename T>
__device__ __forceinline__ int slab_slot(int64_t i, int64_t n, int L)
{
    return (int)(i < L ? i : L + (i - (n - L)));
}

template <typename T>
__device__ __forceinline__ bool in_slab(int64_t i, int64_t n, int L)
{
    return i < L || i >= n - L;
}

// g(t^{n+1}) is evaluated once per step, by the first thread of the H kernel,
// into a device scalar that the E kernel of the same step reads at the source
// node(s) -- no FP64 transcendental in the E stencil.
__device__ __forceinline__ void write_source(const Source &src, const int64_t *d_step, int kstep)
{
    if (src.kind) *src.val = source_value(src, (double)(*d_step + kstep + 1) * src.dt);
}

// ------------------------------------------------------------------- 1-D

template <typename T>
__global__ void k_h1d(const T *__restrict__ ex, T *__restrict__ hy, T *__restrict__ mur, int64_t nz, T ch, Source src,
                      const int64_t *__restrict__ d_step, int kstep)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) write_source(src, d_step, kstep);
    if (k < nz) hy[k] -= ch * (ex[k + 1] - ex[k]);   // mu0 dHy/dt = -dEx/dz
    if (mur) {                                       // E_1^n and E_{nz-1}^n for the Mur ends
        if (k == 1) mur[0] = ex[1];
        if (k == nz - 1) mur[1] = ex[nz - 1];
    }
}

template <typename T>
__global__ void k_e1d(T *__restrict__ ex, const T *__restrict__ hy, int64_t nz, T ce, Source src,
                      const int64_t *__restrict__ d_step, int kstep)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 1 || k >= nz) return;
    T v = ex[k] - ce * (hy[k] - hy[k - 1]);           // eps0 dEx/dt = -dHy/dz - Jx
    if (src.kind && k == src.k) v += (T)*src.val;
    ex[k] = v;
}

template <typename T>
__global__ void k_mur1d(T *__restrict__ ex, const T *__restrict__ mur, int64_t nz, T m)
{
    // E_0^{n+1} = E_1^n + m (E_1^{n+1} - E_0^n), and the mirror image at nz
    if (threadIdx.x == 0) ex[0] = mur[0] + m * (ex[1] - ex[0]);
    if (threadIdx.x == 1) ex[nz] = mur[1] + m * (ex[nz - 1] - ex[nz]);
}

// ------------------------------------------------------------------- 2-D TMz

template <typename T>
__global__ void __launch_bounds__(256) k_h2d(const T *__restrict__ ez, T *__restrict__ hx, T *__restrict__ hy,
                                             int64_t nx, int64_t ny, T ch, T cph, Cpml<T> cp, Source src,
                                             const int64_t *__restrict__ d_step, int kstep)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i == 0 && j == 0) write_source(src, d_step, kstep);
    if (i >= nx || j >= ny) return;
    const int64_t c = j * nx + i;
    const T e = ez[c];
    const T dEy = (j + 1 < ny ? ez[c + nx] : T(0)) - e;   // dEz along y at (i, j+1/2)
    const T dEx = (i + 1 < nx ? ez[c + 1] : T(0)) - e;    // dEz along x at (i+1/2, j)
    T hxv = hx[c], hyv = hy[c];
    const int L = cp.L;
    if (L == 0) {
        hxv -= ch * dEy;                                  // mu0 dHx/dt = -dEz/dy
        hyv += ch * dEx;                                  // mu0 dHy/dt = +dEz/dx
    } else {
        if (in_slab<T>(j, ny, L)) {
            T *p = cp.psi[2] + (int64_t)slab_slot<T>(j, ny, L) * nx + i;
            T ps = cp.bh[1][j] * *p + cp.ah[1][j] * dEy;
            *p = ps;
            hxv -= ch * dEy * cp.ikh[1][j] + cph * ps;
        } else {
            hxv -= ch * dEy;
        }
        if (in_slab<T>(i, nx, L)) {
            T *p = cp.psi[3] + j * (2 * L) + slab_slot<T>(i, nx, L);
            T ps = cp.bh[0][i] * *p + cp.ah[0][i] * dEx;
            *p = ps;
            hyv += ch * dEx * cp.ikh[0][i] + cph * ps;
        } else {
            hyv += ch * dEx;
        }
    }
    hx[c] = hxv;
    hy[c] = hyv;
}

template <typename T>
__global__ void __launch_bounds__(256) k_e2d(T *__restrict__ ez, const T *__restrict__ hx, const T *__restrict__ hy,
                                             int64_t nx, int64_t ny, T ce, T cpe, Cpml<T> cp, Source src,
                                             const int64_t *__restrict__ d_step, int kstep)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i < 1 || j < 1 || i >= nx || j >= ny) return;
    const int64_t c = j * nx + i;
    // E^n is read before any psi store: the compiler cannot prove the psi
    // slabs and Ez apart, so a later load would be a second round trip.
    const T ezc = ez[c];
    const T dHx = hy[c] - hy[c - 1];     // dHy along x
    const T dHy = hx[c] - hx[c - nx];    // dHx along y
    T upd;
    const int L = cp.L;
    if (L == 0) {
        upd = ce * (dHx - dHy);          // eps0 dEz/dt = dHy/dx - dHx/dy - Jz
    } else {
        T px = T(0), py = T(0), kx = T(1), ky = T(1);
        if (in_slab<T>(i, nx, L)) {
            T *p = cp.psi[0] + j * (2 * L) + slab_slot<T>(i, nx, L);
            px = cp.be[0][i] * *p + cp.ae[0][i] * dHx;
            *p = px;
            kx = cp.ike[0][i];
        }
        if (in_slab<T>(j, ny, L)) {
            T *p = cp.psi[1] + (int64_t)slab_slot<T>(j, ny, L) * nx + i;
            py = cp.be[1][j] * *p + cp.ae[1][j] * dHy;
            *p = py;
            ky = cp.ike[1][j];
        }
        upd = ce * (dHx * kx - dHy * ky) + cpe * (px - py);
    }
    T v = ezc + upd;
    if (src.kind && i == src.i && j == src.j) v += (T)*src.val;
    ez[c] = v;
}

// ------------------------------------------------------------------- 3-D
// psi slot 2*f + d: f = Ex,Ey,Ez,Hx,Hy,Hz; d = 0 for the lower-numbered of the
// two curl axes of the component, 1 for the other.  Derivative axis per slot:
//   0:y 1:z | 2:x 3:z | 4:x 5:y | 6:y 7:z | 8:x 9:z | 10:x 11:y
// x-slabs are [nz][ny][2L], y-slabs [nz][2L][nx], z-slabs [2L][ny][nx].

template <typename T>
struct Pml3 {
    const Cpml<T> &cp;
    int64_t nx, ny, nz, i, j, k;
    __device__ __forceinline__ T *slot_ptr(int s, int axis) const
    {
        const int L = cp.L;
        if (axis == 0) return cp.psi[s] + (k * ny + j) * (2 * L) + slab_slot<T>(i, nx, L);
        if (axis == 1) return cp.psi[s] + (k * (2 * L) + slab_slot<T>(j, ny, L)) * nx + i;
        return cp.psi[s] + ((int64_t)slab_slot<T>(k, nz, L) * ny + j) * nx + i;
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_h3d(const T *__restrict__ ex, const T *__restrict__ ey,
                                             const T *__restrict__ ez, T *__restrict__ hx, T *__restrict__ hy,
                                             T *__restrict__ hz, int64_t nx, int64_t ny, int64_t nz, T ch, T cph,
                                             Cpml<T> cp, Source src, const int64_t *__restrict__ d_step, int kstep)
{
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
    const int L = cp.L;
    if (L == 0) {
        // mu0 dH/dt = -curl E
        hxv -= ch * (dEz_y - dEy_z);
        hyv -= ch * (dEx_z - dEz_x);
        hzv -= ch * (dEy_x - dEx_y);
    } else {
        Pml3<T> P{cp, nx, ny, nz, i, j, k};
        const bool sx = in_slab<T>(i, nx, L), sy = in_slab<T>(j, ny, L), sz = in_slab<T>(k, nz, L);
        const T kx = sx ? cp.ikh[0][i] : T(1), ky = sy ? cp.ikh[1][j] : T(1), kz = sz ? cp.ikh[2][k] : T(1);
        T p6 = 0, p7 = 0, p8 = 0, p9 = 0, p10 = 0, p11 = 0;
        if (sy) {
            T *a = P.slot_ptr(6, 1), *b = P.slot_ptr(11, 1);
            p6 = cp.bh[1][j] * *a + cp.ah[1][j] * dEz_y; *a = p6;
            p11 = cp.bh[1][j] * *b + cp.ah[1][j] * dEx_y; *b = p11;
        }
        if (sz) {
            T *a = P.slot_ptr(7, 2), *b = P.slot_ptr(9, 2);
            p7 = cp.bh[2][k] * *a + cp.ah[2][k] * dEy_z; *a = p7;
            p9 = cp.bh[2][k] * *b + cp.ah[2][k] * dEx_z; *b = p9;
        }
        if (sx) {
            T *a = P.slot_ptr(8, 0), *b = P.slot_ptr(10, 0);
            p8 = cp.bh[0][i] * *a + cp.ah[0][i] * dEz_x; *a = p8;
            p10 = cp.bh[0][i] * *b + cp.ah[0][i] * dEy_x; *b = p10;
        }
        hxv -= ch * (dEz_y * ky - dEy_z * kz) + cph * (p6 - p7);
        hyv -= ch * (dEx_z * kz - dEz_x * kx) + cph * (p9 - p8);
        hzv -= ch * (dEy_x * kx - dEx_y * ky) + cph * (p10 - p11);
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
    const int L = cp.L;
    T ux, uy, uz;
    if (L == 0) {
        // eps0 dE/dt = curl H (- J, already applied to Ex)
        ux = ce * (dHz_y - dHy_z);
        uy = ce * (dHx_z - dHz_x);
        uz = ce * (dHy_x - dHx_y);
    } else {
        Pml3<T> P{cp, nx, ny, nz, i, j, k};
        const bool sx = in_slab<T>(i, nx, L), sy = in_slab<T>(j, ny, L), sz = in_slab<T>(k, nz, L);
        const T kx = sx ? cp.ike[0][i] : T(1), ky = sy ? cp.ike[1][j] : T(1), kz = sz ? cp.ike[2][k] : T(1);
        T p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0, p5 = 0;
        if (sy) {
            T *a = P.slot_ptr(0, 1), *b = P.slot_ptr(5, 1);
            p0 = cp.be[1][j] * *a + cp.ae[1][j] * dHz_y; *a = p0;
            p5 = cp.be[1][j] * *b + cp.ae[1][j] * dHx_y; *b = p5;
        }
        if (sz) {
            T *a = P.slot_ptr(1, 2), *b = P.slot_ptr(3, 2);
            p1 = cp.be[2][k] * *a + cp.ae[2][k] * dHy_z; *a = p1;
            p3 = cp.be[2][k] * *b + cp.ae[2][k] * dHx_z; *b = p3;
        }
        if (sx) {
            T *a = P.slot_ptr(2, 0), *b = P.slot_ptr(4, 0);
            p2 = cp.be[0][i] * *a + cp.ae[0][i] * dHz_x; *a = p2;
            p4 = cp.be[0][i] * *b + cp.ae[0][i] * dHy_x; *b = p4;
        }
        ux = ce * (dHz_y * ky - dHy_z * kz) + cpe * (p0 - p1);
        uy = ce * (dHx_z * kz - dHz_x * kx) + cpe * (p3 - p2);
        uz = ce * (dHy_x * kx - dHx_y * ky) + cpe * (p4 - p5);
    }
    if (j > 0 && k > 0) {
        T v = exc + ux;
        if (src.kind) {
            bool hit = src.loc == FDTD_LOC_SHEET
                           ? (k == src.k && i >= src.i0 && i < src.i1 && j >= src.j0 && j < src.j1)
                           : (i == src.i && j == src.j && k == src.k);
            if (hit) v += (T)*src.val;
        }
        ex[c] = v;
    }
    if (i > 0 && k > 0) ey[c] = eyc + uy;
    if (i > 0 && j > 0) ez[c] = ezc + uz;
}

__global__ void k_advance(int64_t *d_step, int64_t by) { *d_step += by; }

// ------------------------------------------------------------------ launchers

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

template <typename T>
void launch_h1d(cudaStream_t st, const T *ex, T *hy, T *mur_state, int64_t nz, T ch, Source src,
                const int64_t *d_step, int kstep)
{
    k_h1d<T><<<cdiv(nz + 1, 256), 256, 0, st>>>(ex, hy, mur_state, nz, ch, src, d_step, kstep);
}
template <typename T>
void launch_e1d(cudaStream_t st, T *ex, const T *hy, int64_t nz, T ce, Source src, const int64_t *d_step, int kstep)
{
    k_e1d<T><<<cdiv(nz + 1, 256), 256, 0, st>>>(ex, hy, nz, ce, src, d_step, kstep);
}
template <typename T>
void launch_mur1d(cudaStream_t st, T *ex, const T *mur_state, int64_t nz, T m)
{
    k_mur1d<T><<<1, 32, 0, st>>>(ex, mur_state, nz, m);
}
template <typename T>
void launch_h2d(cudaStream_t st, const T *ez, T *hx, T *hy, int64_t nx, int64_t ny, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b)
{
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y));
    k_h2d<T><<<g, b, 0, st>>>(ez, hx, hy, nx, ny, ch, cph, cp, src, d_step, kstep);
}
template <typename T>
void launch_e2d(cudaStream_t st, T *ez, const T *hx, const T *hy, int64_t nx, int64_t ny, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b)
{
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y));
    k_e2d<T><<<g, b, 0, st>>>(ez, hx, hy, nx, ny, ce, cpe, cp, src, d_step, kstep);
}
template <typename T>
void launch_h3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b)
{
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
    k_h3d<T><<<g, b, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ch, cph, cp, src, d_step, kstep);
}
template <typename T>
void launch_e3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 b)
{
    dim3 g(cdiv(nx, b.x), cdiv(ny, b.y), cdiv(nz, b.z));
    k_e3d<T><<<g, b, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, ce, cpe, cp, src, d_step, kstep);
}
void launch_advance(cudaStream_t st, int64_t *d_step, int64_t by) { k_advance<<<1, 1, 0, st>>>(d_step, by); }

#define FP_INST(T)                                                                                            \
    template void launch_h1d<T>(cudaStream_t, const T *, T *, T *, int64_t, T, Source, const int64_t *, int);  \
    template void launch_e1d<T>(cudaStream_t, T *, const T *, int64_t, T, Source, const int64_t *, int);      \
    template void launch_mur1d<T>(cudaStream_t, T *, const T *, int64_t, T);                                  \
    template void launch_h2d<T>(cudaStream_t, const T *, T *, T *, int64_t, int64_t, T, T, Cpml<T>, Source,   \
                                const int64_t *, int, dim3);                                                  \
    template void launch_e2d<T>(cudaStream_t, T *, const T *, const T *, int64_t, int64_t, T, T, Cpml<T>,     \
                                Source, const int64_t *, int, dim3);                                          \
    template void launch_h3d<T>(cudaStream_t, T *const[6], int64_t, int64_t, int64_t, T, T, Cpml<T>, Source,  \
                                const int64_t *, int, dim3);                                                  \
    template void launch_e3d<T>(cudaStream_t, T *const[6], int64_t, int64_t, int64_t, T, T, Cpml<T>, Source,  \
                                const int64_t *, int, dim3);
FP_INST(float)
FP_INST(double)

}  // namespace fp

// stencil_common.cuh -- device helpers shared by the curl-stencil kernels:
// CPML slab indexing, the soft-source value and hit test, and the 3-D CPML
// cell updates (psi <- b psi + a dF with the 1/kappa-scaled curl, Eq. 7-12).
#pragma once

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

// CPML H update of one 2-D cell (Eq. 7-12): psi <- b psi + a dE, curl scaled by 1/kappa.
template <typename T>
__device__ __forceinline__ void h2d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t i, int64_t j, T ch, T cph,
                                        T dEy, T dEx, T &hxv, T &hyv)
{
    const int L = cp.L;
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

// CPML curl term of the E update of one 2-D cell.
template <typename T>
__device__ __forceinline__ T e2d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t i, int64_t j, T ce, T cpe,
                                     T dHx, T dHy)
{
    const int L = cp.L;
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
    return ce * (dHx * kx - dHy * ky) + cpe * (px - py);
}

// 3-D psi slot 2*f + d: f = Ex,Ey,Ez,Hx,Hy,Hz; d = 0 for the lower-numbered of
// the two curl axes of the component, 1 for the other.  Derivative axis per slot:
//   0:y 1:z | 2:x 3:z | 4:x 5:y | 6:y 7:z | 8:x 9:z | 10:x 11:y
// x-slabs are [nz][ny][2L], y-slabs [nz][2L][nx], z-slabs [2L][ny][nx].

template <typename T>
struct Pml3 {
    const Cpml<T> &cp;
    int64_t nx, ny, nz, i, j, k;
    __device__ __forceinline__ int64_t off(int axis) const   // element of the cell in a slab of `axis`
    {
        const int L = cp.L;
        if (axis == 0) return (k * ny + j) * (2 * L) + slab_slot<T>(i, nx, L);
        if (axis == 1) return (k * (2 * L) + slab_slot<T>(j, ny, L)) * nx + i;
        return ((int64_t)slab_slot<T>(k, nz, L) * ny + j) * nx + i;
    }
    __device__ __forceinline__ T *slot_ptr(int s, int axis) const { return cp.psi[s] + off(axis); }
};

// CPML H update of one 3-D cell: six psi recursions on the slabs the cell is in,
// read from cp.psi and written to psi_out when store (psi_out == cp.psi: in place).
template <typename T>
__device__ __forceinline__ void h3d_pml_io(const Cpml<T> &cp, T *const *psi_out, bool store, int64_t nx, int64_t ny,
                                           int64_t nz, int64_t i, int64_t j, int64_t k, T ch, T cph, T dEz_y,
                                           T dEy_z, T dEx_z, T dEz_x, T dEy_x, T dEx_y, T &hxv, T &hyv, T &hzv)
{
    const int L = cp.L;
    Pml3<T> P{cp, nx, ny, nz, i, j, k};
    const bool sx = in_slab<T>(i, nx, L), sy = in_slab<T>(j, ny, L), sz = in_slab<T>(k, nz, L);
    const T kx = sx ? cp.ikh[0][i] : T(1), ky = sy ? cp.ikh[1][j] : T(1), kz = sz ? cp.ikh[2][k] : T(1);
    T p6 = 0, p7 = 0, p8 = 0, p9 = 0, p10 = 0, p11 = 0;
    if (sy) {
        const int64_t o = P.off(1);
        p6 = cp.bh[1][j] * cp.psi[6][o] + cp.ah[1][j] * dEz_y;
        p11 = cp.bh[1][j] * cp.psi[11][o] + cp.ah[1][j] * dEx_y;
        if (store) { psi_out[6][o] = p6; psi_out[11][o] = p11; }
    }
    if (sz) {
        const int64_t o = P.off(2);
        p7 = cp.bh[2][k] * cp.psi[7][o] + cp.ah[2][k] * dEy_z;
        p9 = cp.bh[2][k] * cp.psi[9][o] + cp.ah[2][k] * dEx_z;
        if (store) { psi_out[7][o] = p7; psi_out[9][o] = p9; }
    }
    if (sx) {
        const int64_t o = P.off(0);
        p8 = cp.bh[0][i] * cp.psi[8][o] + cp.ah[0][i] * dEz_x;
        p10 = cp.bh[0][i] * cp.psi[10][o] + cp.ah[0][i] * dEy_x;
        if (store) { psi_out[8][o] = p8; psi_out[10][o] = p10; }
    }
    hxv -= ch * (dEz_y * ky - dEy_z * kz) + cph * (p6 - p7);
    hyv -= ch * (dEx_z * kz - dEz_x * kx) + cph * (p9 - p8);
    hzv -= ch * (dEy_x * kx - dEx_y * ky) + cph * (p10 - p11);
}

template <typename T>
__device__ __forceinline__ void h3d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t nz, int64_t i, int64_t j,
                                        int64_t k, T ch, T cph, T dEz_y, T dEy_z, T dEx_z, T dEz_x, T dEy_x, T dEx_y,
                                        T &hxv, T &hyv, T &hzv)
{
    h3d_pml_io<T>(cp, cp.psi, true, nx, ny, nz, i, j, k, ch, cph, dEz_y, dEy_z, dEx_z, dEz_x, dEy_x, dEx_y, hxv, hyv,
                  hzv);
}

// CPML curl terms (ux, uy, uz) of the E update of one 3-D cell; psi read from
// cp.psi, written to psi_out when store.
template <typename T>
__device__ __forceinline__ void e3d_pml_io(const Cpml<T> &cp, T *const *psi_out, bool store, int64_t nx, int64_t ny,
                                           int64_t nz, int64_t i, int64_t j, int64_t k, T ce, T cpe, T dHz_y,
                                           T dHy_z, T dHx_z, T dHz_x, T dHy_x, T dHx_y, T &ux, T &uy, T &uz)
{
    const int L = cp.L;
    Pml3<T> P{cp, nx, ny, nz, i, j, k};
    const bool sx = in_slab<T>(i, nx, L), sy = in_slab<T>(j, ny, L), sz = in_slab<T>(k, nz, L);
    const T kx = sx ? cp.ike[0][i] : T(1), ky = sy ? cp.ike[1][j] : T(1), kz = sz ? cp.ike[2][k] : T(1);
    T p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0, p5 = 0;
    if (sy) {
        const int64_t o = P.off(1);
        p0 = cp.be[1][j] * cp.psi[0][o] + cp.ae[1][j] * dHz_y;
        p5 = cp.be[1][j] * cp.psi[5][o] + cp.ae[1][j] * dHx_y;
        if (store) { psi_out[0][o] = p0; psi_out[5][o] = p5; }
    }
    if (sz) {
        const int64_t o = P.off(2);
        p1 = cp.be[2][k] * cp.psi[1][o] + cp.ae[2][k] * dHy_z;
        p3 = cp.be[2][k] * cp.psi[3][o] + cp.ae[2][k] * dHx_z;
        if (store) { psi_out[1][o] = p1; psi_out[3][o] = p3; }
    }
    if (sx) {
        const int64_t o = P.off(0);
        p2 = cp.be[0][i] * cp.psi[2][o] + cp.ae[0][i] * dHz_x;
        p4 = cp.be[0][i] * cp.psi[4][o] + cp.ae[0][i] * dHy_x;
        if (store) { psi_out[2][o] = p2; psi_out[4][o] = p4; }
    }
    ux = ce * (dHz_y * ky - dHy_z * kz) + cpe * (p0 - p1);
    uy = ce * (dHx_z * kz - dHz_x * kx) + cpe * (p3 - p2);
    uz = ce * (dHy_x * kx - dHx_y * ky) + cpe * (p4 - p5);
}

template <typename T>
__device__ __forceinline__ void e3d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t nz, int64_t i, int64_t j,
                                        int64_t k, T ce, T cpe, T dHz_y, T dHy_z, T dHx_z, T dHz_x, T dHy_x, T dHx_y,
                                        T &ux, T &uy, T &uz)
{
    e3d_pml_io<T>(cp, cp.psi, true, nx, ny, nz, i, j, k, ce, cpe, dHz_y, dHy_z, dHx_z, dHz_x, dHy_x, dHx_y, ux, uy, uz);
}

__device__ __forceinline__ bool source_hits_3d(const Source &src, int64_t i, int64_t j, int64_t k)
{
    return src.loc == FDTD_LOC_SHEET ? (k == src.k && i >= src.i0 && i < src.i1 && j >= src.j0 && j < src.j1)
                                     : (i == src.i && j == src.j && k == src.k);
}

}  // namespace fp

// stencil_common.cuh -- device helpers shared by the curl-stencil kernels:
// CPML slab indexing, the soft-source value and hit test, the fixed-rounding
// 2-D cell updates and the 3-D CPML cell updates (psi <- b psi + a dF with the
// 1/kappa-scaled curl, Eq. 7-12).
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

// Fixed-rounding arithmetic of the 2-D TMz updates.  Every 2-D kernel (one
// cell or four cells a thread, TMA-fed, fused E + H) forms exactly these
// operations through the helpers below, so their results agree bit for bit
// whatever the compiler would contract in each of them.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// E_z curl term outside the CPML: ce (dHy/dx - dHx/dy); E_z^{n+1} = E' + term
// (rn_add), then + g at the source node (rn_add).  e2d_pml_io with kappa 1
// and psi 0 gives exactly this term.
template <typename T>
__device__ __forceinline__ T e2d_term(T ce, T dHx, T dHy)
{
    return rn_mul(ce, rn_sub(dHx, dHy));
}
// H outside the CPML: mu0 dHx/dt = -dEz/dy, mu0 dHy/dt = +dEz/dx.  Product and
// sum are rounded apart, so that the CPML form below with b = a = 0 and
// 1/kappa = 1 (a sub-domain's local layer planes that lie inside the global
// grid) gives exactly this.
template <typename T>
__device__ __forceinline__ T hx_plain(T hx, T ch, T dEy)
{
    return rn_sub(hx, rn_mul(ch, dEy));
}
template <typename T>
__device__ __forceinline__ T hy_plain(T hy, T ch, T dEx)
{
    return rn_add(hy, rn_mul(ch, dEx));
}

// CPML H update of one 2-D cell (Eq. 7-12): psi <- b psi + a dE, curl scaled
// by 1/kappa; psi read from the handle's slabs and written to pout (the same
// slabs for an in-place update).  Outside a slab the axis takes the plain form.
template <typename T>
__device__ __forceinline__ void h2d_pml_io(const Cpml<T> &cp, T *const *pout, int64_t nx, int64_t ny, int64_t i,
                                           int64_t j, T ch, T cph, T dEy, T dEx, T &hxv, T &hyv)
{
    const int L = cp.L;
    if (in_slab<T>(j, ny, L)) {
        const int64_t o = (int64_t)slab_slot<T>(j, ny, L) * nx + i;
        const T ps = rn_fma(cp.bh[1][j], cp.psi[2][o], rn_mul(cp.ah[1][j], dEy));
        pout[2][o] = ps;
        hxv = rn_sub(hxv, rn_fma(rn_mul(ch, dEy), cp.ikh[1][j], rn_mul(cph, ps)));
    } else {
        hxv = hx_plain(hxv, ch, dEy);
    }
    if (in_slab<T>(i, nx, L)) {
        const int64_t o = j * (2 * L) + slab_slot<T>(i, nx, L);
        const T ps = rn_fma(cp.bh[0][i], cp.psi[3][o], rn_mul(cp.ah[0][i], dEx));
        pout[3][o] = ps;
        hyv = rn_add(hyv, rn_fma(rn_mul(ch, dEx), cp.ikh[0][i], rn_mul(cph, ps)));
    } else {
        hyv = hy_plain(hyv, ch, dEx);
    }
}
template <typename T>
__device__ __forceinline__ void h2d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t i, int64_t j, T ch, T cph,
                                        T dEy, T dEx, T &hxv, T &hyv)
{
    h2d_pml_io<T>(cp, cp.psi, nx, ny, i, j, ch, cph, dEy, dEx, hxv, hyv);
}

// CPML curl term of the E update of one 2-D cell; the new psi goes to pout
// only when `store` (a cell the caller owns).  With neither slab it equals
// e2d_term (kappa 1, psi 0).
template <typename T>
__device__ __forceinline__ T e2d_pml_io(const Cpml<T> &cp, T *const *pout, bool store, int64_t nx, int64_t ny,
                                        int64_t i, int64_t j, T ce, T cpe, T dHx, T dHy)
{
    const int L = cp.L;
    T px = T(0), py = T(0), kx = T(1), ky = T(1);
    if (in_slab<T>(i, nx, L)) {
        const int64_t o = j * (2 * L) + slab_slot<T>(i, nx, L);
        px = rn_fma(cp.be[0][i], cp.psi[0][o], rn_mul(cp.ae[0][i], dHx));
        if (store) pout[0][o] = px;
        kx = cp.ike[0][i];
    }
    if (in_slab<T>(j, ny, L)) {
        const int64_t o = (int64_t)slab_slot<T>(j, ny, L) * nx + i;
        py = rn_fma(cp.be[1][j], cp.psi[1][o], rn_mul(cp.ae[1][j], dHy));
        if (store) pout[1][o] = py;
        ky = cp.ike[1][j];
    }
    return rn_fma(ce, rn_fma(dHx, kx, -rn_mul(dHy, ky)), rn_mul(cpe, rn_sub(px, py)));
}
template <typename T>
__device__ __forceinline__ T e2d_pml(const Cpml<T> &cp, int64_t nx, int64_t ny, int64_t i, int64_t j, T ce, T cpe,
                                     T dHx, T dHy)
{
    return e2d_pml_io<T>(cp, cp.psi, true, nx, ny, i, j, ce, cpe, dHx, dHy);
}

// a PEC wall node keeps its E psi: carry it into another slab set
template <typename T>
__device__ __forceinline__ void e2d_psi_carry(const Cpml<T> &cp, T *const *pout, int64_t nx, int64_t ny, int64_t i,
                                              int64_t j)
{
    const int L = cp.L;
    if (in_slab<T>(i, nx, L)) {
        const int64_t o = j * (2 * L) + slab_slot<T>(i, nx, L);
        pout[0][o] = cp.psi[0][o];
    }
    if (in_slab<T>(j, ny, L)) {
        const int64_t o = (int64_t)slab_slot<T>(j, ny, L) * nx + i;
        pout[1][o] = cp.psi[1][o];
    }
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

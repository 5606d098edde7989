// kinetic.cu -- the phase-space kernel: per plasma cell ("slot") the
// Crank-Nicolson update of the anisotropic distribution (Sec. 5.2, Eq. 22,
// the printed f_1x update)
//     df_j^{n+1/2} = alpha_j df_j^{n-1/2} + beta_j (n E^n)
// on every velocity node j, the current moment (Eq. 24, the Jx sum)
//     J^{n+1/2} = sum_j w'_j df_j^{n+1/2},   w'_j = -e w_j
// reduced with compensated (TwoSum) arithmetic, and the Ampere source term
// applied to the cell's own E in place: E^n <- E^n - (dt/eps0) J^{n+1/2}
// (the curl is added afterwards by the E stencil kernel; the E update is
// linear, so the order of the two additions only changes rounding).
//
// Layout: rows of `pitch` elements, [slot][node], pitch = a power-of-two
// number of 16-byte vectors >= nnode (padding nodes have alpha = beta = w = 0
// and stay 0).  L lanes share a row, each lane holding VPL >= 4 vectors when
// the row has that many; a warp covers 32/L rows.  The whole row is loaded
// before any arithmetic so each lane has VPL 16-byte loads in flight, the
// loads/stores use the streaming (evict-first) cache hint because delta f is
// far larger than L2, and the per-node tables sit in shared memory.
// BF16 storage: FP32 arithmetic, stochastic rounding on store with 16 random
// bits per node from Philox4x32-7 keyed by the seed and counted by
// (slot, vector, step).
#include "kinetic_impl.cuh"

namespace fp {

int kinetic_pitch(int nnode, int f_dtype)
{
    const int vec = f_dtype == FDTD_DF_BF16 ? 8 : (f_dtype == FDTD_DF_F64 ? 2 : 4);
    int nv = (nnode + vec - 1) / vec;
    int p2 = 1;
    while (p2 < nv) p2 <<= 1;
    return p2 * vec;
}

int kinetic_candidates(int nnode_pitch, int f_dtype, int (*out)[2])
{
    const int vec = f_dtype == FDTD_DF_BF16 ? 8 : (f_dtype == FDTD_DF_F64 ? 2 : 4);
    return kinetic_shape_candidates(nnode_pitch / vec, out);
}

cudaError_t dispatch_kinetic_bf16(cudaStream_t st, const KinArgs<float> &a, int num_sms, int vpl, int l, int bps);
cudaError_t dispatch_kinetic_f64(cudaStream_t st, const KinArgs<double> &a, int num_sms, int vpl, int l, int bps);

template <>
cudaError_t launch_kinetic<float>(cudaStream_t st, const KinArgs<float> &a, int f_dtype, int num_sms, int vpl, int l,
                                  int bps)
{
    if (a.nslots == 0) return cudaSuccess;
    if (vpl <= 0) {
        int c[8][2];
        kinetic_candidates(a.pitch, f_dtype, c);
        vpl = c[0][0];
        l = c[0][1];
    }
    if (f_dtype == FDTD_DF_F32) return dispatch_kinetic<float, float>(st, a, num_sms, vpl, l, bps);
    if (f_dtype == FDTD_DF_BF16) return dispatch_kinetic_bf16(st, a, num_sms, vpl, l, bps);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_kinetic<double>(cudaStream_t st, const KinArgs<double> &a, int f_dtype, int num_sms, int vpl, int l,
                                   int bps)
{
    if (a.nslots == 0) return cudaSuccess;
    if (vpl <= 0) {
        int c[8][2];
        kinetic_candidates(a.pitch, f_dtype, c);
        vpl = c[0][0];
        l = c[0][1];
    }
    if (f_dtype == FDTD_DF_F64) return dispatch_kinetic_f64(st, a, num_sms, vpl, l, bps);
    return cudaErrorInvalidValue;
}

}  // namespace fp

// ===================================================================
// Nonlinear mode: the advection of delta f itself by the acceleration
// a = -(e/m) E, in flux form with donor-cell fluxes through the faces between
// neighbouring v_par nodes and zero flux through +-vmax (so sum_j df_j dV_j is
// conserved exactly), with the elastic collisions acting on the part of
// delta f that is odd in v_par:
//   odd^{n+1/2}  = alpha odd^{n-1/2} + beta n E + dt (1 + alpha)/2 A_odd
//   even^{n+1/2} = even^{n-1/2} + dt A_even,   A_j = -(Phi_{a+1/2} - Phi_{a-1/2}) / dv_par
// (dt (1 + alpha)/2 = 2 dt / (2 + dt nu)).  One warp per row: the old row is
// staged in shared memory because every node reads its v_par neighbours and
// its mirror node.  Node order j = a * nperp + b (a: v_par index).
// ===================================================================

namespace fp {

template <typename T>
__global__ void __launch_bounds__(256) k_kinetic_nl(KinArgs<T> a, int npar, int nperp, T dvpar, T qm, T dt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nn = npar * nperp;
    T *s_al = reinterpret_cast<T *>(smem_raw), *s_be = s_al + a.pitch, *s_w = s_be + a.pitch;
    T *s_row = s_w + a.pitch + (threadIdx.x >> 5) * a.pitch;   // one row per warp
    for (int t = threadIdx.x; t < 3 * a.pitch; t += blockDim.x) s_al[t] = a.tab[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    T *df = reinterpret_cast<T *>(a.df);
    for (int64_t row = wg; row < a.nslots; row += nw) {
        const int32_t cell = a.slot_cell[row];
        const T E = a.E[cell];
        const T nE = a.dens[row] * E;
        const T acc = -qm * E;
        T *g = df + row * a.pitch;
        for (int j = lane; j < nn; j += 32) s_row[j] = g[j];
        __syncwarp();
        T s = T(0), c = T(0);
        for (int j = lane; j < nn; j += 32) {
            const int ia = j / nperp, ib = j - ia * nperp;
            const int m = (npar - 1 - ia) * nperp + ib;
            // A at node j and at its mirror: donor-cell fluxes through the faces of each
            auto adv = [&](int aa) -> T {
                T lo = T(0), hi = T(0);
                if (aa > 0) lo = acc * (acc > T(0) ? s_row[(aa - 1) * nperp + ib] : s_row[aa * nperp + ib]);
                if (aa < npar - 1) hi = acc * (acc > T(0) ? s_row[aa * nperp + ib] : s_row[(aa + 1) * nperp + ib]);
                return -(hi - lo) / dvpar;
            };
            const T Aj = adv(ia), Am = adv(npar - 1 - ia);
            const T odd = T(0.5) * (s_row[j] - s_row[m]), even = T(0.5) * (s_row[j] + s_row[m]);
            const T aodd = T(0.5) * (Aj - Am), aeven = T(0.5) * (Aj + Am);
            const T al = s_al[j];
            const T x = even + dt * aeven + al * odd + s_be[j] * nE + dt * (T(1) + al) * T(0.5) * aodd;
            g[j] = x;
            T hi2, lo2;
            two_sum(s, mul_rn(s_w[j], x), hi2, lo2);
            s = hi2;
            c += lo2;
        }
        __syncwarp();
        const T J = row_reduce<T, 32>(s, c);
        if (lane == 0) {
            a.jslot[row] = J;
            a.E[cell] = E - a.cj * J;
        }
    }
}

template <typename T>
cudaError_t launch_kinetic_nl(cudaStream_t st, const KinArgs<T> &a, int npar, int nperp, double dvpar, double qm,
                              double dt, int num_sms)
{
    if (a.nslots == 0) return cudaSuccess;
    const size_t smem = (3 + 8) * (size_t)a.pitch * sizeof(T);
    auto kern = k_kinetic_nl<T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (a.nslots + 7) / 8;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * std::max(per_sm, 1));
    kern<<<(unsigned)std::max<int64_t>(blocks, 1), 256, smem, st>>>(a, npar, nperp, (T)dvpar, (T)qm, (T)dt);
    return cudaGetLastError();
}

template cudaError_t launch_kinetic_nl<float>(cudaStream_t, const KinArgs<float> &, int, int, double, double, double,
                                              int);
template cudaError_t launch_kinetic_nl<double>(cudaStream_t, const KinArgs<double> &, int, int, double, double,
                                               double, int);

}  // namespace fp

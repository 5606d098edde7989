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
                                  int bps, int stages)
{
    if (a.nslots == 0) return cudaSuccess;
    if (vpl <= 0) {
        int c[8][2];
        kinetic_candidates(a.pitch, f_dtype, c);
        vpl = c[0][0];
        l = c[0][1];
    }
    if (stages > 0) return launch_kinetic_ring(st, a, f_dtype, num_sms, vpl, l, bps, stages);
    if (f_dtype == FDTD_DF_F32) return dispatch_kinetic<float, float>(st, a, num_sms, vpl, l, bps);
    if (f_dtype == FDTD_DF_BF16) return dispatch_kinetic_bf16(st, a, num_sms, vpl, l, bps);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_kinetic<double>(cudaStream_t st, const KinArgs<double> &a, int f_dtype, int num_sms, int vpl, int l,
                                   int bps, int stages)
{
    if (a.nslots == 0) return cudaSuccess;
    if (stages > 0) return cudaErrorInvalidValue;   // the ring kernel streams FP32 / BF16 rows only
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
    pdl_enter();
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
    launch_pdl(kern, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), smem, st, a, npar, nperp, (T)dvpar, (T)qm, (T)dt);
    return cudaGetLastError();
}

template cudaError_t launch_kinetic_nl<float>(cudaStream_t, const KinArgs<float> &, int, int, double, double, double,
                                              int);
template cudaError_t launch_kinetic_nl<double>(cudaStream_t, const KinArgs<double> &, int, int, double, double,
                                               double, int);

// --------------------------------------------------------- evolving F0
// Speed grid with an evolving isotropic part (the F0 equation of the two-term
// expansion, Sec. 5.2).  Per row, with E = E^n:
//   F0' = F0'(table) + (g_{k+1} - g_{k-1}) / (2 gam)   (g mirrored at v = 0, 0 past the last node)
//   F1  <- alpha F1 + bq F0' n E,   J = sum w' F1 (TwoSum), E -= dt/eps0 J
//   g   += dt [ (e E / 3m) (Phi_{k+1/2} - Phi_{k-1/2}) + (Psi_{k+1/2} - Psi_{k-1/2}) ] / (v_k^2 gam)
// with the heating flux Phi = (a_k + a_{k+1}) / (2 v_{k+1/2}), a = v^3 (F1_old + F1_new) / (2n), and
// the elastic flux Psi = (m/M) v^3 nu (F0 + (k Tg/(m v)) dF0/dv) at the cell edge, both zero at
// v = 0 and past the last node.  The F0 table holds, per node, [f0 | f0' | bq | v^3 | 1/(v^2 gam) |
// 1/(2 v_e) | (m/M) v_e^3 nu_e | k Tg/(m v_e gam)] with v_e the node's upper edge (edge entries 0 at
// and past the last node), so the kernels multiply only.
//
// Fast kernel: L lanes per row, each lane owns one 16-byte vector of VEC consecutive nodes; the
// neighbours one node across a lane boundary come from segment shuffles.  Bytes per node: delta f
// and g, each read and written once (streaming).

template <typename T>
struct F0Tab {
    const T *al, *w, *f0, *f0p, *bq, *v3, *ivg, *e1, *c1, *c2;
};

template <typename T, int L>
__global__ void __launch_bounds__(256) k_kinetic_f0(KinArgs<T> a, F0Args<T> f)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.pitch;
    T *s = reinterpret_cast<T *>(smem_raw);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        s[t] = a.tab[t];               // alpha
        s[P + t] = a.tab[2 * P + t];   // w' = -e w
    }
    for (int t = threadIdx.x; t < 8 * P; t += blockDim.x) s[2 * P + t] = f.tab[t];
    __syncthreads();
    const F0Tab<T> tb{s, s + P, s + 2 * P, s + 3 * P, s + 4 * P, s + 5 * P, s + 6 * P, s + 7 * P, s + 8 * P, s + 9 * P};

    using V = typename Vec<T>::type;
    constexpr int VEC = Vec<T>::n;
    constexpr int R = 32 / L;
    const int lane = threadIdx.x & 31;
    const int sub = lane / L, l = lane % L;
    const int k0 = l * VEC;            // first node of this lane
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int k1 = k0 + VEC < P ? k0 + VEC : k0;   // one node past the lane (its edge entries are 0 at the end)
    V *df = reinterpret_cast<V *>(a.df);
    V *gv = reinterpret_cast<V *>(f.g);
    const int vpr = P / VEC;

    // Software pipeline: the next row's vectors, E and density are loaded while this row is
    // updated (two rows of loads in flight per lane), its cell index one further row ahead so the
    // E gather does not wait on it.  Rows have distinct cells: reading the next row's E before this
    // row's E store is safe.
    const int64_t stride = nw * R;
    auto fetch = [&](int64_t r, int32_t c, V &xv, V &gw, T &Ev, T &nv) {
        if (r < a.nslots) {
            const int64_t i = r * vpr + l;
            xv = __ldcs(df + i);
            gw = __ldcs(gv + i);
            Ev = a.E[c];
            nv = __ldg(a.dens + r);
        }
    };
    int64_t row = wg * R + sub;
    int32_t cell = row < a.nslots ? __ldg(a.slot_cell + row) : 0;
    int32_t cell_next = row + stride < a.nslots ? __ldg(a.slot_cell + row + stride) : 0;
    V xv{}, gw{};
    T Ev = T(0), nv = T(1);
    fetch(row, cell, xv, gw, Ev, nv);
    for (int64_t base = wg * R; base < a.nslots; base += stride) {
        row = base + sub;
        const bool valid = row < a.nslots;
        const int64_t ri = (valid ? row : 0) * vpr + l;
        T x[VEC], g[VEC];
        const T E = valid ? Ev : T(0), n = valid ? nv : T(1);
        if (valid) {
            unpack(xv, x);
            unpack(gw, g);
        } else {
#pragma unroll
            for (int t = 0; t < VEC; ++t) x[t] = g[t] = T(0);
        }
        const int32_t cell_cur = cell;
        // the next row in flight during this row's update
        const int64_t row_next = row + stride;
        fetch(row_next, cell_next, xv, gw, Ev, nv);
        cell = cell_next;
        cell_next = row_next + stride < a.nslots ? __ldg(a.slot_cell + row_next + stride) : 0;
        // g one node to the left / right of the lane's vector
        T gl = __shfl_up_sync(0xffffffffu, g[VEC - 1], 1, L);
        T gr = __shfl_down_sync(0xffffffffu, g[0], 1, L);
        if (l == 0) gl = g[0];         // mirror at v = 0
        if (l == L - 1) gr = T(0);     // past the last node
        const T nE = n * E;
        T xn[VEC], sum = T(0), cmp = T(0);
        {
            T al[VEC], w[VEC], bq[VEC], f0p[VEC];
            lds<VEC>(tb.al + k0, al); lds<VEC>(tb.w + k0, w); lds<VEC>(tb.bq + k0, bq); lds<VEC>(tb.f0p + k0, f0p);
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
                const T gm = t > 0 ? g[t - 1] : gl, gp = t + 1 < VEC ? g[t + 1] : gr;
                xn[t] = al[t] * x[t] + bq[t] * (f0p[t] + (gp - gm) * f.inv2gam) * nE;
                T hi, lo;
                two_sum(sum, mul_rn(w[t], xn[t]), hi, lo);
                sum = hi;
                cmp += lo;
            }
        }
        // heating and collision fluxes through each node's upper edge
        const T inv_n = T(1) / n;
        T av[VEC];
        {
            T v3[VEC];
            lds<VEC>(tb.v3 + k0, v3);
#pragma unroll
            for (int t = 0; t < VEC; ++t) av[t] = v3[t] * T(0.5) * (x[t] + xn[t]) * inv_n;
        }
        T a_r = __shfl_down_sync(0xffffffffu, av[0], 1, L);
        if (l == L - 1) a_r = T(0);
        T phi[VEC], psi[VEC];
        {
            T f0[VEC], e1[VEC], c1[VEC], c2[VEC];
            lds<VEC>(tb.f0 + k0, f0); lds<VEC>(tb.e1 + k0, e1); lds<VEC>(tb.c1 + k0, c1); lds<VEC>(tb.c2 + k0, c2);
            const T f0_next = tb.f0[k1];
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
                const T an = t + 1 < VEC ? av[t + 1] : a_r;
                phi[t] = (av[t] + an) * e1[t];
                const T F0k = f0[t] + g[t];
                const T F0k1 = (t + 1 < VEC ? f0[t + 1] + g[t + 1] : f0_next + gr);
                psi[t] = c1[t] * (T(0.5) * (F0k + F0k1) + c2[t] * (F0k1 - F0k));
            }
        }
        T phi_l = __shfl_up_sync(0xffffffffu, phi[VEC - 1], 1, L);
        T psi_l = __shfl_up_sync(0xffffffffu, psi[VEC - 1], 1, L);
        if (l == 0) phi_l = psi_l = T(0);
        const T qE = f.qm3 * E;
        T gn[VEC];
        {
            T ivg[VEC];
            lds<VEC>(tb.ivg + k0, ivg);
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
                const T pl = t > 0 ? phi[t - 1] : phi_l, ql = t > 0 ? psi[t - 1] : psi_l;
                gn[t] = g[t] + f.dt * (qE * (phi[t] - pl) + (psi[t] - ql)) * ivg[t];
            }
        }
        const T J = row_reduce<T, L>(sum, cmp);
        if (valid) {
            Store<T>::st(df + ri, xn, uint4{}, uint2{});
            Store<T>::st(gv + ri, gn, uint4{}, uint2{});
            if (l == 0) {
                a.jslot[row] = J;
                a.E[cell_cur] = E - a.cj * J;
            }
        }
    }
}

// Rows of more than 32 vectors: one warp per row, rows staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_kinetic_f0_wide(KinArgs<T> a, F0Args<T> f)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.pitch, nv = f.nv;
    T *s = reinterpret_cast<T *>(smem_raw);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        s[t] = a.tab[t];
        s[P + t] = a.tab[2 * P + t];
    }
    for (int t = threadIdx.x; t < 8 * P; t += blockDim.x) s[2 * P + t] = f.tab[t];
    __syncthreads();
    const F0Tab<T> tb{s, s + P, s + 2 * P, s + 3 * P, s + 4 * P, s + 5 * P, s + 6 * P, s + 7 * P, s + 8 * P, s + 9 * P};
    T *s_old = s + 10 * P + (threadIdx.x >> 5) * 4 * P, *s_new = s_old + P, *s_g = s_new + P, *s_ph = s_g + P;
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    T *df = reinterpret_cast<T *>(a.df);
    for (int64_t row = wg; row < a.nslots; row += nw) {
        const int32_t cell = a.slot_cell[row];
        const T E = a.E[cell];
        const T n = a.dens[row];
        T *d = df + row * P, *g = f.g + row * P;
        for (int j = lane; j < P; j += 32) {
            s_old[j] = d[j];
            s_g[j] = g[j];
        }
        __syncwarp();
        T sum = T(0), cmp = T(0);
        for (int j = lane; j < P; j += 32) {
            const T gm = j > 0 ? s_g[j - 1] : s_g[0];
            const T gp = j + 1 < nv ? s_g[j + 1] : T(0);
            const T xv = tb.al[j] * s_old[j] + tb.bq[j] * (tb.f0p[j] + (gp - gm) * f.inv2gam) * (n * E);
            s_new[j] = xv;
            T hi, lo;
            two_sum(sum, mul_rn(tb.w[j], xv), hi, lo);
            sum = hi;
            cmp += lo;
        }
        __syncwarp();
        const T J = row_reduce<T, 32>(sum, cmp);
        const T inv_n = T(1) / n;
        // fluxes through the upper edge of each node: heating into s_ph, collisions kept per lane
        for (int j = lane; j < P; j += 32) {
            const T a0 = tb.v3[j] * T(0.5) * (s_old[j] + s_new[j]) * inv_n;
            const T a1 = j + 1 < P ? tb.v3[j + 1] * T(0.5) * (s_old[j + 1] + s_new[j + 1]) * inv_n : T(0);
            s_ph[j] = (a0 + a1) * tb.e1[j];
        }
        __syncwarp();
        for (int j = lane; j < P; j += 32) {
            auto psi = [&](int k) -> T {
                const T F0k = tb.f0[k] + s_g[k];
                const T F0k1 = k + 1 < P ? tb.f0[k + 1] + s_g[k + 1] : T(0);
                return tb.c1[k] * (T(0.5) * (F0k + F0k1) + tb.c2[k] * (F0k1 - F0k));
            };
            const T pr = s_ph[j], pl = j > 0 ? s_ph[j - 1] : T(0);
            const T qr = psi(j), ql = j > 0 ? psi(j - 1) : T(0);
            g[j] = s_g[j] + f.dt * (f.qm3 * E * (pr - pl) + (qr - ql)) * tb.ivg[j];
            d[j] = s_new[j];
        }
        if (lane == 0) {
            a.jslot[row] = J;
            a.E[cell] = E - a.cj * J;
        }
        __syncwarp();   // the next row reuses the staging rows
    }
}

template <typename T, int L>
cudaError_t run_kinetic_f0(cudaStream_t st, const KinArgs<T> &a, const F0Args<T> &f, int num_sms)
{
    const size_t smem = 10 * (size_t)a.pitch * sizeof(T);
    auto kern = k_kinetic_f0<T, L>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows_per_block = 8 * (32 / L);
    int64_t blocks = (a.nslots + rows_per_block - 1) / rows_per_block;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * std::max(per_sm, 1));
    launch_pdl(kern, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), smem, st, a, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kinetic_f0(cudaStream_t st, const KinArgs<T> &a, const F0Args<T> &f, int num_sms)
{
    if (a.nslots == 0) return cudaSuccess;
    const int V = a.pitch / Vec<T>::n;   // vectors per row (a power of two)
    switch (V) {
    case 1: return run_kinetic_f0<T, 1>(st, a, f, num_sms);
    case 2: return run_kinetic_f0<T, 2>(st, a, f, num_sms);
    case 4: return run_kinetic_f0<T, 4>(st, a, f, num_sms);
    case 8: return run_kinetic_f0<T, 8>(st, a, f, num_sms);
    case 16: return run_kinetic_f0<T, 16>(st, a, f, num_sms);
    case 32: return run_kinetic_f0<T, 32>(st, a, f, num_sms);
    default: break;
    }
    const size_t smem = (10 + 8 * 4) * (size_t)a.pitch * sizeof(T);
    auto kern = k_kinetic_f0_wide<T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;   // row too long for shared memory
    int64_t blocks = (a.nslots + 7) / 8;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * per_sm);
    launch_pdl(kern, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), smem, st, a, f);
    return cudaGetLastError();
}

template cudaError_t launch_kinetic_f0<float>(cudaStream_t, const KinArgs<float> &, const F0Args<float> &, int);
template cudaError_t launch_kinetic_f0<double>(cudaStream_t, const KinArgs<double> &, const F0Args<double> &, int);

}  // namespace fp

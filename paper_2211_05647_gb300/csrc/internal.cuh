// internal.cuh -- handle layout, device helpers and kernel launchers shared by
// the translation units of the fdtd_plasma library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fdtd_plasma.h"

namespace fp {

// SI constants (CODATA 2018 exact / recommended values)
constexpr double kC0 = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------ programmatic dependent launch
// The kernels of a step are launched with launch_pdl: each may be scheduled
// while its predecessor on the stream is still finishing (the launch latency
// overlaps the predecessor's last wave), and begins with pdl_enter(), which
// waits for the predecessor grid to complete with its memory visible before any
// global access, then lets its own successor be scheduled.  Launched without
// the attribute (or after a non-kernel node) the wait returns at once.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch without programmatic serialization, for kernels that must not share
// SMs with early-launched neighbours: the TMA stencils hold up to ~170 KB of
// shared memory per SM, and dependent CTAs waiting beside them (a different
// shared-memory configuration) stalled the replayed 2-D step by 17 %.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ------------------------------------------------------------------ views

// Per-axis CPML profile at E (integer) and H (half-integer) positions, plus
// the psi slabs.  L == 0 means no CPML.  ik* hold 1/kappa.
template <typename T>
struct Cpml {
    int L;
    const T *be[3], *ae[3], *ike[3];
    const T *bh[3], *ah[3], *ikh[3];
    // 2-D: psi[0] ez_x  [ny][2L], psi[1] ez_y [2L][nx], psi[2] hx_y [2L][nx], psi[3] hy_x [ny][2L]
    // 3-D: slot 2*f + d (f = Ex..Hz, d = first / second curl axis), see fields.cu
    T *psi[12];
};

struct Source {
    int kind, loc;
    double amp, fc, tau, t0, dt;
    int64_t i, j, k, i0, i1, j0, j1;
    double *val;   // device scalar: g(t^{n+1}) of the current step, written by the H kernel
};

// g(t) of the soft source, FP64 on the device
__device__ __forceinline__ double source_value(const Source &s, double t)
{
    double u = (t - s.t0) / s.tau;
    if (s.kind == FDTD_SRC_GAUSS_SINE) return s.amp * sin(6.283185307179586 * s.fc * (t - s.t0)) * exp(-u * u);
    if (s.kind == FDTD_SRC_GAUSS) return s.amp * exp(-u * u);
    return 0.0;
}

template <typename TA>
struct KinArgs {
    const int32_t *slot_cell;  // polarisation node of each slot
    const TA *dens;            // density per slot
    void *df;                  // rows of `pitch` elements
    TA *E;                     // polarisation field (updated in place: E -= cj J)
    TA *jslot;                 // J^{n+1/2} per slot
    const TA *tab;             // [alpha | beta | w'] each `pitch` long, w' = -e w
    int64_t nslots;
    int pitch;
    TA cj;                     // dt / eps0
    uint64_t seed;
    const int64_t *d_step;     // steps done before the chunk
    int kstep;                 // step offset inside the chunk
    int64_t slot_base;         // global index of slot 0 (a sub-domain's rows count the stochastic-rounding
                               // draws like the whole grid's)
    int store_j;               // k_kinetic: store J^{n+1/2} per slot (the last step of a sequence, or
                               // when something reads it every step); E is updated either way
    int *err;                  // set to 1 if a bounded wait of the bulk-copy ring kernel gave up
};

// Isotropic-F0 evolution (speed grid): per-node tables, each `pitch` long,
// [f0 | f0' | bq | v^3 | 1/(v^2 gam) | 1/(2 v_e) | (m/M) v_e^3 nu_e | k Tg/(m v_e gam)]
// with bq = 2 dt (e/m) / (2 + dt nu) and v_e the node's upper cell edge (edge
// entries 0 at and past the last node); g = F0 - F0(table) rows.
template <typename TA>
struct F0Args {
    const TA *tab;
    TA *g;
    int nv;
    TA gam, inv2gam;   // speed-cell width and 1 / (2 gam)
    TA qm3;            // e / (3 m)
    TA mr, kTg_m;      // m / M, k Tg / m
    TA dt;
};

// ---------------------------------------------------------- compensated sums

// Knuth TwoSum: s + e == a + b exactly (round-to-nearest, no contraction).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    s = a + b;
    T z = s - a;
    e = (a - (s - z)) + (b - z);
}

// ------------------------------------------- Philox4x32-7 (Salmon et al. 2011)
// The 7-round variant, which the authors report passes TestU01's BigCrush;
// draws the stochastic-rounding bits, the recorder's sample selection and the
// closure training's initial weights and minibatch permutations.

__device__ __forceinline__ uint4 philox4x32_7(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 7; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Two-lane FP32 arithmetic (add / mul / fma .f32x2 on a register pair): each
// lane rounds exactly as the scalar instruction does, at one issue slot for
// two values.
__device__ __forceinline__ uint64_t f2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_split(uint64_t r)
{
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// FP32 -> BF16 with stochastic rounding: add 16 random bits below the kept
// mantissa and truncate (unbiased: rounds up with probability equal to the
// discarded fraction).
__device__ __forceinline__ uint16_t f32_to_bf16_sr(float x, uint32_t r16)
{
    uint32_t b = __float_as_uint(x);
    if ((b & 0x7f800000u) == 0x7f800000u) return (uint16_t)(b >> 16);   // inf / nan
    return (uint16_t)((b + (r16 & 0xffffu)) >> 16);
}

// -------------------------------------------------------------- launchers

template <typename T>
void launch_h1d(cudaStream_t st, const T *ex, T *hy, T *mur_state, int64_t nz, T ch, Source src,
                const int64_t *d_step, int kstep);
template <typename T>
void launch_e1d(cudaStream_t st, T *ex, const T *hy, int64_t nz, T ce, Source src, const int64_t *d_step, int kstep,
                const T *mur_state, T m);   // mur_state == nullptr: PEC ends
template <typename T>
void launch_h2d(cudaStream_t st, const T *ez, T *hx, T *hy, int64_t nx, int64_t ny, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 block, int cpt);
template <typename T>
void launch_e2d(cudaStream_t st, T *ez, const T *hx, const T *hy, int64_t nx, int64_t ny, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 block, int cpt);
template <typename T>
void launch_h3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ch, T cph, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 block, int cpt);
template <typename T>
void launch_e3d(cudaStream_t st, T *const f[6], int64_t nx, int64_t ny, int64_t nz, T ce, T cpe, Cpml<T> cp,
                Source src, const int64_t *d_step, int kstep, dim3 block, int cpt);
// 2-D / 3-D FP32 fused E^{n+1} + H^{n+3/2}: read fields fin and psi cin.psi, write fout and psi_out
// (2-D: rows > 0 with nx a multiple of 4 selects the column march, rows per block segment)
void launch_eh2d(cudaStream_t st, float *const fin[6], float *const fout[6], float *const psi_out[12], int64_t nx,
                 int64_t ny, float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                 const int64_t *d_step, int kstep, int rows);
void launch_eh3d(cudaStream_t st, float *const fin[6], float *const fout[6], float *const psi_out[12], int64_t nx,
                 int64_t ny, int64_t nz, float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                 const int64_t *d_step, int kstep);
void launch_advance(cudaStream_t st, int64_t *d_step, int64_t by);
// FP32 curl stencils fed by TMA (3-D: 32 x 8 columns walking tz planes along z; 2-D: 32-cell strips
// walking rows in 16-row chunks); the tensor maps describe one field set (nx a multiple of 4; maps made
// with nz == 1 are 2-D); timeouts of their bounded waits set bit 2 of *err
struct TmaMaps;
bool tma_stencil_eligible(int64_t nx, int64_t ny, int64_t nz);
TmaMaps *tma_maps_create(float *const f[6], int64_t nx, int64_t ny, int64_t nz);   // nullptr if not possible
void tma_maps_free(TmaMaps *t);
bool tma_maps_match(const TmaMaps *t, float *const f[6]);
void launch_h3d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, int64_t nz,
                    float ch, float cph, Cpml<float> cp, Source src, const int64_t *d_step, int kstep, int tz, int *err);
void launch_e3d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, int64_t nz,
                    float ce, float cpe, Cpml<float> cp, Source src, int tz, int *err);
// 2-D TMz strips fed by TMA (32-cell strips walking `rows` rows in 8-row chunks; maps made with nz == 1)
void launch_h2d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, float ch, float cph,
                    Cpml<float> cp, Source src, const int64_t *d_step, int kstep, int rows, int *err);
void launch_e2d_tma(cudaStream_t st, const TmaMaps *t, float *const f[6], int64_t nx, int64_t ny, float ce, float cpe,
                    Cpml<float> cp, Source src, int rows, int *err);
// fused E^{n+1} + H^{n+3/2} on TMA-staged planes between field sets 0 and 1 (both given to prepare);
// launch returns false (nothing launched) when fin is neither prepared set
bool tma_fused_prepare(TmaMaps *t, float *const f0[6], float *const f1[6]);
void tma_fused_forget(TmaMaps *t);
bool launch_eh3d_tma(cudaStream_t st, const TmaMaps *t, float *const fin[6], float *const fout[6],
                     float *const psi_out[12], float ce, float cpe, float ch, float cph, Cpml<float> cin, Source src,
                     const int64_t *d_step, int kstep, int tz, int *err);

// GPU compaction of a density array into plasma slots (compact.cu): chunks of kCompactChunk nodes; per
// chunk the number of plasma nodes and the largest density (bad |= 1 on a non-finite or negative value),
// then, from each chunk's exclusive-scan offset, its plasma nodes and densities in index order
constexpr int64_t kCompactChunk = 4096;
struct CompactGeom {
    int ndim;
    int64_t nx, ny, nz, n;   // grid cells per axis; n = length of the polarisation array
};
cudaError_t launch_compact_count(cudaStream_t st, const double *d, const CompactGeom &g, int *counts, double *maxes,
                                 int *bad);
cudaError_t launch_compact_scatter(cudaStream_t st, const double *d, const CompactGeom &g, const int64_t *offsets,
                                   int32_t *cells, double *dens);
// dst[i] = (float)src[i], i < n (round to nearest, as the host conversion)
cudaError_t launch_to_f32(cudaStream_t st, const double *src, float *dst, int64_t n);

// delta-f row pitch (elements) for nnode nodes of the given storage type
int kinetic_pitch(int nnode, int f_dtype);
// launch shape candidates (vectors per lane, lanes per row) for a row pitch; the first is the default
int kinetic_candidates(int pitch, int f_dtype, int (*out)[2]);
// returns cudaErrorInvalidValue for an unsupported combination; vpl <= 0 picks the default shape,
// bps > 0 caps the CTAs per SM; stages > 0 (FP32 / BF16 storage) selects the bulk-copy ring kernel
// with that many shared-memory stages (kinetic_ring.cu)
template <typename TA>
cudaError_t launch_kinetic(cudaStream_t st, const KinArgs<TA> &a, int f_dtype, int num_sms, int vpl = 0, int l = 0,
                           int bps = 0, int stages = 0);
// whether the ring kernel's tables and stages fit in one CTA's shared memory (FP32 / BF16 rows, stages >= 2)
bool kinetic_ring_fits(int pitch, int f_dtype, int l, int stages);
// the bulk-copy ring kernel for an FP32 / BF16 row shape (cudaErrorInvalidValue if the stages do not fit)
cudaError_t launch_kinetic_ring(cudaStream_t st, const KinArgs<float> &a, int f_dtype, int num_sms, int vpl, int l,
                                int bps, int stages);
// nonlinear mode (FP32 / FP64 storage): npar x nperp nodes, v_par spacing dvpar, qm = e/m
template <typename T>
cudaError_t launch_kinetic_f0(cudaStream_t st, const KinArgs<T> &a, const F0Args<T> &f, int num_sms);
template <typename T>
cudaError_t launch_kinetic_nl(cudaStream_t st, const KinArgs<T> &a, int npar, int nperp, double dvpar, double qm,
                              double dt, int num_sms);

struct DiagArgs {
    int ndim;
    int64_t nx, ny, nz;
    const void *f[6];
    int64_t flen[6];
    int precision;
    double ch;        // dt / (mu0 dx)
    double eps0_half_dv, mu0_half_dv;
    const void *df;
    int64_t nslots, nnode;
    int pitch, f_dtype;
    const double *dV; // per node, device
};
// out[0..6): energy, energy_plain, number, number_max_cell, number_abs, finite
// Running-DFT ports: block p averages pol[cells[off[p] .. off[p+1])] and adds
// it times exp(-i 2 pi freq[f] t^{n+1}) dt into acc[p][f][re, im].
template <typename T>
cudaError_t launch_ports(cudaStream_t st, const T *pol, int nports, const int64_t *off, const int64_t *cells,
                         const double *freq, double *acc, int nfreq, double dt, const int64_t *d_step, int kstep);

// Velocity-grid tables (host, FP64): node v_par (speed on the speed grid),
// current weight w, F0 and dF0/dv_par, volume element, |v|, s(|v|)|v| and its
// F0-weighted mean, nu.  velocity_tables() returns false for a bad grid kind;
// check_velocity_model() returns why the F0 / collision model is invalid, or NULL.
struct VTab {
    std::vector<double> v, w, f0, f0p, nu, dV, speed, sv;
    double mean_sv = 0.0;
};
const char *check_velocity_model(const fdtd_plasma_desc &p);
bool velocity_tables(const fdtd_plasma_desc &p, VTab &t);
// collision frequency of node j for a mean collision frequency nu0
inline double node_nu(const fdtd_plasma_desc &p, const VTab &t, size_t j, double nu0)
{
    return p.nu_model == FDTD_NU_CONST ? nu0 : nu0 * t.sv[j] / t.mean_sv;
}

cudaError_t launch_diag(cudaStream_t st, const DiagArgs &a, double *partials, int max_blocks, double *out);

// Faces of a Poynting box: f = 2 * axis + (0 lower, 1 upper); plane[f] is the
// E-node index of the face along its axis, lo/hi the cell range of the box on
// each axis, off[f] the first flat face-point index of face f (off[6] = total).
struct PoyntingBox {
    int64_t lo[3], hi[3];
    int64_t plane[6];
    int64_t off[7];
};
// out[0..6): power through faces x0, x1, y0, y1, z0, z1 along +axis; out[6] net outward
cudaError_t launch_poynting(cudaStream_t st, const DiagArgs &a, const PoyntingBox &b, double dA, double *partials,
                            int max_blocks, double *out);

struct ClosureArgs {
    const int32_t *cell;
    const float *dens;
    float *hist;       // [slot][16] ring of E^{n-15..n}
    float *jprev;      // J^{n-1/2} per slot
    float *jslot;      // J^{n+1/2} per slot (output)
    float *E;
    const float *P;    // packed FP32 network parameters
    int64_t n;
    float inv_es, inv_ns, js, rho, cj, beta;
    const int64_t *d_step;
    int kstep;
    int engine;        // 0: mma.sync warp tiles, 1: tcgen05 (TMEM accumulator)
    int store_j;       // store J^{n+1/2} in jslot (jprev, the state, is always written)
    int *err;          // set to 1 if a bounded wait gave up
};
cudaError_t launch_closure(cudaStream_t st, const ClosureArgs &a, int num_sms);
void launch_hist_push(cudaStream_t st, const int32_t *cell, int64_t n, const float *E, float *hist,
                      const int64_t *d_step, int kstep);
void launch_record(cudaStream_t st, int64_t n, const float *hist, const float *dens, const float *jslot, float *jprev,
                   float *out, int64_t capacity, unsigned long long *count, uint32_t threshold, uint64_t seed,
                   const int64_t *d_step, int kstep);

}  // namespace fp

// Record msg as the library-wide error (fdtd_plasma_last_error(NULL)) and return code.
int fp_set_global_error(int code, const char *msg);

// ------------------------------------------------------------------ handle

struct fdtd_plasma {
    fdtd_grid_desc g;
    fdtd_runtime_desc rt;
    cudaStream_t stream;      // caller's stream
    cudaStream_t cap;         // private stream used for graph capture
    int num_sms;
    double dt;
    int64_t nx, ny, nz;
    size_t esz;               // field element size
    void *f[6];
    int64_t flen[6];
    void *psi[12];
    int64_t psilen[12];
    // second field / psi set for the fused 3-D E+H kernel (allocated on first use)
    void *f2[6];
    void *psi2[12];
    int fuse;                 // FDTD_OPT_FUSED_STENCILS (default 0)
    int fuse_rows;            // FDTD_OPT_FUSED_ROWS: 2-D column-march rows per block (0: the 64 x 16 tiles)
    int auto_fuse_rows;       // the autotuner's choice on 2-D FP32 grids: > 0 runs the fused column march
    // guard bytes around every device allocation ($FDTD_PLASMA_CANARIES=1 at create)
    int canary;
    std::vector<std::pair<char *, size_t>> canary_allocs;   // (user pointer, user bytes)
    void *prof;               // CPML tables
    int64_t prof_len;
    void *mur_state;
    int64_t *d_step;
    double *d_src;            // g(t^{n+1}) of the step in flight
    int *d_err;               // device error word (bounded waits that gave up)
    int64_t steps_done;
    // domain decomposition along the slowest axis (fdtd_plasma_create_subdomain; sd_on = 0: a whole grid):
    // local plane l is global plane sd_origin + l; sd_lo / sd_hi ghost planes (0 or 1) below / above the
    // sd_extent owned ones; sd_half: 1 between the two halves of a step (fdtd_plasma_step_half)
    int sd_on, sd_axis, sd_half;
    int64_t sd_nglobal, sd_origin, sd_extent, sd_lo, sd_hi;
    int64_t slot_base;        // global plasma-slot index of local slot 0
    // plasma
    int has_plasma;
    fdtd_plasma_desc pl;
    int64_t nslots, nnode;
    int pitch;
    int32_t *slot_cell;
    void *dens, *df, *jslot, *tab;
    void *g0, *tab_f0;        // evolve_f0: F0 correction rows and the F0 tables
    double *dV;               // per node (FP64) for the diagnostics
    size_t df_esz;
    size_t df_bytes;          // size of the df allocation (kept by a set_plasma of the same size)
    int64_t nkin;             // slots [0, nkin) take the kinetic update (all, unless a closure is set)
    std::vector<int32_t> h_cells;   // host copies of the slot layout
    std::vector<double> h_dens;
    // learned closure: slots [nkin, nslots)
    int has_closure;
    int64_t ncl;
    float *hist, *jprev, *params;
    fdtd_closure_desc cl;
    // training-data recorder
    // launch shapes (autotuner / cache): kinetic (vectors per lane, lanes per row, CTAs per SM; 0 = default),
    // stencil block (0 = default)
    int kin_vpl, kin_l, kin_bps, kin_stages;   // kinetic launch shape; kin_stages > 0: the bulk-copy ring kernel
    int st_bx, st_by, st_bz, st_cpt;
    int st_tz;                // > 0: 3-D FP32 stencils run the TMA column kernels with tz planes per block
    fp::TmaMaps *tma;         // their tensor maps (field set 0), made on first use
    int has_recording;
    float *rec_out;
    int64_t rec_cap;
    unsigned long long *rec_count;
    uint32_t rec_threshold;
    uint64_t rec_seed;
    // source
    int has_source;
    fdtd_source_desc src;
    // graphs
    cudaGraphExec_t g1, gk;
    cudaGraphExec_t gpow[4];   // 2-, 4-, 8- and 16-step graphs for a call's remainder (captured on first use)
    int gk_steps;
    int graphs_valid;
    // running-DFT ports (device arrays; nports = 0: none)
    int nports, nfreq;
    int64_t *port_off, *port_cells;
    double *port_freq, *port_acc;
    // diagnostics scratch
    double *diag_partials;
    int diag_blocks;
    double *diag_out;
    std::string err;
};

/*
 * fdtd_plasma.h -- C ABI of the GB300 (sm_103a) coupled Yee-FDTD + kinetic
 * electron solver of arXiv 2211.05647.
 *
 * One time step n -> n+1 advances, in this order:
 *   H^{n+1/2}  Yee curl of E^n + CPML psi_h           (Sec. 2, Eq. 1, 7-12)
 *   df^{n+1/2} Crank-Nicolson f_1 update per plasma cell and velocity node,
 *              driven by E^n                           (Sec. 5.2, Eq. 22 and the f_1x update)
 *   J^{n+1/2}  = -e sum_j w_j df_j^{n+1/2}             (Eq. 24 and the Jx sum of Sec. 5.2)
 *   E^{n+1}    Yee curl of H^{n+1/2} + CPML psi_e - dt/eps0 J^{n+1/2}   (Eq. 2-6)
 *   soft source g(t^{n+1}) added at its node(s); first-order Mur ends in 1-D.
 *
 * Conventions (all entry points):
 *   - Every call returns an fdtd_status; nothing throws across the ABI.
 *   - A handle is not thread-safe.  All device work is issued on the stream
 *     given at create time and is asynchronous unless stated.
 *   - The caller owns every pointer it passes; inputs are copied before the
 *     call returns, outputs are written before it returns (for device
 *     destinations: stream-ordered, see fdtd_plasma_read_fields).
 *   - Units are SI.  Fields are stored x-fastest, without padding:
 *       1-D: Ex on nodes k = 0..nz (nz+1 values), Hy on k+1/2 (nz values).
 *       2-D TMz: Ez(i,j), Hx(i,j+1/2), Hy(i+1/2,j): nx*ny values at j*nx+i;
 *                Ez on i==0 or j==0 is a PEC node, nodes i==nx / j==ny are PEC ghosts.
 *       3-D: Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Hx(i,j+1/2,k+1/2)
 *            Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k): nx*ny*nz values at (k*ny+j)*nx+i,
 *            tangential E on the low planes held at 0, high planes are ghosts.
 *   - The kinetic current sits on the polarisation component: Ex (1-D, 3-D)
 *     or Ez (2-D TMz).  Plasma cells are polarisation nodes with density > 0
 *     whose E the curl updates; they are numbered ("slots") in increasing
 *     linear index.
 */
#ifndef FDTD_PLASMA_H
#define FDTD_PLASMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_plasma *fdtd_plasma_t;

typedef enum {
    FDTD_OK = 0,
    FDTD_ERR_INVAL = -1,     /* bad argument, size or combination */
    FDTD_ERR_NOMEM = -2,     /* device allocation failed */
    FDTD_ERR_CUDA = -3,      /* a CUDA call failed; see fdtd_plasma_last_error */
    FDTD_ERR_UNSTABLE = -4,  /* Courant / plasma stability bound violated */
    FDTD_ERR_NONFINITE = -5, /* non-finite input or state */
    FDTD_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
    FDTD_ERR_STATE = -7      /* call not allowed in the handle's current state */
} fdtd_status;

enum { FDTD_F32 = 0, FDTD_F64 = 1 };                      /* field / accumulation precision */
enum { FDTD_DF_F32 = 0, FDTD_DF_BF16 = 1, FDTD_DF_F64 = 2 }; /* storage of delta f */
enum { FDTD_VGRID_SIGNED1D = 0, FDTD_VGRID_CART2D = 1, FDTD_VGRID_SPEED3D = 2 };
enum { FDTD_NU_NSV = 0, FDTD_NU_CONST = 1, FDTD_NU_TABLE = 2 };
enum { FDTD_F0_MAXWELL = 0, FDTD_F0_DRUYVESTEYN = 1 };
enum { FDTD_SRC_NONE = 0, FDTD_SRC_GAUSS_SINE = 1, FDTD_SRC_GAUSS = 2 };
enum { FDTD_LOC_POINT = 0, FDTD_LOC_SHEET = 1 };
enum {                                                      /* fdtd_plasma_read_fields "which" */
    FDTD_EX = 0, FDTD_EY, FDTD_EZ, FDTD_HX, FDTD_HY, FDTD_HZ,
    FDTD_J = 6,  /* J^{n+1/2} per plasma slot, field precision */
    FDTD_DF = 7, /* delta f [slot][node], delta-f storage type, rows packed to nnode */
    FDTD_F0 = 8  /* evolve_f0: F0 - F0(table) per unit density [slot][node], delta-f storage type */
};

/* Grid and boundary description (Sec. 2; CPML of Eq. 7-12). */
typedef struct {
    int32_t ndim;              /* 1, 2 (TMz) or 3 */
    int32_t precision;         /* FDTD_F32 or FDTD_F64 */
    int64_t nx, ny, nz;        /* cells per axis; 1-D uses nz; unused axes ignored */
    double dx;                 /* cell size on every axis (m) */
    double courant;            /* S: dt = S dx / c; must satisfy S^2 ndim < 1 */
    int32_t cpml_cells;        /* 2-D/3-D CPML thickness on every face (0 = PEC walls) */
    int32_t mur;               /* 1-D: 1 = first-order Mur at both ends, 0 = PEC ends */
    double cpml_order;         /* n_cpml of Eq. 9-12 */
    double cpml_sigma_factor;  /* sigma_max = factor (order+1)/(150 pi dx), Eq. 11 */
    double cpml_kappa_max;
    double cpml_alpha_min, cpml_alpha_max;   /* S/m, Eq. 12 */
} fdtd_grid_desc;

/* Runtime plumbing: the stream every call issues on, and an optional device
 * allocator (e.g. a framework's caching allocator).  alloc must return
 * 256-byte aligned device memory or NULL; both callbacks may be NULL, in
 * which case cudaMalloc / cudaFree are used. */
typedef struct {
    void *stream;                                   /* cudaStream_t, NULL = legacy default stream */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
} fdtd_runtime_desc;

/* Soft source, added to the polarisation component after the E update at
 * t^{n+1} (Table 3 pulse):  GAUSS_SINE: amp sin(2 pi fc (t-t0)) exp(-((t-t0)/tau)^2)
 *                            GAUSS:      amp exp(-((t-t0)/tau)^2)
 * POINT: node (i,j,k) (1-D uses k; 2-D uses i,j).  SHEET (3-D): every node
 * (i,j,k) with i0<=i<i1, j0<=j<j1 on plane k. */
typedef struct {
    int32_t kind;
    int32_t location;
    double amp, fc, tau, t0;
    int64_t i, j, k;
    int64_t i0, i1, j0, j1;
} fdtd_source_desc;

/* Kinetic plasma (Sec. 5.2).  density: one double per polarisation node
 * (the field's own length), host or device, copied.  The velocity grid has nv
 * (x nv_perp) midpoint nodes over [-vmax_vth v_th, +vmax_vth v_th] (speed
 * grid: [0, vmax_vth v_th]), v_th = sqrt(e te_ev / m).
 * F0 (isotropic, fixed): f0_model MAXWELL, of temperature te_ev; DRUYVESTEYN,
 * A exp(-(eps/eps0)^2) with eps = m v^2/2 and mean energy 3/2 e te_ev
 * (eps0 = 3/2 e te_ev Gamma(3/4)/Gamma(5/4)).  The signed grid carries the
 * 1-D marginal of F0 and the Cartesian grid the 2-D marginal (for the
 * Druyvesteyn F0 by quadrature over the third component), with their v_par
 * derivatives.
 * Collisions (Eq. 23): NSV: nu_j = N s |v_j| with N s set so that the grid's
 * F0-weighted mean of nu is nu0; CONST: nu_j = nu0; TABLE: nu_j = N s(|v_j|)
 * |v_j|, N set the same way, s(v) linear between the s_n >= 2 points of the
 * table (s_speed strictly ascending, m/s; s_sigma >= 0, any unit: only its
 * shape matters) and held at the end values outside it.  The table is host
 * memory, read during set_plasma only.  |v_j| is |v_par| on the signed grid,
 * sqrt(v_par^2 + v_perp^2) on the Cartesian grid, the speed on the speed grid.
 * f_dtype: FDTD_DF_F32, FDTD_DF_BF16 (FP32 arithmetic, stochastic rounding on
 * store, keyed by seed) or FDTD_DF_F64 (only with FDTD_F64 precision).
 * nonlinear: 1 adds the flux-form advection of delta f in v_par (signed and
 * Cartesian grids only).
 * evolve_f0: 1 lets the isotropic part evolve per cell (speed grid, FP32 or
 * FP64 delta f, no closure): F0 = F0(table) + g, g per unit density, with the
 * two-term F0 equation dF0/dt = (e E / (3 m v^2)) d/dv (v^2 F1) + C0(F0),
 * C0 = (m/M)(1/v^2) d/dv [v^3 nu (F0 + (k Tg/(m v)) dF0/dv)] (elastic
 * collisions with gas atoms of mass ratio mass_ratio = m/M at temperature
 * tg_ev), both in flux form on the speed cells (zero flux at 0 and v_max),
 * heating from the time-centred F1 = delta f / n; the F1 update then uses
 * F0' = F0'(table) + central differences of g. */
typedef struct {
    const double *density;
    int32_t density_on_device;
    int32_t vgrid;
    int32_t nv, nv_perp;
    double te_ev, vmax_vth, nu0;
    int32_t nu_model;
    int32_t f_dtype;
    int32_t nonlinear;
    int32_t f0_model;
    uint64_t seed;
    const double *s_speed;     /* FDTD_NU_TABLE only (else ignored) */
    const double *s_sigma;
    int64_t s_n;
    int32_t evolve_f0;
    int32_t reserved;
    double mass_ratio, tg_ev;  /* evolve_f0 only */
} fdtd_plasma_desc;

/* FP64 diagnostics (computed on the device with FP64 accumulators). */
typedef struct {
    double energy;          /* sum eps0/2 E^2 dV + mu0/2 H . H' dV, H' = H advanced by the vacuum curl
                               of the current E: the Yee invariant of a lossless PEC cavity */
    double energy_plain;    /* sum eps0/2 E^2 dV + mu0/2 H^2 dV */
    double number;          /* sum over plasma cells and nodes of df_j dV_j */
    double number_max_cell; /* max over cells of |sum_j df_j dV_j| */
    double number_abs;      /* sum |df_j| dV_j */
    int64_t finite;         /* 1 if every field and df value is finite */
    int64_t step;           /* steps done */
} fdtd_diag;

/* Create a solver.  Validates the grid (sizes >= 2, dx > 0, CPML thinner
 * than a third of each axis) and the Courant number (FDTD_ERR_UNSTABLE if
 * S^2 ndim >= 1).  Fields start at zero, there is no plasma and no source.
 * rt may be NULL.  On error *out is NULL. */
int fdtd_plasma_create(const fdtd_grid_desc *grid, const fdtd_runtime_desc *rt, fdtd_plasma_t *out);

/* Set (or replace) the soft source.  Validates the node range.
 * Allowed at any time; takes effect from the next step. */
int fdtd_plasma_set_source(fdtd_plasma_t h, const fdtd_source_desc *src);

/* Set the plasma: compacts plasma cells, builds the velocity tables and
 * zeroes delta f and J.  FDTD_ERR_STATE after the first step (call
 * fdtd_plasma_reset first); FDTD_ERR_NONFINITE for a non-finite or negative
 * density; FDTD_ERR_UNSTABLE if (w_p,max dt/2)^2 + S^2 ndim >= 1. */
int fdtd_plasma_set_plasma(fdtd_plasma_t h, const fdtd_plasma_desc *pl);

/* Advance nsteps >= 0 steps, asynchronously on the handle's stream.  The
 * first call after a configuration change captures the step sequence into
 * CUDA graphs; later calls replay them. */
int fdtd_plasma_step(fdtd_plasma_t h, int64_t nsteps);

/* Advance nsteps >= 1 steps like fdtd_plasma_step, but launch each kernel
 * directly (no graph) with CUDA events around each kernel of a step,
 * synchronising after every step.  ms_out[0..4] receive the average duration
 * per step (ms) of the H-stencil kernel, the kinetic (delta f + J) kernel,
 * the closure kernel (0 without a closure), the E-stencil kernel (with the
 * Mur ends in 1-D) and of a whole step.  Meant for measurement; state
 * advances exactly as with step. */
int fdtd_plasma_time_kernels(fdtd_plasma_t h, int64_t nsteps, double *ms_out);

/* Launch-shape autotuner.  Times, with CUDA events on the handle's stream,
 * every candidate shape of the kinetic kernel (vectors per lane x lanes per
 * row x CTAs per SM) and of the curl-stencil kernels (thread-block shape,
 * cells per thread, on FP32 grids the TMA column kernels, and on 2-D FP32
 * grids the fused E + H column march against the best separate pair) on
 * the handle's own buffers, adopts the fastest, and records them in a text
 * cache ($FDTD_PLASMA_TUNE_CACHE, else $HOME/.cache/fdtd_plasma/autotune.txt)
 * keyed by GPU name, kernel, precision and size class; later handles of the
 * same class start from the cached shapes.  The state is saved before and
 * restored bit for bit after (needs one temporary copy of it on the device).
 * Synchronous. */
typedef struct {
    int32_t kin_vpl, kin_l, kin_blocks_per_sm;   /* 0 = no kinetic kernel tuned */
    int32_t block_x, block_y, block_z;           /* 0 = no stencil tuned (1-D) */
    double kin_ms, stencil_ms;                   /* best per-launch times */
    int32_t cells_per_thread;                    /* stencils: 1, or 4 (FP32 rows of a multiple of 4 cells;
                                                    block_x then counts groups of 4 cells) */
    int32_t stencil_tz;                          /* FP32, nx a multiple of 4: > 0 when the TMA stencils won
                                                    -- 32 x 8 threads, each block walking stencil_tz planes
                                                    (3-D) or rows (2-D); 0 = grid-of-cells kernels */
    int32_t kin_stages;                          /* 0 = the register kernel; S > 0 = the bulk-copy ring
                                                    kernel with S shared-memory stages (FP32 / BF16 rows:
                                                    a producer warp copies chunks of 256 / kin_l rows, with
                                                    their cell indices and densities, ahead of eight
                                                    consumer warps; same results bit for bit) */
    int32_t fused_rows;                          /* 2-D FP32, nx a multiple of 4, whole grid: > 0 when the
                                                    fused E + H column march beat the best separate pair
                                                    (rows per block segment; the step sequence then runs
                                                    it, with a second field / psi set, same results bit
                                                    for bit); 0 = separate passes */
} fdtd_tune_result;
int fdtd_plasma_autotune(fdtd_plasma_t h, fdtd_tune_result *out);

/* Guard bytes (no counterpart in the paper; a stand-in for a memory checker):
 * when the environment variable FDTD_PLASMA_CANARIES is "1" at
 * fdtd_plasma_create, every device allocation of the handle gets 256 bytes of
 * a fixed pattern before and after it.  This call synchronises the handle's
 * stream and stores in *corrupted (host) how many allocations have a changed
 * guard byte; FDTD_ERR_STATE when the handle was created without guards. */
int fdtd_plasma_check_canaries(fdtd_plasma_t h, int64_t *corrupted);

/* Self-test of the bounded waits (no counterpart in the paper): the tcgen05
 * kernels wait for their tensor-core results, and the TMA column stencils for
 * their plane loads, on mbarriers with an iteration or wall-clock limit, after which they
 * set an error word (reported as FDTD_ERR_TIMEOUT by fdtd_plasma_diagnostics
 * and by host reads of fdtd_plasma_read_fields) and return instead of hanging.  This launches one
 * CTA that waits, with the same helper, on a barrier nothing arrives at, for
 * max_iter tries (1..2^20), and stores 1 in *gave_up (host) when the wait gave
 * up as designed, 0 if it completed.  Synchronous, on the legacy stream. */
int fdtd_selftest_wait_timeout(uint32_t max_iter, int32_t *gave_up);

/* The same for the wall-clock-bounded wait of the TMA column stencils (the
 * waiting thread sleeps in the barrier between polls): one CTA waits on a
 * barrier nothing arrives at until limit_us microseconds (1..10^6) have
 * passed on the GPU's global timer, then stores 1 in *gave_up (host).
 * Synchronous, on the legacy stream; FDTD_ERR_INVAL for a bad argument. */
int fdtd_selftest_timed_wait(uint32_t limit_us, int32_t *gave_up);

/* Runtime options.  FDTD_OPT_FUSED_STENCILS (default 0): 1 makes the step
 * sequence on 2-D and 3-D FP32 grids fuse each E update with the next H update into
 * one pass (fields and CPML psi double-buffered: one extra copy of them is
 * allocated on first use; the fields are back in place when
 * fdtd_plasma_step returns).  It moves a third fewer bytes; in 3-D it is
 * slower than the two separate passes on GB300, in 2-D (the column march
 * below) faster on large grids, where fdtd_plasma_autotune selects it by
 * itself (fdtd_tune_result.fused_rows; half steps stay allowed then).
 * Results equal the unfused sequence bit for bit in 2-D and where the 3-D TMA
 * column stencils below are selected (their fused pass then runs on
 * TMA-staged planes too), else up to FP32 rounding order.  0 turns the
 * option off (and frees the copy unless the autotuner chose the fused pass).
 * FDTD_OPT_STENCIL_TZ: 0 selects the grid-of-cells stencil kernels; a value
 * tz in 1..1024 selects the TMA kernels (2-D and 3-D FP32, nx a multiple of 4):
 * 32 x 8 threads per block; in 3-D each block walks tz planes along z, in 2-D
 * tz rows (rounded up to a multiple of 8) of a 32-cell strip, in 8-row chunks;
 * planes / chunks are staged in shared memory by tensor copies.  The
 * autotuner sets it too (fdtd_tune_result.stencil_tz).  Results equal the
 * one-cell-per-thread kernels bit for bit.
 * FDTD_OPT_KINETIC_SHAPE: the kinetic kernel's launch shape, value =
 * stages * 10^9 + vpl * 10^6 + l * 1000 + bps (ring stages or 0, vectors per
 * lane, lanes per row, CTAs per SM cap or 0); (vpl, l) must be one of the row
 * length's candidates (the ones fdtd_plasma_autotune times), stages 0 (the
 * register kernel) or 2..64 (the bulk-copy ring kernel: FP32 / BF16 rows of
 * the linear update, stages that fit in one CTA's shared memory); 0 returns
 * to the built-in default.
 * Needs a plasma (after set_plasma).  The autotuner overwrites it.
 * FDTD_OPT_FUSED_ROWS (2-D fused pass, nx a multiple of 4): rows per block
 * segment of the column-march kernel (1..4096, default 8; each warp owns a
 * 128-column strip and marches up the segment with no shared memory); 0
 * selects the 64 x 16 shared-memory tiles instead.  Both equal the unfused
 * sequence up to FP32 rounding order.
 * FDTD_ERR_INVAL for an unknown option or value. */
enum { FDTD_OPT_FUSED_STENCILS = 1, FDTD_OPT_STENCIL_TZ = 2, FDTD_OPT_KINETIC_SHAPE = 3, FDTD_OPT_FUSED_ROWS = 4 };
int fdtd_plasma_set_option(fdtd_plasma_t h, int option, int64_t value);

/* The launch shapes the handle uses now (tuned, cached or default; kinetic
 * fields 0 = the built-in choice); times are 0. */
int fdtd_plasma_launch_shapes(fdtd_plasma_t h, fdtd_tune_result *out);

/* Zero every field, psi, delta f and J and the step counter (keeps the
 * configuration). */
int fdtd_plasma_reset(fdtd_plasma_t h);

/* Copy one quantity out.  bytes must equal its exact size (see
 * fdtd_plasma_quantity_bytes).  dst_is_device = 0: host memory, the call
 * synchronises the handle's stream before returning.  dst_is_device = 1:
 * device memory, stream-ordered on the handle's stream. */
int fdtd_plasma_read_fields(fdtd_plasma_t h, int which, void *dst, size_t bytes, int dst_is_device);

/* Overwrite one quantity (same layout as read_fields; FDTD_J is not
 * writable).  Used to set initial conditions. */
int fdtd_plasma_write_fields(fdtd_plasma_t h, int which, const void *src, size_t bytes, int src_is_device);

/* Byte size of a quantity for read/write_fields (0 if absent). */
size_t fdtd_plasma_quantity_bytes(fdtd_plasma_t h, int which);

/* Number of plasma slots and velocity nodes per slot. */
int fdtd_plasma_plasma_shape(fdtd_plasma_t h, int64_t *nslots, int64_t *nnode);

/* Time step dt (s) and steps done. */
int fdtd_plasma_info(fdtd_plasma_t h, double *dt, int64_t *steps_done);

/* Compute FP64 diagnostics of the current state (synchronises the stream). */
int fdtd_plasma_diagnostics(fdtd_plasma_t h, fdtd_diag *out);

/* Running-DFT ports (Sec. 5.3: the slab's S-parameters S11, S21 come from the
 * spectra of the field at two ports).  Port p is the set of polarisation-field
 * nodes cells[port_offsets[p] .. port_offsets[p+1]) (indices into Ex in 1-D
 * and 3-D, Ez in 2-D, x fastest; port_offsets[0] = 0, every port non-empty).
 * After every step, the port's field E^{n+1} averaged over its nodes is
 * accumulated in FP64 as X[p][f] += E_p(t) exp(-i 2 pi freqs[f] t) dt with
 * t = (n+1) dt.  All arrays are host memory, copied; the call synchronises.
 * set_ports zeroes the sums (as does fdtd_plasma_reset); nports = 0 removes
 * the ports.  The sums are not part of the checkpoint state.
 * S11 = (X_plasma[in] - X_vacuum[in]) / X_vacuum[in] and
 * S21 = X_plasma[out] / X_vacuum[out] with a vacuum run of the same source.
 * Errors: FDTD_ERR_INVAL for counts outside 1..4096 ports / 1..2^20
 * frequencies, NULL arrays, empty ports, nodes outside the field or
 * non-finite frequencies. */
int fdtd_plasma_set_ports(fdtd_plasma_t h, int32_t nports, const int64_t *port_offsets, const int64_t *cells,
                          int32_t nfreq, const double *freqs);

/* Copy the port sums out: out (host) holds nports x nfreq x {re, im} doubles,
 * bytes must be exactly that size; synchronises.  FDTD_ERR_STATE without ports. */
int fdtd_plasma_read_ports(fdtd_plasma_t h, double *out, size_t bytes);

/* Electromagnetic power out of an axis-aligned box at the current step (the
 * Poynting vector S = E x H of the field equations of Sec. 2, Eq. 1-2),
 * computed in FP64 whatever the field precision; synchronises the stream.
 *   box = {i0, i1, j0, j1, k0, k1} (host, 6 values): the faces are the E-node
 *     planes i = i0, i1 (x), j = j0, j1 (y), k = k0, k1 (z); each face sums
 *     over cell indices [lo, hi) of its two in-plane axes.  Axes the grid does
 *     not have are ignored (1-D: only k0, k1, 0 <= k <= nz; 2-D: only x and y).
 *     Used axes need 0 <= lo <= hi < number of E nodes on that axis.
 *   E is E^n; H is time-centred at n, (H^{n-1/2} + H^{n+1/2}) / 2 with the
 *     vacuum curl of E^n, averaged onto the face plane from the H nodes on
 *     either side (nodes off the grid count as 0); face element dx^2 (3-D),
 *     dx (2-D), 1 (1-D).
 *   out (host, 7 doubles): power through faces x0, x1, y0, y1, z0, z1 along
 *     +axis (W, W/m or W/m^2 for 3-D, 2-D, 1-D), out[6] = net outward power
 *     x1 - x0 + y1 - y0 + z1 - z0.
 * Returns FDTD_ERR_INVAL for a NULL argument or a face outside the grid. */
int fdtd_plasma_poynting(fdtd_plasma_t h, const int64_t *box, double *out);

/* Checkpoint: the full state (fields, psi, delta f, J, step counter) in an
 * opaque byte blob of fdtd_plasma_state_bytes() bytes, host or device.
 * load_state requires a handle with the same configuration. */
size_t fdtd_plasma_state_bytes(fdtd_plasma_t h);
int fdtd_plasma_save_state(fdtd_plasma_t h, void *buf, size_t bytes, int buf_is_device);
int fdtd_plasma_load_state(fdtd_plasma_t h, const void *buf, size_t bytes, int buf_is_device);

/* ---------------------------------------------------------------------
 * Learned J closure (not in the paper: a small network standing in for the
 * Sec. 5.2 velocity-space update).  Per plasma cell with n <= n_train_max:
 *   x = [E^{n-15} .. E^n] / e_scale ++ [n / n_scale]          (17 inputs)
 *   y = MLP(x): 17 -> 128 -> 128 -> 1, GELU in its tanh form (Hendrycks &
 *       Gimpel) on both hidden layers,
 *       BF16 tensor-core operands, FP32 accumulation
 *   J^{n+1/2} = rho J^{n-1/2} + beta n E^n + j_scale y
 *       (beta n E^n is the Drude increment of a constant-collision plasma, so
 *       the network learns the kinetic correction; rho = beta = 0 gives the
 *       direct form J = j_scale y)
 *   E^n <- E^n - dt/eps0 J^{n+1/2}
 * Cells with n > n_train_max keep the kinetic update.
 * Parameters: FDTD_MLP_NPARAMS FP32 values packed
 *   W1[17][128] b1[128] W2[128][128] b2[128] W3[128] b3[1]  (row-major, y = ((x W1 + b1) ...)). */
#define FDTD_MLP_NIN 17
#define FDTD_MLP_NHID 128
#define FDTD_MLP_NPARAMS 18945

typedef struct {
    const float *params;        /* FDTD_MLP_NPARAMS floats, host or device, copied */
    int32_t params_on_device;
    int32_t engine;             /* 0: mma.sync warp tiles; 1: tcgen05 MMA with a tensor-memory
                                   accumulator (bounded completion waits: a wait that gives up makes
                                   fdtd_plasma_diagnostics return FDTD_ERR_TIMEOUT) */
    double e_scale, j_scale, n_scale, rho, n_train_max;
    double beta;                /* Drude increment coefficient (A m / V per unit density) */
} fdtd_closure_desc;

/* Switch a plasma to the closure (FP32 grids, after set_plasma, before the
 * first step).  Re-lays the slots out: kinetic (fallback) cells first, then
 * closure cells, each in increasing cell index; FDTD_J follows that order,
 * FDTD_DF holds only the kinetic rows. */
int fdtd_plasma_set_closure(fdtd_plasma_t h, const fdtd_closure_desc *c);
int fdtd_plasma_closure_shape(fdtd_plasma_t h, int64_t *n_kinetic, int64_t *n_closure);

/* Training-data recorder (kinetic FP32 runs): from the next step on, every
 * plasma cell keeps a 16-step ring of E^n, and each (cell, step) pair is
 * selected with probability `rate` by a counter-based draw keyed by `seed`;
 * a selected pair appends [E^{n-15} .. E^n, n, J^{n+1/2}, J^{n-1/2}] (19
 * floats) at samples[19 * atomicAdd(count, 1)] while that index is below
 * capacity (the counter keeps counting).  samples and count are caller-owned
 * device memory; the caller zeroes count. */
int fdtd_plasma_set_recording(fdtd_plasma_t h, float *samples, int64_t capacity, unsigned long long *count, double rate,
                              uint64_t seed);

/* Training / inference of the closure network on caller-owned device
 * buffers (stream-ordered on `stream`):
 *   forward  : y[b] = MLP(x[b]) for x [batch][17]
 *   loss_grad: loss = mean (y - target)^2 and its gradient (packed like the
 *              parameters, overwritten) -- forward and backward contractions
 *              on BF16 tensor-core tiles with FP32 accumulation, one CTA per
 *              128-row tile, the tiles' gradients summed in a fixed order
 *              (deterministic); workspace of fdtd_mlp_workspace_bytes(batch)
 *              bytes (one gradient per tile: about 74 KB per 128 rows)
 *   adam     : one Adam step (Kingma & Ba, bias-corrected, step count t >= 1)
 *              on params with first / second moments m, v. */
size_t fdtd_mlp_workspace_bytes(int64_t batch);
int fdtd_mlp_forward(const float *params, const float *x, int64_t batch, float *y, void *stream);
/* The same forward on the 5th-generation tensor cores (tcgen05 MMA into a
 * tensor-memory accumulator, one warpgroup per 128-row tile).  Its internal
 * completion waits are bounded: if one gives up, *err (device int, caller
 * zeroed) is set to 1 and the affected outputs are NaN. */
int fdtd_mlp_forward_tc(const float *params, const float *x, int64_t batch, float *y, int *err, void *stream);
int fdtd_mlp_loss_grad(const float *params, const float *x, const float *target, int64_t batch, float *grad,
                       float *loss, void *workspace, size_t workspace_bytes, void *stream);
int fdtd_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t n, int64_t t, double lr, double beta1,
                  double beta2, double eps, void *stream);

/* Closure training pipeline on recorded samples (caller-owned device
 * buffers; see fdtd_plasma_set_recording for the 19-float sample layout).
 *
 * fdtd_closure_scales: the closure desc's normalisation and Drude part.
 *   rho  = (2 - dt nu_mean) / (2 + dt nu_mean),
 *   beta = 2 dt (e^2/m) / (2 + dt nu_mean)  -- the Crank-Nicolson f_1x update
 *          and Jx sum of Sec. 5.2 with nu(v) = nu_mean, which reduce to a
 *          Drude current (rho = beta = 0 when increment == 0: direct form);
 *   n_scale = n_c = eps0 m omega0^2 / e^2 (critical density at omega0, rad/s);
 *   e_scale = RMS of the 16 recorded E values over all samples;
 *   j_scale = RMS of r = J^{n+1/2} - rho J^{n-1/2} - beta n E^n over all
 *             samples (eps0 omega0 e_scale if every r is 0).
 *   FP64 sums on the device; `out` is host memory (the stream is
 *   synchronised).  workspace: fdtd_closure_workspace_bytes() bytes of device
 *   memory.  Errors: FDTD_ERR_INVAL (NULL, n < 1, dt / omega0 not > 0),
 *   FDTD_ERR_NONFINITE (E all zero or not finite).
 * fdtd_closure_dataset: network inputs x [n][17] = [E^{n-15..n} / e_scale,
 *   n / n_scale] and targets t [n] = r / j_scale, computed in FP64, stored
 *   FP32 (device, stream-ordered).
 * fdtd_mlp_init: seeded He-style initial parameters (W1 ~ N(0, 2/17),
 *   W2 ~ N(0, 2/128), W3 ~ N(0, 1/128), biases 0; Philox4x32-7 + Box-Muller).
 * fdtd_mlp_gather: rows first .. first + batch - 1 of a seeded permutation of
 *   [0, n) for `epoch` (a four-round Feistel network with cycle walking),
 *   copied to xb [batch][17], tb [batch]; needs first + batch <= n.
 * fdtd_mlp_train_epoch: one epoch of minibatch training: for each of the
 *   n / batch full batches of the epoch's permuted order (the ragged tail is
 *   left out), the same loss and gradient as fdtd_mlp_loss_grad on the rows
 *   fdtd_mlp_gather would give, then the Adam step of fdtd_mlp_adam with step
 *   count iter0 + b + 1 and the cosine-decayed rate lr (1 + cos(pi (iter0 + b)
 *   / total_iters)) / 2 -- bit for bit those calls, in two kernel launches a
 *   batch (the rows are read through the permutation; the tiles' gradients
 *   are summed and applied in one kernel).  *loss_mean (device double)
 *   receives the mean of the batch losses.  m, v: FDTD_MLP_NPARAMS floats
 *   each (zeroed by the caller before the first epoch); grad is not used (may
 *   be NULL); workspace of fdtd_mlp_train_workspace_bytes(batch) bytes.
 *   Nothing is synchronised. */
typedef struct {
    double e_scale, j_scale, n_scale, rho, beta;
} fdtd_closure_scales_t;
size_t fdtd_closure_workspace_bytes(void);
int fdtd_closure_scales(const float *samples, int64_t n, double omega0, double dt, double nu_mean, int increment,
                        fdtd_closure_scales_t *out, void *workspace, size_t workspace_bytes, void *stream);
int fdtd_closure_dataset(const float *samples, int64_t n, const fdtd_closure_scales_t *sc, float *x, float *t,
                         void *stream);
int fdtd_mlp_init(float *params, uint64_t seed, void *stream);
int fdtd_mlp_gather(const float *x, const float *t, int64_t n, uint64_t seed, int64_t epoch, int64_t first,
                    int64_t batch, float *xb, float *tb, void *stream);
size_t fdtd_mlp_train_workspace_bytes(int64_t batch);
int fdtd_mlp_train_epoch(float *params, float *grad, float *m, float *v, const float *x, const float *t, int64_t n,
                         int64_t batch, uint64_t seed, int64_t epoch, int64_t iter0, int64_t total_iters, double lr,
                         double beta1, double beta2, double eps, double *loss_mean, void *workspace,
                         size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------
 * Batches of independent 1-D runs (same step as above, per run), advanced by
 * one persistent kernel launch per fdtd_batch_step call (graph-captured).
 * Runs may differ in nz, Mur / PEC ends, density profile, nu0 and source;
 * they must share dx, courant, precision, the velocity grid, te, nu model and
 * f_dtype.  Runs are bin-packed onto thread-block clusters of 8 CTAs; a
 * cluster steps its runs with hardware cluster barriers between the H and E
 * half-steps, and clusters never wait for each other.
 * run descriptors: grid.ndim must be 1; plasma.density may be NULL (vacuum),
 * else nz+1 doubles (host or device); source.kind may be FDTD_SRC_NONE. */
typedef struct fdtd_batch *fdtd_batch_t;

typedef struct {
    fdtd_grid_desc grid;
    fdtd_plasma_desc plasma;
    fdtd_source_desc source;
} fdtd_run_desc;

/* Create a batch (copies every input).  Errors as fdtd_plasma_create / set_plasma. */
int fdtd_batch_create(const fdtd_run_desc *runs, int32_t nruns, const fdtd_runtime_desc *rt, fdtd_batch_t *out);
/* Advance every run by nsteps (asynchronous on the batch's stream). */
int fdtd_batch_step(fdtd_batch_t b, int64_t nsteps);
/* One quantity of one run: FDTD_EX (nz+1), FDTD_HY (nz), FDTD_J (per slot),
 * FDTD_DF (packed rows); sizes as fdtd_batch_quantity_bytes. */
int fdtd_batch_read(fdtd_batch_t b, int32_t run, int which, void *dst, size_t bytes, int dst_is_device);
/* Overwrite a field of one run (FDTD_EX: nz+1 values, FDTD_HY: nz, in the
 * batch precision; host or device source, copied on the batch's stream and
 * synchronised for host sources).  Other quantities: FDTD_ERR_INVAL. */
int fdtd_batch_write(fdtd_batch_t b, int32_t run, int which, const void *src, size_t bytes, int src_is_device);
size_t fdtd_batch_quantity_bytes(fdtd_batch_t b, int32_t run, int which);
/* dt, steps done, total cells, total phase-space nodes, clusters launched and
 * CTAs per cluster (any pointer may be NULL). */
/* Row-shape autotuner of the batched kernel (no counterpart in the paper):
 * times a few steps of every candidate shape for the batch's row length
 * (vectors per lane x lanes per row; FP32 and BF16 rows have two or three,
 * FP64 rows one) on the batch's own buffers, keeps the fastest (a later
 * candidate must be more than 1 % faster than the built-in first one) and
 * restores the state bit for bit (needs one temporary copy of it on the
 * device).  The cluster packing stays as created.  Synchronous; outputs
 * (host, each may be NULL): the shape kept and its time per step in ms. */
int fdtd_batch_autotune(fdtd_batch_t b, int32_t *vpl, int32_t *lanes, double *ms_per_step);
int fdtd_batch_info(fdtd_batch_t b, double *dt, int64_t *steps, int64_t *cells, int64_t *nodes, int32_t *nclusters,
                    int32_t *cluster_ctas);
const char *fdtd_batch_last_error(fdtd_batch_t b);
void fdtd_batch_destroy(fdtd_batch_t b);

/* ---------------------------------------------------------------------
 * Allocation-free diagnostics.  The paper has no counterpart: this is a
 * library service for callers that cannot allocate device memory when they
 * need a diagnostic -- monitoring or watchdog code that must not take the
 * allocator's locks or trigger cudaMalloc's implicit synchronisation,
 * frameworks that route every device allocation through their own pool, and
 * code running close to the device's memory limit.  It computes the same
 * quantities as fdtd_plasma_diagnostics (energy, energy_plain, number,
 * number_max_cell, number_abs, finite -> out[0..5]) from caller-owned device
 * arrays, allocating nothing (no cudaMalloc, no cudaFree, no allocating
 * library call).
 *   in   : the arrays, in the layouts of fdtd_plasma_read_fields (fields by
 *          FDTD_EX..FDTD_HZ, NULL where the dimensionality has none; delta f
 *          as packed [nslots][nnode] rows of f_dtype, dV one double per node;
 *          df and dV may be NULL when nslots == 0).
 *   out  : 6 doubles; device memory (out_is_device = 1, stream-ordered) or
 *          host memory (out_is_device = 0, the stream is synchronised).
 *   stream: cudaStream_t the work is issued on (NULL = legacy default stream).
 * Scratch is a fixed file-scope device array of 8192 tiles (about 459 KB per
 * GPU that loads the library, held until the process exits).  A call needs
 * ceil(field nodes / 65536) + ceil(nslots / 16384) tiles; more returns
 * FDTD_ERR_INVAL with a message (fdtd_plasma_last_error(NULL)).  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so the address stays right
 * after cudaDeviceReset; the first call on a device may also load the
 * library's device code, so make that first call before any stream capture.
 * All calls share the
 * array: calls that overlap on the GPU race (serialise them, e.g. on one
 * stream).  Nothing needs clearing between calls. */
typedef struct {
    int32_t ndim;            /* 1, 2 or 3 */
    int32_t precision;       /* FDTD_F32 or FDTD_F64: element type of the fields */
    int64_t nx, ny, nz;      /* cells, as in fdtd_grid_desc */
    double dx, courant;      /* as in fdtd_grid_desc (fix the vacuum curl of the energy) */
    const void *fields[6];   /* device arrays, index FDTD_EX..FDTD_HZ */
    const void *df;          /* device delta f rows, or NULL */
    int32_t f_dtype;         /* FDTD_DF_F32 / FDTD_DF_BF16 / FDTD_DF_F64 */
    int32_t reserved;
    int64_t nslots, nnode;
    const double *dV;        /* device, nnode volume elements */
} fdtd_diag_arrays;

int fdtd_diagnostics_noalloc(const fdtd_diag_arrays *in, double *out, int out_is_device, void *stream);

/* ---------------------------------------------------------------------
 * Domain decomposition (several GPUs, or several sub-domains on one).  The
 * curl stencils (Sec. 2, Eq. 1-6) couple a cell only to its neighbours, so a
 * grid splits along its slowest axis (y of a 2-D TMz grid, z of a 3-D one)
 * into slabs that exchange one plane of tangential fields per half step: the
 * H update of plane k needs E on plane k + 1 (Eq. 1), the E update of plane k
 * needs H on plane k - 1 (Eq. 2-6).  The delta-f rows, the J moment and the
 * Ampere term are cell-local and never move.
 *
 * fdtd_plasma_create_subdomain: a handle for the owned planes
 *   [offset, offset + extent) of the global grid `global` along `axis`, plus
 *   one ghost plane below (when offset > 0) and one above (when offset +
 *   extent < n_global).  The split axis's CPML profile is the global one at the
 *   planes' global positions, so a sub-domain computes its owned cells bit for
 *   bit as the whole grid does.  set_source takes global coordinates (only the
 *   owner of the source's plane keeps it); set_plasma takes the GLOBAL density
 *   array (pol nodes of the whole grid) and keeps its owned planes, numbering
 *   its plasma slots after the global slots below it (stochastic-rounding
 *   draws equal the whole grid's); read/write_fields and FDTD_J/FDTD_DF cover
 *   the local arrays, ghost planes included (local plane l is global plane
 *   offset - (offset > 0) + l).  Not on sub-domains: the closure, the recorder,
 *   ports, the fused stencil pass.  Errors: FDTD_ERR_INVAL (1-D grids, axis not
 *   the slowest, extent < 2, range outside the axis), as fdtd_plasma_create.
 * fdtd_plasma_step_half: half 0 = H^{n+1/2}; half 1 = delta f, J, E^{n+1}
 *   (and the step counter).  A sub-domain with neighbours steps only this way
 *   (fdtd_plasma_step returns FDTD_ERR_STATE):
 *     unpack E from above; half 0; unpack H from below; half 1
 *   with the neighbours' pack calls before each unpack.  Halves must
 *   alternate, starting with 0 (FDTD_ERR_STATE otherwise).  Stream-ordered.
 * fdtd_plasma_halo_pack / _unpack: copy a halo between the handle's fields and
 *   a caller buffer of fdtd_plasma_halo_bytes(h, which) bytes (device:
 *   stream-ordered on the handle's stream; host: synchronous).
 *   FDTD_HALO_E: pack = the tangential E of the first owned plane (for the
 *     neighbour below), unpack = into the ghost plane above (from the
 *     neighbour above);
 *   FDTD_HALO_H: pack = the tangential H of the last owned plane (for the
 *     neighbour above), unpack = into the ghost plane below.
 *   Layout: the components one after another (3-D: Ex, Ey or Hx, Hy planes of
 *   nx * ny values; 2-D: the Ez or Hx row of nx values), field precision.
 *   FDTD_ERR_STATE when the handle has no neighbour on that side or is not a
 *   sub-domain. */
typedef struct {
    int32_t axis;          /* 1 (2-D grids, y) or 2 (3-D grids, z): the slowest axis */
    int32_t reserved;
    int64_t n_global;      /* cells of the global grid along the axis (= nz or ny of `global`) */
    int64_t offset;        /* first owned cell along the axis */
    int64_t extent;        /* owned cells along the axis (>= 2) */
} fdtd_subdomain_desc;
enum { FDTD_HALO_E = 0, FDTD_HALO_H = 1 };
int fdtd_plasma_create_subdomain(const fdtd_grid_desc *global, const fdtd_subdomain_desc *sd,
                                 const fdtd_runtime_desc *rt, fdtd_plasma_t *out);
int fdtd_plasma_step_half(fdtd_plasma_t h, int half);
size_t fdtd_plasma_halo_bytes(fdtd_plasma_t h, int which);
int fdtd_plasma_halo_pack(fdtd_plasma_t h, int which, void *dst, int dst_is_device);
int fdtd_plasma_halo_unpack(fdtd_plasma_t h, int which, const void *src, int src_is_device);

/* Last error message of the handle (or of the last failed create when h is
 * NULL).  Valid until the next call on the same handle. */
const char *fdtd_plasma_last_error(fdtd_plasma_t h);

/* Release everything the handle owns.  NULL-safe.  Synchronises the stream. */
void fdtd_plasma_destroy(fdtd_plasma_t h);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_PLASMA_H */

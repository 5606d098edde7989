// capi.cu -- the C ABI of include/fdtd_plasma.h: handle lifetime, parameter
// derivation (time step, CPML profiles of Eq. 9-12, velocity tables of the
// Sec. 5.2 update), plasma-cell compaction, CUDA-graph capture of the step
// sequence, stream-ordered I/O, FP64 diagnostics and checkpoints.
//
// Every coefficient is derived here from the paper's formulas, in FP64 on the
// host, then rounded once to the field precision.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <vector>

#include <sys/stat.h>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

using namespace fp;

namespace {

constexpr int kChunk = 32;            // steps per replay of the chunk graph
constexpr int kFuseRowsDefault = 8;   // rows per block segment of the 2-D fused column march
constexpr uint64_t kStateMagic = 0x4644544450534d31ull;

thread_local std::string g_create_error;

int fail(fdtd_plasma *h, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(fdtd_plasma *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

int cuda_fail(fdtd_plasma *h, cudaError_t e, const char *what)
{
    return fail(h, FDTD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);      \
    } while (0)

// Canary pads: with h->canary every allocation gets kCanaryPad guard bytes of
// kCanaryByte before and after the user range (alignment is kept: the pad is
// 256 bytes); fdtd_plasma_check_canaries compares them with the pattern.
// NVTX range around a public entry point (visible in Nsight Systems / Compute timelines)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr size_t kCanaryPad = 256;
constexpr unsigned char kCanaryByte = 0xA5;

void *dalloc_raw(fdtd_plasma *h, size_t bytes);

void *dalloc(fdtd_plasma *h, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (!h->canary) return dalloc_raw(h, bytes);
    char *raw = static_cast<char *>(dalloc_raw(h, bytes + 2 * kCanaryPad));
    if (!raw) return nullptr;
    if (cudaMemset(raw, kCanaryByte, kCanaryPad) != cudaSuccess ||
        cudaMemset(raw + kCanaryPad + bytes, kCanaryByte, kCanaryPad) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {   // done before any work on the handle's stream
        cudaGetLastError();
        if (h->rt.free) h->rt.free(raw, h->rt.alloc_ctx);
        else cudaFree(raw);
        return nullptr;
    }
    h->canary_allocs.push_back({raw + kCanaryPad, bytes});
    return raw + kCanaryPad;
}

void *dalloc_raw(fdtd_plasma *h, size_t bytes)
{
    void *p = nullptr;
    if (h->rt.alloc) {
        p = h->rt.alloc(bytes, h->rt.alloc_ctx);
        if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {   // the 16-byte vector stencils rely on it
            h->err = "the allocator callback returned memory that is not 256-byte aligned";
            if (h->rt.free) h->rt.free(p, h->rt.alloc_ctx);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dfree(fdtd_plasma *h, void *p)
{
    if (!p) return;
    if (h->canary) {
        auto &v = h->canary_allocs;
        for (size_t q = 0; q < v.size(); ++q)
            if (v[q].first == p) {
                v.erase(v.begin() + (std::ptrdiff_t)q);
                p = static_cast<char *>(p) - kCanaryPad;
                break;
            }
    }
    if (h->rt.free) h->rt.free(p, h->rt.alloc_ctx);
    else cudaFree(p);
}

// ------------------------------------------------------------- CPML tables

// One axis of n cells, L-cell layers at both ends, at E (x = i dx) or H
// (x = (i+1/2) dx) positions: sigma = smax (rho/delta)^m, kappa = 1 +
// (kmax-1)(rho/delta)^m, alpha = amin + (amax-amin)(1-rho/delta) (Eq. 12),
// smax = factor (m+1)/(150 pi dx) (Eq. 11), b = exp(-(sigma/kappa+alpha)dt/eps0)
// (Eq. 9), a = sigma (b-1)/(dx (sigma kappa + alpha kappa^2)) (Eq. 10).
void cpml_axis(const fdtd_grid_desc &g, double dt, int64_t n, bool at_h, std::vector<double> &b,
               std::vector<double> &a, std::vector<double> &ik)
{
    const int64_t L = g.cpml_cells;
    const double delta = (double)L * g.dx;
    const double smax = g.cpml_sigma_factor * (g.cpml_order + 1.0) / (150.0 * kPi * g.dx);
    b.assign(n, 0.0);
    a.assign(n, 0.0);
    ik.assign(n, 1.0);
    for (int64_t i = 0; i < n; ++i) {
        const double x = ((double)i + (at_h ? 0.5 : 0.0)) * g.dx;
        double rho;
        if (x < delta) rho = delta - x;
        else if (x > (double)(n - L) * g.dx) rho = x - (double)(n - L) * g.dx;
        else continue;
        const double r = rho / delta;
        const double rm = std::pow(r, g.cpml_order);
        const double sig = smax * rm;
        const double kap = 1.0 + (g.cpml_kappa_max - 1.0) * rm;
        const double alp = g.cpml_alpha_min + (g.cpml_alpha_max - g.cpml_alpha_min) * (1.0 - r);
        const double bb = std::exp(-(sig / kap + alp) * dt / kEps0);
        const double den = g.dx * (sig * kap + alp * kap * kap);
        b[i] = bb;
        a[i] = (sig > 0.0 && den > 0.0) ? sig * (bb - 1.0) / den : 0.0;
        ik[i] = 1.0 / kap;
    }
}

// ------------------------------------------------------------------ misc

int64_t pol_len(const fdtd_plasma *h) { return h->g.ndim == 1 ? h->nz + 1 : h->nx * h->ny * h->nz; }
int pol_comp(const fdtd_plasma *h) { return h->g.ndim == 2 ? FDTD_EZ : FDTD_EX; }

bool pol_updated(const fdtd_plasma *h, int64_t c)
{
    if (h->g.ndim == 1) return c >= 1 && c <= h->nz - 1;
    const int64_t i = c % h->nx, j = (c / h->nx) % h->ny, k = c / (h->nx * h->ny);
    if (h->g.ndim == 2) return i >= 1 && j >= 1;
    (void)i;
    return j >= 1 && k >= 1;
}

void free_closure(fdtd_plasma *h)
{
    dfree(h, h->hist); dfree(h, h->jprev); dfree(h, h->params);
    h->hist = h->jprev = h->params = nullptr;
    h->has_closure = 0;
    h->has_recording = 0;
    h->ncl = 0;
    h->nkin = h->nslots;
}

void free_plasma(fdtd_plasma *h)
{
    free_closure(h);
    dfree(h, h->slot_cell); dfree(h, h->dens); dfree(h, h->df); dfree(h, h->jslot); dfree(h, h->tab);
    dfree(h, h->dV); dfree(h, h->g0); dfree(h, h->tab_f0);
    h->slot_cell = nullptr; h->dens = h->df = h->jslot = h->tab = nullptr; h->dV = nullptr;
    h->g0 = h->tab_f0 = nullptr;
    h->has_plasma = 0;
    h->nslots = 0;
    h->nkin = 0;
    h->nnode = 0;
    h->h_cells.clear();
    h->h_dens.clear();
}

// The plasma slots of a whole grid's density array (host or device, pol_len values), compacted on the
// GPU: cells in increasing index with their densities (FP64) and the largest density; FDTD_ERR_NONFINITE
// for a value that is not finite or is negative.
// The device copy of the result (densities FP64 [ns], then cells int32 [ns]) is handed to the caller in
// *dev_slots (to be freed with dfree) when ns > 0, so the slot arrays are filled device to device.
int compact_on_gpu(fdtd_plasma *h, const fdtd_plasma_desc *p, int64_t np, std::vector<int32_t> &cells,
                   std::vector<double> &dslot, double &nmax, void **dev_slots)
{
    *dev_slots = nullptr;
    const int64_t nb = (np + kCompactChunk - 1) / kCompactChunk;
    const CompactGeom g{h->g.ndim, h->nx, h->ny, h->nz, np};
    void *dtmp = nullptr, *scr = nullptr, *out = nullptr;
    auto release = [&]() { dfree(h, dtmp); dfree(h, scr); dfree(h, out); };
    const double *d = static_cast<const double *>(p->density);
    if (!p->density_on_device) {
        dtmp = dalloc(h, (size_t)np * 8);
        if (!dtmp) return fail(h, FDTD_ERR_NOMEM, "density upload buffer (%lld values)", (long long)np);
        cudaError_t e = cudaMemcpyAsync(dtmp, p->density, (size_t)np * 8, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) { release(); return cuda_fail(h, e, "density upload"); }
        d = static_cast<const double *>(dtmp);
    }
    // scratch: offsets (int64) | maxes (double) | counts (int) | bad (int)
    scr = dalloc(h, (size_t)nb * 20 + 256);
    if (!scr) { release(); return fail(h, FDTD_ERR_NOMEM, "compaction scratch"); }
    int64_t *d_off = static_cast<int64_t *>(scr);
    double *d_max = reinterpret_cast<double *>(d_off + nb);
    int *d_cnt = reinterpret_cast<int *>(d_max + nb), *d_bad = d_cnt + nb;
    std::vector<int> cnt((size_t)nb);
    std::vector<double> mx((size_t)nb);
    std::vector<int64_t> off((size_t)nb);
    int bad = 0;
    cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = launch_compact_count(h->stream, d, g, d_cnt, d_max, d_bad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, (size_t)nb * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx.data(), d_max, (size_t)nb * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { release(); return cuda_fail(h, e, "plasma compaction (count)"); }
    if (bad) { release(); return fail(h, FDTD_ERR_NONFINITE, "density must be finite and >= 0"); }
    int64_t ns = 0;
    nmax = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        off[(size_t)b] = ns;
        ns += cnt[(size_t)b];
        nmax = std::max(nmax, mx[(size_t)b]);
    }
    cells.resize((size_t)ns);
    dslot.resize((size_t)ns);
    if (ns) {
        out = dalloc(h, (size_t)ns * 12 + 256);
        if (!out) { release(); return fail(h, FDTD_ERR_NOMEM, "compaction output (%lld cells)", (long long)ns); }
        double *d_dens = static_cast<double *>(out);
        int32_t *d_cells = reinterpret_cast<int32_t *>(d_dens + ns);
        e = cudaMemcpyAsync(d_off, off.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_compact_scatter(h->stream, d, g, d_off, d_cells, d_dens);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cells.data(), d_cells, (size_t)ns * 4, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dslot.data(), d_dens, (size_t)ns * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { release(); return cuda_fail(h, e, "plasma compaction (scatter)"); }
        *dev_slots = out;
        out = nullptr;
    } else {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { release(); return cuda_fail(h, e, "plasma compaction"); }
    }
    release();
    return FDTD_OK;
}

void drop_graphs(fdtd_plasma *h)
{
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->gk) cudaGraphExecDestroy(h->gk);
    h->g1 = h->gk = nullptr;
    for (auto &g : h->gpow) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    h->graphs_valid = 0;
}

template <typename T>
Cpml<T> cpml_view(fdtd_plasma *h)
{
    Cpml<T> c{};
    c.L = h->g.ndim >= 2 ? h->g.cpml_cells : 0;
    if (!c.L) return c;
    const T *base = reinterpret_cast<const T *>(h->prof);
    int64_t n[3] = {h->nx, h->ny, h->nz};
    int64_t off = 0;
    for (int ax = 0; ax < h->g.ndim; ++ax) {
        c.be[ax] = base + off; off += n[ax];
        c.ae[ax] = base + off; off += n[ax];
        c.ike[ax] = base + off; off += n[ax];
        c.bh[ax] = base + off; off += n[ax];
        c.ah[ax] = base + off; off += n[ax];
        c.ikh[ax] = base + off; off += n[ax];
    }
    for (int q = 0; q < 12; ++q) c.psi[q] = reinterpret_cast<T *>(h->psi[q]);
    return c;
}

Source source_view(fdtd_plasma *h)
{
    Source s{};
    if (!h->has_source) return s;
    s.kind = h->src.kind; s.loc = h->src.location;
    s.amp = h->src.amp; s.fc = h->src.fc; s.tau = h->src.tau; s.t0 = h->src.t0; s.dt = h->dt;
    s.i = h->src.i; s.j = h->src.j; s.k = h->src.k;
    s.i0 = h->src.i0; s.i1 = h->src.i1; s.j0 = h->src.j0; s.j1 = h->src.j1;
    s.val = h->d_src;
    return s;
}

dim3 stencil_block(const fdtd_plasma *h)
{
    if (h->st_bx > 0) return dim3(h->st_bx, h->st_by, h->g.ndim == 3 ? h->st_bz : 1);
    return h->g.ndim == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1);
}

// cells per thread of the curl stencils: tuned, else 4 in 2-D (measured
// faster on GB300) and 1 in 3-D (the four-cell 3-D kernels need 80 registers
// and lose more to the lower occupancy than they save in instructions)
int stencil_cpt(const fdtd_plasma *h)
{
    if (h->st_cpt > 0) return h->st_cpt;
    return h->g.ndim == 2 ? 4 : 1;
}

template <typename T>
KinArgs<T> kin_args(fdtd_plasma *h, int kstep)
{
    KinArgs<T> a{};
    a.slot_cell = h->slot_cell;
    a.dens = reinterpret_cast<const T *>(h->dens);
    a.df = h->df;
    a.E = reinterpret_cast<T *>(h->f[pol_comp(h)]);
    a.jslot = reinterpret_cast<T *>(h->jslot);
    a.tab = reinterpret_cast<const T *>(h->tab);
    a.nslots = h->nkin;
    a.pitch = h->pitch;
    a.cj = (T)(h->dt / kEps0);
    a.seed = h->pl.seed;
    a.d_step = h->d_step;
    a.kstep = kstep;
    a.slot_base = h->slot_base;
    a.store_j = 1;
    a.err = h->d_err;
    return a;
}

// ---------------------------------------------------------------- tune cache
// Text file, one entry per line: "<key> <v0> <v1> <v2>", keyed by GPU name,
// kernel, precision and shape class.  Path: $FDTD_PLASMA_TUNE_CACHE, else
// $HOME/.cache/fdtd_plasma/autotune.txt.

std::string tune_cache_path()
{
    const char *p = std::getenv("FDTD_PLASMA_TUNE_CACHE");
    if (p && *p) return p;
    const char *home = std::getenv("HOME");
    return std::string(home ? home : ".") + "/.cache/fdtd_plasma/autotune.txt";
}

std::string gpu_key()
{
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "gpu";
    std::string n = prop.name;
    for (char &c : n)
        if (c == ' ') c = '_';
    return n;
}

int log2_bucket(int64_t n)
{
    int b = 0;
    while (n > 1) { n >>= 1; ++b; }
    return b;
}

std::string kin_key(const fdtd_plasma *h)
{
    std::ostringstream o;
    o << gpu_key() << "|kinetic|dtype" << h->pl.f_dtype << "|pitch" << h->pitch << "|rows2^" << log2_bucket(h->nkin);
    return o.str();
}

std::string stencil_key(const fdtd_plasma *h)
{
    std::ostringstream o;
    o << gpu_key() << "|stencil" << h->g.ndim << "d|prec" << h->g.precision << "|cells2^"
      << log2_bucket(h->nx * h->ny * h->nz) << "|cpml" << (h->g.cpml_cells > 0) << "|rows4="
      << (h->g.precision == FDTD_F32 && h->nx % 4 == 0);
    return o.str();
}

std::map<std::string, std::vector<int>> read_cache()
{
    std::map<std::string, std::vector<int>> m;
    std::ifstream f(tune_cache_path());
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string k;
        std::vector<int> v;
        int x;
        if (!(in >> k)) continue;
        while (in >> x) v.push_back(x);
        if (v.size() >= 3 && v.size() <= 6) m[k] = v;
    }
    return m;
}

void write_cache(const std::map<std::string, std::vector<int>> &m)
{
    const std::string path = tune_cache_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    std::ofstream f(path, std::ios::trunc);
    for (const auto &kv : m) {
        f << kv.first;
        for (int x : kv.second) f << " " << x;
        f << "\n";
    }
}

void apply_cached_kinetic(fdtd_plasma *h)
{
    auto m = read_cache();
    auto it = m.find(kin_key(h));
    if (it != m.end()) {
        h->kin_vpl = it->second[0]; h->kin_l = it->second[1]; h->kin_bps = it->second[2];
        h->kin_stages = it->second.size() >= 4 ? it->second[3] : 0;
    }
}

void apply_cached_stencil(fdtd_plasma *h)
{
    auto m = read_cache();
    auto it = m.find(stencil_key(h));
    if (it != m.end() && it->second.size() >= 4) {
        h->st_bx = it->second[0]; h->st_by = it->second[1]; h->st_bz = it->second[2]; h->st_cpt = it->second[3];
        h->st_tz = it->second.size() >= 5 ? it->second[4] : 0;
        h->auto_fuse_rows = it->second.size() >= 6 && !h->sd_on ? it->second[5] : 0;
    }
}

// Field / psi sets: set 0 is h->f / h->psi (where the state lives between
// calls), set 1 the second copy used by the fused 3-D E+H kernel.
template <typename T>
struct FieldSet {
    T *f[6];
    Cpml<T> cp;
};

template <typename T>
FieldSet<T> field_set(fdtd_plasma *h, int set)
{
    FieldSet<T> fs{};
    for (int q = 0; q < 6; ++q) fs.f[q] = reinterpret_cast<T *>(set ? h->f2[q] : h->f[q]);
    fs.cp = cpml_view<T>(h);
    if (set)
        for (int q = 0; q < 12; ++q) fs.cp.psi[q] = reinterpret_cast<T *>(h->psi2[q]);
    return fs;
}

// the TMA column kernels' tensor maps when they are the selected 3-D stencils for this field set
// (FP32, set 0); nullptr = run the grid-of-cells kernels
template <typename T>
const TmaMaps *tma_for(fdtd_plasma *h, const FieldSet<T> &fs)
{
    if (sizeof(T) != 4 || h->g.ndim < 2 || h->st_tz <= 0) return nullptr;
    if (!h->tma) h->tma = tma_maps_create(reinterpret_cast<float *const *>(h->f), h->nx, h->ny, h->nz);
    return tma_maps_match(h->tma, reinterpret_cast<float *const *>(fs.f)) ? h->tma : nullptr;
}

template <typename T>
cudaError_t part_h(fdtd_plasma *h, cudaStream_t st, int kstep, const FieldSet<T> &fs)
{
    const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
    const T ch = (T)(h->dt / (mu0 * h->g.dx)), cph = (T)(h->dt / mu0);
    T *const *f = fs.f;
    const Source src = source_view(h);
    if (h->g.ndim == 1)
        launch_h1d<T>(st, f[FDTD_EX], f[FDTD_HY], h->g.mur ? (T *)h->mur_state : nullptr, h->nz, ch, src, h->d_step,
                      kstep);
    else if (h->g.ndim == 2) {
        if constexpr (sizeof(T) == 4) {
            if (const TmaMaps *t = tma_for(h, fs)) {
                launch_h2d_tma(st, t, f, h->nx, h->ny, ch, cph, fs.cp, src, h->d_step, kstep, h->st_tz, h->d_err);
                return cudaGetLastError();
            }
        }
        launch_h2d<T>(st, f[FDTD_EZ], f[FDTD_HX], f[FDTD_HY], h->nx, h->ny, ch, cph, fs.cp, src, h->d_step, kstep,
                      stencil_block(h), stencil_cpt(h));
    }
    else {
        if constexpr (sizeof(T) == 4) {
            if (const TmaMaps *t = tma_for(h, fs)) {
                launch_h3d_tma(st, t, f, h->nx, h->ny, h->nz, ch, cph, fs.cp, src, h->d_step, kstep, h->st_tz,
                               h->d_err);
                return cudaGetLastError();
            }
        }
        launch_h3d<T>(st, const_cast<T *const *>(f), h->nx, h->ny, h->nz, ch, cph, fs.cp, src, h->d_step, kstep,
                      stencil_block(h), stencil_cpt(h));
    }
    return cudaGetLastError();
}

// the work between the H and E updates: E-history push, kinetic update (E -= dt/eps0 J), closure, recorder.
// J^{n+1/2} per slot is stored on the last step of a sequence (what read_fields and checkpoints see between
// step calls) and on every step while the recorder, which reads it, is on.
template <typename T>
cudaError_t part_mid(fdtd_plasma *h, cudaStream_t st, int kstep, const FieldSet<T> &fs, cudaEvent_t *ev,
                     bool last = true)
{
    T *E = fs.f[pol_comp(h)];
    const bool rec = h->has_recording && sizeof(T) == 4;
    if (rec)
        launch_hist_push(st, h->slot_cell, h->nslots, reinterpret_cast<const float *>(E), h->hist, h->d_step, kstep);
    if (h->has_plasma && h->nkin > 0) {
        KinArgs<T> a = kin_args<T>(h, kstep);
        a.E = E;
        a.store_j = last || rec;
        cudaError_t e;
        if (h->pl.evolve_f0) {
            const double vth = std::sqrt(kQe * h->pl.te_ev / kMe);
            const double gam = h->pl.vmax_vth * vth / h->pl.nv;
            F0Args<T> f{};
            f.tab = reinterpret_cast<const T *>(h->tab_f0);
            f.g = reinterpret_cast<T *>(h->g0);
            f.nv = h->pl.nv;
            f.gam = (T)gam;
            f.inv2gam = (T)(1.0 / (2.0 * gam));
            f.qm3 = (T)(kQe / kMe / 3.0);
            f.mr = (T)h->pl.mass_ratio;
            f.kTg_m = (T)(kQe * h->pl.tg_ev / kMe);
            f.dt = (T)h->dt;
            e = launch_kinetic_f0<T>(st, a, f, h->num_sms);
        } else if (h->pl.nonlinear) {
            const double vth = std::sqrt(kQe * h->pl.te_ev / kMe);
            const double dvpar = 2.0 * h->pl.vmax_vth * vth / h->pl.nv;
            const int nperp = h->pl.vgrid == FDTD_VGRID_CART2D ? h->pl.nv_perp : 1;
            e = launch_kinetic_nl<T>(st, a, h->pl.nv, nperp, dvpar, kQe / kMe, h->dt, h->num_sms);
        } else {
            e = launch_kinetic<T>(st, a, h->pl.f_dtype, h->num_sms, h->kin_vpl, h->kin_l, h->kin_bps, h->kin_stages);
        }
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[2], st);
    if (h->has_closure && h->ncl > 0 && sizeof(T) == 4) {
        ClosureArgs c{};
        c.cell = h->slot_cell + h->nkin;
        c.dens = reinterpret_cast<const float *>(h->dens) + h->nkin;
        c.hist = h->hist;
        c.jprev = h->jprev;
        c.jslot = reinterpret_cast<float *>(h->jslot) + h->nkin;
        c.E = reinterpret_cast<float *>(E);
        c.P = h->params;
        c.n = h->ncl;
        c.inv_es = (float)(1.0 / h->cl.e_scale);
        c.inv_ns = (float)(1.0 / h->cl.n_scale);
        c.js = (float)h->cl.j_scale;
        c.rho = (float)h->cl.rho;
        c.beta = (float)h->cl.beta;
        c.cj = (float)(h->dt / kEps0);
        c.d_step = h->d_step;
        c.kstep = kstep;
        c.engine = h->cl.engine;
        c.store_j = last;
        c.err = h->d_err;
        cudaError_t e = launch_closure(st, c, h->num_sms);
        if (e != cudaSuccess) return e;
    }
    if (rec)
        launch_record(st, h->nslots, h->hist, reinterpret_cast<const float *>(h->dens),
                      reinterpret_cast<const float *>(h->jslot), h->jprev, h->rec_out, h->rec_cap, h->rec_count,
                      h->rec_threshold, h->rec_seed, h->d_step, kstep);
    return cudaGetLastError();
}

template <typename T>
cudaError_t part_e(fdtd_plasma *h, cudaStream_t st, int kstep, const FieldSet<T> &fs)
{
    const T ce = (T)(h->dt / (kEps0 * h->g.dx)), cpe = (T)(h->dt / kEps0);
    T *const *f = fs.f;
    const Source src = source_view(h);
    if (h->g.ndim == 1) {
        const T m = (T)((kC0 * h->dt - h->g.dx) / (kC0 * h->dt + h->g.dx));
        launch_e1d<T>(st, f[FDTD_EX], f[FDTD_HY], h->nz, ce, src, h->d_step, kstep,
                      h->g.mur ? (const T *)h->mur_state : nullptr, m);
    } else if (h->g.ndim == 2) {
        if constexpr (sizeof(T) == 4) {
            if (const TmaMaps *t = tma_for(h, fs)) {
                launch_e2d_tma(st, t, f, h->nx, h->ny, ce, cpe, fs.cp, src, h->st_tz, h->d_err);
                return cudaGetLastError();
            }
        }
        launch_e2d<T>(st, f[FDTD_EZ], f[FDTD_HX], f[FDTD_HY], h->nx, h->ny, ce, cpe, fs.cp, src, h->d_step, kstep,
                      stencil_block(h), stencil_cpt(h));
    } else {
        if constexpr (sizeof(T) == 4) {
            if (const TmaMaps *t = tma_for(h, fs)) {
                launch_e3d_tma(st, t, f, h->nx, h->ny, h->nz, ce, cpe, fs.cp, src, h->st_tz, h->d_err);
                return cudaGetLastError();
            }
        }
        launch_e3d<T>(st, const_cast<T *const *>(f), h->nx, h->ny, h->nz, ce, cpe, fs.cp, src, h->d_step, kstep,
                      stencil_block(h), stencil_cpt(h));
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t part_ports(fdtd_plasma *h, cudaStream_t st, int kstep, const FieldSet<T> &fs)
{
    if (h->nports <= 0) return cudaSuccess;
    return launch_ports<T>(st, fs.f[pol_comp(h)], h->nports, h->port_off, h->port_cells, h->port_freq, h->port_acc,
                           h->nfreq, h->dt, h->d_step, kstep);
}

// enqueue one step n -> n+1 on field set 0 (kstep = offset of this step inside
// the chunk); ev (optional) receives records before H, before the kinetic
// kernel, before the closure kernel, before E and after E.
template <typename T>
cudaError_t enqueue_step(fdtd_plasma *h, cudaStream_t st, int kstep, cudaEvent_t *ev = nullptr, bool last = true)
{
    const FieldSet<T> fs = field_set<T>(h, 0);
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = part_h<T>(h, st, kstep, fs);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    e = part_mid<T>(h, st, kstep, fs, ev, last);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], st);
    e = part_e<T>(h, st, kstep, fs);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], st);
    return part_ports<T>(h, st, kstep, fs);
}

void free_second_set(fdtd_plasma *h)
{
    tma_fused_forget(h->tma);
    for (int q = 0; q < 6; ++q) { dfree(h, h->f2[q]); h->f2[q] = nullptr; }
    for (int q = 0; q < 12; ++q) { dfree(h, h->psi2[q]); h->psi2[q] = nullptr; }
}

// allocate the second field / psi set when the fused sequence applies; on failure the steps run unfused
void ensure_second_set(fdtd_plasma *h)
{
    if ((!h->fuse && h->auto_fuse_rows <= 0) || h->g.ndim < 2 || h->g.precision != FDTD_F32 || h->f2[FDTD_EZ]) return;
    bool ok = true;
    for (int q = 0; q < 6 && ok; ++q)
        if (h->flen[q]) ok = (h->f2[q] = dalloc(h, h->flen[q] * h->esz)) != nullptr;
    for (int q = 0; q < 12 && ok; ++q)
        if (h->psi[q]) ok = (h->psi2[q] = dalloc(h, h->psilen[q] * h->esz)) != nullptr;
    if (!ok) {
        free_second_set(h);
        h->err.clear();
    }
}

// whether the step sequence fuses E^{n+1} with H^{n+3/2} (2-D / 3-D FP32 by option, 2-D FP32 by the
// autotuner's choice; second field set allocated)
bool fused_stencils(const fdtd_plasma *h)
{
    const bool on = h->fuse || (h->auto_fuse_rows > 0 && h->g.ndim == 2);
    return on && h->g.ndim >= 2 && h->g.precision == FDTD_F32 && h->f2[FDTD_EZ] != nullptr;
}

// rows per segment of the 2-D column march: the option's when fusion was asked for, else the autotuner's
int fuse_rows_of(const fdtd_plasma *h) { return h->fuse ? h->fuse_rows : h->auto_fuse_rows; }

// nsteps steps: H_0, then per step the middle part and either E_k alone (then
// H_{k+1} on the same set) or the fused E_k + H_{k+1} from one set into the
// other.  The number of fused transitions is kept even so the sequence ends on
// set 0; with an odd count the first transition runs unfused.
template <typename T>
cudaError_t enqueue_seq(fdtd_plasma *h, cudaStream_t st, int nsteps)
{
    const bool fuse = sizeof(T) == 4 && fused_stencils(h);
    // the fused pass on TMA-staged planes when the TMA column stencils are selected (3-D FP32)
    bool tma_fused = false;
    if (fuse && h->g.ndim == 3 && h->st_tz > 0) {
        if (!h->tma) h->tma = tma_maps_create(reinterpret_cast<float *const *>(h->f), h->nx, h->ny, h->nz);
        tma_fused = h->tma && tma_fused_prepare(h->tma, reinterpret_cast<float *const *>(h->f),
                                                reinterpret_cast<float *const *>(h->f2));
    }
    const int trans = nsteps - 1;
    const int unfused_first = fuse && (trans % 2) ? 1 : 0;
    int set = 0;
    cudaError_t e = part_h<T>(h, st, 0, field_set<T>(h, set));
    if (e != cudaSuccess) return e;
    for (int k = 0; k < nsteps; ++k) {
        const FieldSet<T> fs = field_set<T>(h, set);
        const bool last = k == nsteps - 1;
        e = part_mid<T>(h, st, k, fs, nullptr, last);
        if (e != cudaSuccess) return e;
        if (!last && fuse && k >= unfused_first) {
            const FieldSet<T> to = field_set<T>(h, set ^ 1);
            const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
            if constexpr (sizeof(T) == 4) {
                const float ce = (float)(h->dt / (kEps0 * h->g.dx)), cpe = (float)(h->dt / kEps0);
                const float ch = (float)(h->dt / (mu0 * h->g.dx)), cph = (float)(h->dt / mu0);
                if (h->g.ndim == 3) {
                    if (!(tma_fused && launch_eh3d_tma(st, h->tma, fs.f, to.f, to.cp.psi, ce, cpe, ch, cph, fs.cp,
                                                       source_view(h), h->d_step, k, h->st_tz, h->d_err)))
                        launch_eh3d(st, fs.f, to.f, to.cp.psi, h->nx, h->ny, h->nz, ce, cpe, ch, cph, fs.cp,
                                    source_view(h), h->d_step, k);
                }
                else
                    launch_eh2d(st, fs.f, to.f, to.cp.psi, h->nx, h->ny, ce, cpe, ch, cph, fs.cp, source_view(h),
                                h->d_step, k, fuse_rows_of(h));
            }
            set ^= 1;
            e = part_ports<T>(h, st, k, to);
            if (e != cudaSuccess) return e;
            continue;
        }
        e = part_e<T>(h, st, k, fs);
        if (e == cudaSuccess) e = part_ports<T>(h, st, k, fs);
        if (e == cudaSuccess && !last) e = part_h<T>(h, st, k + 1, fs);
        if (e != cudaSuccess) return e;
    }
    return set == 0 ? cudaGetLastError() : cudaErrorInvalidValue;   // the state must end on set 0
}

cudaError_t enqueue(fdtd_plasma *h, cudaStream_t st, int nsteps)
{
    cudaError_t e = h->g.precision == FDTD_F64 ? enqueue_seq<double>(h, st, nsteps) : enqueue_seq<float>(h, st, nsteps);
    if (e != cudaSuccess) return e;
    launch_advance(st, h->d_step, nsteps);
    return cudaGetLastError();
}

int capture(fdtd_plasma *h, int nsteps, cudaGraphExec_t *out)
{
    cudaGraph_t graph = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = enqueue(h, h->cap, nsteps);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h, e, "capturing the step sequence");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return FDTD_OK;
}

size_t field_bytes(const fdtd_plasma *h, int q) { return h->f[q] ? (size_t)h->flen[q] * h->esz : 0; }

}  // namespace

int fp_set_global_error(int code, const char *msg)
{
    g_create_error = msg;
    return code;
}

// =================================================================== ABI

extern "C" {

}  // extern "C"

namespace {

// Sub-domain of a grid decomposed along its slowest axis: the grid desc given
// to create_impl is then the GLOBAL grid; the handle holds the owned planes
// [offset, offset + extent) plus one ghost plane on each side that has a
// neighbour.
struct SubInfo {
    int axis;
    int64_t n_global, offset, extent;
};

int create_impl(const fdtd_grid_desc *g, const fdtd_runtime_desc *rt, fdtd_plasma_t *out, const SubInfo *sd)
{
    if (!out) return fail(nullptr, FDTD_ERR_INVAL, "out is NULL");
    *out = nullptr;
    if (!g) return fail(nullptr, FDTD_ERR_INVAL, "grid is NULL");
    if (g->ndim < 1 || g->ndim > 3) return fail(nullptr, FDTD_ERR_INVAL, "ndim must be 1, 2 or 3");
    if (g->precision != FDTD_F32 && g->precision != FDTD_F64) return fail(nullptr, FDTD_ERR_INVAL, "bad precision");
    if (!(g->dx > 0.0) || !std::isfinite(g->dx)) return fail(nullptr, FDTD_ERR_INVAL, "dx must be > 0");
    if (!(g->courant > 0.0) || !std::isfinite(g->courant)) return fail(nullptr, FDTD_ERR_INVAL, "courant must be > 0");
    if (g->courant * g->courant * g->ndim >= 1.0)
        return fail(nullptr, FDTD_ERR_UNSTABLE, "Courant number %g violates S^2 ndim < 1", g->courant);
    int64_t n[3] = {g->ndim >= 2 ? g->nx : 1, g->ndim >= 2 ? g->ny : 1, g->ndim == 2 ? 1 : g->nz};
    const int64_t n_full[3] = {n[0], n[1], n[2]};   // the global grid (= n unless a sub-domain)
    int64_t sd_lo = 0, sd_hi = 0;
    if (sd) {
        // the slowest axis of the grid is split: y in 2-D (TMz), z in 3-D
        if (g->ndim < 2 || sd->axis != g->ndim - 1)
            return fail(nullptr, FDTD_ERR_INVAL, "sub-domains split 2-D grids along y (axis 1), 3-D grids along z (axis 2)");
        if (sd->n_global != n[sd->axis] || sd->offset < 0 || sd->extent < 2 || sd->offset + sd->extent > sd->n_global)
            return fail(nullptr, FDTD_ERR_INVAL, "sub-domain [offset, offset + extent) must lie in the global axis, extent >= 2");
        sd_lo = sd->offset > 0 ? 1 : 0;
        sd_hi = sd->offset + sd->extent < sd->n_global ? 1 : 0;
        n[sd->axis] = sd->extent + sd_lo + sd_hi;
    }
    for (int ax = 0; ax < 3; ++ax) {
        const bool used = (g->ndim == 1) ? ax == 2 : (g->ndim == 2 ? ax < 2 : true);
        if (used && (n[ax] < 3 || n[ax] > (int64_t)1 << 30))
            return fail(nullptr, FDTD_ERR_INVAL, "axis %d size %lld out of range [3, 2^30]", ax, (long long)n[ax]);
    }
    const int64_t ncell = n[0] * n[1] * n[2];
    if (ncell > ((int64_t)1 << 31) - 1) return fail(nullptr, FDTD_ERR_INVAL, "grid has more than 2^31-1 nodes");
    if (g->cpml_cells < 0) return fail(nullptr, FDTD_ERR_INVAL, "cpml_cells < 0");
    if (g->ndim == 1 && g->cpml_cells) return fail(nullptr, FDTD_ERR_INVAL, "1-D uses Mur or PEC ends, not CPML");
    if (g->ndim >= 2 && g->mur) return fail(nullptr, FDTD_ERR_INVAL, "Mur ends are 1-D only");
    if (g->cpml_cells) {
        for (int ax = 0; ax < g->ndim; ++ax)
            if (3 * (int64_t)g->cpml_cells >= n_full[ax])
                return fail(nullptr, FDTD_ERR_INVAL, "CPML thicker than a third of axis %d", ax);
        if (!(g->cpml_order > 0) || !(g->cpml_kappa_max >= 1.0) || !(g->cpml_sigma_factor >= 0) ||
            g->cpml_alpha_min < 0 || g->cpml_alpha_max < g->cpml_alpha_min)
            return fail(nullptr, FDTD_ERR_INVAL, "bad CPML parameters");
    }

    fdtd_plasma *h = new (std::nothrow) fdtd_plasma();
    if (h) {
        h->fuse = 0;
        h->fuse_rows = kFuseRowsDefault;
        const char *cv = std::getenv("FDTD_PLASMA_CANARIES");
        h->canary = cv && cv[0] == '1';
    }
    if (!h) return fail(nullptr, FDTD_ERR_NOMEM, "host allocation failed");
    h->g = *g;
    if (sd) {
        h->sd_on = 1;
        h->sd_axis = sd->axis;
        h->sd_nglobal = sd->n_global;
        h->sd_extent = sd->extent;
        h->sd_lo = sd_lo;
        h->sd_hi = sd_hi;
        h->sd_origin = sd->offset - sd_lo;
        if (sd->axis == 1) h->g.ny = n[1];     // the handle's grid desc is the local one
        else h->g.nz = n[2];
    }
    if (rt) h->rt = *rt;
    h->stream = (cudaStream_t)h->rt.stream;
    h->nx = n[0]; h->ny = n[1]; h->nz = n[2];
    h->dt = g->courant * g->dx / kC0;
    h->esz = g->precision == FDTD_F64 ? 8 : 4;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        int r = cuda_fail(nullptr, ce, "device setup");
        delete h;
        return r;
    }
    int rc = FDTD_OK;
    auto bail = [&](int code, const char *what) {
        g_create_error = h->err.empty() ? std::string(what) : std::string(what) + ": " + h->err;
        fdtd_plasma_destroy(h);
        return code;
    };
    // fields
    if (g->ndim == 1) {
        h->flen[FDTD_EX] = h->nz + 1;
        h->flen[FDTD_HY] = h->nz;
    } else if (g->ndim == 2) {
        h->flen[FDTD_EZ] = h->flen[FDTD_HX] = h->flen[FDTD_HY] = ncell;
    } else {
        for (int q = 0; q < 6; ++q) h->flen[q] = ncell;
    }
    for (int q = 0; q < 6; ++q)
        if (h->flen[q]) {
            h->f[q] = dalloc(h, h->flen[q] * h->esz);
            if (!h->f[q]) return bail(FDTD_ERR_NOMEM, "field allocation failed");
        }
    // CPML: profiles + psi slabs
    if (g->ndim >= 2 && g->cpml_cells) {
        const int64_t L2 = 2 * (int64_t)g->cpml_cells;
        std::vector<double> tabs;
        for (int ax = 0; ax < g->ndim; ++ax) {
            // a sub-domain's split axis takes the global profile at its planes' global positions: its local
            // layer planes that are not in a global layer get b = a = 0, 1/kappa = 1, so psi stays 0 there and
            // the update equals the interior one exactly
            const int64_t off = (h->sd_on && ax == h->sd_axis) ? h->sd_origin : 0;
            for (int at_h = 0; at_h < 2; ++at_h) {
                std::vector<double> b, a, ik;
                cpml_axis(*g, h->dt, n_full[ax], at_h != 0, b, a, ik);
                tabs.insert(tabs.end(), b.begin() + off, b.begin() + off + n[ax]);
                tabs.insert(tabs.end(), a.begin() + off, a.begin() + off + n[ax]);
                tabs.insert(tabs.end(), ik.begin() + off, ik.begin() + off + n[ax]);
            }
        }
        h->prof_len = (int64_t)tabs.size();
        h->prof = dalloc(h, tabs.size() * h->esz);
        if (!h->prof) return bail(FDTD_ERR_NOMEM, "CPML table allocation failed");
        if (h->esz == 8) {
            rc = cudaMemcpy(h->prof, tabs.data(), tabs.size() * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> t32(tabs.begin(), tabs.end());
            rc = cudaMemcpy(h->prof, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice);
        }
        if (rc != cudaSuccess) return bail(FDTD_ERR_CUDA, "CPML table upload failed");
        if (g->ndim == 2) {
            h->psilen[0] = h->psilen[3] = h->ny * L2;   // x-slabs
            h->psilen[1] = h->psilen[2] = L2 * h->nx;   // y-slabs
        } else {
            const int64_t xs = h->nz * h->ny * L2, ys = h->nz * L2 * h->nx, zs = L2 * h->ny * h->nx;
            const int axis_of_slot[12] = {1, 2, 0, 2, 0, 1, 1, 2, 0, 2, 0, 1};
            for (int q = 0; q < 12; ++q) h->psilen[q] = axis_of_slot[q] == 0 ? xs : (axis_of_slot[q] == 1 ? ys : zs);
        }
        for (int q = 0; q < 12; ++q)
            if (h->psilen[q]) {
                h->psi[q] = dalloc(h, h->psilen[q] * h->esz);
                if (!h->psi[q]) return bail(FDTD_ERR_NOMEM, "psi allocation failed");
            }
    }
    h->mur_state = dalloc(h, 4 * 8);
    h->d_step = (int64_t *)dalloc(h, 256);
    h->d_src = (double *)dalloc(h, 256);
    h->d_err = (int *)dalloc(h, 256);
    h->diag_blocks = h->num_sms * 4;
    h->diag_partials = (double *)dalloc(h, (size_t)h->diag_blocks * 7 * sizeof(double));
    h->diag_out = (double *)dalloc(h, 8 * sizeof(double));
    if (!h->mur_state || !h->d_step || !h->d_src || !h->d_err || !h->diag_partials || !h->diag_out)
        return bail(FDTD_ERR_NOMEM, "small allocation failed");
    if (g->ndim >= 2) apply_cached_stencil(h);
    rc = fdtd_plasma_reset(h);
    if (rc != FDTD_OK) {
        g_create_error = h->err;
        fdtd_plasma_destroy(h);
        return rc;
    }
    cudaError_t se = cudaStreamSynchronize(h->stream);
    if (se != cudaSuccess) return bail(FDTD_ERR_CUDA, cudaGetErrorString(se));
    *out = h;
    return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_plasma_create(const fdtd_grid_desc *g, const fdtd_runtime_desc *rt, fdtd_plasma_t *out)
{
    return create_impl(g, rt, out, nullptr);
}

int fdtd_plasma_create_subdomain(const fdtd_grid_desc *global, const fdtd_subdomain_desc *sd,
                                 const fdtd_runtime_desc *rt, fdtd_plasma_t *out)
{
    if (!sd) return fail(nullptr, FDTD_ERR_INVAL, "subdomain desc is NULL");
    SubInfo si{sd->axis, sd->n_global, sd->offset, sd->extent};
    return create_impl(global, rt, out, &si);
}

int fdtd_plasma_check_canaries(fdtd_plasma_t h, int64_t *corrupted)
{
    NvtxRange nvtx_("fdtd_plasma_check_canaries");
    if (!h || !corrupted) return FDTD_ERR_INVAL;
    if (!h->canary) return fail(h, FDTD_ERR_STATE, "canaries are off (set FDTD_PLASMA_CANARIES=1 before create)");
    CK(h, cudaStreamSynchronize(h->stream));
    std::vector<unsigned char> pad(2 * kCanaryPad);
    int64_t bad = 0;
    for (const auto &a : h->canary_allocs) {
        CK(h, cudaMemcpy(pad.data(), a.first - kCanaryPad, kCanaryPad, cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(pad.data() + kCanaryPad, a.first + a.second, kCanaryPad, cudaMemcpyDeviceToHost));
        for (unsigned char c : pad)
            if (c != kCanaryByte) {
                ++bad;
                break;
            }
    }
    *corrupted = bad;
    return FDTD_OK;
}

int fdtd_plasma_set_option(fdtd_plasma_t h, int option, int64_t value)
{
    if (!h) return FDTD_ERR_INVAL;
    if (option == FDTD_OPT_FUSED_STENCILS) {
        if (value != 0 && value != 1) return fail(h, FDTD_ERR_INVAL, "FDTD_OPT_FUSED_STENCILS takes 0 or 1");
        if (value && h->sd_on) return fail(h, FDTD_ERR_STATE, "sub-domains exchange halos between the E and H passes");
        CK(h, cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        h->fuse = (int)value;
        if (!h->fuse && h->auto_fuse_rows <= 0) free_second_set(h);
        return FDTD_OK;
    }
    if (option == FDTD_OPT_FUSED_ROWS) {
        if (value < 0 || value > 4096) return fail(h, FDTD_ERR_INVAL, "FDTD_OPT_FUSED_ROWS takes 0 .. 4096");
        CK(h, cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        h->fuse_rows = (int)value;
        return FDTD_OK;
    }
    if (option == FDTD_OPT_STENCIL_TZ) {
        if (value < 0 || value > 1024) return fail(h, FDTD_ERR_INVAL, "FDTD_OPT_STENCIL_TZ takes 0 .. 1024");
        if (value > 0) {
            if (h->g.ndim < 2 || h->g.precision != FDTD_F32)
                return fail(h, FDTD_ERR_INVAL, "the TMA stencils run on 2-D and 3-D FP32 grids");
            if (!h->tma) h->tma = tma_maps_create(reinterpret_cast<float *const *>(h->f), h->nx, h->ny, h->nz);
            if (!h->tma) return fail(h, FDTD_ERR_INVAL, "the TMA stencils need nx a multiple of 4");
        }
        CK(h, cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        h->st_tz = (int)value;
        if (value > 0) { h->st_bx = 32; h->st_by = 8; h->st_bz = 1; h->st_cpt = 1; }
        return FDTD_OK;
    }
    if (option == FDTD_OPT_KINETIC_SHAPE) {
        if (!h->has_plasma) return fail(h, FDTD_ERR_STATE, "FDTD_OPT_KINETIC_SHAPE needs a plasma (set_plasma first)");
        const int stages = (int)(value / 1000000000), vpl = (int)(value / 1000000 % 1000),
                  l = (int)(value / 1000 % 1000), bps = (int)(value % 1000);
        if (value != 0) {
            int cand[32][2];
            const int nc = kinetic_candidates(h->pitch, h->pl.f_dtype, cand);
            bool ok = false;
            for (int c = 0; c < nc; ++c) ok |= cand[c][0] == vpl && cand[c][1] == l;
            if (value < 0 || !ok)
                return fail(h, FDTD_ERR_INVAL, "FDTD_OPT_KINETIC_SHAPE: %lld is not a candidate shape of this row length",
                            (long long)value);
            if (stages > 0 && (stages > 64 || h->pl.nonlinear || h->pl.evolve_f0 ||
                               !kinetic_ring_fits(h->pitch, h->pl.f_dtype, l, stages)))
                return fail(h, FDTD_ERR_INVAL,
                            "FDTD_OPT_KINETIC_SHAPE: %d ring stages (2..64 that fit in shared memory; FP32 / BF16 rows "
                            "of the linear update only)",
                            stages);
        }
        CK(h, cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        h->kin_vpl = vpl;
        h->kin_l = l;
        h->kin_bps = bps;
        h->kin_stages = stages;
        return FDTD_OK;
    }
    return fail(h, FDTD_ERR_INVAL, "unknown option %d", option);
}

int fdtd_plasma_launch_shapes(fdtd_plasma_t h, fdtd_tune_result *out)
{
    if (!h || !out) return FDTD_ERR_INVAL;
    *out = fdtd_tune_result{};
    out->kin_vpl = h->kin_vpl;
    out->kin_l = h->kin_l;
    out->kin_blocks_per_sm = h->kin_bps;
    out->kin_stages = h->kin_stages;
    if (h->g.ndim >= 2) {
        const dim3 b = stencil_block(h);
        out->block_x = (int32_t)b.x; out->block_y = (int32_t)b.y; out->block_z = (int32_t)b.z;
        out->cells_per_thread = stencil_cpt(h);
        out->stencil_tz = h->st_tz;
        out->fused_rows = h->g.ndim == 2 && h->g.precision == FDTD_F32 && !h->sd_on && (h->fuse || h->auto_fuse_rows > 0)
                              ? fuse_rows_of(h)
                              : 0;
    }
    return FDTD_OK;
}

int fdtd_plasma_reset(fdtd_plasma_t h)
{
    if (!h) return FDTD_ERR_INVAL;
    for (int q = 0; q < 6; ++q)
        if (h->f[q]) CK(h, cudaMemsetAsync(h->f[q], 0, field_bytes(h, q), h->stream));
    for (int q = 0; q < 12; ++q)
        if (h->psi[q]) CK(h, cudaMemsetAsync(h->psi[q], 0, h->psilen[q] * h->esz, h->stream));
    if (h->has_plasma) {
        CK(h, cudaMemsetAsync(h->df, 0, (size_t)h->nkin * h->pitch * h->df_esz, h->stream));
        if (h->g0) CK(h, cudaMemsetAsync(h->g0, 0, (size_t)h->nkin * h->pitch * h->df_esz, h->stream));
        CK(h, cudaMemsetAsync(h->jslot, 0, (size_t)(h->nslots ? h->nslots : 1) * h->esz, h->stream));
    }
    if (h->hist) CK(h, cudaMemsetAsync(h->hist, 0, (size_t)(h->has_closure ? h->ncl : h->nslots) * 16 * 4, h->stream));
    if (h->jprev) CK(h, cudaMemsetAsync(h->jprev, 0, (size_t)(h->has_closure ? h->ncl : h->nslots) * 4, h->stream));
    if (h->port_acc) CK(h, cudaMemsetAsync(h->port_acc, 0, (size_t)h->nports * h->nfreq * 2 * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->mur_state, 0, 32, h->stream));
    CK(h, cudaMemsetAsync(h->d_step, 0, sizeof(int64_t), h->stream));
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    h->steps_done = 0;
    h->sd_half = 0;
    return FDTD_OK;
}

int fdtd_plasma_set_source(fdtd_plasma_t h, const fdtd_source_desc *s)
{
    if (!h || !s) return FDTD_ERR_INVAL;
    if (s->kind == FDTD_SRC_NONE) {
        h->has_source = 0;
        drop_graphs(h);
        return FDTD_OK;
    }
    if (s->kind != FDTD_SRC_GAUSS_SINE && s->kind != FDTD_SRC_GAUSS) return fail(h, FDTD_ERR_INVAL, "bad source kind");
    if (!(s->tau > 0) || !std::isfinite(s->amp) || !std::isfinite(s->fc) || !std::isfinite(s->t0) || !std::isfinite(s->tau))
        return fail(h, FDTD_ERR_INVAL, "source parameters must be finite, tau > 0");
    const int nd = h->g.ndim;
    fdtd_source_desc loc = *s;
    if (h->sd_on) {
        // global coordinates: a sub-domain keeps the source only when it owns the source's plane
        int64_t &c = h->sd_axis == 1 ? loc.j : loc.k;
        if (c < 1 || c >= h->sd_nglobal) return fail(h, FDTD_ERR_INVAL, "source node outside the updated nodes");
        c -= h->sd_origin;
        if (c < h->sd_lo || c >= h->sd_lo + h->sd_extent) {
            h->src = *s;
            h->has_source = 0;
            drop_graphs(h);
            return FDTD_OK;
        }
        s = &loc;
    }
    if (s->location == FDTD_LOC_POINT) {
        bool ok;
        if (nd == 1) ok = s->k >= 1 && s->k <= h->nz - 1;
        else if (nd == 2) ok = s->i >= 1 && s->i < h->nx && s->j >= 1 && s->j < h->ny;
        else ok = s->i >= 0 && s->i < h->nx && s->j >= 1 && s->j < h->ny && s->k >= 1 && s->k < h->nz;
        if (!ok) return fail(h, FDTD_ERR_INVAL, "source node outside the updated nodes");
    } else if (s->location == FDTD_LOC_SHEET) {
        if (nd != 3) return fail(h, FDTD_ERR_INVAL, "sheet sources are 3-D only");
        if (!(s->k >= 1 && s->k < h->nz && s->i0 >= 0 && s->i1 <= h->nx && s->i0 < s->i1 && s->j0 >= 1 &&
              s->j1 <= h->ny && s->j0 < s->j1))
            return fail(h, FDTD_ERR_INVAL, "sheet outside the updated Ex nodes");
    } else {
        return fail(h, FDTD_ERR_INVAL, "bad source location");
    }
    h->src = *s;
    h->has_source = 1;
    drop_graphs(h);
    return FDTD_OK;
}

int fdtd_plasma_set_plasma(fdtd_plasma_t h, const fdtd_plasma_desc *p)
{
    NvtxRange nvtx_("fdtd_plasma_set_plasma");
    if (!h || !p) return FDTD_ERR_INVAL;
    if (h->steps_done != 0) return fail(h, FDTD_ERR_STATE, "set_plasma after stepping: call fdtd_plasma_reset first");
    if (!p->density) return fail(h, FDTD_ERR_INVAL, "density is NULL");
    if (p->vgrid < 0 || p->vgrid > 2) return fail(h, FDTD_ERR_INVAL, "bad vgrid");
    if (p->nv < 2 || (p->vgrid == FDTD_VGRID_CART2D && p->nv_perp < 1))
        return fail(h, FDTD_ERR_INVAL, "nv too small");
    if (!(p->te_ev > 0) || !(p->vmax_vth > 0) || !(p->nu0 >= 0) || !std::isfinite(p->nu0))
        return fail(h, FDTD_ERR_INVAL, "te_ev, vmax_vth must be > 0 and nu0 >= 0");
    if (const char *why = check_velocity_model(*p)) return fail(h, FDTD_ERR_INVAL, "%s", why);
    const bool f64 = h->g.precision == FDTD_F64;
    if (f64 ? p->f_dtype != FDTD_DF_F64 : (p->f_dtype != FDTD_DF_F32 && p->f_dtype != FDTD_DF_BF16))
        return fail(h, FDTD_ERR_INVAL, "f_dtype does not match the field precision");
    if (p->nonlinear && (p->vgrid == FDTD_VGRID_SPEED3D || p->f_dtype == FDTD_DF_BF16))
        return fail(h, FDTD_ERR_INVAL, "the nonlinear mode needs a v_par grid (signed or Cartesian) and FP32/FP64 delta f");
    if (p->evolve_f0 && (p->vgrid != FDTD_VGRID_SPEED3D || p->f_dtype == FDTD_DF_BF16 || p->nonlinear))
        return fail(h, FDTD_ERR_INVAL, "evolve_f0 needs the speed grid and FP32/FP64 delta f (not the nonlinear mode)");
    if (p->evolve_f0 && (!(p->mass_ratio >= 0) || !std::isfinite(p->mass_ratio) || !(p->tg_ev >= 0) ||
                         !std::isfinite(p->tg_ev)))
        return fail(h, FDTD_ERR_INVAL, "evolve_f0: mass_ratio and tg_ev must be finite and >= 0");
    const int64_t nnode = p->vgrid == FDTD_VGRID_CART2D ? (int64_t)p->nv * p->nv_perp : p->nv;
    const int pitch = kinetic_pitch((int)nnode, p->f_dtype);
    const int vec = p->f_dtype == FDTD_DF_BF16 ? 8 : (p->f_dtype == FDTD_DF_F64 ? 2 : 4);
    if (pitch / vec > 512) return fail(h, FDTD_ERR_INVAL, "too many velocity nodes for this storage type");

    // density: compact the plasma cells
    const int64_t np = pol_len(h);
    std::vector<double> dens(h->sd_on ? np : 0);
    int64_t slot_base = 0;
    if (h->sd_on) {
        // a sub-domain reads its planes of the global density array; its slots are numbered after the
        // global plasma slots below its first owned plane
        const int64_t plane = h->sd_axis == 1 ? h->nx : h->nx * h->ny;
        const int64_t npg = plane * h->sd_nglobal;
        std::vector<double> all(npg);
        if (p->density_on_device) CK(h, cudaMemcpy(all.data(), p->density, npg * 8, cudaMemcpyDeviceToHost));
        else std::memcpy(all.data(), p->density, npg * 8);
        const int64_t first = (h->sd_origin + h->sd_lo) * plane;
        for (int64_t c = 0; c < first; ++c) {
            const int64_t i = c % h->nx, j = (c / h->nx) % h->ny, k = c / plane;
            const bool upd = h->sd_axis == 1 ? (i >= 1 && c / h->nx >= 1) : (j >= 1 && k >= 1);
            if (all[c] > 0.0 && upd) ++slot_base;
        }
        std::memcpy(dens.data(), all.data() + h->sd_origin * plane, np * 8);
        for (int64_t c = 0; c < np; ++c) {     // ghost planes carry no plasma
            const int64_t l = c / plane;
            if (l < h->sd_lo || l >= h->sd_lo + h->sd_extent) dens[c] = 0.0;
        }
    }
    std::vector<int32_t> cells;
    std::vector<double> dslot;
    double nmax = 0.0;
    // the compaction's device copy of the slots (whole grids), freed on every way out
    struct DevSlots {
        fdtd_plasma *h;
        void *p = nullptr;
        ~DevSlots() { dfree(h, p); }
    } dev_slots{h};
    if (!h->sd_on) {
        // a whole grid: the density stays on (or goes once to) the device and is compacted there
        const int rc = compact_on_gpu(h, p, np, cells, dslot, nmax, &dev_slots.p);
        if (rc != FDTD_OK) return rc;
    } else {
        for (int64_t c = 0; c < np; ++c) {
            const double d = dens[c];
            if (!std::isfinite(d) || d < 0.0) return fail(h, FDTD_ERR_NONFINITE, "density must be finite and >= 0");
            if (d > 0.0 && pol_updated(h, c)) {
                cells.push_back((int32_t)c);
                dslot.push_back(d);
                if (d > nmax) nmax = d;
            }
        }
    }
    // plasma-modified stability of Yee + Crank-Nicolson current: (w_p dt/2)^2 + S^2 ndim < 1
    const double wp = std::sqrt(nmax * kQe * kQe / (kEps0 * kMe));
    if (std::pow(wp * h->dt / 2, 2) + h->g.courant * h->g.courant * h->g.ndim >= 1.0)
        return fail(h, FDTD_ERR_UNSTABLE, "plasma frequency %g rad/s too high for dt %g", wp, h->dt);

    VTab t;
    fdtd_plasma_desc pd = *p;
    if (!velocity_tables(pd, t)) return fail(h, FDTD_ERR_INVAL, "bad velocity grid");
    // folded tables: alpha, beta, w' = -e w (padding nodes: 0)
    std::vector<double> tab(3 * (size_t)pitch, 0.0);
    for (int64_t j = 0; j < nnode; ++j) {
        const double nu = t.nu[j];
        tab[j] = (2.0 - h->dt * nu) / (2.0 + h->dt * nu);
        tab[pitch + j] = 2.0 * h->dt * (kQe / kMe) * t.f0p[j] / (2.0 + h->dt * nu);
        tab[2 * pitch + j] = -kQe * t.w[j];
    }
    // evolve_f0 tables (padding 0): f0, f0', bq = 2 dt (e/m) / (2 + dt nu), v^3, 1/(v^2 gam), and for
    // the upper cell edge v_e = (j+1) gam of each node but the last: 1/(2 v_e), (m/M) v_e^3 nu_e
    // (nu_e the mean of the two nodes), k Tg / (m v_e gam)
    std::vector<double> tabf0(p->evolve_f0 ? 8 * (size_t)pitch : 0, 0.0);
    if (p->evolve_f0) {
        const double gam = 2.0 * t.v[0];
        const double kTg_m = kQe * p->tg_ev / kMe;
        for (int64_t j = 0; j < nnode; ++j) {
            const double v = t.v[j];
            tabf0[j] = t.f0[j];
            tabf0[pitch + j] = t.f0p[j];
            tabf0[2 * pitch + j] = 2.0 * h->dt * (kQe / kMe) / (2.0 + h->dt * t.nu[j]);
            tabf0[3 * pitch + j] = v * v * v;
            tabf0[4 * pitch + j] = 1.0 / (v * v * gam);
            if (j + 1 < nnode) {
                const double ve = (double)(j + 1) * gam;
                tabf0[5 * pitch + j] = 1.0 / (2.0 * ve);
                tabf0[6 * pitch + j] = p->mass_ratio * ve * ve * ve * 0.5 * (t.nu[j] + t.nu[j + 1]);
                tabf0[7 * pitch + j] = kTg_m / (ve * gam);
            }
        }
    }

    drop_graphs(h);
    // a delta-f array of the same size is kept (set_plasma on a reset solver with the same plasma layout):
    // only zeroed below, not freed and allocated again
    const size_t df_need = (cells.empty() ? 1 : cells.size()) * (size_t)pitch *
                           (p->f_dtype == FDTD_DF_BF16 ? 2 : (p->f_dtype == FDTD_DF_F64 ? 8 : 4));
    void *keep_df = nullptr;
    if (h->df && h->df_bytes == df_need) {
        keep_df = h->df;
        h->df = nullptr;
    }
    free_plasma(h);
    const size_t ns = cells.size();
    h->pl = *p;
    h->pl.density = nullptr;
    h->pl.s_speed = h->pl.s_sigma = nullptr;   // caller memory, read above only
    h->pl.s_n = 0;
    h->nslots = (int64_t)ns;
    h->nnode = nnode;
    h->pitch = pitch;
    h->df_esz = p->f_dtype == FDTD_DF_BF16 ? 2 : (p->f_dtype == FDTD_DF_F64 ? 8 : 4);
    // slot index and density arrays in multiples of four entries: the ring kernel's bulk copies of them are
    // rounded up to 16 bytes
    h->slot_cell = (int32_t *)dalloc(h, ((ns + 3) & ~(size_t)3) * 4);
    h->dens = dalloc(h, ((ns + 3) & ~(size_t)3) * h->esz);
    h->df = keep_df ? keep_df : dalloc(h, df_need);
    h->df_bytes = df_need;
    h->jslot = dalloc(h, (ns ? ns : 1) * h->esz);
    h->tab = dalloc(h, tab.size() * h->esz);
    h->dV = (double *)dalloc(h, nnode * 8);
    if (p->evolve_f0) {
        h->g0 = dalloc(h, (ns ? ns : 1) * pitch * h->df_esz);
        h->tab_f0 = dalloc(h, 8 * (size_t)pitch * h->esz);
    }
    if (!h->slot_cell || !h->dens || !h->df || !h->jslot || !h->tab || !h->dV ||
        (p->evolve_f0 && (!h->g0 || !h->tab_f0))) {
        free_plasma(h);
        return fail(h, FDTD_ERR_NOMEM, "plasma allocation failed (%zu cells x %d nodes)", ns, pitch);
    }
    h->has_plasma = 1;
    h->slot_base = slot_base;
    h->nkin = (int64_t)ns;
    h->kin_vpl = h->kin_l = h->kin_bps = h->kin_stages = 0;
    apply_cached_kinetic(h);
    if (ns && dev_slots.p) {   // device to device from the compaction (densities converted to FP32 there)
        const double *d_dens = static_cast<const double *>(dev_slots.p);
        const int32_t *d_cells = reinterpret_cast<const int32_t *>(d_dens + ns);
        CK(h, cudaMemcpyAsync(h->slot_cell, d_cells, ns * 4, cudaMemcpyDeviceToDevice, h->stream));
        if (h->esz == 8) CK(h, cudaMemcpyAsync(h->dens, d_dens, ns * 8, cudaMemcpyDeviceToDevice, h->stream));
        else CK(h, launch_to_f32(h->stream, d_dens, static_cast<float *>(h->dens), (int64_t)ns));
    } else if (ns) {
        CK(h, cudaMemcpy(h->slot_cell, cells.data(), ns * 4, cudaMemcpyHostToDevice));
        if (h->esz == 8) {
            CK(h, cudaMemcpy(h->dens, dslot.data(), ns * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> d32(dslot.begin(), dslot.end());
            CK(h, cudaMemcpy(h->dens, d32.data(), ns * 4, cudaMemcpyHostToDevice));
        }
    }
    if (h->esz == 8) {
        CK(h, cudaMemcpy(h->tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> t32(tab.begin(), tab.end());
        CK(h, cudaMemcpy(h->tab, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice));
    }
    h->h_cells = std::move(cells);
    h->h_dens = std::move(dslot);
    CK(h, cudaMemcpy(h->dV, t.dV.data(), nnode * 8, cudaMemcpyHostToDevice));
    if (p->evolve_f0) {
        if (h->esz == 8) {
            CK(h, cudaMemcpy(h->tab_f0, tabf0.data(), tabf0.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> t32(tabf0.begin(), tabf0.end());
            CK(h, cudaMemcpy(h->tab_f0, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice));
        }
        CK(h, cudaMemsetAsync(h->g0, 0, (ns ? ns : 1) * pitch * h->df_esz, h->stream));
    }
    CK(h, cudaMemsetAsync(h->df, 0, (ns ? ns : 1) * pitch * h->df_esz, h->stream));
    CK(h, cudaMemsetAsync(h->jslot, 0, (ns ? ns : 1) * h->esz, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

int fdtd_plasma_step(fdtd_plasma_t h, int64_t nsteps)
{
    NvtxRange nvtx_("fdtd_plasma_step");
    if (!h) return FDTD_ERR_INVAL;
    if (nsteps < 0) return fail(h, FDTD_ERR_INVAL, "nsteps < 0");
    if (h->sd_on && (h->sd_lo || h->sd_hi || h->sd_half))
        return fail(h, FDTD_ERR_STATE, "a sub-domain with neighbours steps by fdtd_plasma_step_half, exchanging halos");
    if (nsteps == 0) return FDTD_OK;
    if (!h->graphs_valid) {
        ensure_second_set(h);
        int rc = capture(h, 1, &h->g1);
        if (rc == FDTD_OK) rc = capture(h, kChunk, &h->gk);
        if (rc != FDTD_OK) {
            drop_graphs(h);
            return rc;
        }
        h->gk_steps = kChunk;
        h->graphs_valid = 1;
    }
    // the remainder (< 32 steps) as 16-, 8-, 4-, 2- and 1-step graphs: few launches, and the fused
    // stencil pass inside each of them; the ones this call needs are captured before anything runs
    const int64_t rem = nsteps % h->gk_steps;
    for (int b = 3; b >= 0; --b) {
        if (!((rem >> (b + 1)) & 1) || h->gpow[b]) continue;
        const int rc = capture(h, 2 << b, &h->gpow[b]);
        if (rc != FDTD_OK) {
            drop_graphs(h);
            return rc;
        }
    }
    for (int64_t c = nsteps / h->gk_steps; c > 0; --c) CK(h, cudaGraphLaunch(h->gk, h->stream));
    for (int b = 3; b >= 0; --b)
        if ((rem >> (b + 1)) & 1) CK(h, cudaGraphLaunch(h->gpow[b], h->stream));
    if (rem & 1) CK(h, cudaGraphLaunch(h->g1, h->stream));
    h->steps_done += nsteps;
    return FDTD_OK;
}

int fdtd_plasma_step_half(fdtd_plasma_t h, int half)
{
    NvtxRange nvtx_("fdtd_plasma_step_half");
    if (!h || (half != 0 && half != 1)) return FDTD_ERR_INVAL;
    if (h->fuse) return fail(h, FDTD_ERR_STATE, "half steps do not run the fused stencil pass (FDTD_OPT_FUSED_STENCILS)");
    if (half != h->sd_half)
        return fail(h, FDTD_ERR_STATE, half ? "half 1 needs half 0 of the step first" : "half 1 of the step is pending");
    const FieldSet<float> f32 = field_set<float>(h, 0);
    const FieldSet<double> f64 = field_set<double>(h, 0);
    const bool dbl = h->g.precision == FDTD_F64;
    cudaError_t e;
    if (half == 0) {
        e = dbl ? part_h<double>(h, h->stream, 0, f64) : part_h<float>(h, h->stream, 0, f32);
        if (e != cudaSuccess) return cuda_fail(h, e, "H half step");
        h->sd_half = 1;
        return FDTD_OK;
    }
    e = dbl ? part_mid<double>(h, h->stream, 0, f64, nullptr) : part_mid<float>(h, h->stream, 0, f32, nullptr);
    if (e == cudaSuccess) e = dbl ? part_e<double>(h, h->stream, 0, f64) : part_e<float>(h, h->stream, 0, f32);
    if (e == cudaSuccess) e = dbl ? part_ports<double>(h, h->stream, 0, f64) : part_ports<float>(h, h->stream, 0, f32);
    if (e == cudaSuccess) {
        launch_advance(h->stream, h->d_step, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "E half step");
    h->sd_half = 0;
    h->steps_done += 1;
    return FDTD_OK;
}

namespace {
// the field planes a halo carries: 3-D (split along z) the x- and y-components of the plane, 2-D TMz (split
// along y) Ez or Hx of the row; E: the tangential E the neighbour below needs for its H update, H: the
// tangential H the neighbour above needs for its E update
int halo_comps(const fdtd_plasma *h, int which, int comp[2])
{
    if (h->g.ndim == 3) {
        comp[0] = which == FDTD_HALO_E ? FDTD_EX : FDTD_HX;
        comp[1] = which == FDTD_HALO_E ? FDTD_EY : FDTD_HY;
        return 2;
    }
    comp[0] = which == FDTD_HALO_E ? FDTD_EZ : FDTD_HX;
    return 1;
}

int64_t halo_plane(const fdtd_plasma *h) { return h->g.ndim == 3 ? h->nx * h->ny : h->nx; }

int halo_copy(fdtd_plasma *h, int which, bool pack, void *buf, int buf_is_device)
{
    if (!h || !buf || (which != FDTD_HALO_E && which != FDTD_HALO_H)) return FDTD_ERR_INVAL;
    if (!h->sd_on) return fail(h, FDTD_ERR_STATE, "halos belong to sub-domains (fdtd_plasma_create_subdomain)");
    // pack E: first owned plane (for the neighbour below); unpack E: top ghost plane (from the neighbour above);
    // pack H: last owned plane (for the neighbour above); unpack H: bottom ghost plane (from the neighbour below)
    const bool need_below = (which == FDTD_HALO_E) == pack;
    if (need_below ? !h->sd_lo : !h->sd_hi)
        return fail(h, FDTD_ERR_STATE, "no neighbour %s this sub-domain for that halo", need_below ? "below" : "above");
    int64_t l;
    if (which == FDTD_HALO_E) l = pack ? h->sd_lo : h->sd_lo + h->sd_extent;
    else l = pack ? h->sd_lo + h->sd_extent - 1 : 0;
    int comp[2];
    const int nc = halo_comps(h, which, comp);
    const size_t bytes = (size_t)halo_plane(h) * h->esz;
    for (int q = 0; q < nc; ++q) {
        char *field = static_cast<char *>(h->f[comp[q]]) + (size_t)l * bytes;
        char *b = static_cast<char *>(buf) + (size_t)q * bytes;
        const cudaMemcpyKind kind = buf_is_device ? cudaMemcpyDeviceToDevice
                                                  : (pack ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
        CK(h, pack ? cudaMemcpyAsync(b, field, bytes, kind, h->stream) : cudaMemcpyAsync(field, b, bytes, kind, h->stream));
    }
    if (!buf_is_device) CK(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}
}  // namespace

size_t fdtd_plasma_halo_bytes(fdtd_plasma_t h, int which)
{
    if (!h || !h->sd_on || (which != FDTD_HALO_E && which != FDTD_HALO_H)) return 0;
    int comp[2];
    return (size_t)halo_comps(h, which, comp) * (size_t)halo_plane(h) * h->esz;
}

int fdtd_plasma_halo_pack(fdtd_plasma_t h, int which, void *dst, int dst_is_device)
{
    NvtxRange nvtx_("fdtd_plasma_halo_pack");
    return halo_copy(h, which, true, dst, dst_is_device);
}

int fdtd_plasma_halo_unpack(fdtd_plasma_t h, int which, const void *src, int src_is_device)
{
    NvtxRange nvtx_("fdtd_plasma_halo_unpack");
    return halo_copy(h, which, false, const_cast<void *>(src), src_is_device);
}

int fdtd_plasma_set_closure(fdtd_plasma_t h, const fdtd_closure_desc *c)
{
    NvtxRange nvtx_("fdtd_plasma_set_closure");
    if (!h || !c || !c->params) return FDTD_ERR_INVAL;
    if (h->sd_on) return fail(h, FDTD_ERR_STATE, "the closure runs on whole grids, not on sub-domains");
    if (!h->has_plasma) return fail(h, FDTD_ERR_STATE, "set_closure needs a plasma (set_plasma first)");
    if (h->steps_done != 0) return fail(h, FDTD_ERR_STATE, "set_closure after stepping: call fdtd_plasma_reset first");
    if (h->g.precision != FDTD_F32) return fail(h, FDTD_ERR_INVAL, "the closure runs on FP32 grids");
    if (h->pl.evolve_f0) return fail(h, FDTD_ERR_INVAL, "the closure replaces a fixed-F0 plasma (evolve_f0 is set)");
    if (!(c->e_scale > 0) || !(c->n_scale > 0) || !std::isfinite(c->j_scale) || !std::isfinite(c->rho) ||
        !std::isfinite(c->beta) ||
        !(c->n_train_max >= 0))
        return fail(h, FDTD_ERR_INVAL, "closure scales must be finite, e_scale and n_scale > 0");
    std::vector<float> P(FDTD_MLP_NPARAMS);
    if (c->engine != 0 && c->engine != 1) return fail(h, FDTD_ERR_INVAL, "closure engine must be 0 or 1");
    if (c->params_on_device) CK(h, cudaMemcpy(P.data(), c->params, P.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(P.data(), c->params, P.size() * 4);
    for (float v : P)
        if (!std::isfinite(v)) return fail(h, FDTD_ERR_NONFINITE, "closure parameters must be finite");
    // re-layout: kinetic (fallback) slots first, closure slots after, each in cell order
    std::vector<int32_t> cells;
    std::vector<double> dens;
    for (size_t q = 0; q < h->h_cells.size(); ++q)
        if (h->h_dens[q] > c->n_train_max) { cells.push_back(h->h_cells[q]); dens.push_back(h->h_dens[q]); }
    const int64_t nk = (int64_t)cells.size();
    for (size_t q = 0; q < h->h_cells.size(); ++q)
        if (!(h->h_dens[q] > c->n_train_max)) { cells.push_back(h->h_cells[q]); dens.push_back(h->h_dens[q]); }
    const int64_t ns = (int64_t)cells.size(), nc = ns - nk;
    drop_graphs(h);
    free_closure(h);
    dfree(h, h->slot_cell); dfree(h, h->dens); dfree(h, h->df); dfree(h, h->jslot);
    h->slot_cell = (int32_t *)dalloc(h, ((ns + 3) & ~(int64_t)3) * 4);
    h->dens = dalloc(h, ((ns + 3) & ~(int64_t)3) * 4);
    h->df_bytes = (nk ? nk : 1) * h->pitch * h->df_esz;
    h->df = dalloc(h, h->df_bytes);
    h->jslot = dalloc(h, (ns ? ns : 1) * 4);
    h->hist = (float *)dalloc(h, (nc ? nc : 1) * 16 * 4);
    h->jprev = (float *)dalloc(h, (nc ? nc : 1) * 4);
    h->params = (float *)dalloc(h, P.size() * 4);
    if (!h->slot_cell || !h->dens || !h->df || !h->jslot || !h->hist || !h->jprev || !h->params) {
        free_plasma(h);
        return fail(h, FDTD_ERR_NOMEM, "closure allocation failed");
    }
    std::vector<float> d32(dens.begin(), dens.end());
    if (ns) CK(h, cudaMemcpy(h->slot_cell, cells.data(), ns * 4, cudaMemcpyHostToDevice));
    if (ns) CK(h, cudaMemcpy(h->dens, d32.data(), ns * 4, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->params, P.data(), P.size() * 4, cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->df, 0, (nk ? nk : 1) * h->pitch * h->df_esz));
    CK(h, cudaMemset(h->jslot, 0, (ns ? ns : 1) * 4));
    CK(h, cudaMemset(h->hist, 0, (nc ? nc : 1) * 16 * 4));
    CK(h, cudaMemset(h->jprev, 0, (nc ? nc : 1) * 4));
    h->h_cells = cells;
    h->h_dens = dens;
    h->nkin = nk;
    h->ncl = nc;
    h->cl = *c;
    h->cl.params = nullptr;
    h->has_closure = 1;
    return FDTD_OK;
}

int fdtd_plasma_closure_shape(fdtd_plasma_t h, int64_t *n_kinetic, int64_t *n_closure)
{
    if (!h) return FDTD_ERR_INVAL;
    if (n_kinetic) *n_kinetic = h->nkin;
    if (n_closure) *n_closure = h->ncl;
    return FDTD_OK;
}

int fdtd_plasma_set_recording(fdtd_plasma_t h, float *samples, int64_t capacity, unsigned long long *count,
                              double rate, uint64_t seed)
{
    if (!h) return FDTD_ERR_INVAL;
    if (h->sd_on) return fail(h, FDTD_ERR_STATE, "the recorder runs on whole grids, not on sub-domains");
    if (!h->has_plasma || h->has_closure) return fail(h, FDTD_ERR_STATE, "recording needs a kinetic plasma, no closure");
    if (h->g.precision != FDTD_F32) return fail(h, FDTD_ERR_INVAL, "recording runs on FP32 grids");
    if (!samples || !count || capacity < 1 || !(rate > 0) || rate > 1)
        return fail(h, FDTD_ERR_INVAL, "recording needs a buffer, a counter, capacity >= 1 and 0 < rate <= 1");
    drop_graphs(h);
    if (!h->hist) {
        const int64_t ns = h->nslots ? h->nslots : 1;
        h->hist = (float *)dalloc(h, ns * 16 * 4);
        h->jprev = (float *)dalloc(h, ns * 4);
        if (!h->hist || !h->jprev) return fail(h, FDTD_ERR_NOMEM, "recorder allocation failed");
        CK(h, cudaMemset(h->hist, 0, ns * 16 * 4));
        CK(h, cudaMemset(h->jprev, 0, ns * 4));
    }
    h->rec_out = samples;
    h->rec_cap = capacity;
    h->rec_count = count;
    h->rec_threshold = rate >= 1.0 ? 0xffffffffu : (uint32_t)(rate * 4294967296.0);
    h->rec_seed = seed;
    h->has_recording = 1;
    return FDTD_OK;
}

}  // extern "C"

namespace {

// A later candidate replaces the best so far only when it is more than 1 % faster: candidates that
// time within noise of each other do not flip from run to run (the built-in shapes come first).
constexpr double kTuneMargin = 0.99;

template <typename T>
int autotune_t(fdtd_plasma *h, fdtd_tune_result *out)
{
    const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
    const T ch = (T)(h->dt / (mu0 * h->g.dx)), ce = (T)(h->dt / (kEps0 * h->g.dx));
    const T cph = (T)(h->dt / mu0), cpe = (T)(h->dt / kEps0);
    T *f[6];
    for (int q = 0; q < 6; ++q) f[q] = reinterpret_cast<T *>(h->f[q]);
    const Cpml<T> cp = cpml_view<T>(h);
    const Source src = source_view(h);
    cudaStream_t st = h->stream;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    auto time_ms = [&](auto &&launch) -> double {
        launch();   // warm-up (also sets attributes)
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) launch();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 5.0;
    };
    auto m = read_cache();
    out->block_x = out->block_y = out->block_z = out->cells_per_thread = out->stencil_tz = out->fused_rows = 0;
    out->stencil_ms = 0;
    if (h->g.ndim >= 2) {
        static const int s2[][3] = {{32, 8, 1}, {64, 4, 1}, {128, 2, 1}, {256, 1, 1}, {32, 4, 1}, {64, 2, 1}};
        static const int s3[][3] = {{32, 4, 2}, {32, 8, 1}, {32, 2, 4}, {64, 4, 1}, {64, 2, 2}, {128, 2, 1}, {32, 4, 1}};
        const int n = h->g.ndim == 2 ? 6 : 7;
        const bool quads = h->g.precision == FDTD_F32 && h->nx % 4 == 0;
        double best = 1e30;
        for (int cpt : {1, 4}) {
            if (cpt == 4 && !quads) continue;
            for (int c = 0; c < n; ++c) {
                const int *sh = h->g.ndim == 2 ? s2[c] : s3[c];
                const dim3 b(sh[0], sh[1], sh[2]);
                const double ms = time_ms([&] {
                    if (h->g.ndim == 2) {
                        launch_h2d<T>(st, f[FDTD_EZ], f[FDTD_HX], f[FDTD_HY], h->nx, h->ny, ch, cph, cp, src, h->d_step,
                                      0, b, cpt);
                        launch_e2d<T>(st, f[FDTD_EZ], f[FDTD_HX], f[FDTD_HY], h->nx, h->ny, ce, cpe, cp, src, h->d_step,
                                      0, b, cpt);
                    } else {
                        launch_h3d<T>(st, f, h->nx, h->ny, h->nz, ch, cph, cp, src, h->d_step, 0, b, cpt);
                        launch_e3d<T>(st, f, h->nx, h->ny, h->nz, ce, cpe, cp, src, h->d_step, 0, b, cpt);
                    }
                });
                if (ms < best * kTuneMargin) {
                    best = ms;
                    out->block_x = sh[0]; out->block_y = sh[1]; out->block_z = sh[2]; out->cells_per_thread = cpt;
                }
            }
        }
        // FP32: the TMA kernels (2-D: rows per block; 3-D: planes per block)
        if constexpr (sizeof(T) == 4) {
            if (!h->tma) h->tma = tma_maps_create(f, h->nx, h->ny, h->nz);
            if (h->g.ndim == 2 && h->tma) {
                for (int rows : {32, 48, 64, 96, 128}) {
                    if (rows > 4 * h->ny) continue;
                    const double ms = time_ms([&] {
                        launch_h2d_tma(st, h->tma, f, h->nx, h->ny, ch, cph, cp, src, h->d_step, 0, rows, h->d_err);
                        launch_e2d_tma(st, h->tma, f, h->nx, h->ny, ce, cpe, cp, src, rows, h->d_err);
                    });
                    if (ms < best * kTuneMargin) {
                        best = ms;
                        out->block_x = 32; out->block_y = 8; out->block_z = 1; out->cells_per_thread = 1;
                        out->stencil_tz = rows;
                    }
                }
            }
            if (h->g.ndim == 3 && h->tma) {
                for (int tz : {8, 12, 16, 24, 32}) {
                    if (tz > 2 * h->nz) continue;
                    const double ms = time_ms([&] {
                        launch_h3d_tma(st, h->tma, f, h->nx, h->ny, h->nz, ch, cph, cp, src, h->d_step, 0, tz,
                                       h->d_err);
                        launch_e3d_tma(st, h->tma, f, h->nx, h->ny, h->nz, ce, cpe, cp, src, tz, h->d_err);
                    });
                    if (ms < best * kTuneMargin) {
                        best = ms;
                        out->block_x = 32; out->block_y = 8; out->block_z = 1; out->cells_per_thread = 1;
                        out->stencil_tz = tz;
                    }
                }
            }
        }
        // 2-D FP32 on a whole grid: the fused E + H column march (one launch a step, from this set into the
        // second) against the best separate pair
        out->fused_rows = 0;
        if constexpr (sizeof(T) == 4) {
            if (h->g.ndim == 2 && h->nx % 4 == 0 && !h->sd_on) {
                h->auto_fuse_rows = kFuseRowsDefault;   // lets ensure_second_set allocate the second set
                ensure_second_set(h);
                if (h->f2[FDTD_EZ]) {
                    float *fo[6], *po[12];
                    for (int q = 0; q < 6; ++q) fo[q] = reinterpret_cast<float *>(h->f2[q]);
                    for (int q = 0; q < 12; ++q) po[q] = reinterpret_cast<float *>(h->psi2[q]);
                    for (int rows : {4, 8, 16, 32}) {
                        const double ms = time_ms([&] {
                            launch_eh2d(st, f, fo, po, h->nx, h->ny, ce, cpe, ch, cph, cp, src, h->d_step, 0, rows);
                        });
                        if (ms < best * kTuneMargin) {
                            best = ms;
                            out->fused_rows = rows;
                        }
                    }
                }
                h->auto_fuse_rows = out->fused_rows;
                if (!h->fuse && h->auto_fuse_rows <= 0) free_second_set(h);
            }
        }
        h->st_bx = out->block_x; h->st_by = out->block_y; h->st_bz = out->block_z; h->st_cpt = out->cells_per_thread;
        h->st_tz = out->stencil_tz;
        out->stencil_ms = best;
        m[stencil_key(h)] = {out->block_x,        out->block_y,    out->block_z,
                             out->cells_per_thread, out->stencil_tz, out->fused_rows};
    }
    out->kin_vpl = out->kin_l = out->kin_blocks_per_sm = out->kin_stages = 0;
    out->kin_ms = 0;
    if (h->has_plasma && h->nkin > 0 && !h->pl.nonlinear && !h->pl.evolve_f0) {
        int cand[8][2];
        const int nc = kinetic_candidates(h->pitch, h->pl.f_dtype, cand);
        // (ring stages, CTAs per SM cap): the register kernel, then the bulk-copy ring (FP32 / BF16 rows).
        // Each candidate is timed where it runs, between the H and E stencils of whole steps (events around
        // the middle part, as fdtd_plasma_time_kernels does): timed back to back on their own, some ring
        // shapes that lose inside the step looked fastest.
        static const int variants[][2] = {{0, 0}, {0, 2}, {0, 3}, {2, 0}, {3, 0}, {4, 0}, {6, 0}};
        cudaEvent_t ev[5];
        for (int q = 0; q < 5; ++q) CK(h, cudaEventCreate(&ev[q]));
        auto time_in_step = [&](bool &bad) -> double {
            double acc = 0.0;
            for (int r = 0; r < 6 && !bad; ++r) {
                cudaError_t e = enqueue_step<T>(h, st, 0, ev, true);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    bad = true;
                    break;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[1], ev[2]);
                if (r > 0) acc += ms;   // the first step is the warm-up
            }
            return acc / 5.0;
        };
        const int keep[3] = {h->kin_vpl, h->kin_l, h->kin_bps}, keep_stages = h->kin_stages;
        // the timing steps leave no trace outside the saved state: no port spectra, no recorded samples
        const int keep_ports = h->nports, keep_rec = h->has_recording;
        h->nports = 0;
        h->has_recording = 0;
        double best = 1e30;
        for (int c = 0; c < nc; ++c)
            for (const auto &vr : variants) {
                if (vr[0] > 0 && (h->pl.f_dtype == FDTD_DF_F64 || !kinetic_ring_fits(h->pitch, h->pl.f_dtype,
                                                                                       cand[c][1], vr[0])))
                    continue;
                bool bad = false;
                h->kin_vpl = cand[c][0]; h->kin_l = cand[c][1]; h->kin_bps = vr[1]; h->kin_stages = vr[0];
                const double ms = time_in_step(bad);
                if (!bad && ms < best * kTuneMargin) {
                    best = ms;
                    out->kin_vpl = cand[c][0]; out->kin_l = cand[c][1]; out->kin_blocks_per_sm = vr[1];
                    out->kin_stages = vr[0];
                }
            }
        for (int q = 0; q < 5; ++q) cudaEventDestroy(ev[q]);
        h->nports = keep_ports;
        h->has_recording = keep_rec;
        if (best >= 1e30) {   // nothing ran: keep the shape in use
            out->kin_vpl = keep[0]; out->kin_l = keep[1]; out->kin_blocks_per_sm = keep[2];
            out->kin_stages = keep_stages;
        }
        h->kin_vpl = out->kin_vpl; h->kin_l = out->kin_l; h->kin_bps = out->kin_blocks_per_sm;
        h->kin_stages = out->kin_stages;
        out->kin_ms = best;
        m[kin_key(h)] = {out->kin_vpl, out->kin_l, out->kin_blocks_per_sm, out->kin_stages};
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(h, cudaGetLastError());
    write_cache(m);
    return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_plasma_autotune(fdtd_plasma_t h, fdtd_tune_result *out)
{
    NvtxRange nvtx_("fdtd_plasma_autotune");
    if (!h || !out) return FDTD_ERR_INVAL;
    // the candidates run on the live buffers: save the state and restore it bit for bit afterwards
    const size_t nb = fdtd_plasma_state_bytes(h);
    void *blob = dalloc(h, nb);
    if (!blob) return fail(h, FDTD_ERR_NOMEM, "autotune: no room for the state copy (%zu bytes)", nb);
    int rc = fdtd_plasma_save_state(h, blob, nb, 1);
    const int64_t steps = h->steps_done;
    if (rc == FDTD_OK) rc = h->g.precision == FDTD_F64 ? autotune_t<double>(h, out) : autotune_t<float>(h, out);
    const int rc2 = fdtd_plasma_load_state(h, blob, nb, 1);
    h->steps_done = steps;
    dfree(h, blob);
    drop_graphs(h);
    return rc != FDTD_OK ? rc : rc2;
}

int fdtd_plasma_time_kernels(fdtd_plasma_t h, int64_t nsteps, double *ms_out)
{
    NvtxRange nvtx_("fdtd_plasma_time_kernels");
    if (!h || !ms_out || nsteps < 1) return FDTD_ERR_INVAL;
    cudaEvent_t ev[5];
    for (int q = 0; q < 5; ++q) CK(h, cudaEventCreate(&ev[q]));
    double acc[5] = {0, 0, 0, 0, 0};
    int rc = FDTD_OK;
    for (int64_t s = 0; s < nsteps && rc == FDTD_OK; ++s) {
        const bool last = s == nsteps - 1;   // J stored on the last step, as in a step sequence
        cudaError_t e = h->g.precision == FDTD_F64 ? enqueue_step<double>(h, h->stream, 0, ev, last)
                                                   : enqueue_step<float>(h, h->stream, 0, ev, last);
        if (e == cudaSuccess) {
            launch_advance(h->stream, h->d_step, 1);
            e = cudaEventSynchronize(ev[4]);
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e, "timed step");
            break;
        }
        float ms;
        for (int q = 0; q < 4; ++q) {
            cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
            acc[q] += ms;
        }
        cudaEventElapsedTime(&ms, ev[0], ev[4]);
        acc[4] += ms;
        h->steps_done += 1;
    }
    for (int q = 0; q < 5; ++q) cudaEventDestroy(ev[q]);
    if (rc != FDTD_OK) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    for (int q = 0; q < 5; ++q) ms_out[q] = acc[q] / (double)nsteps;
    return FDTD_OK;
}

size_t fdtd_plasma_quantity_bytes(fdtd_plasma_t h, int which)
{
    if (!h) return 0;
    if (which >= 0 && which <= 5) return field_bytes(h, which);
    if (which == FDTD_J) return h->has_plasma ? (size_t)h->nslots * h->esz : 0;
    if (which == FDTD_DF) return h->has_plasma ? (size_t)h->nkin * h->nnode * h->df_esz : 0;
    if (which == FDTD_F0) return h->has_plasma && h->g0 ? (size_t)h->nkin * h->nnode * h->df_esz : 0;
    return 0;
}

// the device error word: bit 1 closure tensor-core waits, bit 2 TMA stencil waits
static const char *wait_error_text(int errw)
{
    if (errw & 2) return "a bounded device wait gave up (TMA stencil kernel)";
    return "a bounded device wait gave up (closure kernel)";
}

static int copy_quantity(fdtd_plasma_t h, int which, void *host_or_dev, size_t bytes, int is_device, bool out)
{
    if (!h || !host_or_dev) return FDTD_ERR_INVAL;
    const size_t need = fdtd_plasma_quantity_bytes(h, which);
    if (need == 0) return fail(h, FDTD_ERR_INVAL, "quantity %d is absent", which);
    if (bytes != need) return fail(h, FDTD_ERR_INVAL, "quantity %d needs %zu bytes, got %zu", which, need, bytes);
    const cudaMemcpyKind kind = out ? (is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                                    : (is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (which == FDTD_DF || which == FDTD_F0) {
        void *rows = which == FDTD_DF ? h->df : h->g0;
        const size_t row = (size_t)h->nnode * h->df_esz, dpitch = (size_t)h->pitch * h->df_esz;
        if (out)
            CK(h, cudaMemcpy2DAsync(host_or_dev, row, rows, dpitch, row, h->nkin, kind, h->stream));
        else
            CK(h, cudaMemcpy2DAsync(rows, dpitch, host_or_dev, row, row, h->nkin, kind, h->stream));
    } else {
        void *dev = which == FDTD_J ? h->jslot : h->f[which];
        if (out) CK(h, cudaMemcpyAsync(host_or_dev, dev, bytes, kind, h->stream));
        else CK(h, cudaMemcpyAsync(dev, host_or_dev, bytes, kind, h->stream));
    }
    if (!is_device) {
        int errw = 0;
        if (out) CK(h, cudaMemcpyAsync(&errw, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (errw) return fail(h, FDTD_ERR_TIMEOUT, "%s", wait_error_text(errw));
    }
    return FDTD_OK;
}

int fdtd_plasma_read_fields(fdtd_plasma_t h, int which, void *dst, size_t bytes, int dst_is_device)
{
    NvtxRange nvtx_("fdtd_plasma_read_fields");
    return copy_quantity(h, which, dst, bytes, dst_is_device, true);
}

int fdtd_plasma_write_fields(fdtd_plasma_t h, int which, const void *src, size_t bytes, int src_is_device)
{
    NvtxRange nvtx_("fdtd_plasma_write_fields");
    if (h && which == FDTD_J) return fail(h, FDTD_ERR_INVAL, "J is not writable");
    return copy_quantity(h, which, const_cast<void *>(src), bytes, src_is_device, false);
}

int fdtd_plasma_plasma_shape(fdtd_plasma_t h, int64_t *nslots, int64_t *nnode)
{
    if (!h) return FDTD_ERR_INVAL;
    if (nslots) *nslots = h->nslots;
    if (nnode) *nnode = h->nnode;
    return FDTD_OK;
}

int fdtd_plasma_info(fdtd_plasma_t h, double *dt, int64_t *steps)
{
    if (!h) return FDTD_ERR_INVAL;
    if (dt) *dt = h->dt;
    if (steps) *steps = h->steps_done;
    return FDTD_OK;
}

int fdtd_plasma_diagnostics(fdtd_plasma_t h, fdtd_diag *out)
{
    NvtxRange nvtx_("fdtd_plasma_diagnostics");
    if (!h || !out) return FDTD_ERR_INVAL;
    const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
    DiagArgs a{};
    a.ndim = h->g.ndim;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    for (int q = 0; q < 6; ++q) { a.f[q] = h->f[q]; a.flen[q] = h->flen[q]; }
    a.precision = h->g.precision;
    a.ch = h->dt / (mu0 * h->g.dx);
    const double dv = std::pow(h->g.dx, h->g.ndim);
    a.eps0_half_dv = 0.5 * kEps0 * dv;
    a.mu0_half_dv = 0.5 * mu0 * dv;
    a.df = h->df;
    a.nslots = h->has_plasma ? h->nkin : 0;
    a.nnode = h->nnode;
    a.pitch = h->pitch;
    a.f_dtype = h->pl.f_dtype;
    a.dV = h->dV;
    CK(h, launch_diag(h->stream, a, h->diag_partials, h->diag_blocks, h->diag_out));
    double o[6];
    CK(h, cudaMemcpyAsync(o, h->diag_out, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    int errw = 0;
    CK(h, cudaMemcpyAsync(&errw, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (errw) return fail(h, FDTD_ERR_TIMEOUT, "%s", wait_error_text(errw));
    out->energy = o[0];
    out->energy_plain = o[1];
    out->number = o[2];
    out->number_max_cell = o[3];
    out->number_abs = o[4];
    out->finite = o[5] > 0.5 ? 1 : 0;
    out->step = h->steps_done;
    return FDTD_OK;
}

void free_ports(fdtd_plasma *h)
{
    dfree(h, h->port_off); dfree(h, h->port_cells); dfree(h, h->port_freq); dfree(h, h->port_acc);
    h->port_off = h->port_cells = nullptr;
    h->port_freq = h->port_acc = nullptr;
    h->nports = h->nfreq = 0;
}

int fdtd_plasma_set_ports(fdtd_plasma_t h, int32_t nports, const int64_t *port_offsets, const int64_t *cells,
                          int32_t nfreq, const double *freqs)
{
    NvtxRange nvtx_("fdtd_plasma_set_ports");
    if (!h) return FDTD_ERR_INVAL;
    if (h->sd_on && nports) return fail(h, FDTD_ERR_STATE, "ports run on whole grids, not on sub-domains");
    if (nports == 0) {
        drop_graphs(h);
        free_ports(h);
        return FDTD_OK;
    }
    if (nports < 0 || nports > 4096 || nfreq < 1 || nfreq > (1 << 20) || !port_offsets || !cells || !freqs)
        return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_set_ports: bad counts or NULL array");
    if (port_offsets[0] != 0) return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_set_ports: port_offsets[0] must be 0");
    const int64_t np = pol_len(h);
    for (int p = 0; p < nports; ++p)
        if (!(port_offsets[p + 1] > port_offsets[p]))
            return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_set_ports: port %d has no nodes", p);
    const int64_t ncell = port_offsets[nports];
    for (int64_t q = 0; q < ncell; ++q)
        if (cells[q] < 0 || cells[q] >= np)
            return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_set_ports: node %lld outside the polarisation field",
                        (long long)cells[q]);
    for (int f = 0; f < nfreq; ++f)
        if (!std::isfinite(freqs[f])) return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_set_ports: non-finite frequency");
    drop_graphs(h);
    free_ports(h);
    h->port_off = (int64_t *)dalloc(h, (nports + 1) * sizeof(int64_t));
    h->port_cells = (int64_t *)dalloc(h, ncell * sizeof(int64_t));
    h->port_freq = (double *)dalloc(h, nfreq * sizeof(double));
    h->port_acc = (double *)dalloc(h, (size_t)nports * nfreq * 2 * sizeof(double));
    if (!h->port_off || !h->port_cells || !h->port_freq || !h->port_acc) {
        free_ports(h);
        return fail(h, FDTD_ERR_NOMEM, "fdtd_plasma_set_ports: allocation failed");
    }
    CK(h, cudaMemcpyAsync(h->port_off, port_offsets, (nports + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaMemcpyAsync(h->port_cells, cells, ncell * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->port_freq, freqs, nfreq * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemsetAsync(h->port_acc, 0, (size_t)nports * nfreq * 2 * sizeof(double), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));   // the host arrays may go away after return
    h->nports = nports;
    h->nfreq = nfreq;
    return FDTD_OK;
}

int fdtd_plasma_read_ports(fdtd_plasma_t h, double *out, size_t bytes)
{
    NvtxRange nvtx_("fdtd_plasma_read_ports");
    if (!h || !out) return FDTD_ERR_INVAL;
    const size_t need = (size_t)h->nports * h->nfreq * 2 * sizeof(double);
    if (h->nports == 0) return fail(h, FDTD_ERR_STATE, "fdtd_plasma_read_ports: no ports set");
    if (bytes != need) return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_read_ports: need %zu bytes", need);
    CK(h, cudaMemcpyAsync(out, h->port_acc, need, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

int fdtd_plasma_poynting(fdtd_plasma_t h, const int64_t *box, double *out)
{
    NvtxRange nvtx_("fdtd_plasma_poynting");
    if (!h || !box || !out) return FDTD_ERR_INVAL;
    const int nd = h->g.ndim;
    // E-node extent per axis; axes a 1-D or 2-D grid does not have are ignored
    const int64_t ne[3] = {nd == 1 ? 1 : h->nx, nd == 1 ? 1 : h->ny, nd == 1 ? h->nz + 1 : nd == 2 ? 1 : h->nz};
    const bool used[3] = {nd >= 2, nd >= 2, nd != 2};
    PoyntingBox b{};
    for (int ax = 0; ax < 3; ++ax) {
        b.lo[ax] = used[ax] ? box[2 * ax] : 0;
        b.hi[ax] = used[ax] ? box[2 * ax + 1] : 0;
        if (used[ax] && !(0 <= b.lo[ax] && b.lo[ax] <= b.hi[ax] && b.hi[ax] < ne[ax]))
            return fail(h, FDTD_ERR_INVAL, "fdtd_plasma_poynting: box faces must satisfy 0 <= lo <= hi < E nodes");
        b.plane[2 * ax] = b.lo[ax];
        b.plane[2 * ax + 1] = b.hi[ax];
    }
    b.off[0] = 0;
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1;
        int64_t np = 0;
        if (nd == 1) np = ax == 2 ? 1 : 0;
        else if (nd == 2) np = ax == 2 ? 0 : (ax == 0 ? b.hi[1] - b.lo[1] : b.hi[0] - b.lo[0]);
        else {
            const int u = ax == 0 ? 1 : 0, w = ax == 2 ? 1 : 2;
            np = (b.hi[u] - b.lo[u]) * (b.hi[w] - b.lo[w]);
        }
        b.off[f + 1] = b.off[f] + np;
    }
    const double mu0 = 1.0 / (kEps0 * kC0 * kC0);
    DiagArgs a{};
    a.ndim = nd;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    for (int q = 0; q < 6; ++q) { a.f[q] = h->f[q]; a.flen[q] = h->flen[q]; }
    a.precision = h->g.precision;
    a.ch = h->dt / (mu0 * h->g.dx);
    const double dA = nd == 3 ? h->g.dx * h->g.dx : nd == 2 ? h->g.dx : 1.0;
    CK(h, launch_poynting(h->stream, a, b, dA, h->diag_partials, h->diag_blocks, h->diag_out));
    CK(h, cudaMemcpyAsync(out, h->diag_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

// ------------------------------------------------------------ checkpoints
// blob: 8 x uint64 header, then fields, psi, df (raw rows), J, mur state, step

static size_t state_parts(fdtd_plasma_t h, std::vector<std::pair<void *, size_t>> &parts)
{
    parts.clear();
    for (int q = 0; q < 6; ++q)
        if (h->f[q]) parts.push_back({h->f[q], field_bytes(h, q)});
    for (int q = 0; q < 12; ++q)
        if (h->psi[q]) parts.push_back({h->psi[q], (size_t)h->psilen[q] * h->esz});
    if (h->has_plasma && h->nslots) {
        if (h->nkin) parts.push_back({h->df, (size_t)h->nkin * h->pitch * h->df_esz});
        if (h->nkin && h->g0) parts.push_back({h->g0, (size_t)h->nkin * h->pitch * h->df_esz});
        parts.push_back({h->jslot, (size_t)h->nslots * h->esz});
    }
    const int64_t nh = h->has_closure ? h->ncl : (h->has_recording ? h->nslots : 0);
    if (nh && h->hist) {
        parts.push_back({h->hist, (size_t)nh * 16 * 4});
        parts.push_back({h->jprev, (size_t)nh * 4});
    }
    parts.push_back({h->mur_state, 32});
    parts.push_back({h->d_step, sizeof(int64_t)});
    size_t tot = 64;
    for (auto &p : parts) tot += p.second;
    return tot;
}

size_t fdtd_plasma_state_bytes(fdtd_plasma_t h)
{
    if (!h) return 0;
    std::vector<std::pair<void *, size_t>> parts;
    return state_parts(h, parts);
}

int fdtd_plasma_save_state(fdtd_plasma_t h, void *buf, size_t bytes, int dev)
{
    NvtxRange nvtx_("fdtd_plasma_save_state");
    if (!h || !buf) return FDTD_ERR_INVAL;
    std::vector<std::pair<void *, size_t>> parts;
    const size_t need = state_parts(h, parts);
    if (bytes != need) return fail(h, FDTD_ERR_INVAL, "state needs %zu bytes, got %zu", need, bytes);
    uint64_t hdr[8] = {kStateMagic, (uint64_t)h->g.ndim, (uint64_t)(h->nx * h->ny * h->nz), (uint64_t)h->nslots,
                       (uint64_t)h->pitch, (uint64_t)h->df_esz, (uint64_t)h->esz, (uint64_t)h->steps_done};
    const cudaMemcpyKind k_out = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(h, cudaMemcpyAsync(buf, hdr, 64, dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, h->stream));
    size_t off = 64;
    for (auto &p : parts) {
        CK(h, cudaMemcpyAsync((char *)buf + off, p.first, p.second, k_out, h->stream));
        off += p.second;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

int fdtd_plasma_load_state(fdtd_plasma_t h, const void *buf, size_t bytes, int dev)
{
    NvtxRange nvtx_("fdtd_plasma_load_state");
    if (!h || !buf) return FDTD_ERR_INVAL;
    std::vector<std::pair<void *, size_t>> parts;
    const size_t need = state_parts(h, parts);
    if (bytes != need) return fail(h, FDTD_ERR_INVAL, "state needs %zu bytes, got %zu", need, bytes);
    uint64_t hdr[8];
    CK(h, cudaMemcpy(hdr, buf, 64, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    if (hdr[0] != kStateMagic || hdr[1] != (uint64_t)h->g.ndim || hdr[2] != (uint64_t)(h->nx * h->ny * h->nz) ||
        hdr[3] != (uint64_t)h->nslots || hdr[4] != (uint64_t)h->pitch || hdr[5] != (uint64_t)h->df_esz ||
        hdr[6] != (uint64_t)h->esz)
        return fail(h, FDTD_ERR_STATE, "state blob does not match this handle's configuration");
    const cudaMemcpyKind k_in = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = 64;
    for (auto &p : parts) {
        CK(h, cudaMemcpyAsync(p.first, (const char *)buf + off, p.second, k_in, h->stream));
        off += p.second;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->steps_done = (int64_t)hdr[7];
    return FDTD_OK;
}

const char *fdtd_plasma_last_error(fdtd_plasma_t h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

void fdtd_plasma_destroy(fdtd_plasma_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    free_plasma(h);
    for (int q = 0; q < 6; ++q) dfree(h, h->f[q]);
    for (int q = 0; q < 12; ++q) dfree(h, h->psi[q]);
    dfree(h, h->prof);
    dfree(h, h->mur_state);
    dfree(h, h->d_step);
    dfree(h, h->d_src);
    dfree(h, h->d_err);
    free_ports(h);
    free_second_set(h);
    tma_maps_free(h->tma);
    dfree(h, h->diag_partials);
    dfree(h, h->diag_out);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

}  // extern "C"

// compact.cu -- the plasma cells of a density array on the GPU: the
// polarisation nodes with density > 0 whose E the curl updates (PEC and Mur
// end nodes never carry plasma), in increasing node index, with their
// densities; also the largest density and whether every value is finite and
// >= 0.  Two passes over fixed chunks of the array: per chunk a count and a
// maximum, then (after the host's exclusive scan of the counts) per chunk an
// in-order scatter -- the same slot list the host loop over the array gives.
#include "internal.cuh"

namespace fp {

constexpr int kCompactThreads = 256;

__device__ __forceinline__ bool compact_updated(const CompactGeom &g, int64_t c)
{
    if (g.ndim == 1) return c >= 1 && c <= g.nz - 1;
    const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    if (g.ndim == 2) return i >= 1 && j >= 1;
    return j >= 1 && k >= 1;
}

__global__ void __launch_bounds__(kCompactThreads) k_compact_count(const double *__restrict__ d, CompactGeom g,
                                                                   int *__restrict__ counts,
                                                                   double *__restrict__ maxes, int *__restrict__ bad)
{
    __shared__ int sc[kCompactThreads / 32];
    __shared__ double sm[kCompactThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kCompactChunk, c1 = min(c0 + kCompactChunk, g.n);
    int cnt = 0, b = 0;
    double mx = 0.0;
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const double v = d[c];
        if (!isfinite(v) || v < 0.0) b = 1;
        if (v > 0.0 && compact_updated(g, c)) {
            ++cnt;
            mx = fmax(mx, v);
        }
    }
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    b = __any_sync(0xffffffffu, b);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sc[w] = cnt;
        sm[w] = mx;
        if (b) atomicOr(bad, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        double m = 0.0;
        for (int q = 0; q < kCompactThreads / 32; ++q) {
            t += sc[q];
            m = fmax(m, sm[q]);
        }
        counts[blockIdx.x] = t;
        maxes[blockIdx.x] = m;
    }
}

// chunk b writes its plasma cells, in index order, from slot offsets[b] on
__global__ void __launch_bounds__(kCompactThreads) k_compact_scatter(const double *__restrict__ d, CompactGeom g,
                                                                     const int64_t *__restrict__ offsets,
                                                                     int32_t *__restrict__ cells,
                                                                     double *__restrict__ dens)
{
    __shared__ int sw[kCompactThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kCompactChunk, c1 = min(c0 + kCompactChunk, g.n);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t base = offsets[blockIdx.x];
    for (int64_t r0 = c0; r0 < c1; r0 += blockDim.x) {
        const int64_t c = r0 + threadIdx.x;
        double v = 0.0;
        bool on = false;
        if (c < c1) {
            v = d[c];
            on = v > 0.0 && compact_updated(g, c);
        }
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) sw[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < kCompactThreads / 32; ++q) {
            before += q < w ? sw[q] : 0;
            total += sw[q];
        }
        if (on) {
            const int64_t s = base + before + __popc(m & ((1u << lane) - 1u));
            cells[s] = (int32_t)c;
            dens[s] = v;
        }
        base += total;
        __syncthreads();
    }
}

cudaError_t launch_compact_count(cudaStream_t st, const double *d, const CompactGeom &g, int *counts, double *maxes,
                                 int *bad)
{
    const int64_t nb = (g.n + kCompactChunk - 1) / kCompactChunk;
    if (nb > 0) k_compact_count<<<(unsigned)nb, kCompactThreads, 0, st>>>(d, g, counts, maxes, bad);
    return cudaGetLastError();
}

cudaError_t launch_compact_scatter(cudaStream_t st, const double *d, const CompactGeom &g, const int64_t *offsets,
                                   int32_t *cells, double *dens)
{
    const int64_t nb = (g.n + kCompactChunk - 1) / kCompactChunk;
    if (nb > 0) k_compact_scatter<<<(unsigned)nb, kCompactThreads, 0, st>>>(d, g, offsets, cells, dens);
    return cudaGetLastError();
}

__global__ void k_to_f32(const double *__restrict__ src, float *__restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

cudaError_t launch_to_f32(cudaStream_t st, const double *src, float *dst, int64_t n)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_to_f32<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace fp

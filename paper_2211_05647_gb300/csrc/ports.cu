// ports.cu -- running-DFT port probes (Sec. 5.3: the slab's S-parameters come
// from spectra of the field at two ports).  Once per step, after the E update,
// each port's polarisation field E^{n+1} is averaged over its nodes and added
// into X[p][f] += E_p(t) exp(-i 2 pi f t) dt, t = t^{n+1}, in FP64.
// One block per port: the block reduces the port's nodes, then its threads
// stride over the frequencies.
#include "internal.cuh"

namespace fp {

template <typename T>
__global__ void __launch_bounds__(256) k_ports(const T *__restrict__ pol, const int64_t *__restrict__ off,
                                               const int64_t *__restrict__ cells, const double *__restrict__ freq,
                                               double *__restrict__ acc, int nfreq, double dt,
                                               const int64_t *__restrict__ d_step, int kstep)
{
    pdl_enter();
    __shared__ double red[8];
    __shared__ double mean_dt;
    const int p = blockIdx.x;
    const int64_t b = off[p], e = off[p + 1];
    double s = 0.0;
    for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) s += (double)pol[cells[q]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        mean_dt = t / (double)(e - b) * dt;
    }
    __syncthreads();
    const double tn = (double)(*d_step + kstep + 1) * dt;
    double *a = acc + (int64_t)p * nfreq * 2;
    for (int f = threadIdx.x; f < nfreq; f += blockDim.x) {
        double sn, cs;
        sincos(2.0 * kPi * freq[f] * tn, &sn, &cs);
        a[2 * f] += mean_dt * cs;
        a[2 * f + 1] -= mean_dt * sn;
    }
}

template <typename T>
cudaError_t launch_ports(cudaStream_t st, const T *pol, int nports, const int64_t *off, const int64_t *cells,
                         const double *freq, double *acc, int nfreq, double dt, const int64_t *d_step, int kstep)
{
    launch_pdl(k_ports<T>, dim3(nports), dim3(256), 0, st, pol, off, cells, freq, acc, nfreq, dt, d_step, kstep);
    return cudaGetLastError();
}

template cudaError_t launch_ports<float>(cudaStream_t, const float *, int, const int64_t *, const int64_t *,
                                         const double *, double *, int, double, const int64_t *, int);
template cudaError_t launch_ports<double>(cudaStream_t, const double *, int, const int64_t *, const int64_t *,
                                          const double *, double *, int, double, const int64_t *, int);

}  // namespace fp

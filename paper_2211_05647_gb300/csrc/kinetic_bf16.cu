// kinetic_bf16.cu -- BF16-storage instances of the plasma-row kernel (FP32
// arithmetic, stochastic rounding on store); see kinetic_impl.cuh.
#include "kinetic_impl.cuh"

namespace fp {

cudaError_t dispatch_kinetic_bf16(cudaStream_t st, const KinArgs<float> &a, int num_sms, int vpl, int l, int bps)
{
    return dispatch_kinetic<__nv_bfloat16, float>(st, a, num_sms, vpl, l, bps);
}

}  // namespace fp

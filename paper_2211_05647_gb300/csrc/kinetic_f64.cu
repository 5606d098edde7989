// kinetic_f64.cu -- FP64 instances of the plasma-row kernel (the validation
// instantiation); see kinetic_impl.cuh.
#include "kinetic_impl.cuh"

namespace fp {

cudaError_t dispatch_kinetic_f64(cudaStream_t st, const KinArgs<double> &a, int num_sms, int vpl, int l, int bps)
{
    return dispatch_kinetic<double, double>(st, a, num_sms, vpl, l, bps);
}

}  // namespace fp

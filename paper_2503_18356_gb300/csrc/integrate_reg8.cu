// Register-resident FP32 integrator, node bucket N <= 8.
#include "integrate.cuh"

namespace grins {

cudaError_t launch_integrate_fp32_reg8(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    return launch_reg_bucket<8>(a, st, num_sms);
}

}  // namespace grins

// Register-resident FP32 integrator, node bucket N <= 16.
#include "integrate.cuh"

namespace grins {

cudaError_t launch_integrate_fp32_reg16(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    return launch_reg_bucket<16>(a, st, num_sms);
}

}  // namespace grins

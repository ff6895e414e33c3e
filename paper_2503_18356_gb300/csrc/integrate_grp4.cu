// Lane-group FP32 integrator, up to 4 node rows per lane.
#include "integrate_grp.cuh"

namespace grins {

cudaError_t launch_integrate_grp4(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    return launch_grp_bucket<4, GRINS_GRP_MINB>(a, st, num_sms);
}

}  // namespace grins

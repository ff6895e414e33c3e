// Lane-group FP32 integrator, up to 8 node rows per lane.
#include "integrate_grp.cuh"

namespace grins {

cudaError_t launch_integrate_grp8(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    return launch_grp_bucket<8, GRINS_GRP_MINB>(a, st, num_sms);
}

}  // namespace grins

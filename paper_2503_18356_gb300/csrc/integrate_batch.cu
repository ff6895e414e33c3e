// Batched lane-group FP32 integrator: many networks in one launch.
#include "integrate_grp.cuh"

namespace grins {

namespace {

template <int WARPS, int MINB>
cudaError_t launch_batch_warps(const BatchArgs &b, cudaStream_t st, int num_sms, int smem_limit)
{
    auto kern = dp5_grp_batch_kernel<8, WARPS, MINB>;
    const int region = b.warp_bytes + (int)((sizeof(IntegrateArgs) + 127) / 128 * 128);
    const int smem = WARPS * region;
    if (smem > smem_limit) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)(num_sms * per_sm), WARPS * kWarp, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_integrate_batch(const BatchArgs &b, int warps, cudaStream_t st, int num_sms, int smem_limit)
{
    if (b.n_jobs <= 0) return cudaSuccess;
    if (warps == 2) return launch_batch_warps<2, 6>(b, st, num_sms, smem_limit);
    return launch_batch_warps<4, 3>(b, st, num_sms, smem_limit);
}

}  // namespace grins

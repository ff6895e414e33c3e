// The job loop of a plan's compiled launch (PlanArgs): each warp starts on
// the job where its SM's share of the total work falls, then visits every
// job in turn; for each, it copies the job's arguments into its shared-memory
// region (the integrator reads them with broadcast loads) and, unless the
// job's solves are all handed out, runs the job's body, which integrates
// solves from the job's counter until none is left.  `call(body, args,
// wbase)` runs body `body` (a switch over the plan's compiled bodies).
#pragma once

#include "common.cuh"

namespace grins {

template <typename F>
__device__ __forceinline__ void plan_run(const PlanArgs &p, F &&call)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = (int)(blockDim.x >> 5);
    unsigned char *wbase = smem + warp * p.region_bytes;
    IntegrateArgs *ja = reinterpret_cast<IntegrateArgs *>(wbase + p.gather_bytes);
    // every warp of an SM starts on the same job and visits the jobs in the
    // same order, so the warps sharing an SM's instruction cache mostly run
    // one body at a time (the bodies are long straight-line code)
    unsigned smid = 0, nsm = 1;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
    (void)W;
    const double share = ((double)smid + 0.5) / (double)(nsm > 0 ? nsm : 1);
    int b0 = 0;
    while (b0 + 1 < p.n_jobs && p.cum_work[b0] <= share) ++b0;
#pragma unroll 1
    for (int k = 0; k < p.n_jobs; ++k) {
        const int jb = (b0 + k) % p.n_jobs;
        const unsigned *src = reinterpret_cast<const unsigned *>(p.jobs + jb);
        unsigned *dst = reinterpret_cast<unsigned *>(ja);
        for (int i = lane; i < (int)(sizeof(IntegrateArgs) / 4); i += kWarp) dst[i] = src[i];
        __syncwarp();
        // one warp-uniform decision: skip a job whose solves are all handed out
        unsigned long long q = 0;
        if (lane == 0) q = *reinterpret_cast<volatile unsigned long long *>(ja->queue);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q < (unsigned long long)(ja->n_sets * (long long)ja->n_ics)) call(p.body_of[jb], *ja, wbase);
        __syncwarp();
    }
}

}  // namespace grins

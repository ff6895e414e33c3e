// Order of the borderline re-pass (see IntegrateArgs::tail_items): the
// solves the FP32 pass listed are re-integrated (double-float or FP64) from their
// checkpoints, and their lengths differ widely -- a checkpoint taken early
// leaves a long stretch to t_end.  Handing them out longest first
// (longest-processing-time-first scheduling) lets the long ones start while
// the many short ones fill the gaps, so the re-pass launch does not end on a
// few long solves running alone.  The length is estimated by the attempts
// the FP32 pass took after the checkpoint, in 64 buckets (a counting sort;
// the order within a bucket is arbitrary, and each solve's result is
// independent of it).
#include "common.cuh"

namespace grins {

namespace {

constexpr int kTailBuckets = 64;

__global__ void __launch_bounds__(1024) tail_order_kernel(const IntegrateArgs::TailItem *in,
                                                          IntegrateArgs::TailItem *out,
                                                          const unsigned long long *n_in, long long cap,
                                                          int max_work)
{
    __shared__ unsigned long long cnt[kTailBuckets], pos[kTailBuckets];
    const unsigned long long listed = *n_in;
    const long long n = listed < (unsigned long long)cap ? (long long)listed : cap;
    for (int b = threadIdx.x; b < kTailBuckets; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int width = max_work / kTailBuckets + 1;
    auto bucket = [&](int w) {
        const int b = w / width;
        return b < 0 ? 0 : (b >= kTailBuckets ? kTailBuckets - 1 : b);
    };
    // warp-aggregated counting: the lanes of a warp with the same bucket
    // (__match_any_sync) take their slots with one atomic (whole warps step
    // through the list together, so every lane reaches the match)
    const int lane = threadIdx.x & 31;
    const long long wbase = threadIdx.x - lane;
    for (long long i0 = wbase; i0 < n; i0 += blockDim.x) {
        const long long i = i0 + lane;
        const int b = i < n ? bucket(in[i].work) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        if (b >= 0 && lane == __ffs(grp) - 1) atomicAdd(&cnt[b], (unsigned long long)__popc(grp));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int b = kTailBuckets - 1; b >= 0; --b) { pos[b] = s; s += cnt[b]; }
    }
    __syncthreads();
    for (long long i0 = wbase; i0 < n; i0 += blockDim.x) {
        const long long i = i0 + lane;
        IntegrateArgs::TailItem it{};
        int b = -1;
        if (i < n) { it = in[i]; b = bucket(it.work); }
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(grp) - 1;
        unsigned long long base = 0;
        if (b >= 0 && lane == leader) base = atomicAdd(&pos[b], (unsigned long long)__popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        const unsigned long long p = base + __popc(grp & ((1u << lane) - 1u));
        if (b >= 0 && p < (unsigned long long)n) out[p] = it;
    }
}

}  // namespace

cudaError_t launch_tail_order(const IntegrateArgs::TailItem *in, IntegrateArgs::TailItem *out,
                              const unsigned long long *n_in, long long cap, int max_work, cudaStream_t st)
{
    tail_order_kernel<<<1, 1024, 0, st>>>(in, out, n_in, cap, max_work);
    return cudaGetLastError();
}

}  // namespace grins

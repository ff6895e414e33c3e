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
    for (long long i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[bucket(in[i].work)], 1ull);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int b = kTailBuckets - 1; b >= 0; --b) { pos[b] = s; s += cnt[b]; }
    }
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const IntegrateArgs::TailItem it = in[i];
        const unsigned long long p = atomicAdd(&pos[bucket(it.work)], 1ull);
        if (p < (unsigned long long)n) out[p] = it;
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

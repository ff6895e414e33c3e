// Issue-rate probe of the arithmetic units the kernels of this library are
// bound by: the special-function unit (ex2.approx, lg2.approx, rcp.approx,
// the operations of the FP32 integrator's edge terms, node logarithms and
// divisions), the FP32 fused multiply-add and the FP64 multiply-add,
// multiply and add (polish, dedupe, the plain FP64 solver and the FP64 form
// of the re-pass).  The rates, in operations per clock
// per SM, are the denominators of the integrator's and the FP64 kernels'
// rooflines on the device the library runs on.
//
// Method: one block of 1024 threads per SM (its dynamic shared memory
// request leaves no room for a second), each thread running independent
// chains of the operation under test for a fixed count (8 chains; 16 for the
// FMAs: the FP64 FMA's latency is long, and the compiler issues pairs of
// independent FP32 FMAs as one packed f32x2 instruction, so the FP32 rate
// counts lane operations of packed code); the block reads the SM clock (clock64)
// after a barrier before and after the loop.  A block's rate = its threads x
// chains x iterations / its clock delta; the probe reports the median over
// blocks.  Each chain step is one operation of the kind under test plus, for
// the special functions, at most one FP32 add that keeps the chain's values
// finite (the add goes to the FMA pipe, which has eight times the
// special-function unit's throughput, so it does not bound the loop).  The
// FP32 FMA loop is unrolled fourfold so that the loop counter and branch
// (3 instructions per pass) take under 5 % of the issue slots.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace grins {
namespace {

constexpr int kRateThreads = 1024;
constexpr int kRateIters = 2048;

template <int OP> struct RateShape {
    static constexpr int chains = OP >= 3 ? 16 : 8;   // the FMAs and the FP64 operations
    static constexpr int unroll = OP == 3 ? 4 : 1;
};

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_lg2(float x)
{
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_rcp(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// OP: 0 ex2, 1 lg2, 2 rcp, 3 FP32 FMA, 4 FP64 FMA, 5 FP64 multiply, 6 FP64 add.  cycles[b] <- block b's
// clock delta; sink[b] <- a value depending on every chain (keeps the loop).
template <int OP>
__global__ void __launch_bounds__(kRateThreads) rate_kernel(long long *cycles, double *sink, int n_blocks)
{
    constexpr int CH = RateShape<OP>::chains;
    const int b = blockIdx.x;
    float f[CH];
    double d[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        f[c] = 0.25f + 0.01f * (float)((threadIdx.x + c) & 15);
        d[c] = (double)f[c];
    }
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll RateShape<OP>::unroll
    for (int i = 0; i < kRateIters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if constexpr (OP == 0) f[c] = mufu_ex2(-f[c]);                  // stays in (0.5, 1]
            else if constexpr (OP == 1) f[c] = mufu_lg2(f[c] + 1.5f);       // stays in (0.58, 1.6)
            else if constexpr (OP == 2) f[c] = mufu_rcp(f[c] + 1.0f);       // stays in (0.5, 1)
            else if constexpr (OP == 3) f[c] = fmaf(f[c], 0.999f, 0.001f);  // fixed point 1
            else if constexpr (OP == 4) d[c] = fma(d[c], 0.999, 0.001);
            else if constexpr (OP == 5) d[c] = __dmul_rn(d[c], 0.999999);   // decays slowly, stays normal
            else d[c] = __dadd_rn(d[c], 1e-9);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += (OP >= 4) ? d[c] : (double)f[c];
    // one value per block: any thread's value keeps its chains live
    if (threadIdx.x == 0 && b < n_blocks) {
        cycles[b] = t1 - t0;
        sink[b] = s;
    }
}

template <int OP>
cudaError_t run_rate(int n_sm, int smem, long long *d_cycles, double *d_sink, cudaStream_t st, double &rate)
{
    cudaError_t e = cudaFuncSetAttribute(rate_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    rate_kernel<OP><<<n_sm, kRateThreads, smem, st>>>(d_cycles, d_sink, n_sm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<long long> cyc((size_t)n_sm);
    if ((e = cudaMemcpyAsync(cyc.data(), d_cycles, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    std::vector<double> r;
    for (long long c : cyc)
        if (c > 0) r.push_back((double)kRateThreads * RateShape<OP>::chains * kRateIters / (double)c);
    if (r.empty()) return cudaErrorUnknown;
    std::sort(r.begin(), r.end());
    rate = r[r.size() / 2];
    return cudaSuccess;
}

}  // namespace

cudaError_t measure_unit_rates(double *rates, cudaStream_t st, long long *d_cycles, double *d_sink, int n_sm)
{
    int dev = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    // more than half an SM's shared memory: one block per SM
    const int smem = smem_sm / 2 + 1024;
    if ((e = run_rate<0>(n_sm, smem, d_cycles, d_sink, st, rates[0])) != cudaSuccess) return e;
    if ((e = run_rate<1>(n_sm, smem, d_cycles, d_sink, st, rates[1])) != cudaSuccess) return e;
    if ((e = run_rate<2>(n_sm, smem, d_cycles, d_sink, st, rates[2])) != cudaSuccess) return e;
    if ((e = run_rate<3>(n_sm, smem, d_cycles, d_sink, st, rates[3])) != cudaSuccess) return e;
    if ((e = run_rate<4>(n_sm, smem, d_cycles, d_sink, st, rates[4])) != cudaSuccess) return e;
    if ((e = run_rate<5>(n_sm, smem, d_cycles, d_sink, st, rates[5])) != cudaSuccess) return e;
    return run_rate<6>(n_sm, smem, d_cycles, d_sink, st, rates[6]);
}

}  // namespace grins

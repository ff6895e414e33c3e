// Generic-N integrator instantiations, the Hill-exponent scan and the
// precision/size dispatch of the integrator.
#include "integrate_generic.cuh"

namespace grins {

cudaError_t launch_integrate_fp32_reg8(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_fp32_reg16(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_fp32_reg24(const IntegrateArgs &a, cudaStream_t st, int num_sms);

namespace {

// Largest Hill exponent n over all sets of the batch -> *out (atomic max).
__global__ void nmax_scan_kernel(const unsigned char *params, ParamLayout L, int64_t n_sets,
                                 unsigned long long *out)
{
    const long long total = n_sets * (long long)L.E;
    unsigned m = 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long s = g / L.E;
        const int e = (int)(g - s * L.E);
        m = max(m, (unsigned)params[s * L.stride + L.off_n + e]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, (unsigned long long)m);
}

}  // namespace

cudaError_t launch_integrate_fp32(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    const int N = a.topo.N;
    if (N > 24) return launch_dp5_generic<float>(a, st, num_sms);
    // register kernel for exponents <= 6, generic kernel otherwise; both are
    // queued and each returns at once unless the scanned exponent selects it
    unsigned long long *nmax = a.queue + 1;
    if (a.topo.E > 0) {
        const long long total = a.n_sets * (long long)a.topo.E;
        long long blocks = (total + 255) / 256;
        if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
        if (blocks < 1) blocks = 1;
        nmax_scan_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.params, a.L, a.n_sets, nmax);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    IntegrateArgs r = a;
    r.nmax = nmax;
    cudaError_t e;
    if (N <= 8) e = launch_integrate_fp32_reg8(r, st, num_sms);
    else if (N <= 16) e = launch_integrate_fp32_reg16(r, st, num_sms);
    else e = launch_integrate_fp32_reg24(r, st, num_sms);
    if (e != cudaSuccess) return e;
    IntegrateArgs g = a;
    g.nmax = nmax;
    g.gate = 2;
    return launch_dp5_generic<float>(g, st, num_sms);
}

cudaError_t launch_integrate_fp64(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    return launch_dp5_generic<double>(a, st, num_sms);
}

}  // namespace grins

// Distinct steady states per parameter set (Sec. 3.1: the multistability of a
// parameter set is the number of unique steady states it reaches over its
// initial conditions; Sec. 2.1.3: states are compared after G/k
// normalisation).
//
// Per set, in IC order, a converged state with normalised coordinates
// v_i = (x_i * k_i) / G_i joins the first representative r with
// max_i |v_i - r_i| <= tol, or becomes a new representative.  All arithmetic
// is IEEE double with explicit round-to-nearest operations (no contraction),
// so the result is bit-identical on any launch shape.  One thread per set;
// the representatives' IC indices are kept in registers for the first 32 and
// recovered from the state ids already written beyond that.
#include "common.cuh"

namespace grins {

namespace {

constexpr int kRepCache = 32;

__device__ __forceinline__ double norm_coord(double x, double k, double G)
{
    return __ddiv_rn(__dmul_rn(x, k), G);
}

__global__ void unique_kernel(const UniqueArgs a)
{
    const int N = a.L.N;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_sets;
         s += (long long)gridDim.x * blockDim.x) {
        const unsigned char *blk = a.params + s * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *X = a.states + s * (long long)a.n_ics * N;
        const uint8_t *st = a.status + s * (long long)a.n_ics;
        int32_t *sid = a.state_id + s * (long long)a.n_ics;
        int rep_ic[kRepCache];
        int n_rep = 0;
        for (int c = 0; c < a.n_ics; ++c) {
            if (st[c] != GRINS_SS_CONVERGED) { sid[c] = -1; continue; }
            const double *x = X + (long long)c * N;
            int joined = -1;
            for (int r = 0; r < n_rep && joined < 0; ++r) {
                int rc;
                if (r < kRepCache) {
                    rc = rep_ic[r];
                } else {   // the r-th representative is the first IC whose id is r
                    rc = 0;
                    while (sid[rc] != r) ++rc;
                }
                const double *xr = X + (long long)rc * N;
                double dmax = 0.0;
                for (int i = 0; i < N; ++i) {
                    const double d = fabs(__dsub_rn(norm_coord(x[i], K[i], G[i]), norm_coord(xr[i], K[i], G[i])));
                    dmax = d > dmax ? d : dmax;
                }
                if (dmax <= a.tol) joined = r;
            }
            if (joined < 0) {
                if (n_rep < kRepCache) rep_ic[n_rep] = c;
                joined = n_rep++;
            }
            sid[c] = joined;
        }
        a.n_unique[s] = n_rep;
    }
}

}  // namespace

cudaError_t launch_unique(const UniqueArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_sets <= 0) return cudaSuccess;
    long long blocks = (a.n_sets + 127) / 128;
    const long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    unique_kernel<<<(unsigned)blocks, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace grins

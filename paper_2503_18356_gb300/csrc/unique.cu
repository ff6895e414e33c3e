// Distinct steady states per parameter set (Sec. 3.1: the multistability of a
// parameter set is the number of unique steady states it reaches over its
// initial conditions; Sec. 2.1.3: states are compared after G/k
// normalisation).
//
// Per set, in IC order, a converged state with normalised coordinates
// v_i = (x_i * k_i) / G_i joins the first representative r with
// max_i |v_i - r_i| <= tol, or becomes a new representative.  All arithmetic
// is IEEE double with explicit round-to-nearest operations (no contraction),
// so the result is bit-identical on any launch shape.
//
// One warp per set, lanes over nodes: each converged state is normalised
// once (coalesced loads, one division per coordinate), the representatives'
// coordinates stay in shared memory, and a comparison is a warp vote -- the
// maximum is at most tol exactly when no coordinate difference exceeds tol
// (a NaN difference never raises the maximum, as in the sequential form) and
// 0 <= tol.  Representatives beyond the shared-memory capacity are
// normalised again when compared.
#include "common.cuh"

namespace grins {

namespace {

constexpr int kWarps = 8;              // warps per block
constexpr int kRepDoubles = 640;       // per warp: representatives' coordinates (5 KB)
constexpr int kVPL = 2;                // candidate coordinates per lane in registers
static_assert(kVPL * kWarp >= kMaxNodes, "every node of a network has a lane slot");
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double norm_coord(double x, double k, double G)
{
    return __ddiv_rn(__dmul_rn(x, k), G);
}

__global__ void __launch_bounds__(kWarps * kWarp) unique_kernel(const UniqueArgs a)
{
    __shared__ double reps[kWarps][kRepDoubles];
    const int N = a.L.N, I = a.n_ics;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x / kWarp;
    const int rcap = N > 0 ? kRepDoubles / N : 0;
    double *rv = reps[w];
    const double tol = a.tol;
    const bool tol_ok = 0.0 <= tol;
    for (long long s = (long long)blockIdx.x * kWarps + w; s < a.n_sets; s += (long long)gridDim.x * kWarps) {
        const unsigned char *blk = a.params + s * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *X = a.states + s * (long long)I * N;
        const uint8_t *st = a.status + s * (long long)I;
        int32_t *sid = a.state_id + s * (long long)I;
        int n_rep = 0;
        for (int c = 0; c < I; ++c) {
            if (st[c] != GRINS_SS_CONVERGED) {
                if (lane == 0) sid[c] = -1;
                __syncwarp();          // the id is read by every lane when recovering a representative
                continue;
            }
            const double *x = X + (long long)c * N;
            double v[kVPL];
#pragma unroll
            for (int m = 0; m < kVPL; ++m) {
                const int i = lane + kWarp * m;
                v[m] = i < N ? norm_coord(x[i], K[i], G[i]) : 0.0;
            }
            int joined = -1;
            for (int r = 0; r < n_rep; ++r) {
                const double *xr = nullptr;
                if (r >= rcap) {       // the r-th representative is the first IC whose id is r
                    int rc = 0;
                    while (rc < c && sid[rc] != r) ++rc;
                    xr = X + (long long)rc * N;
                }
                bool ok = true;
#pragma unroll
                for (int m = 0; m < kVPL; ++m) {
                    const int i = lane + kWarp * m;
                    if (i < N) {
                        const double vr = r < rcap ? rv[r * N + i] : norm_coord(xr[i], K[i], G[i]);
                        ok = ok && !(fabs(__dsub_rn(v[m], vr)) > tol);
                    }
                }
                if (__all_sync(FULL, ok) && tol_ok) { joined = r; break; }
            }
            if (joined < 0) {
                if (n_rep < rcap) {
#pragma unroll
                    for (int m = 0; m < kVPL; ++m) {
                        const int i = lane + kWarp * m;
                        if (i < N) rv[n_rep * N + i] = v[m];
                    }
                }
                joined = n_rep++;
            }
            if (lane == 0) sid[c] = joined;
            __syncwarp();
        }
        if (lane == 0) a.n_unique[s] = n_rep;
    }
}

}  // namespace

cudaError_t launch_unique(const UniqueArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_sets <= 0) return cudaSuccess;
    long long blocks = (a.n_sets + kWarps - 1) / kWarps;
    const long long cap = (long long)num_sms * 4;
    if (blocks > cap) blocks = cap;
    unique_kernel<<<(unsigned)blocks, kWarps * kWarp, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace grins

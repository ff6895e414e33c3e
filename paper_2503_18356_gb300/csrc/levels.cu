// Levels of G/k-normalised expression, state labels and multistability
// (Sec. 2.1.3: nodes are coarse-grained into levels "based on the global
// distribution" of the normalised values; a state is the concatenation of
// its nodes' levels and a set's multistability its number of distinct
// states, Sec. 3.1).  The reading of the unspecified boundary rule is the
// one declared in grins_racipe.h; this file holds the two device passes:
//   * gk_histogram_kernel: one warp per set, lanes over nodes; every node of
//     every converged solve goes to bin floor(v n_bins) of v = (x k) / G
//     (IEEE FP64, rounded as written; clamped to the first and last bin);
//     lanes of a warp that hit the same bin add once (match + popc) into
//     the block's shared histogram, which is added to the global one at the
//     end (64-bit counts throughout);
//   * level_states_kernel: one warp per set, lanes over nodes; a node's
//     level is the number of boundary bins below its bin, the label packs
//     the levels (two 32-bit OR reductions over the warp), and the set's
//     distinct labels are counted lanes over ICs (each compared with the
//     set's earlier converged solves).
#include "common.cuh"

namespace grins {

namespace {

constexpr int kLevelWarps = 8;          // warps per block
constexpr int kLevelVPL = 2;            // nodes per lane
constexpr unsigned FULL = 0xffffffffu;
static_assert(kLevelVPL * kWarp >= kMaxNodes, "every node of a network has a lane slot");

__device__ __forceinline__ int gk_bin(double x, double k, double G, int n_bins)
{
    const double f = __dmul_rn(__ddiv_rn(__dmul_rn(x, k), G), (double)n_bins);
    if (!(f >= 0.0)) return 0;
    if (f >= (double)n_bins) return n_bins - 1;
    return (int)f;
}

__global__ void __launch_bounds__(kLevelWarps * kWarp) gk_histogram_kernel(const LevelArgs a)
{
    extern __shared__ unsigned long long hist[];          // [n_bins]
    const int N = a.L.N, I = a.n_ics, B = a.n_bins;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x / kWarp;
    for (int b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0ull;
    __syncthreads();
    for (long long s = (long long)blockIdx.x * kLevelWarps + w; s < a.n_sets;
         s += (long long)gridDim.x * kLevelWarps) {
        const unsigned char *blk = a.params + s * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        for (int c = 0; c < I; ++c) {
            if (a.status[s * I + c] != GRINS_SS_CONVERGED) continue;
            const double *x = a.states + (s * I + c) * (long long)N;
#pragma unroll
            for (int m = 0; m < kLevelVPL; ++m) {
                const int i = lane + kWarp * m;
                const unsigned act = __ballot_sync(FULL, i < N);
                if (i < N) {
                    const int b = gk_bin(x[i], K[i], G[i], B);
                    const unsigned peers = __match_any_sync(act, b);
                    if (lane == __ffs(peers) - 1) atomicAdd(&hist[b], (unsigned long long)__popc(peers));
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x)
        if (hist[b]) atomicAdd(&a.counts[b], hist[b]);
}

__global__ void __launch_bounds__(kLevelWarps * kWarp) level_states_kernel(const LevelArgs a)
{
    const int N = a.L.N, I = a.n_ics, B = a.n_bins, W = a.width;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x / kWarp;
    for (long long s = (long long)blockIdx.x * kLevelWarps + w; s < a.n_sets;
         s += (long long)gridDim.x * kLevelWarps) {
        const unsigned char *blk = a.params + s * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        const uint8_t *st = a.status + s * I;
        unsigned long long *lab = a.labels + s * I;
        for (int c = 0; c < I; ++c) {
            if (st[c] != GRINS_SS_CONVERGED) {
                if (lane == 0) lab[c] = ~0ull;
                continue;
            }
            const double *x = a.states + (s * I + c) * (long long)N;
            unsigned long long part = 0ull;
#pragma unroll
            for (int m = 0; m < kLevelVPL; ++m) {
                const int i = lane + kWarp * m;
                if (i < N) {
                    const int b = gk_bin(x[i], K[i], G[i], B);
                    unsigned long long lev = 0ull;
                    for (int t = 0; t < a.n_bounds; ++t) lev += a.bounds[t] < b ? 1ull : 0ull;
                    part |= lev << (i * W);
                }
            }
            const unsigned lo = __reduce_or_sync(FULL, (unsigned)part);
            const unsigned hi = __reduce_or_sync(FULL, (unsigned)(part >> 32));
            if (lane == 0) lab[c] = ((unsigned long long)hi << 32) | lo;
        }
        __syncwarp();                   // the labels are read back by every lane
        int fresh = 0;
        for (int c = lane; c < I; c += kWarp) {
            if (st[c] != GRINS_SS_CONVERGED) continue;
            const unsigned long long l = lab[c];
            bool seen = false;
            for (int c2 = 0; c2 < c && !seen; ++c2) seen = st[c2] == GRINS_SS_CONVERGED && lab[c2] == l;
            fresh += seen ? 0 : 1;
        }
        const int n = (int)__reduce_add_sync(FULL, (unsigned)fresh);
        if (lane == 0) {
            a.n_states[s] = n;
            atomicAdd(&a.multi_hist[n], 1ull);
        }
    }
}

long long level_blocks(long long n_sets, int num_sms)
{
    long long blocks = (n_sets + kLevelWarps - 1) / kLevelWarps;
    const long long cap = (long long)num_sms * 4;
    return blocks > cap ? cap : (blocks < 1 ? 1 : blocks);
}

}  // namespace

cudaError_t launch_gk_histogram(const LevelArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_sets <= 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned long long) * (size_t)a.n_bins;
    gk_histogram_kernel<<<(unsigned)level_blocks(a.n_sets, num_sms), kLevelWarps * kWarp, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_level_states(const LevelArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_sets <= 0) return cudaSuccess;
    level_states_kernel<<<(unsigned)level_blocks(a.n_sets, num_sms), kLevelWarps * kWarp, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace grins

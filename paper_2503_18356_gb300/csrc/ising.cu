// Boolean Ising formalism (Sec. 2.2, Eq. 3): node i turns on when
// sum_j J_ij s_j > 0, off when it is < 0, and keeps its state on a tie;
// J_ij = +1 (activating edge j -> i), -1 (inhibiting).  One thread per
// trajectory: the state is one 64-bit word (bit i = node i on), and a
// node's field is two population counts against the bit masks of its
// activating and inhibiting sources -- with inactive nodes counted as -1,
// h = 2 |s & A_i| - |A_i| - 2 |s & I_i| + |I_i|; counted as 0 (the 0/1
// encoding), h = |s & A_i| - |s & I_i|.  Synchronous mode updates every
// node at once; asynchronous mode one node per step, drawn uniformly from
// the trajectory's Philox4x64-10 stream (draw d = word d % 4 of the block
// with counter (trajectory, d / 4, 0, 0), key (seed, "ISINGBO"); draw 0
// is the random initial state, draw 1 + k picks step k's node).  A
// trajectory stops at a fixed point (status converged, steps = updates
// applied before it) or after max_steps updates.
#include "common.cuh"

namespace grins {

namespace {

constexpr uint64_t kTagIsing = 0x4953494E47424Full;   // "ISINGBO"

__device__ __forceinline__ unsigned long long ising_sync(const IsingArgs &a, unsigned long long s)
{
    unsigned long long t = s;
    for (int i = 0; i < a.N; ++i) {
        const int ha = __popcll(s & a.act[i]), hi = __popcll(s & a.inh[i]);
        const int h = a.enc01 ? ha - hi : 2 * ha - a.n_act[i] - 2 * hi + a.n_inh[i];
        if (h > 0) t |= 1ull << i;
        else if (h < 0) t &= ~(1ull << i);
    }
    return t;
}

__device__ __forceinline__ uint64_t ising_draw(const IsingArgs &a, long long traj, uint64_t d)
{
    const U64x4 r = philox4x64_10((uint64_t)traj, d / 4, 0, 0, a.seed, kTagIsing);
    switch (d % 4) {
    case 0: return r.v[0];
    case 1: return r.v[1];
    case 2: return r.v[2];
    default: return r.v[3];
    }
}

__global__ void ising_kernel(const IsingArgs a)
{
    const unsigned long long mask = a.N == 64 ? ~0ull : ((1ull << a.N) - 1ull);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_traj;
         t += (long long)gridDim.x * blockDim.x) {
        unsigned long long s = (a.init ? a.init[t] : ising_draw(a, t, 0)) & mask;
        int k = 0;
        uint8_t st = GRINS_SS_MAXSTEPS;
        for (;;) {
            const unsigned long long next = ising_sync(a, s);
            if (next == s) { st = GRINS_SS_CONVERGED; break; }
            if (k >= a.max_steps) break;
            if (a.mode == 0) {
                s = next;
            } else {
                // node uniform in [0, N - 1] from the draw's top 32 bits (multiply-shift)
                const uint64_t r = ising_draw(a, t, 1 + (uint64_t)k);
                const int i = (int)(((r >> 32) * (uint64_t)a.N) >> 32);
                s = (s & ~(1ull << i)) | (next & (1ull << i));
            }
            ++k;
        }
        a.final_state[t] = s;
        a.steps[t] = k;
        a.status[t] = st;
    }
}

}  // namespace

cudaError_t launch_ising(const IsingArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_traj <= 0) return cudaSuccess;
    long long blocks = (a.n_traj + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    if (blocks > cap) blocks = cap;
    ising_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace grins

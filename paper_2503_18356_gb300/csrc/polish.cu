// FP64 Newton polish and residual certificate of converged steady states.
//
// A steady state is a zero of Eq. 1: f_i(x) = G_i prod_e F_e(x_src) - k_i x_i.
// From the state the integrator stopped at, Newton steps x <- x + d with
// J d = -f(x) are taken in double precision, J analytic:
//     J_ij = G_i P_i sum_{e: src(e)=j, dst(e)=i} F_e'(x_j) / F_e(x_j) - k_i [i=j],
//     F_e = (a p + b) / (1 + p), p = (x/T)^n,
//     F_e'/F_e = (a - b) n p / ((1 + p)(a p + b) x).
// Converged when rho = max_i |f_i| / (G_i / k_i) < tol.  A solve whose
// Newton step moves a G/k-normalised coordinate by more than max_move, whose
// Jacobian is singular, or that does not reach tol within `iters` steps keeps
// its unpolished state and gets status GRINS_SS_POLISH_FAIL.
// One warp per solve: lanes over rows (targets) for the residual and
// Jacobian, Gaussian elimination with partial pivoting in shared memory.
#include "integrate.cuh"

namespace grins {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * kWarp) polish_kernel(const PolishArgs a)
{
    __shared__ double sJ[WARPS][NMAX][NMAX + 1];
    __shared__ double sx[WARPS][NMAX];
    __shared__ double sb[WARPS][NMAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int N = a.topo.N;
    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    double (*J)[NMAX + 1] = sJ[w];
    double *x = sx[w];
    double *b = sb[w];

    for (long long idx = (long long)blockIdx.x * WARPS + w; idx < a.n_solves;
         idx += (long long)gridDim.x * WARPS) {
        if (a.status[idx] != GRINS_SS_CONVERGED) {
            if (lane == 0 && a.err_est) a.err_est[idx] = -1.0f;
            continue;
        }
        const long long set = idx / a.n_ics;
        const unsigned char *blk = a.params + set * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *T = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *lam = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nn = blk + a.L.off_n;
        double *state = a.states + idx * N;
        for (int i = lane; i < N; i += kWarp) x[i] = state[i];
        __syncwarp();

        bool ok = false;
        double last_move = 0.0, rho = 0.0;
        for (int it = 0; it <= a.iters; ++it) {
            // residual and Jacobian rows, lanes over targets
            double rloc = 0.0;
            for (int i = lane; i < N; i += kWarp) {
                for (int j = 0; j < N; ++j) J[i][j] = 0.0;
                double P = 1.0;
                for (int c = a.topo.off[i]; c < a.topo.off[i + 1]; ++c) {
                    int e = a.topo.edge[c], s = a.topo.src[c];
                    if (!GRINS_OK_IDX(e >= 0 && e < a.topo.E && s >= 0 && s < N && N <= NMAX, 21, c)) e = s = 0;
                    const double xs = fmax(x[s], 0.0);
                    const double r = xs / T[e];
                    const int n = nn[e];
                    double p = 1.0, pm1 = 1.0, base = r;
                    for (int m = n; m; m >>= 1) { if (m & 1) p *= base; base *= base; }
                    base = r;
                    for (int m = n - 1; m > 0; m >>= 1) { if (m & 1) pm1 *= base; base *= base; }
                    const bool act = a.topo.sign[c] > 0;
                    const double aa = act ? 1.0 : lam[e];
                    const double bb = act ? 1.0 / lam[e] : 1.0;
                    const double num = fma(aa, p, bb), den = 1.0 + p;
                    P *= num / den;
                    // d log F / dx = (a - b) n r^(n-1) / (T (1 + p)(a p + b))
                    J[i][s] += (aa - bb) * (double)n * pm1 / (T[e] * den * num);
                }
                const double f = G[i] * P - K[i] * x[i];
                b[i] = -f;
                for (int j = 0; j < N; ++j) J[i][j] *= G[i] * P;
                J[i][i] -= K[i];
                rloc = fmax(rloc, fabs(f) / (G[i] / K[i]));
            }
            rho = warp_max(rloc);
            __syncwarp();
            if (rho < a.tol) { ok = true; break; }
            if (it == a.iters || !(rho == rho)) break;

            // Gaussian elimination with partial pivoting
            bool singular = false;
            for (int c = 0; c < N; ++c) {
                double best = -1.0;
                int piv = c;
                for (int r = c + lane; r < N; r += kWarp) {
                    const double v = fabs(J[r][c]);
                    if (v > best) { best = v; piv = r; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(FULL, best, o);
                    const int op = __shfl_xor_sync(FULL, piv, o);
                    if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
                }
                if (!(best > 0.0)) { singular = true; break; }
                if (piv != c) {
                    for (int j = lane; j < N; j += kWarp) {
                        const double tmp = J[c][j]; J[c][j] = J[piv][j]; J[piv][j] = tmp;
                    }
                    if (lane == 0) { const double tb = b[c]; b[c] = b[piv]; b[piv] = tb; }
                }
                __syncwarp();
                const double inv = 1.0 / J[c][c];
                for (int r = c + 1 + lane; r < N; r += kWarp) {
                    const double m = J[r][c] * inv;
                    for (int j = c + 1; j < N; ++j) J[r][j] -= m * J[c][j];
                    b[r] -= m * b[c];
                }
                __syncwarp();
            }
            if (singular) break;
            // back substitution (b becomes the Newton step)
            for (int r = N - 1; r >= 0; --r) {
                double s = 0.0;
                for (int j = r + 1 + lane; j < N; j += kWarp) s += J[r][j] * b[j];
                s = warp_sum(s);
                if (lane == 0) b[r] = (b[r] - s) / J[r][r];
                __syncwarp();
            }
            double mv = 0.0;
            for (int i = lane; i < N; i += kWarp) mv = fmax(mv, fabs(b[i]) * (K[i] / G[i]));
            mv = warp_max(mv);
            if (!(mv <= a.max_move)) break;
            for (int i = lane; i < N; i += kWarp) x[i] += b[i];
            last_move = mv;
            __syncwarp();
        }
        if (ok) {
            for (int i = lane; i < N; i += kWarp) state[i] = x[i];
            if (lane == 0 && a.err_est) a.err_est[idx] = (float)(last_move > 0.0 ? last_move : rho);
        } else {
            if (lane == 0) {
                a.status[idx] = GRINS_SS_POLISH_FAIL;
                if (a.err_est) a.err_est[idx] = -1.0f;
            }
        }
        __syncwarp();
    }
}

template <int NMAX, int WARPS>
cudaError_t launch_bucket(const PolishArgs &a, cudaStream_t st, int num_sms)
{
    auto kern = polish_kernel<NMAX, WARPS>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * kWarp, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)num_sms * per_sm;
    const long long need = (a.n_solves + WARPS - 1) / WARPS;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, WARPS * kWarp, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_polish(const PolishArgs &a, cudaStream_t st, int num_sms)
{
    if (a.n_solves <= 0) return cudaSuccess;
    const int N = a.topo.N;
    if (N <= 8) return launch_bucket<8, 8>(a, st, num_sms);
    if (N <= 16) return launch_bucket<16, 8>(a, st, num_sms);
    if (N <= 32) return launch_bucket<32, 4>(a, st, num_sms);
    return launch_bucket<64, 1>(a, st, num_sms);
}

}  // namespace grins

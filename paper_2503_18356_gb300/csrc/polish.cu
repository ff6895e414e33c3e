// Newton polish and FP64 residual certificate of converged steady states.
//
// A steady state is a zero of Eq. 1: f_i(x) = G_i prod_e F_e(x_src) - k_i x_i.
// From the state the integrator stopped at, the polish takes chord-Newton
// steps x <- x + d with J0 d = -f(x) (mixed-precision iterative refinement):
//   * f is evaluated in FP64 at every step (the quantity being certified);
//   * the analytic Jacobian is evaluated once, at the starting state, in
//     FP32, and factorised once (LU with partial pivoting, FP32):
//       J_ij = G_i P_i sum_{e: src(e)=j, dst(e)=i} F_e'(x_j) / F_e(x_j) - k_i [i=j],
//       F_e = (a p + b) / (1 + p), p = (x/T)^n,
//       F_e'/F_e = (a - b) n p / ((1 + p)(a p + b) x);
//   * the step is solved in FP32 and added to the FP64 state.
// Starting within ~1e-5 of the fixed point, each step shrinks the error by
// about the FP32 Jacobian's relative error times its condition number, so
// two or three steps reach an FP64 residual of 1e-12 while every operation
// but the residual runs at FP32 rate.
// Converged when rho = max_i |f_i| / (G_i / k_i) < tol.  A solve whose step
// moves a G/k-normalised coordinate by more than max_move, whose Jacobian is
// singular, or that does not reach tol within `iters` steps keeps its
// unpolished state and gets status GRINS_SS_POLISH_FAIL.
// One warp per solve: lanes over rows (targets).
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

__device__ __forceinline__ float warp_maxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// x^n for a small non-negative integer n, by repeated squaring
template <typename Real>
__device__ __forceinline__ Real ipow(Real x, int n)
{
    Real p = (Real)1, b = x;
    for (; n; n >>= 1) {
        if (n & 1) p *= b;
        b *= b;
    }
    return p;
}

template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * kWarp) polish_kernel(const PolishArgs a)
{
    __shared__ float sJ[WARPS][NMAX][NMAX + 1];   // FP32 Jacobian, then its LU factors
    __shared__ double sx[WARPS][NMAX];            // FP64 state
    __shared__ float sb[WARPS][NMAX];             // FP32 right-hand side, then the step
    __shared__ int spiv[WARPS][NMAX];             // pivot row of each elimination step
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int N = a.topo.N;
    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    float (*J)[NMAX + 1] = sJ[w];
    double *x = sx[w];
    float *b = sb[w];
    int *piv = spiv[w];

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

        // f_i in FP64 for the rows of this lane -> b (FP32, negated); returns
        // rho.  Each factor of Eq. 2 is written without divisions,
        //     F_e = (lam x^n + T^n) / ((x^n + T^n) c),  c = lam (activating), 1,
        // (numerator and denominator of (lam p + 1) / ((1 + p) c) times T^n),
        // and the products are divided once per eight factors (x^n, T^n stay
        // below ~1e24, so eight factors stay finite).  With `jac` row i of
        // the Jacobian is filled in as well.
        auto residual = [&](bool jac) -> double {
            double rloc = 0.0;
            for (int i = lane; i < N; i += kWarp) {
                if (jac)
                    for (int j = 0; j < N; ++j) J[i][j] = 0.0f;
                double P = 1.0, num = 1.0, den = 1.0;
                int cnt = 0;
                for (int c = a.topo.off[i]; c < a.topo.off[i + 1]; ++c) {
                    int e = a.topo.edge[c], s = a.topo.src[c];
                    if (!GRINS_OK_IDX(e >= 0 && e < a.topo.E && s >= 0 && s < N && N <= NMAX, 21, c)) e = s = 0;
                    const bool act = a.topo.sign[c] > 0;
                    const int n = nn[e];
                    const double l = lam[e], Te = T[e];
                    const double xs = fmax(x[s], 0.0);
                    const double xn = ipow(xs, n), tn = ipow(Te, n);
                    num *= fma(l, xn, tn);
                    den *= act ? (xn + tn) * l : xn + tn;
                    if (++cnt == 8) { P *= num / den; num = den = 1.0; cnt = 0; }
                    if (jac) {
                        // d log F / dx = n p (lam - 1) / (x (lam p + 1)(1 + p)),
                        // p = (x/T)^n, in FP32 (the Jacobian only steers the
                        // iteration); at x = 0 only n = 1 leaves a slope
                        const float lf = (float)l, xf = (float)xs;
                        float dl;
                        if (xf > 0.0f) {
                            const float pf = (float)fmin(xn / tn, 1e30);
                            dl = (float)n * (lf - 1.0f) / xf * (pf / (1.0f + pf)) / fmaf(lf, pf, 1.0f);
                        } else {
                            dl = n == 1 ? (lf - 1.0f) / (float)Te : 0.0f;
                        }
                        J[i][s] += dl;   // scaled by G_i P_i below
                    }
                }
                P *= num / den;
                const double f = G[i] * P - K[i] * x[i];
                b[i] = (float)(-f);
                if (jac) {
                    const float gp = (float)(G[i] * P);
                    for (int j = 0; j < N; ++j) J[i][j] *= gp;
                    J[i][i] -= (float)K[i];
                }
                rloc = fmax(rloc, fabs(f) * (K[i] / G[i]));
            }
            return warp_max(rloc);
        };

        bool ok = false, singular = false;
        double last_move = 0.0;
        double rho = residual(true);
        __syncwarp();
        if (rho < a.tol) ok = true;

        // LU of the FP32 Jacobian with partial pivoting; multipliers kept
        // below the diagonal, row swaps recorded in piv
        if (!ok) {
            for (int c = 0; c < N; ++c) {
                float best = -1.0f;
                int pr = c;
                for (int r = c + lane; r < N; r += kWarp) {
                    const float v = fabsf(J[r][c]);
                    if (v > best) { best = v; pr = r; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(FULL, best, o);
                    const int op = __shfl_xor_sync(FULL, pr, o);
                    if (ob > best || (ob == best && op < pr)) { best = ob; pr = op; }
                }
                if (!(best > 0.0f)) { singular = true; break; }
                if (lane == 0) piv[c] = pr;
                if (pr != c) {
                    for (int j = lane; j < N; j += kWarp) {
                        const float t = J[c][j]; J[c][j] = J[pr][j]; J[pr][j] = t;
                    }
                }
                __syncwarp();
                const float inv = 1.0f / J[c][c];
                for (int r = c + 1 + lane; r < N; r += kWarp) {
                    const float m = J[r][c] * inv;
                    J[r][c] = m;
                    for (int j = c + 1; j < N; ++j) J[r][j] = fmaf(-m, J[c][j], J[r][j]);
                }
                __syncwarp();
            }
        }

        // chord iterations: solve J0 d = -f(x) in FP32, x += d in FP64
        for (int it = 0; !ok && !singular && it < a.iters; ++it) {
            if (lane == 0)
                for (int c = 0; c < N; ++c) {
                    const int pr = piv[c];
                    if (pr != c) { const float t = b[c]; b[c] = b[pr]; b[pr] = t; }
                }
            __syncwarp();
            for (int c = 0; c < N; ++c) {                 // forward (unit lower)
                const float bc = b[c];
                for (int r = c + 1 + lane; r < N; r += kWarp) b[r] = fmaf(-J[r][c], bc, b[r]);
                __syncwarp();
            }
            for (int c = N - 1; c >= 0; --c) {            // backward (upper)
                if (lane == 0) b[c] = b[c] / J[c][c];
                __syncwarp();
                const float bc = b[c];
                for (int r = lane; r < c; r += kWarp) b[r] = fmaf(-J[r][c], bc, b[r]);
                __syncwarp();
            }
            float mv = 0.0f;
            for (int i = lane; i < N; i += kWarp) mv = fmaxf(mv, fabsf(b[i]) * (float)(K[i] / G[i]));
            mv = warp_maxf(mv);
            if (!(mv <= (float)a.max_move)) break;
            for (int i = lane; i < N; i += kWarp) x[i] += (double)b[i];
            last_move = mv;
            __syncwarp();
            rho = residual(false);
            __syncwarp();
            if (rho < a.tol) ok = true;
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

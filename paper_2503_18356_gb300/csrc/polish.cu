// Newton polish and FP64 residual certificate of converged steady states.
//
// A steady state is a zero of Eq. 1: f_i(x) = G_i prod_e F_e(x_src) - k_i x_i.
// From the state the integrator stopped at, the polish takes chord-Newton
// steps x <- x + d with J0 d = -f(x) (mixed-precision iterative refinement):
//   * f is evaluated in FP64 at every step (the quantity being certified):
//     a row's f_i = (G_i nu_i - k_i x_i de_i) / de_i, with nu_i and de_i the
//     products of its factors' numerators and denominators (below), forms
//     the cancelling difference in FP64 and takes the quotient by an
//     approximate FP64 reciprocal (one special-function instruction instead
//     of an FP64 division; relative error below 1e-6, measured on this GPU
//     over 4M inputs spanning 2^-1000 .. 2^1000 -- rho is compared with tol
//     to that relative accuracy, far finer than the threshold needs, and the
//     step, from an FP32 Jacobian, is unaffected);
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
//
// FP64 runs at a small fraction of the FP32 rate on this GPU (a warp's FP64
// instruction occupies the SM's FP64 pipe for about 16 cycles), so the
// residual is arranged to issue few FP64 warp instructions, each with most
// lanes busy.  A warp takes a work unit of one parameter set and up to
// kUnitIcs of its initial conditions, and polishes the unit's converged
// solves one after another:
//   * once per unit, lanes over edges (CSR order) tabulate lambda, T^n and
//     c T^n below with the edge's source, exponent and sign in shared
//     memory (multiplications only), lanes over nodes the row constants --
//     the parameters are the set's, shared by its ICs;
//   * per residual, lanes over nodes tabulate x^1 .. x^6, lanes over edges
//     form each factor's numerator lambda x^n + T^n and denominator
//     c x^n + c T^n (one FMA each), and lanes over rows (targets) multiply
//     their factors and form f_i;
//   * the Jacobian is filled edge by edge in FP32; the LU runs in shared
//     memory, the substitutions with the right-hand side in registers (one
//     row per lane, values passed by shuffles).
#include <climits>

#include "integrate.cuh"

namespace grins {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kPow = 6;          // x^1 .. x^6 tabulated per node
constexpr int kUnitIcs = 5;      // initial conditions per work unit (22-node workload, 10 ICs per set:
                                 // 2 / 4 / 5 / 10 -> 6.61 / 6.45 / 6.37 / 6.37 ms; with fixed shares of
                                 // units, 1 / 4 / 16 -> 8.95 / 8.10 / 8.30 ms)

__device__ __forceinline__ float warp_maxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// NaN -> +inf, so that the warp maxima of rho and of the step (fmaxf drops
// NaN operands) see a non-finite residual or step
__device__ __forceinline__ float nan_to_inf(float v) { return v == v ? v : __int_as_float(0x7f800000); }

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

// Approximate FP64 reciprocal (one special-function instruction; inputs
// and results below the normal range flush to zero)
__device__ __forceinline__ double rcp_approx64(double v)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
    return r;
}

// Bytes of the per-warp edge tables for E edges: FP64 c T^n, lambda, T^n,
// factor numerator and denominator; int (src << 9 | act << 8 | n) and
// target row; FP32 (T, lambda).
__host__ __device__ constexpr long long polish_edge_bytes(int E)
{
    return (long long)(E > 0 ? E : 1) * (5 * 8 + 2 * 4 + 8);
}

template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * kWarp) polish_kernel(const PolishArgs a)
{
    constexpr int RPL = NMAX > kWarp ? NMAX / kWarp : 1;   // rows per lane
    __shared__ float sJ[WARPS][NMAX][NMAX + 1];   // FP32 Jacobian, then its LU factors
    __shared__ double sx[WARPS][NMAX];            // FP64 state
    __shared__ double sxp[WARPS][kPow][NMAX];     // x^1 .. x^6 per node
    __shared__ float sgp[WARPS][NMAX];            // G_i P_i at the starting state
    __shared__ float sxf[WARPS][NMAX];            // FP32 max(x, 0) at the starting state
    __shared__ int spiv[WARPS][NMAX];             // pivot row of each elimination step
    __shared__ int sperm[WARPS][NMAX];            // row permutation of the LU
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int N = a.topo.N, E = a.topo.E;
    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    float (*J)[NMAX + 1] = sJ[w];
    double *x = sx[w];
    double (*xp)[NMAX] = sxp[w];
    float *gp = sgp[w];
    float *xf32 = sxf[w];
    int *piv = spiv[w];
    int *perm = sperm[w];
    const int Eb = E > 0 ? E : 1;
    unsigned char *eb = dsm + (long long)w * polish_edge_bytes(E);
    double *cb_e = reinterpret_cast<double *>(eb);
    double *a_e = cb_e + Eb;
    double *b_e = a_e + Eb;
    double *num_e = b_e + Eb;
    double *den_e = num_e + Eb;
    int *code_e = reinterpret_cast<int *>(den_e + Eb);
    int *row_e = code_e + Eb;
    float2 *tl_e = reinterpret_cast<float2 *>(row_e + Eb);

    // target row of every CSR position (the topology's, fixed)
    for (int i = lane; i < N; i += kWarp)
        for (int c = a.topo.off[i]; c < a.topo.off[i + 1]; ++c) row_e[c] = i;
    const int upc = (a.n_ics + kUnitIcs - 1) / kUnitIcs;      // units per set
    // list mode: one unit per listed solve
    const bool list = a.items != nullptr;
    long long n_units = a.n_ics > 0 ? a.n_solves / a.n_ics * upc : 0;
    if (list) n_units = (long long)min(*a.n_items, (unsigned long long)a.n_solves);
    const bool dyn = a.queue != nullptr;
    auto next_unit = [&](long long u) -> long long {
        if (!dyn) return u + (long long)gridDim.x * WARPS;
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(a.queue, 1ull);
        return (long long)__shfl_sync(FULL, v, 0);
    };
    for (long long u = dyn ? next_unit(0) : (long long)blockIdx.x * WARPS + w; u < n_units; u = next_unit(u)) {
        long long set;
        int ic0, ic1;
        if (list) {
            long long idx = a.items[u].idx;
            if (!GRINS_OK_IDX(idx >= 0 && idx < a.n_solves, 24, idx)) idx = 0;
            set = idx / a.n_ics;
            ic0 = (int)(idx - set * a.n_ics);
            ic1 = ic0 + 1;
            // the re-pass left its final status marked: clear the mark
            if (lane == 0) a.status[idx] = (uint8_t)(a.status[idx] & ~kStatusListed);
            __syncwarp();
        } else {
            set = u / upc;
            ic0 = (int)(u - set * upc) * kUnitIcs;
            ic1 = min(ic0 + kUnitIcs, a.n_ics);
        }
        if (a.cancel != nullptr && grins_cancelled(a.cancel)) {
            // cancelled: the unit's converged solves stay unpolished
            for (int ic = ic0 + lane; ic < ic1; ic += kWarp) {
                const long long idx = set * a.n_ics + ic;
                const uint8_t st = a.status[idx];
                if (st == GRINS_SS_CONVERGED) a.status[idx] = GRINS_SS_CANCELLED;
                if (a.err_est && !(st & kStatusListed)) a.err_est[idx] = -1.0f;
            }
            continue;
        }
        // a unit without converged solves needs no tables
        bool any = false;
        for (int ic = ic0 + lane; ic < ic1; ic += kWarp) {
            const long long idx = set * a.n_ics + ic;
            const uint8_t st = a.status[idx];
            any = any || st == GRINS_SS_CONVERGED;
            // a solve listed for the re-pass (running beside this polish)
            // is left alone: the list-mode polish after it sets its outputs
            if (st != GRINS_SS_CONVERGED && !(st & kStatusListed) && a.err_est) a.err_est[idx] = -1.0f;
        }
        if (!__any_sync(FULL, any)) continue;
        const unsigned char *blk = a.params + set * a.L.stride;
        const double *G = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *K = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *T = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *lam = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nn = blk + a.L.off_n;

        // edge tables (lanes over CSR positions) and row constants of the set
        for (int c = lane; c < E; c += kWarp) {
            int e = a.topo.edge[c], s = a.topo.src[c];
            if (!GRINS_OK_IDX(e >= 0 && e < E && s >= 0 && s < N && N <= NMAX, 21, c)) e = s = 0;
            const int n = nn[e];
            const bool act = a.topo.sign[c] > 0;
            const double Te = T[e], l = lam[e], tn = ipow(Te, n);
            a_e[c] = l;
            b_e[c] = tn;
            cb_e[c] = act ? l * tn : tn;
            code_e[c] = (s << 9) | (act ? 256 : 0) | n;
            tl_e[c] = make_float2((float)Te, (float)l);
        }
        double Gr[RPL], Kr[RPL];
        float kg[RPL];
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const int i = lane + kWarp * k;
            Gr[k] = 1.0; Kr[k] = 0.0; kg[k] = 0.0f;
            if (i < N) {
                Gr[k] = G[i]; Kr[k] = K[i];
                kg[k] = div_approx((float)Kr[k], (float)Gr[k]);
            }
        }
        __syncwarp();

        for (int ic = ic0; ic < ic1; ++ic) {
            const long long idx = set * a.n_ics + ic;
            if (a.status[idx] != GRINS_SS_CONVERGED) continue;
            double *state = a.states + idx * N;
            for (int i = lane; i < N; i += kWarp) x[i] = state[i];
            __syncwarp();

            // f in FP64 -> b = -f (FP32, one entry per row of this lane); returns
            // rho.  Each factor of Eq. 2 is written without divisions,
            //     F_e = (lam x^n + T^n) / (c x^n + c T^n),
            // c = lam activating, 1 inhibiting (numerator and denominator of
            // (lam p + 1) / ((1 + p) c) times T^n), and a row's running
            // products are divided once per eight factors (x^n, T^n stay
            // below ~1e24 and lam c below ~1e4, so eight factors stay
            // finite).  With `jac` the FP32 Jacobian is filled in as well.
            float b[RPL];
            auto residual = [&](bool jac) -> float {
                for (int i = lane; i < N; i += kWarp) {
                    const double v = fmax(x[i], 0.0);
                    const double v2 = v * v, v4 = v2 * v2;
                    xp[0][i] = v; xp[1][i] = v2; xp[2][i] = v2 * v;
                    xp[3][i] = v4; xp[4][i] = v4 * v; xp[5][i] = v2 * v4;
                    if (jac) xf32[i] = (float)v;
                }
                __syncwarp();
                for (int c = lane; c < E; c += kWarp) {
                    const int code = code_e[c], s = code >> 9, n = code & 255;
                    const double xn = (n >= 1 && n <= kPow) ? xp[n - 1][s] : ipow(fmax(x[s], 0.0), n);
                    num_e[c] = fma(a_e[c], xn, b_e[c]);
                    den_e[c] = fma((code & 256) ? a_e[c] : 1.0, xn, cb_e[c]);
                }
                __syncwarp();
                float rloc = 0.0f;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int i = lane + kWarp * k;
                    b[k] = 0.0f;
                    if (i < N) {
                        double P = Gr[k], nu = 1.0, de = 1.0;
                        int cnt = 0;
                        for (int c = a.topo.off[i]; c < a.topo.off[i + 1]; ++c) {
                            nu *= num_e[c];
                            de *= den_e[c];
                            if (++cnt == 8) { P *= nu / de; nu = de = 1.0; cnt = 0; }
                        }
                        // f = (G nu - k x de) / de: the difference in FP64,
                        // the quotient to about FP32 accuracy
                        const double pn = P * nu, kx = Kr[k] * x[i], rde = rcp_approx64(de);
                        const double f = fma(-kx, de, pn) * rde;
                        b[k] = (float)(-f);
                        if (jac) gp[i] = (float)(pn * rde);
                        rloc = fmaxf(rloc, nan_to_inf(fabsf(b[k]) * kg[k]));
                    }
                }
                if (jac) {
                    // J_is = G_i P_i dlog F_e / dx_s for the edge e = (s -> i)
                    // (one edge per pair), then J_ii -= k_i.  dlog F / dx =
                    // n p (lam - 1) / (x (lam p + 1)(1 + p)), p = (x/T)^n, in
                    // FP32 (the Jacobian only steers the iteration); at x = 0
                    // only n = 1 leaves a slope.
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + kWarp * k;
                        if (i < N)
                            for (int j = 0; j < N; ++j) J[i][j] = 0.0f;
                    }
                    __syncwarp();
                    for (int c = lane; c < E; c += kWarp) {
                        const int code = code_e[c], s = code >> 9, n = code & 255, i = row_e[c];
                        const float2 tl = tl_e[c];
                        const float xf = xf32[s];
                        float dl;
                        if (xf > 0.0f) {
                            const float pf = fminf(ipow(xf * div_approx(1.0f, tl.x), n), 1e30f);
                            dl = (float)n * (tl.y - 1.0f) * pf * div_approx(1.0f, xf * (1.0f + pf)) *
                                 div_approx(1.0f, fmaf(tl.y, pf, 1.0f));
                        } else {
                            dl = n == 1 ? (tl.y - 1.0f) * div_approx(1.0f, tl.x) : 0.0f;
                        }
                        J[i][s] = gp[i] * dl;
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + kWarp * k;
                        if (i < N) J[i][i] -= (float)Kr[k];
                    }
                }
                return warp_maxf(rloc);
            };

            bool ok = false, singular = false;
            float last_move = 0.0f;
            float rho = residual(true);
            __syncwarp();
            if ((double)rho < a.tol) ok = true;

            // LU of the FP32 Jacobian with partial pivoting; multipliers kept
            // below the diagonal, reciprocals of the pivots on it, and the row
            // swaps composed into perm ((P b)_r = b_perm[r])
            if (!ok) {
                for (int c = 0; c < N; ++c) {
                    float best = -1.0f;
                    int pr = c;
                    for (int r = c + lane; r < N; r += kWarp) {
                        const float v = fabsf(J[r][c]);
                        if (v > best) { best = v; pr = r; }
                    }
                    // largest magnitude over the warp, lowest row among equals
                    const unsigned key = best >= 0.0f ? __float_as_uint(best) + 1u : 0u;
                    const unsigned mx = __reduce_max_sync(FULL, key);
                    pr = __reduce_min_sync(FULL, key == mx ? pr : INT_MAX);
                    if (mx <= 1u) { singular = true; break; }     // no candidate, or only zeros
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
                if (!singular) {
                    for (int c = lane; c < N; c += kWarp) J[c][c] = 1.0f / J[c][c];
                    if (lane == 0) {
                        // the swaps in order applied to the identity
                        for (int c = 0; c < N; ++c) perm[c] = c;
                        for (int c = 0; c < N; ++c) {
                            const int p = piv[c];
                            const int t = perm[c]; perm[c] = perm[p]; perm[p] = t;
                        }
                    }
                    __syncwarp();
                }
            }

            // b of row r (warp-uniform r) from the lane holding it
            auto row_value = [&](int r) -> float {
                float v = b[0];
#pragma unroll
                for (int k = 1; k < RPL; ++k)
                    if (r >= kWarp * k) v = b[k];
                return __shfl_sync(FULL, v, r & (kWarp - 1));
            };

            // chord iterations: solve J0 d = -f(x) in FP32, x += d in FP64
            for (int it = 0; !ok && !singular && it < a.iters; ++it) {
                // b <- P b
                float pb[RPL];
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int i = lane + kWarp * k;
                    const int p = i < N ? perm[i] : 0;
                    float v = 0.0f;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const float t = __shfl_sync(FULL, b[q], p & (kWarp - 1));
                        if (p >> 5 == q) v = t;
                    }
                    pb[k] = v;
                }
#pragma unroll
                for (int k = 0; k < RPL; ++k) b[k] = pb[k];
                for (int c = 0; c < N; ++c) {                 // forward (unit lower)
                    const float bc = row_value(c);
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + kWarp * k;
                        if (i > c && i < N) b[k] = fmaf(-J[i][c], bc, b[k]);
                    }
                }
                for (int c = N - 1; c >= 0; --c) {            // backward (upper, reciprocal diagonal)
#pragma unroll
                    for (int k = 0; k < RPL; ++k)
                        if (lane + kWarp * k == c) b[k] *= J[c][c];
                    const float bc = row_value(c);
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + kWarp * k;
                        if (i < c) b[k] = fmaf(-J[i][c], bc, b[k]);
                    }
                }
                float mv = 0.0f;
#pragma unroll
                for (int k = 0; k < RPL; ++k)
                    if (lane + kWarp * k < N) mv = fmaxf(mv, nan_to_inf(fabsf(b[k]) * kg[k]));
                mv = warp_maxf(mv);
                if (!(mv <= (float)a.max_move)) break;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int i = lane + kWarp * k;
                    if (i < N) x[i] += (double)b[k];
                }
                last_move = mv;
                __syncwarp();
                rho = residual(false);
                __syncwarp();
                if ((double)rho < a.tol) ok = true;
            }
            if (ok) {
                for (int i = lane; i < N; i += kWarp) state[i] = x[i];
                if (lane == 0 && a.err_est) a.err_est[idx] = last_move > 0.0f ? last_move : rho;
            } else {
                if (lane == 0) {
                    a.status[idx] = GRINS_SS_POLISH_FAIL;
                    if (a.err_est) a.err_est[idx] = -1.0f;
                }
            }
            __syncwarp();
        }
    }
}

template <int NMAX, int WARPS>
cudaError_t launch_bucket(const PolishArgs &a, cudaStream_t st, int num_sms)
{
    auto kern = polish_kernel<NMAX, WARPS>;
    const long long dyn = WARPS * polish_edge_bytes(a.topo.E);
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    cudaFuncAttributes fa;
    err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    if (dyn + (long long)fa.sharedSizeBytes > optin) return cudaErrorInvalidConfiguration;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * kWarp, (size_t)dyn);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)num_sms * per_sm;
    const long long units = a.n_ics > 0 ? a.n_solves / a.n_ics * ((a.n_ics + kUnitIcs - 1) / kUnitIcs) : 0;
    const long long need = (units + WARPS - 1) / WARPS;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, WARPS * kWarp, (size_t)dyn, st>>>(a);
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

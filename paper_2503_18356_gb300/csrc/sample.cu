// Parameter and initial-condition sampler (Sec. 2.1.2, Table 1).
//
// One thread per (parameter set, Philox block): block c of set s yields the
// draws 4c .. 4c+3 of that set's stream, each mapped to one parameter.
// Draw layout of a set (2N + 3E draws):
//   [0, N) G_i   [N, 2N) k_i   [2N, 2N+E) threshold_e   [2N+E, 2N+2E) lambda_e
//   [2N+2E, 2N+3E) n_e
// Floating-point maps use explicit round-to-nearest intrinsics so that no
// multiply-add is contracted: the values are reproducible bit for bit.
#include "common.cuh"

namespace grins {

namespace {

__device__ __forceinline__ double affine_rn(double lo, double span, double u)
{
    return __dadd_rn(lo, __dmul_rn(span, u));
}

// A continuous parameter over [lo, hi] under a GRINS_DIST_* other than
// Table 1's: log-uniform, or normal / log-normal around the range's middle
// with a sixth of the range as standard deviation, clamped (Box-Muller on
// the draw's two 32-bit halves).  u is the draw's unit (stratified under a
// Latin hypercube), r the raw draw.  The steps are those of the host's
// draw; the log, exp and cos of the device agree with the host's to a few
// ulp.
__device__ double dist_draw(int dist, double lo, double hi, double u, uint64_t r)
{
    if (dist == GRINS_DIST_LOGUNIFORM) {
        const double a = log(lo), b = log(hi);
        return exp(affine_rn(a, __dsub_rn(b, a), u));
    }
    const double uh = __dmul_rn(__dadd_rn((double)(r >> 32), 0.5), 0x1.0p-32);
    const double ul = __dmul_rn(__dadd_rn((double)(r & 0xffffffffull), 0.5), 0x1.0p-32);
    const double z = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, log(uh))), cos(__dmul_rn(6.283185307179586, ul)));
    if (dist == GRINS_DIST_NORMAL) {
        const double x = __dadd_rn(__ddiv_rn(__dadd_rn(lo, hi), 2.0), __dmul_rn(z, __ddiv_rn(__dsub_rn(hi, lo), 6.0)));
        return fmin(hi, fmax(lo, x));
    }
    const double a = log(lo), b = log(hi);
    const double x = exp(__dadd_rn(__ddiv_rn(__dadd_rn(a, b), 2.0), __dmul_rn(z, __ddiv_rn(__dsub_rn(b, a), 6.0))));
    return fmin(hi, fmax(lo, x));
}

// Latin hypercube stratum of set s (< S) for draw index d: a keyed
// permutation of [0, S) -- a 4-round Feistel network on 2h bits (2^(2h) >=
// S) whose round function is word 0 of Philox4x64-10 at counter (d, round,
// right half, 0), key (seed, kTagLhs), walked until it lands below S.
__device__ uint64_t lhs_stratum(uint64_t seed, uint64_t d, uint64_t s, uint64_t S)
{
    int nb = 2;
    while (nb < 62 && (1ull << nb) < S) ++nb;
    const int h = (nb + 1) / 2;
    const uint64_t hm = (1ull << h) - 1ull;
    uint64_t x = s;
    do {
        uint64_t L = x >> h, R = x & hm;
        for (uint64_t rd = 0; rd < 4; ++rd) {
            const uint64_t F = philox4x64_10(d, rd, R, 0, seed, kTagLhs).v[0] & hm;
            const uint64_t t = L ^ F;
            L = R;
            R = t;
        }
        x = (L << h) | R;
    } while (x >= S);
    return x;
}

// Coordinate d of Sobol point s in Gray-code order: the shift XOR the
// direction numbers of the set bits of s ^ (s >> 1).
__device__ __forceinline__ double sobol_unit(const SampleArgs &a, uint64_t d, uint64_t s)
{
    const uint32_t *V = a.sobol_v + d * 32;
    uint32_t x = __ldg(a.sobol_v + (size_t)a.sobol_dims * 32 + d);
    for (uint64_t g = s ^ (s >> 1); g; g &= g - 1) x ^= __ldg(V + (__ffsll((long long)g) - 1));
    return __dmul_rn((double)x, 0x1.0p-32);
}

// The unit of draw d of set s: its own draw, under a Latin hypercube
// (stratum + draw) / S, or the Sobol coordinate.
__device__ __forceinline__ double draw_unit(const SampleArgs &a, uint64_t d, uint64_t s, uint64_t x)
{
    if (a.sobol_v) return sobol_unit(a, d, s);
    if (a.lhs_sets <= 0) return unit_double(x);
    const uint64_t p = lhs_stratum(a.seed, d, s, (uint64_t)a.lhs_sets);
    return __ddiv_rn(__dadd_rn((double)p, unit_double(x)), (double)a.lhs_sets);
}

// Draw d of a set from its per-parameter row (grins_param_range): G, k and
// lambda by the row's distribution (an inhibiting lambda under Table 1 in
// the inverse range), T as the row's multiplier range times the source's
// median, n uniform over the row's integers (stratified: floor(u count)).
__device__ __forceinline__ void row_draw(const SampleArgs &a, int d, double u, uint64_t x, double *G, double *k,
                                         double *T, double *lam, uint8_t *nn)
{
    const int N = a.L.N, E = a.L.E;
    const grins_param_range p = a.prange[d];
    if (d < 2 * N) {
        const double v = p.dist ? dist_draw(p.dist, p.lo, p.hi, u, x) : affine_rn(p.lo, __dsub_rn(p.hi, p.lo), u);
        if (d < N) G[d] = v; else k[d - N] = v;
    } else if (d < 2 * N + E) {
        const int e = d - 2 * N;
        T[e] = __dmul_rn(affine_rn(p.lo, __dsub_rn(p.hi, p.lo), u), a.edge_median[e]);
    } else if (d < 2 * N + 2 * E) {
        const int e = d - 2 * N - E;
        if (p.dist) lam[e] = dist_draw(p.dist, p.lo, p.hi, u, x);
        else if (a.edge_sign[e] > 0) lam[e] = affine_rn(p.lo, __dsub_rn(p.hi, p.lo), u);
        else {
            const double vlo = __ddiv_rn(1.0, p.hi);
            lam[e] = __ddiv_rn(1.0, affine_rn(vlo, __dsub_rn(__ddiv_rn(1.0, p.lo), vlo), u));
        }
    } else {
        const int e = d - 2 * N - 2 * E;
        const int lo = (int)p.lo, count = (int)p.hi - lo + 1;
        if (a.lhs_sets > 0 || a.sobol_v) {
            const int m = (int)__dmul_rn(u, (double)count);
            nn[e] = (uint8_t)(lo + (m < count ? m : count - 1));
        } else {
            nn[e] = (uint8_t)unit_int(x, lo, count);
        }
    }
}

// OTHER: some class uses a distribution besides Table 1's (a separate
// instantiation, so that the Table 1 kernel carries no log, exp or cos).
template <bool OTHER>
__global__ void sample_params_kernel(SampleArgs a)
{
    const int N = a.L.N, E = a.L.E;
    const int n_draws = 2 * N + 3 * E;
    const int blocks_per_set = (n_draws + 3) / 4;
    const int64_t total = a.n_sets * blocks_per_set;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s_local = gid / blocks_per_set;
        const int c = (int)(gid - s_local * blocks_per_set);
        const uint64_t s = (uint64_t)(a.set0 + s_local);
        U64x4 r = philox4x64_10(s, (uint64_t)c, 0, 0, a.seed, kTagParams);
        unsigned char *blk = a.params + s_local * a.L.stride;
        double *G = reinterpret_cast<double *>(blk + a.L.off_G);
        double *k = reinterpret_cast<double *>(blk + a.L.off_k);
        double *T = reinterpret_cast<double *>(blk + a.L.off_T);
        double *lam = reinterpret_cast<double *>(blk + a.L.off_lam);
        uint8_t *nn = blk + a.L.off_n;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int d = 4 * c + w;
            if (d >= n_draws) break;
            const uint64_t x = r.v[w];
            const double u = OTHER ? draw_unit(a, (uint64_t)d, s, x) : unit_double(x);
            if (OTHER && a.prange) {
                row_draw(a, d, u, x, G, k, T, lam, nn);
                continue;
            }
            if (d < N) {
                G[d] = OTHER && a.dist_G ? dist_draw(a.dist_G, a.G_min, a.G_hi, u, x) : affine_rn(a.G_min, a.G_span, u);
            } else if (d < 2 * N) {
                k[d - N] = OTHER && a.dist_k ? dist_draw(a.dist_k, a.k_min, a.k_hi, u, x)
                                             : affine_rn(a.k_min, a.k_span, u);
            } else if (d < 2 * N + E) {
                const int e = d - 2 * N;
                T[e] = __dmul_rn(affine_rn(a.thr_lo, a.thr_span, u), a.edge_median[e]);
            } else if (d < 2 * N + 2 * E) {
                const int e = d - 2 * N - E;
                const bool act = a.edge_sign[e] > 0;
                if (act) lam[e] = OTHER && a.dist_la ? dist_draw(a.dist_la, a.la_min, a.la_hi, u, x)
                                                     : affine_rn(a.la_min, a.la_span, u);
                else lam[e] = OTHER && a.dist_li ? dist_draw(a.dist_li, a.li_min, a.li_max, u, x)
                                                 : __ddiv_rn(1.0, affine_rn(a.vi_min, a.vi_span, u));
            } else {
                const int e = d - 2 * N - 2 * E;
                if (OTHER && (a.lhs_sets > 0 || a.sobol_v)) {
                    const int m = (int)__dmul_rn(u, (double)a.n_count);
                    nn[e] = (uint8_t)(a.n_min + (m < a.n_count ? m : a.n_count - 1));
                } else {
                    nn[e] = (uint8_t)unit_int(x, a.n_min, a.n_count);
                }
            }
        }
        // zero the tail padding once per set
        if (c == 0) {
            for (int64_t b = a.L.off_n + E; b < a.L.stride; ++b) blk[b] = 0;
        }
    }
}

// Unit initial conditions: u in [0, 1) per (IC, node), or, with rows, the
// fraction of G/k that row i's distribution gives over [lo, hi].
__global__ void sample_ics_kernel(int N, uint64_t seed, int n_ics, double *u, const grins_param_range *rows)
{
    const int blocks_per_ic = (N + 3) / 4;
    const int64_t total = (int64_t)n_ics * blocks_per_ic;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int ic = (int)(gid / blocks_per_ic);
        const int c = (int)(gid - (int64_t)ic * blocks_per_ic);
        U64x4 r = philox4x64_10((uint64_t)ic, (uint64_t)c, 0, 0, seed, kTagIcs);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int i = 4 * c + w;
            if (i >= N) continue;
            const double v = unit_double(r.v[w]);
            if (!rows) {
                u[(int64_t)ic * N + i] = v;
            } else {
                const grins_param_range p = rows[i];
                u[(int64_t)ic * N + i] = p.dist ? dist_draw(p.dist, p.lo, p.hi, v, r.v[w])
                                                : affine_rn(p.lo, __dsub_rn(p.hi, p.lo), v);
            }
        }
    }
}

int grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_sample_params(const SampleArgs &a, cudaStream_t st)
{
    if (a.n_sets <= 0) return cudaSuccess;
    const int n_draws = 2 * a.L.N + 3 * a.L.E;
    const int64_t work = a.n_sets * ((n_draws + 3) / 4);
    if (a.dist_G || a.dist_k || a.dist_la || a.dist_li || a.lhs_sets > 0 || a.sobol_v || a.prange)
        sample_params_kernel<true><<<grid_for(work, 256), 256, 0, st>>>(a);
    else
        sample_params_kernel<false><<<grid_for(work, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sample_ics(int N, uint64_t seed, int n_ics, double *u, const grins_param_range *rows,
                              cudaStream_t st)
{
    if (n_ics <= 0) return cudaSuccess;
    const int64_t work = (int64_t)n_ics * ((N + 3) / 4);
    sample_ics_kernel<<<grid_for(work, 256), 256, 0, st>>>(N, seed, n_ics, u, rows);
    return cudaGetLastError();
}

}  // namespace grins

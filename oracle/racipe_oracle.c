/*
 * RACIPE oracle: a plain, slow, FP64 CPU statement of what the RACIPE
 * ensemble path computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table
 * or constant generator with the CUDA library: every formula below is
 * restated from the paper (GRiNS, arXiv 2503.18356) and from the published
 * definitions of the numerical methods it names.
 *
 * Contents (each function cites the passage it follows):
 *   - Philox4x64-10 counter-based generator (Salmon et al., SC'11), the one
 *     random source of the sampler; pinned against numpy's Philox.
 *   - Shifted Hill function, Eq. 2, and the RACIPE node equation, Eq. 1.
 *   - Parameter and initial-condition sampling, Sec. 2.1.2 and Table 1,
 *     including the inverse-range inhibitory fold change and the
 *     half-functional threshold rule.
 *   - Dormand-Prince 5(4) with FSAL and step-size control (Dormand & Prince
 *     1980; Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4), run to the
 *     steady-state condition of Sec. 2.1.3, with optional output at grid
 *     times (Sec. 2.1.3, time series).
 *   - Newton polish of a converged state (steady state = Eq. 1 equal to 0).
 *   - Per-parameter-set steady-state dedupe (Sec. 3.1, multistability).
 *   - Tsitouras 5(4) (Tsitouras 2011), the paper's own integrator, as the
 *     second tableau of the same stepper.
 *   - Levels of G/k-normalised expression, level labels and the
 *     multistability histogram (Sec. 2.1.3, Sec. 3.1).
 *   - The Boolean Ising formalism, synchronous and asynchronous (Eq. 3).
 *   - Log-uniform, normal and log-normal parameter distributions, the
 *     Latin-hypercube and Sobol sets, the per-parameter range table with
 *     per-node medians, and initial conditions from per-node ranges (the
 *     samplers and the range file of Sec. 2.1.2).
 *
 * Parity status: every function here is pinned by a CPU test against
 * closed forms, library routines (numpy Philox, scipy DOP853, scipy
 * quadrature) or brute force; none is "parity unpinned".
 *
 * Compiled with -O2 -ffp-contract=off: every floating-point expression is
 * evaluated as written, one IEEE rounding per operation, no FMA.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Status codes of one solve (outcome of one (parameter set, IC) pair)  */
/* ------------------------------------------------------------------ */
enum { ORC_CONVERGED = 0, ORC_TEND = 1, ORC_MAXSTEPS = 2, ORC_NONFINITE = 3,
       ORC_POLISH_FAIL = 4 };

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11).  Ten rounds of the 4-word Philox S-box  */
/* with the published multipliers and Weyl key increments.              */
/* ------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                       uint64_t out[4])
{
    const uint64_t mult0 = 0xD2E7470EE14C6C93ULL;
    const uint64_t mult1 = 0xCA5A826395121157ULL;
    const uint64_t weyl0 = 0x9E3779B97F4A7C15ULL;  /* golden ratio */
    const uint64_t weyl1 = 0xBB67AE8584CAA73BULL;  /* sqrt(3) - 1 */
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)mult0 * x0;
        unsigned __int128 p1 = (unsigned __int128)mult1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Draw number d of the stream (key, c0): word d%4 of the block with
 * counter (c0, d/4, 0, 0). */
static uint64_t draw64(uint64_t key0, uint64_t key1, uint64_t c0, uint64_t d)
{
    uint64_t ctr[4] = { c0, d / 4, 0, 0 };
    uint64_t key[2] = { key0, key1 };
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return out[d % 4];
}

/* Uniform double in [0, 1) from the top 53 bits. */
double orc_u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* Uniform integer in [lo, hi] from the top 32 bits (multiply-shift). */
int32_t orc_uint_range(uint64_t r, int32_t lo, int32_t hi)
{
    uint64_t span = (uint64_t)(int64_t)(hi - lo + 1);
    return lo + (int32_t)(((r >> 32) * span) >> 32);
}

/* Stream keys (second key word; the first is the user's seed). */
#define ORC_TAG_PARAMS 0x52414349504550ULL  /* "RACIPEP" */
#define ORC_TAG_ICS    0x52414349504549ULL  /* "RACIPEI" */
#define ORC_KEY_MEDIAN 0x48414C4646554E43ULL /* "HALFFUNC", fixed */

/* ------------------------------------------------------------------ */
/* Parameter ranges, Table 1 (defaults set by orc_default_ranges).      */
/* ------------------------------------------------------------------ */
typedef struct {
    double G_min, G_max;           /* production rate */
    double k_min, k_max;           /* degradation rate */
    double lam_act_min, lam_act_max; /* activating fold change (>= 1) */
    double lam_inh_min, lam_inh_max; /* inhibiting fold change (<= 1) */
    int32_t n_min, n_max;          /* Hill coefficient, integer */
    double thr_lo, thr_hi;         /* half-functional factors */
    int32_t median_samples;        /* samples per median estimate */
    int32_t median_mode;           /* 0 = per in-degree class, 1 = unregulated */
    int32_t dist_G, dist_k, dist_lam_act, dist_lam_inh;   /* distribution per class, below */
    int64_t lhs_sets;              /* > 0: Latin hypercube over this many sets (below) */
    int32_t sobol;                 /* 0 off, 1 Sobol points, 2 scrambled (below) */
    int32_t sobol_dims;
    const int64_t *sobol_poly;     /* [sobol_dims] primitive polynomials, bit j = coeff. of x^j */
    const int64_t *sobol_m;        /* [sobol_dims][sobol_m_cols] initial m_1 .. m_s */
    int32_t sobol_m_cols;
    const struct orc_param_range *param_ranges;  /* [2N + 3E] rows, or NULL (below) */
} orc_ranges;

/* A per-parameter range row (Sec. 2.1.2: the parameter range file, with a */
/* distribution per parameter), rows in the order G[N], k[N], T[E],        */
/* lambda[E], n[E]: G, k, lambda by dist over [lo, hi] (an inhibiting      */
/* lambda under dist 0 in Table 1's inverse range); T the multiplier range */
/* of the source's median; n the integers lo..hi.                          */
typedef struct orc_param_range {
    int32_t dist, reserved;
    double lo, hi;
} orc_param_range;

void orc_default_ranges(orc_ranges *r)
{
    r->G_min = 1.0;   r->G_max = 100.0;
    r->k_min = 0.1;   r->k_max = 1.0;
    r->lam_act_min = 1.0;  r->lam_act_max = 100.0;
    r->lam_inh_min = 0.01; r->lam_inh_max = 1.0;
    r->n_min = 1; r->n_max = 6;
    r->thr_lo = 0.02; r->thr_hi = 1.98;
    r->median_samples = 10000;
    r->median_mode = 0;
    r->dist_G = r->dist_k = r->dist_lam_act = r->dist_lam_inh = 0;
    r->lhs_sets = 0;
    r->sobol = 0;
    r->sobol_dims = 0;
    r->sobol_poly = NULL;
    r->sobol_m = NULL;
    r->sobol_m_cols = 0;
    r->param_ranges = NULL;
}

/* Affine map of a unit draw onto [lo, hi]: lo + (hi - lo) * u. */
static double affine(double lo, double hi, double u) { return lo + (hi - lo) * u; }

/* The paper's samplers besides Table 1's (Sec. 2.1.2), for one continuous */
/* parameter over [lo, hi] from one 64-bit draw x: dist 0 uniform (Table 1),*/
/* 1 log-uniform: exp(U[log lo, log hi]), 2 normal: mean (lo + hi) / 2,    */
/* standard deviation (hi - lo) / 6, clamped to [lo, hi], 3 log-normal: the */
/* same in log space, then exp.  The normal deviate is Box-Muller on the    */
/* draw's two 32-bit halves h, l: u = (h + 1/2) 2^-32, v = (l + 1/2) 2^-32, */
/* z = sqrt(-2 log u) cos(2 pi v).                                          */
static double param_draw_u(int32_t dist, double lo, double hi, double uu, uint64_t x)
{
    if (dist == 1) return exp(affine(log(lo), log(hi), uu));
    if (dist == 2 || dist == 3) {
        double u = ((double)(x >> 32) + 0.5) * 0x1.0p-32;
        double v = ((double)(x & 0xffffffffULL) + 0.5) * 0x1.0p-32;
        double z = sqrt(-2.0 * log(u)) * cos(6.283185307179586 * v);
        double y;
        if (dist == 2) {
            y = (lo + hi) / 2.0 + z * ((hi - lo) / 6.0);
        } else {
            double a = log(lo), b = log(hi);
            y = exp((a + b) / 2.0 + z * ((b - a) / 6.0));
        }
        return y < lo ? lo : (y > hi ? hi : y);
    }
    return affine(lo, hi, uu);
}

static double param_draw(int32_t dist, double lo, double hi, uint64_t x)
{
    return param_draw_u(dist, lo, hi, orc_u01(x), x);
}

/* Activating fold change: uniform on [lam_act_min, lam_act_max] (Table 1),
 * or the class's distribution; uu is the draw's unit. */
static double lam_activating_u(const orc_ranges *r, double uu, uint64_t x)
{
    return param_draw_u(r->dist_lam_act, r->lam_act_min, r->lam_act_max, uu, x);
}

/* Inhibiting fold change, Sec. 2.1.2: drawn uniformly in the inverse range
 * [1/max, 1/min] and then inverted (Table 1), or the class's distribution
 * over [lam_inh_min, lam_inh_max]. */
static double lam_inhibiting_u(const orc_ranges *r, double uu, uint64_t x)
{
    if (r->dist_lam_inh != 0) return param_draw_u(r->dist_lam_inh, r->lam_inh_min, r->lam_inh_max, uu, x);
    double v_lo = 1.0 / r->lam_inh_max;
    double v_hi = 1.0 / r->lam_inh_min;
    return 1.0 / affine(v_lo, v_hi, uu);
}

static double lam_activating(const orc_ranges *r, uint64_t x) { return lam_activating_u(r, orc_u01(x), x); }
static double lam_inhibiting(const orc_ranges *r, uint64_t x) { return lam_inhibiting_u(r, orc_u01(x), x); }

/* Latin hypercube (Sec. 2.1.2, the paper's other samplers): with       */
/* lhs_sets = S > 0, draw d of set s < S takes the unit (p + u) / S,    */
/* u its own draw and p = pi_d(s), pi_d a keyed permutation of [0, S):  */
/* a balanced 4-round Feistel network on 2h bits (h = ceil(b / 2), b    */
/* the bits of S - 1, at least 2), round function word 0 of             */
/* Philox4x64-10 at counter (d, round, right half, 0) with key (seed,   */
/* ORC_TAG_LHS) masked to h bits, applied again while the result is     */
/* not below S (cycle walking, Black and Rogaway 2002).                 */
#define ORC_TAG_LHS 0x5241434950454CULL    /* "RACIPEL" */

uint64_t orc_lhs_stratum(uint64_t seed, uint64_t d, uint64_t s, uint64_t S)
{
    int b = 2;
    while (b < 62 && (1ULL << b) < S) ++b;
    int h = (b + 1) / 2;
    uint64_t hm = (1ULL << h) - 1ULL, x = s;
    do {
        uint64_t L = x >> h, R = x & hm;
        for (uint64_t rd = 0; rd < 4; ++rd) {
            uint64_t ctr[4] = { d, rd, R, 0 }, key[2] = { seed, ORC_TAG_LHS }, out[4];
            orc_philox4x64_10(ctr, key, out);
            uint64_t nR = L ^ (out[0] & hm);
            L = R;
            R = nR;
        }
        x = (L << h) | R;
    } while (x >= S);
    return x;
}

/* Sobol sequence (Sec. 2.1.2, the paper's default sampler).  Coordinate */
/* d of point s, as a 32-bit integer x (the unit is x 2^-32):           */
/*  - direction integers (Bratley and Fox 1988): dimension 0 has m_k = 1; */
/*    dimension d >= 1, with primitive polynomial                        */
/*    x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1, takes its given m_1..m_s    */
/*    and m_k = m_(k-s) XOR 2^s m_(k-s) XOR sum_i 2^i a_i m_(k-i) beyond;  */
/*    direction number b (0-based) is m_(b+1) 2^(31-b);                  */
/*  - point s in Gray-code order (Antonov and Saleev 1979): the XOR of    */
/*    the direction numbers of the set bits of s XOR (s >> 1);           */
/*  - scrambled (Matousek 1998): digit j of the result (j = 1 the most   */
/*    significant) is the parity of x AND M_j, M_j = digit j plus the     */
/*    digits above it taken from the low 32 bits of Philox4x64-10 word 0  */
/*    at counter (d, j, 0, 0), key (seed, ORC_TAG_SOBOL); then XOR the     */
/*    low 32 bits of word 0 at counter (d, 0, 0, 0) (digital shift).      */
#define ORC_TAG_SOBOL 0x52414349504553ULL  /* "RACIPES" */

static uint32_t low32_draw(uint64_t seed, uint64_t d, uint64_t j)
{
    uint64_t ctr[4] = { d, j, 0, 0 }, key[2] = { seed, ORC_TAG_SOBOL }, out[4];
    orc_philox4x64_10(ctr, key, out);
    return (uint32_t)(out[0] & 0xFFFFFFFFULL);
}

uint32_t orc_sobol_x(const orc_ranges *r, uint64_t seed, uint64_t d, uint64_t s)
{
    uint64_t m[33];
    if (d == 0) {
        for (int k = 1; k <= 32; ++k) m[k] = 1;
    } else {
        uint64_t p = (uint64_t)r->sobol_poly[d];
        int deg = 0;
        for (int j = 0; j < 64; ++j) if ((p >> j) & 1ULL) deg = j;
        for (int k = 1; k <= deg; ++k) m[k] = (uint64_t)r->sobol_m[d * (uint64_t)r->sobol_m_cols + (uint64_t)(k - 1)];
        for (int k = deg + 1; k <= 32; ++k) {
            uint64_t v = m[k - deg] ^ (m[k - deg] << deg);
            for (int i = 1; i <= deg - 1; ++i) {
                uint64_t a_i = (p >> (deg - i)) & 1ULL;
                if (a_i) v ^= m[k - i] << i;
            }
            m[k] = v;
        }
    }
    uint64_t g = s ^ (s >> 1);
    uint32_t x = 0;
    for (int b = 0; b < 32; ++b)
        if ((g >> b) & 1ULL) x ^= (uint32_t)(m[b + 1] << (31 - b));
    if (r->sobol != 2) return x;
    uint32_t y = 0;
    for (int j = 1; j <= 32; ++j) {
        int bit = 32 - j;
        uint32_t Mj = 1U << bit;
        if (j >= 2) Mj |= low32_draw(seed, d, (uint64_t)j) & (0xFFFFFFFFU << (bit + 1));
        uint32_t t = x & Mj, par = 0;
        while (t) { par ^= 1U; t &= t - 1U; }
        y |= par << bit;
    }
    return y ^ low32_draw(seed, d, 0);
}

/* The unit of draw d of set s: u01 of its draw, the stratified one, or the
 * Sobol coordinate. */
static double unit_of(const orc_ranges *r, uint64_t seed, uint64_t d, uint64_t s, uint64_t x)
{
    if (r->sobol) return (double)orc_sobol_x(r, seed, d, s) * 0x1p-32;
    if (r->lhs_sets <= 0) return orc_u01(x);
    return ((double)orc_lhs_stratum(seed, d, s, (uint64_t)r->lhs_sets) + orc_u01(x)) / (double)r->lhs_sets;
}

/* ------------------------------------------------------------------ */
/* Shifted Hill function, Eq. 2, written exactly as printed:            */
/*   H = B0^n / (B0^n + B^n) + lambda * B^n / (B0^n + B^n).             */
/* B is an expression level; negative values (which the model never    */
/* produces) are read as 0.                                            */
/* ------------------------------------------------------------------ */
double orc_shifted_hill(double B, double B0, double n, double lam)
{
    if (B < 0.0) B = 0.0;
    double b0n = pow(B0, n);
    double bn = pow(B, n);
    return b0n / (b0n + bn) + lam * bn / (b0n + bn);
}

/* One edge's factor in Eq. 1: H/lambda for an activating edge, H for an
 * inhibiting one. */
static double edge_factor(int sign, double B, double T, double n, double lam)
{
    double h = orc_shifted_hill(B, T, n, lam);
    return sign > 0 ? h / lam : h;
}

/* ------------------------------------------------------------------ */
/* Network (signed, directed edge list, Sec. 2.1.1).                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n_nodes, n_edges;
    const int32_t *src, *dst;
    const int8_t *sign;            /* +1 activation, -1 inhibition */
} orc_net;

/* One parameter set, 2N + 3E values (Sec. 2.1.2). */
typedef struct {
    const double *G, *k;           /* [N] */
    const double *T, *lam;         /* [E] */
    const int32_t *n;              /* [E] */
} orc_params;

/* Eq. 1: f_i(x) = G_i * prod_{e into i} factor_e(x_src(e)) - k_i * x_i. */
void orc_rhs(const orc_net *net, const orc_params *p, const double *x, double *f)
{
    int N = net->n_nodes;
    for (int i = 0; i < N; ++i) f[i] = p->G[i];
    for (int e = 0; e < net->n_edges; ++e) {
        int s = net->src[e], t = net->dst[e];
        f[t] = f[t] * edge_factor(net->sign[e], x[s], p->T[e], (double)p->n[e], p->lam[e]);
    }
    for (int i = 0; i < N; ++i) f[i] = f[i] - p->k[i] * x[i];
}

/* Steady-state residual: rho(x) = max_i |f_i| / (G_i / k_i). */
static double residual_rho(int N, const orc_params *p, const double *f)
{
    double rho = 0.0;
    for (int i = 0; i < N; ++i) {
        double r = fabs(f[i]) / (p->G[i] / p->k[i]);
        if (!(r <= rho)) rho = r;   /* NaN propagates */
    }
    return rho;
}

double orc_rho(const orc_net *net, const orc_params *p, const double *x)
{
    double f[1024];
    if (net->n_nodes > 1024) return NAN;
    orc_rhs(net, p, x, f);
    return residual_rho(net->n_nodes, p, f);
}

/* ------------------------------------------------------------------ */
/* Half-functional rule (Table 1 threshold row; Sec. 2.1.2).            */
/* The threshold of an edge out of node j is U[thr_lo, thr_hi] times    */
/* the median steady-state level M_j of node j.  For an unregulated j   */
/* the steady state is G/k, so M0 = median(G/k).  For a j with `a`      */
/* activating and `b` inhibiting inputs, the level is simulated from    */
/* its regulation: (G/k) * prod over inputs of the edge factor, each    */
/* input at an unregulated level G'/k', with its threshold drawn from   */
/* U[thr_lo, thr_hi] * M0 and n, lambda from Table 1.  The median over  */
/* `median_samples` seeded samples is M(a, b).  Draw layout of sample   */
/* s: 0 -> G, 1 -> k, then per input m (activating ones first) the five */
/* draws 2+5m .. 6+5m -> G', k', threshold, lambda, n.                  */
/* ------------------------------------------------------------------ */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double median_of(double *v, int K)
{
    qsort(v, (size_t)K, sizeof(double), cmp_double);
    if (K % 2 == 1) return v[K / 2];
    return (v[K / 2 - 1] + v[K / 2]) / 2.0;
}

/* Fills out[0..K) with the samples of class (a, b) given M0 (unused for
 * a = b = 0).  Exposed for the tests. */
void orc_median_samples(int32_t a, int32_t b, const orc_ranges *r, double M0,
                        double *out)
{
    int K = r->median_samples;
    uint64_t key1 = ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
    for (int s = 0; s < K; ++s) {
        double G = param_draw(r->dist_G, r->G_min, r->G_max, draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 0));
        double k = param_draw(r->dist_k, r->k_min, r->k_max, draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 1));
        double level = G / k;
        for (int m = 0; m < a + b; ++m) {
            uint64_t d = 2 + 5 * (uint64_t)m;
            double Gs = param_draw(r->dist_G, r->G_min, r->G_max, draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 0));
            double ks = param_draw(r->dist_k, r->k_min, r->k_max, draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 1));
            double T = affine(r->thr_lo, r->thr_hi, orc_u01(draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 2))) * M0;
            uint64_t xl = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 3);
            int32_t n = orc_uint_range(draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 4), r->n_min, r->n_max);
            int sign = m < a ? +1 : -1;
            double lam = sign > 0 ? lam_activating(r, xl) : lam_inhibiting(r, xl);
            level = level * edge_factor(sign, Gs / ks, T, (double)n, lam);
        }
        out[s] = level;
    }
}

double orc_median(int32_t a, int32_t b, const orc_ranges *r)
{
    int K = r->median_samples;
    double *v = (double *)malloc(sizeof(double) * (size_t)K);
    if (!v) return NAN;
    orc_median_samples(0, 0, r, 0.0, v);
    double M0 = median_of(v, K);
    double M = M0;
    if ((a != 0 || b != 0) && r->median_mode == 0) {
        orc_median_samples(a, b, r, M0, v);
        M = median_of(v, K);
    }
    free(v);
    return M;
}

/* ------------------------------------------------------------------ */
/* Sampling, Sec. 2.1.2 and Table 1.  Parameter set s uses the stream  */
/* key (seed, TAG_PARAMS), counter word 0 = s, draws:                   */
/*   [0, N)        G_i          [N, 2N)        k_i                      */
/*   [2N, 2N+E)    threshold_e  [2N+E, 2N+2E)  lambda_e                 */
/*   [2N+2E, 2N+3E) n_e                                                 */
/* IC number c uses key (seed, TAG_ICS), counter word 0 = c, draw i ->  */
/* the unit level u_{c,i}; the initial condition of node i under set s  */
/* is u_{c,i} * G_i / k_i (Sec. 2.1.2, between a node's minimum 0 and   */
/* maximum G/k; the same unit ICs are used for every set, Sec. 3.1).    */
/* ------------------------------------------------------------------ */
/* A continuous parameter from its row: G, k, activating lambda by the    */
/* row's distribution; an inhibiting lambda under dist 0 in the inverse    */
/* range [1/hi, 1/lo], inverted (Table 1's rule).                          */
static double row_param(const orc_param_range *p, int inh, double uu, uint64_t x)
{
    if (inh && p->dist == 0) return 1.0 / affine(1.0 / p->hi, 1.0 / p->lo, uu);
    return param_draw_u(p->dist, p->lo, p->hi, uu, x);
}

/* Sets from a per-parameter table: the class sampler's draws and units,  */
/* each parameter taking its own row.                                      */
static void sample_rows(const orc_net *net, const orc_ranges *r, uint64_t seed, int64_t set0, int64_t n_sets,
                        const double *Msrc, double *G, double *k, double *T, double *lam, int32_t *n)
{
    int N = net->n_nodes, E = net->n_edges;
    const orc_param_range *P = r->param_ranges;
    int strat = r->lhs_sets > 0 || r->sobol;
    for (int64_t s = 0; s < n_sets; ++s) {
        uint64_t c0 = (uint64_t)(set0 + s);
        for (int d = 0; d < 2 * N + 3 * E; ++d) {
            uint64_t x = draw64(seed, ORC_TAG_PARAMS, c0, (uint64_t)d);
            double uu = unit_of(r, seed, (uint64_t)d, c0, x);
            const orc_param_range *p = &P[d];
            if (d < N) G[s * N + d] = row_param(p, 0, uu, x);
            else if (d < 2 * N) k[s * N + (d - N)] = row_param(p, 0, uu, x);
            else if (d < 2 * N + E) {
                int e = d - 2 * N;
                T[s * E + e] = affine(p->lo, p->hi, uu) * Msrc[net->src[e]];
            } else if (d < 2 * N + 2 * E) {
                int e = d - 2 * N - E;
                lam[s * E + e] = row_param(p, net->sign[e] < 0, uu, x);
            } else {
                int e = d - 2 * N - 2 * E;
                int lo = (int)p->lo, hi = (int)p->hi, cnt = hi - lo + 1;
                if (strat) {
                    int m = (int)(uu * (double)cnt);
                    n[s * E + e] = lo + (m < cnt ? m : cnt - 1);
                } else {
                    n[s * E + e] = orc_uint_range(x, lo, hi);
                }
            }
        }
    }
}

/* The half-functional medians M_j of every node (Sec. 2.1.2).  Class      */
/* ranges: the median of node j's in-degree class (orc_median).  A         */
/* per-parameter table: node j's own rows -- first its unregulated median  */
/* M0_j, the median of G_j / k_j over median_samples draws (stream key     */
/* (ORC_KEY_MEDIAN, 2^63 + 2j), draws 0 and 1); then, if j has inputs and  */
/* the per-in-degree mode is on, the median of G_j / k_j times the Hill    */
/* factor of each in-edge (edge order; the q-th in-edge takes draws 2 + 5q */
/* .. 6 + 5q: G and k of its source from the source's rows, the threshold  */
/* multiplier from the edge's T row times M0 of the source, lambda and n   */
/* from the edge's rows), key (ORC_KEY_MEDIAN, 2^63 + 2j + 1).              */
void orc_node_medians(const orc_net *net, const orc_ranges *r, double *M)
{
    int N = net->n_nodes, E = net->n_edges;
    if (!r->param_ranges) {
        for (int j = 0; j < N; ++j) {
            int a = 0, b = 0;
            for (int e = 0; e < E; ++e)
                if (net->dst[e] == j) { if (net->sign[e] > 0) ++a; else ++b; }
            M[j] = orc_median(a, b, r);
        }
        return;
    }
    const orc_param_range *P = r->param_ranges;
    int K = r->median_samples;
    double *v = (double *)malloc(sizeof(double) * (size_t)K);
    double *M0 = (double *)malloc(sizeof(double) * (size_t)N);
    for (int j = 0; j < N; ++j) {
        uint64_t key1 = (1ULL << 63) + 2ULL * (uint64_t)j;
        for (int s = 0; s < K; ++s) {
            uint64_t xg = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 0);
            uint64_t xk = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 1);
            v[s] = row_param(&P[j], 0, orc_u01(xg), xg) / row_param(&P[N + j], 0, orc_u01(xk), xk);
        }
        M0[j] = median_of(v, K);
        M[j] = M0[j];
    }
    for (int j = 0; j < N && r->median_mode == 0; ++j) {
        int has_inputs = 0;
        for (int e = 0; e < E; ++e) if (net->dst[e] == j) has_inputs = 1;
        if (!has_inputs) continue;
        uint64_t key1 = (1ULL << 63) + 2ULL * (uint64_t)j + 1ULL;
        for (int s = 0; s < K; ++s) {
            uint64_t xg = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 0);
            uint64_t xk = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, 1);
            double level = row_param(&P[j], 0, orc_u01(xg), xg) / row_param(&P[N + j], 0, orc_u01(xk), xk);
            int q = 0;
            for (int e = 0; e < E; ++e) {
                if (net->dst[e] != j) continue;
                int src = net->src[e];
                uint64_t d = 2 + 5 * (uint64_t)q;
                uint64_t x0 = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 0);
                uint64_t x1 = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 1);
                uint64_t x2 = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 2);
                uint64_t x3 = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 3);
                uint64_t x4 = draw64(ORC_KEY_MEDIAN, key1, (uint64_t)s, d + 4);
                double Gs = row_param(&P[src], 0, orc_u01(x0), x0);
                double ks = row_param(&P[N + src], 0, orc_u01(x1), x1);
                const orc_param_range *pt = &P[2 * N + e], *pl = &P[2 * N + E + e], *pn = &P[2 * N + 2 * E + e];
                double Tq = affine(pt->lo, pt->hi, orc_u01(x2)) * M0[src];
                double lq = row_param(pl, net->sign[e] < 0, orc_u01(x3), x3);
                int32_t nq = orc_uint_range(x4, (int32_t)pn->lo, (int32_t)pn->hi);
                level = level * edge_factor(net->sign[e], Gs / ks, Tq, (double)nq, lq);
                ++q;
            }
            v[s] = level;
        }
        M[j] = median_of(v, K);
    }
    free(v);
    free(M0);
}

void orc_sample_params(const orc_net *net, const orc_ranges *r, uint64_t seed,
                       int64_t set0, int64_t n_sets,
                       double *G, double *k, double *T, double *lam, int32_t *n)
{
    int N = net->n_nodes, E = net->n_edges;
    /* Median per source node (class or per-parameter). */
    double *Msrc = (double *)malloc(sizeof(double) * (size_t)N);
    orc_node_medians(net, r, Msrc);
    if (r->param_ranges) {
        sample_rows(net, r, seed, set0, n_sets, Msrc, G, k, T, lam, n);
        free(Msrc);
        return;
    }
    for (int64_t s = 0; s < n_sets; ++s) {
        uint64_t c0 = (uint64_t)(set0 + s);
        double *Gs = G + s * N, *ks = k + s * N, *Ts = T + s * E, *ls = lam + s * E;
        int32_t *ns = n + s * E;
        for (int i = 0; i < N; ++i) {
            uint64_t xg = draw64(seed, ORC_TAG_PARAMS, c0, (uint64_t)i);
            uint64_t xk = draw64(seed, ORC_TAG_PARAMS, c0, (uint64_t)(N + i));
            Gs[i] = param_draw_u(r->dist_G, r->G_min, r->G_max, unit_of(r, seed, (uint64_t)i, c0, xg), xg);
            ks[i] = param_draw_u(r->dist_k, r->k_min, r->k_max, unit_of(r, seed, (uint64_t)(N + i), c0, xk), xk);
        }
        for (int e = 0; e < E; ++e) {
            uint64_t dt = (uint64_t)(2 * N + e), dl = (uint64_t)(2 * N + E + e), dn = (uint64_t)(2 * N + 2 * E + e);
            uint64_t xt = draw64(seed, ORC_TAG_PARAMS, c0, dt);
            uint64_t xl = draw64(seed, ORC_TAG_PARAMS, c0, dl);
            uint64_t rn = draw64(seed, ORC_TAG_PARAMS, c0, dn);
            double ul = unit_of(r, seed, dl, c0, xl);
            Ts[e] = affine(r->thr_lo, r->thr_hi, unit_of(r, seed, dt, c0, xt)) * Msrc[net->src[e]];
            ls[e] = net->sign[e] > 0 ? lam_activating_u(r, ul, xl) : lam_inhibiting_u(r, ul, xl);
            if (r->lhs_sets > 0 || r->sobol) {
                int cnt = r->n_max - r->n_min + 1;
                int m = (int)(unit_of(r, seed, dn, c0, rn) * (double)cnt);
                ns[e] = r->n_min + (m < cnt ? m : cnt - 1);
            } else {
                ns[e] = orc_uint_range(rn, r->n_min, r->n_max);
            }
        }
    }
    free(Msrc);
}

void orc_sample_ics(int32_t n_nodes, uint64_t seed, int32_t n_ics, double *u)
{
    for (int c = 0; c < n_ics; ++c)
        for (int i = 0; i < n_nodes; ++i)
            u[(int64_t)c * n_nodes + i] = orc_u01(draw64(seed, ORC_TAG_ICS, (uint64_t)c, (uint64_t)i));
}

/* Initial conditions from updated ranges (Sec. 2.1.2: regenerated from the */
/* range file, with a distribution per node): the same draw as above, the  */
/* fraction of node i's maximum G_i / k_i taken by row i's distribution    */
/* over [lo, hi] instead of uniformly over [0, 1).                          */
void orc_sample_ics_ranges(int32_t n_nodes, uint64_t seed, int32_t n_ics, const orc_param_range *rows, double *u)
{
    for (int c = 0; c < n_ics; ++c)
        for (int i = 0; i < n_nodes; ++i) {
            uint64_t x = draw64(seed, ORC_TAG_ICS, (uint64_t)c, (uint64_t)i);
            u[(int64_t)c * n_nodes + i] = param_draw(rows[i].dist, rows[i].lo, rows[i].hi, x);
        }
}

/* ------------------------------------------------------------------ */
/* Dormand-Prince 5(4) (Dormand & Prince 1980, "A family of embedded    */
/* Runge-Kutta formulae"), seven stages, first-same-as-last.            */
/* ------------------------------------------------------------------ */
static const double DP_C[7] = { 0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0 };
static const double DP_A[7][6] = {
    { 0 },
    { 1.0 / 5.0 },
    { 3.0 / 40.0, 9.0 / 40.0 },
    { 44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0 },
    { 19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0 },
    { 9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0 },
    { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0 },
};
/* 5th-order weights (equal to the last row of A) and embedded 4th order. */
static const double DP_B5[7] = { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                                 -2187.0 / 6784.0, 11.0 / 84.0, 0.0 };
static const double DP_B4[7] = { 5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                 -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0 };

/* ------------------------------------------------------------------ */
/* Tsitouras 5(4) (Ch. Tsitouras 2011, "Runge-Kutta pairs of order 5(4) */
/* satisfying only the first column simplifying assumption", Comput.    */
/* Math. Appl. 62), seven stages, first-same-as-last: the paper's       */
/* solver (diffrax Tsit5, Sec. 3.1).  The 5th-order weights are the last*/
/* row of A; the embedded weights are written as b5 - (b5 - b4) with    */
/* the published error coefficients b5 - b4.                            */
/* ------------------------------------------------------------------ */
static const double TS_C[7] = { 0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0 };
static const double TS_A[7][6] = {
    { 0 },
    { 0.161 },
    { -0.008480655492356989, 0.335480655492357 },
    { 2.897153057105493, -6.359448489975075, 4.3622954328695815 },
    { 5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525 },
    { 5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401, -0.028269050394068383 },
    { 0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081,
      2.324710524099774 },
};
static const double TS_B5[7] = { 0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742,
                                 -3.290069515436081, 2.324710524099774, 0.0 };
static const double TS_B4[7] = {
    0.09646076681806523 - -0.00178001105222577714, 0.01 - -0.0008164344596567469,
    0.4798896504144996 - 0.007880878010261995, 1.379008574103742 - -0.1447110071732629,
    -3.290069515436081 - 0.5823571654525552, 2.324710524099774 - -0.45808210592918697,
    0.0 - 0.015151515151515152 };

typedef struct {
    const double *c, (*a)[6], *b5, *b4;
} orc_tableau_t;

static orc_tableau_t tableau_of(int32_t method)
{
    orc_tableau_t t = { DP_C, DP_A, DP_B5, DP_B4 };
    if (method == 1) { t.c = TS_C; t.a = TS_A; t.b5 = TS_B5; t.b4 = TS_B4; }
    return t;
}

/* The Butcher tableau of a method (0 Dormand-Prince, 1 Tsitouras) for   */
/* tests: c[7], a[7][7] (row-major, zero above the diagonal), b5, b4.    */
void orc_tableau(int32_t method, double *c, double *a, double *b5, double *b4)
{
    orc_tableau_t t = tableau_of(method);
    for (int i = 0; i < 7; ++i) {
        c[i] = t.c[i]; b5[i] = t.b5[i]; b4[i] = t.b4[i];
        for (int j = 0; j < 7; ++j) a[i * 7 + j] = j < i && j < 6 ? t.a[i][j] : 0.0;
    }
}

typedef struct {
    double rtol, atol, t0, t_end, ss_tol;
    int64_t max_steps;
    const double *t_grid;          /* NULL: no time series */
    int32_t n_t;
    double h_fixed;                /* > 0: fixed step, no control, no steady-state stop */
    int32_t method;                /* 0 Dormand-Prince 5(4), 1 Tsitouras 5(4) */
} orc_opts;

typedef struct {
    int32_t status;
    double t_final;
    int64_t n_attempts, n_accepted;
} orc_result;

#define ORC_NMAX 256

/* One step of size h of the 5(4) pair t from (y, k1 = f(y)); fills      */
/* k[0..6], y5, y4.                                                      */
static void dp5_step(const orc_net *net, const orc_params *p, const orc_tableau_t *t, const double *y,
                     double h, double k[7][ORC_NMAX], double *y5, double *y4)
{
    int N = net->n_nodes;
    double z[ORC_NMAX];
    for (int s = 1; s < 7; ++s) {
        for (int i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc = acc + t->a[s][j] * k[j][i];
            z[i] = y[i] + h * acc;
        }
        orc_rhs(net, p, z, k[s]);
    }
    for (int i = 0; i < N; ++i) {
        double a5 = 0.0, a4 = 0.0;
        for (int j = 0; j < 7; ++j) { a5 = a5 + t->b5[j] * k[j][i]; a4 = a4 + t->b4[j] * k[j][i]; }
        y5[i] = y[i] + h * a5;
        y4[i] = y[i] + h * a4;
    }
}

static double rms_scaled(int N, const double *v, const double *y, const double *y2,
                         double atol, double rtol)
{
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
        double m = fabs(y[i]);
        if (y2 && fabs(y2[i]) > m) m = fabs(y2[i]);
        double q = v[i] / (atol + rtol * m);
        s = s + q * q;
    }
    return sqrt(s / N);
}

static int all_finite(int N, const double *v)
{
    for (int i = 0; i < N; ++i) if (!isfinite(v[i])) return 0;
    return 1;
}

/* Integrates Eq. 1 from x0 at t0 until the steady-state condition
 * (Sec. 2.1.3) rho(f(y)) < ss_tol holds at an accepted step, or t_end is
 * reached, or max_steps attempts are spent.  With a time grid, steps are
 * shortened to land on every grid time and the state there is written to
 * series[g * N + i]; grid times after termination get the final state.
 * With h_fixed > 0 the method runs with that fixed step to t_end (used to
 * measure its order).  o->method picks the 5(4) pair: 0 Dormand-Prince,
 * 1 Tsitouras (the paper's solver); both take the step control above. */
orc_result orc_solve(const orc_net *net, const orc_params *p, const double *x0,
                     const orc_opts *o, double *x_out, double *series)
{
    int N = net->n_nodes;
    orc_result res = { ORC_TEND, o->t0, 0, 0 };
    const orc_tableau_t tab = tableau_of(o->method);
    double y[ORC_NMAX], y5[ORC_NMAX], y4[ORC_NMAX], err[ORC_NMAX];
    double k[7][ORC_NMAX];
    memcpy(y, x0, sizeof(double) * N);
    double t = o->t0;
    int g = 0;                     /* next grid index */
    while (series && g < o->n_t && o->t_grid[g] <= t) {
        memcpy(series + (int64_t)g * N, y, sizeof(double) * N); ++g;
    }
    orc_rhs(net, p, y, k[0]);
    int fixed = o->h_fixed > 0.0;
    if (!fixed && residual_rho(N, p, k[0]) < o->ss_tol) {
        res.status = ORC_CONVERGED;
        goto finish;
    }
    double h;
    if (fixed) {
        h = o->h_fixed;
    } else {
        /* Starting step (Hairer, Norsett & Wanner, Sec. II.4). */
        double d0 = rms_scaled(N, y, y, NULL, o->atol, o->rtol);
        double d1 = rms_scaled(N, k[0], y, NULL, o->atol, o->rtol);
        double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        double y1[ORC_NMAX], f1[ORC_NMAX], df[ORC_NMAX];
        for (int i = 0; i < N; ++i) y1[i] = y[i] + h0 * k[0][i];
        orc_rhs(net, p, y1, f1);
        for (int i = 0; i < N; ++i) df[i] = f1[i] - k[0][i];
        double d2 = rms_scaled(N, df, y, NULL, o->atol, o->rtol) / h0;
        double dm = d1 > d2 ? d1 : d2;
        double h1 = dm <= 1e-15 ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / 5.0);
        h = fmin(100.0 * h0, h1);
    }
    double span = o->t_end - o->t0;
    if (h > span) h = span;
    int rejected = 0;
    for (;;) {
        if (t >= o->t_end) { res.status = ORC_TEND; break; }
        if (res.n_attempts >= o->max_steps) { res.status = ORC_MAXSTEPS; break; }
        /* Land exactly on the next grid time or on t_end. */
        double h_try = h;
        double t_stop = o->t_end;
        int to_grid = 0;
        if (series && g < o->n_t && o->t_grid[g] < t_stop) { t_stop = o->t_grid[g]; to_grid = 1; }
        int clipped = 0;
        if (t + h_try >= t_stop) { h_try = t_stop - t; clipped = 1; }
        dp5_step(net, p, &tab, y, h_try, k, y5, y4);
        res.n_attempts++;
        for (int i = 0; i < N; ++i) err[i] = y5[i] - y4[i];
        if (!all_finite(N, y5) || !all_finite(N, k[6])) { res.status = ORC_NONFINITE; break; }
        double en = fixed ? 0.0 : rms_scaled(N, err, y, y5, o->atol, o->rtol);
        if (!isfinite(en)) { res.status = ORC_NONFINITE; break; }
        if (en < 1.0) {
            res.n_accepted++;
            t = clipped ? t_stop : t + h_try;
            memcpy(y, y5, sizeof(double) * N);
            memcpy(k[0], k[6], sizeof(double) * N);   /* first same as last */
            if (clipped && to_grid) {
                while (g < o->n_t && o->t_grid[g] <= t) {
                    memcpy(series + (int64_t)g * N, y, sizeof(double) * N); ++g;
                }
            }
            if (!fixed && residual_rho(N, p, k[0]) < o->ss_tol) { res.status = ORC_CONVERGED; break; }
            if (!fixed) {
                /* Step-size controller: safety 0.9, factor in [0.2, 10],
                 * no growth right after a rejected attempt. */
                double fac = en == 0.0 ? 10.0 : 0.9 * pow(en, -1.0 / 5.0);
                if (fac > 10.0) fac = 10.0;
                if (rejected && fac > 1.0) fac = 1.0;
                h = h_try * fac;
            }
            rejected = 0;
        } else {
            double fac = 0.9 * pow(en, -1.0 / 5.0);
            if (fac < 0.2) fac = 0.2;
            h = h_try * fac;
            rejected = 1;
        }
        if (!fixed && h < 1e-14 * (fabs(t) > 1.0 ? fabs(t) : 1.0)) { res.status = ORC_NONFINITE; break; }
    }
finish:
    res.t_final = t;
    memcpy(x_out, y, sizeof(double) * N);
    while (series && g < o->n_t) {
        memcpy(series + (int64_t)g * N, y, sizeof(double) * N); ++g;
    }
    return res;
}

/* ------------------------------------------------------------------ */
/* Newton polish.  A steady state is a zero of Eq. 1.  From the state   */
/* the integrator stopped at, Newton iterations x <- x + d with         */
/* J d = -f(x), J by central differences, solved by Gaussian            */
/* elimination with partial pivoting, until rho(x) < tol.               */
/* Returns 0 when rho < tol, 1 when max_iter is spent, 2 if J singular. */
/* ------------------------------------------------------------------ */
static int lu_solve(int N, double *A, double *b)
{
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r) if (fabs(A[r * N + c]) > fabs(A[piv * N + c])) piv = r;
        if (A[piv * N + c] == 0.0) return 2;
        if (piv != c) {
            for (int j = 0; j < N; ++j) { double tmp = A[c * N + j]; A[c * N + j] = A[piv * N + j]; A[piv * N + j] = tmp; }
            double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
        }
        for (int r = c + 1; r < N; ++r) {
            double m = A[r * N + c] / A[c * N + c];
            for (int j = c; j < N; ++j) A[r * N + j] = A[r * N + j] - m * A[c * N + j];
            b[r] = b[r] - m * b[c];
        }
    }
    for (int r = N - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < N; ++j) s = s - A[r * N + j] * b[j];
        b[r] = s / A[r * N + r];
    }
    return 0;
}

int32_t orc_polish(const orc_net *net, const orc_params *p, double *x, double tol,
                   int32_t max_iter, double *rho_out, double *step_out)
{
    int N = net->n_nodes;
    double f[ORC_NMAX], fp[ORC_NMAX], fm[ORC_NMAX], xp[ORC_NMAX];
    double *J = (double *)malloc(sizeof(double) * (size_t)N * N);
    int32_t rc = 1;
    double last_step = 0.0;
    for (int it = 0; it <= max_iter; ++it) {
        orc_rhs(net, p, x, f);
        double rho = residual_rho(N, p, f);
        if (rho_out) *rho_out = rho;
        if (rho < tol) { rc = 0; break; }
        if (it == max_iter) break;
        for (int j = 0; j < N; ++j) {
            double scale = fabs(x[j]) > 1e-6 * p->G[j] / p->k[j] ? fabs(x[j]) : 1e-6 * p->G[j] / p->k[j];
            double dx = 6e-6 * scale;
            memcpy(xp, x, sizeof(double) * N);
            xp[j] = x[j] + dx; orc_rhs(net, p, xp, fp);
            xp[j] = x[j] - dx; orc_rhs(net, p, xp, fm);
            for (int i = 0; i < N; ++i) J[i * N + j] = (fp[i] - fm[i]) / (2.0 * dx);
        }
        for (int i = 0; i < N; ++i) f[i] = -f[i];
        if (lu_solve(N, J, f) != 0) { rc = 2; break; }
        last_step = 0.0;
        for (int i = 0; i < N; ++i) {
            x[i] = x[i] + f[i];
            double s = fabs(f[i]) / (p->G[i] / p->k[i]);
            if (s > last_step) last_step = s;
        }
    }
    if (step_out) *step_out = last_step;
    free(J);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Steady-state dedupe for one parameter set (Sec. 3.1: the             */
/* multistability of a set is its number of unique steady states over   */
/* its initial conditions).  States are compared after G/k              */
/* normalisation (Sec. 2.1.3), v_i = (x_i * k_i) / G_i.  In IC order,   */
/* each converged state joins the first representative r with           */
/* max_i |v_i - r_i| <= tol, or becomes a new representative.           */
/* state_id = representative index, -1 for solves that did not converge.*/
/* Returns the number of representatives.                               */
/* ------------------------------------------------------------------ */
int32_t orc_dedupe(int32_t N, int32_t n_ics, const double *states, const uint8_t *status,
                   const double *G, const double *k, double tol, int32_t *state_id)
{
    int32_t n_rep = 0;
    int32_t *rep_ic = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_ics > 0 ? n_ics : 1));
    for (int c = 0; c < n_ics; ++c) {
        state_id[c] = -1;
        if (status[c] != ORC_CONVERGED) continue;
        const double *x = states + (int64_t)c * N;
        int joined = -1;
        for (int r = 0; r < n_rep && joined < 0; ++r) {
            const double *xr = states + (int64_t)rep_ic[r] * N;
            double dmax = 0.0;
            for (int i = 0; i < N; ++i) {
                double v = (x[i] * k[i]) / G[i];
                double vr = (xr[i] * k[i]) / G[i];
                double d = fabs(v - vr);
                if (d > dmax) dmax = d;
            }
            if (dmax <= tol) joined = r;
        }
        if (joined < 0) { rep_ic[n_rep] = c; joined = n_rep; ++n_rep; }
        state_id[c] = joined;
    }
    free(rep_ic);
    return n_rep;
}

/* ------------------------------------------------------------------ */
/* Whole path for a range of parameter sets: for every (set, IC) solve, */
/* optionally polish converged states, then dedupe each set.            */
/* Arrays are indexed by the set's position in the range.               */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t polish;                /* 1: Newton polish of converged states */
    double polish_tol;             /* rho target of the polish */
    int32_t polish_iters;
    double dedupe_tol;
} orc_path_opts;

void orc_run_sets(const orc_net *net, const double *G, const double *k, const double *T,
                  const double *lam, const int32_t *n, int64_t n_sets,
                  const double *ic_unit, int32_t n_ics, const orc_opts *o,
                  const orc_path_opts *po,
                  double *states, uint8_t *status, double *t_final, int64_t *n_attempts,
                  double *series, int32_t *state_id, int32_t *n_unique)
{
    int N = net->n_nodes, E = net->n_edges;
    double x0[ORC_NMAX];
    for (int64_t s = 0; s < n_sets; ++s) {
        orc_params p = { G + s * N, k + s * N, T + s * E, lam + s * E, n + s * E };
        for (int c = 0; c < n_ics; ++c) {
            int64_t idx = s * n_ics + c;
            for (int i = 0; i < N; ++i) x0[i] = (ic_unit[(int64_t)c * N + i] * p.G[i]) / p.k[i];
            double *xo = states + idx * N;
            double *sr = series ? series + idx * (int64_t)o->n_t * N : NULL;
            orc_result r = orc_solve(net, &p, x0, o, xo, sr);
            if (r.status == ORC_CONVERGED && po->polish) {
                double xp[ORC_NMAX];
                memcpy(xp, xo, sizeof(double) * N);
                double rho, stp;
                if (orc_polish(net, &p, xp, po->polish_tol, po->polish_iters, &rho, &stp) == 0)
                    memcpy(xo, xp, sizeof(double) * N);
                else
                    r.status = ORC_POLISH_FAIL;
            }
            status[idx] = (uint8_t)r.status;
            if (t_final) t_final[idx] = r.t_final;
            if (n_attempts) n_attempts[idx] = r.n_attempts;
        }
        if (state_id && n_unique)
            n_unique[s] = orc_dedupe(N, n_ics, states + s * n_ics * (int64_t)N, status + s * n_ics,
                                     p.G, p.k, po->dedupe_tol, state_id + s * n_ics);
    }
}

/* ------------------------------------------------------------------ */
/* Levels of G/k-normalised expression (Sec. 2.1.3 analysis: nodes are  */
/* coarse-grained into levels "based on the global distribution" of the */
/* normalised values, a state is the concatenation of its nodes' levels,*/
/* and a set's multistability is its number of distinct states; Sec.    */
/* 3.1).  The paper does not say how the level boundaries are chosen;   */
/* the reading taken here:                                              */
/*   * v = (x k) / G of every node of every converged solve is put in   */
/*     one of n_bins equal bins on [0, 1] (v below 0 in the first, v at */
/*     or above 1 in the last) -- one histogram over all nodes and sets;*/
/*   * the counts are smoothed with the binomial weights C(2m, j),      */
/*     j = 0..2m, centred (zero outside the bins), in integers;         */
/*   * modes are merged by persistence: runs of equal smoothed counts   */
/*     are peaks (higher than their neighbours; an end run needs only   */
/*     its one neighbour lower) and valleys (lower than both            */
/*     neighbours); valleys are taken from the highest down (ties: the  */
/*     lower bin first), each joining the two groups of modes beside    */
/*     it; the group with the lower highest peak (ties: the one on the  */
/*     right) is absorbed, and the valley is a boundary when twice its  */
/*     count is at most that peak and the peak is at least 1/64 of the  */
/*     histogram's highest count; its bin is the valley run's middle    */
/*     (lower middle); at most max_b boundaries are kept, the lowest    */
/*     valleys first (ties: the lower bin), reported in bin order;      */
/*   * a value's level is the number of boundaries whose bin is below   */
/*     its own; a solve's label packs its nodes' levels, node i in bits */
/*     [i*w, i*w + w), w = bits for (boundaries + 1) levels; a solve    */
/*     that did not converge has the label 2^64 - 1.                    */
/* ------------------------------------------------------------------ */
int32_t orc_gk_bin(double x, double k, double G, int32_t n_bins)
{
    double f = ((x * k) / G) * (double)n_bins;
    if (!(f >= 0.0)) return 0;
    if (f >= (double)n_bins) return n_bins - 1;
    return (int32_t)f;
}

/* Adds the bins of n_sets sets of n_ics solves (states [S][I][N],      */
/* status [S][I], per-set G and k [S][N]) to counts[n_bins].            */
void orc_gk_histogram(int32_t N, int32_t n_ics, int64_t n_sets, const double *states,
                      const uint8_t *status, const double *G, const double *k, int32_t n_bins,
                      uint64_t *counts)
{
    for (int64_t s = 0; s < n_sets; ++s)
        for (int c = 0; c < n_ics; ++c) {
            if (status[s * n_ics + c] != ORC_CONVERGED) continue;
            const double *x = states + (s * n_ics + c) * (int64_t)N;
            for (int i = 0; i < N; ++i)
                counts[orc_gk_bin(x[i], k[s * N + i], G[s * N + i], n_bins)] += 1;
        }
}

static uint64_t binom(int n, int j)
{
    uint64_t r = 1;
    for (int t = 1; t <= j; ++t) r = r * (uint64_t)(n - j + t) / (uint64_t)t;
    return r;
}

/* Boundary bins of the histogram counts[n_bins] (reading above) into   */
/* bins_out[<= max_b]; returns their number.                            */
int32_t orc_level_boundaries(const uint64_t *counts, int32_t n_bins, int32_t m, int32_t max_b,
                             int32_t *bins_out)
{
    if (n_bins < 3 || max_b < 1) return 0;
    uint64_t *sm = (uint64_t *)calloc((size_t)n_bins, sizeof(uint64_t));
    for (int b = 0; b < n_bins; ++b)
        for (int j = 0; j <= 2 * m; ++j) {
            int src = b + j - m;
            if (src >= 0 && src < n_bins) sm[b] += binom(2 * m, j) * counts[src];
        }
    uint64_t top = 0;
    for (int b = 0; b < n_bins; ++b) if (sm[b] > top) top = sm[b];
    /* runs of equal counts: start, end, value, kind (1 peak, -1 valley) */
    int nr = 0;
    int *r0 = (int *)malloc(sizeof(int) * (size_t)n_bins), *r1 = (int *)malloc(sizeof(int) * (size_t)n_bins);
    int *kind = (int *)malloc(sizeof(int) * (size_t)n_bins);
    for (int b = 0; b < n_bins;) {
        int e = b;
        while (e + 1 < n_bins && sm[e + 1] == sm[b]) ++e;
        r0[nr] = b; r1[nr] = e; ++nr;
        b = e + 1;
    }
    for (int r = 0; r < nr; ++r) {
        int lo_l = r > 0 && sm[r0[r - 1]] < sm[r0[r]], lo_r = r + 1 < nr && sm[r0[r + 1]] < sm[r0[r]];
        int hi_l = r > 0 && sm[r0[r - 1]] > sm[r0[r]], hi_r = r + 1 < nr && sm[r0[r + 1]] > sm[r0[r]];
        kind[r] = 0;
        if ((lo_l || r == 0) && (lo_r || r == nr - 1) && nr > 1) kind[r] = 1;
        if (hi_l && hi_r) kind[r] = -1;
    }
    /* groups of peaks: each peak run is a group (highest peak value and
       its run index for ties); a valley joins the groups of the nearest
       peaks on its two sides */
    int *grp = (int *)malloc(sizeof(int) * (size_t)nr);      /* run -> group root (peaks only) */
    uint64_t *gmax = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nr);
    int *gpos = (int *)malloc(sizeof(int) * (size_t)nr);
    for (int r = 0; r < nr; ++r) { grp[r] = r; gmax[r] = sm[r0[r]]; gpos[r] = r; }
    int nv = 0;
    int *vr = (int *)malloc(sizeof(int) * (size_t)nr);
    for (int r = 0; r < nr; ++r) if (kind[r] == -1) vr[nv++] = r;
    /* valleys from the highest down, ties: lower bin first */
    for (int a = 1; a < nv; ++a)
        for (int t = a; t > 0; --t) {
            uint64_t va = sm[r0[vr[t]]], vb = sm[r0[vr[t - 1]]];
            if (va > vb || (va == vb && r0[vr[t]] < r0[vr[t - 1]])) { int x = vr[t]; vr[t] = vr[t - 1]; vr[t - 1] = x; }
            else break;
        }
    int *cb = (int *)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
    uint64_t *cv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nv > 0 ? nv : 1));
    int nc = 0;
    for (int a = 0; a < nv; ++a) {
        int v = vr[a];
        int pl = v - 1, pr = v + 1;                 /* nearest peaks beside the valley */
        while (kind[pl] != 1) --pl;
        while (kind[pr] != 1) ++pr;
        int gl = pl, gr = pr;
        while (grp[gl] != gl) gl = grp[gl];
        while (grp[gr] != gr) gr = grp[gr];
        /* the absorbed group: the lower highest peak, ties the right one */
        int young = gmax[gl] < gmax[gr] ? gl : (gmax[gr] < gmax[gl] ? gr : (gpos[gl] > gpos[gr] ? gl : gr));
        int old = young == gl ? gr : gl;
        uint64_t d = sm[r0[v]];
        if (2 * d <= gmax[young] && 64 * gmax[young] >= top) { cb[nc] = (r0[v] + r1[v]) / 2; cv[nc] = d; ++nc; }
        grp[young] = old;
    }
    int keep = nc < max_b ? nc : max_b;
    for (int a = 0; a < keep; ++a) {          /* selection by (value, bin) */
        int best = a;
        for (int t = a + 1; t < nc; ++t)
            if (cv[t] < cv[best] || (cv[t] == cv[best] && cb[t] < cb[best])) best = t;
        int tb = cb[a]; cb[a] = cb[best]; cb[best] = tb;
        uint64_t tv = cv[a]; cv[a] = cv[best]; cv[best] = tv;
    }
    for (int a = 1; a < keep; ++a)            /* insertion sort by bin */
        for (int t = a; t > 0 && cb[t - 1] > cb[t]; --t) {
            int tb = cb[t]; cb[t] = cb[t - 1]; cb[t - 1] = tb;
        }
    for (int a = 0; a < keep; ++a) bins_out[a] = cb[a];
    free(sm); free(r0); free(r1); free(kind); free(grp); free(gmax); free(gpos); free(vr); free(cb); free(cv);
    return keep;
}

/* Labels [S][I] (reading above), distinct labels among each set's      */
/* converged solves n_states[S], and multi_hist[k] += number of sets    */
/* with k distinct states (k = 0..n_ics).  Returns 0, or -1 when N      */
/* levels do not fit in 64 bits.                                        */
int32_t orc_level_states(int32_t N, int32_t n_ics, int64_t n_sets, const double *states,
                         const uint8_t *status, const double *G, const double *k, int32_t n_bins,
                         const int32_t *bounds, int32_t n_b, uint64_t *labels, int32_t *n_states,
                         uint64_t *multi_hist)
{
    int w = 0;
    while ((1 << w) < n_b + 1) ++w;
    if ((int64_t)N * w > 64) return -1;
    for (int64_t s = 0; s < n_sets; ++s) {
        int32_t distinct = 0;
        for (int c = 0; c < n_ics; ++c) {
            int64_t idx = s * n_ics + c;
            if (status[idx] != ORC_CONVERGED) { labels[idx] = UINT64_MAX; continue; }
            const double *x = states + idx * N;
            uint64_t lab = 0;
            for (int i = 0; i < N; ++i) {
                int bin = orc_gk_bin(x[i], k[s * N + i], G[s * N + i], n_bins);
                uint64_t lev = 0;
                for (int t = 0; t < n_b; ++t) lev += bounds[t] < bin;
                lab |= lev << (i * w);
            }
            labels[idx] = lab;
            int seen = 0;
            for (int c2 = 0; c2 < c && !seen; ++c2)
                seen = status[s * n_ics + c2] == ORC_CONVERGED && labels[s * n_ics + c2] == lab;
            if (!seen) ++distinct;
        }
        n_states[s] = distinct;
        multi_hist[distinct] += 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Boolean Ising formalism (Sec. 2.2, Eq. 3): node i becomes active    */
/* when sum_j J_ij s_j > 0, inactive when it is < 0, and keeps its      */
/* state when it is 0; J_ij = +1 for an activating edge j -> i, -1 for  */
/* an inhibiting one.  A state is a word of N bits, bit i set = node i  */
/* active (s_i = +1); an inactive node counts as s_i = -1, or as 0 with */
/* enc01 (the 0/1 encoding).  Synchronous mode updates every node at    */
/* once; asynchronous mode updates one node per step, chosen uniformly  */
/* (draw 1 + k of the stream (seed, ORC_TAG_ISING, trajectory) for step */
/* k, orc_uint_range over [0, N-1]).  Initial states: given, or draw 0  */
/* of the same stream masked to N bits.  A trajectory stops at a fixed  */
/* point (no node would change: status CONVERGED, steps = updates       */
/* applied before it) or after max_steps updates (status MAXSTEPS).     */
/* ------------------------------------------------------------------ */
#define ORC_TAG_ISING 0x4953494E47424FULL   /* "ISINGBO" */

static int ising_field(const orc_net *net, int i, uint64_t s, int enc01)
{
    int h = 0;
    for (int e = 0; e < net->n_edges; ++e) {
        if (net->dst[e] != i) continue;
        int sj = ((s >> net->src[e]) & 1ULL) ? 1 : (enc01 ? 0 : -1);
        h += net->sign[e] * sj;
    }
    return h;
}

/* The state after updating node i of s. */
static uint64_t ising_node(const orc_net *net, int i, uint64_t s, int enc01)
{
    int h = ising_field(net, i, s, enc01);
    if (h > 0) return s | (1ULL << i);
    if (h < 0) return s & ~(1ULL << i);
    return s;
}

/* The state after updating every node of s at once. */
static uint64_t ising_sync(const orc_net *net, uint64_t s, int enc01)
{
    uint64_t t = s;
    for (int i = 0; i < net->n_nodes; ++i) {
        uint64_t u = ising_node(net, i, s, enc01);
        t = (t & ~(1ULL << i)) | (u & (1ULL << i));
    }
    return t;
}

/* Runs n_traj trajectories; mode 0 synchronous, 1 asynchronous.        */
/* Returns 0, or -1 for more than 64 nodes.                             */
int32_t orc_ising_run(const orc_net *net, int32_t mode, int32_t enc01, uint64_t seed, int64_t n_traj,
                      const uint64_t *init, int32_t max_steps, uint64_t *final, int32_t *steps,
                      uint8_t *status)
{
    int N = net->n_nodes;
    if (N > 64) return -1;
    uint64_t mask = N == 64 ? ~0ULL : ((1ULL << N) - 1ULL);
    for (int64_t t = 0; t < n_traj; ++t) {
        uint64_t s = init ? init[t] & mask : draw64(seed, ORC_TAG_ISING, (uint64_t)t, 0) & mask;
        int32_t k = 0;
        uint8_t st = ORC_MAXSTEPS;
        for (;;) {
            uint64_t next = ising_sync(net, s, enc01);
            if (next == s) { st = ORC_CONVERGED; break; }
            if (k >= max_steps) break;
            if (mode == 0) {
                s = next;
            } else {
                int i = orc_uint_range(draw64(seed, ORC_TAG_ISING, (uint64_t)t, 1 + (uint64_t)k), 0, N - 1);
                s = ising_node(net, i, s, enc01);
            }
            ++k;
        }
        final[t] = s; steps[t] = k; status[t] = st;
    }
    return 0;
}

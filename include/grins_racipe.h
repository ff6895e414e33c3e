/*
 * grins_racipe.h -- C ABI of the GB300 RACIPE ensemble solver
 * (libgrins_racipe.so).
 *
 * RACIPE (GRiNS, arXiv 2503.18356, Sec. 2.1) integrates, for a fixed signed
 * directed gene-regulatory network, one trajectory of the node equation
 * (Eq. 1, with the shifted Hill function of Eq. 2) per pair (random
 * parameter set, random initial condition), runs it to steady state, and
 * reduces each parameter set's results to its distinct steady states.
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  "d_" arguments are DEVICE pointers (CUDA global
 *     memory of the current device), everything else is host memory.
 *   - Every device buffer is owned by the caller; the library never frees
 *     it and never keeps it after the call returns.  The handle owns its
 *     own copy of the topology, the half-functional median table and a
 *     small device workspace (work-queue counters).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that launch kernels are asynchronous on that stream;
 *     results are valid once the stream reaches the call's work.
 *   - Argument errors are reported before any work is queued, with a
 *     status other than GRINS_OK and a message for grins_last_error().
 *     CUDA launch or allocation failures return GRINS_E_CUDA / GRINS_E_NOMEM.
 *     The outcome of each individual solve is never an error: it is written
 *     to that solve's status byte (grins_solve_status).
 *   - A handle may be used from one host thread at a time.  Distinct handles
 *     are independent.
 *
 * Layout of one parameter set (2N + 3E values, Sec. 2.1.2), in the byte
 * block d_params[set * grins_racipe_param_stride(h) ...]:
 *     double G[N]      production rate of node i
 *     double k[N]      degradation rate of node i
 *     double T[E]      threshold of edge e (edge order = creation order)
 *     double lam[E]    fold change of edge e (>= 1 activating, <= 1 inhibiting)
 *     uint8  n[E]      integer Hill coefficient of edge e
 *     (zero padding to a multiple of 16 bytes)
 * Unit initial conditions: double u[n_ics][N] in [0, 1); solve (s, c) starts
 * from x0_i = (u[c][i] * G_i) / k_i (Sec. 2.1.2: between a node's minimum 0
 * and maximum G/k; the same ICs serve every parameter set, Sec. 3.1).
 */
#ifndef GRINS_RACIPE_H
#define GRINS_RACIPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grins_racipe *grins_racipe_t;   /* opaque, library-owned */

typedef enum {
    GRINS_OK = 0,
    GRINS_E_INVALID_ARG = 1,   /* null pointer, bad size, bad option value */
    GRINS_E_TOPOLOGY = 2,      /* invalid edge list */
    GRINS_E_NOMEM = 3,         /* host or device allocation failed */
    GRINS_E_CUDA = 4,          /* a CUDA call or kernel launch failed */
    GRINS_E_BUDGET = 5,        /* request exceeds a documented limit */
    GRINS_E_CANCELLED = 6
} grins_status;

/* Per-solve outcome, one byte per (set, IC). */
typedef enum {
    GRINS_SS_CONVERGED = 0,    /* steady-state condition met (Sec. 2.1.3) */
    GRINS_SS_TEND = 1,         /* reached t_end first */
    GRINS_SS_MAXSTEPS = 2,     /* spent max_steps step attempts */
    GRINS_SS_NONFINITE = 3,    /* NaN/Inf or step-size underflow */
    GRINS_SS_POLISH_FAIL = 4,  /* converged, but the FP64 polish did not certify it;
                                  the unpolished state is returned */
    GRINS_SS_CANCELLED = 5     /* not finished: the call's cancel flag was set before
                                  the solve started (or, in the polish, before its
                                  converged state was polished); its state is not a
                                  result */
} grins_solve_status;

enum { GRINS_FP64 = 0, GRINS_FP32 = 1 };                       /* precision */
enum { GRINS_TAIL_DD = 0, GRINS_TAIL_FP64 = 1 };                 /* tail_precision */
enum { GRINS_METHOD_DOPRI5 = 0, GRINS_METHOD_TSIT5 = 1 };        /* 5(4) pair */
enum { GRINS_MEDIAN_PER_INDEGREE = 0, GRINS_MEDIAN_UNREGULATED = 1 };
/* Distribution of a continuous parameter class over its [min, max] range
 * (the paper's samplers besides Table 1's, Sec. 2.1.2):
 *   GRINS_DIST_TABLE1      uniform; for the inhibiting fold change, uniform
 *                          in the inverse range and inverted (the default)
 *   GRINS_DIST_LOGUNIFORM  exp(U[log min, log max])
 *   GRINS_DIST_NORMAL      mean (min + max) / 2, s.d. (max - min) / 6,
 *                          clamped to [min, max]
 *   GRINS_DIST_LOGNORMAL   the same in log space, then exp
 * The normal deviate is Box-Muller on the draw's two 32-bit halves,
 * u_hi, u_lo = (half + 1/2) 2^-32: sqrt(-2 log u_hi) cos(2 pi u_lo). */
enum { GRINS_DIST_TABLE1 = 0, GRINS_DIST_LOGUNIFORM = 1, GRINS_DIST_NORMAL = 2, GRINS_DIST_LOGNORMAL = 3 };

/* One row of a per-parameter range table (Sec. 2.1.2: the generated
 * parameter range file, with a distribution per parameter).  Rows follow
 * the layout of a parameter set: G[N], k[N], T[E], lam[E], n[E].
 *   G, k, lam: dist (GRINS_DIST_*) over [lo, hi]; an inhibiting lam needs
 *              hi <= 1 and, under GRINS_DIST_TABLE1, is drawn in the
 *              inverse range and inverted (Table 1); an activating lam
 *              needs lo >= 1;
 *   T:         the multiplier range of the source's median (Table 1:
 *              [0.02, 1.98]), uniform; dist must be 0;
 *   n:         integers lo..hi (1 <= lo <= hi <= 255), uniform; dist 0. */
typedef struct {
    int32_t dist;
    int32_t reserved;          /* set to 0 */
    double lo, hi;
} grins_param_range;

/* Sampling ranges, Table 1 (Sec. 2.1.2).  grins_racipe_default_ranges fills
 * the defaults: G [1,100], k [0.1,1], activating lambda [1,100], inhibiting
 * lambda [0.01,1] (drawn in the inverse range and inverted), integer n [1,6],
 * thresholds in [0.02, 1.98] x the median level of the source node (the
 * half-functional rule), 10000 samples per median, per-in-degree medians. */
typedef struct {
    double G_min, G_max;
    double k_min, k_max;
    double lam_act_min, lam_act_max;
    double lam_inh_min, lam_inh_max;
    int32_t n_min, n_max;
    double thr_lo, thr_hi;
    int32_t median_samples;
    int32_t median_mode;       /* GRINS_MEDIAN_* */
    int32_t dist_G, dist_k;            /* GRINS_DIST_* of G, k */
    int32_t dist_lam_act, dist_lam_inh;/* and of the two fold changes (the
                                          half-functional medians use them too) */
    int64_t lhs_sets;                  /* > 0: Latin hypercube over sets
                                          [0, lhs_sets) -- draw d of set s
                                          takes the unit (pi_d(s) + u) / lhs_sets,
                                          u its own draw, pi_d a permutation of
                                          the sets per draw index (a 4-round
                                          Feistel network on 2h bits, 2^(2h) >=
                                          lhs_sets, round function word 0 of
                                          Philox4x64-10 with counter (d, round,
                                          right half, 0) and key (seed,
                                          0x5241434950454C), cycle-walked into
                                          range); Hill coefficients n_min +
                                          floor(unit n_count); Table 1 and
                                          log-uniform classes only; 0 = off */
    int32_t sobol;                     /* GRINS_SOBOL_* (below); 0 = off */
    int32_t sobol_dims;                /* rows of the two tables, >= 2N + 3E */
    const int64_t *sobol_poly;         /* host [sobol_dims], read during the call */
    const int64_t *sobol_m;            /* host [sobol_dims][sobol_m_cols] */
    int32_t sobol_m_cols;
    int32_t reserved;                  /* set to 0 (keeps the struct free of padding) */
    const grins_param_range *param_ranges; /* host [2N + 3E], read during the
                                          call, or NULL.  Non-NULL: every
                                          parameter takes its own row (the
                                          class fields above are unused but
                                          median_samples and median_mode), and
                                          the medians are per node (below) */
    const grins_param_range *ic_ranges;  /* host [N], read during the call, or
                                          NULL: initial condition of node i as
                                          a fraction of its maximum G_i / k_i
                                          drawn by row i's dist over [lo, hi],
                                          0 <= lo <= hi <= 1 (lo > 0 for the
                                          log distributions); NULL = uniform
                                          on [0, 1) (Sec. 2.1.2) */
} grins_racipe_ranges;

/* Sobol sets (Sec. 2.1.2: the paper's default sampler).  With sobol != 0,
 * draw d (0 <= d < 2N + 3E, the order of the layout above) of set s takes
 * the unit x 2^-32, x the 32-bit coordinate d of point s of the Sobol
 * sequence in Gray-code order (Antonov and Saleev 1979): x = XOR of V_d[b]
 * over the set bits b of s ^ (s >> 1), s < 2^32.  Direction numbers
 * (Bratley and Fox 1988): V_d[b] = m_{b+1} 2^(31-b), with m_k = 1 for
 * dimension 0 and, for d >= 1, sobol_m[d][k-1] for k <= s_d and
 *   m_k = m_{k-s} ^ (m_{k-s} << s) ^ XOR_{i=1}^{s-1} a_i (m_{k-i} << i)
 * beyond, where sobol_poly[d] holds the primitive polynomial
 * x^s + a_1 x^(s-1) + ... + a_{s-1} x + 1 with bit j the coefficient of x^j
 * (s its highest set bit, 1 <= s <= min(sobol_m_cols, 32), each given m_k
 * odd and below 2^k).  The table of Joe and Kuo (2008) as scipy ships it has
 * this form.  GRINS_SOBOL_SCRAMBLED adds a linear matrix scramble and a
 * digital shift (Matousek 1998), drawn from Philox4x64-10 with key (seed,
 * 0x52414349504553): digit j (1 = most significant, bit 32 - j) of the
 * scrambled coordinate is the parity of x AND M_j, M_j bit 32 - j plus the
 * bits above it taken from the low word of the draw at counter (d, j, 0, 0);
 * the shift is the low word at counter (d, 0, 0, 0).  Hill coefficients take
 * n_min + floor(unit n_count); Table 1 and log-uniform classes only; not
 * with lhs_sets. */
enum { GRINS_SOBOL_OFF = 0, GRINS_SOBOL_PLAIN = 1, GRINS_SOBOL_SCRAMBLED = 2 };

/* Solver controls (Sec. 2.1.3: tolerances, start and end time, stop at
 * steady state, optional time points).  grins_solver_default_opts fills:
 * FP32 + polish, rtol 1e-6, atol 1e-9, t0 0, t_end 200, ss_tol 1e-6,
 * max_steps 100000, no time grid, polish_tol 1e-13, polish_iters 16,
 * polish_max_move 0.1, ss_tighten 0.3, method GRINS_METHOD_DOPRI5,
 * tail_rtol 1e-9, tail_start 20, tail_rho 10, tail_late 0.2, tail_work 96,
 * tail_precision GRINS_TAIL_DD. */
typedef struct {
    int32_t precision;         /* GRINS_FP32 or GRINS_FP64 integration */
    int32_t polish;            /* 1: FP64 Newton polish of each converged state */
    double rtol, atol;         /* local error tolerances of the 5(4) pair */
    double t0, t_end;
    double ss_tol;             /* converged when max_i |dx_i/dt| / (G_i/k_i) < ss_tol */
    int64_t max_steps;         /* step attempts (accepted + rejected) per solve */
    const double *t_grid;      /* HOST pointer to n_t increasing times in [t0, t_end];
                                  NULL / 0 = no time series */
    int32_t n_t;
    double polish_tol;         /* polish succeeds when the FP64 residual < polish_tol */
    int32_t polish_iters;      /* polish steps at most (chord-Newton steps, see
                                  grins_racipe_polish) */
    double polish_max_move;    /* reject a polish that moves a G/k-normalised
                                  coordinate by more than this in one step (a
                                  guard against a jump to another fixed point;
                                  the default lets the polish finish solves the
                                  steady-state test stopped along a slow mode,
                                  ~1e-2 G/k from their fixed point) */
    double ss_tighten;         /* once a solve's residual max_i |dx_i/dt| / (G_i/k_i) is
                                  below 10 ss_tol, its error tolerances are scaled by
                                  this factor (0 < ss_tighten <= 1; 1 = never): with
                                  ss_tol near rtol, the integrator's own error level
                                  would otherwise sit at the steady-state threshold */
    int32_t method;            /* the embedded 5(4) pair: GRINS_METHOD_DOPRI5
                                  (Dormand-Prince) or GRINS_METHOD_TSIT5 (Tsitouras
                                  2011, the paper's Tsit5, Sec. 3.1); both take the
                                  same step control and steady-state test.  Tsit5
                                  runs on the kernels compiled for the network (FP32
                                  and FP64 register records); calls without one --
                                  no register layout, run-time compiles off -- and
                                  plans and the server take Dormand-Prince only
                                  (GRINS_E_INVALID_ARG otherwise) */
    /* Borderline re-pass (FP32 integrations; tail_rtol = 0 turns it off).
     * Near t_end the steady-state decision of Sec. 2.1.3 is decided by a
     * residual max_i |dx_i/dt| / (G_i/k_i) that has fallen to about ss_tol,
     * and at rtol ~ ss_tol the integrated state is not accurate enough to
     * place it on the right side: the residual can cross ss_tol early, late
     * or, where it dips and rises again, not at all.  So the FP32 pass keeps
     * a checkpoint -- its first accepted state with residual below
     * tail_start * ss_tol -- and a solve whose decision is borderline
     *   - t_end reached with a final residual below tail_rho * ss_tol, or
     *   - converged at t with t_end - t < tail_late * (t - t_c), t_c the
     *     checkpoint's time (the crossing could move past t_end),
     * and that took at most tail_work attempts after its checkpoint (longer
     * stretches -- slow oscillations that hover near ss_tol -- would hold
     * the re-pass for many times the rest of its work and keep their FP32
     * result), is integrated again from its checkpoint to t_end at rtol
     * tail_rtol (atol scaled by tail_rtol / rtol), no tightening, which sets
     * its state, status and t_final; d_n_steps counts the attempts of both
     * passes, and grins_racipe_tail_stats reports the re-pass's share.  The
     * re-pass computes in tail_precision: GRINS_TAIL_DD (default)
     * double-float -- each value a pair of FP32 numbers, about 48 significant
     * bits, which this GPU runs several times faster than FP64 -- or
     * GRINS_TAIL_FP64.  Runs when the kernels compiled for the network are
     * available (FP32 and re-pass register records) and there is no time
     * grid; otherwise the call proceeds without it.  Plans, the server and
     * grins_racipe_integrate_static do not run it. */
    double tail_rtol;
    double tail_start;
    double tail_rho;
    double tail_late;
    int32_t tail_work;
    int32_t tail_precision;    /* GRINS_TAIL_DD or GRINS_TAIL_FP64 */
    void *pass_event;          /* profiling hook, NULL = none: a cudaEvent_t that
                                  grins_racipe_integrate records on its stream after
                                  the integration pass and before the re-pass and the
                                  polish, so a caller can time the integrator alone */
    const volatile int32_t *cancel; /* NULL = none: an int32 the GPU can read (pinned
                                  host memory mapped for the device, or device
                                  memory), polled by the integrators and the polish
                                  each time they take their next work item (a solve,
                                  a parameter set or a polish unit).  Once it is
                                  nonzero no further work starts: solves in flight
                                  finish, every solve not yet started -- and every
                                  converged solve not yet polished -- gets
                                  GRINS_SS_CANCELLED, and the call completes as
                                  usual (it returns GRINS_OK; the statuses tell) */
} grins_solver_opts;

void grins_racipe_default_ranges(grins_racipe_ranges *r);
void grins_solver_default_opts(grins_solver_opts *o);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *grins_last_error(void);

/* Number of device allocations (cudaMalloc, cudaMallocAsync and
 * cudaMallocFromPoolAsync calls) the library has made in this process, over
 * all handles, plans and servers: a diagnostic that shows whether a call
 * allocated (compare the count before and after it).  Thread-safe. */
int64_t grins_device_allocations(void);

/* Measured issue rates of the arithmetic units that bound this library's
 * kernels on the current device, in operations per clock per SM (host array
 * of seven doubles): rates[0] ex2.approx.f32, rates[1] lg2.approx.f32,
 * rates[2] rcp.approx.f32 (the special-function unit: the FP32
 * integrator's edge powers, node logarithms and divisions of Eq. 2),
 * rates[3] FP32 fused multiply-add, rates[4] FP64 fused multiply-add,
 * rates[5] FP64 multiply, rates[6] FP64 add (the polish, the dedupe, the
 * plain FP64 solver).  These are the denominators of
 * the kernels' rooflines.  One block of 1024 threads per SM runs eight
 * independent chains of each operation for a fixed count and reads the SM
 * clock around the loop; a rate is the median over blocks, so it does not
 * depend on the clock frequency.  Takes a few milliseconds; allocates two
 * small device buffers (freed before returning) and synchronises `stream`.
 * Errors: GRINS_E_INVALID_ARG (rates NULL), GRINS_E_NOMEM, GRINS_E_CUDA. */
grins_status grins_unit_rates(double *rates, void *stream);

/* Library version string. */
const char *grins_version(void);

/* Builds a handle from a signed, directed edge list (Sec. 2.1.1; the parser
 * accepts activation and inhibition links only).  Host arrays of length
 * n_edges: src[e] -> dst[e] with sign[e] = +1 (activation) or -1
 * (inhibition).  They are copied.  Self-loops are allowed.
 * Errors: GRINS_E_TOPOLOGY for n_nodes < 1 or > 64, n_edges < 0 or > 4096,
 * an index out of range, a sign other than +1/-1, or a repeated (src, dst)
 * pair; GRINS_E_INVALID_ARG for null pointers; GRINS_E_CUDA / NOMEM when
 * the device workspace cannot be created.  Uses the current CUDA device. */
grins_status grins_racipe_create(int32_t n_nodes, int32_t n_edges, const int32_t *src,
                                 const int32_t *dst, const int8_t *sign,
                                 grins_racipe_t *out);

/* Frees the handle and its device workspace (synchronises the device). */
grins_status grins_racipe_destroy(grins_racipe_t h);

/* Bytes per parameter set in d_params (see the layout above); -1 on a
 * null handle. */
int64_t grins_racipe_param_stride(grins_racipe_t h);

/* Host copy of the per-node median levels M_j used by the half-functional
 * threshold rule for the given ranges (NULL = defaults): out[n_nodes].
 * M_j depends on node j's in-degree class (#activating, #inhibiting
 * inputs), Sec. 2.1.2 and Table 1 threshold row.
 * With a per-parameter table, node j's medians use its own rows: the
 * unregulated median M0_j of G_j / k_j (median_samples draws of Philox
 * key (0x48414C4646554E43, 2^63 + 2j), counter (sample, draw / 4), word draw %
 * 4: G draw 0, k draw 1), and, when j has inputs and median_mode is
 * per-in-degree, the median M_j of G_j / k_j times one Hill factor per
 * in-edge e (edge order, q-th in-edge draws 2 + 5q .. 6 + 5q: G and k of
 * the source from its rows, T = multiplier x M0_src, lam, n from e's rows)
 * under key (0x48414C4646554E43, 2^63 + 2j + 1); else M_j = M0_j. */
grins_status grins_racipe_node_medians(grins_racipe_t h, const grins_racipe_ranges *r,
                                       double *out);

/* Samples parameter sets set0 .. set0+n_sets-1 into d_params (bytes
 * [n_sets][param_stride]) and, if d_ic_unit is not NULL, the unit initial
 * conditions d_ic_unit[n_ics][N] (doubles), following Sec. 2.1.2 and
 * Table 1 (r = NULL: defaults).  Counter-based: set s is the same whether
 * it is drawn alone or in any batch, on any device.  Errors:
 * GRINS_E_INVALID_ARG for bad ranges (min > max, non-positive G/k/lambda
 * bounds, activating lambda below 1, inhibiting lambda above 1, n outside
 * [1, 255], median_samples < 1), n_sets < 0, set0 < 0, n_ics < 0, or a
 * null d_params with n_sets > 0, and for the Sobol, table and
 * initial-condition options the conditions stated with them.
 * Host work and synchronisation: the half-functional medians are computed
 * on the host once per ranges (cached on the handle, under a lock); the
 * first call on a handle uploads its edge medians and waits for its stream;
 * a later call whose medians differ, and any call with Sobol tables or
 * per-parameter or initial-condition rows, stages them in a stream-ordered
 * device buffer (cudaMallocAsync, freed after the sampler on the same
 * stream) and does not wait. */
grins_status grins_racipe_sample_params(grins_racipe_t h, const grins_racipe_ranges *r,
                                        uint64_t seed, int64_t set0, int64_t n_sets,
                                        int32_t n_ics, void *d_params, double *d_ic_unit,
                                        void *stream);

/* Integrates every (set, IC) pair: n_sets parameter sets from d_params
 * (layout above) times n_ics unit ICs, with Dormand-Prince 5(4) (FSAL,
 * per-solve step control) until the steady-state condition, t_end or
 * max_steps; then (o->polish) an FP64 Newton polish of each converged
 * state.  Outputs, indexed [set][ic]:
 *   d_states  double [n_sets][n_ics][N]  final (polished) state
 *   d_status  uint8  [n_sets][n_ics]     grins_solve_status
 *   d_t_final double [n_sets][n_ics]     time at termination   (nullable)
 *   d_err_est float  [n_sets][n_ics]     G/k-normalised size of the last
 *                                        polish step; -1 if not polished (nullable)
 *   d_n_steps int32  [n_sets][n_ics]     step attempts           (nullable)
 *   d_series  double [n_sets][n_ics][n_t][N] states at o->t_grid (required
 *                                        iff n_t > 0); grid times after
 *                                        termination hold the final state
 * When the borderline re-pass runs (FP32, o->tail_rtol > 0) and o->polish is
 * set, the polish of the solves the re-pass does not take runs on a second
 * stream of the handle beside the re-pass, and the re-passed solves are
 * polished after both; the call forks that stream from `stream` and joins it
 * back with events, so all of its work is ordered on `stream` as usual and
 * the results are those of the polish run after the re-pass.
 * Errors: GRINS_E_INVALID_ARG for null required pointers, n_ics < 1,
 * n_sets < 0, non-positive tolerances, t_end <= t0, a grid that is not
 * increasing inside [t0, t_end], or max_steps < 1. */
grins_status grins_racipe_integrate(grins_racipe_t h, const grins_solver_opts *o,
                                    const void *d_params, int64_t n_sets,
                                    const double *d_ic_unit, int32_t n_ics,
                                    double *d_states, uint8_t *d_status, double *d_t_final,
                                    float *d_err_est, int32_t *d_n_steps, double *d_series,
                                    void *stream);

/* Which FP32 integrator kernel the handle's integrate calls use, as text:
 * the lane-group layout (lanes per solve L, node rows R, edge positions P)
 * and whether the kernel specialised to this network at run time (NVRTC)
 * is in use, or why not (before the first FP32 integrate call it reports
 * that nothing has been compiled yet); after an FP64 integrate call, a
 * second clause says which FP64 kernel ran.  The string is owned by the
 * handle and valid until the next call on it. */
const char *grins_racipe_integrator(grins_racipe_t h);

/* ----------------------------------------------------------------- plans
 * Batched form of the path (the production "batching" form of the hot
 * path; the paper's simulator runs one network per call): many networks of
 * uneven node and edge counts and uneven ensemble sizes are integrated in
 * one persistent launch -- each warp visits the jobs in turn and takes
 * solves from each job's work counter -- followed by each job's FP64 polish
 * (o->polish) and dedupe.  The work is captured once into a CUDA graph;
 * grins_racipe_plan_run replays it. */
typedef struct grins_racipe_plan *grins_racipe_plan_t;   /* opaque, library-owned */

/* One job of a plan: a network handle and its device buffers, laid out as
 * for grins_racipe_integrate and grins_racipe_unique_states. */
typedef struct {
    grins_racipe_t net;          /* the network (must outlive the plan) */
    const void *d_params;        /* [n_sets][param_stride] bytes */
    int64_t n_sets;
    const double *d_ic_unit;     /* [n_ics][N] unit initial conditions */
    int32_t n_ics;
    double *d_states;            /* [n_sets][n_ics][N] */
    uint8_t *d_status;           /* [n_sets][n_ics] */
    double *d_t_final;           /* [n_sets][n_ics], nullable */
    int32_t *d_n_steps;          /* [n_sets][n_ics], nullable */
    float *d_err_est;            /* [n_sets][n_ics], nullable */
    int32_t *d_state_id;         /* [n_sets][n_ics] dedupe output, nullable */
    int32_t *d_n_unique;         /* [n_sets] dedupe output; both or neither */
    double dedupe_tol;           /* max-norm tolerance of the dedupe (G/k scale) */
} grins_racipe_job;

/* Builds a plan for n_jobs jobs with the solver options o (FP32, no time
 * grid).  The integration runs in one of three forms:
 *   * one persistent launch of a kernel built for the plan: every distinct
 *     register layout among the jobs' networks gets the integrator compiled
 *     for it as a device function (NVRTC, in parallel on host threads,
 *     cached per layout and register cap), linked (nvJitLink) under one
 *     dispatcher; the warps of an SM start on the same job and visit the
 *     jobs in the same order, so they mostly run one body at a time;
 *   * one persistent launch of the run-time-layout kernel (no compile);
 *   * per job the integrator compiled for its network, each on one of up to
 *     16 branches of the graph, so that jobs run concurrently.
 * The jobs' polish and dedupe run on the graph's branches.
 * autotune = 0: the run-time-layout launch with 4 warps per block and 1
 * extra slot per scheduling domain.  autotune = 1: each form and its knobs
 * -- warps per block and resident blocks per SM (the register cap of every
 * body) of the compiled launch, block size and slots per domain of the
 * run-time-layout launch -- is timed on the first sixteenth of every job's
 * sets and the fastest kept (this runs kernels on `stream` and writes to the
 * jobs' output buffers).  autotune = 2: the per-job form without timing.
 * autotune = 3: the compiled launch, 4 warps x 3 blocks per SM, without
 * timing.  The jobs' buffers must stay valid for the plan's lifetime; their
 * contents are read when the plan runs.  Plans run no borderline re-pass
 * (grins_solver_opts.tail_rtol is ignored).  Errors: GRINS_E_INVALID_ARG for
 * bad options or jobs (networks on another device, missing buffers,
 * precision other than FP32, a time grid); GRINS_E_BUDGET when a network has
 * no lane-group layout of at most 8 node rows, a form needs more shared
 * memory than the device has, or (autotune = 3) the compiled form is not
 * available (no register layout, no NVRTC or nvJitLink). */
grins_status grins_racipe_plan_create(const grins_solver_opts *o, const grins_racipe_job *jobs,
                                      int32_t n_jobs, int32_t autotune, void *stream,
                                      grins_racipe_plan_t *out);

/* Replays the plan's graph on `stream` (asynchronous). */
grins_status grins_racipe_plan_run(grins_racipe_plan_t p, void *stream);

/* The chosen configuration and the autotuner's timings, as text. */
const char *grins_racipe_plan_info(grins_racipe_plan_t p);

/* Frees the plan (synchronises the device). */
grins_status grins_racipe_plan_destroy(grins_racipe_plan_t p);

/* ---------------------------------------------------------------- server
 * Serving form of the path (the paper's simulator is a batch library; this
 * is the production "serving" form): ensemble requests -- a network, a
 * sampling seed, n_sets x n_ics, solver options -- are admitted by a worker
 * thread in arrival order while the number in flight and the HBM budget
 * allow.  Each admitted request gets its own stream and device buffers
 * (from a private stream-ordered memory pool) and runs sample -> integrate
 * -> polish -> dedupe; requests admitted while others run execute
 * concurrently on the device (continuous batching).  Results stay in device
 * memory until the request is released.  A network handle must not be used
 * by other threads while it has requests queued or running; two requests on
 * one network run one after the other. */
typedef struct grins_racipe_server *grins_racipe_server_t;   /* opaque */

typedef struct {
    int32_t max_inflight;      /* requests running at once (streams), 1..64 */
    int64_t hbm_budget_bytes;  /* device memory all admitted requests may hold */
    /* Run-time compiled integrator (FP32 requests).  jit = 1: a request whose
     * work n_sets * n_ics * n_edges is at least jit_min_work starts, at
     * submission, a background compile of the integrator for its network
     * (unless one exists) and is admitted once the compile is done, or after
     * jit_max_wait_s, whichever comes first; it then runs the compiled kernel
     * if ready.  Smaller requests, and every request with jit = 0, run the
     * run-time-layout kernel unless an earlier call compiled one for the
     * network.  A request waiting for its compile does not hold back later
     * requests. */
    int32_t jit;
    double jit_min_work;
    double jit_max_wait_s;
} grins_server_config;

enum { GRINS_REQ_QUEUED = 0, GRINS_REQ_RUNNING = 1, GRINS_REQ_DONE = 2, GRINS_REQ_FAILED = 3,
       GRINS_REQ_CANCELLED = 4 };

typedef struct {
    int32_t state;             /* GRINS_REQ_* */
    int32_t error;             /* grins_status of a failed request */
    int64_t n_sets;
    int32_t n_ics;
    int64_t bytes;             /* device memory the request holds until released */
    double queued_s;           /* submission -> admission (so far, if queued) */
    double latency_s;          /* submission -> results ready; -1 if not done */
} grins_request_info;

/* Defaults: 8 in flight, 32 GiB budget, jit = 1, jit_min_work = 2e6,
 * jit_max_wait_s = 1. */
void grins_server_default_config(grins_server_config *c);

/* Starts a server (and its worker thread) on the current device; c = NULL
 * for the defaults.  Errors: GRINS_E_INVALID_ARG for a bad config. */
grins_status grins_racipe_server_create(const grins_server_config *c, grins_racipe_server_t *out);

/* Queues a request: parameter sets 0 .. n_sets-1 of `seed` (ranges r, NULL
 * = defaults) with n_ics ICs on network `net`, integrated with o (no time
 * grid) and deduplicated with dedupe_tol.  Returns at once with its id; the
 * tables r points to (Sobol, per-parameter and initial-condition rows) are
 * copied, so the caller may free them on return.  The half-functional
 * medians of in-degree classes not yet computed in the process (host work,
 * tens of milliseconds per class) are computed by the server's preparation
 * thread, the classes of one network in parallel; the request waits in the
 * queue for them (later requests are not held back).  A per-parameter
 * table's medians are computed in the calling thread.
 * Errors: GRINS_E_INVALID_ARG for bad arguments, GRINS_E_BUDGET when the
 * request alone needs more than the whole HBM budget. */
grins_status grins_racipe_server_submit(grins_racipe_server_t sv, grins_racipe_t net,
                                        const grins_racipe_ranges *r, uint64_t seed, int64_t n_sets,
                                        int32_t n_ics, const grins_solver_opts *o, double dedupe_tol,
                                        int64_t *request_id);

/* Waits (timeout_s < 0: without limit) for the request to finish and
 * reports its state and timings in *info (nullable). */
grins_status grins_racipe_server_wait(grins_racipe_server_t sv, int64_t request_id, double timeout_s,
                                      grins_request_info *info);

/* Cancels a request.  Queued: it never runs (state GRINS_REQ_CANCELLED, no
 * results).  Running: its kernels start no further work -- solves in flight
 * finish, the others get GRINS_SS_CANCELLED (through a per-slot flag in
 * pinned host memory mapped for the device, grins_solver_opts.cancel) -- and
 * it ends in GRINS_REQ_CANCELLED with error GRINS_E_CANCELLED; its results
 * can still be copied (the statuses tell which solves finished).  Finished:
 * no effect.  Returns at once; grins_racipe_server_wait waits for the end.
 * Errors: GRINS_E_INVALID_ARG for an unknown request. */
grins_status grins_racipe_server_cancel(grins_racipe_server_t sv, int64_t request_id);

/* Copies a finished request's results into caller buffers (each nullable):
 * states double [n_sets][n_ics][N], status uint8 [n_sets][n_ics],
 * n_unique int32 [n_sets], state_id int32 [n_sets][n_ics], n_steps int32
 * [n_sets][n_ics] (step attempts per solve). */
grins_status grins_racipe_server_copy_results(grins_racipe_server_t sv, int64_t request_id,
                                              double *d_states, uint8_t *d_status, int32_t *d_n_unique,
                                              int32_t *d_state_id, int32_t *d_n_steps, void *stream);

/* Frees a finished request's device memory and forgets it. */
grins_status grins_racipe_server_release(grins_racipe_server_t sv, int64_t request_id);

/* Stops the worker, waits for running requests and frees everything. */
grins_status grins_racipe_server_destroy(grins_racipe_server_t sv);

/* Largest time grid (o->n_t) that grins_racipe_integrate_static accepts. */
#define GRINS_STATIC_MAX_GRID 4096

/* The integrate call (same arguments, outputs and errors as
 * grins_racipe_integrate) for callers that must not allocate device memory
 * during a call: code that runs inside a host framework owning every device
 * allocation, a real-time loop where cudaMalloc/cudaFree would synchronise
 * the device or block, or a sandbox whose allocation quota is already spent.
 * The paper has no counterpart; this is an ABI convenience.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call
 *     (grins_device_allocations does not move across a call).  Its scratch
 *     (work-queue counter, check words and the device copy of the time
 *     grid) is one fixed array of about 33 KB inside the library, present on
 *     every device that loads the library until the process exits.  Inputs
 *     and outputs are still the caller's buffers.
 *   - Kernel: it compiles nothing.  The kernel compiled for the network is
 *     used only when an earlier grins_racipe_integrate call in this process,
 *     with the same precision and method, compiled and loaded it; otherwise
 *     the FP32 run-time-layout kernel or the generic FP64 kernel runs -- the
 *     same equations, step control and steady-state test, so states agree
 *     within the integration tolerance, but step counts (d_n_steps) and the
 *     last digits can differ from grins_racipe_integrate's.  The Tsitouras
 *     pair has no such fallback: without the compiled kernel it returns
 *     GRINS_E_INVALID_ARG.
 *   - The first call on each device (and again after the device's context
 *     is replaced, e.g. by cudaDeviceReset) looks up that array's device
 *     address with cudaGetSymbolAddress, with the device current.  That
 *     lookup can load the library's device code onto the device (lazy module
 *     loading): make the first call before any stream capture.
 *   - Every call, from any handle or thread, shares the one array; the call
 *     clears the counters it needs before launching, and the array keeps the
 *     last call's contents otherwise.  Calls whose work overlaps on the GPU
 *     (different streams, or different host threads) race on it: serialise
 *     them.
 *   - Extra error: GRINS_E_BUDGET when o->n_t > GRINS_STATIC_MAX_GRID. */
grins_status grins_racipe_integrate_static(grins_racipe_t h, const grins_solver_opts *o,
                                           const void *d_params, int64_t n_sets,
                                           const double *d_ic_unit, int32_t n_ics,
                                           double *d_states, uint8_t *d_status,
                                           double *d_t_final, float *d_err_est,
                                           int32_t *d_n_steps, double *d_series, void *stream);

/* The borderline re-pass of the last FP32 grins_racipe_integrate call on h
 * (see grins_solver_opts.tail_rtol): *n_solves = solves it re-integrated
 * (in tail_precision), *n_attempts = their step attempts in the re-pass;
 * both 0 when that call did not run it.  Copies two counters from the device after synchronising
 * `stream` (the stream of that call).  Errors: GRINS_E_INVALID_ARG for null
 * pointers. */
grins_status grins_racipe_tail_stats(grins_racipe_t h, void *stream, int64_t *n_solves, int64_t *n_attempts);

/* Newton polish of states already integrated (the step integrate runs when
 * o->polish is set; exposed so a caller can polish separately).  For every
 * solve with status GRINS_SS_CONVERGED: chord-Newton steps on Eq. 1 = 0 --
 * the residual in double precision at every step, the analytic Jacobian
 * evaluated and LU-factorised once in single precision, the step added in
 * double precision (mixed-precision iterative refinement) -- until the FP64
 * residual max_i |f_i| / (G_i / k_i) < o->polish_tol (at most
 * o->polish_iters steps).
 * Success overwrites d_states[set][ic][:] and writes the G/k-normalised size
 * of the last step to d_err_est (nullable); failure (singular
 * Jacobian, a step moving a normalised coordinate by more than
 * o->polish_max_move, or no convergence) keeps the state and sets the status
 * to GRINS_SS_POLISH_FAIL.  Other statuses are left alone (err_est = -1).
 * Only the polish_* fields of o are read.  Errors: GRINS_E_INVALID_ARG for
 * null pointers, n_ics < 1, n_sets < 0 or bad polish options. */
grins_status grins_racipe_polish(grins_racipe_t h, const grins_solver_opts *o,
                                 const void *d_params, int64_t n_sets, int32_t n_ics,
                                 double *d_states, uint8_t *d_status, float *d_err_est,
                                 void *stream);

/* Distinct steady states per parameter set (Sec. 3.1: multistability is
 * the number of unique steady states a set reaches over its ICs).  States
 * are G/k-normalised (Sec. 2.1.3), v_i = (x_i * k_i) / G_i in FP64; in IC
 * order, each converged state joins the first representative whose
 * max-norm distance is <= tol, else it becomes a new one.
 *   d_state_id int32 [n_sets][n_ics]  representative index, -1 unless converged
 *   d_n_unique int32 [n_sets]         number of representatives
 * Deterministic and independent of launch shape.  Errors:
 * GRINS_E_INVALID_ARG for null pointers, n_ics < 1 or > 4096, tol < 0. */
grins_status grins_racipe_unique_states(grins_racipe_t h, const void *d_params,
                                        const double *d_states, const uint8_t *d_status,
                                        int64_t n_sets, int32_t n_ics, double tol,
                                        int32_t *d_state_id, int32_t *d_n_unique,
                                        void *stream);

/* ---------------------------------------------------------------- levels
 * Levels of G/k-normalised expression, state labels and multistability
 * (Sec. 2.1.3: "nodes can be discretised into levels based on the global
 * distribution of normalised G/k values"; a state is the concatenation of
 * its nodes' levels and a set's multistability its number of distinct
 * states, Sec. 3.1).  The paper does not say how the boundaries between
 * levels are chosen; the reading implemented here:
 *   1. grins_racipe_gk_histogram: one histogram of v = (x_i k_i) / G_i (FP64)
 *      over every node of every converged solve, n_bins equal bins on
 *      [0, 1] -- bin floor(v n_bins), v below 0 in bin 0, at or above 1 in
 *      the last bin;
 *   2. grins_level_boundaries (host): the counts smoothed with the
 *      binomial weights C(2m, j), j = 0..2m, m = half_width (integers,
 *      zero beyond the ends); modes merged by persistence: maximal runs of
 *      equal smoothed counts are peaks (higher than their neighbours; an
 *      end run needs only its one neighbour lower) and valleys (lower than
 *      both neighbours); valleys from the highest down (ties: lower bin
 *      first) join the groups of peaks on their two sides, the group with
 *      the lower highest peak (ties: the one on the right) is absorbed,
 *      and the valley is a boundary when twice its count is at most that
 *      peak and the peak is at least 1/64 of the highest smoothed count;
 *      its bin is the run's middle (lower middle); at most max_boundaries
 *      are kept, lowest valleys first (ties: lower bin), reported in
 *      increasing bin order;
 *   3. grins_racipe_level_states: a value's level is the number of
 *      boundary bins below its bin; a solve's label packs its nodes'
 *      levels, node i in bits [i w, i w + w), w the bits of (boundaries +
 *      1) levels; per set, the number of distinct labels among its
 *      converged solves, and a histogram of those numbers over sets.
 * All three are exact (integer results, the FP64 normalisation rounded as
 * written), independent of launch shape and batch split. */

/* Adds the bins of the converged solves of n_sets sets to d_counts.
 *   d_params  the sets' parameter block (as for grins_racipe_integrate)
 *   d_states  double [n_sets][n_ics][N], d_status uint8 [n_sets][n_ics]
 *   d_counts  uint64 [n_bins], device, caller-zeroed; accumulates, so
 *             batches of sets add up to one histogram
 * Asynchronous on stream.  Errors: GRINS_E_INVALID_ARG for a NULL handle or
 * buffer, n_ics outside [1, 4096], n_bins outside [2, 4096]. */
grins_status grins_racipe_gk_histogram(grins_racipe_t h, const void *d_params,
                                       const double *d_states, const uint8_t *d_status,
                                       int64_t n_sets, int32_t n_ics, int32_t n_bins,
                                       unsigned long long *d_counts, void *stream);

/* Level boundaries of a histogram (host memory in and out, no GPU).
 *   h_counts  uint64 [n_bins]; half_width m >= 0 (0: no smoothing)
 *   h_bins    int32 [max_boundaries], filled with *n_out boundary bins in
 *             increasing order
 * Errors: GRINS_E_INVALID_ARG for NULL pointers, n_bins outside [2, 4096],
 * half_width outside [0, 8] (the smoothed counts stay exact in 64 bits up
 * to 2^48 values), max_boundaries outside [1, 16]. */
grins_status grins_level_boundaries(const unsigned long long *h_counts, int32_t n_bins,
                                    int32_t half_width, int32_t max_boundaries, int32_t *h_bins,
                                    int32_t *n_out);

/* Level labels, distinct states per set and the multistability histogram.
 *   h_bounds      int32 [n_bounds] boundary bins (host), increasing, in
 *                 [0, n_bins); n_bounds in [0, 16]
 *   d_labels      uint64 [n_sets][n_ics]: packed levels; 2^64 - 1 for a solve
 *                 that did not converge
 *   d_n_states    int32 [n_sets]: distinct labels among the set's converged
 *                 solves
 *   d_multi_hist  uint64 [n_ics + 1], caller-zeroed, accumulates: entry k
 *                 counts the sets with k distinct states
 * Asynchronous on stream.  Errors: GRINS_E_INVALID_ARG for a NULL handle or
 * buffer, bad sizes or unordered boundaries; GRINS_E_BUDGET when N nodes'
 * levels do not fit in 64 bits. */
grins_status grins_racipe_level_states(grins_racipe_t h, const void *d_params,
                                       const double *d_states, const uint8_t *d_status,
                                       int64_t n_sets, int32_t n_ics, int32_t n_bins,
                                       const int32_t *h_bounds, int32_t n_bounds,
                                       unsigned long long *d_labels, int32_t *d_n_states,
                                       unsigned long long *d_multi_hist, void *stream);

/* ----------------------------------------------------------------- Ising
 * Boolean Ising formalism on the handle's network (Sec. 2.2, Eq. 3): node i
 * turns on when sum_j J_ij s_j > 0, off when it is < 0, and keeps its
 * state on a tie; J_ij = +1 for an activating edge j -> i, -1 for an
 * inhibiting one.  A state is a 64-bit word, bit i set = node i on (s_i =
 * +1); an off node counts as s_i = -1, or as 0 with enc01 (the 0/1
 * encoding).  GRINS_ISING_SYNC updates every node at once,
 * GRINS_ISING_ASYNC one node per step, chosen uniformly from the
 * trajectory's counter-based stream: Philox4x64-10 with key (seed,
 * 0x4953494E47424F), draw d = word d % 4 of the block with counter
 * (trajectory, d / 4, 0, 0); step k takes draw 1 + k and the node
 * ((draw >> 32) * N) >> 32.  A trajectory stops at a fixed point (no node
 * would change: status GRINS_SS_CONVERGED, steps = updates applied before
 * it) or after max_steps updates (GRINS_SS_MAXSTEPS).
 *   d_init   uint64 [n_traj] initial states, or NULL: draw 0 of each
 *            trajectory's stream, masked to N bits
 *   d_final  uint64 [n_traj], d_steps int32 [n_traj], d_status uint8 [n_traj]
 * Asynchronous on stream.  Errors: GRINS_E_INVALID_ARG for a NULL handle or
 * output buffer, an unknown mode, n_traj < 0 or max_steps < 0. */
enum { GRINS_ISING_SYNC = 0, GRINS_ISING_ASYNC = 1 };
grins_status grins_ising_run(grins_racipe_t h, int32_t mode, int32_t enc01, uint64_t seed, int64_t n_traj,
                             const unsigned long long *d_init, int32_t max_steps,
                             unsigned long long *d_final, int32_t *d_steps, uint8_t *d_status,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRINS_RACIPE_H */

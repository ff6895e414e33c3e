// Internal definitions shared by the CUDA translation units of
// libgrins_racipe.so: parameter-block layout, device topology, kernel
// argument structs, the device Philox generator and launch declarations.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#endif

#include "grins_racipe.h"

namespace grins {

constexpr int kMaxNodes = 64;     // kernels are bucketed up to this N
constexpr int kMaxEdges = 4096;
constexpr int kWarp = 32;

// Byte layout of one parameter set (2N + 3E values, Sec. 2.1.2):
// double G[N], k[N], T[E], lam[E]; uint8 n[E]; padded to 16 bytes.
struct ParamLayout {
    int32_t N, E;
    int32_t off_G, off_k, off_T, off_lam, off_n;
    int64_t stride;
};

__host__ __device__ inline ParamLayout make_layout(int N, int E)
{
    ParamLayout L;
    L.N = N; L.E = E;
    L.off_G = 0;
    L.off_k = 8 * N;
    L.off_T = 16 * N;
    L.off_lam = 16 * N + 8 * E;
    L.off_n = 16 * N + 16 * E;
    int64_t bytes = (int64_t)16 * N + 16 * E + E;
    L.stride = (bytes + 15) / 16 * 16;
    return L;
}

// Network on the device, in-edges grouped by target (CSR).
struct DevTopo {
    int32_t N, E;
    const int32_t *off;       // [N+1] first CSR position of each target's inputs
    const int32_t *src;       // [E] source node of CSR position
    const int32_t *edge;      // [E] creation-order edge index of CSR position
    const int8_t *sign;       // [E] +1 activation / -1 inhibition
};

// ---------------------------------------------------------------- sampler
struct SampleArgs {
    ParamLayout L;
    const int8_t *edge_sign;     // [E] creation order
    const double *edge_median;   // [E] creation order: median level of the edge's source
    uint64_t seed;
    int64_t set0, n_sets;
    double G_min, G_span, k_min, k_span;
    double la_min, la_span;      // activating lambda
    double vi_min, vi_span;      // inverse inhibiting lambda
    double thr_lo, thr_span;
    int32_t n_min, n_count;
    int32_t dist_G, dist_k, dist_la, dist_li;   // GRINS_DIST_* per class
    double G_hi, k_hi, la_hi;                   // range ends (non-Table-1 draws)
    int64_t lhs_sets;                           // > 0: Latin hypercube over this many sets
    const uint32_t *sobol_v;                    // non-null: Sobol units; [D][32] direction
                                                // numbers (scrambled), then [D] shifts
    int sobol_dims;                             // D = 2N + 3E
    const grins_param_range *prange;            // non-null: per-parameter rows [2N + 3E]
    double li_min, li_max;                      // inhibiting lambda range (non-Table-1 draws)
    unsigned char *params;
};

#ifndef __CUDACC_RTC__
cudaError_t launch_sample_params(const SampleArgs &a, cudaStream_t st);
cudaError_t launch_sample_ics(int N, uint64_t seed, int n_ics, double *u, const grins_param_range *rows,
                              cudaStream_t st);
#endif

// ------------------------------------------------------------- integrator
// Lane-group layout of a network (built by the host at create time): the
// nodes sorted by in-degree and dealt out in R rows of L nodes; row r's
// in-edges fill D_r = row_deg[r] positions starting at row_off[r]; position
// p of lane j holds edge pos_edge[p * L + j] (-1: neutral padding) whose
// source value sits pos_off[p * L + j] bytes into a group's gather column.
constexpr int kGrpMaxRows = 16;
struct GrpTopo {
    int32_t L, R, P;
    const int32_t *pos_edge;     // [P * L] creation-order edge index or -1
    const int32_t *pos_off;      // [P * L] gather byte offset of the source
    const int32_t *row_node;     // [R * L] node of slot (r, j) or -1
    const int32_t *row_link;     // [R * L] 1: slot (r, j) continues slot (link_to[r], j)
    int32_t row_off[kGrpMaxRows];
    int32_t row_deg[kGrpMaxRows];
    int32_t link_to[kGrpMaxRows];  // row a row's continuation products multiply into, -1 none
};

struct IntegrateArgs {
    DevTopo topo;
    ParamLayout L;
    const unsigned char *params;
    int64_t n_sets;
    const double *ic_unit;       // [n_ics][N]
    int32_t n_ics;
    double rtol, atol, t0, t_end, ss_tol;
    double ss_near;              // residual below which the tolerances tighten (10 ss_tol)
    double ss_gain;              // factor on the squared error norm there (1 / ss_tighten^2)
    // the same in FP32 (filled with them): FP32 kernels read these as
    // constant operands instead of converting the doubles in the loop
    float f_rtol, f_atol, f_t_end, f_ss_tol, f_ss_near, f_ss_gain;
    int64_t max_steps;
    int32_t max_steps32;         // max_steps clamped to the int32 range (filled with the copies above)
    int32_t method;              // 5(4) pair: 0 Dormand-Prince, 1 Tsitouras (compiled kernels only)
    const double *t_grid;        // device copy, [n_t]
    int32_t n_t;
    double *states;              // [S][I][N]
    uint8_t *status;             // [S][I]
    double *t_final;             // nullable
    int32_t *n_steps;            // nullable
    double *series;              // [S][I][n_t][N] or null
    unsigned long long *queue;   // work counter, zero before launch
    unsigned long long *check;   // checked builds: first violation (code, info)
    int32_t slots;               // parameter-set slots per warp (upper bound)
    int32_t smem_limit;          // opt-in shared memory per block, bytes
    GrpTopo grp;                 // lane-group layout (grp.L == 0: not available)
    const void *grp_jit;         // host: kernel compiled for this layout, or null
    // Borderline re-pass (FP32 register-record kernel writes, FP64 one reads;
    // all null / zero when off).  The FP32 pass keeps a checkpoint -- the
    // first accepted state with residual < tail_chk -- and, for a solve whose
    // steady-state decision falls near t_end (t_end reached with final
    // residual < tail_rho, or converged with t_end - t < tail_late (t - t_c))
    // and which took at most tail_work attempts after its checkpoint, leaves
    // that state in `states`, appends (solve, t_c, those attempts) to
    // tail_items and bumps tail_n.  The re-pass, given the same list,
    // integrates each from its checkpoint to its status.
    struct TailItem { int64_t idx; float t; int32_t work; };
    TailItem *tail_items;        // [n_sets * n_ics] capacity
    unsigned long long *tail_n;  // [2]: items appended, re-pass attempts spent on them
    float f_tail_chk, f_tail_rho, f_tail_late;
    int32_t tail_work;
    // list mode: the statuses the re-pass writes keep kStatusListed (a
    // list-mode polish after it clears the mark; a polish running beside it
    // must not take these solves even once their status is final)
    int32_t tail_mark;
    const volatile int32_t *cancel;   // nullable: nonzero stops the hand-out of work (grins_solver_opts.cancel)
};

// Jobs of one batched launch (a plan): per-job arguments as for a single
// network (device array), the cumulative share of work up to each job, and
// the shared-memory bytes each warp's integration region takes.
struct BatchArgs {
    const IntegrateArgs *jobs;   // [n_jobs], device
    const double *cum_work;      // [n_jobs], device: cumulative work fraction
    int32_t n_jobs;
    int32_t warp_bytes;          // max over jobs of the per-warp layout (multiple of 128)
};

// One compiled launch for a plan (grins_racipe_plan_*): every job's
// register-record integrator, compiled for its network's layout, in one
// kernel; job b runs body body_of[b].  Warp w starts on the job where its
// share of the total work falls and visits every job in turn, integrating
// its solves from the job's counter until they are all handed out.  A warp's
// shared-memory region is region_bytes: its gather buffers (gather_bytes,
// the largest layout's), then a copy of the job's arguments.
struct PlanArgs {
    const IntegrateArgs *jobs;   // [n_jobs], device
    const double *cum_work;      // [n_jobs], device: cumulative work fraction
    const int32_t *body_of;      // [n_jobs], device
    int32_t n_jobs;
    int32_t gather_bytes;
    int32_t region_bytes;
};

// Maximum N served by the FP32 / FP64 integrator buckets.
#ifndef __CUDACC_RTC__
// Run-time compiled lane-group kernel for one layout (jit.cu): compiled on
// first use (grp_jit_kernel) or only looked up (grp_jit_lookup); kind is
// kJitRegisters (records in registers) or kJitShared (records in shared
// memory).  The returned pointer is an opaque handle for launch_grp_jit.
// kJitRegisters64 / kJitRegistersDD: records in registers in FP64 or in
// double-float (dd.cuh: the borderline re-pass).
enum JitKind { kJitShared = 0, kJitRegisters = 1, kJitRegisters64 = 2, kJitRegistersDD = 3 };
// method: the 5(4) pair of a register-record kernel (0 Dormand-Prince,
// 1 Tsitouras) in its low bits, plus kJitSeries for a kernel that writes
// time series (register-record kernels without it compile the grid logic
// out) and kJitTail for one taking part in the borderline re-pass; the
// shared-record kernel runs Dormand-Prince only and ignores both flags.
constexpr int kJitMethodMask = 15;
constexpr int kJitSeries = 16;
constexpr int kJitTail = 32;      // with the borderline re-pass (checkpoints / list mode)
constexpr int kJitCancel = 64;    // polling a cancel flag (grins_solver_opts.cancel)
const void *grp_jit_kernel(const GrpTopo &g, int kind, std::string *why, int method = 0);
const void *grp_jit_lookup(const GrpTopo &g, int kind, int method = 0);
// Starts (once) a background compile for layout g: 1 ready, 0 compiling, -1
// failed or unavailable.
int grp_jit_prefetch(const GrpTopo &g, int kind, int method = 0);
cudaError_t launch_grp_jit(const void *kern, const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_fp32(const IntegrateArgs &a, cudaStream_t st, int num_sms);
// Batched lane-group launch with `warps` warps per block (2 or 4); smem =
// dynamic shared memory per block.  Returns cudaErrorInvalidConfiguration
// when it does not fit.
cudaError_t launch_integrate_batch(const BatchArgs &b, int warps, cudaStream_t st, int num_sms,
                                   int smem_limit);
cudaError_t launch_integrate_fp64(const IntegrateArgs &a, cudaStream_t st, int num_sms);
// The plan kernel for the given layouts (body i compiled for layouts[i];
// FP32 Dormand-Prince, no time series, no re-pass) with `minb` resident
// blocks of `warps` warps per SM, built on first use and cached; null with
// the reason in *why.
const void *grp_jit_plan_kernel(const GrpTopo *layouts, int n_layouts, int warps, int minb, bool cancel,
                                std::string *why);
// Launch of a plan kernel: grid of resident blocks, smem = warps x region.
cudaError_t launch_plan_ct(const void *kern, const PlanArgs &p, cudaStream_t st, int num_sms, int smem_limit);
// The borderline re-pass list `in` (n_in[0] items) copied to `out` longest
// first (by the FP32 pass's attempts after the checkpoint, in buckets of
// max_work / 64), for the re-pass.
// Issue rates of ex2.approx, lg2.approx, rcp.approx, FP32 FMA, FP64 FMA,
// FP64 multiply and FP64 add (rates[0..6], operations per clock per SM) on
// the current device, from one block per SM of n_sm; d_cycles / d_sink:
// n_sm entries each (rates.cu).
cudaError_t measure_unit_rates(double *rates, cudaStream_t st, long long *d_cycles, double *d_sink, int n_sm);

cudaError_t launch_tail_order(const IntegrateArgs::TailItem *in, IntegrateArgs::TailItem *out,
                              const unsigned long long *n_in, long long cap, int max_work, cudaStream_t st);
#endif

// ----------------------------------------------------------------- polish
struct PolishArgs {
    DevTopo topo;
    ParamLayout L;
    const unsigned char *params;
    int64_t n_solves;            // S * I
    int32_t n_ics;
    double *states;              // in/out
    uint8_t *status;             // in/out
    float *err_est;              // nullable
    double tol, max_move;
    int32_t iters;
    unsigned long long *check;   // checked builds: first violation (code, info)
    const volatile int32_t *cancel;   // nullable: nonzero marks unpolished converged solves cancelled
    // list mode (non-null): polish only the solves of the re-pass list
    // (items[0 .. *n_items)), one solve per work unit
    const IntegrateArgs::TailItem *items;
    const unsigned long long *n_items;
    // non-null: warps take work units from this counter (zeroed by the
    // caller) instead of a fixed share -- the work of a unit varies with its
    // converged solves, and a polish beside another kernel starts its
    // blocks at different times
    unsigned long long *queue;
};

// Status byte of a solve the FP32 pass listed for the borderline re-pass:
// its FP32 status with this bit set, until the re-pass writes the final one
// (a polish running beside the re-pass leaves such solves alone).
constexpr uint8_t kStatusListed = 0x80;

#ifndef __CUDACC_RTC__
cudaError_t launch_polish(const PolishArgs &a, cudaStream_t st, int num_sms);
#endif

// ----------------------------------------------------------------- unique
struct UniqueArgs {
    ParamLayout L;
    const unsigned char *params;
    const double *states;
    const uint8_t *status;
    int64_t n_sets;
    int32_t n_ics;
    double tol;
    int32_t *state_id;
    int32_t *n_unique;
};

#ifndef __CUDACC_RTC__
cudaError_t launch_unique(const UniqueArgs &a, cudaStream_t st, int num_sms);
#endif

// ----------------------------------------------------------------- levels
constexpr int kMaxLevelBounds = 16;
struct LevelArgs {
    ParamLayout L;
    const unsigned char *params;
    const double *states;
    const uint8_t *status;
    int64_t n_sets;
    int32_t n_ics;
    int32_t n_bins;
    unsigned long long *counts;          // gk histogram [n_bins], accumulated
    int32_t n_bounds;                    // boundary bins, increasing
    int32_t bounds[kMaxLevelBounds];
    int32_t width;                       // label bits per node
    unsigned long long *labels;          // [S][I]
    int32_t *n_states;                   // [S]
    unsigned long long *multi_hist;      // [I + 1], accumulated
};

#ifndef __CUDACC_RTC__
cudaError_t launch_gk_histogram(const LevelArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_level_states(const LevelArgs &a, cudaStream_t st, int num_sms);
#endif

// ------------------------------------------------------------------ Ising
struct IsingArgs {
    int32_t N, mode, enc01, max_steps;
    uint64_t seed;
    int64_t n_traj;
    const unsigned long long *init;      // [n_traj] or null: random from the seed
    unsigned long long *final_state;     // [n_traj]
    int32_t *steps;                      // [n_traj]
    uint8_t *status;                     // [n_traj]
    unsigned long long act[kMaxNodes];   // per node: bits of its activating sources
    unsigned long long inh[kMaxNodes];   // and of its inhibiting ones
    int32_t n_act[kMaxNodes], n_inh[kMaxNodes];
};

#ifndef __CUDACC_RTC__
cudaError_t launch_ising(const IsingArgs &a, cudaStream_t st, int num_sms);
#endif

// ---------------------------------------------------------- cancellation
#ifdef __CUDACC__
// The cancel flag of a call (nullable), read by lane 0 and broadcast: the
// same answer on every lane of the warp.
__device__ __forceinline__ bool grins_cancelled(const volatile int32_t *flag)
{
    int v = 0;
    if (flag != nullptr && (threadIdx.x & 31) == 0) v = *flag;
    return __shfl_sync(0xffffffffu, v, 0) != 0;
}

// After a cancel: hands out every parameter set left in a set counter
// (queue, sets of n_ics solves), 32 at a time, and marks their solves
// GRINS_SS_CANCELLED; warp-uniform.
__device__ __forceinline__ void grins_cancel_sets(unsigned long long *queue, long long n_sets, int n_ics,
                                                  uint8_t *status)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (;;) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(queue, 32ull);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if ((long long)b0 >= n_sets) return;
        const long long b1 = (long long)b0 + 32 < n_sets ? (long long)b0 + 32 : n_sets;
        for (long long i = (long long)b0 * n_ics + lane; i < b1 * n_ics; i += 32) status[i] = GRINS_SS_CANCELLED;
    }
}
#endif

// ------------------------------------------------------------- device RNG
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// four-word Philox bijection with the published multipliers and Weyl key
// increments.  Used as a keyed hash of (stream key, counter): draw d of
// the stream (key, c0) is word d % 4 of the block with counter
// (c0, d / 4, 0, 0).
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                uint64_t c3, uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    U64x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Stream tags (second key word; the first is the user's seed) and the
// fixed key of the half-functional median samples.
constexpr uint64_t kTagParams = 0x52414349504550ull;  // "RACIPEP"
constexpr uint64_t kTagIcs = 0x52414349504549ull;     // "RACIPEI"
constexpr uint64_t kTagLhs = 0x5241434950454Cull;     // "RACIPEL": Latin hypercube permutations
constexpr uint64_t kTagSobol = 0x52414349504553ull;   // "RACIPES": Sobol scramble
constexpr uint64_t kKeyMedian = 0x48414C4646554E43ull; // "HALFFUNC"

// [0, 1) from the top 53 bits; exact.
__host__ __device__ __forceinline__ double unit_double(uint64_t r)
{
    return (double)(r >> 11) * 0x1.0p-53;
}

// Integer in [lo, lo + count) from the top 32 bits (multiply-shift).
__host__ __device__ __forceinline__ int32_t unit_int(uint64_t r, int32_t lo, int32_t count)
{
    return lo + (int32_t)(((r >> 32) * (uint64_t)count) >> 32);
}

}  // namespace grins

// Persistent Dormand-Prince 5(4) integrator for RACIPE ensembles.
//
// Model (GRiNS, Sec. 2.1.1, Eq. 1 and Eq. 2): for every node i
//     dx_i/dt = G_i * prod_{e into i} F_e(x_src(e)) - k_i x_i,
//     F_e = H^S / lambda (activating), H^S (inhibiting),
//     H^S(B) = lambda + (1 - lambda) / (1 + (B/T)^n).
// Written over p = (B/T)^n both factors are (a p + b) / (1 + p) with
//     activating: a = 1,      b = 1/lambda
//     inhibiting: a = lambda, b = 1,
// so a node's inputs are multiplied as one numerator and one denominator
// product and divided once per chunk of four inputs.
//
// Execution model (one GPU, persistent grid):
//   * every warp is independent; it owns `slots` parameter-set slots in
//     shared memory, each holding one set's derived coefficients;
//   * a lane integrates one (set, initial condition) solve with its own
//     step size; lanes serve ICs of the warp's slots, so a warp holds a
//     few parameter sets at once when a set has fewer ICs than lanes;
//   * a lane that terminates writes its result and takes the next pending
//     IC of a slot; a slot whose ICs are all done is refilled with the next
//     parameter set from a device-wide atomic work counter;
//   * the state y and the stage derivatives k1..k7 live in registers (node
//     loops unrolled to the bucket size NMAX), the stage input is staged per
//     lane in shared memory ([node][lane], conflict-free) because inputs are
//     gathered through the runtime topology.
// Integration follows Dormand & Prince (1980) with first-same-as-last, the
// RMS error norm scaled by atol + rtol * max(|y|, |y_new|), and the
// controller h <- h * clamp(0.9 err^(-1/5), 0.2, 10) (no growth right after a
// rejection).  A solve stops when max_i |f_i| / (G_i / k_i) < ss_tol on an
// accepted step (Sec. 2.1.3), at t_end, or after max_steps attempts.
#pragma once

#include "common.cuh"

namespace grins {

// Dormand-Prince 5(4) tableau (Dormand & Prince 1980); e = b5 - b4.
namespace dp {
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                 a54 = -212.0 / 729.0;
constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                 a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                 b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
constexpr double e1 = 71.0 / 57600.0, e3 = -71.0 / 16695.0, e4 = 71.0 / 1920.0,
                 e5 = -17253.0 / 339200.0, e6 = 22.0 / 525.0, e7 = -1.0 / 40.0;
}  // namespace dp

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------------
// Checked mode (-DGRINS_CHECKED): every computed shared/global index of the
// integrator and polish kernels is range- and alignment-checked; the first
// violation is recorded in the handle's check words (kernel argument
// `check`: code, info; no trap) and the access is redirected to a safe
// address.  Off in normal builds.
// ------------------------------------------------------------------------
#ifdef GRINS_CHECKED
__device__ __forceinline__ bool grins_check(unsigned long long *w, bool ok, unsigned code, long long info)
{
    if (!ok && w && atomicCAS(w, 0ull, (unsigned long long)code) == 0ull) w[1] = (unsigned long long)info;
    return ok;
}
#define GRINS_OK_IDX(cond, code, info) grins_check(grins_chk, (cond), (code), (long long)(info))
#else
#define GRINS_OK_IDX(cond, code, info) true
#endif

// ------------------------------------------------------------------------
// Precision policies of the generic kernel.
//   scratch(z):  what the input gather reads for a source node (B = max(z, 0))
//   edge(...):   multiplies one input into (num, den)
// p = (B / T)^n by repeated squaring, clamped so that a chunk of four
// denominators cannot overflow (FP32: 2^30, a factor changes by < 1e-7
// relative; FP64: 2^200).
// ------------------------------------------------------------------------
template <typename Real> struct Prec;

template <> struct Prec<float> {
    struct alignas(16) Edge { float invT, n, a, b; };
    __device__ static __forceinline__ float scratch(float z) { return fmaxf(z, 0.0f); }
    __device__ static __forceinline__ void edge(const Edge &q, float s, float &num, float &den)
    {
        const float r = s * q.invT;
        int m = (int)q.n;
        float p = 1.0f, base = r;
        while (m) {
            if (m & 1) p *= base;
            base *= base;
            m >>= 1;
        }
        p = fminf(p, 0x1.0p30f);
        num *= fmaf(q.a, p, q.b);
        den = fmaf(den, p, den);
    }
    __device__ static __forceinline__ float ratio(float num, float den) { return __fdividef(num, den); }
    __device__ static Edge make_edge(double T, double lam, int n, int sign)
    {
        Edge q;
        q.invT = (float)(1.0 / T);
        q.n = (float)n;
        q.a = sign > 0 ? 1.0f : (float)lam;
        q.b = sign > 0 ? (float)(1.0 / lam) : 1.0f;
        return q;
    }
};

template <> struct Prec<double> {
    struct alignas(16) Edge { double invT, n, a, b; };
    __device__ static __forceinline__ double scratch(double z) { return fmax(z, 0.0); }
    __device__ static __forceinline__ void edge(const Edge &q, double s, double &num, double &den)
    {
        const double r = s * q.invT;
        int m = (int)q.n;
        double p = 1.0, base = r;
        while (m) {
            if (m & 1) p *= base;
            base *= base;
            m >>= 1;
        }
        p = fmin(p, 0x1.0p200);
        num *= fma(q.a, p, q.b);
        den = fma(den, p, den);
    }
    __device__ static __forceinline__ double ratio(double num, double den) { return num / den; }
    __device__ static Edge make_edge(double T, double lam, int n, int sign)
    {
        Edge q;
        q.invT = 1.0 / T;
        q.n = (double)n;
        q.a = sign > 0 ? 1.0 : lam;
        q.b = sign > 0 ? 1.0 / lam : 1.0;
        return q;
    }
};


// ------------------------------------------------------------------------
// Shared state of a warp
// ------------------------------------------------------------------------
struct SlotMeta {
    long long set;   // parameter set index, -1 = empty
    int next_ic;     // next IC to hand out
    int active;      // lanes currently integrating this slot
};

// Hill exponents served by the power table of the register kernel.
constexpr int kPowTable = 6;

// One input edge of the register kernel: the power-table offset of
// (source node, n) for this parameter set, T^-n, and the factor
// coefficients a, b of (a p + b) / (1 + p).
struct alignas(16) PowEdge {
    int off;
    float invTn, a, b;
};

// Shared-memory layout of the register kernel (per block):
//   topology: CSR offsets [NMAX+1] | CSR sources [E]
//   per warp: z [NMAX][32] | powers [NMAX][6][32] | slot meta [S] | slots [S]
//   slot:     G [NMAX] | k [NMAX] | k/G [NMAX] | edges [E] (PowEdge)
template <int NMAX>
struct RegLayout {
    static __host__ __device__ int topo_bytes(int E) { return ((NMAX + 1 + E) * 4 + 15) / 16 * 16; }
    static __host__ __device__ int z_bytes() { return NMAX * kWarp * 4; }
    static __host__ __device__ int pow_bytes() { return NMAX * kPowTable * kWarp * 4; }
    static __host__ __device__ int meta_bytes(int S) { return (S * (int)sizeof(SlotMeta) + 15) / 16 * 16; }
    static __host__ __device__ int node_bytes() { return (3 * NMAX * 4 + 15) / 16 * 16; }
    static __host__ __device__ int slot_bytes(int E)
    {
        int b = node_bytes() + E * (int)sizeof(PowEdge);
        // consecutive slots start 16 bytes apart modulo 128, so that lanes of
        // different slots reading the same field hit different bank groups
        const int r = b % 128;
        b += (r <= 16) ? (16 - r) : (144 - r);
        return b;
    }
    static __host__ __device__ int warp_bytes(int E, int S)
    {
        return z_bytes() + pow_bytes() + meta_bytes(S) + S * slot_bytes(E);
    }
    static __host__ __device__ int block_bytes(int E, int S, int warps) { return topo_bytes(E) + warps * warp_bytes(E, S); }
};

// ------------------------------------------------------------------------
// Register-resident FP32 kernel (N <= NMAX <= 24, Hill exponents <= 6).
//
// Per stage every lane writes, for each node, z and the powers
// max(z,0)^1..6 into its own bank column of the warp's power table; an input
// edge then reads max(z_src,0)^n with one shared load at the per-set offset
// (src, n) and multiplies by T^-n, so p = (B/T)^n costs one load and one
// multiply.  y and k1..k7 stay in registers (node loops unrolled to NMAX).
// ------------------------------------------------------------------------
template <int NMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * kWarp)
dp5_reg_kernel(const IntegrateArgs a)
{
    constexpr unsigned FULL = 0xffffffffu;
    using LY = RegLayout<NMAX>;
    extern __shared__ __align__(16) unsigned char smem[];

    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    // exponents above the table: the generic kernel serves this launch
    if (a.nmax && *a.nmax > (unsigned long long)kPowTable) return;

    const int N = a.topo.N, E = a.topo.E, S = a.slots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    int *s_off = reinterpret_cast<int *>(smem);
    int *s_src = s_off + (NMAX + 1);
    for (int i = threadIdx.x; i <= NMAX; i += blockDim.x) s_off[i] = a.topo.off[i < N ? i : N];
    for (int e = threadIdx.x; e < E; e += blockDim.x) s_src[e] = a.topo.src[e];
    __syncthreads();

    unsigned char *wbase = smem + LY::topo_bytes(E) + warp * LY::warp_bytes(E, S);
    float *zs = reinterpret_cast<float *>(wbase) + lane;                          // z[i] at zs[i*32]
    float *pw = reinterpret_cast<float *>(wbase + LY::z_bytes()) + lane;           // pw[(i*6+n-1)*32]
    SlotMeta *meta = reinterpret_cast<SlotMeta *>(wbase + LY::z_bytes() + LY::pow_bytes());
    unsigned char *slot_base = wbase + LY::z_bytes() + LY::pow_bytes() + LY::meta_bytes(S);
    const int slot_bytes = LY::slot_bytes(E);
    const int pow_elems = NMAX * kPowTable * kWarp;

    for (int s = lane; s < S; s += kWarp) { meta[s].set = -1; meta[s].next_ic = 0; meta[s].active = 0; }
    __syncwarp();

    const float rtol = (float)a.rtol, atol = (float)a.atol;
    const float ss_tol = (float)a.ss_tol;
    const float t_end = (float)a.t_end;
    const float invN = 1.0f / (float)N;

    int my_slot = -1, my_ic = 0;
    long long my_set = 0;
    float t = 0.0f, h = 0.0f;
    int steps = 0, gidx = 0;
    bool need_k1 = false, rejected = false, exhausted = false;
    float y[NMAX], k1[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) { y[i] = 1.0f; k1[i] = 0.0f; }

    auto slot_ptr = [&](int s) -> unsigned char * {
        if (!GRINS_OK_IDX(s >= 0 && s < S, 1, s)) s = 0;
        return slot_base + s * slot_bytes;
    };

    // f = Eq. 1 at the stage input z (registers) for this lane's slot
    auto rhs = [&](const float (&z)[NMAX], float (&f)[NMAX], const unsigned char *sp) {
        const float *G = reinterpret_cast<const float *>(sp);
        const float *kd = G + NMAX;
        const PowEdge *ed = reinterpret_cast<const PowEdge *>(sp + LY::node_bytes());
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i < N) {
                const float x1 = fmaxf(z[i], 0.0f);
                const float x2 = x1 * x1, x3 = x2 * x1, x4 = x2 * x2, x5 = x4 * x1, x6 = x3 * x3;
                float *q = pw + i * kPowTable * kWarp;
                q[0] = x1; q[kWarp] = x2; q[2 * kWarp] = x3; q[3 * kWarp] = x4; q[4 * kWarp] = x5; q[5 * kWarp] = x6;
                zs[i * kWarp] = z[i];
            }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i < N) {
                float prod = 1.0f, num = 1.0f, den = 1.0f;
                const int beg = s_off[i], end = s_off[i + 1];
                int cnt = 0;
                for (int e = beg; e < end; ++e) {
                    const PowEdge r = ed[e];
                    int off = r.off;
                    if (!GRINS_OK_IDX(off >= 0 && off < pow_elems && (off & 31) == 0, 2, off)) off = 0;
                    const float p = fminf(pw[off] * r.invTn, 0x1.0p30f);
                    num *= fmaf(r.a, p, r.b);
                    den = fmaf(den, p, den);
                    if (++cnt == 4) { prod *= __fdividef(num, den); num = 1.0f; den = 1.0f; cnt = 0; }
                }
                prod *= __fdividef(num, den);
                f[i] = G[i] * prod - kd[i] * zs[i * kWarp];
            }
        }
        __syncwarp();
    };

    // load parameter set `set` into slot `s` (whole warp)
    auto stage_slot = [&](int s, long long set) {
        unsigned char *sp = slot_ptr(s);
        float *G = reinterpret_cast<float *>(sp);
        float *kd = G + NMAX;
        float *kG = G + 2 * NMAX;
        PowEdge *ed = reinterpret_cast<PowEdge *>(sp + LY::node_bytes());
        GRINS_OK_IDX(((uintptr_t)ed & 15) == 0, 3, (uintptr_t)ed);
        const unsigned char *blk = a.params + set * a.L.stride;
        const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *Td = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nd = blk + a.L.off_n;
        GRINS_OK_IDX(((uintptr_t)Gd & 7) == 0 && set >= 0 && set < a.n_sets, 4, set);
        for (int i = lane; i < NMAX; i += kWarp) {
            if (i < N) {
                const double g = Gd[i], k = kdd[i];
                G[i] = (float)g; kd[i] = (float)k; kG[i] = (float)(k / g);
            } else {
                G[i] = 0.0f; kd[i] = 0.0f; kG[i] = 0.0f;
            }
        }
        for (int e = lane; e < E; e += kWarp) {
            const int ue = a.topo.edge[e];
            int n = (int)nd[ue];
            if (!GRINS_OK_IDX(n >= 1 && n <= kPowTable && ue >= 0 && ue < E, 5, n)) n = 1;
            const double T = Td[ue], lam = ld[ue];
            double Tn = T;
            for (int m = 1; m < n; ++m) Tn *= T;
            const bool act = a.topo.sign[e] > 0;
            PowEdge r;
            r.off = (s_src[e] * kPowTable + (n - 1)) * kWarp;
            r.invTn = (float)(1.0 / Tn);
            r.a = act ? 1.0f : (float)lam;
            r.b = act ? (float)(1.0 / lam) : 1.0f;
            ed[e] = r;
        }
        __syncwarp();
    };

    auto write_series = [&](int g) {
        const long long base = ((my_set * a.n_ics + my_ic) * (long long)a.n_t + g) * N;
        double *dst = a.series + base;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) if (i < N) dst[i] = (double)y[i];
    };

    auto refill = [&]() {
        for (;;) {
            const unsigned idle = __ballot_sync(FULL, my_slot < 0);
            if (idle == 0) return;
            int s_pend = -1;
            for (int s = 0; s < S; ++s)
                if (meta[s].set >= 0 && meta[s].next_ic < a.n_ics) { s_pend = s; break; }
            if (s_pend >= 0) {
                const int first = meta[s_pend].next_ic;
                const int take = min(a.n_ics - first, __popc(idle));
                const int rank = __popc(idle & ((1u << lane) - 1u));
                if (my_slot < 0 && rank < take) {
                    my_slot = s_pend;
                    my_ic = first + rank;
                    my_set = meta[s_pend].set;
                    const unsigned char *blk = a.params + my_set * a.L.stride;
                    const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
                    const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
                    const double *u = a.ic_unit + (long long)my_ic * N;
#pragma unroll
                    for (int i = 0; i < NMAX; ++i)
                        if (i < N) y[i] = (float)((u[i] * Gd[i]) / kdd[i]);
                    t = (float)a.t0;
                    steps = 0;
                    gidx = 0;
                    need_k1 = true;
                    rejected = false;
                    while (gidx < a.n_t && a.t_grid[gidx] <= a.t0) { write_series(gidx); ++gidx; }
                }
                __syncwarp();
                if (lane == 0) { meta[s_pend].next_ic = first + take; meta[s_pend].active += take; }
                __syncwarp();
                continue;
            }
            if (exhausted) return;
            int s_free = -1;
            for (int s = 0; s < S; ++s)
                if (meta[s].set < 0 || (meta[s].next_ic >= a.n_ics && meta[s].active == 0)) { s_free = s; break; }
            if (s_free < 0) return;
            unsigned long long nxt = 0;
            if (lane == 0) nxt = atomicAdd(a.queue, 1ull);
            nxt = __shfl_sync(FULL, nxt, 0);
            if ((long long)nxt >= a.n_sets) {
                exhausted = true;
                __syncwarp();
                if (lane == 0) meta[s_free].set = -1;
                __syncwarp();
                return;
            }
            stage_slot(s_free, (long long)nxt);
            if (lane == 0) { meta[s_free].set = (long long)nxt; meta[s_free].next_ic = 0; meta[s_free].active = 0; }
            __syncwarp();
        }
    };

    auto residual = [&](const float (&f)[NMAX], const unsigned char *sp) -> float {
        const float *kG = reinterpret_cast<const float *>(sp) + 2 * NMAX;
        float r = 0.0f;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) if (i < N) r = fmaxf(r, fabsf(f[i]) * kG[i]);
        return r;
    };

    refill();

    for (;;) {
        const bool working = my_slot >= 0;
        if (!__any_sync(FULL, working)) break;
        const unsigned char *sp = slot_ptr(working ? my_slot : 0);
        bool done = false;
        uint8_t st_code = GRINS_SS_TEND;

        // first derivative and starting step of freshly assigned solves
        if (__any_sync(FULL, need_k1)) {
            float f[NMAX];
            rhs(y, f, sp);
            if (need_k1) {
                need_k1 = false;
                float d0 = 0.0f, d1 = 0.0f;
                bool fin = true;
#pragma unroll
                for (int i = 0; i < NMAX; ++i) {
                    if (i < N) {
                        k1[i] = f[i];
                        fin = fin && isfinite(f[i]);
                        const float sc = atol + rtol * fabsf(y[i]);
                        d0 += (y[i] / sc) * (y[i] / sc);
                        d1 += (f[i] / sc) * (f[i] / sc);
                    }
                }
                d0 = sqrtf(d0 * invN);
                d1 = sqrtf(d1 * invN);
                h = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * d0 / d1;
                h = fminf(h, (float)(a.t_end - a.t0));
                if (!fin) { done = true; st_code = GRINS_SS_NONFINITE; }
                else if (residual(f, sp) < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
            }
        }

        // Every lane runs the six stages (the stage right-hand sides hold
        // warp barriers); idle and finished lanes compute on scratch values
        // and only working lanes act on the result.
        {
            float t_stop = t_end;
            bool to_grid = false;
            if (gidx < a.n_t && (float)a.t_grid[gidx] < t_stop) { t_stop = (float)a.t_grid[gidx]; to_grid = true; }
            float hh = h;
            bool clipped = false;
            if (t + hh >= t_stop) { hh = t_stop - t; clipped = true; }

            float z[NMAX], k2[NMAX], k3[NMAX], k4[NMAX], k5[NMAX], k6[NMAX], k7[NMAX];
#pragma unroll
            for (int i = 0; i < NMAX; ++i) z[i] = y[i] + hh * ((float)dp::a21 * k1[i]);
            rhs(z, k2, sp);
#pragma unroll
            for (int i = 0; i < NMAX; ++i) z[i] = y[i] + hh * ((float)dp::a31 * k1[i] + (float)dp::a32 * k2[i]);
            rhs(z, k3, sp);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                z[i] = y[i] + hh * ((float)dp::a41 * k1[i] + (float)dp::a42 * k2[i] + (float)dp::a43 * k3[i]);
            rhs(z, k4, sp);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                z[i] = y[i] + hh * ((float)dp::a51 * k1[i] + (float)dp::a52 * k2[i] + (float)dp::a53 * k3[i] +
                                    (float)dp::a54 * k4[i]);
            rhs(z, k5, sp);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                z[i] = y[i] + hh * ((float)dp::a61 * k1[i] + (float)dp::a62 * k2[i] + (float)dp::a63 * k3[i] +
                                    (float)dp::a64 * k4[i] + (float)dp::a65 * k5[i]);
            rhs(z, k6, sp);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                z[i] = y[i] + hh * ((float)dp::b1 * k1[i] + (float)dp::b3 * k3[i] + (float)dp::b4 * k4[i] +
                                    (float)dp::b5 * k5[i] + (float)dp::b6 * k6[i]);
            rhs(z, k7, sp);

          if (working && !done) {
            float en = 0.0f;
            bool finite = true;
#pragma unroll
            for (int i = 0; i < NMAX; ++i) {
                if (i < N) {
                    const float err = hh * ((float)dp::e1 * k1[i] + (float)dp::e3 * k3[i] + (float)dp::e4 * k4[i] +
                                            (float)dp::e5 * k5[i] + (float)dp::e6 * k6[i] + (float)dp::e7 * k7[i]);
                    const float sc = atol + rtol * fmaxf(fabsf(y[i]), fabsf(z[i]));
                    const float q = err / sc;
                    en += q * q;
                    finite = finite && isfinite(z[i]) && isfinite(k7[i]);
                }
            }
            en *= invN;                          // squared RMS error norm
            ++steps;
            if (!finite || !isfinite(en)) {
                done = true; st_code = GRINS_SS_NONFINITE;
            } else if (en < 1.0f) {
                const float t_new = clipped ? t_stop : t + hh;
                if (!(t_new > t)) { done = true; st_code = GRINS_SS_NONFINITE; }
                t = t_new;
#pragma unroll
                for (int i = 0; i < NMAX; ++i) { y[i] = z[i]; k1[i] = k7[i]; }
                if (clipped && to_grid) {
                    while (gidx < a.n_t && (float)a.t_grid[gidx] <= t) { write_series(gidx); ++gidx; }
                }
                // controller 0.9 err^(-1/5), err = sqrt(en)
                float fac = en == 0.0f ? 10.0f : 0.9f * powf(en, -0.1f);
                fac = fminf(fac, 10.0f);
                if (rejected) fac = fminf(fac, 1.0f);
                h = hh * fac;
                rejected = false;
                if (!done) {
                    if (residual(k1, sp) < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                    else if (t >= t_end) { done = true; st_code = GRINS_SS_TEND; }
                }
            } else {
                h = hh * fmaxf(0.9f * powf(en, -0.1f), 0.2f);
                rejected = true;
            }
            if (!done && steps >= a.max_steps) { done = true; st_code = GRINS_SS_MAXSTEPS; }
          }
        }

        if (__any_sync(FULL, done)) {
            if (done) {
                const long long idx = my_set * a.n_ics + my_ic;
                if (GRINS_OK_IDX(idx >= 0 && idx < a.n_sets * a.n_ics, 6, idx)) {
                    double *dst = a.states + idx * N;
#pragma unroll
                    for (int i = 0; i < NMAX; ++i) if (i < N) dst[i] = (double)y[i];
                    a.status[idx] = st_code;
                    if (a.t_final) a.t_final[idx] = (double)t;
                    if (a.n_steps) a.n_steps[idx] = steps;
                    while (gidx < a.n_t) { write_series(gidx); ++gidx; }
                }
                atomicSub(&meta[my_slot].active, 1);
                my_slot = -1;
            }
            __syncwarp();
            refill();
        }
    }
}

template <int NMAX>
cudaError_t launch_reg_bucket(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    constexpr int WARPS = 4;
    using LY = RegLayout<NMAX>;
    auto kern = dp5_reg_kernel<NMAX, WARPS>;
    IntegrateArgs b = a;
    int smem = LY::block_bytes(b.topo.E, b.slots, WARPS);
    while (smem > b.smem_limit && b.slots > 1) smem = LY::block_bytes(b.topo.E, --b.slots, WARPS);
    if (smem > b.smem_limit) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long work_warps = (b.n_sets * b.n_ics + 31) / 32 + 1;
    long long blocks = (long long)num_sms * per_sm;
    const long long need = (work_warps + WARPS - 1) / WARPS;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, WARPS * kWarp, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace grins

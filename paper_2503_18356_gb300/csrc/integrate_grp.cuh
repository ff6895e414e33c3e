// Lane-group FP32 Dormand-Prince 5(4) integrator for RACIPE ensembles.
//
// Model (GRiNS, Sec. 2.1.1, Eq. 1 and Eq. 2): for every node i
//     dx_i/dt = G_i * prod_{e into i} F_e(x_src(e)) - k_i x_i,
//     F_e = H^S / lambda (activating), H^S (inhibiting),
//     H^S(B) = lambda + (1 - lambda) / (1 + (B/T)^n).
// With p = (B/T)^n both factors are w (p + u) / (1 + p) with u = 1/lambda
// and w = 1 (activating) or lambda (inhibiting); the w of a node's inputs
// are folded into G'_i = G_i prod_{inhibiting e into i} lambda_e once per
// parameter set.  p = 2^t with t = n log2(B) - n log2(T): log2 of every
// stage value once per node, one FMA and one ex2 per edge.  Numerators and
// denominators are multiplied in chunks of four edges (p clamped to 2^30 so a
// chunk cannot overflow) and divided once per chunk.  A row's edges are
// processed as one straight-line block (up to eight at a time) so their
// dependent shared loads and ex2 latencies overlap.
//
// Execution model (one GPU, persistent grid, warps independent):
//   * a solve (parameter set x initial condition) is spread over a group of
//     L lanes; the network's nodes are sorted by in-degree and dealt out in
//     rows of L nodes, lane j of a group owning node slot (r, j) of every
//     row r; y, k1..k7 and the stage input stay in registers, one entry per
//     row (NPL rows at most);
//   * row r's in-edges occupy D_r positions (the row's largest in-degree,
//     shorter lanes padded with neutral edges), so every lane of the warp
//     runs the same edge loop: per edge one 16-byte shared load of the
//     parameter record (n, -n log2 T, 1/lambda, gather offset) and one
//     shared load of log2 x_src from the warp's gather buffer;
//   * the gather buffer holds log2 of every group's stage input,
//     [row][lane j][group]; a lane reading node (r', j') hits bank
//     j' * 32/L + group, so the host orders each row's edges to give the L
//     lanes distinct source columns where it can; two buffers alternate, so
//     one warp barrier per right-hand side suffices;
//   * parameter records live in slots (one parameter set each, shared by
//     the groups integrating its initial conditions), owned by a half-warp;
//     a group that finishes takes the next pending initial condition of a
//     slot of its half-warp, and a slot whose initial conditions are all
//     done is refilled from the device-wide set counter.
// Integration follows Dormand & Prince (1980) with first-same-as-last, the
// RMS error norm scaled by atol + rtol * max(|y|, |y_new|), and the
// controller h <- h * clamp(0.9 err^(-1/5), 0.2, 10) (no growth right after a
// rejection).  A solve stops when max_i |f_i| / (G_i / k_i) < ss_tol on an
// accepted step (Sec. 2.1.3), at t_end, or after max_steps attempts.
#pragma once

#include "integrate.cuh"
#include "dd.cuh"

// Minimum resident blocks per SM the register allocation targets (4 warps
// per block; 3 -> at most 168 registers per thread).
#ifndef GRINS_GRP_MINB
#define GRINS_GRP_MINB 3
#endif

namespace grins {

// Shared-memory layout of one warp of the group kernel:
//   gather buffers 2 x [R][32] float | slot meta [S] | slots [S]
//   slot: edge records [P][L] float4 (n, -n log2 T, 1/lambda, gather offset)
//         | node records [R][L] float2 (G', k) | [R][L] float k/G | pad
// A half-warp holds the lanes of max(1, L/2) values of j; a slot is padded
// to 16 * max(1, L/2) bytes past a multiple of 128, so that the records the
// half-warp reads at one position from all slots of the warp (at most
// 128 / (16 max(1, L/2)) of them) fall into distinct banks.
struct GrpLayout {
    int L, R, P, S;
    __host__ __device__ int gather_bytes() const { return 2 * R * kWarp * 4; }
    __host__ __device__ int meta_bytes() const { return (S * (int)sizeof(SlotMeta) + 127) / 128 * 128; }
    __host__ __device__ int edge_bytes() const { return P * L * 16; }
    __host__ __device__ int node_bytes() const { return R * L * 8; }
    __host__ __device__ int slot_bytes() const
    {
        const int b = edge_bytes() + node_bytes() + R * L * 4;
        const int step = 16 * (L > 2 ? L / 2 : 1);
        const int r = (b + 128 - step) % 128;   // pad to step mod 128
        return b + (r ? 128 - r : 0);
    }
    __host__ __device__ int warp_bytes() const
    {
        return (gather_bytes() + meta_bytes() + S * slot_bytes() + 127) / 128 * 128;
    }
};

// Dynamic shared memory of one warp of the register-record kernel
// (integrate_rr.cuh): two gather buffers [planes][rows][32] entries of el
// bytes (FP32: 1 plane of log2 x; FP64: 6 planes x .. x^6).
__host__ __device__ constexpr int rr_warp_bytes(int rows, int planes, int el)
{
    return 2 * planes * rows * kWarp * el;
}

// The double-float kernel keeps its edge records in shared memory instead
// of registers (its right-hand side then runs each row's positions as a
// loop, code that fits the instruction cache): after the gather buffers,
// [positions][32 lanes] records of 16 bytes ((1/T)^n and 1/lambda, each a
// pair of FP32 numbers) and [positions][32 lanes] gather addresses.
__host__ __device__ constexpr int rr_dd_warp_bytes(int rows, int positions)
{
    return rr_warp_bytes(rows, 6, 8) + (positions > 0 ? positions : 1) * kWarp * 20;
}

// Lanes of a group are j-major: lane = j * (32 / L) + g, so lane j of every
// group sits in one contiguous block and a group's lanes are 32/L apart.
// Scheduling domains of four consecutive groups: domains per warp.
__host__ __device__ inline int grp_domains(int L)
{
    const int gs = kWarp / L;
    return gs < 4 ? 1 : gs / 4;
}
__device__ __forceinline__ float grp_sum(float v, int L)
{
    for (int o = kWarp / L; o < kWarp; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float grp_max(float v, int L)
{
    for (int o = kWarp / L; o < kWarp; o <<= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ bool grp_all(bool v, int L)
{
    int x = v ? 1 : 0;
    for (int o = kWarp / L; o < kWarp; o <<= 1) x &= __shfl_xor_sync(0xffffffffu, x, o);
    return x != 0;
}

// One edge position: multiplies the factor's numerator p + u into num and
// its denominator 1 + p into den, p = 2^min(n log2 x_src - n log2 T, 30).
struct GrpCtx {
    const float4 *ed;            // this lane's column of the slot's edge records
    const unsigned char *gcol;   // this group's column of the gather buffer
    int L, lim_pi, lim_off;
    unsigned long long *grins_chk;
};

__device__ __forceinline__ void grp_edge(const GrpCtx &c, int pi, float &num, float &den)
{
    unsigned long long *grins_chk = c.grins_chk;
    (void)grins_chk;
    if (!GRINS_OK_IDX(pi >= 0 && pi < c.lim_pi, 32, pi)) pi = 0;
    const float4 e = c.ed[pi];
    int off = __float_as_int(e.w);
    if (!GRINS_OK_IDX(off >= 0 && off < c.lim_off && (off & 3) == 0, 33, off)) off = 0;
    const float ls = *reinterpret_cast<const float *>(c.gcol + off);
    const float pw = ex2_approx(fminf(fmaf(e.x, ls, e.y), 30.0f));
    num *= pw + e.z;
    den = fmaf(den, pw, den);
}

// Product over the D positions of a row starting at record index pi (D is
// the same for every lane of the warp).
//  * Compile-time layout (the kernel compiled at run time for one network,
//    GRINS_GRP_CT): D is a constant, the loop unrolls into one straight-line
//    block per row and rows follow each other without branches.
//  * Run-time layout: chunks of four in a loop, then the remainder.
// One division per four factors keeps the partial products finite.
#ifdef GRINS_GRP_CT
template <int D>
__device__ __forceinline__ float grp_row_ct(const GrpCtx &c, int pi)
{
    float prod = 1.0f;
#pragma unroll
    for (int m = 0; m < D; m += 4) {
        float num = 1.0f, den = 1.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (m + q < D) grp_edge(c, pi + (m + q) * c.L, num, den);
        }
        prod *= div_approx(num, den);
    }
    return prod;
}

// Rows r, r+1, ... of the compile-time layout (GrpRowCt<r>::off / ::deg and
// kGrpCtRows come from the generated prelude of the run-time compile):
// z[r] <- G'_r prod_r - k_r z[r].
template <int r, int NPL>
__device__ __forceinline__ void grp_rows_ct(const GrpCtx &c, const float2 *nd, float (&z)[NPL])
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        const float prod = grp_row_ct<GrpRowCt<r>::deg>(c, GrpRowCt<r>::off * c.L);
        const float2 nr = nd[r * c.L];
        z[r] = fmaf(nr.x, prod, -nr.y * z[r]);
        grp_rows_ct<r + 1, NPL>(c, nd, z);
    }
}
#endif

__device__ __forceinline__ float grp_row_rt(const GrpCtx &c, int pi, int D)
{
    const int pend = pi + D * c.L;
    float prod = 1.0f;
#pragma unroll 1
    for (; pi + 4 * c.L <= pend; pi += 4 * c.L) {
        float num = 1.0f, den = 1.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) grp_edge(c, pi + q * c.L, num, den);
        prod *= div_approx(num, den);
    }
    if (pi < pend) {
        float num = 1.0f, den = 1.0f;
#pragma unroll 1
        for (; pi < pend; pi += c.L) grp_edge(c, pi, num, den);
        prod *= div_approx(num, den);
    }
    return prod;
}

// Body of the lane-group kernel.  NPL: node rows per lane (register arrays);
// LC, RC: lanes per group and rows when fixed at compile time (0: read from
// the launch arguments).
template <int NPL, int WARPS, int LC, int RC>
__device__ __forceinline__ void grp_body(const IntegrateArgs &a, unsigned char *wbase)
{
    constexpr unsigned FULL = 0xffffffffu;
    unsigned long long *grins_chk = a.check;
    (void)grins_chk;

    const GrpTopo &gt = a.grp;
    const int N = a.topo.N, L = LC ? LC : gt.L, R = RC ? RC : gt.R, P = gt.P, S = a.slots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int GS = kWarp / L;                    // groups per warp
    const int j = lane / GS, g = lane - j * GS;  // lane within group, group (j-major)
    const int col = lane;                        // this lane's column in a gather row
    // scheduling domains: four consecutive groups (one lane quad per j), so
    // a 16-byte record load serves a quad from at most its domain's slots
    const int DG = GS < 4 ? GS : 4;              // groups per domain
    const int NDOM = GS / DG;                    // domains per warp
    const int SD = S / NDOM;                     // slots per domain
    const GrpLayout LY{L, R, P, S};

    (void)warp;
    float *gbuf = reinterpret_cast<float *>(wbase);
    SlotMeta *meta = reinterpret_cast<SlotMeta *>(wbase + LY.gather_bytes());
    unsigned char *slot_base = wbase + LY.gather_bytes() + LY.meta_bytes();
    const int slot_bytes = LY.slot_bytes();

    for (int s = lane; s < S; s += kWarp) { meta[s].set = -1; meta[s].next_ic = 0; meta[s].active = 0; }
    // slots start zeroed: records of a slot no set has reached yet still
    // hold an in-range gather offset (0) for groups computing on scratch
#pragma unroll 1
    for (int i = lane; i < S * slot_bytes / 16; i += kWarp)
        reinterpret_cast<float4 *>(slot_base)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
    for (int i = lane; i < 2 * R * kWarp; i += kWarp) gbuf[i] = 0.0f;
    __syncwarp();

    const float rtol = a.f_rtol, atol = a.f_atol;
    const float ss_tol = a.f_ss_tol;
    const float t_end = a.f_t_end;
    const float invN = 1.0f / (float)N;

    int my_slot = -1, my_ic = 0;
    long long my_set = 0;
    float t = 0.0f, h = 0.0f;
    int steps = 0, gidx = 0, buf = 0;
    bool near = false;               // residual below ss_near: tolerances tightened
    const float ss_near = a.f_ss_near, ss_gain = a.f_ss_gain;
    bool need_k1 = false, rejected = false, exhausted = false;
    // y: state; k1..k6: stage derivatives; z: stage input, overwritten by
    // the right-hand side.  The last stage input (the fifth-order solution)
    // is built in k2, which no later stage reads, and its right-hand side
    // (k7) is left in z.
    float y[NPL], k1[NPL], k2[NPL], k3[NPL], k4[NPL], k5[NPL], k6[NPL], z[NPL];
#pragma unroll
    for (int r = 0; r < NPL; ++r) y[r] = k1[r] = k2[r] = k3[r] = k4[r] = k5[r] = k6[r] = z[r] = 0.0f;

    auto slot_ptr = [&](int s) -> unsigned char * {
        if (!GRINS_OK_IDX(s >= 0 && s < S, 31, s)) s = 0;
        return slot_base + s * slot_bytes;
    };

    // z <- Eq. 1 at the stage input z, for this lane's rows
    auto rhs = [&](const unsigned char *sp) {
        float *gb = gbuf + buf * (R * kWarp);
        buf ^= 1;
#pragma unroll
        for (int r = 0; r < NPL; ++r)
            if (r < R) gb[r * kWarp + col] = lg2_approx(fabsf(z[r]));   // |z|: see rr_put
        __syncwarp();
        GrpCtx c;
        c.ed = reinterpret_cast<const float4 *>(sp) + j;
        c.gcol = reinterpret_cast<const unsigned char *>(gb) + 4 * g;
        c.L = L;
        c.lim_pi = P * L;
        c.lim_off = R * kWarp * 4;
        c.grins_chk = grins_chk;
        const float2 *nd = reinterpret_cast<const float2 *>(sp + LY.edge_bytes()) + j;
#ifdef GRINS_GRP_CT
        grp_rows_ct<0, NPL>(c, nd, z);
#else
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            if (r < R) {
                const float prod = grp_row_rt(c, gt.row_off[r] * L, gt.row_deg[r]);
                const float2 nr = nd[r * L];
                z[r] = fmaf(nr.x, prod, -nr.y * z[r]);
            }
        }
#endif
    };

    // parameter set `set` -> slot `s` (whole warp)
    auto stage_slot = [&](int s, long long set) {
        unsigned char *sp = slot_ptr(s);
        float4 *ed = reinterpret_cast<float4 *>(sp);
        float2 *nd = reinterpret_cast<float2 *>(sp + LY.edge_bytes());
        float *nkg = reinterpret_cast<float *>(sp + LY.edge_bytes() + LY.node_bytes());
        if (!GRINS_OK_IDX(set >= 0 && set < a.n_sets, 34, set)) set = 0;
        const unsigned char *blk = a.params + set * a.L.stride;
        const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *Td = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nn = blk + a.L.off_n;
#pragma unroll 1
        for (int i = lane; i < P * L; i += kWarp) {
            const int e = gt.pos_edge[i];
            float4 rec;
            rec.w = __int_as_float(gt.pos_off[i]);
            if (e >= 0) {
                const float n = (float)nn[e];
                rec.x = n;
                rec.y = -n * log2f((float)Td[e]);
                rec.z = (float)(1.0 / ld[e]);
            } else {     // neutral edge: F = (p + 1) / (1 + p) = 1
                rec.x = 1.0f; rec.y = -100.0f; rec.z = 1.0f;
            }
            ed[i] = rec;
        }
#pragma unroll 1
        for (int i = lane; i < R * L; i += kWarp) {
            const int node = gt.row_node[i];
            float2 rec = make_float2(0.0f, 1.0f);
            float kg = 0.0f;
            if (node >= 0) {
                const double G = Gd[node], k = kdd[node];
                double Gp = G;
#pragma unroll 1
                for (int c = a.topo.off[node]; c < a.topo.off[node + 1]; ++c)
                    if (a.topo.sign[c] < 0) Gp *= ld[a.topo.edge[c]];
                rec.x = (float)Gp;
                rec.y = (float)k;
                kg = (float)(k / G);
            }
            nd[i] = rec;
            nkg[i] = kg;
        }
        __syncwarp();
    };

    auto write_series = [&](int gi) {
        double *dst = a.series + ((my_set * a.n_ics + my_ic) * (long long)a.n_t + gi) * N;
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            if (r < R) {
                const int node = gt.row_node[r * L + j];
                if (node >= 0) dst[node] = (double)y[r];
            }
        }
    };

    // Work assignment.  Each half-warp (the whole warp when a group spans
    // more than half of it) is a scheduling domain with its own slots: a
    // 16-byte shared load serves a half-warp in one pass when its lanes read
    // at most four distinct 16-byte records, which two slots of a half-warp
    // of two-lane groups never exceed.
    auto refill = [&]() {
        if (a.cancel != nullptr && !exhausted && grins_cancelled(a.cancel)) {
            // cancelled: the initial conditions still pending in this warp's
            // slots and every set left in the counter are marked, not started
#pragma unroll 1
            for (int sl = 0; sl < NDOM * SD; ++sl) {
                const long long set = meta[sl].set;
                const int first = meta[sl].next_ic;
                if (set >= 0 && first < a.n_ics)
                    for (int ic = first + lane; ic < a.n_ics; ic += kWarp) a.status[set * a.n_ics + ic] = GRINS_SS_CANCELLED;
                __syncwarp();
                if (lane == 0 && set >= 0 && first < a.n_ics) meta[sl].next_ic = a.n_ics;
                __syncwarp();
            }
            grins_cancel_sets(a.queue, a.n_sets, a.n_ics, a.status);
            exhausted = true;
            return;
        }
#pragma unroll 1
        for (int d = 0; d < NDOM; ++d) {
            // the domain's groups are bits d*DG .. d*DG+DG-1 of the ballot
            // below (taken at the lanes j = 0, lane = g)
            const unsigned dmask = (DG == 32 ? FULL : ((1u << DG) - 1u)) << (d * DG);
            const bool in_dom = g / DG == d;
            const int s_lo = d * SD, s_hi = s_lo + SD;
#pragma unroll 1
            for (;;) {
                // one bit per idle group of the domain, at its first lane
                const unsigned idle = __ballot_sync(FULL, my_slot < 0 && j == 0) & dmask;
                if (idle == 0) break;
                int s_pend = -1;
#pragma unroll 1
                for (int s = s_lo; s < s_hi; ++s)
                    if (meta[s].set >= 0 && meta[s].next_ic < a.n_ics) { s_pend = s; break; }
                if (s_pend >= 0) {
                    const int first = meta[s_pend].next_ic;
                    const int take = min(a.n_ics - first, __popc(idle));
                    const int rank = __popc(idle & ((1u << g) - 1u));
                    if (in_dom && my_slot < 0 && rank < take) {
                        my_slot = s_pend;
                        my_ic = first + rank;
                        my_set = meta[s_pend].set;
                        const unsigned char *blk = a.params + my_set * a.L.stride;
                        const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
                        const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
                        const double *u = a.ic_unit + (long long)my_ic * N;
#pragma unroll
                        for (int r = 0; r < NPL; ++r) {
                            y[r] = 0.0f;
                            if (r < R) {
                                const int node = gt.row_node[r * L + j];
                                if (node >= 0) y[r] = __fdividef((float)u[node] * (float)Gd[node], (float)kdd[node]);
                            }
                        }
                        t = (float)a.t0;
                        steps = 0;
                        gidx = 0;
                        need_k1 = true;
                        rejected = false;
                        near = false;
#pragma unroll 1
                        while (gidx < a.n_t && a.t_grid[gidx] <= a.t0) { write_series(gidx); ++gidx; }
                    }
                    __syncwarp();
                    if (lane == 0) { meta[s_pend].next_ic = first + take; meta[s_pend].active += take; }
                    __syncwarp();
                    continue;
                }
                if (exhausted) break;
                int s_free = -1;
#pragma unroll 1
                for (int s = s_lo; s < s_hi; ++s)
                    if (meta[s].set < 0 || (meta[s].next_ic >= a.n_ics && meta[s].active == 0)) { s_free = s; break; }
                if (s_free < 0) break;
                unsigned long long nxt = 0;
                if (lane == 0) nxt = atomicAdd(a.queue, 1ull);
                nxt = __shfl_sync(FULL, nxt, 0);
                if ((long long)nxt >= a.n_sets) {
                    exhausted = true;
                    __syncwarp();
                    if (lane == 0) meta[s_free].set = -1;
                    __syncwarp();
                    break;
                }
                stage_slot(s_free, (long long)nxt);
                if (lane == 0) { meta[s_free].set = (long long)nxt; meta[s_free].next_ic = 0; meta[s_free].active = 0; }
                __syncwarp();
            }
        }
    };

    // max_i |v_i| k_i / G_i over the group
    auto residual = [&](const float (&v)[NPL], const unsigned char *sp) -> float {
        const float *nkg = reinterpret_cast<const float *>(sp + LY.edge_bytes() + LY.node_bytes()) + j;
        float r = 0.0f;
#pragma unroll
        for (int q = 0; q < NPL; ++q)
            if (q < R) r = fmaxf(r, fabsf(v[q]) * nkg[q * L]);
        return grp_max(r, L);
    };

    // warp-wide: some group is working / has just been given a solve (they
    // change only when a group finishes and the warp refills)
    bool any_work = false, any_new = false;
    auto refresh = [&]() {
        any_work = __any_sync(FULL, my_slot >= 0);
        any_new = __any_sync(FULL, need_k1);
    };
    refill();
    refresh();

#pragma unroll 1
    for (;;) {
        const bool working = my_slot >= 0;
        if (!any_work) break;
        const unsigned char *sp = slot_ptr(working ? my_slot : 0);
        bool done = false;
        int st_code = GRINS_SS_TEND;
        float t_stop = t_end, hh = 0.0f;
        bool to_grid = false, clipped = false;

        // s = 0: first derivative and starting step of freshly assigned
        // solves (only when some group has one); s = 1..6: the stages of one
        // step attempt, f -> k2 .. k6, then k7 (kept in k2).  Every lane runs
        // every right-hand side (they hold warp barriers); idle and finished
        // groups compute on scratch values and only working groups act.
        const int s0 = any_new ? 0 : 1;
        any_new = false;
        auto stage = [&](const int s) {
            if (s == 0) {
#pragma unroll
                for (int r = 0; r < NPL; ++r) z[r] = y[r];
            } else {
                if (s == 1) {
                    if (gidx < a.n_t && (float)a.t_grid[gidx] < t_stop) { t_stop = (float)a.t_grid[gidx]; to_grid = true; }
                    hh = h;
                    if (t + hh >= t_stop) { hh = t_stop - t; clipped = true; }
                }
                if (s == 1) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R) z[r] = y[r] + hh * ((float)dp::a21 * k1[r]);
                } else if (s == 2) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R) z[r] = y[r] + hh * ((float)dp::a31 * k1[r] + (float)dp::a32 * k2[r]);
                } else if (s == 3) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R)
                            z[r] = y[r] + hh * ((float)dp::a41 * k1[r] + (float)dp::a42 * k2[r] +
                                                (float)dp::a43 * k3[r]);
                } else if (s == 4) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R)
                            z[r] = y[r] + hh * ((float)dp::a51 * k1[r] + (float)dp::a52 * k2[r] +
                                                (float)dp::a53 * k3[r] + (float)dp::a54 * k4[r]);
                } else if (s == 5) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R)
                            z[r] = y[r] + hh * ((float)dp::a61 * k1[r] + (float)dp::a62 * k2[r] +
                                                (float)dp::a63 * k3[r] + (float)dp::a64 * k4[r] +
                                                (float)dp::a65 * k5[r]);
                } else {
#pragma unroll
                    for (int r = 0; r < NPL; ++r)
                        if (r < R) {
                            k2[r] = y[r] + hh * ((float)dp::b1 * k1[r] + (float)dp::b3 * k3[r] +
                                                 (float)dp::b4 * k4[r] + (float)dp::b5 * k5[r] +
                                                 (float)dp::b6 * k6[r]);
                            z[r] = k2[r];
                        }
                }
            }
            rhs(sp);
            if (s == 0) {
                float d0 = 0.0f, d1 = 0.0f;
                bool fin = true;
#pragma unroll
                for (int r = 0; r < NPL; ++r) {
                    if (r < R) {
                        fin = fin && isfinite(z[r]);
                        const float isc = __fdividef(1.0f, atol + rtol * fabsf(y[r]));
                        d0 += (y[r] * isc) * (y[r] * isc);
                        d1 += (z[r] * isc) * (z[r] * isc);
                    }
                }
                d0 = sqrtf(grp_sum(d0, L) * invN);
                d1 = sqrtf(grp_sum(d1, L) * invN);
                fin = grp_all(fin, L);
                const float res = residual(z, sp);
                if (need_k1) {
                    need_k1 = false;
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k1[r] = z[r];
                    h = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * d0 / d1;
                    h = fminf(h, (float)(a.t_end - a.t0));
                    if (!fin) { done = true; st_code = GRINS_SS_NONFINITE; }
                    else if (res < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                }
            } else {
                if (s == 1) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k2[r] = z[r];
                } else if (s == 2) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k3[r] = z[r];
                } else if (s == 3) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k4[r] = z[r];
                } else if (s == 4) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k5[r] = z[r];
                } else if (s == 5) {
#pragma unroll
                    for (int r = 0; r < NPL; ++r) k6[r] = z[r];
                }
            }
        };
#if defined(GRINS_GRP_CT) && !defined(GRINS_GRP_ROLL_STAGES)
        // compile-time layout: every stage inlined, so k_{s+1} = z renames
        // registers instead of copying them
        if (s0 == 0) stage(0);
        stage(1); stage(2); stage(3); stage(4); stage(5); stage(6);
#else
#pragma unroll 1
        for (int s = s0; s <= 6; ++s) stage(s);
#endif

        // error estimate and step control; k2 now holds the fifth-order
        // solution and z its derivative k7.  A non-finite stage derivative
        // makes err non-finite -- through the error weights or through the
        // later stages it feeds -- and with it the norm, the only finiteness
        // test needed.
        float en = 0.0f;
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            if (r < R) {
                const float err = hh * ((float)dp::e1 * k1[r] + (float)dp::e3 * k3[r] + (float)dp::e4 * k4[r] +
                                        (float)dp::e5 * k5[r] + (float)dp::e6 * k6[r] + (float)dp::e7 * z[r]);
                const float sc = atol + rtol * fmaxf(fabsf(y[r]), fabsf(k2[r]));
                const float q = div_approx(err, sc);
                en += q * q;
            }
        }
        en = grp_sum(en, L) * invN;                   // squared RMS error norm
        if (near) en *= ss_gain;
        const float res = residual(z, sp);

        if (working && !done) {
            ++steps;
            // controller 0.9 err^(-1/5), err = sqrt(en), evaluated once for
            // accepted and rejected attempts (en = 0 gives +inf, which the
            // growth limit clamps)
            const float fr = 0.9f * ex2_approx(-0.1f * lg2_approx(en));
            if (!isfinite(en)) {
                done = true; st_code = GRINS_SS_NONFINITE;
            } else if (en < 1.0f) {
                const float t_new = clipped ? t_stop : t + hh;
                if (!(t_new > t)) { done = true; st_code = GRINS_SS_NONFINITE; }
                t = t_new;
#pragma unroll
                for (int r = 0; r < NPL; ++r) if (r < R) { y[r] = k2[r]; k1[r] = z[r]; }
                if (clipped && to_grid) {
#pragma unroll 1
                    while (gidx < a.n_t && (float)a.t_grid[gidx] <= t) { write_series(gidx); ++gidx; }
                }
                h = hh * fminf(fr, rejected ? 1.0f : 10.0f);   // no growth right after a rejection
                rejected = false;
                near = res < ss_near;
                if (!done) {
                    if (res < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                    else if (t >= t_end) { done = true; st_code = GRINS_SS_TEND; }
                }
            } else {
                h = hh * fmaxf(fr, 0.2f);
                rejected = true;
            }
            if (!done && steps >= a.max_steps32) { done = true; st_code = GRINS_SS_MAXSTEPS; }
        }

        if (__any_sync(FULL, done)) {
            if (done) {
                long long idx = my_set * a.n_ics + my_ic;
                if (!GRINS_OK_IDX(idx >= 0 && idx < a.n_sets * a.n_ics, 35, idx)) idx = 0;
                double *dst = a.states + idx * N;
#pragma unroll
                for (int r = 0; r < NPL; ++r) {
                    if (r < R) {
                        const int node = gt.row_node[r * L + j];
                        if (node >= 0) dst[node] = (double)y[r];
                    }
                }
                if (j == 0) {
                    a.status[idx] = (uint8_t)st_code;
                    if (a.t_final) a.t_final[idx] = (double)t;
                    if (a.n_steps) a.n_steps[idx] = steps;
                }
#pragma unroll 1
                while (gidx < a.n_t) { write_series(gidx); ++gidx; }
                if (j == 0) atomicSub(&meta[my_slot].active, 1);
                my_slot = -1;
            }
            __syncwarp();
            refill();
            refresh();
        }
    }
}

// Single network: warp w of the block owns bytes [w * warp_bytes, ...) of
// the block's dynamic shared memory.
template <int NPL, int WARPS, int LC, int RC>
__device__ __forceinline__ void grp_body(const IntegrateArgs &a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const GrpLayout LY{LC ? LC : a.grp.L, RC ? RC : a.grp.R, a.grp.P, a.slots};
    grp_body<NPL, WARPS, LC, RC>(a, smem + (threadIdx.x >> 5) * LY.warp_bytes());
}

#ifndef __CUDACC_RTC__
// Many networks in one launch (a plan, grins_racipe_plan_create): warp w
// starts on the job where its share of the total work falls and then visits
// every job in turn, integrating sets from that job's work counter until it
// is exhausted.  The job's arguments are copied into the warp's shared
// memory (after its fixed-size integration region) so the body reads them
// with broadcast loads.
template <int NPL, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * kWarp, MINB)
dp5_grp_batch_kernel(const BatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int region = b.warp_bytes + (int)((sizeof(IntegrateArgs) + 127) / 128 * 128);
    unsigned char *wbase = smem + warp * region;
    IntegrateArgs *ja = reinterpret_cast<IntegrateArgs *>(wbase + b.warp_bytes);
    const double share = ((double)(blockIdx.x * WARPS + warp) + 0.5) / ((double)gridDim.x * WARPS);
    int b0 = 0;
    while (b0 + 1 < b.n_jobs && b.cum_work[b0] <= share) ++b0;
    for (int k = 0; k < b.n_jobs; ++k) {
        const int jb = (b0 + k) % b.n_jobs;
        const unsigned *src = reinterpret_cast<const unsigned *>(b.jobs + jb);
        unsigned *dst = reinterpret_cast<unsigned *>(ja);
        for (int i = lane; i < (int)(sizeof(IntegrateArgs) / 4); i += kWarp) dst[i] = src[i];
        __syncwarp();
        // one warp-uniform decision: skip a job whose sets are all handed out
        unsigned long long q = 0;
        if (lane == 0) q = *reinterpret_cast<volatile unsigned long long *>(ja->queue);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q < (unsigned long long)ja->n_sets) grp_body<NPL, WARPS, 0, 0>(*ja, wbase);
        __syncwarp();
    }
}

template <int NPL, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * kWarp, MINB)
dp5_grp_kernel(const IntegrateArgs a)
{
    grp_body<NPL, WARPS, 0, 0>(a);
}

template <int NPL, int MINB>
cudaError_t launch_grp_bucket(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    constexpr int WARPS = 4;
    auto kern = dp5_grp_kernel<NPL, WARPS, MINB>;
    IntegrateArgs b = a;
    const int ndom = grp_domains(b.grp.L);
    GrpLayout LY{b.grp.L, b.grp.R, b.grp.P, b.slots};
    while (WARPS * LY.warp_bytes() > b.smem_limit && LY.S > ndom) LY.S = (b.slots -= ndom);
    const int smem = WARPS * LY.warp_bytes();
    if (smem > b.smem_limit) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int groups = kWarp / b.grp.L;
    const long long work_warps = (b.n_sets * b.n_ics + groups - 1) / groups + 1;
    long long blocks = (long long)num_sms * per_sm;
    const long long need = (work_warps + WARPS - 1) / WARPS;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, WARPS * kWarp, smem, st>>>(b);
    return cudaGetLastError();
}
#endif  // __CUDACC_RTC__

}  // namespace grins

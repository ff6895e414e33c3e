// Generic persistent Dormand-Prince 5(4) kernel for any N (runtime size).
//
// Same model, solver and work distribution as the register-resident kernel
// of integrate.cuh, but every per-lane vector lives in shared memory as
// [vector][node][lane] (each lane owns one bank column, so the accesses are
// conflict-free) and loops over nodes and stages are runtime loops.  It
// serves the double-precision solver and FP32 networks above the register
// buckets.  One warp per block; the block's shared memory holds
//   topology | slot metadata | 9 vectors x N x 32 lanes | slots.
// Vector roles per lane: {0,1} = y and the stage input (swapped on accept),
// {2,3} = k1 and k2 (k7 is written over k2, which no later stage reads, and
// the two swap on accept: first same as last), 4..7 = k3..k6, 8 = the
// gathered form of the stage input, max(z, 0).  Hill powers are taken by
// repeated squaring, so any integer exponent is served.
#pragma once

#include "integrate.cuh"

namespace grins {

template <typename Real> struct DPTable {
    Real a[7][6];
    Real e[7];
};

#define GRINS_DP_TABLE(R)                                                                      \
    {{{0}, {(R)dp::a21}, {(R)dp::a31, (R)dp::a32}, {(R)dp::a41, (R)dp::a42, (R)dp::a43},      \
      {(R)dp::a51, (R)dp::a52, (R)dp::a53, (R)dp::a54},                                        \
      {(R)dp::a61, (R)dp::a62, (R)dp::a63, (R)dp::a64, (R)dp::a65},                            \
      {(R)dp::b1, 0, (R)dp::b3, (R)dp::b4, (R)dp::b5, (R)dp::b6}},                             \
     {(R)dp::e1, 0, (R)dp::e3, (R)dp::e4, (R)dp::e5, (R)dp::e6, (R)dp::e7}}

// Stage coefficients in constant memory (read with warp-uniform indices).
static __constant__ DPTable<float> c_dp_f = GRINS_DP_TABLE(float);
static __constant__ DPTable<double> c_dp_d = GRINS_DP_TABLE(double);

template <typename Real>
__device__ __forceinline__ const DPTable<Real> &dp_table();
template <> __device__ __forceinline__ const DPTable<float> &dp_table<float>() { return c_dp_f; }
template <> __device__ __forceinline__ const DPTable<double> &dp_table<double>() { return c_dp_d; }

struct GenericLayout {
    int N, E, S, real;
    __host__ __device__ int topo_bytes() const { return ((N + 1 + E) * 4 + 15) / 16 * 16; }
    __host__ __device__ int meta_bytes() const { return S * (int)sizeof(SlotMeta); }
    __host__ __device__ int vec_bytes() const { return 9 * N * kWarp * real; }
    __host__ __device__ int node_bytes() const { return (3 * N * real + 15) / 16 * 16; }
    __host__ __device__ int slot_bytes() const
    {
        int b = node_bytes() + E * 4 * real;
        b = (b + 15) / 16 * 16;
        int r = b % 128;
        b += (r <= 16) ? (16 - r) : (144 - r);
        return b;
    }
    __host__ __device__ int total() const { return topo_bytes() + meta_bytes() + vec_bytes() + S * slot_bytes(); }
};

template <typename Real>
__global__ void __launch_bounds__(kWarp)
dp5_generic_kernel(const IntegrateArgs a)
{
    using P = Prec<Real>;
    using Edge = typename P::Edge;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];

    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    const int N = a.topo.N, E = a.topo.E, S = a.slots;
    const int lane = threadIdx.x;
    const GenericLayout LY{N, E, S, (int)sizeof(Real)};
    const DPTable<Real> &tab = dp_table<Real>();

    int *s_off = reinterpret_cast<int *>(smem);
    int *s_src = s_off + (N + 1);
    SlotMeta *meta = reinterpret_cast<SlotMeta *>(smem + LY.topo_bytes());
    Real *vec = reinterpret_cast<Real *>(smem + LY.topo_bytes() + LY.meta_bytes());
    unsigned char *slot_base = smem + LY.topo_bytes() + LY.meta_bytes() + LY.vec_bytes();
    const int slot_bytes = LY.slot_bytes();

    for (int i = lane; i <= N; i += kWarp) s_off[i] = a.topo.off[i];
    for (int e = lane; e < E; e += kWarp) s_src[e] = a.topo.src[e];
    for (int s = lane; s < S; s += kWarp) { meta[s].set = -1; meta[s].next_ic = 0; meta[s].active = 0; }
    __syncwarp();

    auto V = [&](int b, int i) -> Real & {
        if (!GRINS_OK_IDX(b >= 0 && b < 9 && i >= 0 && i < N, 11, b * 1000 + i)) b = i = 0;
        return vec[(b * N + i) * kWarp + lane];
    };

    const Real rtol = (Real)a.rtol, atol = (Real)a.atol;
    const Real ss_tol = (Real)a.ss_tol;
    const Real t_end = (Real)a.t_end;
    const Real invN = (Real)1 / (Real)N;

    int my_slot = -1, my_ic = 0;
    long long my_set = 0;
    Real t = 0, h = 0;
    int steps = 0, gidx = 0, yb = 0, kb1 = 2;
    bool need_k1 = false, rejected = false, exhausted = false;
    bool near = false;                 // residual below ss_near: tolerances tightened

    auto slot_ptr = [&](int s) -> unsigned char * {
        if (!GRINS_OK_IDX(s >= 0 && s < S, 13, s)) s = 0;
        return slot_base + s * slot_bytes;
    };

    // f(stage input in vector zb) -> vector out
    auto rhs = [&](int zb, int out, const unsigned char *sp) {
        const Real *G = reinterpret_cast<const Real *>(sp);
        const Real *kd = G + N;
        const Edge *ed = reinterpret_cast<const Edge *>(sp + LY.node_bytes());
        __syncwarp();
        for (int i = 0; i < N; ++i) {
            Real prod = 1, num = 1, den = 1;
            const int beg = s_off[i], end = s_off[i + 1];
            int cnt = 0;
            for (int e = beg; e < end; ++e) {
                GRINS_OK_IDX(e >= 0 && e < E && s_src[e] >= 0 && s_src[e] < N, 12, e);
                P::edge(ed[e], V(8, s_src[e]), num, den);
                if (++cnt == 4) { prod *= P::ratio(num, den); num = 1; den = 1; cnt = 0; }
            }
            prod *= P::ratio(num, den);
            V(out, i) = G[i] * prod - kd[i] * V(zb, i);
        }
        __syncwarp();
    };

    auto stage_slot = [&](int s, long long set) {
        unsigned char *sp = slot_ptr(s);
        Real *G = reinterpret_cast<Real *>(sp);
        Real *kd = G + N;
        Real *kG = G + 2 * N;
        Edge *ed = reinterpret_cast<Edge *>(sp + LY.node_bytes());
        const unsigned char *blk = a.params + set * a.L.stride;
        const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *Td = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nd = blk + a.L.off_n;
        for (int i = lane; i < N; i += kWarp) {
            const double g = Gd[i], k = kdd[i];
            G[i] = (Real)g; kd[i] = (Real)k; kG[i] = (Real)(k / g);
        }
        for (int e = lane; e < E; e += kWarp) {
            const int ue = a.topo.edge[e];
            ed[e] = P::make_edge(Td[ue], ld[ue], (int)nd[ue], (int)a.topo.sign[e]);
        }
        __syncwarp();
    };

    auto write_series = [&](int g) {
        double *dst = a.series + (((long long)my_set * a.n_ics + my_ic) * a.n_t + g) * N;
        for (int i = 0; i < N; ++i) dst[i] = (double)V(yb, i);
    };

    auto refill = [&]() {
        if (a.cancel != nullptr && !exhausted && grins_cancelled(a.cancel)) {
            // cancelled: the initial conditions still pending in this warp's
            // slots and every set left in the counter are marked, not started
            for (int sl = 0; sl < S; ++sl) {
                const long long set = meta[sl].set;
                const int first = meta[sl].next_ic;
                if (set >= 0 && first < a.n_ics)
                    for (int ic = first + lane; ic < a.n_ics; ic += 32) a.status[set * a.n_ics + ic] = GRINS_SS_CANCELLED;
                __syncwarp();
                if (lane == 0 && set >= 0 && first < a.n_ics) meta[sl].next_ic = a.n_ics;
                __syncwarp();
            }
            grins_cancel_sets(a.queue, a.n_sets, a.n_ics, a.status);
            exhausted = true;
            return;
        }
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
                    yb = 0; kb1 = 2;
                    for (int i = 0; i < N; ++i) V(yb, i) = (Real)((u[i] * Gd[i]) / kdd[i]);
                    t = (Real)a.t0;
                    steps = 0; gidx = 0;
                    need_k1 = true; rejected = false; near = false;
                    if (a.n_t > 0) {
                        while (gidx < a.n_t && a.t_grid[gidx] <= a.t0) { write_series(gidx); ++gidx; }
                    }
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

    auto residual = [&](int kb, const unsigned char *sp) -> Real {
        const Real *kG = reinterpret_cast<const Real *>(sp) + 2 * N;
        Real r = 0;
        for (int i = 0; i < N; ++i) r = fmax(r, fabs(V(kb, i)) * kG[i]);
        return r;
    };

    refill();

    for (;;) {
        const bool working = my_slot >= 0;
        if (!__any_sync(FULL, working)) break;
        const unsigned char *sp = slot_ptr(working ? my_slot : 0);
        bool done = false;
        uint8_t st_code = GRINS_SS_TEND;
        const int zb = yb ^ 1;

        if (__any_sync(FULL, need_k1)) {
            for (int i = 0; i < N; ++i) { const Real yi = V(yb, i); V(zb, i) = yi; V(8, i) = P::scratch(yi); }
            const int out = need_k1 ? kb1 : 5 - kb1;
            rhs(zb, out, sp);
            if (need_k1) {
                need_k1 = false;
                Real d0 = 0, d1 = 0;
                bool fin = true;
                for (int i = 0; i < N; ++i) {
                    const Real yi = V(yb, i), fi = V(kb1, i);
                    fin = fin && isfinite(fi);
                    const Real sc = atol + rtol * fabs(yi);
                    d0 += (yi / sc) * (yi / sc);
                    d1 += (fi / sc) * (fi / sc);
                }
                d0 = sqrt(d0 * invN);
                d1 = sqrt(d1 * invN);
                h = (d0 < (Real)1e-5 || d1 < (Real)1e-5) ? (Real)1e-6 : (Real)0.01 * d0 / d1;
                h = fmin(h, (Real)(a.t_end - a.t0));
                if (!fin) { done = true; st_code = GRINS_SS_NONFINITE; }
                else if (residual(kb1, sp) < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
            }
        }

        // Every lane runs the stages (idle and finished lanes on scratch
        // values); only working lanes act on the result.
        Real t_stop = t_end;
        bool to_grid = false;
        if (a.n_t > 0 && gidx < a.n_t && (Real)a.t_grid[gidx] < t_stop) { t_stop = (Real)a.t_grid[gidx]; to_grid = true; }
        Real hh = h;
        bool clipped = false;
        if (t + hh >= t_stop) { hh = t_stop - t; clipped = true; }
        const int kb2 = 5 - kb1;
#pragma unroll 1
        for (int s = 1; s <= 6; ++s) {
            for (int i = 0; i < N; ++i) {
                Real acc = tab.a[s][0] * V(kb1, i);
                if (s > 1 && s < 6) acc += tab.a[s][1] * V(kb2, i);
                for (int j = 2; j < s; ++j) acc += tab.a[s][j] * V(2 + j, i);
                const Real z = V(yb, i) + hh * acc;
                V(zb, i) = z;
                V(8, i) = P::scratch(z);
            }
            rhs(zb, s == 1 || s == 6 ? kb2 : 2 + s, sp);
        }
        if (working && !done) {
            Real en = 0;
            bool finite = true;
            for (int i = 0; i < N; ++i) {
                const Real k7 = V(kb2, i), z = V(zb, i);
                const Real err = hh * (tab.e[0] * V(kb1, i) + tab.e[2] * V(4, i) + tab.e[3] * V(5, i) +
                                       tab.e[4] * V(6, i) + tab.e[5] * V(7, i) + tab.e[6] * k7);
                const Real sc = atol + rtol * fmax(fabs(V(yb, i)), fabs(z));
                const Real q = err / sc;
                en += q * q;
                finite = finite && isfinite(z) && isfinite(k7);
            }
            en *= invN;
            if (near) en *= (Real)a.ss_gain;
            ++steps;
            if (!finite || !isfinite(en)) {
                done = true; st_code = GRINS_SS_NONFINITE;
            } else if (en < (Real)1) {
                const Real t_new = clipped ? t_stop : t + hh;
                if (!(t_new > t)) { done = true; st_code = GRINS_SS_NONFINITE; }
                t = t_new;
                yb ^= 1;
                kb1 = kb2;
                if (clipped && to_grid) {
                    while (gidx < a.n_t && (Real)a.t_grid[gidx] <= t) { write_series(gidx); ++gidx; }
                }
                Real fac = en == (Real)0 ? (Real)10 : (Real)0.9 * pow(en, (Real)-0.1);
                fac = fmin(fac, (Real)10);
                if (rejected) fac = fmin(fac, (Real)1);
                h = hh * fac;
                rejected = false;
                if (!done) {
                    const Real res = residual(kb1, sp);
                    near = res < (Real)a.ss_near;
                    if (res < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                    else if (t >= t_end) { done = true; st_code = GRINS_SS_TEND; }
                }
            } else {
                h = hh * fmax((Real)0.9 * pow(en, (Real)-0.1), (Real)0.2);
                rejected = true;
            }
            if (!done && steps >= a.max_steps) { done = true; st_code = GRINS_SS_MAXSTEPS; }
        }

        if (__any_sync(FULL, done)) {
            if (done) {
                long long idx = my_set * a.n_ics + my_ic;
                if (!GRINS_OK_IDX(idx >= 0 && idx < a.n_sets * a.n_ics, 14, idx)) idx = 0;
                double *dst = a.states + idx * N;
                for (int i = 0; i < N; ++i) dst[i] = (double)V(yb, i);
                a.status[idx] = st_code;
                if (a.t_final) a.t_final[idx] = (double)t;
                if (a.n_steps) a.n_steps[idx] = steps;
                if (a.n_t > 0) { while (gidx < a.n_t) { write_series(gidx); ++gidx; } }
                atomicSub(&meta[my_slot].active, 1);
                my_slot = -1;
            }
            __syncwarp();
            refill();
        }
    }
}

template <typename Real>
cudaError_t launch_dp5_generic(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    IntegrateArgs b = a;
    GenericLayout LY{b.topo.N, b.topo.E, b.slots, (int)sizeof(Real)};
    while (LY.total() > b.smem_limit && LY.S > 1) LY.S = --b.slots;
    const int smem = LY.total();
    if (smem > b.smem_limit) return cudaErrorInvalidConfiguration;
    auto kern = dp5_generic_kernel<Real>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarp, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long need = (b.n_sets * b.n_ics + 31) / 32 + 1;
    long long blocks = (long long)num_sms * per_sm;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, kWarp, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace grins

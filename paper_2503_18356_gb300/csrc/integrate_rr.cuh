// Lane-group FP32 Dormand-Prince 5(4) integrator with the parameter records
// in registers, compiled at run time for one network's row layout.
//
// Model, lane mapping, gather buffer and step control are those of the
// shared-memory-record kernel (integrate_grp.cuh; GRiNS Sec. 2.1.1, Eq. 1
// and Eq. 2 written as products of w (p + u) / (1 + p), p = 2^t,
// t = n log2 x_src - n log2 T).  What differs:
//   * a lane keeps the records of its own edge positions in registers --
//     n, -n log2 T and 1/lambda as FP32 pairs, and the shared-memory address
//     of each position's source entry -- together with G', k and k/G of its
//     rows, loaded when it starts a solve.  The edge loop then issues one
//     shared load per edge (the source value) where the shared-record kernel
//     issues two, one of them 16 bytes wide;
//   * edges are taken two at a time with the packed FP32 pair instructions
//     (fma/add/mul .f32x2 of sm_100 and later), each pair component carrying
//     at most four factors (p <= 2^30) before its division;
//   * work is handed out one solve at a time from a set-major counter, so
//     no parameter-set slots are needed.
// The rows (GrpRowCt<r>: position offset and degree; kGrpCtRows) are
// compile-time constants generated for the network, and the stages of an
// attempt are written out, so every register array is indexed by constants
// and the gather buffer of each right-hand side is an immediate offset.
//
// FP64 instantiation (the plain FP64 GPU solver): the same body with double
// states and records; its edge term is exact rather than log-domain -- the
// gather buffer holds x, x^2 .. x^6 of every stage value and an edge forms
// p = x^n (1/T)^n with one multiply (n <= 6, Table 1; an edge with a larger
// n makes its solve non-finite), numerators and denominators divided once
// per eight factors.
#pragma once

#include "integrate_grp.cuh"

namespace grins {

// Pair offset of row r: rows before it take ceil(deg / 2) pairs each.
template <int r> struct RrQ {
    static constexpr int off = RrQ<r - 1>::off + (GrpRowCt<r - 1>::deg + 1) / 2;
};
template <> struct RrQ<0> { static constexpr int off = 0; };

constexpr int kRrP = GrpRowCt<kGrpCtRows - 1>::off + GrpRowCt<kGrpCtRows - 1>::deg;   // positions per lane
constexpr int kRrQ = RrQ<kGrpCtRows>::off;                                              // pairs per lane
constexpr int kRrPa = kRrP > 0 ? kRrP : 1;
constexpr int kRrQa = kRrQ > 0 ? kRrQ : 1;

__device__ __forceinline__ unsigned rr_smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Gather-buffer accesses and the warp barrier as ordered inline PTX: the
// buffer offset of a right-hand side is an immediate.
template <int OFF>
__device__ __forceinline__ float rr_lds(unsigned addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
    return v;
}

template <int OFF>
__device__ __forceinline__ void rr_sts(unsigned addr, float v)
{
    asm volatile("st.shared.f32 [%0+%1], %2;" ::"r"(addr), "n"(OFF), "f"(v) : "memory");
}

__device__ __forceinline__ void rr_syncwarp()
{
    asm volatile("bar.warp.sync %0;" ::"r"(0xffffffffu) : "memory");
}

template <int NPL>
struct RrRecs {
    unsigned ga[kRrPa];                    // shared address of each position's source entry (buffer 0)
    float2 n[kRrQa], c[kRrQa], u[kRrQa];   // n, -n log2 T, 1/lambda, two positions per pair
    float Gp[NPL], k[NPL], kg[NPL];        // G' = G prod_inh lambda, k, k/G of this lane's rows
};

// A chunk of five or six factors shares one division: the y component of
// its first pair carries an extra factor 2^-60 in numerator and denominator
// alike (its record holds -n log2 T - 60 and 2^-60 / lambda), which keeps
// both products of six factors of at most 2^30 + 1 within FP32 range.
template <int r>
__device__ constexpr bool rr_scaled_pair(int i)
{
    constexpr int D = GrpRowCt<r>::deg, NP = D / 2;
    constexpr bool TAIL = (D & 1) != 0;
    if (i % 4 != 0 || i >= NP) return false;
    const int np = NP - i < 4 ? NP - i : 4;
    const bool tail = TAIL && i + np >= NP && np < 4;
    const int f = 2 * np + (tail ? 1 : 0);
    return f >= 5 && f <= 6;
}

// Positions P, P+1 (record pair Q) into (num, den); FIRST starts the chunk,
// SC: its y component is scaled by 2^-60 (rr_scaled_pair).
template <int BO, int P, int Q, bool FIRST, bool SC, int NPL>
__device__ __forceinline__ void rr_pair(const RrRecs<NPL> &q, float2 &num, float2 &den)
{
    const float2 s = make_float2(rr_lds<BO>(q.ga[P]), rr_lds<BO>(q.ga[P + 1]));
    const float2 t = __ffma2_rn(q.n[Q], s, q.c[Q]);
    const float2 pw = make_float2(ex2_approx(fminf(t.x, 30.0f)), ex2_approx(fminf(t.y, SC ? -30.0f : 30.0f)));
    const float2 a = __fadd2_rn(pw, q.u[Q]);
    if constexpr (FIRST) {
        num = a;
        den = __fadd2_rn(pw, make_float2(1.0f, SC ? 0x1p-60f : 1.0f));
    } else {
        num = __fmul2_rn(num, a);
        den = __ffma2_rn(den, pw, den);
    }
}

// Position P alone (component x of record pair Q).
template <int BO, int P, int Q, bool FIRST, int NPL>
__device__ __forceinline__ void rr_single(const RrRecs<NPL> &q, float &num, float &den)
{
    const float s = rr_lds<BO>(q.ga[P]);
    const float pw = ex2_approx(fminf(fmaf(q.n[Q].x, s, q.c[Q].x), 30.0f));
    if constexpr (FIRST) {
        num = pw + q.u[Q].x;
        den = pw + 1.0f;
    } else {
        num *= pw + q.u[Q].x;
        den = fmaf(den, pw, den);
    }
}

template <int BO, int P0, int Q0, int I, int NP, bool SC, int NPL>
__device__ __forceinline__ void rr_pairs(const RrRecs<NPL> &q, float2 &num, float2 &den)
{
    if constexpr (I < NP) {
        rr_pair<BO, P0 + 2 * I, Q0 + I, I == 0, SC && I == 0, NPL>(q, num, den);
        rr_pairs<BO, P0, Q0, I + 1, NP, SC, NPL>(q, num, den);
    }
}

// NP (1..4) pairs from position P0 / pair Q0, plus the row's last (odd)
// position when TAIL: the product of their factors.  Up to four factors in
// all share one division; more keep the two components apart (each holds at
// most four) and divide each.
template <int BO, int P0, int Q0, int NP, bool TAIL, int NPL>
__device__ __forceinline__ float rr_chunk(const RrRecs<NPL> &q)
{
    float2 num, den;
    constexpr int F = 2 * NP + (TAIL ? 1 : 0);
    rr_pairs<BO, P0, Q0, 0, NP, F >= 5 && F <= 6, NPL>(q, num, den);
    if constexpr (TAIL) rr_single<BO, P0 + 2 * NP, Q0 + NP, false, NPL>(q, num.x, den.x);
    if constexpr (F <= 6)
        return div_approx(num.x * num.y, den.x * den.y);
    else
        return div_approx(num.x, den.x) * div_approx(num.y, den.y);
}

// Product over a row of NP pairs (+ TAIL) in chunks of four pairs; the odd
// position joins the last chunk when it has room, else forms its own.
template <int BO, int P0, int Q0, int NP, bool TAIL, int C, int NPL>
__device__ __forceinline__ float rr_row_prod(const RrRecs<NPL> &q)
{
    constexpr int first = 4 * C;
    if constexpr (first >= NP) {
        if constexpr (TAIL && NP % 4 == 0) {
            float num, den;
            rr_single<BO, P0 + 2 * NP, Q0 + NP, true, NPL>(q, num, den);
            return div_approx(num, den);
        } else {
            return 1.0f;
        }
    } else {
        constexpr int np = NP - first < 4 ? NP - first : 4;
        constexpr bool tail_here = TAIL && first + np >= NP && np < 4;
        const float f = rr_chunk<BO, P0 + 2 * first, Q0 + first, np, tail_here, NPL>(q);
        if constexpr (first + 4 >= NP && !(TAIL && NP % 4 == 0))
            return f;
        else
            return f * rr_row_prod<BO, P0, Q0, NP, TAIL, C + 1, NPL>(q);
    }
}

__device__ __forceinline__ float rr_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rr_fma(double a, double b, double c) { return fma(a, b, c); }

// prod[r] <- the product of row r's factors, rows r, r+1, ...
template <int BO, int r, int NPL>
__device__ __forceinline__ void rr_prods(const RrRecs<NPL> &q, float (&prod)[NPL])
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int D = GrpRowCt<r>::deg;
        prod[r] = rr_row_prod<BO, GrpRowCt<r>::off, RrQ<r>::off, D / 2, (D & 1) != 0, 0, NPL>(q);
        rr_prods<BO, r + 1, NPL>(q, prod);
    }
}

// Continuations: a lane whose slot in row r continues its slot in row
// GrpRowCt<r>::link (lk[r]) multiplies its row-r partial product into it.
template <int r, int NPL, typename Real>
__device__ __forceinline__ void rr_links(const bool (&lk)[NPL], Real (&prod)[NPL])
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int t = GrpRowCt<r>::link;
        if constexpr (t >= 0 && t < NPL) prod[t] *= lk[r] ? prod[r] : (Real)1;
        rr_links<r + 1, NPL, Real>(lk, prod);
    }
}

// z[r] <- G'_r prod_r - k_r z[r]
template <int NPL, typename Recs, typename Real>
__device__ __forceinline__ void rr_update(const Recs &q, const Real (&prod)[NPL], Real (&z)[NPL])
{
#pragma unroll
    for (int r = 0; r < NPL; ++r) z[r] = rr_fma(q.Gp[r], prod[r], -q.k[r] * z[r]);
}

// log2 of this lane's stage values into its column of the buffer at BO.
// The log-domain edge term reads a stage value through |z| (an operand
// modifier of the log2, no instruction) where Eq. 2 reads a negative value
// as 0: a small overshoot -delta << T below zero gives the same factor to
// within (delta / T)^n, and the exact solution never goes below zero, so
// only a stage far off the trajectory -- an inaccurate attempt -- sees a
// difference.
template <int BO, int r, int NPL>
__device__ __forceinline__ void rr_put(const float (&z)[NPL], unsigned own)
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        rr_sts<BO + r * kWarp * 4>(own, lg2_approx(fabsf(z[r])));
        rr_put<BO, r + 1, NPL>(z, own);
    }
}

// z <- Eq. 1 at the stage input z through gather buffer B (0 or 1)
template <int B, int NPL>
__device__ __forceinline__ void rr_rhs(const RrRecs<NPL> &q, const bool (&lk)[NPL], float (&z)[NPL], unsigned own)
{
    constexpr int BO = B * NPL * kWarp * 4;
    rr_put<BO, 0, NPL>(z, own);
    rr_syncwarp();
    float prod[NPL];
    rr_prods<BO, 0, NPL>(q, prod);
    rr_links<0, NPL, float>(lk, prod);
    rr_update<NPL>(q, prod, z);
}

// ------------------------------------------------------------------ FP64
constexpr int kRr64Pow = 6;                   // planes x .. x^6 of the FP64 gather buffer

template <int OFF>
__device__ __forceinline__ double rr_lds64(unsigned addr)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(addr), "n"(OFF));
    return v;
}

template <int OFF>
__device__ __forceinline__ void rr_sts64(unsigned addr, double v)
{
    asm volatile("st.shared.f64 [%0+%1], %2;" ::"r"(addr), "n"(OFF), "d"(v) : "memory");
}

template <int NPL>
struct RrRecs64 {
    unsigned ga[kRrPa];                 // shared address of each position's x^n entry (buffer 0)
    double itn[kRrPa], u[kRrPa];        // (1/T)^n, 1/lambda (neutral: 0, 1)
    double Gp[NPL], k[NPL], kg[NPL];
};

// Product of the D factors of a row from position P0, one division per
// eight factors (p <= 2^120, so eight stay finite).
template <int BO, int P0, int D, int I, int NPL>
__device__ __forceinline__ void rr64_acc(const RrRecs64<NPL> &q, double &prod, double &num, double &den)
{
    if constexpr (I < D) {
        const double p = fmin(rr_lds64<BO>(q.ga[P0 + I]) * q.itn[P0 + I], 0x1.0p120);
        num *= p + q.u[P0 + I];
        den = fma(den, p, den);
        if constexpr (I % 8 == 7) { prod *= num / den; num = 1.0; den = 1.0; }
        rr64_acc<BO, P0, D, I + 1, NPL>(q, prod, num, den);
    }
}

template <int BO, int r, int NPL>
__device__ __forceinline__ void rr64_prods(const RrRecs64<NPL> &q, double (&prod)[NPL])
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int D = GrpRowCt<r>::deg;
        double p = 1.0, num = 1.0, den = 1.0;
        rr64_acc<BO, GrpRowCt<r>::off, D, 0, NPL>(q, p, num, den);
        if constexpr (D % 8 != 0) p *= num / den;
        prod[r] = p;
        rr64_prods<BO, r + 1, NPL>(q, prod);
    }
}

// x .. x^6 of this lane's stage values (x clamped to [0, 1e6]) into plane q
// of its column of the buffer at BO
template <int BO, int r, int NPL>
__device__ __forceinline__ void rr64_put(const double (&z)[NPL], unsigned own)
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int PL = NPL * kWarp * 8, RO = r * kWarp * 8;
        const double x = fmin(fmax(z[r], 0.0), 1e6);
        const double x2 = x * x, x4 = x2 * x2;
        rr_sts64<BO + RO>(own, x);
        rr_sts64<BO + PL + RO>(own, x2);
        rr_sts64<BO + 2 * PL + RO>(own, x2 * x);
        rr_sts64<BO + 3 * PL + RO>(own, x4);
        rr_sts64<BO + 4 * PL + RO>(own, x4 * x);
        rr_sts64<BO + 5 * PL + RO>(own, x2 * x4);
        rr64_put<BO, r + 1, NPL>(z, own);
    }
}

template <int B, int NPL>
__device__ __forceinline__ void rr_rhs(const RrRecs64<NPL> &q, const bool (&lk)[NPL], double (&z)[NPL], unsigned own)
{
    constexpr int BO = B * kRr64Pow * NPL * kWarp * 8;
    rr64_put<BO, 0, NPL>(z, own);
    rr_syncwarp();
    double prod[NPL];
    rr64_prods<BO, 0, NPL>(q, prod);
    rr_links<0, NPL, double>(lk, prod);
    rr_update<NPL>(q, prod, z);
}

// FP64 records of row r from parameter block blk; col = this group's column
// address of plane 0 in buffer 0.
template <int r, int NPL, int L>
__device__ __forceinline__ void rr_load_rows(RrRecs64<NPL> &q, const IntegrateArgs &a, const unsigned char *blk,
                                             int j, unsigned col)
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int D = GrpRowCt<r>::deg, P0 = GrpRowCt<r>::off;
        const double *Td = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nn = blk + a.L.off_n;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int e = a.grp.pos_edge[(P0 + d) * L + j];
            double itn = 0.0, u = 1.0;
            int plane = 0;
            if (e >= 0) {
                const int ne = nn[e];
                const double it = 1.0 / Td[e];
                double pn = it;
#pragma unroll 1
                for (int m = 1; m < ne; ++m) pn *= it;
                const bool ok = ne >= 1 && ne <= kRr64Pow;
                itn = ok ? fmin(pn, 1e30) : __longlong_as_double(0x7ff8000000000000ll);
                plane = ok ? ne - 1 : 0;
                u = 1.0 / ld[e];
            }
            q.itn[P0 + d] = itn;
            q.u[P0 + d] = u;
            q.ga[P0 + d] = col + 2 * a.grp.pos_off[(P0 + d) * L + j] + plane * (NPL * kWarp * 8);
        }
        rr_load_rows<r + 1, NPL, L>(q, a, blk, j, col);
    }
}

// ------------------------------------------------------------ by precision
template <typename Real, int NPL> struct RrSel { using Recs = RrRecs<NPL>; static constexpr int planes = 1; };
template <int NPL> struct RrSel<double, NPL> { using Recs = RrRecs64<NPL>; static constexpr int planes = kRr64Pow; };

__device__ __forceinline__ float rr_div(float a, float b) { return div_approx(a, b); }
__device__ __forceinline__ double rr_div(double a, double b) { return a / b; }
__device__ __forceinline__ float rr_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double rr_abs(double a) { return fabs(a); }
__device__ __forceinline__ float rr_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rr_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rr_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double rr_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float rr_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double rr_sqrt(double a) { return sqrt(a); }

// A tolerance argument in the kernel's precision (FP32 kernels read the
// launcher's FP32 copy).
template <typename Real>
__device__ __forceinline__ Real rr_argr(double d, float f)
{
    if constexpr (sizeof(Real) == 4) return f;
    else return d;
}

template <typename Real>
__device__ __forceinline__ Real rr_gsum(Real v, int L)
{
    for (int o = kWarp / L; o < kWarp; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename Real>
__device__ __forceinline__ Real rr_gmax(Real v, int L)
{
    for (int o = kWarp / L; o < kWarp; o <<= 1) v = rr_max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Records of row r (positions d = 0 .. deg-1) from parameter block blk.
template <int r, int NPL, int L>
__device__ __forceinline__ void rr_load_rows(RrRecs<NPL> &q, const IntegrateArgs &a, const unsigned char *blk, int j,
                                             unsigned)
{
    if constexpr (r < kGrpCtRows && r < NPL) {
        constexpr int D = GrpRowCt<r>::deg, P0 = GrpRowCt<r>::off, Q0 = RrQ<r>::off;
        const double *Td = reinterpret_cast<const double *>(blk + a.L.off_T);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const uint8_t *nn = blk + a.L.off_n;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int e = a.grp.pos_edge[(P0 + d) * L + j];
            float n = 1.0f, c = -100.0f, u = 1.0f;     // neutral: (p + 1) / (1 + p) = 1
            if (e >= 0) {
                n = (float)nn[e];
                c = -n * log2f((float)Td[e]);
                u = __frcp_rn((float)ld[e]);
            }
            if ((d & 1) && rr_scaled_pair<r>(d / 2)) { c -= 60.0f; u *= 0x1p-60f; }
            if (d & 1) { q.n[Q0 + d / 2].y = n; q.c[Q0 + d / 2].y = c; q.u[Q0 + d / 2].y = u; }
            else       { q.n[Q0 + d / 2].x = n; q.c[Q0 + d / 2].x = c; q.u[Q0 + d / 2].x = u; }
        }
        rr_load_rows<r + 1, NPL, L>(q, a, blk, j, 0u);
    }
}

// Stage combinations out[r] = (ADD_Y ? y[r] : 0) + hh (c1 k1[r] + c2 k2[r]
// + ...), the sum taken left to right.  FP32 rows go two at a time through
// the packed pair instructions (each component rounds as the scalar
// operation would); an odd last row and FP64 rows go one at a time.
template <int NPL>
__device__ __forceinline__ void rr_acc2(float2 &s, int r, float c, const float (&k)[NPL])
{
    s = __ffma2_rn(make_float2(c, c), make_float2(k[r], k[r + 1]), s);
}
template <int NPL, typename... Ts>
__device__ __forceinline__ void rr_acc2(float2 &s, int r, float c, const float (&k)[NPL], const Ts &...ts)
{
    rr_acc2<NPL>(s, r, c, k);
    rr_acc2<NPL>(s, r, ts...);
}
template <int NPL, typename Real>
__device__ __forceinline__ void rr_acc1(Real &s, int r, Real c, const Real (&k)[NPL])
{
    s = rr_fma(c, k[r], s);
}
template <int NPL, typename Real, typename... Ts>
__device__ __forceinline__ void rr_acc1(Real &s, int r, Real c, const Real (&k)[NPL], const Ts &...ts)
{
    rr_acc1<NPL, Real>(s, r, c, k);
    rr_acc1<NPL, Real>(s, r, ts...);
}

template <bool ADD_Y, int NPL, typename... Ts>
__device__ __forceinline__ void rr_comb(float (&out)[NPL], const float (&y)[NPL], float hh, float c,
                                        const float (&k)[NPL], const Ts &...ts)
{
#pragma unroll
    for (int r = 0; r + 1 < NPL; r += 2) {
        float2 s = __fmul2_rn(make_float2(c, c), make_float2(k[r], k[r + 1]));
        if constexpr (sizeof...(Ts) > 0) rr_acc2<NPL>(s, r, ts...);
        const float2 o = ADD_Y ? __ffma2_rn(make_float2(hh, hh), s, make_float2(y[r], y[r + 1]))
                               : __fmul2_rn(make_float2(hh, hh), s);
        out[r] = o.x;
        out[r + 1] = o.y;
    }
    if constexpr (NPL % 2 == 1) {
        constexpr int r = NPL - 1;
        float s = c * k[r];
        if constexpr (sizeof...(Ts) > 0) rr_acc1<NPL, float>(s, r, ts...);
        out[r] = ADD_Y ? fmaf(hh, s, y[r]) : hh * s;
    }
}

template <bool ADD_Y, int NPL, typename... Ts>
__device__ __forceinline__ void rr_comb(double (&out)[NPL], const double (&y)[NPL], double hh, double c,
                                        const double (&k)[NPL], const Ts &...ts)
{
#pragma unroll
    for (int r = 0; r < NPL; ++r) {
        double s = c * k[r];
        if constexpr (sizeof...(Ts) > 0) rr_acc1<NPL, double>(s, r, ts...);
        out[r] = ADD_Y ? fma(hh, s, y[r]) : hh * s;
    }
}

// The 5(4) pair of the integrator: M = 0 Dormand-Prince (b2 = e2 = 0),
// M = 1 Tsitouras (the paper's Tsit5).
template <int M> struct RrTab;
template <> struct RrTab<0> {
    static constexpr double a21 = dp::a21, a31 = dp::a31, a32 = dp::a32, a41 = dp::a41, a42 = dp::a42,
                            a43 = dp::a43, a51 = dp::a51, a52 = dp::a52, a53 = dp::a53, a54 = dp::a54,
                            a61 = dp::a61, a62 = dp::a62, a63 = dp::a63, a64 = dp::a64, a65 = dp::a65;
    static constexpr double b1 = dp::b1, b2 = 0.0, b3 = dp::b3, b4 = dp::b4, b5 = dp::b5, b6 = dp::b6;
    static constexpr double e1 = dp::e1, e2 = 0.0, e3 = dp::e3, e4 = dp::e4, e5 = dp::e5, e6 = dp::e6,
                            e7 = dp::e7;
};
template <> struct RrTab<1> {
    static constexpr double a21 = ts::a21, a31 = ts::a31, a32 = ts::a32, a41 = ts::a41, a42 = ts::a42,
                            a43 = ts::a43, a51 = ts::a51, a52 = ts::a52, a53 = ts::a53, a54 = ts::a54,
                            a61 = ts::a61, a62 = ts::a62, a63 = ts::a63, a64 = ts::a64, a65 = ts::a65;
    static constexpr double b1 = ts::b1, b2 = ts::b2, b3 = ts::b3, b4 = ts::b4, b5 = ts::b5, b6 = ts::b6;
    static constexpr double e1 = ts::e1, e2 = ts::e2, e3 = ts::e3, e4 = ts::e4, e5 = ts::e5, e6 = ts::e6,
                            e7 = ts::e7;
};

// Body of the register-record kernel: NPL rows, WARPS warps per block, L
// lanes per solve, Real = float (log-domain edge terms) or double (power
// table), M the 5(4) pair (RrTab).
template <int NPL, int WARPS, int L, typename Real = float, int M = 0>
__device__ __forceinline__ void rr_body(const IntegrateArgs &a)
{
    using T = RrTab<M>;
    constexpr bool F64 = sizeof(Real) == 8;
    constexpr int EL = (int)sizeof(Real);                 // bytes per gather entry
    constexpr int PLN = RrSel<Real, NPL>::planes;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int GS = kWarp / L;                // groups per warp
    unsigned long long *grins_chk = a.check;
    (void)grins_chk;
    const int N = a.topo.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = lane / GS, g = lane - j * GS;  // lane within group, group (j-major)

    float *gbuf = reinterpret_cast<float *>(smem) + warp * (2 * PLN * NPL * kWarp * EL / 4);
    const unsigned base = rr_smem_addr(gbuf);
    const unsigned own = base + EL * lane;
#pragma unroll 1
    for (int i = lane; i < 2 * PLN * NPL * kWarp * EL / 4; i += kWarp) gbuf[i] = 0.0f;

    typename RrSel<Real, NPL>::Recs q;
#pragma unroll
    for (int p = 0; p < kRrPa; ++p) {
        int off = p < kRrP ? a.grp.pos_off[p * L + j] : 0;
        if (!GRINS_OK_IDX(off >= 0 && off < NPL * kWarp * 4 && (off & 3) == 0, 33, off)) off = 0;
        q.ga[p] = base + (EL / 4) * off + EL * g;
    }
    if constexpr (F64) {
#pragma unroll
        for (int p = 0; p < kRrPa; ++p) { q.itn[p] = 0.0; q.u[p] = 1.0; }
    } else {
#pragma unroll
        for (int i = 0; i < kRrQa; ++i) {
            q.n[i] = make_float2(1.0f, 1.0f);
            q.c[i] = make_float2(-100.0f, -100.0f);
            q.u[i] = make_float2(1.0f, 1.0f);
        }
    }
#pragma unroll
    bool lk[NPL];                     // continuation flags of this lane's slots
#pragma unroll
    for (int r = 0; r < NPL; ++r) lk[r] = a.grp.row_link != nullptr && a.grp.row_link[r * L + j] != 0;
    for (int r = 0; r < NPL; ++r) { q.Gp[r] = 0; q.k[r] = 1; q.kg[r] = 0; }
    rr_syncwarp();

    const Real rtol = rr_argr<Real>(a.rtol, a.f_rtol), atol = rr_argr<Real>(a.atol, a.f_atol);
    const Real ss_tol = rr_argr<Real>(a.ss_tol, a.f_ss_tol);
    const Real t_end = rr_argr<Real>(a.t_end, a.f_t_end);
    const Real invN = (Real)1 / (Real)N;
    // FP64 list mode: the solves to integrate are the borderline ones the
    // FP32 pass listed, each from its checkpoint (state in `states`, time in
    // the list); FP32 tail mode: keep checkpoints and list borderline solves
    const bool from_list = F64 && a.tail_items != nullptr;
    const bool tail_on = !F64 && a.tail_items != nullptr;
    const long long n_solves = a.n_sets * (long long)a.n_ics;
    const unsigned long long listed = from_list ? *a.tail_n : 0ull;
    const long long total = from_list ? (listed < (unsigned long long)n_solves ? (long long)listed : n_solves) : n_solves;
    const float tail_chk = tail_on ? a.f_tail_chk : -1.0f;
    bool has_chk = false;            // this solve's checkpoint is written
    Real t_c = 0;                    // and its time
    int steps_c = 0;                 // and the attempts before it

    long long my_set = 0;
    int my_ic = 0;
    bool working = false, exhausted = false;
    Real t = 0, h = 0;
    int steps = 0, gidx = 0;
    bool near = false;               // residual below ss_near: tolerances tightened
    const Real ss_near = rr_argr<Real>(a.ss_near, a.f_ss_near), ss_gain = rr_argr<Real>(a.ss_gain, a.f_ss_gain);
    bool need_k1 = false, rejected = false;
    Real y[NPL], k1[NPL], k2[NPL], k3[NPL], k4[NPL], k5[NPL], k6[NPL], z[NPL];
#pragma unroll
    for (int r = 0; r < NPL; ++r) y[r] = k1[r] = k2[r] = k3[r] = k4[r] = k5[r] = k6[r] = z[r] = 0;

    auto write_series = [&](int gi) {
        double *dst = a.series + ((my_set * a.n_ics + my_ic) * (long long)a.n_t + gi) * N;
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            const int node = a.grp.row_node[r * L + j];
            if (node >= 0) dst[node] = (double)y[r];
        }
    };

    // item it = set * n_ics + ic -> this lane's records, rows and state
    auto start = [&](long long it) {
        if (!GRINS_OK_IDX(it >= 0 && it < total, 35, it)) it = 0;
        Real t_start = (Real)a.t0;
        if (from_list) {
            const typename IntegrateArgs::TailItem ti = a.tail_items[it];
            it = ti.idx;
            if (!GRINS_OK_IDX(it >= 0 && it < n_solves, 36, it)) it = 0;
            t_start = (Real)ti.t;
        }
        my_set = it / a.n_ics;
        my_ic = (int)(it - my_set * a.n_ics);
        const unsigned char *blk = a.params + my_set * a.L.stride;
        const double *Gd = reinterpret_cast<const double *>(blk + a.L.off_G);
        const double *kdd = reinterpret_cast<const double *>(blk + a.L.off_k);
        const double *ld = reinterpret_cast<const double *>(blk + a.L.off_lam);
        const double *u0 = a.ic_unit + (long long)my_ic * N;
        rr_load_rows<0, NPL, L>(q, a, blk, j, base + EL * g);
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            const int node = a.grp.row_node[r * L + j];
            q.Gp[r] = 0; q.k[r] = 1; q.kg[r] = 0; y[r] = 0;
            if (node >= 0) {
                const double G = Gd[node], k = kdd[node];
                double Gp = G;
#pragma unroll 1
                for (int c = a.topo.off[node]; c < a.topo.off[node + 1]; ++c)
                    if (a.topo.sign[c] < 0) Gp *= ld[a.topo.edge[c]];
                q.Gp[r] = (Real)Gp;
                q.k[r] = (Real)k;
                q.kg[r] = (Real)(k / G);
                if constexpr (F64) y[r] = from_list ? a.states[it * N + node] : u0[node] * G / k;
                else y[r] = __fdividef((float)u0[node] * (float)G, (float)k);
            }
        }
        t = (Real)t_start;
        has_chk = false;
        steps = 0;
        gidx = 0;
        need_k1 = true;
        rejected = false;
        near = false;
        working = true;
#pragma unroll 1
        while (gidx < a.n_t && a.t_grid[gidx] <= a.t0) { write_series(gidx); ++gidx; }
    };

    // idle groups take the next solves; one counter update per warp
    auto fetch = [&]() {
        const bool want = !working && !exhausted;
        const unsigned m = __ballot_sync(FULL, want && j == 0);   // bit g: group g
        if (m == 0) return;
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(a.queue, (unsigned long long)__popc(m));
        b0 = __shfl_sync(FULL, b0, 0);
        if (want) {
            const long long it = (long long)b0 + __popc(m & ((1u << g) - 1u));
            if (it < total) start(it);
            else exhausted = true;
        }
    };

    auto residual = [&](const Real (&v)[NPL]) -> Real {
        Real r = 0;
#pragma unroll
        for (int i = 0; i < NPL; ++i) r = rr_max(r, rr_abs(v[i]) * q.kg[i]);
        return rr_gmax(r, L);
    };

    // warp-wide: some group is working / has just started a solve (they
    // change only when a group finishes and the warp fetches)
    bool any_work = false, any_new = false;
    auto refresh = [&]() {
        any_work = __any_sync(FULL, working);
        any_new = __any_sync(FULL, need_k1);
    };
    fetch();
    refresh();

#pragma unroll 1
    for (;;) {
        if (!any_work) break;
        bool done = false;
        int st_code = GRINS_SS_TEND;

        // first derivative and starting step of freshly started solves
        // (only when some group has one); idle and finished groups compute on
        // scratch values throughout and only working groups act
        if (any_new) {
            any_new = false;
            rr_syncwarp();                        // buffer 1 was read by the last stage
#pragma unroll
            for (int r = 0; r < NPL; ++r) z[r] = y[r];
            rr_rhs<1>(q, lk, z, own);
            Real d0 = 0, d1 = 0;
            bool fin = true;
#pragma unroll
            for (int r = 0; r < NPL; ++r) {
                fin = fin && isfinite(z[r]);
                const Real isc = rr_div((Real)1, atol + rtol * rr_abs(y[r]));
                d0 += (y[r] * isc) * (y[r] * isc);
                d1 += (z[r] * isc) * (z[r] * isc);
            }
            d0 = rr_sqrt(rr_gsum(d0, L) * invN);
            d1 = rr_sqrt(rr_gsum(d1, L) * invN);
            fin = grp_all(fin, L);
            const Real res = residual(z);
            if (need_k1) {
                need_k1 = false;
#pragma unroll
                for (int r = 0; r < NPL; ++r) k1[r] = z[r];
                h = (d0 < (Real)1e-5 || d1 < (Real)1e-5) ? (Real)1e-6 : (Real)0.01 * d0 / d1;
                h = rr_min(h, t_end - t);
                if (!fin) { done = true; st_code = GRINS_SS_NONFINITE; }
                else if (res < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                else if (!(t < t_end)) { done = true; st_code = GRINS_SS_TEND; }   // a checkpoint at t_end
            }
        }

        Real t_stop = t_end;
        bool to_grid = false, clipped = false;
        if (gidx < a.n_t && (Real)a.t_grid[gidx] < t_stop) { t_stop = (Real)a.t_grid[gidx]; to_grid = true; }
        Real hh = h;
        if (t + hh >= t_stop) { hh = t_stop - t; clipped = true; }

        rr_comb<true>(z, y, hh, (Real)T::a21, k1);
        rr_rhs<0>(q, lk, z, own);
#pragma unroll
        for (int r = 0; r < NPL; ++r) k2[r] = z[r];
        rr_comb<true>(z, y, hh, (Real)T::a31, k1, (Real)T::a32, k2);
        rr_rhs<1>(q, lk, z, own);
#pragma unroll
        for (int r = 0; r < NPL; ++r) k3[r] = z[r];
        rr_comb<true>(z, y, hh, (Real)T::a41, k1, (Real)T::a42, k2, (Real)T::a43, k3);
        rr_rhs<0>(q, lk, z, own);
#pragma unroll
        for (int r = 0; r < NPL; ++r) k4[r] = z[r];
        rr_comb<true>(z, y, hh, (Real)T::a51, k1, (Real)T::a52, k2, (Real)T::a53, k3, (Real)T::a54, k4);
        rr_rhs<1>(q, lk, z, own);
#pragma unroll
        for (int r = 0; r < NPL; ++r) k5[r] = z[r];
        rr_comb<true>(z, y, hh, (Real)T::a61, k1, (Real)T::a62, k2, (Real)T::a63, k3, (Real)T::a64, k4,
                      (Real)T::a65, k5);
        rr_rhs<0>(q, lk, z, own);
#pragma unroll
        for (int r = 0; r < NPL; ++r) k6[r] = z[r];
        Real ev[NPL];                                 // error estimates
        if constexpr (M == 0) {
            // fifth-order solution in k2 (b2 = 0: no later stage reads k2)
            rr_comb<true>(k2, y, hh, (Real)T::b1, k1, (Real)T::b3, k3, (Real)T::b4, k4, (Real)T::b5, k5,
                          (Real)T::b6, k6);
#pragma unroll
            for (int r = 0; r < NPL; ++r) z[r] = k2[r];
            rr_rhs<1>(q, lk, z, own);                 // z = k7
            rr_comb<false>(ev, y, hh, (Real)T::e1, k1, (Real)T::e3, k3, (Real)T::e4, k4, (Real)T::e5, k5,
                           (Real)T::e6, k6, (Real)T::e7, z);
        } else {
            Real yn[NPL];                             // fifth-order solution
            rr_comb<true>(yn, y, hh, (Real)T::b1, k1, (Real)T::b2, k2, (Real)T::b3, k3, (Real)T::b4, k4,
                          (Real)T::b5, k5, (Real)T::b6, k6);
#pragma unroll
            for (int r = 0; r < NPL; ++r) z[r] = yn[r];
            rr_rhs<1>(q, lk, z, own);                 // z = k7
            rr_comb<false>(ev, y, hh, (Real)T::e1, k1, (Real)T::e2, k2, (Real)T::e3, k3, (Real)T::e4, k4,
                           (Real)T::e5, k5, (Real)T::e6, k6, (Real)T::e7, z);
#pragma unroll
            for (int r = 0; r < NPL; ++r) k2[r] = yn[r];   // the new state where the other pair keeps it
        }

        // A non-finite stage derivative makes err non-finite -- through the
        // error weights or through the later stages it feeds -- and with it
        // the norm, which is therefore the only finiteness test needed (the
        // new state is finite whenever every stage derivative is).
        Real en = 0;
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
            const Real err = ev[r];
            const Real sc = atol + rtol * rr_max(rr_abs(y[r]), rr_abs(k2[r]));
            const Real qq = rr_div(err, sc);
            en += qq * qq;
        }
        en = rr_gsum(en, L) * invN;                   // squared RMS error norm
        if (near) en *= ss_gain;
        const Real res = residual(z);

        // step control of the working groups: controller 0.9 err^(-1/5),
        // err = sqrt(en), evaluated once (en = 0 gives +inf, which the growth
        // limit clamps); growth at most 10, none right after a rejection,
        // shrinking at most to 0.2
        const bool act = working && !done;
        const bool fin = isfinite(en);
        const bool acc = act && fin && en < (Real)1;
        const float fr = 0.9f * ex2_approx(-0.1f * lg2_approx((float)en));
        const float fac = acc ? fminf(fr, rejected ? 1.0f : 10.0f) : fmaxf(fr, 0.2f);
        const Real t_new = clipped ? t_stop : t + hh;
        if (act) {
            ++steps;
            h = hh * (Real)fac;
            rejected = !acc;
            if (!fin || (acc && !(t_new > t))) { done = true; st_code = GRINS_SS_NONFINITE; }
        }
        if (acc) {
            t = t_new;
#pragma unroll
            for (int r = 0; r < NPL; ++r) { y[r] = k2[r]; k1[r] = z[r]; }
            near = res < ss_near;
            if constexpr (!F64) {
                if (res < tail_chk && !has_chk && !done) {
                    // checkpoint: the first accepted state below tail_chk
                    has_chk = true;
                    t_c = t;
                    steps_c = steps;
                    double *dst = a.states + (my_set * a.n_ics + my_ic) * N;
#pragma unroll
                    for (int r = 0; r < NPL; ++r) {
                        const int node = a.grp.row_node[r * L + j];
                        if (node >= 0) dst[node] = (double)y[r];
                    }
                }
            }
            if (!done) {
                if (res < ss_tol) { done = true; st_code = GRINS_SS_CONVERGED; }
                else if (t >= t_end) { done = true; st_code = GRINS_SS_TEND; }
            }
            if (clipped && to_grid) {
#pragma unroll 1
                while (gidx < a.n_t && (Real)a.t_grid[gidx] <= t) { write_series(gidx); ++gidx; }
            }
        }
        if (act && !done && steps >= a.max_steps32) { done = true; st_code = GRINS_SS_MAXSTEPS; }

        if (__any_sync(FULL, done)) {
            if (done) {
                long long idx = my_set * a.n_ics + my_ic;
                if (!GRINS_OK_IDX(idx >= 0 && idx < n_solves, 35, idx)) idx = 0;
                // a borderline decision goes to the FP64 pass: t_end reached
                // with the residual close to ss_tol, or converged so late that
                // the time the residual took to fall from the checkpoint's
                // level says the crossing may lie past t_end
                bool relist = false;
                if constexpr (!F64) {
                    if (has_chk && steps - steps_c <= a.tail_work) {
                        if (st_code == GRINS_SS_TEND) relist = res < a.f_tail_rho;
                        else if (st_code == GRINS_SS_CONVERGED) relist = t_end - t < a.f_tail_late * (t - t_c);
                    }
                }
                if (!relist) {
                    double *dst = a.states + idx * N;
#pragma unroll
                    for (int r = 0; r < NPL; ++r) {
                        const int node = a.grp.row_node[r * L + j];
                        if (node >= 0) dst[node] = (double)y[r];
                    }
                }
                if (j == 0) {
                    a.status[idx] = (uint8_t)st_code;
                    if (a.t_final) a.t_final[idx] = (double)t;
                    if (from_list) {
                        atomicAdd(a.tail_n + 1, (unsigned long long)steps);
                        if (a.n_steps) a.n_steps[idx] += steps;      // after the FP32 pass's attempts
                    } else if (a.n_steps) {
                        a.n_steps[idx] = steps;
                    }
                    if (relist) {
                        const unsigned long long k = atomicAdd(a.tail_n, 1ull);
                        // at most one entry per solve: the list holds n_sets * n_ics
                        if (k < (unsigned long long)n_solves)
                            a.tail_items[k] = typename IntegrateArgs::TailItem{idx, (float)t_c, steps - steps_c};
                    }
                }
#pragma unroll 1
                while (gidx < a.n_t) { write_series(gidx); ++gidx; }
                working = false;
            }
            fetch();
            refresh();
        }
    }
}

}  // namespace grins

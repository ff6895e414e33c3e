// Shared pieces of the Dormand-Prince 5(4) integrators for RACIPE ensembles:
// the tableau, approximate log2/exp2, the checked-mode index macro, the
// precision policies of the generic kernel and the per-warp slot metadata.
//
// Model (GRiNS, Sec. 2.1.1, Eq. 1 and Eq. 2): for every node i
//     dx_i/dt = G_i * prod_{e into i} F_e(x_src(e)) - k_i x_i,
//     F_e = H^S / lambda (activating), H^S (inhibiting),
//     H^S(B) = lambda + (1 - lambda) / (1 + (B/T)^n).
// Written over p = (B/T)^n both factors are (a p + b) / (1 + p) with
//     activating: a = 1,      b = 1/lambda
//     inhibiting: a = lambda, b = 1.
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

// Tsitouras 5(4) (Ch. Tsitouras 2011, Comput. Math. Appl. 62; the paper's
// Tsit5, Sec. 3.1): stage coefficients, 5th-order weights (the last row of
// A, first-same-as-last) and error weights e = b5 - b4.  Unlike
// Dormand-Prince, b2 and e2 are not zero.
namespace ts {
constexpr double a21 = 0.161;
constexpr double a31 = -0.008480655492356989, a32 = 0.335480655492357;
constexpr double a41 = 2.897153057105493, a42 = -6.359448489975075, a43 = 4.3622954328695815;
constexpr double a51 = 5.325864828439257, a52 = -11.748883564062828, a53 = 7.4955393428898365,
                 a54 = -0.09249506636175525;
constexpr double a61 = 5.86145544294642, a62 = -12.92096931784711, a63 = 8.159367898576159,
                 a64 = -0.071584973281401, a65 = -0.028269050394068383;
constexpr double b1 = 0.09646076681806523, b2 = 0.01, b3 = 0.4798896504144996, b4 = 1.379008574103742,
                 b5 = -3.290069515436081, b6 = 2.324710524099774;
constexpr double e1 = -0.00178001105222577714, e2 = -0.0008164344596567469, e3 = 0.007880878010261995,
                 e4 = -0.1447110071732629, e5 = 0.5823571654525552, e6 = -0.45808210592918697,
                 e7 = 0.015151515151515152;
}  // namespace ts

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

// a / b as a times the approximate reciprocal of b (one MUFU.RCP, no range
// handling): for |b| in [2^-126, 2^126], relative error within a few ulp.
// The integrators' divisors stay inside that range (chunk denominators in
// [1, 2^121], error scales >= atol).
__device__ __forceinline__ float div_approx(float a, float b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return a * r;
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

}  // namespace grins

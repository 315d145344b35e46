// dim_ff.cuh -- float-float (FF) arithmetic and the cell physics of the
// FP32-bulk form of the split step, shared by the per-grid kernels
// (dim_bulkff.cu) and the batched persistent kernel (dim_batch.cu).
//
// Why: on GB300 the FP64 pipe issues about one sixty-fourth of the FP32 rate
// (measured: 1.05 TFLOP/s FP64 FMA against 78 TFLOP/s FP32 FMA), so a kernel
// is FP64-bound as soon as it runs more than a few FP64 instructions per cell.
// The FP32-bulk form therefore runs no FP64 instruction inside a step.  The
// state is carried as pairs of floats (hi + lo, 47-48 significant bits) and the
// quantities that need more than FP32 -- where the stiffened-gas "cold" energy
// a_k g_k pinf_k/(g_k - 1) or the kinetic energy cancels against a small
// thermal part, and the volume fraction whose complement 1 - alpha_2 must keep
// its digits near alpha -> 0, 1 -- are formed in FF; everything else (the
// MUSCL/HLLC flux arithmetic, the relaxation roots, the Chebyshev stencil
// sweeps) runs in FP32.  Conversions between the caller's FP64 planes and the
// FF planes use integer operations on the bit patterns only.
//
// FF arithmetic: Knuth's two-sum, the fast two-sum (|a| >= |b|) and the exact
// product by fused multiply-add (Dekker's two-product with an FMA), combined
// in the usual double-float algorithms (Dekker 1971; Hida, Li & Bailey 2001).
// Every operation below is an explicit round-to-nearest intrinsic, so the
// compiler neither contracts nor reorders them.
#pragma once
#include <cuda.h>

#include "dim_device.cuh"

namespace dimk {

struct ff {
    float h, l;  // value h + l, |l| <= ulp(h) / 2
};

__device__ __forceinline__ ff ff_of(float h) { return ff{h, 0.f}; }
__device__ __forceinline__ ff ff_one() { return ff{1.f, 0.f}; }

// s + e = a + b exactly, for |a| >= |b| or a = 0
__device__ __forceinline__ ff ff_qts(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff ff_ts(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// p + e = a b exactly
__device__ __forceinline__ ff ff_tp(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_ts(a.h, b.h);
    return ff_qts(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    const ff s = ff_ts(a.h, b);
    return ff_qts(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    const ff p = ff_tp(a.h, b);
    return ff_qts(p.h, __fmaf_rn(a.l, b, p.l));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const ff p = ff_tp(a.h, b.h);
    return ff_qts(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
// quotient: FP32 estimate, FF remainder, one correction
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdividef(a.h, b.h);
    const ff r = ff_sub(a, ff_mul_f(b, q1));
    return ff_qts(q1, __fdividef(r.h, b.h));
}
// a - b rounded to one float (the exact difference of the high parts plus the low parts)
__device__ __forceinline__ float ff_diff_f(ff a, ff b)
{
    const ff s = ff_ts(a.h, -b.h);
    return __fadd_rn(s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l)));
}
__device__ __forceinline__ float ff_f(ff a) { return __fadd_rn(a.h, a.l); }

// ---------------------------------------------------------------------------
// FP64 <-> FF on the integer pipe
// ---------------------------------------------------------------------------
// hi = the double's sign, exponent and leading 23 mantissa bits (truncated);
// lo = the next 23 mantissa bits, scaled; then renormalised.  Relative error
// below 2^-46.  Magnitudes below 2^-126 become zero; below 2^-80 the low part
// is dropped (relative error 2^-23 there); above the float range the value is
// rounded to a float (infinity) -- none occurs in an admissible state.
__device__ __forceinline__ ff ff_from_d(double x)
{
    const unsigned hi32 = (unsigned)__double2hiint(x), lo32 = (unsigned)__double2loint(x);
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const int ef = e - 896;  // biased float exponent of x
    if (ef < 1) return ff{__uint_as_float(sign), 0.f};
    if (ef > 254) return ff{__double2float_rn(x), 0.f};
    const float h = __uint_as_float(sign | ((unsigned)ef << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
    const unsigned r = (lo32 & 0x1fffffffu) >> 6;  // 23 bits of weight 2^(e - 1069)
    // r as a float without a conversion instruction: 2^23 + r is exact in the
    // mantissa, then subtract 2^23
    float l = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.0f);
    const int es = e - 942;  // float exponent field of 2^(e - 1069)
    l = es >= 1 ? __fmul_rn(l, __uint_as_float((unsigned)es << 23)) : 0.f;
    return ff_qts(h, sign ? -l : l);
}

// h + l as the nearest-below double: the two significands aligned on a 64-bit
// integer (l carries at most 24 bits below h's 24), one renormalisation shift
__device__ __forceinline__ double ff_to_d(ff a)
{
    const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
    const int eh = (int)((hb >> 23) & 0xffu);
    const unsigned long long sign = (unsigned long long)(hb & 0x80000000u) << 32;
    if (eh == 0) return __longlong_as_double((long long)sign);
    long long M = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // weight 2^(eh - 179)
    const int el = (int)((lb >> 23) & 0xffu);
    if (el != 0) {
        long long m = (long long)((lb & 0x7fffffu) | 0x800000u);  // weight 2^(el - 150)
        const int s = el - eh + 29;
        m = s >= 0 ? (m << s) : (s > -40 ? (m >> -s) : 0);
        M += ((lb ^ hb) & 0x80000000u) ? -m : m;
    }
    int ed = eh + 896;  // biased double exponent
    if (M >= (1LL << 53)) {
        M >>= 1;
        ed += 1;
    } else if (M < (1LL << 52)) {
        M <<= 1;
        ed -= 1;
    }
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)ed << 52) | ((unsigned long long)M & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ ff ld_ff(const float2 *P, size_t i)
{
    const float2 v = P[i];
    return ff{v.x, v.y};
}
__device__ __forceinline__ void st_ff(float2 *P, size_t i, ff a) { P[i] = make_float2(a.h, a.l); }

// ---------------------------------------------------------------------------
// Constants of the FP32-bulk kernels, built on the host from DevParams
// ---------------------------------------------------------------------------
struct FFP {
    float g[2], gm1[2], igm1[2], pinf[2], gpinf[2], cv[2], mu[2], k0[2], src[2];
    ff cold[2];   // gamma_k pinf_k / (gamma_k - 1): the cold energy per unit volume fraction
    ff dcold;     // cold_1 - cold_2
    ff pinf_ff[2];
    ff g_ff[2], gm1_ff[2], cv_ff[2], gcv_ff[2];  // gamma_k, gamma_k - 1, Cv_k, (gamma_k - 1) Cv_k
    ff B1_ff;
    float B1;     // pinf_1 - pinf_2
    float cfl, idx, idy, idx2, idy2;
    float inv_Tref, k_exp;
    int k_pow;
};

// TMA descriptors of the FP32-bulk heat stage's planes (2D, nx x ny floats):
// the two iterate planes, T0, C0 = T0 + tau V Ia, tau V and Lam
struct LimMaps {
    CUtensorMap va, vb, T0, C0, tV, L;
};

// ---------------------------------------------------------------------------
// Cell physics
// ---------------------------------------------------------------------------
// p_k = (g_k - 1) E_k / a_k - g_k pinf_k (Eq. eos_stiffened), formed as
// (g_k - 1) (E_k / a_k - cold_k) with the quotient and the difference in FF
__device__ __forceinline__ float ff_phase_p(const FFP &f, int k, ff E, ff a)
{
    if (f.pinf[k] == 0.f) return f.gm1[k] * __fdividef(ff_f(E), ff_f(a));
    return f.gm1[k] * ff_f(ff_sub(ff_div(E, a), f.cold[k]));
}
// the same phase pressure as a pair
__device__ __forceinline__ ff ff_phase_pf(const FFP &f, int k, ff E, ff a)
{
    const ff e = ff_div(E, a);
    return ff_mul(f.pinf[k] == 0.f ? e : ff_sub(e, f.cold[k]), f.gm1_ff[k]);
}

// mixture sound speed c^2 = (a1 A1 + a2 A2) / rho, A_k = g_k (p_k + pinf_k) (Sec. 3.1, Eq. AK)
__device__ __forceinline__ float ff_sound(const FFP &f, float a1, float a2, float p1, float p2, float rho)
{
    return sqrtf(__fdividef(a1 * f.g[0] * (p1 + f.pinf[0]) + a2 * f.g[1] * (p2 + f.pinf[1]), rho));
}

// conductivity lambda_k(T) = k0_k (T / T_ref)^k_exp in FP32
__device__ __forceinline__ float ff_cond(const FFP &f, int k, float T)
{
    if (f.k_pow == 0) return f.k0[k];
    const float t = T * f.inv_Tref;
    if (f.k_pow > 0) {
        float r = t;
        for (int i = 1; i < f.k_pow; i++) r *= t;
        return f.k0[k] * r;
    }
    return f.k0[k] * __powf(t, f.k_exp);
}

// max over the active axes of (|u_axis| + c)/h_axis for one FF state (Sec. 3.1,
// the mixture sound speed of Eq. AK), NaN flagged in st: the per-cell arithmetic
// of the CFL kernel, of the heat kernel that forms the next step's maximum and
// of the batched step.  Every operation after the phase pressures is an
// intrinsic, which the compiler never contracts, so all of them round it alike
// and give the same time step.
__device__ __forceinline__ float ff_wave_speed(const DevParams &p, const FFP &f, const ff *q, unsigned &st)
{
    const ff a1 = ff_sub(ff_one(), q[7]);
    const float p1 = ff_phase_p(f, 0, q[4], a1), p2 = ff_phase_p(f, 1, q[5], q[7]);
    const float rho = __fadd_rn(ff_f(q[0]), ff_f(q[1]));
    const float A1 = __fmul_rn(__fmul_rn(ff_f(a1), f.g[0]), __fadd_rn(p1, f.pinf[0]));
    const float A2 = __fmul_rn(__fmul_rn(ff_f(q[7]), f.g[1]), __fadd_rn(p2, f.pinf[1]));
    const float cs = sqrtf(__fdividef(__fadd_rn(A1, A2), rho));
    float m = 0.f;
    if (p.nx > 1) {
        const float s = __fmul_rn(__fadd_rn(fabsf(__fdividef(ff_f(q[2]), rho)), cs), f.idx);
        m = fmaxf(m, s);
        if (isnan(s)) st |= DIM_ST_NAN;
    }
    if (p.ny > 1) {
        const float s = __fmul_rn(__fadd_rn(fabsf(__fdividef(ff_f(q[3]), rho)), cs), f.idy);
        m = fmaxf(m, s);
        if (isnan(s)) st |= DIM_ST_NAN;
    }
    return m;
}

// end-of-step admissibility of an FF state (q in the global plane order):
// alpha_2 and alpha_1 = 1 - alpha_2 positive, m_k > 0, E_k > alpha_k pinf_k, no NaN
__device__ __forceinline__ unsigned ff_check(const FFP &f, const ff *q)
{
    const ff a1 = ff_sub(ff_one(), q[7]);
    unsigned st = 0;
    const bool ok = q[7].h > 0.f && a1.h > 0.f && q[0].h > 0.f && q[1].h > 0.f &&
                    ff_diff_f(q[4], ff_mul(a1, f.pinf_ff[0])) > 0.f && ff_diff_f(q[5], ff_mul(q[7], f.pinf_ff[1])) > 0.f;
    if (!ok) st |= DIM_ST_NONPHYS;
#pragma unroll
    for (int k = 0; k < NQ; k++)
        if (isnan(q[k].h)) st |= DIM_ST_NAN;
    return st;
}

// Below this minor-phase fraction an FP32 relaxation root is accurate enough:
// the relaxed pressure moves by ~3e9 Pa per unit error of the fraction, and
// the FP32 root's error is ~1e-7 of the minor fraction (< 3e-3 Pa here), so
// the float-float Newton correction runs only in mixed cells.
constexpr float kNewtonFraction = 1e-5f;

// Pressure relaxation (Sec. 3.3, three steps) of one cell in place.
// Step (1): with dE_k = -p_I da_k and p_I the relaxed pressure x, the EOS gives
// a_k(x) - a_k^0 = d_k(x) = a_k^0 (p_k^0 - x) / (g_k (x + pinf_k)); the volume
// constraint d_1(x) + d_2(x) = 0, multiplied by g_1 g_2 (x + pinf_1)(x + pinf_2), is
//   a_1^0 g_2 (p_1^0 - x)(x + pinf_2) + a_2^0 g_1 (p_2^0 - x)(x + pinf_1) = 0,
// the same quadratic as in the conserved variables but written in the phase
// pressures (the cancellation of E_k against the cold energy is done in FF when
// p_k^0 is formed).  Its larger root (the one with x + pinf_k > 0) is solved in
// FP32 and corrected by one Newton step on d_1 + d_2 evaluated in FF: where a
// stiff phase is present the relaxed pressure moves by about
// da (cold_1 - cold_2) / sum(a_k / (g_k - 1)) per error da of the volume
// fraction, so the fraction must carry more than FP32 digits.  The minor
// phase's fraction takes a_m^0 + d_m(x), the major one 1 - a_m.
// Step (2): p^(2) from sum_k a_k' (p + g_k pinf_k)/(g_k - 1) = rho e, written
// as the change against the phase energies before the step (mis = rho e - E_1 -
// E_2 in FF, the cold energy moved by da_2 in FF).  Step (3):
// E_k = a_k' p^(2) / (g_k - 1) + a_k' cold_k, so both phases end at p^(2).
__device__ __forceinline__ unsigned ff_prelax(const FFP &f, ff *q)
{
    const ff a2 = q[7], a1 = ff_sub(ff_one(), a2);
    const ff P1 = ff_phase_pf(f, 0, q[4], a1), P2 = ff_phase_pf(f, 1, q[5], a2);
    const float p1 = ff_f(P1), p2 = ff_f(P2);
    const float A1 = ff_f(a1), A2 = ff_f(a2);
    const float w1 = A1 * f.g[1], w2 = A2 * f.g[0];
    // qa x^2 - qb x - qc = 0 (qa > 0): larger root without cancellation
    const float qa = w1 + w2;
    const float qb = w1 * (p1 - f.pinf[1]) + w2 * (p2 - f.pinf[0]);
    const float qc = w1 * p1 * f.pinf[1] + w2 * p2 * f.pinf[0];
    float disc = qb * qb + 4.f * qa * qc;
    unsigned st = 0;
    if (disc < 0.f) {
        st |= DIM_ST_NOROOT;
        disc = 0.f;
    }
    const float sq = sqrtf(disc);
    const float x = qb >= 0.f ? __fdividef(qb + sq, 2.f * qa) : __fdividef(2.f * qc, sq - qb);
    ff a2n, da2;
    const bool minor2 = A2 <= 0.5f;
    if (fminf(A1, A2) >= kNewtonFraction) {
        // d_k(x) in FF, their x-derivatives in FP32, one Newton step
        const ff y1 = ff_add_f(f.pinf_ff[0], x), y2 = ff_add_f(f.pinf_ff[1], x);
        const ff d1 = ff_div(ff_mul(a1, ff_add_f(P1, -x)), ff_mul(y1, f.g_ff[0]));
        const ff d2 = ff_div(ff_mul(a2, ff_add_f(P2, -x)), ff_mul(y2, f.g_ff[1]));
        const float e1 = ff_f(y1), e2 = ff_f(y2);
        const float dd1 = -__fdividef(A1 * (p1 + f.pinf[0]), f.g[0] * e1 * e1);
        const float dd2 = -__fdividef(A2 * (p2 + f.pinf[1]), f.g[1] * e2 * e2);
        const float dx = -__fdividef(ff_f(ff_add(d1, d2)), dd1 + dd2);
        if (minor2) {
            da2 = ff_add_f(d2, dd2 * dx);
        } else {
            da2 = ff_neg(ff_add_f(d1, dd1 * dx));
        }
    } else if (minor2) {  // a nearly pure cell: the FP32 root and change suffice
        da2 = ff_of(A2 * __fdividef(p2 - x, f.g[1] * (x + f.pinf[1])));
    } else {
        da2 = ff_of(-A1 * __fdividef(p1 - x, f.g[0] * (x + f.pinf[0])));
    }
    if (minor2) a2n = ff_add(a2, da2);
    else a2n = ff_sub(ff_one(), ff_sub(a1, da2));
    const ff a1n = ff_sub(ff_one(), a2n);
    // rho e - E_1 - E_2 with the kinetic energy (rho u)^2 / (2 rho) in FF
    const ff rho = ff_add(q[0], q[1]);
    const ff ke = ff_mul_f(ff_div(ff_add(ff_mul(q[2], q[2]), ff_mul(q[3], q[3])), rho), 0.5f);
    const float mis = ff_f(ff_sub(ff_sub(q[6], ke), ff_add(q[4], q[5])));
    const float th = mis + A1 * p1 * f.igm1[0] + A2 * p2 * f.igm1[1];
    const float num = ff_f(ff_add_f(ff_mul(f.dcold, da2), th));
    const float A1n = ff_f(a1n), A2n = ff_f(a2n);
    const float pr = __fdividef(num, A1n * f.igm1[0] + A2n * f.igm1[1]);
    q[4] = ff_add_f(ff_mul(a1n, f.cold[0]), A1n * pr * f.igm1[0]);
    q[5] = ff_add_f(ff_mul(a2n, f.cold[1]), A2n * pr * f.igm1[1]);
    q[7] = a2n;
    if (!(a2n.h > 0.f && a1n.h > 0.f && q[0].h > 0.f && q[1].h > 0.f && pr + f.pinf[0] > 0.f && pr + f.pinf[1] > 0.f))
        st |= DIM_ST_NONPHYS;
    if (isnan(pr) || isnan(a2n.h)) st |= DIM_ST_NAN;
    return st;
}

// p,T equilibrium at fixed m_k and rho e (Sec. 3.4.1 end state, Sec. 3.4.2
// projection), with E_k = C_k T + a_k pinf_k (C_k = m_k Cv_k), p_1 = p_2 = p and
// T_1 = T_2 = T.  The EOS gives a_k = G_k C_k T / (p + pinf_k) (G_k = gamma_k - 1);
// the volume constraint gives T = 1 / sum_k G_k C_k / (p + pinf_k); the energy
// rho e = sum_k a_k (p + g_k pinf_k)/(g_k - 1) then leaves one equation in p,
//   F(p) = sum_k G_k C_k W_k / (p + pinf_k) - C = 0,  W_k = rho e - pinf_k,
// the same equilibrium as the alpha-quadratic of the FP64 kernels written in
// the common pressure.  With y = p + pinf_2 and B_1 = pinf_1 - pinf_2 it is the
// quadratic C y^2 + (C B_1 - G_1 C_1 W_1 - G_2 C_2 W_2) y - G_2 C_2 W_2 B_1 = 0,
// whose middle coefficient cancels to about -C p where a stiff phase dominates:
// it is formed in FF, the positive root taken in FP32, and in mixed cells one
// Newton step on F evaluated in FF gives y to FF precision.  Then
// g_k = G_k C_k / (p + pinf_k), T = 1 / (g_1 + g_2), a_2 = g_2 / (g_1 + g_2) (the
// minor phase's fraction directly, the major one as 1 - minor; in FF in mixed
// cells, from FP32 quotients where the minor fraction is below kNewtonFraction),
// and
// E_k = a_k p / (g_k - 1) + a_k cold_k, the second E_k = rho e - the first.
// Returns T (FP32), a_2 and the phase energies.
__device__ __forceinline__ unsigned ff_equilibrium(const FFP &f, ff m1, ff m2, ff rhoe, float &T, ff &a2n, ff &E1,
                                                   ff &E2)
{
    const ff GC1 = ff_mul(m1, f.gcv_ff[0]), GC2 = ff_mul(m2, f.gcv_ff[1]);
    const ff C = ff_add(ff_mul(m1, f.cv_ff[0]), ff_mul(m2, f.cv_ff[1]));
    const ff W1 = ff_sub(rhoe, f.pinf_ff[0]), W2 = ff_sub(rhoe, f.pinf_ff[1]);
    const ff GW1 = ff_mul(GC1, W1), GW2 = ff_mul(GC2, W2);
    const float Cf = ff_f(C), B1 = f.B1;
    const float qb = ff_f(ff_sub(ff_mul(C, f.B1_ff), ff_add(GW1, GW2)));
    const float qc = -ff_f(GW2) * B1;  // C y^2 + qb y + qc = 0
    unsigned st = 0;
    float disc = qb * qb - 4.f * Cf * qc;
    if (disc < 0.f) {
        st |= DIM_ST_NOROOT;
        disc = 0.f;
    }
    const float sq = sqrtf(disc);
    float y = qb <= 0.f ? __fdividef(sq - qb, 2.f * Cf) : __fdividef(-2.f * qc, qb + sq);
    if (B1 == 0.f) y = __fdividef(ff_f(ff_add(GW1, GW2)), Cf);  // linear: C y = sum G_k C_k W_k
    const ff Y2 = ff_of(y), Y1 = ff_add_f(f.B1_ff, y);
    ff Yb = Y2, Ya = Y1;
    // Newton step on F in FF, in mixed cells (the minor fraction g_m / (g_1 + g_2)
    // estimated in FP32 from the root)
    const float g1e = __fdividef(ff_f(GC1), ff_f(Y1)), g2e = __fdividef(ff_f(GC2), y);
    bool minor2;
    if (fminf(g1e, g2e) >= kNewtonFraction * (g1e + g2e)) {
        const ff t1 = ff_div(GW1, Y1), t2 = ff_div(GW2, Y2);
        const float dF = -__fdividef(ff_f(t1), ff_f(Y1)) - __fdividef(ff_f(t2), y);
        const float dy = -__fdividef(ff_f(ff_sub(ff_add(t1, t2), C)), dF);
        Yb = ff_add_f(Y2, dy);
        Ya = ff_add_f(Y1, dy);
        const ff g1 = ff_div(GC1, Ya), g2 = ff_div(GC2, Yb);
        const ff gs = ff_add(g1, g2);
        T = __fdividef(1.f, ff_f(gs));
        minor2 = ff_f(g2) <= ff_f(g1);
        a2n = minor2 ? ff_div(g2, gs) : ff_sub(ff_one(), ff_div(g1, gs));
    } else {
        // a nearly pure cell: T and the minor fraction from the FP32 quotients
        // (their FP32 digits are all the state keeps of a fraction below
        // kNewtonFraction), the major fraction as 1 - minor in FF
        const float gs = g1e + g2e;
        T = __fdividef(1.f, gs);
        minor2 = g2e <= g1e;
        const float am = __fdividef(minor2 ? g2e : g1e, gs);
        a2n = minor2 ? ff_of(am) : ff_add_f(ff_one(), -am);
    }
    const ff a1n = ff_sub(ff_one(), a2n);
    const float p = ff_f(ff_sub(Yb, f.pinf_ff[1]));  // y - pinf_2
    if (minor2) {
        E2 = ff_add_f(ff_mul(a2n, f.cold[1]), ff_f(a2n) * p * f.igm1[1]);
        E1 = ff_sub(rhoe, E2);
    } else {
        E1 = ff_add_f(ff_mul(a1n, f.cold[0]), ff_f(a1n) * p * f.igm1[0]);
        E2 = ff_sub(rhoe, E1);
    }
    if (!(a2n.h > 0.f && a1n.h > 0.f && T > 0.f && p + f.pinf[0] > 0.f && p + f.pinf[1] > 0.f)) st |= DIM_ST_NONPHYS;
    if (isnan(T) || isnan(a2n.h)) st |= DIM_ST_NAN;
    return st;
}

// mixture temperature of a cell in thermal equilibrium: (E_1 + E_2 - a_1 pinf_1 - a_2 pinf_2) / C
__device__ __forceinline__ float ff_mixture_T(const FFP &f, float m1, float m2, ff E1, ff E2, ff a2)
{
    const ff a1 = ff_sub(ff_one(), a2);
    const float th = ff_diff_f(ff_add(E1, E2), ff_add(ff_mul(a1, f.pinf_ff[0]), ff_mul(a2, f.pinf_ff[1])));
    return __fdividef(th, m1 * f.cv[0] + m2 * f.cv[1]);
}

// conduction coefficients at (T, a): V = 1/(C + B_1^2/K), K = T^2 sum_k G_k C_k / a_k^2,
// Lam = sum_k a_k lambda_k(T) (Sec. 3.4.2), FP32
__device__ __forceinline__ void ff_heat_coeffs(const FFP &f, float m1, float m2, float T, ff a2, float &V, float &Lam)
{
    const float a2f = ff_f(a2), a1f = ff_f(ff_sub(ff_one(), a2));
    const float C1 = m1 * f.cv[0], C2 = m2 * f.cv[1];
    const float r1 = __fdividef(f.gm1[0] * C1 * T, a1f * a1f);
    const float r2 = __fdividef(f.gm1[1] * C2 * T, a2f * a2f);
    const float K = T * (r1 + r2);
    V = __fdividef(1.f, C1 + C2 + f.B1 * __fdividef(f.B1, K));
    Lam = a1f * ff_cond(f, 0, T) + a2f * ff_cond(f, 1, T);
}

// block-wide max of non-negative floats into a double accumulator (one
// conversion per block)
__device__ __forceinline__ void block_max_to_f(unsigned long long *acc, float v)
{
    __shared__ float s_wf[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_wf[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        float x = l < nw ? s_wf[l] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (l == 0) atomic_max_pos(acc, (double)x);
    }
}

// warp-wide minimum of positive floats (NaN ignored) into an accumulator that
// holds bits(+inf) - bits(min) (a max accumulator, 0 when empty: the map is
// decreasing for positive floats), without a block barrier; the atomic is
// issued only when the warp's value improves on the accumulator's, which after
// the first warps of a launch it rarely does
__device__ __forceinline__ void warp_min_pos_bits(unsigned *acc, float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const unsigned key = 0x7f800000u - __float_as_uint(v);
    if ((threadIdx.x & 31) == 0 && v > 0.f && key > *(volatile unsigned *)acc) atomicMax(acc, key);
}

// ---------------------------------------------------------------------------
// FP32 face arithmetic of the sweep (MUSCL + HLLC), as the FP64 kernel but in
// FP32 on the thermal and kinetic energies (the cold energies travel with the
// FF volume-fraction flux)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float minmodf(float a, float b)
{
    if (a > 0.f && b > 0.f) return fminf(a, b);
    if (a < 0.f && b < 0.f) return fmaxf(a, b);
    return 0.f;
}

// In a stiff phase the phase energy E_k = a_k (p_k + g_k pinf_k)/(g_k - 1) is
// dominated by the cold part a_k cold_k, while the pressure lives in the
// thermal part Et_k = a_k p_k/(g_k - 1).  The FP32 HLLC carries Et_k and the
// kinetic energy; across an acoustic wave the star state E_k* = chi E_k splits
// as Et_k* = chi Et_k + (chi - 1) a_k cold_k with chi - 1 = (S* - u)/(S_K - S*),
// and u* a_k* cold_k travels with the FF volume-fraction flux.
struct FaceF {
    float un, ut, rho, p, c, C1, C2;
    float q[7];  // m1, m2, rho u_n, rho u_t, Et1, Et2, Et1 + Et2 + rho|u|^2/2
};

__device__ __forceinline__ void face_state_f(const FFP &f, float a1, float a2, const float *w, FaceF &s)
{
    const float m1 = w[0], m2 = w[1], un = w[2], ut = w[3], p1 = w[4], p2 = w[5];
    const float rho = m1 + m2;
    const float Et1 = a1 * p1 * f.igm1[0];
    const float Et2 = a2 * p2 * f.igm1[1];
    s.un = un;
    s.ut = ut;
    s.rho = rho;
    s.p = a1 * p1 + a2 * p2;
    s.c = ff_sound(f, a1, a2, p1, p2, rho);
    s.C1 = a1 * f.cold[0].h;
    s.C2 = a2 * f.cold[1].h;
    s.q[0] = m1;
    s.q[1] = m2;
    s.q[2] = rho * un;
    s.q[3] = rho * ut;
    s.q[4] = Et1;
    s.q[5] = Et2;
    s.q[6] = Et1 + Et2 + 0.5f * rho * (un * un + ut * ut);
}

// HLLC (Davis speeds, x/t = 0 state) in FP32; F[0..6] and u* = F[7]; returns
// the side (0 left, 1 right) whose alpha_2 the x/t = 0 state carries
__device__ __forceinline__ int hllc_f(const FaceF &L, const FaceF &R, float *F)
{
    const float SL = fminf(L.un - L.c, R.un - R.c);
    const float SR = fmaxf(L.un + L.c, R.un + R.c);
    const float Ss = __fdividef(R.p - L.p + L.rho * L.un * (SL - L.un) - R.rho * R.un * (SR - R.un),
                                L.rho * (SL - L.un) - R.rho * (SR - R.un));
    float q[7], us, ps;
    int side;
    if (SL >= 0.f) {
#pragma unroll
        for (int k = 0; k < 7; k++) q[k] = L.q[k];
        us = L.un;
        ps = L.p;
        side = 0;
    } else if (SR >= 0.f) {
        const bool left = Ss >= 0.f;
        const FaceF &K = left ? L : R;
        const float SK = left ? SL : SR;
        const float rd = __fdividef(1.f, SK - Ss);
        const float chi = (SK - K.un) * rd;
        const float chim1 = (Ss - K.un) * rd;
        q[0] = chi * K.q[0];
        q[1] = chi * K.q[1];
        q[2] = chi * K.rho * Ss;
        q[3] = chi * K.rho * K.ut;
        q[4] = chi * K.q[4] + chim1 * K.C1;
        q[5] = chi * K.q[5] + chim1 * K.C2;
        q[6] = chi * (K.q[6] + (Ss - K.un) * (K.rho * Ss + __fdividef(K.p, SK - K.un))) + chim1 * (K.C1 + K.C2);
        us = Ss;
        ps = K.p + K.rho * (SK - K.un) * (Ss - K.un);
        side = left ? 0 : 1;
    } else {
#pragma unroll
        for (int k = 0; k < 7; k++) q[k] = R.q[k];
        us = R.un;
        ps = R.p;
        side = 1;
    }
    F[0] = us * q[0];
    F[1] = us * q[1];
    F[2] = us * q[2] + ps;
    F[3] = us * q[3];
    F[4] = us * q[4];
    F[5] = us * q[5];
    F[6] = us * (q[6] + ps);
    F[7] = us;
    return side;
}

__device__ __forceinline__ int bc_mapf(int a, int len, int bc)
{
    if (a >= 0 && a < len) return a;
    if (bc == DIM_BC_PERIODIC) return ((a % len) + len) % len;
    return a < 0 ? 0 : len - 1;
}

// dynamic shared memory of one FF sweep tile
__host__ __device__ constexpr size_t sweepff_smem(int TN, int TL)
{
    return sizeof(float2) * ((size_t)NQ * (TN + 4) * TL + (size_t)(TN + 1) * TL) +
           sizeof(float) * (6 * (size_t)(TN + 4) * TL + 8 * (size_t)(TN + 1) * TL);
}

// One tile (TN cells along the sweep axis x TL lines, first cell a0, first line
// t0) of the FP32-bulk sweep: PVT-consistent minmod MUSCL (Sec. 3.6) on
// (alpha_2, m_1, m_2, u_n, u_t, p_1, p_2), HLLC fluxes, the update with the
// non-conservative term R(U_i) du* (Sec. 3.1), and the pressure relaxation
// (Sec. 3.3) when relax != 0.  dtdx = dt / h of the axis.  States in FF planes.
// BOUND: also the minimum density of the updated cells into sc->vbound (the
// last sweep of a step that runs the viscous stage)
template <int AXIS, int TN, int TL, bool BOUND = false>
__device__ __forceinline__ void sweepff_tile(const DevParams &p, const FFP &f, const float2 *Uin, float2 *Uout,
                                             float dtdx, Scalars *sc, int relax, int check, int a0, int t0,
                                             void *smem)
{
    constexpr int NE = TN + 4;
    constexpr int NL = NE * TL;
    constexpr int NFL = TN + 1;
    constexpr int NF = NFL * TL;
    float2 *sU = (float2 *)smem;      // [8][NL] conserved state (FF)
    float2 *sF7 = sU + NQ * NL;       // [NF] volume-fraction flux u* alpha_2 (FF)
    float *sW = (float *)(sF7 + NF);  // [6][NL] m1, m2, u_n, u_t, p1, p2
    float *sF = sW + 6 * NL;          // [8][NF] F0..F6, u*
    const int n = p.n;
    const int len = AXIS == 0 ? p.nx : p.ny;
    const int ntr = AXIS == 0 ? p.ny : p.nx;
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    auto cidx = [&](int e, int l) { return AXIS == 0 ? l * NE + e : e * TL + l; };
    auto fidx = [&](int fc, int l) { return AXIS == 0 ? l * NFL + fc : fc * TL + l; };
    auto S = [&](int k, int i) { return ff{sU[k * NL + i].x, sU[k * NL + i].y}; };

    for (int li = threadIdx.x; li < NL; li += blockDim.x) {
        int e, l;
        if (AXIS == 0) {
            l = li / NE;
            e = li - l * NE;
        } else {
            e = li / TL;
            l = li - e * TL;
        }
        const int tr = min(t0 + l, ntr - 1);
        const int al = bc_mapf(a0 - 2 + e, len, p.bc[AXIS]);
        const int x = AXIS == 0 ? al : tr, y = AXIS == 0 ? tr : al;
        const size_t c = (size_t)y * p.nx + x;
        ff q[NQ];
        q[0] = ld_ff(Uin, c);
        q[1] = ld_ff(Uin, n + c);
        q[2] = ld_ff(Uin, QN * (size_t)n + c);
        q[3] = ld_ff(Uin, QT * (size_t)n + c);
#pragma unroll
        for (int k = 4; k < NQ; k++) q[k] = ld_ff(Uin, k * (size_t)n + c);
#pragma unroll
        for (int k = 0; k < NQ; k++) sU[k * NL + li] = make_float2(q[k].h, q[k].l);
        const ff a1 = ff_sub(ff_one(), q[7]);
        const float rho = ff_f(q[0]) + ff_f(q[1]);
        sW[0 * NL + li] = ff_f(q[0]);
        sW[1 * NL + li] = ff_f(q[1]);
        sW[2 * NL + li] = __fdividef(ff_f(q[2]), rho);
        sW[3 * NL + li] = __fdividef(ff_f(q[3]), rho);
        sW[4 * NL + li] = ff_phase_p(f, 0, q[4], a1);
        sW[5 * NL + li] = ff_phase_p(f, 1, q[5], q[7]);
    }
    __syncthreads();

    for (int fi = threadIdx.x; fi < NF; fi += blockDim.x) {
        int fc, l;
        if (AXIS == 0) {
            l = fi / NFL;
            fc = fi - l * NFL;
        } else {
            fc = fi / TL;
            l = fi - fc * TL;
        }
        const int iL = cidx(fc + 1, l), iR = cidx(fc + 2, l);
        ff aL = S(7, iL), aR = S(7, iR);
        float wl[6], wr[6];
        if (p.limiter != DIM_LIMITER_NONE) {
            const int iLL = cidx(fc, l), iRR = cidx(fc + 3, l);
            const bool ob = p.limiter == DIM_LIMITER_OVERBEE;
            // volume fraction: differences in FF (a fraction near 1 keeps the
            // digits of its complement), limited slope in FP32
            const float dm = ff_diff_f(aL, S(7, iLL)), dc = ff_diff_f(aR, aL), dp = ff_diff_f(S(7, iRR), aR);
            float sl = minmodf(dm, dc), sr = minmodf(dc, dp);
            if (ob) {
                sl *= 2.f;
                sr *= 2.f;
            }
            aL = ff_add_f(aL, 0.5f * sl);
            aR = ff_add_f(aR, -0.5f * sr);
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float *Wk = sW + k * NL;
                float s1 = minmodf(Wk[iL] - Wk[iLL], Wk[iR] - Wk[iL]);
                float s2 = minmodf(Wk[iR] - Wk[iL], Wk[iRR] - Wk[iR]);
                if (ob && k <= 1) {  // m1, m2
                    s1 *= 2.f;
                    s2 *= 2.f;
                }
                wl[k] = Wk[iL] + 0.5f * s1;
                wr[k] = Wk[iR] - 0.5f * s2;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 6; k++) {
                wl[k] = sW[k * NL + iL];
                wr[k] = sW[k * NL + iR];
            }
        }
        FaceF L, R;
        face_state_f(f, ff_f(ff_sub(ff_one(), aL)), ff_f(aL), wl, L);
        face_state_f(f, ff_f(ff_sub(ff_one(), aR)), ff_f(aR), wr, R);
        float F[8];
        const int side = hllc_f(L, R, F);
#pragma unroll
        for (int k = 0; k < 8; k++) sF[k * NF + fi] = F[k];
        const ff F7 = ff_mul_f(side ? aR : aL, F[7]);
        sF7[fi] = make_float2(F7.h, F7.l);
    }
    __syncthreads();

    unsigned st = 0;
    float rmin = __int_as_float(0x7f800000);  // +inf
    for (int oi = threadIdx.x; oi < TN * TL; oi += blockDim.x) {
        int i, l;
        if (AXIS == 0) {
            l = oi / TN;
            i = oi - l * TN;
        } else {
            i = oi / TL;
            l = oi - i * TL;
        }
        const int al = a0 + i, tr = t0 + l;
        if (al >= len || tr >= ntr) continue;
        const int ci = cidx(i + 2, l), fm = fidx(i, l), fp = fidx(i + 1, l);
        const ff a2 = S(7, ci), a1 = ff_sub(ff_one(), a2);
        // du* exactly as a pair, so that alpha du* and the alpha flux difference cancel
        const ff du = ff_ts(sF[7 * NF + fp], -sF[7 * NF + fm]);
        const float duf = ff_f(du);
        const float R4 = ff_f(a1) * sW[4 * NL + ci], R5 = ff_f(a2) * sW[5 * NL + ci];
        ff q[NQ];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            float inc = dtdx * (sF[k * NF + fp] - sF[k * NF + fm]);
            if (k == 4) inc += dtdx * R4 * duf;
            if (k == 5) inc += dtdx * R5 * duf;
            q[k] = ff_add_f(S(k, ci), -inc);
        }
        // alpha_2 += dt/dx (alpha_2 du* - (F7+ - F7-)); the cold energies travel
        // with the volume-fraction fluxes: u* a_2* cold_2 = cold_2 F7 and
        // u* a_1* cold_1 = cold_1 (u* - F7)
        const ff dF7 = ff_sub(ff{sF7[fp].x, sF7[fp].y}, ff{sF7[fm].x, sF7[fm].y});
        q[7] = ff_add(a2, ff_mul_f(ff_sub(ff_mul(a2, du), dF7), dtdx));
        const ff c1 = ff_mul_f(ff_mul(ff_sub(du, dF7), f.cold[0]), dtdx);
        const ff c2 = ff_mul_f(ff_mul(dF7, f.cold[1]), dtdx);
        q[4] = ff_sub(q[4], c1);
        q[5] = ff_sub(q[5], c2);
        q[6] = ff_sub(q[6], ff_add(c1, c2));
        ff o[NQ] = {q[0], q[1], q[0], q[0], q[4], q[5], q[6], q[7]};
        o[QN] = q[2];
        o[QT] = q[3];
        if (relax) {
            const unsigned s = ff_prelax(f, o);
            if (s & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= s & DIM_ST_NAN;
        }
        if (check) st |= ff_check(f, o);
        if constexpr (BOUND) rmin = fminf(rmin, ff_f(o[0]) + ff_f(o[1]));  // the viscous kernels' rho
        const int x = AXIS == 0 ? al : tr, y = AXIS == 0 ? tr : al;
        const size_t c = (size_t)y * p.nx + x;
#pragma unroll
        for (int k = 0; k < NQ; k++) st_ff(Uout, k * (size_t)n + c, o[k]);
    }
    flag(sc, st);
    if constexpr (BOUND) warp_min_pos_bits(&sc->vbound, rmin);
    __syncthreads();  // the shared tile is reused by the next tile of a persistent block
}

// FP32 stencil operators of the parabolic stages
__device__ __forceinline__ float lapf(const DevParams &p, const Nb &nb, int c, const float *v, const float *L,
                                      float idx2, float idy2)
{
    float r = 0.f;
    const float vc = v[c], Lc = L[c];
    if (p.nx > 1) {
        const float fl = nb.xm >= 0 ? 0.5f * (L[nb.xm] + Lc) * (vc - v[nb.xm]) * idx2 : 0.f;
        const float fr = nb.xp >= 0 ? 0.5f * (Lc + L[nb.xp]) * (v[nb.xp] - vc) * idx2 : 0.f;
        r += fr - fl;
    }
    if (p.ny > 1) {
        const float fl = nb.ym >= 0 ? 0.5f * (L[nb.ym] + Lc) * (vc - v[nb.ym]) * idy2 : 0.f;
        const float fr = nb.yp >= 0 ? 0.5f * (Lc + L[nb.yp]) * (v[nb.yp] - vc) * idy2 : 0.f;
        r += fr - fl;
    }
    return r;
}

__device__ __forceinline__ float gershf(const DevParams &p, const Nb &nb, int c, const float *V, const float *L,
                                        float idx2, float idy2)
{
    const float Lc = L[c];
    float s = 0.f;
    if (p.nx > 1) {
        const float fl = nb.xm >= 0 ? 0.5f * (L[nb.xm] + Lc) : 0.f;
        const float fr = nb.xp >= 0 ? 0.5f * (Lc + L[nb.xp]) : 0.f;
        s += (fl + fr) * idx2;
    }
    if (p.ny > 1) {
        const float fl = nb.ym >= 0 ? 0.5f * (L[nb.ym] + Lc) : 0.f;
        const float fr = nb.yp >= 0 ? 0.5f * (Lc + L[nb.yp]) : 0.f;
        s += (fl + fr) * idy2;
    }
    return 2.f * V[c] * s;
}

}  // namespace dimk

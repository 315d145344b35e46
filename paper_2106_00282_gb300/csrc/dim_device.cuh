// dim_device.cuh -- device building blocks of the split step (sm_103a).
//
// Stiffened-gas thermodynamics, the three-step pressure relaxation, the p,T
// equilibrium used by the temperature relaxation and the conduction
// projection, the HLLC face solver and a bounded grid-wide barrier for the
// cooperative (persistent) parabolic kernels.
//
// Paper: Zhang, Menshov, Wang & Shen, arXiv:2106.00282 (equations cited at the
// functions).  Phase 0 is the dense phase, phase 1 the gas; alpha = alpha_2.
#pragma once
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "../../include/dim.h"

namespace dimk {

constexpr int NQ = 8;     // conserved planes
constexpr int PMAX = 64;  // largest Chebyshev parameter count a launch supports

// Parameters as passed by value to every kernel.
struct DevParams {
    double g[2], pinf[2], cv[2];
    double gm1[2];      // gamma_k - 1
    double inv_gm1[2];  // 1 / (gamma_k - 1)
    double gpinf[2];    // gamma_k pinf_k
    double k0[2], k_exp, T_ref, inv_Tref;
    int k_pow;          // conductivity exponent: 0 constant, 1..8 integer power, -1 general
    double mu[2];
    double cfl;
    double dx, dy, idx, idy, idx2, idy2;  // spacing, 1/h and 1/h^2
    int nx, ny, n;
    int limiter, bc[2], trelax, n_outer, p_policy, p_fixed, p_min, p_max;
    int trelax_iters;  // simple iterations of DIM_TRELAX_MIDPOINT
    int heat_alpha;    // DIM_HEAT_ALPHA_PROJECTION or DIM_HEAT_ALPHA_LINEAR
    int precision;  // DIM_PRECISION_FP64 or DIM_PRECISION_FP32_BULK
    double src[2];  // external heat source intensities I_k
    // 1: the Chebyshev lambda_max of every LIM solve is read from the context
    // scalars (a replayed schedule) instead of being reduced from the state
    int frozen;
    // roots of T_P: beta[(P-1)*PMAX + m-1] = cos((2m-1) pi / (2P)), m = 1..P,
    // tabulated on the host (libm) once per context
    const double *beta;
};

// Device scalars of one context.  The fields before `status` are cleared at
// the start of every step / stage call; status and the barrier generation
// persist.
struct Scalars {
    unsigned long long smax;     // max (|u|+c)/h of the step (bits of a non-negative double)
    unsigned long long lam[12];  // Gershgorin lambda_max per LIM solve (heat iterations 0..7, viscous x, y)
    int P[12];                   // Chebyshev parameter count used: [0] heat, [1] viscous x, [2] viscous y
    // FP32-bulk form: the minimum density of the state after the step's last
    // hyperbolic sweep, as bits(+inf) - bits(rho_min) (0: none recorded); it
    // bounds lambda_max of the viscous solves
    unsigned int vbound;
    float dt32;                  // FP32-bulk form: cfl / smax, written once per step by the CFL kernel
    unsigned int wave_blocks;    // FP32-bulk form: blocks of the CFL kernel that have finished
    unsigned int bar_count;      // grid barrier: arrivals of the current generation
    unsigned int status;         // DIM_ST_* bits
    unsigned int bar_gen;        // grid barrier: generation
    // FP32-bulk form, outside the per-step reset: a heat kernel that also forms
    // the next step's CFL maximum accumulates it here and counts its finished
    // blocks; the last one moves it to smax (with dt32) and clears both
    unsigned long long smax_next;
    unsigned int heat_blocks;
};
constexpr int LAM_VX = 8, LAM_VY = 9;

// scratch planes of the parabolic stages (n doubles each)
// hist (may be null): every LIM iterate is kept there instead of in the
// ping-pong planes -- heat: per outer iteration it, 2 P_it planes
// (T_it, alpha_it, v^1 .. v^{2P_it - 2}); viscous: u^1 .. u^{2P-2}, w^1 .. w^{2P-2}
struct HeatScratch {
    double *T0, *V, *L, *va, *vb, *Ti, *Ai, *Ia;  // Ia = a1 I1 + a2 I2 (external source)
    double *hist;
    double *Lfx, *Lfy;  // face means of Lam at the face after each cell along x, y
    double *tV, *tf;    // tau V and tau (V Ia) of each cell (the LIM sweeps' coefficients)
};
// planes of the viscous stage's per-face values, stored at the face after each cell
enum { VF_FN, VF_FT, VF_W, VF_A1W, VF_A1FN, VF_A1FT, VF_A2W, VF_A2FN, VF_A2FT, VF_N };
struct ViscScratch {
    double *V, *A2, *u0, *w0, *ua, *ub, *wa, *wb;
    double *hist;
    double *LN, *LM;  // face coefficients 4/3 mu_f and mu_f
    double *F;        // VF_N face planes of the conservative last sweep
    double *tV;       // tau V of each cell
};
constexpr int SCRATCH_PLANES = 8 + 2 + VF_N + 1;  // parabolic scratch of a context

__device__ __forceinline__ double dmax_bits(unsigned long long b) { return __longlong_as_double((long long)b); }

__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ void flag(Scalars *sc, unsigned bits)
{
    if (bits) atomicOr(&sc->status, bits);
}

// ---------------------------------------------------------------------------
// IEEE-754 ordering decided on the integer pipe.  On GB300 an FP64 compare or
// min/max issues on the same narrow FP64 pipe as the arithmetic (one warp
// instruction per 64 cycles per scheduler); these take the same decisions as
// the IEEE comparisons (NaN compares false, -0 == +0) from the bit patterns.
// ---------------------------------------------------------------------------
constexpr long long kAbsMask = 0x7FFFFFFFFFFFFFFFLL, kInfBits = 0x7FF0000000000000LL;
__device__ __forceinline__ long long bits_of(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool nan_i(double x) { return (bits_of(x) & kAbsMask) > kInfBits; }
__device__ __forceinline__ bool gt0_i(double x)  // x > 0
{
    long long b = bits_of(x);
    return b > 0 && b <= kInfBits;
}
__device__ __forceinline__ bool ge0_i(double x)  // x >= 0
{
    long long b = bits_of(x);
    return (b >= 0 && b <= kInfBits) || b == LLONG_MIN;
}
__device__ __forceinline__ bool lt0_i(double x)  // x < 0
{
    long long b = bits_of(x), m = b & kAbsMask;
    return b < 0 && m != 0 && m <= kInfBits;
}
__device__ __forceinline__ bool le0_i(double x)  // x <= 0
{
    long long b = bits_of(x);
    return (b < 0 && (b & kAbsMask) <= kInfBits) || b == 0;
}
// key monotone in the value, -0 and +0 both 0
__device__ __forceinline__ long long okey(double x)
{
    long long b = bits_of(x);
    return b >= 0 ? b : (LLONG_MIN - b);
}
__device__ __forceinline__ bool lt_i(double x, double y)  // x < y
{
    return !nan_i(x) && !nan_i(y) && okey(x) < okey(y);
}

// ---------------------------------------------------------------------------
// Stiffened gas (Eqs. eos_stiffened, eos_stiffened2 with q_k = 0)
// ---------------------------------------------------------------------------
// p_k = (gamma_k - 1) E_k / alpha_k - gamma_k pinf_k, E_k = alpha_k rho_k e_k
__device__ __forceinline__ double sg_p(const DevParams &p, int k, double Ek, double ak)
{
    return p.gm1[k] * Ek / ak - p.gpinf[k];
}
// E_k = alpha_k (p + gamma_k pinf_k) / (gamma_k - 1)
__device__ __forceinline__ double sg_E(const DevParams &p, int k, double pr, double ak)
{
    return ak * (pr + p.gpinf[k]) * p.inv_gm1[k];
}
// minmod(a, b): the smaller-magnitude argument when both have the same sign and
// neither is zero, else 0 -- decided on the integer pipe (same result as the
// IEEE comparisons, NaN gives 0)
__device__ __forceinline__ double minmod(double a, double b)
{
    long long ia = bits_of(a), ib = bits_of(b);
    long long ma = ia & kAbsMask, mb = ib & kAbsMask;
    bool same = (ia ^ ib) >= 0 && ma != 0 && mb != 0 && ma <= kInfBits && mb <= kInfBits;
    return same ? (ma < mb ? a : b) : 0.0;
}

// A_k = rho_k c_k^2 = gamma_k (p_k + pinf_k)  (Eq. AK)
__device__ __forceinline__ double sg_A(const DevParams &p, int k, double pr) { return p.g[k] * (pr + p.pinf[k]); }

// mixture sound speed c^2 = Y1 c1^2 + Y2 c2^2 (Sec. 3.1) = (a1 A1 + a2 A2) / rho
__device__ __forceinline__ double mix_c(const DevParams &p, double a1, double p1, double a2, double p2, double rho)
{
    return sqrt((a1 * sg_A(p, 0, p1) + a2 * sg_A(p, 1, p2)) / rho);
}

__device__ __forceinline__ double cell_c(const DevParams &p, double m1, double m2, double E1, double E2, double a2)
{
    double a1 = 1.0 - a2;
    double p1 = sg_p(p, 0, E1, a1), p2 = sg_p(p, 1, E2, a2);
    return mix_c(p, a1, p1, a2, p2, m1 + m2);
}

// conductivity lambda_k(T) = k0_k (T / T_ref)^k_exp
__device__ __forceinline__ double cond(const DevParams &p, int k, double T)
{
    if (p.k_pow == 0) return p.k0[k];
    double t = T * p.inv_Tref;
    if (p.k_pow > 0) {
        double r = t;
        for (int i = 1; i < p.k_pow; i++) r = r * t;
        return p.k0[k] * r;
    }
    return p.k0[k] * pow(t, p.k_exp);
}

// end-of-step admissibility: alpha in (0,1), m_k > 0, p_k + pinf_k > 0, no NaN.
// With alpha_k > 0, p_k + pinf_k = (gamma_k - 1)(E_k - alpha_k pinf_k)/alpha_k > 0
// is tested as E_k > alpha_k pinf_k (no division).
__device__ __forceinline__ unsigned check_state(const DevParams &p, const double *q)
{
    unsigned st = 0;
    double a2 = q[7], a1 = 1.0 - a2;
    if (!(gt0_i(a2) && lt_i(a2, 1.0) && gt0_i(q[0]) && gt0_i(q[1]) && lt_i(a1 * p.pinf[0], q[4]) &&
          lt_i(a2 * p.pinf[1], q[5])))
        st |= DIM_ST_NONPHYS;
#pragma unroll
    for (int k = 0; k < NQ; k++)
        if (nan_i(q[k])) st |= DIM_ST_NAN;
    return st;
}

// ---------------------------------------------------------------------------
// Pressure relaxation, Sec. 3.3 (three steps), on one cell in place.
// q in the global plane order.  Returns DIM_ST_* bits of inadmissible results.
// ---------------------------------------------------------------------------
// Step (1): with p_I the relaxed pressure, dE_k = -p da_k and the EOS give
// a_k(p) = (A_k + B_k p) / (gamma_k (p + pinf_k)), A_k = (g_k-1) E_k^0,
// B_k = (g_k-1) a_k^0; a_1(p) + a_2(p) = 1 is a quadratic whose larger root is
// the unique one with p + pinf_k > 0.  Step (2): p from the mixture energy.
// Step (3): E_k = E_k(p, a_k).
__device__ __forceinline__ unsigned prelax(const DevParams &p, double *q)
{
    const double g1 = p.g[0], g2 = p.g[1];
    double a2 = q[7], a1 = 1.0 - a2;
    double ak1 = p.gm1[0] * q[4], bk1 = p.gm1[0] * a1, ek1 = p.gpinf[0];
    double ak2 = p.gm1[1] * q[5], bk2 = p.gm1[1] * a2, ek2 = p.gpinf[1];
    double A = g1 * g2 - bk1 * g2 - bk2 * g1;
    double B = g1 * ek2 + ek1 * g2 - (ak1 * g2 + bk1 * ek2 + ak2 * g1 + bk2 * ek1);
    double C = ek1 * ek2 - ak1 * ek2 - ak2 * ek1;
    double disc = B * B - 4.0 * A * C;
    unsigned st = 0;
    if (lt0_i(disc)) { st |= DIM_ST_NOROOT; disc = 0.0; }
    double sq = sqrt(disc);
    double pr = le0_i(B) ? (sq - B) / (2.0 * A) : (2.0 * C) / (-B - sq);
    double a2n = (ak2 + bk2 * pr) / (g2 * pr + ek2);
    double a1n = 1.0 - a2n;
    double rho = q[0] + q[1];
    double rhoe = q[6] - 0.5 * (q[2] * q[2] + q[3] * q[3]) / rho;
    double p2 = (rhoe - (a1n * p.g[0] * p.pinf[0] * p.inv_gm1[0] + a2n * p.g[1] * p.pinf[1] * p.inv_gm1[1])) /
                (a1n * p.inv_gm1[0] + a2n * p.inv_gm1[1]);
    q[4] = sg_E(p, 0, p2, a1n);
    q[5] = sg_E(p, 1, p2, a2n);
    q[7] = a2n;
    if (!(gt0_i(a2n) && lt_i(a2n, 1.0) && gt0_i(q[0]) && gt0_i(q[1]) && gt0_i(p2 + p.pinf[0]) &&
          gt0_i(p2 + p.pinf[1])))
        st |= DIM_ST_NONPHYS;
    if (nan_i(p2) || nan_i(a2n)) st |= DIM_ST_NAN;
    return st;
}

// ---------------------------------------------------------------------------
// p,T equilibrium at fixed m_k and rho e (Sec. 3.4.1 end state; Sec. 3.4.2
// projection).  With E_k = C_k T + a_k pinf_k: rho e = C T + pinf_1 - B1 a and
// p1 = p2:  G1C1 T/(1-a) - G2C2 T/a = B1; eliminating T,
//   qa a^2 + qb a + qc = 0, qa = B1 (G + C), qb = E G - B1 G2C2 - C B1,
//   qc = -E G2C2, E = rho e - pinf_1;  admissible root (sqrt(d) - qb)/(2 qa).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned equilibrium(const DevParams &p, double m1, double m2, double rhoe, double &T,
                                                double &a)
{
    double C1 = m1 * p.cv[0], C2 = m2 * p.cv[1], C = C1 + C2;
    double G1C1 = p.gm1[0] * C1, G2C2 = p.gm1[1] * C2, G = G1C1 + G2C2;
    double B1 = p.pinf[0] - p.pinf[1];
    double E = rhoe - p.pinf[0];
    double qa = B1 * (G + C);
    double qb = E * G - B1 * G2C2 - C * B1;
    double qc = -E * G2C2;
    double disc = qb * qb - 4.0 * qa * qc;
    unsigned st = 0;
    if (lt0_i(disc)) { st |= DIM_ST_NOROOT; disc = 0.0; }
    double sq = sqrt(disc);
    a = gt0_i(qb) ? (-2.0 * qc) / (qb + sq) : (sq - qb) / (2.0 * qa);
    T = (E + B1 * a) / C;
    if (!(gt0_i(a) && lt_i(a, 1.0) && gt0_i(T))) st |= DIM_ST_NONPHYS;
    if (nan_i(a) || nan_i(T)) st |= DIM_ST_NAN;
    return st;
}

// The implicit discretization of the relaxation ODEs, Eqs. ht_eq2_TR_dis and
// ht_eq3_TR_dis, in the unknowns (T', a'):
//   B2 C1 (T' - T1^0) + (B1 + B2) C2 (T' - T2^0) = 0,  C2 (T' - T2^0) + B2 (a' - a^0) = 0,
// B2 from Eq. B2_2 at the averages T_k^av = (T_k^0 + T')/2, a^av = (a^0 + a')/2,
// taken as pinf_2 minus the fraction (differentiating p1 = p2 at fixed m_k and
// total energy fixes that sign; the printed form adds pinf_2).  p.trelax_iters
// simple iterations from T' = Eq. Taverage, a' = a^0; each iterate conserves
// C T' + pinf_1 - B1 a' exactly.
__device__ __forceinline__ unsigned trelax_midpoint(const DevParams &p, double m1, double m2, double E1, double E2,
                                                    double a0, double &T, double &a)
{
    const double C1 = m1 * p.cv[0], C2 = m2 * p.cv[1];
    const double G1 = p.gm1[0], G2 = p.gm1[1];
    const double B1 = p.pinf[0] - p.pinf[1];
    // phase temperatures before the stage: E_k = C_k T_k + a_k pinf_k
    const double T10 = (E1 - (1.0 - a0) * p.pinf[0]) / C1;
    const double T20 = (E2 - a0 * p.pinf[1]) / C2;
    double Tp = (C1 * T10 + C2 * T20) / (C1 + C2);
    double ap = a0;
    for (int it = 0; it < p.trelax_iters; it++) {
        double T1a = 0.5 * (T10 + Tp), T2a = 0.5 * (T20 + Tp);
        double a2a = 0.5 * (a0 + ap), a1a = 1.0 - a2a;
        double num = G1 * C1 * T1a / (a1a * a1a) + G1 * p.pinf[0] / a1a + G2 * C2 * T2a / (a2a * a2a) +
                     G2 * p.pinf[1] / a2a;
        double den = G1 / a1a + G2 / a2a;
        double B2 = p.pinf[1] - num / den;
        Tp = (B2 * C1 * T10 + (B1 + B2) * C2 * T20) / (B2 * C1 + (B1 + B2) * C2);
        ap = a0 - C2 * (Tp - T20) / B2;
    }
    T = Tp;
    a = ap;
    unsigned st = 0;
    if (!(gt0_i(ap) && lt_i(ap, 1.0) && gt0_i(Tp))) st |= DIM_ST_NONPHYS;
    if (nan_i(ap) || nan_i(Tp)) st |= DIM_ST_NAN;
    return st;
}

// the temperature-relaxation stage of one cell: (T, a) from the phase energies
__device__ __forceinline__ unsigned trelax_cell(const DevParams &p, double m1, double m2, double E1, double E2,
                                                double a0, double &T, double &a)
{
    if (p.trelax == DIM_TRELAX_MIDPOINT) return trelax_midpoint(p, m1, m2, E1, E2, a0, T, a);
    return equilibrium(p, m1, m2, E1 + E2, T, a);
}

// mixture temperature of a cell in thermal equilibrium (energy form of Eq. Taverage)
__device__ __forceinline__ double mixture_T(const DevParams &p, double m1, double m2, double E1, double E2, double a2)
{
    double C = m1 * p.cv[0] + m2 * p.cv[1];
    return (E1 + E2 - (1.0 - a2) * p.pinf[0] - a2 * p.pinf[1]) / C;
}

// conduction coefficients at (T, a): V = dT/d(rho e) = 1/(C + B1^2/K),
// K = T sum_k (p + pinf_k)/a_k = T^2 sum_k G_k C_k / a_k^2, and Lam = sum_k a_k lambda_k(T)
__device__ __forceinline__ void heat_coeffs(const DevParams &p, double m1, double m2, double T, double a2, double &V,
                                            double &Lam)
{
    double a1 = 1.0 - a2;
    double C1 = m1 * p.cv[0], C2 = m2 * p.cv[1];
    double B1 = p.pinf[0] - p.pinf[1];
    double r1 = p.gm1[0] * C1 * T / (a1 * a1);
    double r2 = p.gm1[1] * C2 * T / (a2 * a2);
    double K = T * (r1 + r2);
    V = 1.0 / (C1 + C2 + B1 * B1 / K);
    Lam = a1 * cond(p, 0, T) + a2 * cond(p, 1, T);
}

// U = d alpha / d(rho e) = -B1 V / K on the equilibrium manifold at (T, a), for
// the V that heat_coeffs gives there (Eq. ht_eq3_ht, linear update)
__device__ __forceinline__ double heat_U(const DevParams &p, double m1, double m2, double T, double a2, double V)
{
    double a1 = 1.0 - a2;
    double C1 = m1 * p.cv[0], C2 = m2 * p.cv[1];
    double B1 = p.pinf[0] - p.pinf[1];
    double r1 = p.gm1[0] * C1 * T / (a1 * a1);
    double r2 = p.gm1[1] * C2 * T / (a2 * a2);
    double K = T * (r1 + r2);
    return -(B1 * V) / K;
}

// ---------------------------------------------------------------------------
// Chebyshev local-iteration parameters (Sec. 3.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cheb_P(const DevParams &p, double tau, double lam, unsigned &capped)
{
    int pf = (int)ceil(3.14159265358979323846 / 4.0 * sqrt(tau * lam + 1.0));
    capped = 0;
    if (p.p_policy == DIM_P_FIXED) return p.p_fixed;
    int P = pf;
    if (p.p_policy == DIM_P_CLAMP && P < p.p_min) P = p.p_min;
    if (P > p.p_max) P = p.p_max;
    if (P < pf) capped = DIM_ST_PCAP;
    return P;
}

// P of the viscous solve: the formula capped at p_max (fixed / clamped stage
// counts belong to the heat-conduction solve)
__device__ __forceinline__ int cheb_P_visc(const DevParams &p, double tau, double lam, unsigned &capped)
{
    int pf = (int)ceil(3.14159265358979323846 / 4.0 * sqrt(tau * lam + 1.0));
    int P = pf > p.p_max ? p.p_max : pf;
    capped = P < pf ? DIM_ST_PCAP : 0u;
    return P;
}

// b_1..b_{2P-1} = (a_P..a_2, a_P..a_1), a_m = lam (beta_1 - beta_m)/(1 + beta_1),
// beta_m = cos((2m-1) pi/(2P)) in decreasing order.  One entry per thread of a block.
__device__ __forceinline__ void cheb_schedule_block(const DevParams &p, int P, double lam, double *sb)
{
    const double *beta = p.beta + (P - 1) * PMAX;
    double beta1 = beta[0];
    for (int s = threadIdx.x; s < 2 * P - 1; s += blockDim.x) {
        int m = s < P - 1 ? P - s : 2 * P - 1 - s;  // index of a_m used at position s
        sb[s] = lam * (beta1 - beta[m - 1]) / (1.0 + beta1);
    }
}

// ---------------------------------------------------------------------------
// Bounded grid barrier for cooperative launches.  All blocks of the grid are
// co-resident (cudaLaunchCooperativeKernel), so the wait ends; a wait that
// exceeds ~2e9 cycles sets DIM_ST_TIMEOUT and returns false, and the caller
// leaves the kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// Bounded wait while *word == value: false after limit SM clock cycles.
constexpr long long kWaitLimit = 2000000000LL;  // ~1 s at 2 GHz
__device__ __forceinline__ bool wait_while_equal(const unsigned *word, unsigned value, long long limit)
{
    const long long t0 = clock64();
    while (ld_acquire_u32(word) == value) {
        __nanosleep(40);
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ bool grid_barrier(Scalars *sc)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_u32(&sc->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&sc->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&sc->bar_count, 0u);
            __threadfence();
            atomicAdd(&sc->bar_gen, 1u);
        } else if (!wait_while_equal(&sc->bar_gen, gen, kWaitLimit)) {
            atomicOr(&sc->status, DIM_ST_TIMEOUT);
            ok = 0;
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// block-wide max of a non-negative double into an accumulator
__device__ __forceinline__ void block_max_to(unsigned long long *acc, double v)
{
    __shared__ double s_w[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        double x = l < nw ? s_w[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (l == 0) atomic_max_pos(acc, x);
    }
}

// ---------------------------------------------------------------------------
// stencil neighbourhood of a cell and reading a device accumulator
// ---------------------------------------------------------------------------
// cell (i, j) of index c and its neighbours with the boundary rule; returns -1
// for a transmissive wall (no flux through that face)
struct Nb {
    int xm, xp, ym, yp;
};

__device__ __forceinline__ Nb neighbours(const DevParams &p, int c)
{
    Nb r;
    int j = c / p.nx, i = c - j * p.nx;
    r.xm = r.xp = r.ym = r.yp = -1;
    if (p.nx > 1) {
        if (i > 0) r.xm = c - 1;
        else if (p.bc[0] == DIM_BC_PERIODIC) r.xm = c + p.nx - 1;
        if (i < p.nx - 1) r.xp = c + 1;
        else if (p.bc[0] == DIM_BC_PERIODIC) r.xp = c - (p.nx - 1);
    }
    if (p.ny > 1) {
        if (j > 0) r.ym = c - p.nx;
        else if (p.bc[1] == DIM_BC_PERIODIC) r.ym = c + (p.ny - 1) * p.nx;
        if (j < p.ny - 1) r.yp = c + p.nx;
        else if (p.bc[1] == DIM_BC_PERIODIC) r.yp = c - (p.ny - 1) * p.nx;
    }
    return r;
}

__device__ __forceinline__ double read_acc(const unsigned long long *a)
{
    unsigned long long v = *(volatile const unsigned long long *)a;
    return dmax_bits(v);
}

}  // namespace dimk

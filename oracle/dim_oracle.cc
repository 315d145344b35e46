/*
 * dim_oracle.cc -- plain FP64 CPU oracle of the split time step of the reduced
 * two-temperature Baer-Nunziato (six-equation) model of Zhang, Menshov, Wang &
 * Shen, "Diffuse interface relaxation model for two-phase compressible flows
 * with diffusion processes" (arXiv:2106.00282).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement that the CUDA path is checked against.  Only tests/, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every stage follows the paper's order and notation, one loop over cells or
 * faces per formula, no blocking and no fusion:
 *   - stiffened-gas EOS, Eqs. (eos_stiffened), (eos_stiffened2), q_k = 0;
 *   - mixture sound speed c^2 = Y1 c1^2 + Y2 c2^2 (Sec. 3.1);
 *   - vector form U, F = uU + (a1p1+a2p2)D, R (Eq. vectorForm);
 *   - Godunov/HLLC update with the non-conservative R term (Sec. 3.1),
 *     dimensional splitting;
 *   - PVT-consistent MUSCL: one homogeneous limiter (minmod) for alpha_2 and
 *     alpha_k rho_k (Sec. 3.6, Eqs. rhostar_high1/2, rec_scheme1/2);
 *   - viscous step by the local-iteration method (Sec. 3.2);
 *   - pressure relaxation in the three steps of Sec. 3.3;
 *   - temperature relaxation (Sec. 3.4.1) as the exact p,T-equilibrium;
 *   - heat conduction by Algorithm 1 with the Chebyshev local-iteration
 *     method, Eqs. (LIM), (LIM_last), (ht_eq2_ht), (qk_dis).
 * Where the paper is silent or inconsistent the reading taken is stated at the
 * point of use (sign of B2, Chebyshev root order, sign of L_h, face
 * coefficients, v^(0), ...).
 *
 * The stage arithmetic is written once, as templates over the scalar type R:
 *   R = double  is the oracle itself (every exported orc_* entry point);
 *   R = Dual    (a value and one tangent component, forward-mode
 *               differentiation) gives the exact tangent-linear map of the same
 *               operations, orc_step_tangent.  Branches (limiters, HLLC wave
 *               regions, Davis bounds) follow the value; the CFL time step and
 *               every Chebyshev lambda_max are taken from the value only (frozen),
 *               so the tangent is that of the map with the step's schedule held
 *               fixed.
 * A Dual's value part goes through exactly the operations a double would, so
 * the value of a tangent run equals the oracle bit for bit.
 *
 * State layout: 8 planes of nx*ny doubles, cell (i,j) at j*nx+i, planes
 *   0 m1 = a1 rho1, 1 m2 = a2 rho2, 2 rho u, 3 rho v,
 *   4 E1 = a1 rho1 e1, 5 E2 = a2 rho2 e2, 6 rho E, 7 alpha_2.
 * Phase 1 is the dense phase (liquid / solid), phase 2 the gas.
 *
 * Schedule record of one step (ORC_SCHED doubles): [0] S, the CFL maximum of
 * (|u_d| + c)/h_d (dt = cfl/S); [1..8] lambda_max of the heat solves of outer
 * iterations 0..7; [9], [10] lambda_max of the viscous solves along x and y.
 *
 * Build: g++ -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * oracle rounds every operation exactly as written).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

#define NQ 8
#define ORC_PI 3.14159265358979323846
#define ORC_SCHED 11

/* status bits returned by every entry point (0 = fine) */
#define ORC_NONPHYS 1u /* alpha outside (0,1), m_k <= 0, p+pinf <= 0, T <= 0 */
#define ORC_NAN 2u
#define ORC_NOROOT 4u
#define ORC_TRANSIENT 8u /* a relaxation stage met an inadmissible phase state that a later stage of the
                          * same step repaired (e.g. the first step at a sharp interface); not an error */
#define ORC_PCAP 32u /* the formula asked for more than p_max Chebyshev parameters; P = p_max used */
#define ORC_EINVAL 64u

extern "C" {
typedef struct {
    double gamma[2], pinf[2], cv[2];
    double k0[2], k_exp, T_ref; /* lambda_k(T) = k0_k (T/T_ref)^k_exp */
    double mu[2];
    double cfl;
    int limiter;  /* 0: first order, 1: minmod MUSCL, 2: Overbee on alpha_2 and alpha_k rho_k with minmod
                   * on u and p_k, 3: Overbee on alpha_2 only (the inconsistent combination of Sec. 4.1) */
    int bc[2];    /* per axis: 0 transmissive, 1 periodic */
    int trelax;   /* 0: off (no T relaxation, no conduction), 1: exact equilibrium, 2: the implicit midpoint
                   * scheme of Sec. 3.4.1 with trelax_iters simple iterations */
    int n_outer;  /* outer iterations of Algorithm 1 */
    int p_policy; /* 0: P by formula, 1: fixed p_fixed, 2: clamp(formula, p_min, p_max) */
    int p_fixed, p_min, p_max;
    int precision; /* unused: the oracle is FP64 */
    double src[2]; /* external heat source intensities I_k, I_k = alpha_k I_k (Eq. I) */
    int heat_alpha;   /* heat stage (T, alpha) update: 0 projection onto the equilibrium manifold,
                       * 1 linear, T += tau V (L_h u_hat + I), alpha += tau U (L_h u_hat + I) */
    int trelax_iters; /* simple iterations of the midpoint temperature relaxation (trelax 2) */
} orc_params;
}

/* ------------------------------------------------------------------------- */
/* Forward-mode dual numbers: (value, tangent), the rules of differentiation. */
/* ------------------------------------------------------------------------- */
template <typename B>
struct DualT {
    B v, d;
    DualT() = default;
    DualT(B x) : v(x), d(0) {}
    DualT(B x, B t) : v(x), d(t) {}
    friend DualT operator+(DualT a, DualT b) { return DualT(a.v + b.v, a.d + b.d); }
    friend DualT operator-(DualT a, DualT b) { return DualT(a.v - b.v, a.d - b.d); }
    friend DualT operator-(DualT a) { return DualT(-a.v, -a.d); }
    /* d(ab) = a db + b da */
    friend DualT operator*(DualT a, DualT b) { return DualT(a.v * b.v, a.d * b.v + a.v * b.d); }
    /* d(a/b) = (da - (a/b) db) / b */
    friend DualT operator/(DualT a, DualT b)
    {
        B q = a.v / b.v;
        return DualT(q, (a.d - q * b.d) / b.v);
    }
    friend DualT &operator+=(DualT &a, DualT b) { a = a + b; return a; }
    friend DualT &operator-=(DualT &a, DualT b) { a = a - b; return a; }
    friend bool operator<(DualT a, DualT b) { return a.v < b.v; }
    friend bool operator>(DualT a, DualT b) { return a.v > b.v; }
    friend bool operator<=(DualT a, DualT b) { return a.v <= b.v; }
    friend bool operator>=(DualT a, DualT b) { return a.v >= b.v; }
    /* d sqrt(a) = da / (2 sqrt(a)) */
    friend DualT sqrt(DualT a)
    {
        B s = std::sqrt(a.v);
        return DualT(s, a.d / (B(2) * s));
    }
    friend DualT fabs(DualT a) { return a.v < 0 ? -a : a; }
    friend DualT fmin(DualT a, DualT b) { return b.v < a.v ? b : a; }
    friend DualT fmax(DualT a, DualT b) { return b.v > a.v ? b : a; }
    /* d a^e = e a^(e-1) da for a constant exponent */
    friend DualT pow(DualT a, double e) { return DualT(std::pow(a.v, B(e)), B(e) * std::pow(a.v, B(e) - 1) * a.d); }
    friend double val(DualT x) { return (double)x.v; }
    friend bool is_nan(DualT x) { return std::isnan(x.v); }
};
/* the tangent of the oracle: double values and tangents */
typedef DualT<double> Dual;
/* the same in extended precision (long double), a reference for the
 * rounding error of the double tangent on badly conditioned states */
typedef DualT<long double> DualL;
static inline double val(double x) { return x; }
static inline bool is_nan(double x) { return isnan(x); }

/* Operation counting (test infrastructure): a double that counts the
 * floating-point operations applied to state-dependent values -- + and -,
 * *, /, sqrt, pow; comparisons, min/max, abs and selects are free -- so that
 * running a stage once on it counts the stage's algorithmic work. */
static unsigned long long g_ops[5]; /* add/sub, mul, div, sqrt, pow */
struct Cnt {
    double v;
    Cnt() = default;
    Cnt(double x) : v(x) {}
    friend Cnt operator+(Cnt a, Cnt b) { g_ops[0]++; return Cnt(a.v + b.v); }
    friend Cnt operator-(Cnt a, Cnt b) { g_ops[0]++; return Cnt(a.v - b.v); }
    friend Cnt operator-(Cnt a) { return Cnt(-a.v); }
    friend Cnt operator*(Cnt a, Cnt b) { g_ops[1]++; return Cnt(a.v * b.v); }
    friend Cnt operator/(Cnt a, Cnt b) { g_ops[2]++; return Cnt(a.v / b.v); }
    friend Cnt &operator+=(Cnt &a, Cnt b) { a = a + b; return a; }
    friend Cnt &operator-=(Cnt &a, Cnt b) { a = a - b; return a; }
    friend bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
    friend bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
    friend bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
    friend bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
    friend Cnt sqrt(Cnt a) { g_ops[3]++; return Cnt(std::sqrt(a.v)); }
    friend Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }
    friend Cnt fmin(Cnt a, Cnt b) { return b.v < a.v ? b : a; }
    friend Cnt fmax(Cnt a, Cnt b) { return b.v > a.v ? b : a; }
    friend Cnt pow(Cnt a, double e) { g_ops[4]++; return Cnt(std::pow(a.v, e)); }
    friend double val(Cnt x) { return x.v; }
    friend bool is_nan(Cnt x) { return std::isnan(x.v); }
};

/* Branch record (test infrastructure for derivative checks): every value-decided
 * branch of the sweep -- the operand minmod returns, the Davis min / max, the
 * HLLC wave region -- can be recorded on one run and replayed on another, so
 * that a perturbed run follows the nominal run's branches (the branch-frozen
 * map, whose central differences converge to the tangent).  Off by default. */
static struct {
    int mode; /* 0 off, 1 record, 2 replay */
    unsigned char *buf;
    size_t pos, cap;
    int overflow;
} g_tape;

static int branch(int decided)
{
    if (g_tape.mode == 1) {
        if (g_tape.pos < g_tape.cap) g_tape.buf[g_tape.pos] = (unsigned char)decided;
        else g_tape.overflow = 1;
        g_tape.pos++;
        return decided;
    }
    if (g_tape.mode == 2) {
        if (g_tape.pos < g_tape.cap) return g_tape.buf[g_tape.pos++];
        g_tape.overflow = 1;
    }
    return decided;
}

/* the parameters as the stage arithmetic sees them: the conductivity
 * coefficients, viscosities and source intensities carry the scalar type (so a
 * tangent run can differentiate with respect to them), the rest are constants */
template <typename R>
struct prm {
    double gamma[2], pinf[2], cv[2];
    R k0[2];
    double k_exp, T_ref;
    R mu[2];
    double cfl;
    int limiter, bc[2], trelax, n_outer, p_policy, p_fixed, p_min, p_max;
    R src[2];
    int heat_alpha, trelax_iters;
};

/* dparams (may be NULL): tangents of (k0_1, k0_2, mu_1, mu_2, I_1, I_2) */
template <typename R>
static prm<R> make_prm(const orc_params *P, const double *dparams);

template <>
prm<double> make_prm<double>(const orc_params *P, const double *)
{
    prm<double> q;
    for (int k = 0; k < 2; k++) {
        q.gamma[k] = P->gamma[k]; q.pinf[k] = P->pinf[k]; q.cv[k] = P->cv[k];
        q.k0[k] = P->k0[k]; q.mu[k] = P->mu[k]; q.src[k] = P->src[k]; q.bc[k] = P->bc[k];
    }
    q.k_exp = P->k_exp; q.T_ref = P->T_ref; q.cfl = P->cfl;
    q.limiter = P->limiter; q.trelax = P->trelax; q.n_outer = P->n_outer; q.p_policy = P->p_policy;
    q.p_fixed = P->p_fixed; q.p_min = P->p_min; q.p_max = P->p_max;
    q.heat_alpha = P->heat_alpha; q.trelax_iters = P->trelax_iters;
    return q;
}

template <typename B>
static prm<DualT<B>> make_prm_dual(const orc_params *P, const double *dp)
{
    prm<DualT<B>> q;
    for (int k = 0; k < 2; k++) {
        q.gamma[k] = P->gamma[k]; q.pinf[k] = P->pinf[k]; q.cv[k] = P->cv[k];
        q.k0[k] = DualT<B>(P->k0[k], dp ? dp[k] : 0.0);
        q.mu[k] = DualT<B>(P->mu[k], dp ? dp[2 + k] : 0.0);
        q.src[k] = DualT<B>(P->src[k], dp ? dp[4 + k] : 0.0);
        q.bc[k] = P->bc[k];
    }
    q.k_exp = P->k_exp; q.T_ref = P->T_ref; q.cfl = P->cfl;
    q.limiter = P->limiter; q.trelax = P->trelax; q.n_outer = P->n_outer; q.p_policy = P->p_policy;
    q.p_fixed = P->p_fixed; q.p_min = P->p_min; q.p_max = P->p_max;
    q.heat_alpha = P->heat_alpha; q.trelax_iters = P->trelax_iters;
    return q;
}
template <>
prm<Cnt> make_prm<Cnt>(const orc_params *P, const double *)
{
    prm<Cnt> q;
    for (int k = 0; k < 2; k++) {
        q.gamma[k] = P->gamma[k]; q.pinf[k] = P->pinf[k]; q.cv[k] = P->cv[k];
        q.k0[k] = Cnt(P->k0[k]); q.mu[k] = Cnt(P->mu[k]); q.src[k] = Cnt(P->src[k]);
        q.bc[k] = P->bc[k];
    }
    q.k_exp = P->k_exp; q.T_ref = P->T_ref; q.cfl = P->cfl;
    q.limiter = P->limiter; q.trelax = P->trelax; q.n_outer = P->n_outer; q.p_policy = P->p_policy;
    q.p_fixed = P->p_fixed; q.p_min = P->p_min; q.p_max = P->p_max;
    q.heat_alpha = P->heat_alpha; q.trelax_iters = P->trelax_iters;
    return q;
}

template <>
prm<Dual> make_prm<Dual>(const orc_params *P, const double *dp)
{
    return make_prm_dual<double>(P, dp);
}
template <>
prm<DualL> make_prm<DualL>(const orc_params *P, const double *dp)
{
    return make_prm_dual<long double>(P, dp);
}

/* ------------------------------------------------------------------------- */
/* Thermodynamics: stiffened gas, Eqs. (eos_stiffened), (eos_stiffened2).    */
/* ------------------------------------------------------------------------- */

/* phase pressure from E_k = a_k rho_k e_k:  p_k = (g_k-1) E_k / a_k - g_k pinf_k */
template <typename R>
static R phase_p(const prm<R> *P, int k, R Ek, R ak)
{
    return (P->gamma[k] - 1.0) * Ek / ak - P->gamma[k] * P->pinf[k];
}

/* the material constant 1/(gamma_k - 1) of Eq. (eos_stiffened) */
template <typename R>
static double inv_gm1(const prm<R> *P, int k)
{
    return 1.0 / (P->gamma[k] - 1.0);
}

/* phase energy per mixture volume from (p, a_k): E_k = a_k (p + g pinf)/(g-1) */
template <typename R>
static R phase_E(const prm<R> *P, int k, R p, R ak)
{
    return ak * (p + P->gamma[k] * P->pinf[k]) * inv_gm1(P, k);
}

/* A_k = rho_k c_k^2 = gamma_k (p_k + pinf_k)  (Eq. AK) */
template <typename R>
static R phase_A(const prm<R> *P, int k, R p)
{
    return P->gamma[k] * (p + P->pinf[k]);
}

/* mixture sound speed c^2 = Y1 c1^2 + Y2 c2^2 (Sec. 3.1); with Y_k = a_k rho_k / rho
 * and rho_k c_k^2 = A_k (Eq. AK) this is c^2 = (a1 A1 + a2 A2) / rho */
template <typename R>
static R mixture_c(const prm<R> *P, R a1, R p1, R a2, R p2, R rho)
{
    return sqrt((a1 * phase_A(P, 0, p1) + a2 * phase_A(P, 1, p2)) / rho);
}

/* conductivity law lambda_k(T) = k0_k (T / T_ref)^k_exp */
template <typename R>
static R lambda_k(const prm<R> *P, int k, R T)
{
    R t = T * (1.0 / P->T_ref);
    double e = P->k_exp;
    if (e == 0.0) return P->k0[k];
    if (e == floor(e) && e > 0.0 && e <= 8.0) {
        R r = t;
        for (int n = 1; n < (int)e; n++) r = r * t;
        return P->k0[k] * r;
    }
    return P->k0[k] * pow(t, e);
}

/* ------------------------------------------------------------------------- */
/* Initial data: (alpha_2, p, T, u, v) with both phases at the cell's (p, T). */
/* ------------------------------------------------------------------------- */
extern "C" unsigned orc_from_primitive(const orc_params *Pp, int nx, int ny, const double *prim, double *U)
{
    prm<double> Pv = make_prm<double>(Pp, NULL);
    const prm<double> *P = &Pv;
    int n = nx * ny;
    unsigned st = 0;
    for (int c = 0; c < n; c++) {
        double a2 = prim[0 * n + c], p = prim[1 * n + c], T = prim[2 * n + c];
        double u = prim[3 * n + c], v = prim[4 * n + c];
        double a1 = 1.0 - a2;
        /* Eq. eos_stiffened2 with q = 0: rho_k = (p + pinf_k) / ((g_k - 1) Cv_k T) */
        double rho1 = (p + P->pinf[0]) / ((P->gamma[0] - 1.0) * P->cv[0] * T);
        double rho2 = (p + P->pinf[1]) / ((P->gamma[1] - 1.0) * P->cv[1] * T);
        double m1 = a1 * rho1, m2 = a2 * rho2, rho = m1 + m2;
        double E1 = phase_E(P, 0, p, a1), E2 = phase_E(P, 1, p, a2);
        U[0 * n + c] = m1;
        U[1 * n + c] = m2;
        U[2 * n + c] = rho * u;
        U[3 * n + c] = rho * v;
        U[4 * n + c] = E1;
        U[5 * n + c] = E2;
        U[6 * n + c] = E1 + E2 + 0.5 * rho * (u * u + v * v);
        U[7 * n + c] = a2;
        if (!(a2 > 0.0 && a2 < 1.0 && T > 0.0 && p + P->pinf[0] > 0.0 && p + P->pinf[1] > 0.0))
            st |= ORC_NONPHYS;
    }
    return st;
}

/* ------------------------------------------------------------------------- */
/* Time step from the CFL condition with the mixture sound speed (Sec. 3.1): */
/*   dt = cfl / S,  S = max_cells max_d (|u_d| + c) / h_d  over active axes. */
/* ------------------------------------------------------------------------- */
template <typename R>
static R cell_sound_speed(const prm<R> *P, const R *U, int n, int c)
{
    R m1 = U[0 * n + c], m2 = U[1 * n + c];
    R a2 = U[7 * n + c], a1 = 1.0 - a2;
    R rho = m1 + m2;
    R p1 = phase_p(P, 0, U[4 * n + c], a1);
    R p2 = phase_p(P, 1, U[5 * n + c], a2);
    return mixture_c(P, a1, p1, a2, p2, rho);
}

/* S of a state (a value: the time step is never differentiated) */
template <typename R>
static double wave_max(const prm<R> *P, int nx, int ny, double dx, double dy, const R *U)
{
    int n = nx * ny;
    double smax = 0.0;
    for (int c = 0; c < n; c++) {
        R rho = U[0 * n + c] + U[1 * n + c];
        R cs = cell_sound_speed(P, U, n, c);
        if (nx > 1) {
            double s = val((fabs(U[2 * n + c] / rho) + cs) * (1.0 / dx));
            if (s > smax) smax = s;
        }
        if (ny > 1) {
            double s = val((fabs(U[3 * n + c] / rho) + cs) * (1.0 / dy));
            if (s > smax) smax = s;
        }
    }
    return smax;
}

extern "C" double orc_dt(const orc_params *P, int nx, int ny, double dx, double dy, const double *U)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return P->cfl / wave_max(&Pv, nx, ny, dx, dy, U);
}

/* ------------------------------------------------------------------------- */
/* Hyperbolic sweep along one axis (Sec. 3.1, 3.6).                          */
/* ------------------------------------------------------------------------- */

/* primitive vector W = (alpha_2, m1, m2, u_n, u_t, p1, p2) of a line cell;
 * the line-local conserved order is (m1, m2, rho u_n, rho u_t, E1, E2, rhoE, a2) */
template <typename R>
static void line_prims(const prm<R> *P, const R *q, R *w)
{
    R a2 = q[7], a1 = 1.0 - a2;
    R rho = q[0] + q[1];
    w[0] = a2;
    w[1] = q[0];
    w[2] = q[1];
    w[3] = q[2] / rho;
    w[4] = q[3] / rho;
    w[5] = phase_p(P, 0, q[4], a1);
    w[6] = phase_p(P, 1, q[5], a2);
}

template <typename R>
static R minmod(R a, R b)
{
    int d = 0; /* 0: zero, 1: a, 2: b */
    if (a > 0.0 && b > 0.0) d = a < b ? 1 : 2;
    else if (a < 0.0 && b < 0.0) d = a > b ? 1 : 2;
    d = branch(d);
    return d == 1 ? a : (d == 2 ? b : R(0.0));
}

/* Overbee slope: the limiter phi(r) = max(0, min(2r, 2)) (the upper boundary of
 * the TVD region; the paper cites the limiter without printing it), i.e. twice
 * the minmod slope -- homogeneous of degree 1 like minmod (Sec. 3.6) */
template <typename R>
static R overbee(R a, R b)
{
    return 2.0 * minmod(a, b);
}

template <typename R>
struct face_state {
    R a2, m1, m2, un, ut, rho, p, c;
    R q[NQ]; /* conserved face state, line-local order */
};

/* conserved state and mixture quantities from a reconstructed W */
template <typename R>
static void face_from_w(const prm<R> *P, const R *w, face_state<R> *s)
{
    R a2 = w[0], a1 = 1.0 - a2;
    R m1 = w[1], m2 = w[2], un = w[3], ut = w[4], p1 = w[5], p2 = w[6];
    R rho = m1 + m2;
    R E1 = phase_E(P, 0, p1, a1), E2 = phase_E(P, 1, p2, a2);
    s->a2 = a2; s->m1 = m1; s->m2 = m2; s->un = un; s->ut = ut;
    s->rho = rho;
    s->p = a1 * p1 + a2 * p2;
    s->c = mixture_c(P, a1, p1, a2, p2, rho);
    s->q[0] = m1; s->q[1] = m2;
    s->q[2] = rho * un; s->q[3] = rho * ut;
    s->q[4] = E1; s->q[5] = E2;
    s->q[6] = E1 + E2 + 0.5 * rho * (un * un + ut * ut);
    s->q[7] = a2;
}

/* HLLC solution at xi = x/t = 0 and its flux F(U*) = u* U* + p* D(u*) with
 * D = [0 0 1 0 0 0 u* 0] (Eq. vectorForm).  Davis wave-speed bounds; across the
 * acoustic waves the phase masses and phase energies scale like the density
 * and alpha_2 is unchanged, so an isolated contact is resolved exactly. */
template <typename R>
static void hllc(const face_state<R> *L, const face_state<R> *Rt, R *F, R *ustar)
{
    R sl1 = L->un - L->c, sl2 = Rt->un - Rt->c, sr1 = L->un + L->c, sr2 = Rt->un + Rt->c;
    /* fmin / fmax, the operand recorded */
    R SL = branch(sl2 < sl1 ? 1 : 0) ? sl2 : sl1;
    R SR = branch(sr2 > sr1 ? 1 : 0) ? sr2 : sr1;
    R Ss = (Rt->p - L->p + L->rho * L->un * (SL - L->un) - Rt->rho * Rt->un * (SR - Rt->un)) /
           (L->rho * (SL - L->un) - Rt->rho * (SR - Rt->un));
    R q[NQ], us, ps;
    const face_state<R> *K;
    R SK;
    int region = 0.0 <= SL ? 0 : (0.0 <= SR ? (0.0 <= Ss ? 1 : 2) : 3);
    region = branch(region);
    if (region == 0) {
        for (int k = 0; k < NQ; k++) q[k] = L->q[k];
        us = L->un; ps = L->p;
    } else if (region <= 2) {
        if (region == 1) { K = L; SK = SL; } else { K = Rt; SK = SR; }
        R chi = (SK - K->un) / (SK - Ss);
        q[0] = chi * K->q[0];
        q[1] = chi * K->q[1];
        q[2] = chi * K->rho * Ss;
        q[3] = chi * K->rho * K->ut;
        q[4] = chi * K->q[4];
        q[5] = chi * K->q[5];
        q[6] = chi * (K->q[6] + (Ss - K->un) * (K->rho * Ss + K->p / (SK - K->un)));
        q[7] = K->a2;
        us = Ss;
        ps = K->p + K->rho * (SK - K->un) * (Ss - K->un);
    } else {
        for (int k = 0; k < NQ; k++) q[k] = Rt->q[k];
        us = Rt->un; ps = Rt->p;
    }
    F[0] = us * q[0];
    F[1] = us * q[1];
    F[2] = us * q[2] + ps;
    F[3] = us * q[3];
    F[4] = us * q[4];
    F[5] = us * q[5];
    F[6] = us * (q[6] + ps);
    F[7] = us * q[7];
    *ustar = us;
}

/* one line of n cells, ext holds n+4 cells (2 ghosts per side) in the
 * line-local order, 8 values per cell; out receives the n updated cells */
template <typename R>
static void line_update(const prm<R> *P, int n, double dtdx, const R *ext, R *out)
{
    int ne = n + 4;
    R *W = (R *)malloc(sizeof(R) * 7 * ne);
    R *S = (R *)calloc(7 * ne, sizeof(R));
    R *F = (R *)malloc(sizeof(R) * NQ * (n + 1));
    R *us = (R *)malloc(sizeof(R) * (n + 1));
    for (int e = 0; e < ne; e++) line_prims(P, ext + NQ * e, W + 7 * e);
    /* MUSCL slopes: sigma_e = minmod(W_e - W_{e-1}, W_{e+1} - W_e) on every
     * component of W, the same limiter for alpha_2 and m_k (Sec. 3.6) */
    /* limiter 2: Overbee on alpha_2, m1, m2 (components 0-2), minmod on the rest;
     * limiter 3: Overbee on alpha_2 only */
    if (P->limiter >= 1)
        for (int e = 1; e <= n + 2; e++)
            for (int k = 0; k < 7; k++) {
                R dm = W[7 * e + k] - W[7 * (e - 1) + k], dp = W[7 * (e + 1) + k] - W[7 * e + k];
                int ob = (P->limiter == 2 && k <= 2) || (P->limiter == 3 && k == 0);
                S[7 * e + k] = ob ? overbee(dm, dp) : minmod(dm, dp);
            }
    /* face f (f = 0..n) lies between extended cells f+1 and f+2 */
    for (int f = 0; f <= n; f++) {
        R wl[7], wr[7];
        face_state<R> sl, sr;
        for (int k = 0; k < 7; k++) {
            wl[k] = W[7 * (f + 1) + k] + 0.5 * S[7 * (f + 1) + k];
            wr[k] = W[7 * (f + 2) + k] - 0.5 * S[7 * (f + 2) + k];
        }
        face_from_w(P, wl, &sl);
        face_from_w(P, wr, &sr);
        hllc(&sl, &sr, F + NQ * f, us + f);
    }
    /* Godunov update with the non-conservative term R(U_i^n)(u*_{i+1/2} - u*_{i-1/2}),
     * R = [0 0 0 0 a1p1 a2p2 0 -a2] (Sec. 3.1): only the phase-energy and
     * volume-fraction rows carry it */
    for (int i = 0; i < n; i++) {
        const R *q = ext + NQ * (i + 2);
        const R *w = W + 7 * (i + 2);
        R a2 = w[0], a1 = 1.0 - a2;
        R Rv[NQ] = {R(0.0), R(0.0), R(0.0), R(0.0), a1 * w[5], a2 * w[6], R(0.0), -a2};
        R du = us[i + 1] - us[i];
        for (int k = 0; k < NQ; k++) {
            R v = q[k] - dtdx * (F[NQ * (i + 1) + k] - F[NQ * i + k]);
            if (k == 4 || k == 5 || k == 7) v = v - dtdx * Rv[k] * du;
            out[NQ * i + k] = v;
        }
    }
    free(W); free(S); free(F); free(us);
}

/* ghost index of extended position e (0..n+3) of a line of n cells */
static int ghost_src(int e, int n, int bc)
{
    int i = e - 2;
    if (i >= 0 && i < n) return i;
    if (bc == 1) return ((i % n) + n) % n;
    return i < 0 ? 0 : n - 1;
}

/* one directional sweep (axis 0: x, 1: y) without relaxation */
template <typename R>
static unsigned sweep_t(const prm<R> *P, int nx, int ny, double dx, double dy, int axis, double dt, R *U)
{
    int n = nx * ny;
    int len = axis == 0 ? nx : ny, nlines = axis == 0 ? ny : nx;
    double h = axis == 0 ? dx : dy;
    int qn = axis == 0 ? 2 : 3, qt = axis == 0 ? 3 : 2;
    int map[NQ] = {0, 1, qn, qt, 4, 5, 6, 7};
    R *ext = (R *)malloc(sizeof(R) * NQ * (len + 4));
    R *out = (R *)malloc(sizeof(R) * NQ * len);
    for (int l = 0; l < nlines; l++) {
        for (int e = 0; e < len + 4; e++) {
            int i = ghost_src(e, len, P->bc[axis]);
            int c = axis == 0 ? l * nx + i : i * nx + l;
            for (int k = 0; k < NQ; k++) ext[NQ * e + k] = U[map[k] * n + c];
        }
        line_update(P, len, dt / h, ext, out);
        for (int i = 0; i < len; i++) {
            int c = axis == 0 ? l * nx + i : i * nx + l;
            for (int k = 0; k < NQ; k++) U[map[k] * n + c] = out[NQ * i + k];
        }
    }
    free(ext); free(out);
    return 0;
}

extern "C" unsigned orc_sweep(const orc_params *P, int nx, int ny, double dx, double dy, int axis, double dt,
                              double *U)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return sweep_t(&Pv, nx, ny, dx, dy, axis, dt, U);
}

/* ------------------------------------------------------------------------- */
/* Instantaneous pressure relaxation, the three steps of Sec. 3.3.           */
/* ------------------------------------------------------------------------- */
/* (1) with p_I equal to the relaxed pressure p, dE_k = -p da_k and the SG EOS
 *     give a_k(p) = (g_k-1)(E_k^0 + p a_k^0) / (g_k (p + pinf_k)); the
 *     saturation sum a_1(p) + a_2(p) = 1 is a quadratic A p^2 + B p + C = 0
 *     whose larger root is the unique one with p + pinf_k > 0 for both k;
 * (2) p2 = p(a^(1), rho e) from the mixture energy rho e = rho E - |rho u|^2/(2 rho);
 * (3) E_k = E_k(p2, a_k^(1)). */
template <typename R>
static unsigned prelax_cell(const prm<R> *P, R *U, int n, int c)
{
    unsigned st = 0;
    double g1 = P->gamma[0], g2 = P->gamma[1], pi1 = P->pinf[0], pi2 = P->pinf[1];
    R m1 = U[0 * n + c], m2 = U[1 * n + c];
    R a2 = U[7 * n + c], a1 = 1.0 - a2;
    R E1 = U[4 * n + c], E2 = U[5 * n + c];
    /* a_k(p) = (ak + bk p) / (dk p + ek) */
    R ak1 = (g1 - 1.0) * E1, bk1 = (g1 - 1.0) * a1;
    double dk1 = g1, ek1 = g1 * pi1;
    R ak2 = (g2 - 1.0) * E2, bk2 = (g2 - 1.0) * a2;
    double dk2 = g2, ek2 = g2 * pi2;
    R A = dk1 * dk2 - bk1 * dk2 - bk2 * dk1;
    R B = dk1 * ek2 + ek1 * dk2 - (ak1 * dk2 + bk1 * ek2 + ak2 * dk1 + bk2 * ek1);
    R C = ek1 * ek2 - ak1 * ek2 - ak2 * ek1;
    R disc = B * B - 4.0 * A * C;
    if (disc < 0.0) { st |= ORC_NOROOT; disc = 0.0; }
    R sq = sqrt(disc);
    R p = B <= 0.0 ? (sq - B) / (2.0 * A) : (2.0 * C) / (-B - sq);
    R a2n = (ak2 + bk2 * p) / (dk2 * p + ek2);
    R a1n = 1.0 - a2n;
    /* step (2): pressure from the conservative mixture energy */
    R rho = m1 + m2;
    R mu = U[2 * n + c], mv = U[3 * n + c];
    R rhoe = U[6 * n + c] - 0.5 * (mu * mu + mv * mv) / rho;
    double i1 = inv_gm1(P, 0), i2 = inv_gm1(P, 1);
    R p2 = (rhoe - (a1n * g1 * pi1 * i1 + a2n * g2 * pi2 * i2)) / (a1n * i1 + a2n * i2);
    /* step (3) */
    U[4 * n + c] = phase_E(P, 0, p2, a1n);
    U[5 * n + c] = phase_E(P, 1, p2, a2n);
    U[7 * n + c] = a2n;
    if (!(a2n > 0.0 && a2n < 1.0 && m1 > 0.0 && m2 > 0.0 && p2 + pi1 > 0.0 && p2 + pi2 > 0.0))
        st |= ORC_NONPHYS;
    if (is_nan(p2) || is_nan(a2n)) st |= ORC_NAN;
    return st;
}

template <typename R>
static unsigned prelax_t(const prm<R> *P, int ncell, R *U)
{
    unsigned st = 0;
    for (int c = 0; c < ncell; c++) st |= prelax_cell(P, U, ncell, c);
    return st;
}

extern "C" unsigned orc_prelax(const orc_params *P, int ncell, double *U)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return prelax_t(&Pv, ncell, U);
}

/* ------------------------------------------------------------------------- */
/* Temperature relaxation (Sec. 3.4.1): exact p,T equilibrium.              */
/* ------------------------------------------------------------------------- */
/* At fixed m_k (C_k = m_k Cv_k) and fixed rho e the SG phase energies are
 * E_k = C_k T_k + a_k pinf_k, so with T1 = T2 = T
 *   rho e = C T + pinf_1 - B1 alpha,  C = C1 + C2,  B1 = pinf_1 - pinf_2,
 * and p1 = p2 reads  G1 C1 T/(1-alpha) - G2 C2 T/alpha = B1  (G_k = g_k - 1).
 * Eliminating T gives  qa alpha^2 + qb alpha + qc = 0 with
 *   qa = B1 (G + C), qb = E G - B1 G2C2 - C B1, qc = -E G2C2,
 *   G = G1C1 + G2C2, E = rho e - pinf_1;
 * the admissible root (alpha in (0,1), T > 0) is (sqrt(disc) - qb)/(2 qa) for
 * either sign of qa, evaluated without cancellation.  This is the state the
 * relaxation ODEs (ht_eq2_TR), (ht_eq3_TR) drive to, with B2 taken with the
 * sign that keeps p1 = p2 along the path (B2 = pinf_2 - p/r0). */
template <typename R>
static unsigned equilibrium(const prm<R> *P, R m1, R m2, R rhoe, R *T, R *a2)
{
    R C1 = m1 * P->cv[0], C2 = m2 * P->cv[1], C = C1 + C2;
    R G1C1 = (P->gamma[0] - 1.0) * C1, G2C2 = (P->gamma[1] - 1.0) * C2, G = G1C1 + G2C2;
    double B1 = P->pinf[0] - P->pinf[1];
    R E = rhoe - P->pinf[0];
    R qa = B1 * (G + C);
    R qb = E * G - B1 * G2C2 - C * B1;
    R qc = -E * G2C2;
    R disc = qb * qb - 4.0 * qa * qc;
    unsigned st = 0;
    if (disc < 0.0) { st |= ORC_NOROOT; disc = 0.0; }
    R sq = sqrt(disc);
    R a = qb > 0.0 ? (-2.0 * qc) / (qb + sq) : (sq - qb) / (2.0 * qa);
    *a2 = a;
    *T = (E + B1 * a) / C;
    if (!(a > 0.0 && a < 1.0 && *T > 0.0)) st |= ORC_NONPHYS;
    if (is_nan(a) || is_nan(*T)) st |= ORC_NAN;
    return st;
}

/* mixture temperature of a cell in thermal equilibrium, from the energy:
 * rho e = C T + a1 pinf_1 + a2 pinf_2  (Eq. Taverage with T1 = T2) */
template <typename R>
static R cell_T(const prm<R> *P, const R *U, int n, int c)
{
    R a2 = U[7 * n + c], a1 = 1.0 - a2;
    R C = U[0 * n + c] * P->cv[0] + U[1 * n + c] * P->cv[1];
    return (U[4 * n + c] + U[5 * n + c] - a1 * P->pinf[0] - a2 * P->pinf[1]) / C;
}

/* The paper's own discretization of the relaxation ODEs (ht_eq2_TR),
 * (ht_eq3_TR): Eqs. (ht_eq2_TR_dis), (ht_eq3_TR_dis), unknowns (T', a2'),
 *   B2 C1 (T' - T1^0) + (B1 + B2) C2 (T' - T2^0) = 0,
 *   C2 (T' - T2^0) + B2 (a2' - a2^0) = 0,
 * B2 evaluated at the averages T_k^av = (T_k^0 + T')/2, a2^av = (a2^0 + a2')/2.
 * B2 is Eq. (B2_2) with the sign that keeps dp1 = dp2 along the path (the
 * printed form adds pinf_2 to the fraction; differentiating p1 = p2 at fixed
 * m_k and fixed total energy subtracts it from pinf_2):
 *   B2 = pinf_2 - [G1 C1 T1/a1^2 + G1 pinf_1/a1 + G2 C2 T2/a2^2 + G2 pinf_2/a2]
 *                 / [G1/a1 + G2/a2],   G_k = g_k - 1 (Grueneisen, SG).
 * The system is solved by simple iteration, a fixed number of times, from
 * T' = Eq. (Taverage), a2' = a2^0.  Every iterate satisfies both equations for
 * its B2, so the total energy C T' + pinf_1 - B1 a2' is conserved whatever the
 * count; with pinf_1 = pinf_2 the temperature is Eq. (Taverage) exactly. */
template <typename R>
static unsigned trelax_midpoint(const prm<R> *P, R m1, R m2, R E1, R E2, R a20, R *T, R *a2)
{
    R C1 = m1 * P->cv[0], C2 = m2 * P->cv[1];
    double G1 = P->gamma[0] - 1.0, G2 = P->gamma[1] - 1.0;
    double B1 = P->pinf[0] - P->pinf[1];
    /* phase temperatures before the stage: E_k = C_k T_k + a_k pinf_k */
    R T10 = (E1 - (1.0 - a20) * P->pinf[0]) / C1;
    R T20 = (E2 - a20 * P->pinf[1]) / C2;
    R Tp = (C1 * T10 + C2 * T20) / (C1 + C2);
    R ap = a20;
    for (int it = 0; it < P->trelax_iters; it++) {
        R T1a = 0.5 * (T10 + Tp), T2a = 0.5 * (T20 + Tp);
        R a2a = 0.5 * (a20 + ap), a1a = 1.0 - a2a;
        R num = G1 * C1 * T1a / (a1a * a1a) + G1 * P->pinf[0] / a1a + G2 * C2 * T2a / (a2a * a2a) +
                G2 * P->pinf[1] / a2a;
        R den = G1 / a1a + G2 / a2a;
        R B2 = P->pinf[1] - num / den;
        Tp = (B2 * C1 * T10 + (B1 + B2) * C2 * T20) / (B2 * C1 + (B1 + B2) * C2);
        ap = a20 - C2 * (Tp - T20) / B2;
    }
    *T = Tp;
    *a2 = ap;
    unsigned st = 0;
    if (!(ap > 0.0 && ap < 1.0 && Tp > 0.0)) st |= ORC_NONPHYS;
    if (is_nan(ap) || is_nan(Tp)) st |= ORC_NAN;
    return st;
}

template <typename R>
static unsigned trelax_t(const prm<R> *P, int ncell, R *U)
{
    unsigned st = 0;
    int n = ncell;
    for (int c = 0; c < n; c++) {
        R m1 = U[0 * n + c], m2 = U[1 * n + c];
        R rhoe = U[4 * n + c] + U[5 * n + c];
        R T, a2;
        if (P->trelax == 2)
            st |= trelax_midpoint(P, m1, m2, U[4 * n + c], U[5 * n + c], U[7 * n + c], &T, &a2);
        else
            st |= equilibrium(P, m1, m2, rhoe, &T, &a2);
        U[4 * n + c] = m1 * P->cv[0] * T + (1.0 - a2) * P->pinf[0];
        U[5 * n + c] = m2 * P->cv[1] * T + a2 * P->pinf[1];
        U[7 * n + c] = a2;
    }
    return st;
}

extern "C" unsigned orc_trelax(const orc_params *P, int ncell, double *U)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return trelax_t(&Pv, ncell, U);
}

/* ------------------------------------------------------------------------- */
/* Chebyshev local-iteration method (Sec. 3.2, Eqs. LIM, LIM_last).           */
/* ------------------------------------------------------------------------- */
/* P = ceil(pi/4 sqrt(tau lambda_max + 1)) (Sec. 3.2), then the policy: fixed P,
 * or clamp to [p_min, p_max].  The formula is capped at p_max as well: with the
 * paper's parameter order the roundoff of the recurrence grows with P
 * (intermediate factors reach tau lambda_max), so large P is not usable in
 * finite precision. */
static int cheb_P_formula(double tau, double lam_max)
{
    return (int)ceil(ORC_PI / 4.0 * sqrt(tau * lam_max + 1.0));
}

template <typename R>
static int cheb_P(const prm<R> *P, double tau, double lam_max)
{
    int pf = cheb_P_formula(tau, lam_max);
    if (P->p_policy == 1) return P->p_fixed;
    if (P->p_policy == 2 && pf < P->p_min) pf = P->p_min;
    if (pf > P->p_max) pf = P->p_max;
    return pf;
}

extern "C" int orc_cheb_P(const orc_params *P, double tau, double lam_max)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return cheb_P(&Pv, tau, lam_max);
}

template <typename R>
static unsigned cheb_capped(const prm<R> *P, double tau, double lam_max, int Pn)
{
    return (P->p_policy != 1 && Pn < cheb_P_formula(tau, lam_max)) ? ORC_PCAP : 0u;
}

/* P of the viscous solve: the formula (capped at p_max); the fixed / clamped
 * stage counts of a configuration are those of the heat-conduction solve */
template <typename R>
static int cheb_P_viscous(const prm<R> *P, double tau, double lam_max)
{
    int pf = cheb_P_formula(tau, lam_max);
    return pf > P->p_max ? P->p_max : pf;
}

/* b_1..b_{2P-1} = (a_P .. a_2, a_P .. a_1), a_m = lam (beta_1 - beta_m)/(1 + beta_1),
 * beta_m = cos((2m-1) pi / (2P)) the roots of T_P.  The roots are taken in their
 * natural (decreasing) order so that beta_1 is the largest and every a_m >= 0
 * (the ascending order the text names makes a_m negative and the iteration
 * unstable). */
extern "C" void orc_cheb_schedule(int Pn, double lam, double *b)
{
    double *beta = (double *)malloc(sizeof(double) * (Pn + 1));
    double *a = (double *)malloc(sizeof(double) * (Pn + 1));
    for (int m = 1; m <= Pn; m++) beta[m] = cos((2.0 * m - 1.0) * ORC_PI / (2.0 * Pn));
    for (int m = 1; m <= Pn; m++) a[m] = lam * (beta[1] - beta[m]) / (1.0 + beta[1]);
    for (int s = 0; s < Pn - 1; s++) b[s] = a[Pn - s];
    for (int s = 0; s < Pn; s++) b[Pn - 1 + s] = a[Pn - s];
    free(beta); free(a);
}

/* Discrete operator L_h v = div(Lam grad v) in flux-difference form (Eq. qk_dis):
 * (L v)_i = Fx_{i+1/2} - Fx_{i-1/2} + Fy_{j+1/2} - Fy_{j-1/2},
 * F_{i+1/2} = Lam_{i+1/2} (v_{i+1} - v_i) / h^2; Lam on faces is given.
 * Face arrays: lx[j*(nx+1)+i] is the face left of cell i, ly[j*nx+i] the face
 * below cell (i,j) (ny+1 rows).  Transmissive walls carry zero face
 * coefficient; periodic axes wrap.  An axis of extent 1 is inactive. */
template <typename R>
struct orc_op {
    int nx, ny;
    double dx, dy;
    int bc[2];
    R *lx, *ly;
    double idx2, idy2; /* the 1/h^2 factors of Eq. (qk_dis), formed once per grid */
    int only;          /* -1: both axes; 0 / 1: the operator along x / y only (viscous step) */
};

template <typename R>
static void op_init(orc_op<R> *o, int nx, int ny, double dx, double dy, const int *bc)
{
    o->nx = nx; o->ny = ny; o->dx = dx; o->dy = dy;
    o->bc[0] = bc[0]; o->bc[1] = bc[1];
    o->idx2 = 1.0 / (dx * dx);
    o->idy2 = 1.0 / (dy * dy);
    o->only = -1;
    o->lx = (R *)malloc(sizeof(R) * (nx + 1) * ny);
    o->ly = (R *)malloc(sizeof(R) * nx * (ny + 1));
}

template <typename R>
static void op_apply(const orc_op<R> *o, const R *v, R *out)
{
    int nx = o->nx, ny = o->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            R r = 0.0;
            if (nx > 1 && o->only != 1) {
                int il = i == 0 ? nx - 1 : i - 1, ir = i == nx - 1 ? 0 : i + 1;
                R fl = o->lx[j * (nx + 1) + i] * (v[j * nx + i] - v[j * nx + il]) * o->idx2;
                R fr = o->lx[j * (nx + 1) + i + 1] * (v[j * nx + ir] - v[j * nx + i]) * o->idx2;
                r += fr - fl;
            }
            if (ny > 1 && o->only != 0) {
                int jl = j == 0 ? ny - 1 : j - 1, jr = j == ny - 1 ? 0 : j + 1;
                R fl = o->ly[j * nx + i] * (v[j * nx + i] - v[jl * nx + i]) * o->idy2;
                R fr = o->ly[(j + 1) * nx + i] * (v[jr * nx + i] - v[j * nx + i]) * o->idy2;
                r += fr - fl;
            }
            out[j * nx + i] = r;
        }
}

/* face coefficients as the arithmetic mean of the two cell values (the paper
 * does not specify Lam_{k,i+1/2}); zero on transmissive walls */
template <typename R>
static void op_faces(orc_op<R> *o, const R *lam)
{
    int nx = o->nx, ny = o->ny;
    if (o->only == 1) memset(o->lx, 0, sizeof(R) * (nx + 1) * ny);
    if (o->only == 0) memset(o->ly, 0, sizeof(R) * nx * (ny + 1));
    for (int j = 0; j < ny && o->only != 1; j++)
        for (int i = 0; i <= nx; i++) {
            R v;
            if (i == 0 || i == nx)
                v = o->bc[0] == 1 ? 0.5 * (lam[j * nx + nx - 1] + lam[j * nx + 0]) : R(0.0);
            else
                v = 0.5 * (lam[j * nx + i - 1] + lam[j * nx + i]);
            o->lx[j * (nx + 1) + i] = v;
        }
    for (int j = 0; j <= ny && o->only != 0; j++)
        for (int i = 0; i < nx; i++) {
            R v;
            if (j == 0 || j == ny)
                v = o->bc[1] == 1 ? 0.5 * (lam[(ny - 1) * nx + i] + lam[i]) : R(0.0);
            else
                v = 0.5 * (lam[(j - 1) * nx + i] + lam[j * nx + i]);
            o->ly[j * nx + i] = v;
        }
}

/* Gershgorin bound of the spectrum of A = -V L_h: max_i 2 V_i sum_f Lam_f / h_f^2
 * (a value: lambda_max sets the Chebyshev schedule, which is never differentiated) */
template <typename R>
static double op_lam_max(const orc_op<R> *o, const R *V)
{
    int nx = o->nx, ny = o->ny;
    double lm = 0.0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            R s = 0.0;
            if (nx > 1 && o->only != 1) s += (o->lx[j * (nx + 1) + i] + o->lx[j * (nx + 1) + i + 1]) * o->idx2;
            if (ny > 1 && o->only != 0) s += (o->ly[j * nx + i] + o->ly[(j + 1) * nx + i]) * o->idy2;
            double r = val(2.0 * V[j * nx + i] * s);
            if (r > lm) lm = r;
        }
    return lm;
}

/* The first 2P-2 local iterations of Eq. (LIM) for dv/dt = V L_h v:
 *   v^(m) = (v^n + tau b_m v^(m-1) + tau V L_h v^(m-1)) / (1 + tau b_m),
 * v^(0) = v^n; L_h is the (negative semi-definite) discrete diffusion operator,
 * so the sweeps add +tau V L_h (Sec. 3.2's "-tau L_h" is written for the
 * positive operator -L_h).  Returns the predictor u_hat = v^(2P-2); the final,
 * explicit sweep (b_{2P-1} = 0, Eq. LIM_last) is applied by the caller in
 * conservative form. */
template <typename R>
static void lim_predict(const orc_op<R> *o, int Pn, const double *b, double tau, const R *V, const R *v0,
                        const R *f, R *uhat)
{
    int n = o->nx * o->ny;
    R *cur = (R *)malloc(sizeof(R) * n);
    R *nxt = (R *)malloc(sizeof(R) * n);
    R *Lv = (R *)malloc(sizeof(R) * n);
    memcpy(cur, v0, sizeof(R) * n);
    for (int m = 1; m <= 2 * Pn - 2; m++) {
        double bm = b[m - 1];
        double rden = 1.0 / (1.0 + tau * bm); /* the prefactor of Eq. (LIM), once per sweep */
        op_apply(o, cur, Lv);
        for (int c = 0; c < n; c++)
            nxt[c] = (v0[c] + tau * bm * cur[c] + tau * V[c] * Lv[c] + (f ? tau * f[c] : R(0.0))) * rden;
        R *t = cur; cur = nxt; nxt = t;
    }
    memcpy(uhat, cur, sizeof(R) * n);
    free(cur); free(nxt); free(Lv);
}

/* exported for tests: one complete LIM solve (2P-1 iterations, the last one
 * explicit) of dv/dt = V L_h v with cell coefficient lam, returns P */
extern "C" int orc_lim_solve(const orc_params *Pp, int nx, int ny, double dx, double dy, double tau,
                             const double *lam, const double *V, const double *v0, double *v1, double *lam_max_out)
{
    prm<double> Pv = make_prm<double>(Pp, NULL);
    int n = nx * ny;
    orc_op<double> o;
    op_init(&o, nx, ny, dx, dy, Pp->bc);
    op_faces(&o, lam);
    double lm = op_lam_max(&o, V);
    int Pn = cheb_P(&Pv, tau, lm);
    double *b = (double *)malloc(sizeof(double) * (2 * Pn - 1));
    orc_cheb_schedule(Pn, lm, b);
    double *uh = (double *)malloc(sizeof(double) * n);
    double *Lu = (double *)malloc(sizeof(double) * n);
    lim_predict(&o, Pn, b, tau, V, v0, (const double *)NULL, uh);
    op_apply(&o, uh, Lu);
    for (int c = 0; c < n; c++) v1[c] = v0[c] + tau * V[c] * Lu[c];
    if (lam_max_out) *lam_max_out = lm;
    free(o.lx); free(o.ly); free(b); free(uh); free(Lu);
    return Pn;
}

/* lambda_max of a solve: computed (and recorded in *slot when slot != NULL),
 * or, when replaying a recorded schedule, read from *slot */
static double lam_of(double computed, double *slot, int replay)
{
    if (slot && replay) return *slot;
    if (slot) *slot = computed;
    return computed;
}

/* ------------------------------------------------------------------------- */
/* Heat conduction under p,T equilibrium: Algorithm 1 with the LIM.         */
/* ------------------------------------------------------------------------- */
/* On the equilibrium manifold rho e = C T + pinf_1 - B1 alpha with p1 = p2, so
 * dT/d(rho e) = V = 1 / (C + B1^2 / K), K = T sum_k (p + pinf_k)/alpha_k,
 * d alpha/d(rho e) = -B1 V / K, and q1 + q2 = div(Lam grad T), Lam = a1 l1 + a2 l2.
 * Eq. (ht_eq2_ht) is then dT/dt = V L_h T.  Each outer iteration freezes V and
 * Lam at the latest (T, alpha), runs the 2P-2 predictor sweeps from T^n, and
 * applies the last (explicit) sweep conservatively to the mixture energy:
 * rho E += tau L_h u_hat, rho e += tau L_h u_hat, followed by the projection
 * (T, alpha) = equilibrium(m1, m2, rho e) and E_k = C_k T + a_k pinf_k.
 * With heat_alpha = 1 the projection is replaced by the linear update of
 * Eqs. (ht_eq2_ht), (ht_eq3_ht) with the frozen V and U = -B1 V / K.
 * lam_io: NULL, or the 8 lambda_max slots of the schedule record. */
template <typename R>
static unsigned heat_t(const prm<R> *P, int nx, int ny, double dx, double dy, double tau, R *U, int *P_used,
                       double *lam_io, int replay)
{
    int n = nx * ny;
    unsigned st = 0;
    double B1 = P->pinf[0] - P->pinf[1];
    R *T0 = (R *)malloc(sizeof(R) * n);
    R *re0 = (R *)malloc(sizeof(R) * n);
    R *rE0 = (R *)malloc(sizeof(R) * n);
    R *Ti = (R *)malloc(sizeof(R) * n);
    R *ai = (R *)malloc(sizeof(R) * n);
    R *V = (R *)malloc(sizeof(R) * n);
    R *lam = (R *)malloc(sizeof(R) * n);
    R *uh = (R *)malloc(sizeof(R) * n);
    R *q = (R *)malloc(sizeof(R) * n);
    R *Ia = (R *)malloc(sizeof(R) * n); /* I1 + I2 = a1 I1 + a2 I2 (Eq. I) */
    R *f = (R *)malloc(sizeof(R) * n);  /* V (I1 + I2): the f of Eq. (LIM) */
    R *Uc = (R *)malloc(sizeof(R) * n); /* U = d alpha / d(rho e) = -B1 V / K */
    R *a0 = (R *)malloc(sizeof(R) * n);
    orc_op<R> o;
    op_init(&o, nx, ny, dx, dy, P->bc);
    for (int c = 0; c < n; c++) {
        T0[c] = cell_T(P, U, n, c);
        re0[c] = U[4 * n + c] + U[5 * n + c];
        rE0[c] = U[6 * n + c];
        Ti[c] = T0[c];
        ai[c] = U[7 * n + c];
        a0[c] = ai[c];
    }
    int pmax_used = 0;
    int nout = P->n_outer < 1 ? 1 : P->n_outer;
    for (int it = 0; it < nout; it++) {
        for (int c = 0; c < n; c++) {
            R m1 = U[0 * n + c], m2 = U[1 * n + c];
            R T = Ti[c], a2 = ai[c], a1 = 1.0 - a2;
            R C1 = m1 * P->cv[0], C2 = m2 * P->cv[1];
            /* p + pinf_k = G_k C_k T / a_k on the manifold */
            R r1 = (P->gamma[0] - 1.0) * C1 * T / (a1 * a1);
            R r2 = (P->gamma[1] - 1.0) * C2 * T / (a2 * a2);
            R K = T * (r1 + r2);
            V[c] = 1.0 / (C1 + C2 + B1 * B1 / K);
            if (P->heat_alpha == 1) Uc[c] = -(B1 * V[c]) / K;
            lam[c] = a1 * lambda_k(P, 0, T) + a2 * lambda_k(P, 1, T);
            Ia[c] = a1 * P->src[0] + a2 * P->src[1];
            f[c] = V[c] * Ia[c];
        }
        op_faces(&o, lam);
        double lm = lam_of(op_lam_max(&o, V), lam_io ? lam_io + (it < 8 ? it : 7) : NULL, replay);
        int Pn = cheb_P(P, tau, lm);
        st |= cheb_capped(P, tau, lm, Pn);
        if (Pn > pmax_used) pmax_used = Pn;
        double *b = (double *)malloc(sizeof(double) * (2 * Pn - 1));
        orc_cheb_schedule(Pn, lm, b);
        lim_predict(&o, Pn, b, tau, V, T0, f, uh);
        free(b);
        op_apply(&o, uh, q);
        /* the last sweep in conservative form: rho e gains tau (L_h u_hat + I1 + I2) */
        for (int c = 0; c < n; c++) q[c] = q[c] + Ia[c];
        if (P->heat_alpha == 1) {
            /* Eqs. (ht_eq2_ht), (ht_eq3_ht) over the step with the frozen V, U
             * and the same q + I: T = T^n + tau V (q + I), alpha = alpha^n + tau U (q + I);
             * the energy C T + pinf_1 - B1 alpha gains tau (q + I)(C V - B1 U) = tau (q + I) */
            for (int c = 0; c < n; c++) {
                Ti[c] = T0[c] + tau * V[c] * q[c];
                ai[c] = a0[c] + tau * Uc[c] * q[c];
            }
        } else {
            for (int c = 0; c < n; c++) {
                R T, a2;
                st |= equilibrium(P, U[0 * n + c], U[1 * n + c], re0[c] + tau * q[c], &T, &a2);
                Ti[c] = T;
                ai[c] = a2;
            }
        }
    }
    for (int c = 0; c < n; c++) {
        R a2 = ai[c], T = Ti[c];
        U[4 * n + c] = U[0 * n + c] * P->cv[0] * T + (1.0 - a2) * P->pinf[0];
        U[5 * n + c] = U[1 * n + c] * P->cv[1] * T + a2 * P->pinf[1];
        U[6 * n + c] = rE0[c] + tau * q[c];
        U[7 * n + c] = a2;
    }
    if (P_used) *P_used = pmax_used;
    free(T0); free(re0); free(rE0); free(Ti); free(ai); free(V); free(lam); free(uh); free(q); free(Ia); free(f);
    free(Uc); free(a0);
    free(o.lx); free(o.ly);
    return st;
}

extern "C" unsigned orc_heat(const orc_params *P, int nx, int ny, double dx, double dy, double tau, double *U,
                             int *P_used)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return heat_t(&Pv, nx, ny, dx, dy, tau, U, P_used, NULL, 0);
}

/* ------------------------------------------------------------------------- */
/* Viscous step along one axis (Sec. 3.2).                                   */
/* ------------------------------------------------------------------------- */
/* rho du_n/dt = d/dx(4/3 mu du_n/dx) and rho du_t/dt = d/dx(mu du_t/dx) by the
 * LIM with V = 1/rho and mu = a1 mu1 + a2 mu2 (cross-derivative terms are
 * dropped by the directional splitting); the last sweep updates rho u
 * conservatively from the predicted velocity u_hat; rho E and E_k follow the
 * face-flux formulas of Sec. 3.2 with face values taken as two-cell means and
 * u_hat_i in place of u_i.  lam_io: NULL, or the schedule slot of this solve. */
template <typename R>
static unsigned viscous_t(const prm<R> *P, int nx, int ny, double dx, double dy, int axis, double tau, R *U,
                          int *P_used, double *lam_io, int replay)
{
    int n = nx * ny;
    int len = axis == 0 ? nx : ny;
    double h = axis == 0 ? dx : dy;
    int qn = axis == 0 ? 2 : 3, qt = axis == 0 ? 3 : 2;
    if (len < 2) { if (P_used) *P_used = 0; return 0; }
    R *V = (R *)malloc(sizeof(R) * n);
    R *mu = (R *)malloc(sizeof(R) * n);
    R *ln = (R *)malloc(sizeof(R) * n);
    R *un0 = (R *)malloc(sizeof(R) * n);
    R *ut0 = (R *)malloc(sizeof(R) * n);
    R *unh = (R *)malloc(sizeof(R) * n);
    R *uth = (R *)malloc(sizeof(R) * n);
    for (int c = 0; c < n; c++) {
        R rho = U[0 * n + c] + U[1 * n + c];
        R a2 = U[7 * n + c];
        V[c] = 1.0 / rho;
        mu[c] = (1.0 - a2) * P->mu[0] + a2 * P->mu[1];
        ln[c] = 4.0 / 3.0 * mu[c];
        un0[c] = U[qn * n + c] / rho;
        ut0[c] = U[qt * n + c] / rho;
    }
    orc_op<R> o, ot;
    op_init(&o, nx, ny, dx, dy, P->bc);
    op_init(&ot, nx, ny, dx, dy, P->bc);
    double ih = 1.0 / h; /* the 1/dx factor of the face fluxes of Sec. 3.2, formed once */
    /* both operators act along the sweep axis only */
    o.only = axis;
    ot.only = axis;
    op_faces(&o, ln);
    op_faces(&ot, mu);
    double lm = lam_of(op_lam_max(&o, V), lam_io, replay);
    int Pn = cheb_P_viscous(P, tau, lm);
    unsigned st = Pn < cheb_P_formula(tau, lm) ? ORC_PCAP : 0u;
    double *b = (double *)malloc(sizeof(double) * (2 * Pn - 1));
    orc_cheb_schedule(Pn, lm, b);
    lim_predict(&o, Pn, b, tau, V, un0, (const R *)NULL, unh);
    lim_predict(&ot, Pn, b, tau, V, ut0, (const R *)NULL, uth);
    free(b);
    /* conservative last sweep and energy updates, line by line */
    R *newU = (R *)malloc(sizeof(R) * NQ * n);
    memcpy(newU, U, sizeof(R) * NQ * n);
    for (int c = 0; c < n; c++) {
        int i = c % nx, j = c / nx;
        int pos = axis == 0 ? i : j;
        /* neighbours and face coefficients on the two faces of cell c */
        R Fn[2], Ft[2], W[2], aF1[2], aF2[2];
        for (int s = 0; s < 2; s++) {
            /* s = 0: face minus (between pos-1 and pos), s = 1: face plus */
            int fp = pos + s; /* face index 0..len */
            R lnf, lmf;
            int cl, cr;
            if (axis == 0) {
                lnf = o.lx[j * (nx + 1) + fp];
                lmf = ot.lx[j * (nx + 1) + fp];
                int il = fp == 0 ? nx - 1 : fp - 1, ir = fp == nx ? 0 : fp;
                cl = j * nx + il; cr = j * nx + ir;
            } else {
                lnf = o.ly[fp * nx + i];
                lmf = ot.ly[fp * nx + i];
                int jl = fp == 0 ? ny - 1 : fp - 1, jr = fp == ny ? 0 : fp;
                cl = jl * nx + i; cr = jr * nx + i;
            }
            Fn[s] = lnf * (unh[cr] - unh[cl]) * ih;
            Ft[s] = lmf * (uth[cr] - uth[cl]) * ih;
            R ubar = 0.5 * (unh[cl] + unh[cr]);
            R wbar = 0.5 * (uth[cl] + uth[cr]);
            W[s] = ubar * Fn[s] + wbar * Ft[s];
            R a2l = U[7 * n + cl], a2r = U[7 * n + cr];
            aF2[s] = 0.5 * (a2l + a2r);
            aF1[s] = 0.5 * ((1.0 - a2l) + (1.0 - a2r));
        }
        newU[qn * n + c] = U[qn * n + c] + tau * (Fn[1] - Fn[0]) * ih;
        newU[qt * n + c] = U[qt * n + c] + tau * (Ft[1] - Ft[0]) * ih;
        newU[6 * n + c] = U[6 * n + c] + tau * (W[1] - W[0]) * ih;
        newU[4 * n + c] = U[4 * n + c] + tau * (aF1[1] * W[1] - aF1[0] * W[0]) * ih -
                          tau * (unh[c] * (aF1[1] * Fn[1] - aF1[0] * Fn[0]) + uth[c] * (aF1[1] * Ft[1] - aF1[0] * Ft[0])) * ih;
        newU[5 * n + c] = U[5 * n + c] + tau * (aF2[1] * W[1] - aF2[0] * W[0]) * ih -
                          tau * (unh[c] * (aF2[1] * Fn[1] - aF2[0] * Fn[0]) + uth[c] * (aF2[1] * Ft[1] - aF2[0] * Ft[0])) * ih;
    }
    memcpy(U, newU, sizeof(R) * NQ * n);
    if (P_used) *P_used = Pn;
    free(newU); free(V); free(mu); free(ln); free(un0); free(ut0); free(unh); free(uth);
    free(o.lx); free(o.ly); free(ot.lx); free(ot.ly);
    return st;
}

extern "C" unsigned orc_viscous(const orc_params *P, int nx, int ny, double dx, double dy, int axis, double tau,
                                double *U, int *P_used)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return viscous_t(&Pv, nx, ny, dx, dy, axis, tau, U, P_used, NULL, 0);
}

/* ------------------------------------------------------------------------- */
/* One split step: mechanical stage (hyperbolic sweeps x then y, each followed */
/* by pressure relaxation; viscous step; pressure relaxation), temperature    */
/* relaxation, heat conduction (Sec. 3 opening, Sec. 2.4).                    */
/* ------------------------------------------------------------------------- */
template <typename R>
static int viscous_on(const prm<R> *P) { return P->mu[0] > 0.0 || P->mu[1] > 0.0; }
template <typename R>
static int heat_on(const prm<R> *P)
{
    return P->trelax >= 1 && (P->k0[0] > 0.0 || P->k0[1] > 0.0 || P->src[0] > 0.0 || P->src[1] > 0.0);
}

/* end-of-step admissibility: alpha_2 in (0,1), m_k > 0, p_k + pinf_k > 0 */
template <typename R>
static unsigned final_check(const prm<R> *P, int n, const R *U)
{
    unsigned st = 0;
    for (int c = 0; c < n; c++) {
        R a2 = U[7 * n + c], a1 = 1.0 - a2;
        R p1 = phase_p(P, 0, U[4 * n + c], a1), p2 = phase_p(P, 1, U[5 * n + c], a2);
        if (!(a2 > 0.0 && a2 < 1.0 && U[0 * n + c] > 0.0 && U[1 * n + c] > 0.0 && p1 + P->pinf[0] > 0.0 &&
              p2 + P->pinf[1] > 0.0))
            st |= ORC_NONPHYS;
        for (int k = 0; k < NQ; k++)
            if (is_nan(U[k * n + c])) st |= ORC_NAN;
    }
    return st;
}

/* nsteps split steps.  sched: NULL, or nsteps records of ORC_SCHED doubles,
 * written (replay = 0) or read (replay = 1: S and every lambda_max are taken
 * from the record instead of the state). */
template <typename R>
static unsigned step_t(const prm<R> *P, int nx, int ny, double dx, double dy, R *U, int nsteps, double dt_fixed,
                       double *dt_last, int *P_heat, double *sched, int replay)
{
    int n = nx * ny;
    unsigned st = 0, tr = 0;
    int ph = 0;
    for (int s = 0; s < nsteps; s++) {
        double *rec = sched ? sched + (size_t)ORC_SCHED * s : NULL;
        if (rec && !replay) memset(rec, 0, sizeof(double) * ORC_SCHED);
        double dt;
        if (dt_fixed > 0.0) {
            dt = dt_fixed;
        } else {
            double S = rec && replay ? rec[0] : wave_max(P, nx, ny, dx, dy, U);
            if (rec && !replay) rec[0] = S;
            dt = P->cfl / S;
        }
        if (nx > 1) { tr |= sweep_t(P, nx, ny, dx, dy, 0, dt, U); tr |= prelax_t(P, n, U); }
        if (ny > 1) { tr |= sweep_t(P, nx, ny, dx, dy, 1, dt, U); tr |= prelax_t(P, n, U); }
        if (viscous_on(P)) {
            int pv;
            if (nx > 1) tr |= viscous_t(P, nx, ny, dx, dy, 0, dt, U, &pv, rec ? rec + 9 : NULL, replay);
            if (ny > 1) tr |= viscous_t(P, nx, ny, dx, dy, 1, dt, U, &pv, rec ? rec + 10 : NULL, replay);
            tr |= prelax_t(P, n, U);
        }
        if (P->trelax >= 1) {
            tr |= trelax_t(P, n, U);
            if (heat_on(P)) tr |= heat_t(P, nx, ny, dx, dy, dt, U, &ph, rec ? rec + 1 : NULL, replay);
        }
        st |= final_check(P, n, U);
        if (dt_last) *dt_last = dt;
    }
    if (tr & (ORC_NONPHYS | ORC_NOROOT)) st |= ORC_TRANSIENT;
    if (tr & ORC_NAN) st |= ORC_NAN;
    st |= tr & ORC_PCAP;
    if (P_heat) *P_heat = ph;
    return st;
}

extern "C" unsigned orc_step(const orc_params *P, int nx, int ny, double dx, double dy, double *U, int nsteps,
                             double dt_fixed, double *dt_last, int *P_heat)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return step_t(&Pv, nx, ny, dx, dy, U, nsteps, dt_fixed, dt_last, P_heat, NULL, 0);
}

/* nsteps steps recording (replay = 0) or replaying (replay = 1) the schedule */
extern "C" unsigned orc_step_sched(const orc_params *P, int nx, int ny, double dx, double dy, double *U, int nsteps,
                                   double *sched, int replay)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    return step_t(&Pv, nx, ny, dx, dy, U, nsteps, 0.0, NULL, NULL, sched, replay);
}

/* nsteps steps with the schedule and the sweep branches recorded (replay = 0)
 * or replayed (replay = 1).  tape holds tape_cap bytes; *tape_used receives
 * the number of branch decisions the run took.  Returns the status, or
 * ORC_EINVAL when the tape is too small. */
extern "C" unsigned orc_step_frozen(const orc_params *P, int nx, int ny, double dx, double dy, double *U, int nsteps,
                                    double *sched, unsigned char *tape, size_t tape_cap, int replay,
                                    size_t *tape_used)
{
    prm<double> Pv = make_prm<double>(P, NULL);
    g_tape.mode = replay ? 2 : 1;
    g_tape.buf = tape;
    g_tape.cap = tape_cap;
    g_tape.pos = 0;
    g_tape.overflow = 0;
    unsigned st = step_t(&Pv, nx, ny, dx, dy, U, nsteps, 0.0, NULL, NULL, sched, replay);
    if (tape_used) *tape_used = g_tape.pos;
    int over = g_tape.overflow;
    g_tape.mode = 0;
    g_tape.buf = NULL;
    return over ? ORC_EINVAL : st;
}

/* Tangent-linear map of nsteps steps: U (value) and dU (tangent, 8 planes) are
 * advanced together; dparams (6 values or NULL) are the tangents of
 * (k0_1, k0_2, mu_1, mu_2, I_1, I_2).  dt and every lambda_max are frozen at
 * the values of the run (sched, when given, records them). */
template <typename D>
static unsigned tangent_run(const orc_params *P, const double *dparams, int nx, int ny, double dx, double dy,
                            double *U, double *dU, int nsteps, double *sched, const unsigned char *tape,
                            size_t tape_len)
{
    prm<D> Pd = make_prm<D>(P, dparams);
    size_t m = (size_t)NQ * nx * ny;
    D *X = (D *)malloc(sizeof(D) * m);
    for (size_t i = 0; i < m; i++) X[i] = D(U[i], dU[i]);
    if (tape) {
        g_tape.mode = 2;
        g_tape.buf = (unsigned char *)tape;
        g_tape.cap = tape_len;
        g_tape.pos = 0;
        g_tape.overflow = 0;
    }
    unsigned st = step_t(&Pd, nx, ny, dx, dy, X, nsteps, 0.0, NULL, NULL, sched, sched && tape ? 1 : 0);
    if (tape) {
        if (g_tape.overflow || g_tape.pos != tape_len) st |= ORC_EINVAL;
        g_tape.mode = 0;
        g_tape.buf = NULL;
    }
    for (size_t i = 0; i < m; i++) {
        U[i] = (double)X[i].v;
        dU[i] = (double)X[i].d;
    }
    free(X);
    return st;
}

extern "C" unsigned orc_step_tangent(const orc_params *P, const double *dparams, int nx, int ny, double dx, double dy,
                                     double *U, double *dU, int nsteps, double *sched)
{
    return tangent_run<Dual>(P, dparams, nx, ny, dx, dy, U, dU, nsteps, sched, NULL, 0);
}

/* The same tangent with every value and tangent carried in long double, a
 * reference for the rounding error of the double tangent.  sched and tape:
 * the schedule and branch record of the double run (orc_step_frozen), replayed
 * so that the extended run linearizes the same branch-frozen map. */
extern "C" unsigned orc_step_tangent_ext(const orc_params *P, const double *dparams, int nx, int ny, double dx,
                                         double dy, double *U, double *dU, int nsteps, double *sched,
                                         const unsigned char *tape, size_t tape_len)
{
    return tangent_run<DualL>(P, dparams, nx, ny, dx, dy, U, dU, nsteps, sched, tape, tape_len);
}

/* Operation counts of one stage on state U (test infrastructure): stage 0 CFL
 * maximum, 1 / 2 sweep along x / y, 3 pressure relaxation, 4 temperature
 * relaxation, 5 heat conduction (P by the parameters' policy), 6 / 7 viscous
 * step along x / y.  out[0..4] = additions and subtractions, multiplications,
 * divisions, square roots, powers; returns the Chebyshev P used (or 0). */
extern "C" int orc_count_ops(const orc_params *P, int nx, int ny, double dx, double dy, const double *U, int stage,
                             double tau, unsigned long long *out)
{
    prm<Cnt> Pc = make_prm<Cnt>(P, NULL);
    size_t m = (size_t)NQ * nx * ny;
    Cnt *X = (Cnt *)malloc(sizeof(Cnt) * m);
    for (size_t i = 0; i < m; i++) X[i] = Cnt(U[i]);
    for (int k = 0; k < 5; k++) g_ops[k] = 0;
    int Pn = 0;
    switch (stage) {
    case 0: (void)wave_max(&Pc, nx, ny, dx, dy, X); break;
    case 1: sweep_t(&Pc, nx, ny, dx, dy, 0, tau, X); break;
    case 2: sweep_t(&Pc, nx, ny, dx, dy, 1, tau, X); break;
    case 3: prelax_t(&Pc, nx * ny, X); break;
    case 4: trelax_t(&Pc, nx * ny, X); break;
    case 5: heat_t(&Pc, nx, ny, dx, dy, tau, X, &Pn, NULL, 0); break;
    case 6: viscous_t(&Pc, nx, ny, dx, dy, 0, tau, X, &Pn, NULL, 0); break;
    case 7: viscous_t(&Pc, nx, ny, dx, dy, 1, tau, X, &Pn, NULL, 0); break;
    default: break;
    }
    for (int k = 0; k < 5; k++) out[k] = g_ops[k];
    free(X);
    return Pn;
}

/* diagnostics used by the tests: per-cell phase pressures and temperatures */
extern "C" void orc_diagnostics(const orc_params *Pp, int ncell, const double *U, double *out /* 6 planes */)
{
    prm<double> Pv = make_prm<double>(Pp, NULL);
    const prm<double> *P = &Pv;
    int n = ncell;
    for (int c = 0; c < n; c++) {
        double m1 = U[0 * n + c], m2 = U[1 * n + c];
        double a2 = U[7 * n + c], a1 = 1.0 - a2;
        double rho = m1 + m2;
        double p1 = phase_p(P, 0, U[4 * n + c], a1);
        double p2 = phase_p(P, 1, U[5 * n + c], a2);
        double r1 = m1 / a1, r2 = m2 / a2;
        /* T_k = (p_k + pinf_k) / ((g_k - 1) rho_k Cv_k), Eq. eos_stiffened2 */
        out[0 * n + c] = p1;
        out[1 * n + c] = p2;
        out[2 * n + c] = (p1 + P->pinf[0]) / ((P->gamma[0] - 1.0) * r1 * P->cv[0]);
        out[3 * n + c] = (p2 + P->pinf[1]) / ((P->gamma[1] - 1.0) * r2 * P->cv[1]);
        out[4 * n + c] = U[2 * n + c] / rho;
        out[5 * n + c] = U[3 * n + c] / rho;
    }
}

/* heat-stage coefficients at a cell state, exported for the tests:
 * out = (T, V, U_alpha, Lam) with U_alpha = -B1 V / K */
extern "C" void orc_heat_coeffs(const orc_params *Pp, int ncell, const double *U, double *out /* 4 planes */)
{
    prm<double> Pv = make_prm<double>(Pp, NULL);
    const prm<double> *P = &Pv;
    int n = ncell;
    double B1 = P->pinf[0] - P->pinf[1];
    for (int c = 0; c < n; c++) {
        double m1 = U[0 * n + c], m2 = U[1 * n + c];
        double a2 = U[7 * n + c], a1 = 1.0 - a2;
        double T = cell_T(P, U, n, c);
        double C1 = m1 * P->cv[0], C2 = m2 * P->cv[1];
        double r1 = (P->gamma[0] - 1.0) * C1 * T / (a1 * a1);
        double r2 = (P->gamma[1] - 1.0) * C2 * T / (a2 * a2);
        double K = T * (r1 + r2);
        double V = 1.0 / (C1 + C2 + B1 * B1 / K);
        out[0 * n + c] = T;
        out[1 * n + c] = V;
        out[2 * n + c] = -B1 * V / K;
        out[3 * n + c] = a1 * lambda_k(P, 0, T) + a2 * lambda_k(P, 1, T);
    }
}

/* exported for tests: the equilibrium projection of one state */
extern "C" unsigned orc_equilibrium(const orc_params *Pp, double m1, double m2, double rhoe, double *T, double *a2)
{
    prm<double> Pv = make_prm<double>(Pp, NULL);
    return equilibrium(&Pv, m1, m2, rhoe, T, a2);
}

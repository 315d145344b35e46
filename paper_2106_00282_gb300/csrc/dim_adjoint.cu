// dim_adjoint.cu -- adjoint (reverse-mode) kernels of the split step (sm_103a).
//
// Each stage of the step (Sec. 3) is differentiated with its schedule (dt,
// Chebyshev lambda_max, hence P and b_m) and its value-decided branches
// (limiter operand, Davis bounds, HLLC wave region) held fixed:
//
//  * pointwise stages: the pressure relaxation (Sec. 3.3) and the p,T
//    equilibrium (temperature relaxation, Sec. 3.4.1, and the projection of
//    Sec. 3.4.2) are reversed by hand, the admissible roots through their
//    implicit derivatives; the conduction coefficients of Sec. 3.4.2 form
//    their local Jacobian with forward-mode dual numbers and apply its
//    transpose;
//  * the hyperbolic sweep (Sec. 3.1, 3.6): the update of cell i is
//    U_i - dt/h (F_{i+1/2} - F_{i-1/2}) - dt/h R(U_i)(u*_{i+1/2} - u*_{i-1/2});
//    the adjoint of face f's outputs (F, u*) is dt/h times the difference of
//    its two cells' adjoints (and of R.adjoint for u*); each face reverses its
//    HLLC flux and reconstruction by hand into the adjoints of its four
//    stencil cells' primitives, and every cell gathers those and applies the
//    transposed primitive Jacobian;
//  * the LIM solves (Sec. 3.2, Eqs. LIM, LIM_last): the sweeps
//    v^m = (v^0 + tau b_m v^{m-1} + tau V (L v^{m-1} + f)) / (1 + tau b_m) are
//    linear in v for frozen coefficients and L_h is symmetric, so the reverse
//    sweep is  y = vbar^m/(1 + tau b_m),  vbar^{m-1} = tau b_m y + tau L(V y),
//    accumulating the adjoints of v^0, V, the face coefficients and f; the
//    coefficients' own dependence on the state (V, Lam of Sec. 3.4.2, 1/rho
//    and mu of Sec. 3.2) is then transposed pointwise.
// The primal values the kernels need (stage inputs, every LIM iterate) are
// recomputed by the forward kernels and passed in.  Parameter gradients
// (k0_k, mu_k, I_k) are block sums added to 6 device doubles.
#include "dim_device.cuh"

namespace dimk {
namespace {

// ---------------------------------------------------------------------------
// forward-mode dual numbers: a value and N tangent components
// ---------------------------------------------------------------------------
template <int N>
struct Dn {
    double v;
    double d[N];
};

template <int N>
__device__ __forceinline__ Dn<N> dcst(double v)
{
    Dn<N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = 0.0;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> dseed(double v, int k)
{
    Dn<N> r = dcst<N>(v);
    r.d[k] = 1.0;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N> &a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(const Dn<N> &a, double b)
{
    Dn<N> r = a;
    r.v = a.v + b;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator+(double a, const Dn<N> &b)
{
    Dn<N> r = b;
    r.v = a + b.v;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N> &a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N> &a, double b)
{
    Dn<N> r = a;
    r.v = a.v - b;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(double a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a - b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = -b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator-(const Dn<N> &a)
{
    Dn<N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = -a.d[i];
    return r;
}
// d(ab) = b da + a db
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N> &a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(const Dn<N> &a, double b)
{
    Dn<N> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator*(double a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a * b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a * b.d[i];
    return r;
}
// d(a/b) = (da - (a/b) db) / b.  The value is the IEEE quotient (the branch
// decisions of the forward depend on it); the tangents multiply by one
// reciprocal.
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N> &a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(const Dn<N> &a, double b)
{
    Dn<N> r;
    r.v = a.v / b;
    const double ib = 1.0 / b;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * ib;
    return r;
}
template <int N>
__device__ __forceinline__ Dn<N> operator/(double a, const Dn<N> &b)
{
    Dn<N> r;
    r.v = a / b.v;
    const double s = -r.v / b.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = s * b.d[i];
    return r;
}
// d sqrt(a) = da / (2 sqrt(a))
template <int N>
__device__ __forceinline__ Dn<N> dsqrt(const Dn<N> &a)
{
    Dn<N> r;
    r.v = sqrt(a.v);
    const double h = 0.5 / r.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * h;
    return r;
}
// x^e for the conductivity law, derivative e x^(e-1) (k_pow: 0 constant, >0
// integer power by repeated products, <0 general exponent)
template <int N>
__device__ __forceinline__ Dn<N> dpow_law(const DevParams &p, const Dn<N> &t)
{
    if (p.k_pow > 0) {
        Dn<N> r = t;
        for (int i = 1; i < p.k_pow; i++) r = r * t;
        return r;
    }
    Dn<N> r;
    r.v = pow(t.v, p.k_exp);
    double dr = p.k_exp * pow(t.v, p.k_exp - 1.0);
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = dr * t.d[i];
    return r;
}
// value of (T/T_ref)^k_exp as the forward law evaluates it
__device__ __forceinline__ double law_ratio(const DevParams &p, double T)
{
    if (p.k_pow == 0) return 1.0;
    double t = T * p.inv_Tref;
    if (p.k_pow > 0) {
        double r = t;
        for (int i = 1; i < p.k_pow; i++) r = r * t;
        return r;
    }
    return pow(t, p.k_exp);
}

// ---------------------------------------------------------------------------
// the stage formulas in dual arithmetic (same operation order as the forward)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ Dn<N> d_sgE(const DevParams &p, int k, const Dn<N> &pr, const Dn<N> &ak)
{
    return ak * (pr + p.gpinf[k]) * p.inv_gm1[k];
}

// conduction coefficients V = 1/(C + B1^2/K), Lam = sum_k a_k lambda_k(T)
// (Sec. 3.4.2) and the source a1 I1 + a2 I2 (Eq. I) at (m1, m2, T, a2)
template <int N>
__device__ __forceinline__ void d_heat_coeffs(const DevParams &p, const Dn<N> &m1, const Dn<N> &m2, const Dn<N> &T,
                                              const Dn<N> &a2, Dn<N> &V, Dn<N> &Lam, Dn<N> &Ia)
{
    Dn<N> a1 = 1.0 - a2;
    Dn<N> C1 = m1 * p.cv[0], C2 = m2 * p.cv[1];
    const double B1 = p.pinf[0] - p.pinf[1];
    Dn<N> r1 = p.gm1[0] * C1 * T / (a1 * a1);
    Dn<N> r2 = p.gm1[1] * C2 * T / (a2 * a2);
    Dn<N> K = T * (r1 + r2);
    V = 1.0 / (C1 + C2 + B1 * B1 / K);
    if (p.k_pow == 0) {
        Lam = a1 * p.k0[0] + a2 * p.k0[1];
    } else {
        Dn<N> r = dpow_law(p, T * p.inv_Tref);
        Lam = a1 * (p.k0[0] * r) + a2 * (p.k0[1] * r);
    }
    Ia = a1 * p.src[0] + a2 * p.src[1];
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int line_map(int a, int len, int bc)
{
    if (a >= 0 && a < len) return a;
    if (bc == DIM_BC_PERIODIC) return ((a % len) + len) % len;
    return a < 0 ? 0 : len - 1;
}

// neighbours along one axis: -1 at a transmissive wall (zero flux), wrapped
// when periodic, -1 when the axis has a single cell
__device__ __forceinline__ void axis_nb(const DevParams &p, int axis, int c, int &cm, int &cp)
{
    const int x = c % p.nx, y = c / p.nx;
    const int len = axis == 0 ? p.nx : p.ny, i = axis == 0 ? x : y;
    const int stride = axis == 0 ? 1 : p.nx;
    cm = cp = -1;
    if (len < 2) return;
    if (i > 0) cm = c - stride;
    else if (p.bc[axis] == DIM_BC_PERIODIC) cm = c + (len - 1) * stride;
    if (i < len - 1) cp = c + stride;
    else if (p.bc[axis] == DIM_BC_PERIODIC) cp = c - (len - 1) * stride;
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

__device__ __forceinline__ void add_param(double *pbar, int k, double v)
{
    double s = block_sum(v);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(pbar + k, s);
}

#define GRID_LOOP(c, n) for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (n); c += gridDim.x * blockDim.x)


// ---------------------------------------------------------------------------
// the p,T equilibrium (Sec. 3.4.1 / 3.4.2) and its reverse by the implicit
// derivative of the admissible root: qa a^2 + qb a + qc = 0 gives
// da = -(a^2 dqa + a dqb + dqc) / (2 qa a + qb); T = (E + B1 a) / C
// ---------------------------------------------------------------------------
struct EqState {
    double C, G, G2C2, E, qa, qb, B1, a, T;
};

// forward values in the operation order of the forward kernels' equilibrium()
__device__ __forceinline__ EqState eq_fwd(const DevParams &p, double m1, double m2, double rhoe)
{
    EqState q;
    const double C1 = m1 * p.cv[0], C2 = m2 * p.cv[1];
    q.C = C1 + C2;
    const double G1C1 = p.gm1[0] * C1;
    q.G2C2 = p.gm1[1] * C2;
    q.G = G1C1 + q.G2C2;
    q.B1 = p.pinf[0] - p.pinf[1];
    q.E = rhoe - p.pinf[0];
    q.qa = q.B1 * (q.G + q.C);
    q.qb = q.E * q.G - q.B1 * q.G2C2 - q.C * q.B1;
    const double qc = -q.E * q.G2C2;
    double disc = q.qb * q.qb - 4.0 * q.qa * qc;
    if (disc < 0.0) disc = 0.0;
    const double sq = sqrt(disc);
    q.a = q.qb > 0.0 ? (-2.0 * qc) / (q.qb + sq) : (sq - q.qb) / (2.0 * q.qa);
    q.T = (q.E + q.B1 * q.a) / q.C;
    return q;
}

// adjoints (Tb, ab) of (T, a) -> adjoints of (m1, m2, rho e)
__device__ __forceinline__ void eq_rev(const DevParams &p, const EqState &q, double Tb, double ab, double &m1b,
                                       double &m2b, double &reb)
{
    const double iC = 1.0 / q.C;
    double Eb = Tb * iC;
    ab += Tb * q.B1 * iC;
    double Cb = -Tb * q.T * iC;
    const double w = ab / (2.0 * q.qa * q.a + q.qb);
    const double qab = -w * q.a * q.a, qbb = -w * q.a, qcb = -w;
    double Gb = q.B1 * qab;
    Cb += q.B1 * qab;
    Eb += q.G * qbb;
    Gb += q.E * qbb;
    double G2C2b = -q.B1 * qbb;
    Cb -= q.B1 * qbb;
    Eb -= q.G2C2 * qcb;
    G2C2b -= q.E * qcb;
    G2C2b += Gb;
    const double C1b = p.gm1[0] * Gb + Cb, C2b = p.gm1[1] * G2C2b + Cb;
    m1b = p.cv[0] * C1b;
    m2b = p.cv[1] * C2b;
    reb = Eb;
}

// ---------------------------------------------------------------------------
// pointwise stages: Gin = J^T G in place (G: 8 planes)
// ---------------------------------------------------------------------------
// Pressure relaxation (Sec. 3.3) in reverse, per cell.  Forward: a_k(p) =
// (ak_k + bk_k p)/(g_k p + ek_k) with ak_k = (g_k-1)E_k, bk_k = (g_k-1)a_k,
// ek_k = g_k pinf_k; p the admissible root of A p^2 + B p + C = 0, hence
// dp = -(p^2 dA + p dB + dC)/sqrt(disc); a2n = a_2(p); p2 from
// rho e = rho E - |rho u|^2/(2 rho); E_k = a_kn (p2 + g_k pinf_k)/(g_k - 1).
// The outputs are E_1, E_2, alpha_2; m_k, rho u, rho v, rho E pass through.
__global__ void __launch_bounds__(256) k_adj_prelax(const DevParams p, const double *Uin, double *G)
{
    const int n = p.n;
    const double g1 = p.g[0], g2 = p.g[1], ek1 = p.gpinf[0], ek2 = p.gpinf[1];
    const double i1 = p.inv_gm1[0], i2 = p.inv_gm1[1];
    const double c1 = p.g[0] * p.pinf[0] * p.inv_gm1[0], c2 = p.g[1] * p.pinf[1] * p.inv_gm1[1];
    GRID_LOOP(c, n)
    {
        const double m1 = Uin[c], m2 = Uin[n + c], mu = Uin[2 * n + c], mv = Uin[3 * n + c];
        const double E1 = Uin[4 * n + c], E2 = Uin[5 * n + c], rE = Uin[6 * n + c], a2 = Uin[7 * n + c];
        // forward values (the operation order of the forward relaxation)
        const double a1 = 1.0 - a2;
        const double ak1 = p.gm1[0] * E1, bk1 = p.gm1[0] * a1, ak2 = p.gm1[1] * E2, bk2 = p.gm1[1] * a2;
        const double A = g1 * g2 - bk1 * g2 - bk2 * g1;
        const double B = g1 * ek2 + ek1 * g2 - (ak1 * g2 + bk1 * ek2 + ak2 * g1 + bk2 * ek1);
        const double C = ek1 * ek2 - ak1 * ek2 - ak2 * ek1;
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) disc = 0.0;
        const double sq = sqrt(disc);
        const double pr = B <= 0.0 ? (sq - B) / (2.0 * A) : (2.0 * C) / (-B - sq);
        const double Xa = ak2 + bk2 * pr, Ya = g2 * pr + ek2;
        const double a2n = Xa / Ya, a1n = 1.0 - a2n;
        const double rho = m1 + m2;
        const double ke = 0.5 * (mu * mu + mv * mv) / rho;
        const double rhoe = rE - ke;
        const double Nn = rhoe - (a1n * c1 + a2n * c2), Dd = a1n * i1 + a2n * i2;
        const double p2 = Nn / Dd;
        // reverse (shared reciprocals: the adjoint needs no bit-compatibility)
        const double G4 = G[4 * n + c], G5 = G[5 * n + c], G7 = G[7 * n + c];
        const double p2b = G4 * a1n * i1 + G5 * a2n * i2;
        double a1nb = G4 * (p2 + ek1) * i1;
        double a2nb = G5 * (p2 + ek2) * i2 + G7;
        const double rD = 1.0 / Dd, rr = 1.0 / rho, rY = 1.0 / Ya;
        const double Nb = p2b * rD, Db = -p2b * p2 * rD;
        const double rhoeb = Nb;
        a1nb += -Nb * c1 + Db * i1;
        a2nb += -Nb * c2 + Db * i2;
        a2nb -= a1nb;
        const double rEb = rhoeb;
        const double mub = -rhoeb * mu * rr, mvb = -rhoeb * mv * rr;
        const double rhob = rhoeb * ke * rr;
        const double Xb = a2nb * rY, Yb = -a2nb * a2n * rY;
        double ak2b = Xb, bk2b = Xb * pr;
        const double prb = Xb * bk2 + Yb * g2;
        const double w = prb / sq;
        const double Ab = -w * pr * pr, Bb = -w * pr, Cb = -w;
        double bk1b = -Ab * g2;
        bk2b += -Ab * g1;
        double ak1b = -Bb * g2;
        bk1b += -Bb * ek2;
        ak2b += -Bb * g1;
        bk2b += -Bb * ek1;
        ak1b += -Cb * ek2;
        ak2b += -Cb * ek1;
        G[c] += rhob;
        G[n + c] += rhob;
        G[2 * n + c] += mub;
        G[3 * n + c] += mvb;
        G[4 * n + c] = ak1b * p.gm1[0];
        G[5 * n + c] = ak2b * p.gm1[1];
        G[6 * n + c] += rEb;
        G[7 * n + c] = -bk1b * p.gm1[0] + bk2b * p.gm1[1];
    }
}

// temperature relaxation (Sec. 3.4.1): (T, a) = equilibrium(m1, m2, E1 + E2),
// E_k = m_k Cv_k T + a_k pinf_k
__global__ void __launch_bounds__(256) k_adj_trelax(const DevParams p, const double *Uin, double *G)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        // inputs m1, m2, E1, E2; outputs E_k = m_k Cv_k T + a_k pinf_k and alpha_2 = a
        const double m1 = Uin[c], m2 = Uin[n + c];
        const EqState q = eq_fwd(p, m1, m2, Uin[4 * n + c] + Uin[5 * n + c]);
        const double g4 = G[4 * n + c], g5 = G[5 * n + c], g7 = G[7 * n + c];
        const double Tb = g4 * m1 * p.cv[0] + g5 * m2 * p.cv[1];
        const double ab = -g4 * p.pinf[0] + g5 * p.pinf[1] + g7;
        double m1b, m2b, reb;
        eq_rev(p, q, Tb, ab, m1b, m2b, reb);
        G[c] += g4 * p.cv[0] * q.T + m1b;
        G[n + c] += g5 * p.cv[1] * q.T + m2b;
        G[4 * n + c] = reb;
        G[5 * n + c] = reb;
        G[7 * n + c] = 0.0;  // alpha_2 is replaced by the equilibrium value
    }
}

// ---------------------------------------------------------------------------
// hyperbolic sweep (two kernels)
// ---------------------------------------------------------------------------
// The flux (F, u*) of face f depends on its 4-cell stencil only through the
// reconstructed primitives wl (cell f-1) and wr (cell f): 14 values.
// k_adj_sweep_face, per face: the adjoint of the face outputs
// gbar = dt/h (adj_R - adj_L) [and dt/h (R.adj_R - R.adj_L) for u*], the
// hand-written reverse of the HLLC flux with respect to (wl, wr),
// then the transposed reconstruction (slopes: the minmod operand chosen, times
// 1 or 2 for Overbee) -> the adjoint of the primitives W of the 4 stencil
// cells, stored per face (28 values) with the face's u*.
// k_adj_sweep_cell, per cell: the sum over the faces whose stencil holds the
// cell (ghost positions mapped as in the forward), the transposed Jacobian of
// the conversion q -> W, the identity of the update and the cell's own
// R(U_i)(u*_{i+1/2} - u*_{i-1/2}) term.
// k_adj_sweep_prims first stores every cell's primitives W (line-local order)
// once, so that the face kernel does not convert each cell four times.
constexpr int FACE_ADJ_PLANES = 29;  // 4 x 7 primitive adjoints + u*
constexpr int FACE_WORK_PLANES = FACE_ADJ_PLANES + 7;  // + the primitives W

template <int AXIS>
__device__ __forceinline__ void line_cell(const DevParams &p, int l, int pos, int &c)
{
    c = AXIS == 0 ? l * p.nx + pos : pos * p.nx + l;
}

__device__ __forceinline__ void prims_v(const DevParams &p, const double *q, double *w)
{
    double a2 = q[7], a1 = 1.0 - a2;
    double rho = q[0] + q[1];
    w[0] = a2;
    w[1] = q[0];
    w[2] = q[1];
    w[3] = q[2] / rho;
    w[4] = q[3] / rho;
    w[5] = sg_p(p, 0, q[4], a1);
    w[6] = sg_p(p, 1, q[5], a2);
}

// minmod operand choice with the forward's rules: 0 zero, 1 first, 2 second
__device__ __forceinline__ int mm_choice(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? 1 : 2;
    if (a < 0.0 && b < 0.0) return a > b ? 1 : 2;
    return 0;
}

// A face state of Eq. (vectorForm) from reconstructed primitives (values, the
// forward's operation order) and its reverse: the adjoints of (q[8], u_n, p,
// c, rho) -> the adjoint of w = (alpha_2, m1, m2, u_n, u_t, p1, p2).
struct FaceV {
    double a2, a1, m1, m2, un, ut, p1, p2, rho, E1, E2, p, A1, A2, X, c;
    double q[NQ];
};

__device__ __forceinline__ void face_fwd(const DevParams &p, const double *w, FaceV &s)
{
    s.a2 = w[0];
    s.a1 = 1.0 - s.a2;
    s.m1 = w[1];
    s.m2 = w[2];
    s.un = w[3];
    s.ut = w[4];
    s.p1 = w[5];
    s.p2 = w[6];
    s.rho = s.m1 + s.m2;
    s.E1 = sg_E(p, 0, s.p1, s.a1);
    s.E2 = sg_E(p, 1, s.p2, s.a2);
    s.p = s.a1 * s.p1 + s.a2 * s.p2;
    s.A1 = sg_A(p, 0, s.p1);
    s.A2 = sg_A(p, 1, s.p2);
    s.X = s.a1 * s.A1 + s.a2 * s.A2;
    s.c = sqrt(s.X / s.rho);
    s.q[0] = s.m1;
    s.q[1] = s.m2;
    s.q[2] = s.rho * s.un;
    s.q[3] = s.rho * s.ut;
    s.q[4] = s.E1;
    s.q[5] = s.E2;
    s.q[6] = s.E1 + s.E2 + 0.5 * s.rho * (s.un * s.un + s.ut * s.ut);
    s.q[7] = s.a2;
}

// qb: adjoint of q[8]; unb, utb, pb, cb, rhob: direct adjoints of u_n, u_t, p,
// c, rho
__device__ __forceinline__ void face_rev(const DevParams &p, const FaceV &s, const double *qb, double unb,
                                         double utb, double pb, double cb, double rhob, double *wb)
{
    double m1b = qb[0], m2b = qb[1], E1b = qb[4], E2b = qb[5], a2b = qb[7], a1b = 0.0;
    double p1b = 0.0, p2b = 0.0;
    // q2 = rho un, q3 = rho ut
    rhob += qb[2] * s.un + qb[3] * s.ut;
    unb += qb[2] * s.rho;
    utb += qb[3] * s.rho;
    // q6 = E1 + E2 + rho (un^2 + ut^2)/2
    E1b += qb[6];
    E2b += qb[6];
    rhob += qb[6] * 0.5 * (s.un * s.un + s.ut * s.ut);
    unb += qb[6] * s.rho * s.un;
    utb += qb[6] * s.rho * s.ut;
    // c = sqrt(X / rho)
    const double c2b = cb / (2.0 * s.c);
    const double ir = 1.0 / s.rho;
    const double Xb = c2b * ir;
    rhob -= c2b * (s.X * ir) * ir;
    a1b += Xb * s.A1;
    a2b += Xb * s.A2;
    p1b += Xb * s.a1 * p.g[0];
    p2b += Xb * s.a2 * p.g[1];
    // p = a1 p1 + a2 p2
    a1b += pb * s.p1;
    a2b += pb * s.p2;
    p1b += pb * s.a1;
    p2b += pb * s.a2;
    // E_k = a_k (p_k + g_k pinf_k) / (g_k - 1)
    a1b += E1b * (s.p1 + p.gpinf[0]) * p.inv_gm1[0];
    p1b += E1b * s.a1 * p.inv_gm1[0];
    a2b += E2b * (s.p2 + p.gpinf[1]) * p.inv_gm1[1];
    p2b += E2b * s.a2 * p.inv_gm1[1];
    // rho = m1 + m2, a1 = 1 - a2
    m1b += rhob;
    m2b += rhob;
    a2b -= a1b;
    wb[0] = a2b;
    wb[1] = m1b;
    wb[2] = m2b;
    wb[3] = unb;
    wb[4] = utb;
    wb[5] = p1b;
    wb[6] = p2b;
}

// The HLLC flux of the face (the forward's branch rules) and its reverse:
// gF = adjoint of (F[0..7], u*) -> adjoints of wl and wr; returns u*.
__device__ __forceinline__ double face_reverse(const DevParams &p, const double *wl, const double *wr,
                                               const double *gF, double *wlb, double *wrb)
{
    FaceV L, R;
    face_fwd(p, wl, L);
    face_fwd(p, wr, R);
    const double sl1 = L.un - L.c, sl2 = R.un - R.c, sr1 = L.un + L.c, sr2 = R.un + R.c;
    const bool slR = sl2 < sl1, srR = sr2 > sr1;
    const double SL = slR ? sl2 : sl1, SR = srR ? sr2 : sr1;
    const double num = R.p - L.p + L.rho * L.un * (SL - L.un) - R.rho * R.un * (SR - R.un);
    const double den = L.rho * (SL - L.un) - R.rho * (SR - R.un);
    const double Ss = num / den;
    const int region = 0.0 <= SL ? 0 : (0.0 <= SR ? (0.0 <= Ss ? 1 : 2) : 3);
    double qb_L[NQ], qb_R[NQ];
#pragma unroll
    for (int k = 0; k < NQ; k++) qb_L[k] = qb_R[k] = 0.0;
    double unLb = 0.0, unRb = 0.0, pLb = 0.0, pRb = 0.0, cLb = 0.0, cRb = 0.0, rhoLb = 0.0, rhoRb = 0.0;
    double us;
    if (region == 0 || region == 3) {
        const FaceV &K = region == 0 ? L : R;
        us = K.un;
        double *qbK = region == 0 ? qb_L : qb_R;
        double usb = gF[8] + gF[6] * (K.q[6] + K.p);
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            qbK[k] = gF[k] * us;
            if (k != 6) usb += gF[k] * K.q[k];
        }
        // F2 = u* q2 + p*, F6 = u* (q6 + p*)
        const double psb = gF[2] + gF[6] * us;
        if (region == 0) { unLb += usb; pLb += psb; }
        else { unRb += usb; pRb += psb; }
        face_rev(p, L, qb_L, unLb, 0.0, pLb, cLb, rhoLb, wlb);
        face_rev(p, R, qb_R, unRb, 0.0, pRb, cRb, rhoRb, wrb);
        return us;
    } else {
        const bool kl = region == 1;
        const FaceV &K = kl ? L : R;
        const double SK = kl ? SL : SR;
        const double t = SK - K.un, d2 = SK - Ss, chi = t / d2;
        const double e = Ss - K.un, fv = K.rho * Ss + K.p / t, gv = K.q[6] + e * fv;
        double q[NQ];
        q[0] = chi * K.q[0];
        q[1] = chi * K.q[1];
        q[2] = chi * K.rho * Ss;
        q[3] = chi * K.rho * K.ut;
        q[4] = chi * K.q[4];
        q[5] = chi * K.q[5];
        q[6] = chi * gv;
        q[7] = K.a2;
        us = Ss;
        const double ps = K.p + K.rho * t * e;
        // flux
        double qs_b[NQ];
        double usb = gF[8] + gF[6] * (q[6] + ps);
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            qs_b[k] = gF[k] * us;
            if (k != 6) usb += gF[k] * q[k];
        }
        const double psb = gF[2] + gF[6] * us;
        // star state
        double *qbK = kl ? qb_L : qb_R;
        double rhoKb = 0.0, unKb = 0.0, utKb = 0.0, pKb = 0.0, Ssb = usb, tb = 0.0;
        const double chib = qs_b[0] * K.q[0] + qs_b[1] * K.q[1] + qs_b[2] * K.rho * Ss + qs_b[3] * K.rho * K.ut +
                            qs_b[4] * K.q[4] + qs_b[5] * K.q[5] + qs_b[6] * gv;
        qbK[0] += qs_b[0] * chi;
        qbK[1] += qs_b[1] * chi;
        qbK[4] += qs_b[4] * chi;
        qbK[5] += qs_b[5] * chi;
        rhoKb += qs_b[2] * chi * Ss + qs_b[3] * chi * K.ut;
        Ssb += qs_b[2] * chi * K.rho;
        utKb += qs_b[3] * chi * K.rho;
        const double gb = qs_b[6] * chi;
        qbK[6] += gb;
        const double eb1 = gb * fv, fb = gb * e;
        rhoKb += fb * Ss;
        Ssb += fb * K.rho;
        const double it = 1.0 / t;
        pKb += fb * it;
        tb -= fb * K.p * it * it;
        Ssb += eb1;
        unKb -= eb1;
        qbK[7] += qs_b[7];
        // ps = pK + rhoK t e
        pKb += psb;
        rhoKb += psb * t * e;
        tb += psb * K.rho * e;
        const double eb2 = psb * K.rho * t;
        Ssb += eb2;
        unKb -= eb2;
        // chi = t / d2, d2 = SK - Ss, t = SK - unK
        const double id2 = 1.0 / d2;
        const double d1b = chib * id2, d2b = -chib * chi * id2;
        tb += d1b;
        double SKb = d2b + tb;
        Ssb -= d2b;
        unKb -= tb;
        // Ss = num / den
        const double iden = 1.0 / den;
        const double numb = Ssb * iden, denb = -Ssb * Ss * iden;
        double SLb = 0.0, SRb = 0.0;
        pRb += numb;
        pLb -= numb;
        rhoLb += numb * L.un * (SL - L.un) + denb * (SL - L.un);
        unLb += numb * L.rho * (SL - 2.0 * L.un) - denb * L.rho;
        SLb += numb * L.rho * L.un + denb * L.rho;
        rhoRb -= numb * R.un * (SR - R.un) + denb * (SR - R.un);
        unRb -= numb * R.rho * (SR - 2.0 * R.un) - denb * R.rho;
        SRb -= numb * R.rho * R.un + denb * R.rho;
        if (kl) SLb += SKb;
        else SRb += SKb;
        if (kl) { rhoLb += rhoKb; unLb += unKb; pLb += pKb; }
        else { rhoRb += rhoKb; unRb += unKb; pRb += pKb; }
        // Davis bounds: the operand each of S_L, S_R took
        if (slR) { unRb += SLb; cRb -= SLb; }
        else { unLb += SLb; cLb -= SLb; }
        if (srR) { unRb += SRb; cRb += SRb; }
        else { unLb += SRb; cLb += SRb; }
        face_rev(p, L, qb_L, unLb, kl ? utKb : 0.0, pLb, cLb, rhoLb, wlb);
        face_rev(p, R, qb_R, unRb, kl ? 0.0 : utKb, pRb, cRb, rhoRb, wrb);
        return us;
    }
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_adj_sweep_prims(const DevParams p, const double *Uin, double *Wp)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int gmap[NQ] = {0, 1, QN, QT, 4, 5, 6, 7};
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        double q[NQ], w[7];
#pragma unroll
        for (int j = 0; j < NQ; j++) q[j] = Uin[gmap[j] * n + c];
        prims_v(p, q, w);
#pragma unroll
        for (int j = 0; j < 7; j++) Wp[(size_t)j * n + c] = w[j];
    }
}

template <int AXIS>
__global__ void __launch_bounds__(128) k_adj_sweep_face(const DevParams p, const double *Wp, const double *Gout,
                                                        double *fw, double dtdx)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int gmap[NQ] = {0, 1, QN, QT, 4, 5, 6, 7};
    const int n = p.n;
    const int len = AXIS == 0 ? p.nx : p.ny, nlines = AXIS == 0 ? p.ny : p.nx;
    const int nf = (len + 1) * nlines;
    const int bc = p.bc[AXIS];
    const bool lim = p.limiter != DIM_LIMITER_NONE, ob = p.limiter == DIM_LIMITER_OVERBEE;
    GRID_LOOP(fid, nf)
    {
        const int l = fid / (len + 1), f = fid - l * (len + 1);
        double W[4][7];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int c;
            line_cell<AXIS>(p, l, line_map(f - 2 + k, len, bc), c);
#pragma unroll
            for (int j = 0; j < 7; j++) W[k][j] = Wp[(size_t)j * n + c];
        }
        // reconstruction (values and limiter choices as in the forward)
        double wl[7], wr[7];
        int cl[7], cr[7];
#pragma unroll
        for (int j = 0; j < 7; j++) {
            if (lim) {
                const double dml = W[1][j] - W[0][j], dpl = W[2][j] - W[1][j];
                const double dmr = W[2][j] - W[1][j], dpr = W[3][j] - W[2][j];
                cl[j] = mm_choice(dml, dpl);
                cr[j] = mm_choice(dmr, dpr);
                double sl = cl[j] == 1 ? dml : (cl[j] == 2 ? dpl : 0.0);
                double sr = cr[j] == 1 ? dmr : (cr[j] == 2 ? dpr : 0.0);
                if (ob && j <= 2) {
                    sl = 2.0 * sl;
                    sr = 2.0 * sr;
                }
                wl[j] = W[1][j] + 0.5 * sl;
                wr[j] = W[2][j] - 0.5 * sr;
            } else {
                cl[j] = cr[j] = 0;
                wl[j] = W[1][j];
                wr[j] = W[2][j];
            }
        }
        // adjoint of the face outputs: cells f-1 (plus face) and f (minus face)
        double gF[9];
        {
            double rL = 0.0, rR = 0.0;
#pragma unroll
            for (int o = 0; o < NQ; o++) gF[o] = 0.0;
            if (f - 1 >= 0) {
                int c;
                line_cell<AXIS>(p, l, f - 1, c);
                double lam[NQ];
#pragma unroll
                for (int o = 0; o < NQ; o++) lam[o] = Gout[gmap[o] * n + c];
#pragma unroll
                for (int o = 0; o < NQ; o++) gF[o] -= lam[o];
                const double a2 = W[1][0], a1 = 1.0 - a2;
                rL = lam[4] * (a1 * W[1][5]) + lam[5] * (a2 * W[1][6]) - lam[7] * a2;
            }
            if (f < len) {
                int c;
                line_cell<AXIS>(p, l, f, c);
                double lam[NQ];
#pragma unroll
                for (int o = 0; o < NQ; o++) lam[o] = Gout[gmap[o] * n + c];
#pragma unroll
                for (int o = 0; o < NQ; o++) gF[o] += lam[o];
                const double a2 = W[2][0], a1 = 1.0 - a2;
                rR = lam[4] * (a1 * W[2][5]) + lam[5] * (a2 * W[2][6]) - lam[7] * a2;
            }
#pragma unroll
            for (int o = 0; o < NQ; o++) gF[o] *= dtdx;
            gF[8] = dtdx * (rR - rL);
        }
        double wlb[7], wrb[7];
        fw[28 * (size_t)nf + fid] = face_reverse(p, wl, wr, gF, wlb, wrb);
        // transposed reconstruction
        double Wb[4][7];
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 7; j++) Wb[k][j] = 0.0;
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const double h = (ob && j <= 2) ? 1.0 : 0.5;
            // wl = W1 + h * (chosen slope)
            if (cl[j] == 1) { Wb[1][j] += wlb[j] * (1.0 + h); Wb[0][j] -= h * wlb[j]; }
            else if (cl[j] == 2) { Wb[1][j] += wlb[j] * (1.0 - h); Wb[2][j] += h * wlb[j]; }
            else Wb[1][j] += wlb[j];
            // wr = W2 - h * (chosen slope)
            if (cr[j] == 1) { Wb[2][j] += wrb[j] * (1.0 - h); Wb[1][j] += h * wrb[j]; }
            else if (cr[j] == 2) { Wb[2][j] += wrb[j] * (1.0 + h); Wb[3][j] -= h * wrb[j]; }
            else Wb[2][j] += wrb[j];
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 7; j++) fw[(size_t)(7 * k + j) * nf + fid] = Wb[k][j];
    }
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_adj_sweep_cell(const DevParams p, const double *Uin, const double *Gout,
                                                        const double *fw, double *Gin, double dtdx)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int gmap[NQ] = {0, 1, QN, QT, 4, 5, 6, 7};
    const int n = p.n;
    const int len = AXIS == 0 ? p.nx : p.ny, nlines = AXIS == 0 ? p.ny : p.nx;
    const int nf = (len + 1) * nlines;
    const int bc = p.bc[AXIS];
    GRID_LOOP(c, n)
    {
        const int x = c % p.nx, y = c / p.nx;
        const int i = AXIS == 0 ? x : y, l = AXIS == 0 ? y : x;
        const int fbase = l * (len + 1);
        double Wb[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        // faces whose stencil may contain line position i (windows shifted by
        // the period for a periodic axis; every face of a short line)
        const int nwin = len <= 8 ? 1 : (bc == DIM_BC_PERIODIC ? 3 : 1);
        for (int w = 0; w < nwin; w++) {
            int f0, f1;
            if (len <= 8) { f0 = 0; f1 = len; }
            else {
                const int sh = w == 0 ? 0 : (w == 1 ? len : -len);
                f0 = max(i - 1 + sh, 0);
                f1 = min(i + 2 + sh, len);
            }
            for (int f = f0; f <= f1; f++) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (line_map(f - 2 + k, len, bc) != i) continue;
#pragma unroll
                    for (int j = 0; j < 7; j++) Wb[j] += fw[(size_t)(7 * k + j) * nf + fbase + f];
                }
            }
        }
        double q[NQ], lam[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            q[k] = Uin[gmap[k] * n + c];
            lam[k] = Gout[gmap[k] * n + c];
        }
        // transposed Jacobian of q -> W (line-local order), by hand:
        // W = (a2, m1, m2, q2/rho, q3/rho, (g1-1) E1/a1 - g1 pinf1, (g2-1) E2/a2 - g2 pinf2)
        double acc[NQ];
        {
            const double a2 = q[7], a1 = 1.0 - a2, ir = 1.0 / (q[0] + q[1]);
            const double ia1 = 1.0 / a1, ia2 = 1.0 / a2;
            const double u = q[2] * ir, v = q[3] * ir;
            const double rhob = -(Wb[3] * u + Wb[4] * v) * ir;
            const double e1 = Wb[5] * p.gm1[0] * ia1, e2 = Wb[6] * p.gm1[1] * ia2;
            acc[0] = lam[0] + Wb[1] + rhob;
            acc[1] = lam[1] + Wb[2] + rhob;
            acc[2] = lam[2] + Wb[3] * ir;
            acc[3] = lam[3] + Wb[4] * ir;
            acc[4] = lam[4] + e1;
            acc[5] = lam[5] + e2;
            acc[6] = lam[6];
            // d p1/d a2 = +(g1-1) E1/a1^2 (a1 = 1 - a2), d p2/d a2 = -(g2-1) E2/a2^2
            acc[7] = lam[7] + Wb[0] + e1 * q[4] * ia1 - e2 * q[5] * ia2;
        }
        // R(U_i) (u*_{i+1/2} - u*_{i-1/2}): R.lam = lam4 a1 p1 + lam5 a2 p2 - lam7 a2,
        // a_k p_k = (g_k-1) E_k - a_k g_k pinf_k
        const double du = dtdx * (fw[28 * (size_t)nf + fbase + i + 1] - fw[28 * (size_t)nf + fbase + i]);
        acc[4] -= du * lam[4] * p.gm1[0];
        acc[5] -= du * lam[5] * p.gm1[1];
        acc[7] -= du * (lam[4] * p.gpinf[0] - lam[5] * p.gpinf[1] - lam[7]);
#pragma unroll
        for (int k = 0; k < NQ; k++) Gin[gmap[k] * n + c] = acc[k];
    }
}

// ---------------------------------------------------------------------------
// viscous stage along one axis (Sec. 3.2)
// ---------------------------------------------------------------------------
// coefficient planes: V = 1/rho, mu = a1 mu1 + a2 mu2, u0 = rho u_n / rho,
// w0 = rho u_t / rho
template <int AXIS>
__global__ void __launch_bounds__(256) k_adj_visc_prep(const DevParams p, const double *Uin, double *V, double *mu,
                                                       double *u0, double *w0)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        double rho = Uin[c] + Uin[n + c];
        double a2 = Uin[7 * n + c];
        V[c] = 1.0 / rho;
        mu[c] = (1.0 - a2) * p.mu[0] + a2 * p.mu[1];
        u0[c] = Uin[QN * n + c] / rho;
        w0[c] = Uin[QT * n + c] / rho;
    }
}

// the contribution of face (l, r) to J through the conservative last sweep:
// S = sum over s in {l (+), r (-)} of sign_s tau/h [G_s^n Fn + G_s^t Ft +
//     G_s^E W + (G_s^E1 aF1 + G_s^E2 aF2)(W - uh_s Fn - wh_s Ft)]
// with inputs x = (uh_l, uh_r, wh_l, wh_r, a_l, a_r, mu_l, mu_r); xb = dS/dx
// by the hand-written reverse (ih = 1/h; the factor tau/h of the update is
// folded into Gl, Gr by the caller)
__device__ __forceinline__ void visc_face_J(const double *x, const double *Gl, const double *Gr, double ih,
                                            double *xb)
{
    const double ul = x[0], ur = x[1], wl = x[2], wr = x[3], al = x[4], ar = x[5], ml = x[6], mr = x[7];
    // forward values
    const double lnf = 0.5 * (4.0 / 3.0 * ml + 4.0 / 3.0 * mr);
    const double lmf = 0.5 * (ml + mr);
    const double Fn = lnf * (ur - ul) * ih;
    const double Ft = lmf * (wr - wl) * ih;
    const double um = 0.5 * (ul + ur), wm = 0.5 * (wl + wr);
    const double W = um * Fn + wm * Ft;
    const double aF2 = 0.5 * (al + ar);
    const double aF1 = 0.5 * ((1.0 - al) + (1.0 - ar));
    // Gl/Gr: (G^n, G^t, G^E, G^E1, G^E2) of the two cells, each already times tau/h
    const double Kl = Gl[3] * aF1 + Gl[4] * aF2, Kr = Gr[3] * aF1 + Gr[4] * aF2;
    const double Dl = W - ul * Fn - wl * Ft, Dr = W - ur * Fn - wr * Ft;
    // reverse of S = Sl - Sr
    const double Dlb = Kl, Drb = -Kr;
    const double Wb = Gl[2] - Gr[2] + Dlb + Drb;
    const double Fnb = Gl[0] - Gr[0] - Dlb * ul - Drb * ur + Wb * um;
    const double Ftb = Gl[1] - Gr[1] - Dlb * wl - Drb * wr + Wb * wm;
    const double aF1b = Dl * Gl[3] - Dr * Gr[3], aF2b = Dl * Gl[4] - Dr * Gr[4];
    const double umb = Wb * Fn, wmb = Wb * Ft;
    const double fu = Fnb * lnf * ih, fw = Ftb * lmf * ih;
    xb[0] = -Dlb * Fn + 0.5 * umb - fu;
    xb[1] = -Drb * Fn + 0.5 * umb + fu;
    xb[2] = -Dlb * Ft + 0.5 * wmb - fw;
    xb[3] = -Drb * Ft + 0.5 * wmb + fw;
    xb[4] = xb[5] = 0.5 * aF2b - 0.5 * aF1b;
    const double lnfb = Fnb * (ur - ul) * ih, lmfb = Ftb * (wr - wl) * ih;
    xb[6] = xb[7] = lnfb * (0.5 * (4.0 / 3.0)) + 0.5 * lmfb;
}

template <int AXIS>
__global__ void __launch_bounds__(128) k_adj_visc_final(const DevParams p, const double *G, const double *A2,
                                                        const double *mu, const double *uh, const double *wh,
                                                        double *Gin, double *ub, double *wb, double *ab,
                                                        double *mub, double tau)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int n = p.n;
    const double ih = AXIS == 0 ? 1.0 / p.dx : 1.0 / p.dy;
    const double tih = tau * ih;
    GRID_LOOP(c, n)
    {
        int cm, cp;
        axis_nb(p, AXIS, c, cm, cp);
        double su = 0.0, sw = 0.0, sa = 0.0, sm = 0.0;
        for (int sd = 0; sd < 2; sd++) {
            const int nb = sd == 0 ? cm : cp;
            if (nb < 0) continue;
            const int l = sd == 0 ? cm : c, r = sd == 0 ? c : cp;
            double x[8] = {uh[l], uh[r], wh[l], wh[r], A2[l], A2[r], mu[l], mu[r]};
            double Gl[5] = {tih * G[QN * n + l], tih * G[QT * n + l], tih * G[6 * n + l], tih * G[4 * n + l],
                            tih * G[5 * n + l]};
            double Gr[5] = {tih * G[QN * n + r], tih * G[QT * n + r], tih * G[6 * n + r], tih * G[4 * n + r],
                            tih * G[5 * n + r]};
            double xb[8];
            visc_face_J(x, Gl, Gr, ih, xb);
            // this cell is r of the minus face, l of the plus face
            const int o = sd == 0 ? 1 : 0;
            su += xb[0 + o];
            sw += xb[2 + o];
            sa += xb[4 + o];
            sm += xb[6 + o];
        }
#pragma unroll
        for (int k = 0; k < NQ; k++) Gin[k * n + c] = G[k * n + c];
        ub[c] = su;
        wb[c] = sw;
        ab[c] = sa;
        mub[c] = sm;
    }
}

// one reverse LIM sweep of both velocity fields; uprev/wprev = u^{m-1}, w^{m-1}
template <int AXIS>
__global__ void __launch_bounds__(256) k_adj_visc_lim(const DevParams p, const double *V, const double *mu,
                                                      const double *uprev, const double *wprev, const double *ubi,
                                                      const double *wbi, double *ubo, double *wbo, double *u0b,
                                                      double *w0b, double *Vb, double *mub, double tau, double bm,
                                                      double rden)
{
    const int n = p.n;
    const double ih2 = AXIS == 0 ? p.idx2 : p.idy2;
    GRID_LOOP(c, n)
    {
        int cm, cp;
        axis_nb(p, AXIS, c, cm, cp);
        const double mc = mu[c];
        const double yu = rden * ubi[c], yw = rden * wbi[c];
        const double zu = V[c] * yu, zw = V[c] * yw;
        double lu = 0.0, lw = 0.0;      // L(V y) at c
        double Lup = 0.0, Lwp = 0.0;    // L(u^{m-1}) at c
        double mb = 0.0;
        for (int sd = 0; sd < 2; sd++) {
            const int nb = sd == 0 ? cm : cp;
            if (nb < 0) continue;
            const double mn = mu[nb];
            const double lnf = 0.5 * (4.0 / 3.0 * mn + 4.0 / 3.0 * mc), lmf = 0.5 * (mn + mc);
            const double zun = V[nb] * (rden * ubi[nb]), zwn = V[nb] * (rden * wbi[nb]);
            lu += lnf * (zun - zu) * ih2;
            lw += lmf * (zwn - zw) * ih2;
            const double du = uprev[nb] - uprev[c], dw = wprev[nb] - wprev[c];
            Lup += lnf * du * ih2;
            Lwp += lmf * dw * ih2;
            // face coefficient adjoints tau (z_c - z_nb)(u_nb - u_c)/h^2, half to this cell
            const double lnb = tau * (zu - zun) * du * ih2, lmb = tau * (zw - zwn) * dw * ih2;
            mb += 0.5 * (4.0 / 3.0) * lnb + 0.5 * lmb;
        }
        ubo[c] = tau * bm * yu + tau * lu;
        wbo[c] = tau * bm * yw + tau * lw;
        u0b[c] += yu;
        w0b[c] += yw;
        Vb[c] += tau * (yu * Lup + yw * Lwp);
        mub[c] += mb;
    }
}

// V = 1/rho, u0 = rho u_n / rho, w0, mu = a1 mu1 + a2 mu2 -> G
template <int AXIS>
__global__ void __launch_bounds__(256) k_adj_visc_coef(const DevParams p, const double *Uin, const double *u0,
                                                       const double *w0, const double *u0b, const double *w0b,
                                                       const double *ub0, const double *wb0, const double *Vb,
                                                       const double *mub, const double *ab, double *Gin, double *pbar)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const int n = p.n;
    double s2 = 0.0, s3 = 0.0;
    GRID_LOOP(c, n)
    {
        const double rho = Uin[c] + Uin[n + c], a2 = Uin[7 * n + c];
        const double V = 1.0 / rho;
        const double ubt = u0b[c] + ub0[c], wbt = w0b[c] + wb0[c];
        Gin[QN * n + c] += ubt / rho;
        Gin[QT * n + c] += wbt / rho;
        const double rb = -(ubt * u0[c] + wbt * w0[c]) / rho - Vb[c] * V * V;
        Gin[c] += rb;
        Gin[n + c] += rb;
        Gin[7 * n + c] += ab[c] + mub[c] * (p.mu[1] - p.mu[0]);
        s2 += mub[c] * (1.0 - a2);
        s3 += mub[c] * a2;
    }
    add_param(pbar, 2, s2);
    add_param(pbar, 3, s3);
}

// ---------------------------------------------------------------------------
// heat-conduction stage (Sec. 3.4.2, Algorithm 1 with the LIM)
// ---------------------------------------------------------------------------
// (L v)_c with face coefficient the mean of the two cells' Lam (Eq. qk_dis)
__device__ __forceinline__ double lap_v(const DevParams &p, int c, const double *v, const double *L)
{
    double r = 0.0;
    const double vc = v[c], Lc = L[c];
    for (int ax = 0; ax < 2; ax++) {
        int cm, cp;
        axis_nb(p, ax, c, cm, cp);
        const double ih2 = ax == 0 ? p.idx2 : p.idy2;
        const double fl = cm >= 0 ? 0.5 * (L[cm] + Lc) * (vc - v[cm]) * ih2 : 0.0;
        const double fr = cp >= 0 ? 0.5 * (Lc + L[cp]) * (v[cp] - vc) * ih2 : 0.0;
        r += fr - fl;
    }
    return r;
}

// sum over the faces of c of (a_c - a_nb)(v_nb - v_c)/h^2: half of it is the
// adjoint of Lam_c through the two-cell face means
__device__ __forceinline__ double face_lam_adj(const DevParams &p, int c, const double *a, const double *v)
{
    double s = 0.0;
    for (int ax = 0; ax < 2; ax++) {
        int cm, cp;
        axis_nb(p, ax, c, cm, cp);
        const double ih2 = ax == 0 ? p.idx2 : p.idy2;
        if (cm >= 0) s += (a[c] - a[cm]) * (v[cm] - v[c]) * ih2;
        if (cp >= 0) s += (a[c] - a[cp]) * (v[cp] - v[c]) * ih2;
    }
    return s;
}

// T0 = mixture temperature of the stage input; T0bar cleared
__global__ void __launch_bounds__(256) k_adj_heat_prep(const DevParams p, const double *Uin, double *T0, double *T0b)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        T0[c] = mixture_T(p, Uin[c], Uin[n + c], Uin[4 * n + c], Uin[5 * n + c], Uin[7 * n + c]);
        T0b[c] = 0.0;
    }
}

// frozen coefficients of one outer iteration from its (T_it, a_it)
__global__ void __launch_bounds__(256) k_adj_heat_coef_fwd(const DevParams p, const double *Uin, const double *Tit,
                                                           const double *ait, double *V, double *L, double *Ia)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        double v, l;
        heat_coeffs(p, Uin[c], Uin[n + c], Tit[c], ait[c], v, l);
        V[c] = v;
        L[c] = l;
        Ia[c] = (1.0 - ait[c]) * p.src[0] + ait[c] * p.src[1];
    }
}

// adjoint through (T, a) = equilibrium(m1, m2, rho e0 + tau q) of one outer
// iteration; last: the iteration whose result is the stage output
// (E_k = m_k Cv_k T + a_k pinf_k, rho E = rho E0 + tau q, alpha_2 = a)
__global__ void __launch_bounds__(256) k_adj_heat_eq(const DevParams p, const double *Uin, const double *G,
                                                     const double *vM, const double *L, const double *Ia,
                                                     const double *Tb, const double *ab, double *Gin, double *qb,
                                                     double tau, int last)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        const double m1v = Uin[c], m2v = Uin[n + c];
        const double q = lap_v(p, c, vM, L) + Ia[c];
        const EqState eq = eq_fwd(p, m1v, m2v, Uin[4 * n + c] + Uin[5 * n + c] + tau * q);
        double tb, abr, g0 = 0.0, g1 = 0.0, qbc = 0.0;
        if (last) {
            const double g4 = G[4 * n + c], g5 = G[5 * n + c];
            tb = g4 * m1v * p.cv[0] + g5 * m2v * p.cv[1];
            abr = -g4 * p.pinf[0] + g5 * p.pinf[1] + G[7 * n + c];
            g0 = g4 * p.cv[0] * eq.T;
            g1 = g5 * p.cv[1] * eq.T;
            qbc = tau * G[6 * n + c];
#pragma unroll
            for (int k = 0; k < 4; k++) Gin[k * n + c] = G[k * n + c];
            Gin[6 * n + c] = G[6 * n + c];
            Gin[4 * n + c] = 0.0;
            Gin[5 * n + c] = 0.0;
            Gin[7 * n + c] = 0.0;
        } else {
            tb = Tb[c];
            abr = ab[c];
        }
        double m1b, m2b, rb;
        eq_rev(p, eq, tb, abr, m1b, m2b, rb);
        Gin[c] += g0 + m1b;
        Gin[n + c] += g1 + m2b;
        // rho e0 = E1 + E2
        Gin[4 * n + c] += rb;
        Gin[5 * n + c] += rb;
        qb[c] = qbc + tau * rb;
    }
}

// q = L(v^M) + Ia: vbar^M = L(qbar) (L symmetric), Lam and Ia adjoints
__global__ void __launch_bounds__(256) k_adj_heat_q(const DevParams p, const double *qb, const double *vM,
                                                    const double *L, double *vb, double *Lb, double *Iab, double *Vb)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        vb[c] = lap_v(p, c, qb, L);
        Lb[c] = 0.5 * face_lam_adj(p, c, qb, vM);
        Iab[c] = qb[c];
        Vb[c] = 0.0;
    }
}

// face coefficients of the frozen operator times 1/h^2: Lx[c] = (Lam_c +
// Lam_{c+x})/2 / dx^2 at the face after c (0 at a wall), Ly likewise
__global__ void __launch_bounds__(256) k_adj_heat_faces(const DevParams p, const double *L, double *Lx, double *Ly)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        int cm, cp;
        axis_nb(p, 0, c, cm, cp);
        Lx[c] = cp >= 0 ? 0.5 * (L[c] + L[cp]) * p.idx2 : 0.0;
        axis_nb(p, 1, c, cm, cp);
        Ly[c] = cp >= 0 ? 0.5 * (L[c] + L[cp]) * p.idy2 : 0.0;
    }
}

// z = V (vbar / (1 + tau b)) of the first reverse sweep
__global__ void __launch_bounds__(256) k_adj_heat_z(const DevParams p, const double *V, const double *vb, double *z,
                                                    double rden)
{
    const int n = p.n;
    GRID_LOOP(c, n) z[c] = V[c] * (rden * vb[c]);
}

// one reverse predictor sweep: vprev = v^{m-1}; y = vbar^m / (1 + tau b_m),
// z = V y (formed by the previous sweep for every cell); writes vbar^{m-1} and
// the next sweep's z (rden_next = 1/(1 + tau b_{m-1}))
__global__ void __launch_bounds__(256) k_adj_heat_lim(const DevParams p, const double *V, const double *Lx,
                                                      const double *Ly, const double *Ia, const double *vprev,
                                                      const double *vbi, const double *z, double *vbo, double *znext,
                                                      double *T0b, double *Vb, double *Lb, double *Iab, double tau,
                                                      double bm, double rden, double rden_next)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        const double y = rden * vbi[c], zc = z[c], vc = vprev[c];
        double lz = 0.0, lv = 0.0, fl = 0.0;
        for (int ax = 0; ax < 2; ax++) {
            int cm, cp;
            axis_nb(p, ax, c, cm, cp);
            const double *Lf = ax == 0 ? Lx : Ly;
            const double ih2 = ax == 0 ? p.idx2 : p.idy2;
            double fa = 0.0;
            if (cm >= 0) {
                const double f = Lf[cm], dz = z[cm] - zc, dv = vprev[cm] - vc;
                lz += f * dz;
                lv += f * dv;
                fa -= dz * dv;
            }
            if (cp >= 0) {
                const double f = Lf[c], dz = z[cp] - zc, dv = vprev[cp] - vc;
                lz += f * dz;
                lv += f * dv;
                fa -= dz * dv;
            }
            fl += fa * ih2;
        }
        const double vb = tau * bm * y + tau * lz;
        vbo[c] = vb;
        znext[c] = V[c] * (rden_next * vb);
        T0b[c] += y;
        Vb[c] += tau * y * (lv + Ia[c]);
        Lb[c] += 0.5 * tau * fl;
        Iab[c] += tau * V[c] * y;
    }
}

// coefficients (V, Lam, Ia) at (m1, m2, T_it, a_it) -> m1, m2 and (T_it, a_it);
// first: iteration 0, whose (T, a) are the stage input's (T0, alpha_2)
__global__ void __launch_bounds__(256) k_adj_heat_coef(const DevParams p, const double *Uin, const double *Tit,
                                                       const double *ait, const double *Vb, const double *Lb,
                                                       const double *Iab, const double *vb0, double *T0b, double *Tb,
                                                       double *ab, double *Gin, double *pbar, int first)
{
    const int n = p.n;
    double sk0 = 0.0, sk1 = 0.0, si0 = 0.0, si1 = 0.0;
    GRID_LOOP(c, n)
    {
        Dn<4> m1 = dseed<4>(Uin[c], 0), m2 = dseed<4>(Uin[n + c], 1);
        Dn<4> T = dseed<4>(Tit[c], 2), a = dseed<4>(ait[c], 3);
        Dn<4> V, L, I;
        d_heat_coeffs(p, m1, m2, T, a, V, L, I);
        const double vb = Vb[c], lb = Lb[c], ib = Iab[c];
        double g[4];
#pragma unroll
        for (int k = 0; k < 4; k++) g[k] = vb * V.d[k] + lb * L.d[k] + ib * I.d[k];
        Gin[c] += g[0];
        Gin[n + c] += g[1];
        // the LIM start v^0 = T0: its adjoint after the reverse sweeps
        T0b[c] += vb0[c];
        if (first) {
            T0b[c] += g[2];
            Gin[7 * n + c] += g[3];
        } else {
            Tb[c] = g[2];
            ab[c] = g[3];
        }
        const double r = law_ratio(p, Tit[c]);
        sk0 += lb * (1.0 - ait[c]) * r;
        sk1 += lb * ait[c] * r;
        si0 += ib * (1.0 - ait[c]);
        si1 += ib * ait[c];
    }
    add_param(pbar, 0, sk0);
    add_param(pbar, 1, sk1);
    add_param(pbar, 4, si0);
    add_param(pbar, 5, si1);
}

// T0 = (E1 + E2 - a1 pinf_1 - a2 pinf_2)/(m1 Cv_1 + m2 Cv_2) -> G
__global__ void __launch_bounds__(256) k_adj_heat_T0(const DevParams p, const double *Uin, const double *T0b,
                                                     double *Gin)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        const double m1 = Uin[c], m2 = Uin[n + c], a2 = Uin[7 * n + c];
        const double C = m1 * p.cv[0] + m2 * p.cv[1];
        const double T = mixture_T(p, m1, m2, Uin[4 * n + c], Uin[5 * n + c], a2);
        const double tb = T0b[c];
        const double w = tb / C;
        Gin[c] += -w * T * p.cv[0];
        Gin[n + c] += -w * T * p.cv[1];
        Gin[4 * n + c] += w;
        Gin[5 * n + c] += w;
        Gin[7 * n + c] += w * (p.pinf[0] - p.pinf[1]);
    }
}

// ---------------------------------------------------------------------------
// initial data: primbar = (dU/dprim)^T Ubar of the conversion (alpha_2, p, T,
// u, v) -> U with both phases at (p, T) (Eqs. eos_stiffened, eos_stiffened2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_from_primitive(const DevParams p, const double *prim,
                                                            const double *Ub, double *pb)
{
    const int n = p.n;
    GRID_LOOP(c, n)
    {
        Dn<5> a2 = dseed<5>(prim[c], 0), pr = dseed<5>(prim[n + c], 1), T = dseed<5>(prim[2 * n + c], 2);
        Dn<5> u = dseed<5>(prim[3 * n + c], 3), v = dseed<5>(prim[4 * n + c], 4);
        Dn<5> a1 = 1.0 - a2;
        Dn<5> rho1 = (pr + p.pinf[0]) / (p.gm1[0] * p.cv[0] * T);
        Dn<5> rho2 = (pr + p.pinf[1]) / (p.gm1[1] * p.cv[1] * T);
        Dn<5> m1 = a1 * rho1, m2 = a2 * rho2, rho = m1 + m2;
        Dn<5> E1 = d_sgE(p, 0, pr, a1), E2 = d_sgE(p, 1, pr, a2);
        Dn<5> out[NQ];
        out[0] = m1;
        out[1] = m2;
        out[2] = rho * u;
        out[3] = rho * v;
        out[4] = E1;
        out[5] = E2;
        out[6] = E1 + E2 + 0.5 * rho * (u * u + v * v);
        out[7] = a2;
        double r[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            const double g = Ub[k * n + c];
#pragma unroll
            for (int j = 0; j < 5; j++) r[j] += g * out[k].d[j];
        }
#pragma unroll
        for (int j = 0; j < 5; j++) pb[j * n + c] = r[j];
    }
}

int grid_for(int n, int threads)
{
    int b = (n + threads - 1) / threads;
    return b < 152 * 16 ? b : 152 * 16;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (stream-ordered, asynchronous)
// ---------------------------------------------------------------------------
cudaError_t adj_prelax(const DevParams &p, const double *Uin, double *G, cudaStream_t s)
{
    k_adj_prelax<<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, G);
    return cudaGetLastError();
}

cudaError_t adj_trelax(const DevParams &p, const double *Uin, double *G, cudaStream_t s)
{
    k_adj_trelax<<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, G);
    return cudaGetLastError();
}

// fw: FACE_ADJ_PLANES x (nx*ny + max(nx, ny)) doubles of workspace
cudaError_t adj_sweep(const DevParams &p, int axis, const double *Uin, const double *Gout, double *Gin, double dtdx,
                      double *fw, cudaStream_t s)
{
    const int len = axis == 0 ? p.nx : p.ny, nlines = axis == 0 ? p.ny : p.nx;
    const int nf = (len + 1) * nlines;
    double *Wp = fw + (size_t)FACE_ADJ_PLANES * nf;  // 7 planes of n <= nf cells
    if (axis == 0) {
        k_adj_sweep_prims<0><<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, Wp);
        k_adj_sweep_face<0><<<grid_for(nf, 128), 128, 0, s>>>(p, Wp, Gout, fw, dtdx);
        k_adj_sweep_cell<0><<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, Gout, fw, Gin, dtdx);
    } else {
        k_adj_sweep_prims<1><<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, Wp);
        k_adj_sweep_face<1><<<grid_for(nf, 128), 128, 0, s>>>(p, Wp, Gout, fw, dtdx);
        k_adj_sweep_cell<1><<<grid_for(p.n, 256), 256, 0, s>>>(p, Uin, Gout, fw, Gin, dtdx);
    }
    return cudaGetLastError();
}

int adj_face_planes() { return FACE_WORK_PLANES; }

// planes of the viscous adjoint: 11 work planes W[0..10] (V, mu, u0, w0, ub x2,
// wb x2, u0b, w0b, Vb) + ab, mub = 13
constexpr int VISC_WORK_PLANES = 13;

// Reverse of one viscous stage.  hist: u^1..u^M, w^1..w^M (M = 2P - 2);
// b[m-1], m = 1..M: the frozen Chebyshev parameters.  G: adjoint of the stage
// output, Gin: adjoint of the stage input (out).  work: 13 planes.
cudaError_t adj_visc(const DevParams &p, int axis, const double *Uin, const double *hist, int M, const double *b,
                     double tau, const double *G, double *Gin, double *work, double *pbar, cudaStream_t s)
{
    const size_t n = (size_t)p.n;
    double *V = work, *mu = work + n, *u0 = work + 2 * n, *w0 = work + 3 * n;
    double *ubA = work + 4 * n, *ubB = work + 5 * n, *wbA = work + 6 * n, *wbB = work + 7 * n;
    double *u0b = work + 8 * n, *w0b = work + 9 * n, *Vb = work + 10 * n, *ab = work + 11 * n, *mub = work + 12 * n;
    const int gb = grid_for(p.n, 256), gb2 = grid_for(p.n, 128);
    cudaError_t e;
    if (axis == 0) k_adj_visc_prep<0><<<gb, 256, 0, s>>>(p, Uin, V, mu, u0, w0);
    else k_adj_visc_prep<1><<<gb, 256, 0, s>>>(p, Uin, V, mu, u0, w0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double *uh = M > 0 ? hist + (size_t)(M - 1) * n : u0;
    const double *wh = M > 0 ? hist + (size_t)(2 * M - 1) * n : w0;
    if (axis == 0) k_adj_visc_final<0><<<gb2, 128, 0, s>>>(p, G, Uin + 7 * n, mu, uh, wh, Gin, ubA, wbA, ab, mub, tau);
    else k_adj_visc_final<1><<<gb2, 128, 0, s>>>(p, G, Uin + 7 * n, mu, uh, wh, Gin, ubA, wbA, ab, mub, tau);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(u0b, 0, 3 * n * sizeof(double), s)) != cudaSuccess) return e;  // u0b, w0b, Vb
    double *ui = ubA, *uo = ubB, *wi = wbA, *wo = wbB;
    for (int m = M; m >= 1; m--) {
        const double bm = b[m - 1], rden = 1.0 / (1.0 + tau * bm);
        const double *up = m >= 2 ? hist + (size_t)(m - 2) * n : u0;
        const double *wp = m >= 2 ? hist + (size_t)(M + m - 2) * n : w0;
        if (axis == 0)
            k_adj_visc_lim<0><<<gb, 256, 0, s>>>(p, V, mu, up, wp, ui, wi, uo, wo, u0b, w0b, Vb, mub, tau, bm, rden);
        else
            k_adj_visc_lim<1><<<gb, 256, 0, s>>>(p, V, mu, up, wp, ui, wi, uo, wo, u0b, w0b, Vb, mub, tau, bm, rden);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        double *t = ui; ui = uo; uo = t;
        t = wi; wi = wo; wo = t;
    }
    if (axis == 0) k_adj_visc_coef<0><<<gb, 256, 0, s>>>(p, Uin, u0, w0, u0b, w0b, ui, wi, Vb, mub, ab, Gin, pbar);
    else k_adj_visc_coef<1><<<gb, 256, 0, s>>>(p, Uin, u0, w0, u0b, w0b, ui, wi, Vb, mub, ab, Gin, pbar);
    return cudaGetLastError();
}

// planes of the heat adjoint: T0, T0b, V, L, Ia, qb, vb x2, Lb, Iab, Vb, Tb, ab
constexpr int HEAT_WORK_PLANES = 17;

// Reverse of one heat-conduction stage (Algorithm 1, N outer iterations).
// hist: per iteration it, 2 P_it planes (T_it, a_it, v^1..v^{M_it}); Ms[it] =
// 2 P_it - 2; bs: the frozen b of every iteration, concatenated (M_it each).
cudaError_t adj_heat(const DevParams &p, const double *Uin, const double *hist, int N, const int *Ms,
                     const double *bs, double tau, const double *G, double *Gin, double *work, double *pbar,
                     cudaStream_t s)
{
    const size_t n = (size_t)p.n;
    double *T0 = work, *T0b = work + n, *V = work + 2 * n, *L = work + 3 * n, *Ia = work + 4 * n;
    double *qb = work + 5 * n, *vbA = work + 6 * n, *vbB = work + 7 * n, *Lb = work + 8 * n, *Iab = work + 9 * n;
    double *Vb = work + 10 * n, *Tb = work + 11 * n, *ab = work + 12 * n;
    double *Lx = work + 13 * n, *Ly = work + 14 * n, *zA = work + 15 * n, *zB = work + 16 * n;
    const int gb = grid_for(p.n, 256);
    cudaError_t e;
    k_adj_heat_prep<<<gb, 256, 0, s>>>(p, Uin, T0, T0b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // history offsets of the iterations
    size_t off[8];
    size_t boff[8];
    size_t o = 0, ob = 0;
    for (int it = 0; it < N; it++) {
        off[it] = o;
        boff[it] = ob;
        o += (size_t)Ms[it] + 2;
        ob += (size_t)Ms[it];
    }
    for (int it = N - 1; it >= 0; it--) {
        const int M = Ms[it];
        const double *Tit = hist + off[it] * n, *ait = hist + (off[it] + 1) * n;
        auto v_of = [&](int m) -> const double * { return m == 0 ? T0 : hist + (off[it] + 1 + m) * n; };
        k_adj_heat_coef_fwd<<<gb, 256, 0, s>>>(p, Uin, Tit, ait, V, L, Ia);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_adj_heat_eq<<<gb, 256, 0, s>>>(p, Uin, G, v_of(M), L, Ia, Tb, ab, Gin, qb, tau, it == N - 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_adj_heat_q<<<gb, 256, 0, s>>>(p, qb, v_of(M), L, vbA, Lb, Iab, Vb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        double *vi = vbA, *vo = vbB, *zi = zA, *zo = zB;
        auto rden_of = [&](int m) { return 1.0 / (1.0 + tau * bs[boff[it] + m - 1]); };
        if (M >= 1) {
            k_adj_heat_faces<<<gb, 256, 0, s>>>(p, L, Lx, Ly);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_adj_heat_z<<<gb, 256, 0, s>>>(p, V, vi, zi, rden_of(M));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        for (int m = M; m >= 1; m--) {
            const double bm = bs[boff[it] + m - 1], rden = rden_of(m), rnext = m > 1 ? rden_of(m - 1) : 0.0;
            k_adj_heat_lim<<<gb, 256, 0, s>>>(p, V, Lx, Ly, Ia, v_of(m - 1), vi, zi, vo, zo, T0b, Vb, Lb, Iab, tau,
                                              bm, rden, rnext);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            double *t = vi; vi = vo; vo = t;
            t = zi; zi = zo; zo = t;
        }
        k_adj_heat_coef<<<gb, 256, 0, s>>>(p, Uin, Tit, ait, Vb, Lb, Iab, vi, T0b, Tb, ab, Gin, pbar, it == 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_adj_heat_T0<<<gb, 256, 0, s>>>(p, Uin, T0b, Gin);
    return cudaGetLastError();
}

cudaError_t adj_from_primitive(const DevParams &p, const double *prim, const double *Ub, double *pb, cudaStream_t s)
{
    k_adj_from_primitive<<<grid_for(p.n, 256), 256, 0, s>>>(p, prim, Ub, pb);
    return cudaGetLastError();
}

int adj_visc_work_planes() { return VISC_WORK_PLANES; }
int adj_heat_work_planes() { return HEAT_WORK_PLANES; }

}  // namespace dimk

// dim_bulk32.cu -- the FP32-bulk form of the split step (sm_103a).
//
// Same stages and launch structure as the FP64 kernels (dim_sweep.cu,
// dim_parabolic.cu), with the bulk of the flux and stencil arithmetic in FP32:
//   FP32: MUSCL reconstruction of m_k, u_n, u_t, p_k; face states, sound
//         speeds and the HLLC solver; viscous and heat coefficients; every
//         Chebyshev local-iteration sweep (FP32 scratch planes).
//   FP64: the conserved state and its accumulation; the phase pressures at
//         cell centres (p_k = (g_k - 1) E_k / a_k - g_k pinf_k cancels against
//         g_k pinf_k); the volume fraction's reconstruction and flux (so that
//         the minor-phase fraction 1 - alpha_2 keeps its precision near
//         alpha -> 0/1); the pressure relaxation (Sec. 3.3) and the p,T
//         equilibrium (Sec. 3.4) root solves; the Chebyshev parameters b_m.
#include "dim_device.cuh"

namespace dimk {

struct PF {  // FP32 copies of the phase constants
    float g[2], pinf[2], gpinf[2], inv_gm1[2];
};

__device__ __forceinline__ PF pf_of(const DevParams &p)
{
    PF f;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        f.g[k] = (float)p.g[k];
        f.pinf[k] = (float)p.pinf[k];
        f.gpinf[k] = (float)p.gpinf[k];
        f.inv_gm1[k] = (float)p.inv_gm1[k];
    }
    return f;
}

__device__ __forceinline__ float minmodf(float a, float b)
{
    if (a > 0.f && b > 0.f) return fminf(a, b);
    if (a < 0.f && b < 0.f) return fmaxf(a, b);
    return 0.f;
}

// Energies in the FP32 face arithmetic.  In a stiff phase the phase energy
// E_k = a_k (p_k + g_k pinf_k)/(g_k - 1) is dominated by the "cold" part
// C_k = a_k g_k pinf_k/(g_k - 1), while the pressure lives in the small
// thermal part Et_k = a_k p_k/(g_k - 1).  The FP32 HLLC therefore carries only
// the thermal and kinetic energies; across an acoustic wave the star state
// E_k* = chi E_k splits as Et_k* = chi Et_k + (chi - 1) C_k with
// chi - 1 = (S* - u)/(S_K - S*) (no cancellation), and the cold energies are
// transported by the FP64 volume-fraction flux: u* C_k* = u* a_k* g_k pinf_k/(g_k - 1).
struct FaceF {
    float un, ut, rho, p, c, C1, C2;
    float q[7];  // m1, m2, rho u_n, rho u_t, Et1, Et2, Et1 + Et2 + rho|u|^2/2
};

// face state from reconstructed (alpha_1, alpha_2) (FP64, rounded here) and
// W = (m1, m2, u_n, u_t, p1, p2) (FP32)
__device__ __forceinline__ void face_state_f(const PF &f, double a1d, double a2d, const float *w, FaceF &s)
{
    float a1 = (float)a1d, a2 = (float)a2d;
    float m1 = w[0], m2 = w[1], un = w[2], ut = w[3], p1 = w[4], p2 = w[5];
    float rho = m1 + m2;
    float Et1 = a1 * p1 * f.inv_gm1[0];
    float Et2 = a2 * p2 * f.inv_gm1[1];
    s.un = un;
    s.ut = ut;
    s.rho = rho;
    s.p = a1 * p1 + a2 * p2;
    s.c = sqrtf((a1 * f.g[0] * (p1 + f.pinf[0]) + a2 * f.g[1] * (p2 + f.pinf[1])) / rho);
    s.C1 = a1 * f.gpinf[0] * f.inv_gm1[0];
    s.C2 = a2 * f.gpinf[1] * f.inv_gm1[1];
    s.q[0] = m1;
    s.q[1] = m2;
    s.q[2] = rho * un;
    s.q[3] = rho * ut;
    s.q[4] = Et1;
    s.q[5] = Et2;
    s.q[6] = Et1 + Et2 + 0.5f * rho * (un * un + ut * ut);
}

// HLLC (as in the FP64 kernel) in FP32 on the thermal/kinetic energies;
// F[0..6] and u* in FP32; returns the side (0 left, 1 right) whose alpha_2 is
// carried by the x/t = 0 state
__device__ __forceinline__ int hllc_f(const FaceF &L, const FaceF &R, float *F)
{
    float SL = fminf(L.un - L.c, R.un - R.c);
    float SR = fmaxf(L.un + L.c, R.un + R.c);
    float Ss = (R.p - L.p + L.rho * L.un * (SL - L.un) - R.rho * R.un * (SR - R.un)) /
               (L.rho * (SL - L.un) - R.rho * (SR - R.un));
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
        float SK = left ? SL : SR;
        float chi = (SK - K.un) / (SK - Ss);
        float chim1 = (Ss - K.un) / (SK - Ss);
        q[0] = chi * K.q[0];
        q[1] = chi * K.q[1];
        q[2] = chi * K.rho * Ss;
        q[3] = chi * K.rho * K.ut;
        q[4] = chi * K.q[4] + chim1 * K.C1;
        q[5] = chi * K.q[5] + chim1 * K.C2;
        q[6] = chi * (K.q[6] + (Ss - K.un) * (K.rho * Ss + K.p / (SK - K.un))) + chim1 * (K.C1 + K.C2);
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

__device__ __forceinline__ int bc_map32(int a, int len, int bc)
{
    if (a >= 0 && a < len) return a;
    if (bc == DIM_BC_PERIODIC) return ((a % len) + len) % len;
    return a < 0 ? 0 : len - 1;
}

template <int AXIS, int TN, int TL>
__global__ void __launch_bounds__(TN *TL) k_sweep32(const DevParams p, const double *__restrict__ Uin,
                                                    double *__restrict__ Uout, double dt_host, Scalars *sc, int relax,
                                                    int check)
{
    extern __shared__ double smem[];
    constexpr int NE = TN + 4;
    constexpr int NL = NE * TL;
    constexpr int NFL = TN + 1;
    constexpr int NF = NFL * TL;
    double *sU = smem;              // [8][NL] conserved state (FP64)
    double *sP = sU + NQ * NL;      // [2][NL] cell-centre phase pressures (FP64)
    double *sF7 = sP + 2 * NL;      // [NF] volume-fraction flux (FP64)
    float *sW = (float *)(sF7 + NF);  // [6][NL] m1, m2, u_n, u_t, p1, p2 (FP32)
    float *sF = sW + 6 * NL;          // [8][NF] F0..F6, u* (FP32)
    const int n = p.n;
    const int len = AXIS == 0 ? p.nx : p.ny;
    const int ntr = AXIS == 0 ? p.ny : p.nx;
    const int a0 = blockIdx.x * TN;
    const int t0 = blockIdx.y * TL;
    const double dt = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const double dtdx = dt / (AXIS == 0 ? p.dx : p.dy);
    const float dtdxf = (float)dtdx;
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    const PF f = pf_of(p);
    auto cidx = [&](int e, int l) { return AXIS == 0 ? l * NE + e : e * TL + l; };
    auto fidx = [&](int fc, int l) { return AXIS == 0 ? l * NFL + fc : fc * TL + l; };

    for (int li = threadIdx.x; li < NL; li += blockDim.x) {
        int e, l;
        if (AXIS == 0) { l = li / NE; e = li - l * NE; }
        else { e = li / TL; l = li - e * TL; }
        int tr = min(t0 + l, ntr - 1);
        int al = bc_map32(a0 - 2 + e, len, p.bc[AXIS]);
        int x = AXIS == 0 ? al : tr, y = AXIS == 0 ? tr : al;
        int c = y * p.nx + x;
        double q[NQ];
        q[0] = Uin[c];
        q[1] = Uin[n + c];
        q[2] = Uin[QN * n + c];
        q[3] = Uin[QT * n + c];
        q[4] = Uin[4 * n + c];
        q[5] = Uin[5 * n + c];
        q[6] = Uin[6 * n + c];
        q[7] = Uin[7 * n + c];
#pragma unroll
        for (int k = 0; k < NQ; k++) sU[k * NL + li] = q[k];
        double a2 = q[7], a1 = 1.0 - a2;
        double p1 = sg_p(p, 0, q[4], a1), p2 = sg_p(p, 1, q[5], a2);
        sP[li] = p1;
        sP[NL + li] = p2;
        float rho = (float)(q[0] + q[1]);
        sW[0 * NL + li] = (float)q[0];
        sW[1 * NL + li] = (float)q[1];
        sW[2 * NL + li] = (float)q[2] / rho;
        sW[3 * NL + li] = (float)q[3] / rho;
        sW[4 * NL + li] = (float)p1;
        sW[5 * NL + li] = (float)p2;
    }
    __syncthreads();

    for (int fi = threadIdx.x; fi < NF; fi += blockDim.x) {
        int fc, l;
        if (AXIS == 0) { l = fi / NFL; fc = fi - l * NFL; }
        else { fc = fi / TL; l = fi - fc * TL; }
        const int iL = cidx(fc + 1, l), iR = cidx(fc + 2, l);
        const double *A = sU + 7 * NL;
        double aL = A[iL], aR = A[iR];
        float wl[6], wr[6];
        if (p.limiter == DIM_LIMITER_MINMOD) {
            const int iLL = cidx(fc, l), iRR = cidx(fc + 3, l);
            // volume fraction in FP64 (same limiter, Sec. 3.6)
            double sl = minmod(A[iL] - A[iLL], A[iR] - A[iL]);
            double sr = minmod(A[iR] - A[iL], A[iRR] - A[iR]);
            aL = A[iL] + 0.5 * sl;
            aR = A[iR] - 0.5 * sr;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float *Wk = sW + k * NL;
                float s1 = minmodf(Wk[iL] - Wk[iLL], Wk[iR] - Wk[iL]);
                float s2 = minmodf(Wk[iR] - Wk[iL], Wk[iRR] - Wk[iR]);
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
        face_state_f(f, 1.0 - aL, aL, wl, L);
        face_state_f(f, 1.0 - aR, aR, wr, R);
        float F[8];
        int side = hllc_f(L, R, F);
#pragma unroll
        for (int k = 0; k < 8; k++) sF[k * NF + fi] = F[k];
        sF7[fi] = (double)F[7] * (side ? aR : aL);
    }
    __syncthreads();

    unsigned st = 0;
    for (int oi = threadIdx.x; oi < TN * TL; oi += blockDim.x) {
        int i, l;
        if (AXIS == 0) { l = oi / TN; i = oi - l * TN; }
        else { i = oi / TL; l = oi - i * TL; }
        int al = a0 + i, tr = t0 + l;
        if (al >= len || tr >= ntr) continue;
        const int ci = cidx(i + 2, l), fm = fidx(i, l), fp = fidx(i + 1, l);
        double a2 = sU[7 * NL + ci], a1 = 1.0 - a2;
        float duf = sF[7 * NF + fp] - sF[7 * NF + fm];
        double du = (double)sF[7 * NF + fp] - (double)sF[7 * NF + fm];
        float R4 = (float)(a1 * sP[ci]), R5 = (float)(a2 * sP[NL + ci]);
        double qo[NQ];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            float inc = dtdxf * (sF[k * NF + fp] - sF[k * NF + fm]);
            if (k == 4) inc += dtdxf * R4 * duf;
            if (k == 5) inc += dtdxf * R5 * duf;
            qo[k] = sU[k * NL + ci] - (double)inc;
        }
        qo[7] = sU[7 * NL + ci] - dtdx * (sF7[fp] - sF7[fm]) + dtdx * a2 * du;
        // cold energies through the FP64 volume-fraction flux:
        // u* a1* = u* - F7, u* a2* = F7 on each face
        {
            double dF7 = sF7[fp] - sF7[fm];
            double c1 = p.gpinf[0] * p.inv_gm1[0] * (du - dF7), c2 = p.gpinf[1] * p.inv_gm1[1] * dF7;
            qo[4] -= dtdx * c1;
            qo[5] -= dtdx * c2;
            qo[6] -= dtdx * (c1 + c2);
        }
        double q[NQ] = {qo[0], qo[1], 0.0, 0.0, qo[4], qo[5], qo[6], qo[7]};
        q[QN] = qo[2];
        q[QT] = qo[3];
        if (relax) {
            unsigned s = prelax(p, q);
            if (s & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= s & DIM_ST_NAN;
        }
        if (check) st |= check_state(p, q);
        int x = AXIS == 0 ? al : tr, y = AXIS == 0 ? tr : al;
        int c = y * p.nx + x;
#pragma unroll
        for (int k = 0; k < NQ; k++) Uout[k * n + c] = q[k];
    }
    flag(sc, st);
}

// CFL bound and input check; phase pressures in FP64, the rest in FP32
__global__ void k_wave_max32(const DevParams p, const double *__restrict__ U, Scalars *sc)
{
    const int n = p.n;
    const PF f = pf_of(p);
    float m = 0.f;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
        st |= check_state(p, q);
        double a2 = q[7], a1 = 1.0 - a2;
        float p1 = (float)sg_p(p, 0, q[4], a1), p2 = (float)sg_p(p, 1, q[5], a2);
        float rho = (float)(q[0] + q[1]);
        float cs = sqrtf(((float)a1 * f.g[0] * (p1 + f.pinf[0]) + (float)a2 * f.g[1] * (p2 + f.pinf[1])) / rho);
        if (p.nx > 1) {
            float s = (fabsf((float)q[2] / rho) + cs) * (float)p.idx;
            m = fmaxf(m, s);
            if (isnan(s)) st |= DIM_ST_NAN;
        }
        if (p.ny > 1) {
            float s = (fabsf((float)q[3] / rho) + cs) * (float)p.idy;
            m = fmaxf(m, s);
            if (isnan(s)) st |= DIM_ST_NAN;
        }
    }
    block_max_to(&sc->smax, (double)m);
    flag(sc, st);
}

// ---------------------------------------------------------------------------
// parabolic stages in FP32 bulk
// ---------------------------------------------------------------------------
struct HeatScratch32 {
    float *T0, *V, *L, *va, *vb, *Ti;
    double *Ai;  // outer-iteration volume fraction: FP64 (1 - alpha_2 must keep its precision)
};
struct ViscScratch32 {
    float *V, *u0, *w0, *ua, *ub, *wa, *wb;
    double *A2;
};

__device__ __forceinline__ float lapf(const DevParams &p, const Nb &nb, int c, const float *__restrict__ v,
                                      const float *__restrict__ L, float idx2, float idy2)
{
    float r = 0.f;
    float vc = v[c], Lc = L[c];
    if (p.nx > 1) {
        float fl = nb.xm >= 0 ? 0.5f * (L[nb.xm] + Lc) * (vc - v[nb.xm]) * idx2 : 0.f;
        float fr = nb.xp >= 0 ? 0.5f * (Lc + L[nb.xp]) * (v[nb.xp] - vc) * idx2 : 0.f;
        r += fr - fl;
    }
    if (p.ny > 1) {
        float fl = nb.ym >= 0 ? 0.5f * (L[nb.ym] + Lc) * (vc - v[nb.ym]) * idy2 : 0.f;
        float fr = nb.yp >= 0 ? 0.5f * (Lc + L[nb.yp]) * (v[nb.yp] - vc) * idy2 : 0.f;
        r += fr - fl;
    }
    return r;
}

__device__ __forceinline__ float gershf(const DevParams &p, const Nb &nb, int c, const float *__restrict__ V,
                                        const float *__restrict__ L, float idx2, float idy2)
{
    float Lc = L[c];
    float s = 0.f;
    if (p.nx > 1) {
        float fl = nb.xm >= 0 ? 0.5f * (L[nb.xm] + Lc) : 0.f;
        float fr = nb.xp >= 0 ? 0.5f * (Lc + L[nb.xp]) : 0.f;
        s += (fl + fr) * idx2;
    }
    if (p.ny > 1) {
        float fl = nb.ym >= 0 ? 0.5f * (L[nb.ym] + Lc) : 0.f;
        float fr = nb.yp >= 0 ? 0.5f * (Lc + L[nb.yp]) : 0.f;
        s += (fl + fr) * idy2;
    }
    return 2.f * V[c] * s;
}

// V = 1/(C + B1^2/K) and Lam = a1 l1(T) + a2 l2(T) in FP32 (see heat_coeffs)
__device__ __forceinline__ void heat_coeffs_f(const DevParams &p, double m1, double m2, double T, double a2, float &V,
                                              float &Lam)
{
    float a2f = (float)a2, a1f = (float)(1.0 - a2);
    float Tf = (float)T;
    float C1 = (float)(m1 * p.cv[0]), C2 = (float)(m2 * p.cv[1]);
    float B1 = (float)(p.pinf[0] - p.pinf[1]);
    float r1 = (float)p.gm1[0] * C1 * Tf / (a1f * a1f);
    float r2 = (float)p.gm1[1] * C2 * Tf / (a2f * a2f);
    float K = Tf * (r1 + r2);
    V = 1.f / (C1 + C2 + B1 * (B1 / K));
    Lam = (float)(a1f * cond(p, 0, T) + a2f * cond(p, 1, T));
}

__global__ void __launch_bounds__(256) k_heat32(const DevParams p, double *__restrict__ U, HeatScratch32 s,
                                                Scalars *sc, double dt_host, int trelax_first, int check)
{
    __shared__ double s_b[2 * PMAX];
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const double tau = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const float tauf = (float)tau;
    const float idx2 = (float)p.idx2, idy2 = (float)p.idy2;
    const int nout = p.n_outer < 1 ? 1 : (p.n_outer > 8 ? 8 : p.n_outer);
    unsigned st = 0;

    for (int c = t0; c < n; c += nt) {
        double m1 = U[c], m2 = U[n + c], E1 = U[4 * n + c], E2 = U[5 * n + c], a2 = U[7 * n + c];
        double T;
        if (trelax_first) {
            unsigned r = equilibrium(p, m1, m2, E1 + E2, T, a2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            U[4 * n + c] = m1 * p.cv[0] * T + (1.0 - a2) * p.pinf[0];
            U[5 * n + c] = m2 * p.cv[1] * T + a2 * p.pinf[1];
            U[7 * n + c] = a2;
        } else {
            T = mixture_T(p, m1, m2, E1, E2, a2);
        }
        s.T0[c] = (float)T;
        float V, L;
        heat_coeffs_f(p, m1, m2, T, a2, V, L);
        s.V[c] = V;
        s.L[c] = L;
    }
    for (int it = 0; it < nout; it++) {
        if (!grid_barrier(sc)) return;
        float lm = 0.f;
        for (int c = t0; c < n; c += nt) lm = fmaxf(lm, gershf(p, neighbours(p, c), c, s.V, s.L, idx2, idy2));
        block_max_to(&sc->lam[it], (double)lm);
        if (!grid_barrier(sc)) return;
        double lam = read_acc(&sc->lam[it]);
        unsigned capped;
        const int P = cheb_P(p, tau, lam, capped);
        cheb_schedule_block(p, P, lam, s_b);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicMax(&sc->P[0], P);
            if (capped) st |= capped;
        }
        __syncthreads();
        const float *vin = s.T0;
        for (int m = 1; m <= 2 * P - 2; m++) {
            float *vout = (m & 1) ? s.va : s.vb;
            const float tb = (float)(tau * s_b[m - 1]);
            const float rden = (float)(1.0 / (1.0 + tau * s_b[m - 1]));
            for (int c = t0; c < n; c += nt) {
                float Lv = lapf(p, neighbours(p, c), c, vin, s.L, idx2, idy2);
                vout[c] = (s.T0[c] + tb * vin[c] + tauf * s.V[c] * Lv) * rden;
            }
            if (!grid_barrier(sc)) return;
            vin = vout;
        }
        if (it == nout - 1) {
            for (int c = t0; c < n; c += nt) {
                double q = (double)lapf(p, neighbours(p, c), c, vin, s.L, idx2, idy2);
                double m1 = U[c], m2 = U[n + c];
                double rhoe = U[4 * n + c] + U[5 * n + c] + tau * q;
                double T, a2;
                unsigned r = equilibrium(p, m1, m2, rhoe, T, a2);
                double Q[NQ];
                Q[0] = m1;
                Q[1] = m2;
                Q[2] = U[2 * n + c];
                Q[3] = U[3 * n + c];
                Q[4] = m1 * p.cv[0] * T + (1.0 - a2) * p.pinf[0];
                Q[5] = m2 * p.cv[1] * T + a2 * p.pinf[1];
                Q[6] = U[6 * n + c] + tau * q;
                Q[7] = a2;
                U[4 * n + c] = Q[4];
                U[5 * n + c] = Q[5];
                U[6 * n + c] = Q[6];
                U[7 * n + c] = Q[7];
                if (check) st |= check_state(p, Q) | (r & DIM_ST_NAN);
                else if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            }
        } else {
            for (int c = t0; c < n; c += nt) {
                double q = (double)lapf(p, neighbours(p, c), c, vin, s.L, idx2, idy2);
                double T, a2;
                unsigned r = equilibrium(p, U[c], U[n + c], U[4 * n + c] + U[5 * n + c] + tau * q, T, a2);
                if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
                s.Ti[c] = (float)T;
                s.Ai[c] = a2;
            }
            if (!grid_barrier(sc)) return;
            for (int c = t0; c < n; c += nt) {
                float V, L;
                heat_coeffs_f(p, U[c], U[n + c], (double)s.Ti[c], s.Ai[c], V, L);
                s.V[c] = V;
                s.L[c] = L;
            }
        }
    }
    flag(sc, st);
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_visc32(const DevParams p, double *__restrict__ U, ViscScratch32 s,
                                                Scalars *sc, double dt_host, int relax, int check)
{
    __shared__ double s_b[2 * PMAX];
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    constexpr int SLOT = AXIS == 0 ? LAM_VX : LAM_VY;
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const double tau = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const float tauf = (float)tau;
    const float ih2 = (float)(AXIS == 0 ? p.idx2 : p.idy2);
    const float ihf = (float)(AXIS == 0 ? p.idx : p.idy);
    const double ih = AXIS == 0 ? p.idx : p.idy;
    const float mu0 = (float)p.mu[0], mu1 = (float)p.mu[1];
    unsigned st = 0;

    for (int c = t0; c < n; c += nt) {
        float rho = (float)(U[c] + U[n + c]);
        s.V[c] = 1.f / rho;
        s.A2[c] = U[7 * n + c];
        s.u0[c] = (float)U[QN * n + c] / rho;
        s.w0[c] = (float)U[QT * n + c] / rho;
    }
    if (!grid_barrier(sc)) return;
    auto mu_of = [&](int c) {
        float a2 = (float)s.A2[c];
        return (1.f - a2) * mu0 + a2 * mu1;
    };
    auto nbs = [&](int c, int &cm, int &cp) {
        Nb nb = neighbours(p, c);
        cm = AXIS == 0 ? nb.xm : nb.ym;
        cp = AXIS == 0 ? nb.xp : nb.yp;
    };
    float lm = 0.f;
    for (int c = t0; c < n; c += nt) {
        int cm, cp;
        nbs(c, cm, cp);
        float lc = 4.f / 3.f * mu_of(c);
        float fl = cm >= 0 ? 0.5f * (4.f / 3.f * mu_of(cm) + lc) : 0.f;
        float fr = cp >= 0 ? 0.5f * (lc + 4.f / 3.f * mu_of(cp)) : 0.f;
        lm = fmaxf(lm, 2.f * s.V[c] * ((fl + fr) * ih2));
    }
    block_max_to(&sc->lam[SLOT], (double)lm);
    if (!grid_barrier(sc)) return;
    double lam = read_acc(&sc->lam[SLOT]);
    unsigned capped;
    const int P = cheb_P_visc(p, tau, lam, capped);
    cheb_schedule_block(p, P, lam, s_b);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicMax(&sc->P[1 + AXIS], P);
        if (capped) st |= capped;
    }
    __syncthreads();
    const float *uin = s.u0, *win = s.w0;
    for (int m = 1; m <= 2 * P - 2; m++) {
        float *uo = (m & 1) ? s.ua : s.ub;
        float *wo = (m & 1) ? s.wa : s.wb;
        const float tb = (float)(tau * s_b[m - 1]);
        const float rden = (float)(1.0 / (1.0 + tau * s_b[m - 1]));
        for (int c = t0; c < n; c += nt) {
            int cm, cp;
            nbs(c, cm, cp);
            float mc = mu_of(c);
            float mm = cm >= 0 ? 0.5f * (mu_of(cm) + mc) : 0.f;
            float mp = cp >= 0 ? 0.5f * (mc + mu_of(cp)) : 0.f;
            float uc = uin[c], wc = win[c];
            float Lu = (cp >= 0 ? 4.f / 3.f * mp * (uin[cp] - uc) * ih2 : 0.f) -
                       (cm >= 0 ? 4.f / 3.f * mm * (uc - uin[cm]) * ih2 : 0.f);
            float Lw = (cp >= 0 ? mp * (win[cp] - wc) * ih2 : 0.f) - (cm >= 0 ? mm * (wc - win[cm]) * ih2 : 0.f);
            uo[c] = (s.u0[c] + tb * uc + tauf * s.V[c] * Lu) * rden;
            wo[c] = (s.w0[c] + tb * wc + tauf * s.V[c] * Lw) * rden;
        }
        if (!grid_barrier(sc)) return;
        uin = uo;
        win = wo;
    }
    for (int c = t0; c < n; c += nt) {
        int cm, cp;
        nbs(c, cm, cp);
        float mc = mu_of(c);
        float Fn[2], Ft[2], W[2];
        double aF1[2], aF2[2];
        for (int sd = 0; sd < 2; sd++) {
            int cl = sd == 0 ? cm : c, cr = sd == 0 ? c : cp;
            if ((sd == 0 ? cm : cp) < 0) {
                Fn[sd] = Ft[sd] = W[sd] = 0.f;
                aF1[sd] = aF2[sd] = 0.0;
                continue;
            }
            float ml = sd == 0 ? mu_of(cm) : mc, mr = sd == 0 ? mc : mu_of(cp);
            float lmf = 0.5f * (ml + mr);
            Fn[sd] = 4.f / 3.f * lmf * (uin[cr] - uin[cl]) * ihf;
            Ft[sd] = lmf * (win[cr] - win[cl]) * ihf;
            W[sd] = 0.5f * (uin[cl] + uin[cr]) * Fn[sd] + 0.5f * (win[cl] + win[cr]) * Ft[sd];
            double a2l = s.A2[cl], a2r = s.A2[cr];
            aF2[sd] = 0.5 * (a2l + a2r);
            aF1[sd] = 0.5 * ((1.0 - a2l) + (1.0 - a2r));
        }
        double uh = uin[c], wh = win[c];
        double q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
        q[QN] += tau * (double)(Fn[1] - Fn[0]) * ih;
        q[QT] += tau * (double)(Ft[1] - Ft[0]) * ih;
        q[6] += tau * (double)(W[1] - W[0]) * ih;
        q[4] += tau * (aF1[1] * W[1] - aF1[0] * W[0]) * ih -
                tau * (uh * (aF1[1] * Fn[1] - aF1[0] * Fn[0]) + wh * (aF1[1] * Ft[1] - aF1[0] * Ft[0])) * ih;
        q[5] += tau * (aF2[1] * W[1] - aF2[0] * W[0]) * ih -
                tau * (uh * (aF2[1] * Fn[1] - aF2[0] * Fn[0]) + wh * (aF2[1] * Ft[1] - aF2[0] * Ft[0])) * ih;
        if (relax) {
            unsigned r = prelax(p, q);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
        }
        if (check) st |= check_state(p, q);
        U[QN * n + c] = q[QN];
        U[QT * n + c] = q[QT];
        U[4 * n + c] = q[4];
        U[5 * n + c] = q[5];
        U[6 * n + c] = q[6];
        U[7 * n + c] = q[7];
    }
    flag(sc, st);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int SX32_TN = 128, SX32_TL = 1;
constexpr int SY32_TN = 32, SY32_TL = 8;

static size_t sweep32_smem(int TN, int TL)
{
    size_t NL = (size_t)(TN + 4) * TL, NF = (size_t)(TN + 1) * TL;
    return sizeof(double) * (NQ * NL + 2 * NL + NF) + sizeof(float) * (6 * NL + 8 * NF);
}

static int g_heat32_blocks = 0, g_visc32_blocks[2] = {0, 0};

cudaError_t bulk32_setup(int nsm)
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep32<0, SX32_TN, SX32_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep32_smem(SX32_TN, SX32_TL));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sweep32<1, SY32_TN, SY32_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep32_smem(SY32_TN, SY32_TL));
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_heat32, 256, 0);
    if (e != cudaSuccess) return e;
    g_heat32_blocks = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_visc32<0>, 256, 0);
    if (e != cudaSuccess) return e;
    g_visc32_blocks[0] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_visc32<1>, 256, 0);
    if (e != cudaSuccess) return e;
    g_visc32_blocks[1] = b * nsm;
    return cudaSuccess;
}

cudaError_t launch_sweep32(const DevParams &p, int axis, const double *Uin, double *Uout, double dt_host, Scalars *sc,
                           int relax, int check, cudaStream_t s)
{
    if (axis == 0) {
        dim3 grid((p.nx + SX32_TN - 1) / SX32_TN, (p.ny + SX32_TL - 1) / SX32_TL);
        k_sweep32<0, SX32_TN, SX32_TL><<<grid, SX32_TN * SX32_TL, sweep32_smem(SX32_TN, SX32_TL), s>>>(
            p, Uin, Uout, dt_host, sc, relax, check);
    } else {
        dim3 grid((p.ny + SY32_TN - 1) / SY32_TN, (p.nx + SY32_TL - 1) / SY32_TL);
        k_sweep32<1, SY32_TN, SY32_TL><<<grid, SY32_TN * SY32_TL, sweep32_smem(SY32_TN, SY32_TL), s>>>(
            p, Uin, Uout, dt_host, sc, relax, check);
    }
    return cudaGetLastError();
}

cudaError_t launch_wave_max32(const DevParams &p, const double *U, Scalars *sc, cudaStream_t s)
{
    int g = (p.n + 255) / 256 < 152 * 16 ? (p.n + 255) / 256 : 152 * 16;
    k_wave_max32<<<g, 256, 0, s>>>(p, U, sc);
    return cudaGetLastError();
}

static int coop_grid32(int maxb, int n)
{
    int need = (n + 255) / 256;
    return need < maxb ? need : maxb;
}

// the FP32 planes alias the context's 8 FP64 scratch planes (16 FP32 planes)
cudaError_t launch_heat32(const DevParams &p, double *U, double *S, Scalars *sc, double dt_host, int trelax_first,
                          int check, cudaStream_t st)
{
    size_t n = (size_t)p.n;
    float *F = (float *)(S + n);  // six FP32 planes after the FP64 plane 0
    HeatScratch32 hs{F, F + n, F + 2 * n, F + 3 * n, F + 4 * n, F + 5 * n, S};
    DevParams pp = p;
    void *args[] = {(void *)&pp, (void *)&U, (void *)&hs, (void *)&sc, (void *)&dt_host, (void *)&trelax_first,
                    (void *)&check};
    return cudaLaunchCooperativeKernel((const void *)k_heat32, dim3(coop_grid32(g_heat32_blocks, p.n)), dim3(256),
                                       args, 0, st);
}

cudaError_t launch_visc32(const DevParams &p, int axis, double *U, double *S, Scalars *sc, double dt_host, int relax,
                          int check, cudaStream_t st)
{
    size_t n = (size_t)p.n;
    double *A2 = S;  // plane 0 (FP64)
    float *F = (float *)(S + n);
    ViscScratch32 vs{F, F + n, F + 2 * n, F + 3 * n, F + 4 * n, F + 5 * n, F + 6 * n, A2};
    DevParams pp = p;
    void *args[] = {(void *)&pp, (void *)&U, (void *)&vs, (void *)&sc, (void *)&dt_host, (void *)&relax,
                    (void *)&check};
    const void *f = axis == 0 ? (const void *)k_visc32<0> : (const void *)k_visc32<1>;
    return cudaLaunchCooperativeKernel(f, dim3(coop_grid32(g_visc32_blocks[axis], p.n)), dim3(256), args, 0, st);
}

}  // namespace dimk

// dim_bulk32.cuh -- FP32-bulk device building blocks (tile sweep, FP32 face
// states and HLLC, FP32 stencil operators), shared by the per-grid kernels of
// dim_bulk32.cu and the batched persistent kernel of dim_batch.cu.
#pragma once
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

// One tile (TN cells along the sweep axis x TL lines, first cell a0, first line
// t0) of the FP32-bulk sweep; smem as sized by sweep32_smem.  Used by the
// per-grid kernel below and by the batched persistent kernel.
template <int AXIS, int TN, int TL>
__device__ __forceinline__ void sweep32_tile(const DevParams &p, const double *__restrict__ Uin,
                                             double *__restrict__ Uout, double dt, Scalars *sc, int relax, int check,
                                             int a0, int t0, double *smem)
{
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
        double p1 = sg_p<true>(p, 0, q[4], a1), p2 = sg_p<true>(p, 1, q[5], a2);
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
        if (p.limiter != DIM_LIMITER_NONE) {
            const int iLL = cidx(fc, l), iRR = cidx(fc + 3, l);
            const bool ob = p.limiter == DIM_LIMITER_OVERBEE;
            // volume fraction in FP64 (same limiter as alpha_k rho_k, Sec. 3.6)
            double sl = minmod(A[iL] - A[iLL], A[iR] - A[iL]);
            double sr = minmod(A[iR] - A[iL], A[iRR] - A[iR]);
            if (ob) {
                sl = 2.0 * sl;
                sr = 2.0 * sr;
            }
            aL = A[iL] + 0.5 * sl;
            aR = A[iR] - 0.5 * sr;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float *Wk = sW + k * NL;
                float s1 = minmodf(Wk[iL] - Wk[iLL], Wk[iR] - Wk[iL]);
                float s2 = minmodf(Wk[iR] - Wk[iL], Wk[iRR] - Wk[iR]);
                if (ob && k <= 1) {  // m1, m2
                    s1 = 2.f * s1;
                    s2 = 2.f * s2;
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
            unsigned s = prelax<true>(p, q);
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
    __syncthreads();  // the shared tile is reused by the next tile of a persistent block
}


// dynamic shared memory of one FP32 sweep tile
__host__ __device__ constexpr size_t sweep32_smem(int TN, int TL)
{
    return sizeof(double) * ((size_t)NQ * (TN + 4) * TL + 2 * (size_t)(TN + 4) * TL + (size_t)(TN + 1) * TL) +
           sizeof(float) * (6 * (size_t)(TN + 4) * TL + 8 * (size_t)(TN + 1) * TL);
}

// ---------------------------------------------------------------------------
// parabolic stages in FP32 bulk
// ---------------------------------------------------------------------------
struct HeatScratch32 {
    float *T0, *V, *L, *va, *vb, *Ti, *Ia;  // Ia = a1 I1 + a2 I2 (external source)
    double *Ai;  // outer-iteration volume fraction: FP64 (1 - alpha_2 must keep its precision)
};
struct ViscScratch32 {
    float *V, *u0, *w0, *ua, *ub, *wa, *wb;
    double *A2;
};

__device__ __forceinline__ float lapf(const DevParams &p, const Nb &nb, int c, const float *v, const float *L,
                                      float idx2, float idy2)
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

__device__ __forceinline__ float gershf(const DevParams &p, const Nb &nb, int c, const float *V, const float *L,
                                        float idx2, float idy2)
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

}  // namespace dimk

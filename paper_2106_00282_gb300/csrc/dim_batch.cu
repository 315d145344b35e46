// dim_batch.cu -- many independent grids of uneven sizes advanced together in
// one persistent cooperative launch per split step (sm_103a, FP32 bulk).
//
// Every instance keeps the single-grid layout (8 FP64 planes of its own
// nx*ny cells) at its cell offset inside one packed buffer, its own parameters
// (grid, spacing), its own CFL time step, its own lambda_max and Chebyshev
// parameter count.  One launch runs all stages of one step for all instances,
// separated by bounded grid barriers:
//   reset -> CFL maxima -> x sweep (tiles) -> y sweep (tiles)
//   -> viscous x, viscous y -> temperature relaxation + heat conduction,
// each parabolic stage as coefficients -> lambda_max -> per-instance schedule
// -> 2P-2 sweeps (up to the largest P of the batch, idle for instances that
// are done) -> conservative last sweep.  Hyperbolic stages walk a global tile
// list, the others a global list of 2048-cell chunks, each work item finding
// its instance by binary search in prefix sums.  The host captures the
// launch once into a CUDA graph and replays it; an autotuner picks the tile
// shapes and the blocks per SM on the caller's batch.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "dim_bulk32.cuh"

namespace dimk {

constexpr int BCH = 2048;  // cells per chunk

struct BatchDev {
    const DevParams *prm;  // [ninst]
    const long long *off;  // [ninst + 1] cell offsets
    const int *tx, *ty, *ch;  // [ninst + 1] prefix sums of x tiles, y tiles, chunks
    Scalars *sc;           // [ninst]
    Scalars *g;            // grid barrier; P[slot] = largest 2P - 2 of a solve
    double *bs;            // [3][ninst][2 PMAX] Chebyshev schedules (viscous x, viscous y, heat)
    int *Pi;               // [3][ninst] P per instance and solve
    double *U, *U2, *S;
    int ninst;
    int viscous, heat, trelax;
};

__device__ __forceinline__ int find_inst(const int *pre, int n, int t)
{
    int lo = 0, hi = n;  // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// chunk t of the global chunk list: instance, first and last cell
__device__ __forceinline__ int chunk_range(const BatchDev &d, int t, int &c0, int &c1)
{
    int i = find_inst(d.ch, d.ninst, t);
    int k = t - d.ch[i];
    int n = d.prm[i].n;
    c0 = k * BCH;
    c1 = min(c0 + BCH, n);
    return i;
}

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
__device__ void stage_wave(const BatchDev &d)
{
    const int nch = d.ch[d.ninst];
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        const PF f = pf_of(p);
        const int n = p.n;
        const double *U = d.U + 8 * d.off[i];
        float m = 0.f;
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            double q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
            st |= check_state(p, q);
            double a2 = q[7], a1 = 1.0 - a2;
            float p1 = (float)sg_p<true>(p, 0, q[4], a1), p2 = (float)sg_p<true>(p, 1, q[5], a2);
            float rho = (float)(q[0] + q[1]);
            float cs = sqrtf(((float)a1 * f.g[0] * (p1 + f.pinf[0]) + (float)a2 * f.g[1] * (p2 + f.pinf[1])) / rho);
            float sx = (fabsf((float)q[2] / rho) + cs) * (float)p.idx;
            float sy = (fabsf((float)q[3] / rho) + cs) * (float)p.idy;
            m = fmaxf(m, fmaxf(sx, sy));
            if (isnan(sx) || isnan(sy)) st |= DIM_ST_NAN;
        }
        block_max_to(&d.sc[i].smax, (double)m);
        flag(&d.sc[i], st);
    }
}

template <int AXIS, int TN, int TL>
__device__ void stage_sweep(const BatchDev &d, const double *Uin_all, double *Uout_all, double *smem)
{
    const int *pre = AXIS == 0 ? d.tx : d.ty;
    const int nt = pre[d.ninst];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        int i = find_inst(pre, d.ninst, t);
        const DevParams &p = d.prm[i];
        int k = t - pre[i];
        int len = AXIS == 0 ? p.nx : p.ny;
        int nal = (len + TN - 1) / TN;  // tiles along the sweep axis
        int kl = k / nal, ka = k - kl * nal;
        double dt = p.cfl / read_acc(&d.sc[i].smax);
        sweep32_tile<AXIS, TN, TL>(p, Uin_all + 8 * d.off[i], Uout_all + 8 * d.off[i], dt, &d.sc[i], 1, 0, ka * TN,
                                   kl * TL, smem);
    }
}

// per-instance Chebyshev parameters of solve `slot` and the largest sweep count
__device__ void stage_schedule(const BatchDev &d, int slot, int lam_slot, bool viscous)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int per = 2 * PMAX;
    for (int e = tid; e < d.ninst * per; e += nth) {
        int i = e / per, s = e - i * per;
        const DevParams &p = d.prm[i];
        double tau = p.cfl / read_acc(&d.sc[i].smax);
        double lam = read_acc(&d.sc[i].lam[lam_slot]);
        unsigned capped;
        int P = viscous ? cheb_P_visc(p, tau, lam, capped) : cheb_P(p, tau, lam, capped);
        if (s == 0) {
            d.Pi[slot * d.ninst + i] = P;
            atomicMax(&d.g->P[slot], 2 * P - 2);
            atomicMax(&d.sc[i].P[slot], P);
            flag(&d.sc[i], capped);
        }
        if (s < 2 * P - 1) {
            const double *beta = p.beta + (P - 1) * PMAX;
            int m = s < P - 1 ? P - s : 2 * P - 1 - s;
            d.bs[((size_t)slot * d.ninst + i) * per + s] = lam * (beta[0] - beta[m - 1]) / (1.0 + beta[0]);
        }
    }
}

// viscous step along AXIS for all instances (Sec. 3.2), FP32 bulk
template <int AXIS>
__device__ bool stage_visc(const BatchDev &d, int relax)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    constexpr int SLOT = AXIS, LAM = AXIS == 0 ? LAM_VX : LAM_VY;
    const int nch = d.ch[d.ninst];
    // scratch per instance: plane 0 (FP64) alpha snapshot, then FP32 planes V, u0, w0, ua, ub, wa, wb
    auto scr = [&](int i, double *&A2, float *&F) {
        size_t n = (size_t)d.prm[i].n;
        A2 = d.S + 8 * d.off[i];
        F = (float *)(A2 + n);
    };
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        double *U = d.U + 8 * d.off[i];
        double *A2;
        float *F;
        scr(i, A2, F);
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            float rho = (float)(U[c] + U[n + c]);
            F[c] = 1.f / rho;
            A2[c] = U[7 * n + c];
            F[n + c] = (float)U[QN * n + c] / rho;
            F[2 * n + c] = (float)U[QT * n + c] / rho;
        }
    }
    if (!grid_barrier(d.g)) return false;
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        double *A2;
        float *F;
        scr(i, A2, F);
        const float ih2 = (float)(AXIS == 0 ? p.idx2 : p.idy2);
        const float mu0 = (float)p.mu[0], mu1 = (float)p.mu[1];
        float lm = 0.f;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            Nb nb = neighbours(p, c);
            int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
            auto mu_of = [&](int cc) {
                float a = (float)A2[cc];
                return (1.f - a) * mu0 + a * mu1;
            };
            float lc = 4.f / 3.f * mu_of(c);
            float fl = cm >= 0 ? 0.5f * (4.f / 3.f * mu_of(cm) + lc) : 0.f;
            float fr = cp >= 0 ? 0.5f * (lc + 4.f / 3.f * mu_of(cp)) : 0.f;
            lm = fmaxf(lm, 2.f * F[c] * ((fl + fr) * ih2));
        }
        block_max_to(&d.sc[i].lam[LAM], (double)lm);
    }
    if (!grid_barrier(d.g)) return false;
    stage_schedule(d, SLOT, LAM, true);
    if (!grid_barrier(d.g)) return false;
    const int M = *(volatile int *)&d.g->P[SLOT];
    for (int m = 1; m <= M; m++) {
        for (int t = blockIdx.x; t < nch; t += gridDim.x) {
            int c0, c1;
            int i = chunk_range(d, t, c0, c1);
            int P = d.Pi[SLOT * d.ninst + i];
            if (m > 2 * P - 2) continue;
            const DevParams &p = d.prm[i];
            int n = p.n;
            double *A2;
            float *F;
            scr(i, A2, F);
            float *V = F, *u0 = F + n, *w0 = F + 2 * (size_t)n;
            const float *uin = m == 1 ? u0 : (((m - 1) & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n);
            const float *win = m == 1 ? w0 : (((m - 1) & 1) ? F + 5 * (size_t)n : F + 6 * (size_t)n);
            float *uo = (m & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n;
            float *wo = (m & 1) ? F + 5 * (size_t)n : F + 6 * (size_t)n;
            const double tau = p.cfl / read_acc(&d.sc[i].smax);
            const double b = d.bs[((size_t)SLOT * d.ninst + i) * 2 * PMAX + (m - 1)];
            const float tb = (float)(tau * b), rden = (float)(1.0 / (1.0 + tau * b)), tauf = (float)tau;
            const float ih2 = (float)(AXIS == 0 ? p.idx2 : p.idy2);
            const float mu0 = (float)p.mu[0], mu1 = (float)p.mu[1];
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                Nb nb = neighbours(p, c);
                int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
                auto mu_of = [&](int cc) {
                    float a = (float)A2[cc];
                    return (1.f - a) * mu0 + a * mu1;
                };
                float mc = mu_of(c);
                float mm = cm >= 0 ? 0.5f * (mu_of(cm) + mc) : 0.f;
                float mp = cp >= 0 ? 0.5f * (mc + mu_of(cp)) : 0.f;
                float uc = uin[c], wc = win[c];
                float Lu = (cp >= 0 ? 4.f / 3.f * mp * (uin[cp] - uc) * ih2 : 0.f) -
                           (cm >= 0 ? 4.f / 3.f * mm * (uc - uin[cm]) * ih2 : 0.f);
                float Lw = (cp >= 0 ? mp * (win[cp] - wc) * ih2 : 0.f) - (cm >= 0 ? mm * (wc - win[cm]) * ih2 : 0.f);
                uo[c] = (u0[c] + tb * uc + tauf * V[c] * Lu) * rden;
                wo[c] = (w0[c] + tb * wc + tauf * V[c] * Lw) * rden;
            }
        }
        if (!grid_barrier(d.g)) return false;
    }
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        int P = d.Pi[SLOT * d.ninst + i];
        double *U = d.U + 8 * d.off[i];
        double *A2;
        float *F;
        scr(i, A2, F);
        int last = 2 * P - 2;
        const float *uin = last == 0 ? F + n : ((last & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n);
        const float *win = last == 0 ? F + 2 * (size_t)n : ((last & 1) ? F + 5 * (size_t)n : F + 6 * (size_t)n);
        const double tau = p.cfl / read_acc(&d.sc[i].smax);
        const double ih = AXIS == 0 ? p.idx : p.idy;
        const float ihf = (float)ih;
        const float mu0 = (float)p.mu[0], mu1 = (float)p.mu[1];
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            Nb nb = neighbours(p, c);
            int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
            auto mu_of = [&](int cc) {
                float a = (float)A2[cc];
                return (1.f - a) * mu0 + a * mu1;
            };
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
                double a2l = A2[cl], a2r = A2[cr];
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
                unsigned r = prelax<true>(p, q);
                if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
                st |= r & DIM_ST_NAN;
            }
            U[QN * n + c] = q[QN];
            U[QT * n + c] = q[QT];
            U[4 * n + c] = q[4];
            U[5 * n + c] = q[5];
            U[6 * n + c] = q[6];
            U[7 * n + c] = q[7];
        }
        flag(&d.sc[i], st);
    }
    return grid_barrier(d.g);
}

// temperature relaxation + heat conduction for all instances (Sec. 3.4), FP32 bulk
__device__ bool stage_heat(const BatchDev &d)
{
    constexpr int SLOT = 2;
    const int nch = d.ch[d.ninst];
    // scratch per instance: plane 0 (FP64, unused here), FP32 planes T0, V, L, va, vb, Ia
    auto scr = [&](int i) { return (float *)(d.S + 8 * d.off[i] + d.prm[i].n); };
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        double *U = d.U + 8 * d.off[i];
        float *F = scr(i);
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            double m1 = U[c], m2 = U[n + c], T, a2;
            unsigned r = equilibrium<true>(p, m1, m2, U[4 * n + c] + U[5 * n + c], T, a2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            U[4 * n + c] = m1 * p.cv[0] * T + (1.0 - a2) * p.pinf[0];
            U[5 * n + c] = m2 * p.cv[1] * T + a2 * p.pinf[1];
            U[7 * n + c] = a2;
            F[c] = (float)T;
            float V, L;
            heat_coeffs_f(p, m1, m2, T, a2, V, L);
            F[n + c] = V;
            F[2 * n + c] = L;
            F[5 * (size_t)n + c] = (float)((1.0 - a2) * p.src[0] + a2 * p.src[1]);
        }
        flag(&d.sc[i], st);
    }
    if (!grid_barrier(d.g)) return false;
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        float *F = scr(i);
        const float idx2 = (float)p.idx2, idy2 = (float)p.idy2;
        float lm = 0.f;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x)
            lm = fmaxf(lm, gershf(p, neighbours(p, c), c, F + n, F + 2 * (size_t)n, idx2, idy2));
        block_max_to(&d.sc[i].lam[0], (double)lm);
    }
    if (!grid_barrier(d.g)) return false;
    stage_schedule(d, SLOT, 0, false);
    if (!grid_barrier(d.g)) return false;
    const int M = *(volatile int *)&d.g->P[SLOT];
    for (int m = 1; m <= M; m++) {
        for (int t = blockIdx.x; t < nch; t += gridDim.x) {
            int c0, c1;
            int i = chunk_range(d, t, c0, c1);
            int P = d.Pi[SLOT * d.ninst + i];
            if (m > 2 * P - 2) continue;
            const DevParams &p = d.prm[i];
            int n = p.n;
            float *F = scr(i);
            const float *T0 = F, *V = F + n, *L = F + 2 * (size_t)n;
            const float *vin = m == 1 ? T0 : (((m - 1) & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n);
            float *vout = (m & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n;
            const double tau = p.cfl / read_acc(&d.sc[i].smax);
            const double b = d.bs[((size_t)SLOT * d.ninst + i) * 2 * PMAX + (m - 1)];
            const float tb = (float)(tau * b), rden = (float)(1.0 / (1.0 + tau * b)), tauf = (float)tau;
            const float idx2 = (float)p.idx2, idy2 = (float)p.idy2;
            const float *Ia = F + 5 * (size_t)n;
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                float Lv = lapf(p, neighbours(p, c), c, vin, L, idx2, idy2);
                vout[c] = (T0[c] + tb * vin[c] + tauf * V[c] * (Lv + Ia[c])) * rden;
            }
        }
        if (!grid_barrier(d.g)) return false;
    }
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        int P = d.Pi[SLOT * d.ninst + i];
        double *U = d.U + 8 * d.off[i];
        float *F = scr(i);
        int last = 2 * P - 2;
        const float *vin = last == 0 ? F : ((last & 1) ? F + 3 * (size_t)n : F + 4 * (size_t)n);
        const float *L = F + 2 * (size_t)n;
        const double tau = p.cfl / read_acc(&d.sc[i].smax);
        const float idx2 = (float)p.idx2, idy2 = (float)p.idy2;
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            double q = (double)lapf(p, neighbours(p, c), c, vin, L, idx2, idy2) + (double)F[5 * (size_t)n + c];
            double m1 = U[c], m2 = U[n + c];
            double T, a2;
            unsigned r = equilibrium<true>(p, m1, m2, U[4 * n + c] + U[5 * n + c] + tau * q, T, a2);
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
            st |= check_state(p, Q) | (r & DIM_ST_NAN);
        }
        flag(&d.sc[i], st);
    }
    return true;
}

// pointwise temperature relaxation (heat off) with the end-of-step check
__device__ void stage_trelax(const BatchDev &d)
{
    const int nch = d.ch[d.ninst];
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        int n = p.n;
        double *U = d.U + 8 * d.off[i];
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            double q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
            double T, a;
            unsigned r = equilibrium<true>(p, q[0], q[1], q[4] + q[5], T, a);
            q[4] = q[0] * p.cv[0] * T + (1.0 - a) * p.pinf[0];
            q[5] = q[1] * p.cv[1] * T + a * p.pinf[1];
            q[7] = a;
            U[4 * n + c] = q[4];
            U[5 * n + c] = q[5];
            U[7 * n + c] = q[7];
            st |= check_state(p, q) | (r & DIM_ST_NAN);
        }
        flag(&d.sc[i], st);
    }
}

template <int TNX, int TLX, int TNY, int TLY>
__global__ void __launch_bounds__(256) k_batch_step(BatchDev d)
{
    extern __shared__ double smem[];
    // per-instance accumulators of this step
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ninst; i += gridDim.x * blockDim.x) {
        d.sc[i].smax = 0ull;
        for (int s = 0; s < 12; s++) {
            d.sc[i].lam[s] = 0ull;
            d.sc[i].P[s] = 0;
        }
    }
    if (!grid_barrier(d.g)) return;
    stage_wave(d);
    if (!grid_barrier(d.g)) return;
    stage_sweep<0, TNX, TLX>(d, d.U, d.U2, smem);
    if (!grid_barrier(d.g)) return;
    stage_sweep<1, TNY, TLY>(d, d.U2, d.U, smem);
    if (!grid_barrier(d.g)) return;
    if (d.viscous) {
        if (!stage_visc<0>(d, 0)) return;
        if (!stage_visc<1>(d, 1)) return;
    }
    if (d.heat) {
        stage_heat(d);
    } else if (d.trelax) {
        stage_trelax(d);
    }
}

// ---------------------------------------------------------------------------
// variants (tile shapes) and launch
// ---------------------------------------------------------------------------
struct Variant {
    const void *fn;
    int tnx, tlx, tny, tly;
    size_t smem;
};

#define DIM_BATCH_VARIANT(a, b, c, e)                                                          \
    Variant{(const void *)k_batch_step<a, b, c, e>, a, b, c, e,                                \
            sweep32_smem(a, b) > sweep32_smem(c, e) ? sweep32_smem(a, b) : sweep32_smem(c, e)}

static const Variant kVariants[] = {
    DIM_BATCH_VARIANT(256, 1, 32, 8),
    DIM_BATCH_VARIANT(128, 2, 32, 8),
    DIM_BATCH_VARIANT(256, 1, 16, 16),
    DIM_BATCH_VARIANT(128, 2, 16, 16),
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int batch_num_variants() { return kNumVariants; }
void batch_variant_tiles(int v, int *tnx, int *tlx, int *tny, int *tly)
{
    *tnx = kVariants[v].tnx;
    *tlx = kVariants[v].tlx;
    *tny = kVariants[v].tny;
    *tly = kVariants[v].tly;
}

// blocks per SM the variant can keep resident (0 on error)
int batch_variant_setup(int v)
{
    const Variant &V = kVariants[v];
    if (cudaFuncSetAttribute(V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V.smem) != cudaSuccess) return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, V.fn, 256, V.smem) != cudaSuccess) return 0;
    return b;
}

cudaError_t batch_launch(int v, int blocks, const BatchDev &d, cudaStream_t s)
{
    const Variant &V = kVariants[v];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = V.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BatchDev dd = d;
    void *args[] = {(void *)&dd};
    return cudaLaunchKernelExC(&cfg, V.fn, args);
}

// tiles of an nx x ny grid for the x and y sweeps of variant v
void batch_tiles(int v, int nx, int ny, int *tiles_x, int *tiles_y)
{
    const Variant &V = kVariants[v];
    *tiles_x = ((nx + V.tnx - 1) / V.tnx) * ((ny + V.tlx - 1) / V.tlx);
    *tiles_y = ((ny + V.tny - 1) / V.tny) * ((nx + V.tly - 1) / V.tly);
}

}  // namespace dimk

// ---------------------------------------------------------------------------
// host API
// ---------------------------------------------------------------------------
int dim_host_params(const dim_params *hp, int nx, int ny, double dx, double dy, dimk::DevParams *out);
namespace dimk {
cudaError_t launch_from_primitive(const DevParams &p, const double *prim, double *U, Scalars *sc, cudaStream_t s);
}

using dimk::DevParams;
using dimk::Scalars;

struct dim_batch {
    dim_params hp;
    int ninst;
    long long ncell;
    cudaStream_t user;    // caller's stream
    cudaStream_t own;     // non-blocking stream the graph is captured on and replayed
    cudaEvent_t ev_in, ev_out;
    DevParams *prm_h;
    long long *off_h;
    // device tables
    DevParams *prm;
    long long *off;
    int *ch;
    int *tx[dimk::kNumVariants], *ty[dimk::kNumVariants];
    Scalars *sc, *g;
    double *bs, *U2, *S, *beta;
    int *Pi;
    int viscous, heat, trelax;
    int nsm, maxb[dimk::kNumVariants];
    int variant, blocks;
    cudaGraphExec_t gexec;
    double *gU;
    int gvariant, gblocks;
};

static void batch_free(dim_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->prm);
    cudaFree(b->off);
    cudaFree(b->ch);
    for (int v = 0; v < dimk::kNumVariants; v++) {
        cudaFree(b->tx[v]);
        cudaFree(b->ty[v]);
    }
    cudaFree(b->sc);
    cudaFree(b->g);
    cudaFree(b->bs);
    cudaFree(b->U2);
    cudaFree(b->S);
    cudaFree(b->beta);
    cudaFree(b->Pi);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->own) cudaStreamDestroy(b->own);
    free(b->prm_h);
    free(b->off_h);
    free(b);
}

static dimk::BatchDev batch_dev(const dim_batch *b, double *U)
{
    dimk::BatchDev d;
    d.prm = b->prm;
    d.off = b->off;
    d.tx = b->tx[b->variant];
    d.ty = b->ty[b->variant];
    d.ch = b->ch;
    d.sc = b->sc;
    d.g = b->g;
    d.bs = b->bs;
    d.Pi = b->Pi;
    d.U = U;
    d.U2 = b->U2;
    d.S = b->S;
    d.ninst = b->ninst;
    d.viscous = b->viscous;
    d.heat = b->heat;
    d.trelax = b->trelax;
    return d;
}

// one step on the internal stream (no graph)
static cudaError_t batch_step_direct(dim_batch *b, double *U, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->g, 0, offsetof(Scalars, status), s);
    if (e != cudaSuccess) return e;
    return dimk::batch_launch(b->variant, b->blocks, batch_dev(b, U), s);
}

extern "C" {

int dim_batch_init(dim_batch **out, const dim_params *hp, int ninst, const int *nx, const int *ny, const double *dx,
                   const double *dy, void *cuda_stream)
{
    if (!out || !hp || ninst < 1 || !nx || !ny || !dx || !dy) return DIM_EINVAL;
    *out = nullptr;
    if (hp->precision != DIM_PRECISION_FP32_BULK) return DIM_EINVAL;
    dim_batch *b = (dim_batch *)calloc(1, sizeof(dim_batch));
    if (!b) return DIM_ECUDA;
    b->hp = *hp;
    b->ninst = ninst;
    b->user = (cudaStream_t)cuda_stream;
    b->prm_h = (DevParams *)calloc(ninst, sizeof(DevParams));
    b->off_h = (long long *)calloc(ninst + 1, sizeof(long long));
    int *ch_h = (int *)calloc(ninst + 1, sizeof(int));
    int *t_h = (int *)calloc(2 * (ninst + 1), sizeof(int));
    if (!b->prm_h || !b->off_h || !ch_h || !t_h) {
        free(ch_h); free(t_h); batch_free(b);
        return DIM_ECUDA;
    }
    int r = DIM_OK;
    long long off = 0, chunks = 0;
    for (int i = 0; i < ninst && r == DIM_OK; i++) {
        if (nx[i] < 2 || ny[i] < 2) r = DIM_EINVAL;
        else r = dim_host_params(hp, nx[i], ny[i], dx[i], dy[i], &b->prm_h[i]);
        b->off_h[i] = off;
        ch_h[i] = (int)chunks;
        off += (long long)nx[i] * ny[i];
        chunks += ((long long)nx[i] * ny[i] + dimk::BCH - 1) / dimk::BCH;
    }
    b->off_h[ninst] = off;
    ch_h[ninst] = (int)chunks;
    b->ncell = off;
    if (r == DIM_OK && (off > (1LL << 31) / 8 || chunks > (1LL << 30))) r = DIM_EINVAL;
    if (r != DIM_OK) {
        free(ch_h); free(t_h); batch_free(b);
        return r;
    }
    b->viscous = hp->mu[0] > 0.0 || hp->mu[1] > 0.0;
    b->trelax = hp->trelax != DIM_TRELAX_OFF;  // FP32-bulk only: dim_host_params admits no variant
    b->heat = b->trelax && (hp->k0[0] > 0.0 || hp->k0[1] > 0.0 || hp->src[0] > 0.0 || hp->src[1] > 0.0);
    int dev = 0;
    bool ok = cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    // Chebyshev roots, as for dim_init
    const double pi = 3.14159265358979323846;
    double *tab = (double *)calloc((size_t)dimk::PMAX * dimk::PMAX, sizeof(double));
    ok = ok && tab;
    if (ok) {
        for (int P = 1; P <= dimk::PMAX; P++)
            for (int m = 1; m <= P; m++) tab[(P - 1) * dimk::PMAX + (m - 1)] = cos((2.0 * m - 1.0) * pi / (2.0 * P));
    }
    size_t N = (size_t)b->ncell;
    ok = ok && cudaMalloc(&b->beta, sizeof(double) * dimk::PMAX * dimk::PMAX) == cudaSuccess &&
         cudaMemcpy(b->beta, tab, sizeof(double) * dimk::PMAX * dimk::PMAX, cudaMemcpyHostToDevice) == cudaSuccess;
    free(tab);
    for (int i = 0; ok && i < ninst; i++) b->prm_h[i].beta = b->beta;
    ok = ok && cudaMalloc(&b->prm, sizeof(DevParams) * ninst) == cudaSuccess &&
         cudaMemcpy(b->prm, b->prm_h, sizeof(DevParams) * ninst, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMalloc(&b->off, sizeof(long long) * (ninst + 1)) == cudaSuccess &&
         cudaMemcpy(b->off, b->off_h, sizeof(long long) * (ninst + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMalloc(&b->ch, sizeof(int) * (ninst + 1)) == cudaSuccess &&
         cudaMemcpy(b->ch, ch_h, sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice) == cudaSuccess;
    for (int v = 0; ok && v < dimk::kNumVariants; v++) {
        int ax = 0, ay = 0;
        for (int i = 0; i < ninst; i++) {
            int tx_i, ty_i;
            dimk::batch_tiles(v, nx[i], ny[i], &tx_i, &ty_i);
            t_h[i] = ax;
            t_h[ninst + 1 + i] = ay;
            ax += tx_i;
            ay += ty_i;
        }
        t_h[ninst] = ax;
        t_h[2 * ninst + 1] = ay;
        ok = cudaMalloc(&b->tx[v], sizeof(int) * (ninst + 1)) == cudaSuccess &&
             cudaMalloc(&b->ty[v], sizeof(int) * (ninst + 1)) == cudaSuccess &&
             cudaMemcpy(b->tx[v], t_h, sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->ty[v], t_h + ninst + 1, sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice) == cudaSuccess;
        b->maxb[v] = ok ? dimk::batch_variant_setup(v) : 0;
        ok = ok && b->maxb[v] > 0;
    }
    free(ch_h);
    free(t_h);
    ok = ok && cudaMalloc(&b->sc, sizeof(Scalars) * ninst) == cudaSuccess &&
         cudaMemset(b->sc, 0, sizeof(Scalars) * ninst) == cudaSuccess &&
         cudaMalloc(&b->g, sizeof(Scalars)) == cudaSuccess && cudaMemset(b->g, 0, sizeof(Scalars)) == cudaSuccess &&
         cudaMalloc(&b->bs, sizeof(double) * 3 * ninst * 2 * dimk::PMAX) == cudaSuccess &&
         cudaMalloc(&b->Pi, sizeof(int) * 3 * ninst) == cudaSuccess &&
         cudaMalloc(&b->U2, sizeof(double) * 8 * N) == cudaSuccess &&
         cudaMalloc(&b->S, sizeof(double) * 8 * N) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        batch_free(b);
        return DIM_ECUDA;
    }
    b->variant = 0;
    b->blocks = b->maxb[0] * b->nsm;
    *out = b;
    return DIM_OK;
}

void dim_batch_destroy(dim_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->own);
    cudaStreamSynchronize(b->user);
    batch_free(b);
}

int dim_batch_layout(const dim_batch *b, long long *offsets)
{
    if (!b || !offsets) return DIM_EINVAL;
    memcpy(offsets, b->off_h, sizeof(long long) * (b->ninst + 1));
    return DIM_OK;
}

int dim_batch_from_primitive(dim_batch *b, const double *prim, double *U)
{
    if (!b || !prim || !U) return DIM_EINVAL;
    for (int i = 0; i < b->ninst; i++)
        if (dimk::launch_from_primitive(b->prm_h[i], prim + 5 * b->off_h[i], U + 8 * b->off_h[i], b->sc + i,
                                        b->user) != cudaSuccess)
            return DIM_ECUDA;
    return DIM_OK;
}

// the caller's stream -> internal stream -> the caller's stream
static int batch_run(dim_batch *b, double *U, int nsteps, bool use_graph)
{
    if (cudaEventRecord(b->ev_in, b->user) != cudaSuccess || cudaStreamWaitEvent(b->own, b->ev_in, 0) != cudaSuccess)
        return DIM_ECUDA;
    if (use_graph) {
        if (!b->gexec || b->gU != U || b->gvariant != b->variant || b->gblocks != b->blocks) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DIM_ECUDA;
            cudaError_t e = batch_step_direct(b, U, b->own);
            cudaError_t e2 = cudaStreamEndCapture(b->own, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
                if (graph) cudaGraphDestroy(graph);
                return DIM_ECUDA;
            }
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return DIM_ECUDA;
            }
            b->gU = U;
            b->gvariant = b->variant;
            b->gblocks = b->blocks;
        }
        for (int s = 0; s < nsteps; s++)
            if (cudaGraphLaunch(b->gexec, b->own) != cudaSuccess) return DIM_ECUDA;
    } else {
        for (int s = 0; s < nsteps; s++)
            if (batch_step_direct(b, U, b->own) != cudaSuccess) return DIM_ECUDA;
    }
    if (cudaEventRecord(b->ev_out, b->own) != cudaSuccess || cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess)
        return DIM_ECUDA;
    return DIM_OK;
}

int dim_batch_step(dim_batch *b, double *U, int nsteps)
{
    if (!b || !U || nsteps < 0) return DIM_EINVAL;
    return batch_run(b, U, nsteps, true);
}

int dim_batch_autotune(dim_batch *b, const double *U, int *config)
{
    if (!b || !U) return DIM_EINVAL;
    size_t bytes = sizeof(double) * 8 * (size_t)b->ncell;
    double *Ut = nullptr;
    if (cudaMalloc(&Ut, bytes) != cudaSuccess) return DIM_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaStreamSynchronize(b->user) != cudaSuccess) { cudaFree(Ut); return DIM_ECUDA; }
    float best = 1e30f;
    int bv = 0, bb = b->maxb[0] * b->nsm;
    int rc = DIM_OK;
    for (int v = 0; v < dimk::kNumVariants && rc == DIM_OK; v++) {
        for (int per = 1; per <= b->maxb[v] && rc == DIM_OK; per++) {
            if (per != 1 && per != b->maxb[v]) continue;
            b->variant = v;
            b->blocks = per * b->nsm;
            if (cudaMemcpyAsync(Ut, U, bytes, cudaMemcpyDeviceToDevice, b->own) != cudaSuccess ||
                batch_step_direct(b, Ut, b->own) != cudaSuccess || cudaEventRecord(e0, b->own) != cudaSuccess ||
                batch_step_direct(b, Ut, b->own) != cudaSuccess || batch_step_direct(b, Ut, b->own) != cudaSuccess ||
                cudaEventRecord(e1, b->own) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = DIM_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bv = v;
                bb = b->blocks;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(Ut);
    b->variant = bv;
    b->blocks = bb;
    // the trial steps ran on a copy; their status bits are not the caller's
    if (cudaMemset(b->sc, 0, sizeof(Scalars) * b->ninst) != cudaSuccess) rc = DIM_ECUDA;
    if (config) {
        config[0] = bv;
        config[1] = bb;
        dimk::batch_variant_tiles(bv, &config[2], &config[3], &config[4], &config[5]);
    }
    return rc;
}

int dim_batch_status(dim_batch *b, unsigned *flags, unsigned *any)
{
    if (!b) return DIM_EINVAL;
    Scalars *h = (Scalars *)malloc(sizeof(Scalars) * b->ninst);
    if (!h) return DIM_ECUDA;
    if (cudaStreamSynchronize(b->user) != cudaSuccess ||
        cudaMemcpy(h, b->sc, sizeof(Scalars) * b->ninst, cudaMemcpyDeviceToHost) != cudaSuccess) {
        free(h);
        return DIM_ECUDA;
    }
    unsigned a = 0;
    for (int i = 0; i < b->ninst; i++) {
        if (flags) flags[i] = h[i].status;
        a |= h[i].status;
    }
    Scalars g;
    if (cudaMemcpy(&g, b->g, sizeof(Scalars), cudaMemcpyDeviceToHost) == cudaSuccess) a |= g.status;
    if (any) *any = a;
    free(h);
    return DIM_OK;
}

}  // extern "C"

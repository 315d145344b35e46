// dim_batch.cu -- many independent grids of uneven sizes advanced together in
// one persistent cooperative launch per split step (sm_103a, FP32 bulk).
//
// Every instance keeps the single-grid layout (8 planes of its own nx*ny cells)
// at its cell offset inside one packed buffer, its own parameters (grid,
// spacing), its own CFL time step, its own lambda_max and Chebyshev parameter
// count.  A call converts the packed FP64 state to float-float planes once,
// runs its steps on them with the cell arithmetic of the single-grid FP32-bulk
// form (dim_ff.cuh), and converts back.  One launch runs all stages of one
// step for all instances, separated by bounded grid barriers:
//   reset -> CFL maxima -> time steps -> x sweep (tiles) -> y sweep (tiles)
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

#include "dim_ff.cuh"

namespace dimk {

constexpr int BCH = 2048;  // cells per chunk

struct BatchDev {
    const DevParams *prm;  // [ninst]
    const FFP *ffp;        // [ninst]
    const long long *off;  // [ninst + 1] cell offsets
    const int *tx, *ty, *ch;  // [ninst + 1] prefix sums of x tiles, y tiles, chunks
    Scalars *sc;           // [ninst]
    Scalars *g;            // grid barrier; P[slot] = largest 2P - 2 of a solve
    double *bs;            // [3][ninst][2 PMAX] Chebyshev parameters b_m (viscous x, viscous y, heat)
    float *tbf, *rdf;      // [3][ninst][2 PMAX] tau b_m and 1 / (1 + tau b_m)
    float *dtf;            // [ninst] time step of the step
    int *Pi;               // [3][ninst] P per instance and solve
    float2 *U, *U2;        // float-float state planes (packed), sweep ping-pong
    double *S;             // scratch: 8 planes of doubles per instance, used as FP32 planes
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

__device__ __forceinline__ float *scr_f(const BatchDev &d, int i) { return (float *)(d.S + 8 * d.off[i]); }

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
__device__ void stage_wave(const BatchDev &d)
{
    const int nch = d.ch[d.ninst];
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)d.prm[i].n;
        const float2 *U = d.U + 8 * d.off[i];
        float m = 0.f;
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            ff q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = ld_ff(U, k * n + c);
            st |= ff_check(f, q);
            m = fmaxf(m, ff_wave_speed(d.prm[i], f, q, st));  // the per-grid CFL kernel's arithmetic
        }
        block_max_to_f(&d.sc[i].smax, m);
        flag(&d.sc[i], st);
    }
}

// the time step of every instance, once per step
__device__ void stage_dt(const BatchDev &d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ninst; i += gridDim.x * blockDim.x)
        d.dtf[i] = (float)(d.prm[i].cfl / read_acc(&d.sc[i].smax));
}

template <int AXIS, int TN, int TL>
__device__ void stage_sweep(const BatchDev &d, const float2 *Uin_all, float2 *Uout_all, void *smem)
{
    const int *pre = AXIS == 0 ? d.tx : d.ty;
    const int nt = pre[d.ninst];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int i = find_inst(pre, d.ninst, t);
        const DevParams &p = d.prm[i];
        const FFP &f = d.ffp[i];
        const int k = t - pre[i];
        const int len = AXIS == 0 ? p.nx : p.ny;
        const int nal = (len + TN - 1) / TN;  // tiles along the sweep axis
        const int kl = k / nal, ka = k - kl * nal;
        const float dtdx = d.dtf[i] * (AXIS == 0 ? f.idx : f.idy);
        sweepff_tile<AXIS, TN, TL>(p, f, Uin_all + 8 * d.off[i], Uout_all + 8 * d.off[i], dtdx, &d.sc[i], 1, 0,
                                   ka * TN, kl * TL, smem);
    }
}

// per-instance Chebyshev parameters of solve `slot` (FP64 from the root table,
// then tau b_m and 1/(1 + tau b_m) in FP32) and the largest sweep count
__device__ void stage_schedule(const BatchDev &d, int slot, int lam_slot, bool viscous)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int per = 2 * PMAX;
    for (int e = tid; e < d.ninst * per; e += nth) {
        const int i = e / per, s = e - i * per;
        const DevParams &p = d.prm[i];
        const double tau = p.cfl / read_acc(&d.sc[i].smax);
        const double lam = read_acc(&d.sc[i].lam[lam_slot]);
        unsigned capped;
        const int P = viscous ? cheb_P_visc(p, tau, lam, capped) : cheb_P(p, tau, lam, capped);
        if (s == 0) {
            d.Pi[slot * d.ninst + i] = P;
            atomicMax(&d.g->P[slot], 2 * P - 2);
            atomicMax(&d.sc[i].P[slot], P);
            flag(&d.sc[i], capped);
        }
        if (s < 2 * P - 1) {
            const double *beta = p.beta + (P - 1) * PMAX;
            const int m = s < P - 1 ? P - s : 2 * P - 1 - s;
            const double b = lam * (beta[0] - beta[m - 1]) / (1.0 + beta[0]);
            const size_t o = ((size_t)slot * d.ninst + i) * per + s;
            d.bs[o] = b;
            d.tbf[o] = (float)(tau * b);
            d.rdf[o] = (float)(1.0 / (1.0 + tau * b));
        }
    }
}

// viscous step along AXIS for all instances (Sec. 3.2), FP32 bulk; scratch per
// instance (FP32 planes): V, a1, a2, u0, w0, ua, ub, wa, wb
template <int AXIS>
__device__ bool stage_visc(const BatchDev &d, int relax)
{
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    constexpr int SLOT = AXIS, LAM = AXIS == 0 ? LAM_VX : LAM_VY;
    const int nch = d.ch[d.ninst];
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const size_t n = (size_t)d.prm[i].n;
        const float2 *U = d.U + 8 * d.off[i];
        float *F = scr_f(d, i);
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const float rho = ff_f(ld_ff(U, c)) + ff_f(ld_ff(U, n + c));
            const ff a2 = ld_ff(U, 7 * n + c);
            F[c] = __fdividef(1.f, rho);
            F[n + c] = ff_f(ff_sub(ff_one(), a2));
            F[2 * n + c] = ff_f(a2);
            F[3 * n + c] = __fdividef(ff_f(ld_ff(U, QN * n + c)), rho);
            F[4 * n + c] = __fdividef(ff_f(ld_ff(U, QT * n + c)), rho);
        }
    }
    if (!grid_barrier(d.g)) return false;
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)p.n;
        const float *F = scr_f(d, i);
        const float ih2 = AXIS == 0 ? f.idx2 : f.idy2;
        const float mu0 = f.mu[0], mu1 = f.mu[1];
        auto mu_of = [&](int cc) { return F[n + cc] * mu0 + F[2 * n + cc] * mu1; };
        float lm = 0.f;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const Nb nb = neighbours(p, c);
            const int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
            const float lc = 4.f / 3.f * mu_of(c);
            const float fl = cm >= 0 ? 0.5f * (4.f / 3.f * mu_of(cm) + lc) : 0.f;
            const float fr = cp >= 0 ? 0.5f * (lc + 4.f / 3.f * mu_of(cp)) : 0.f;
            lm = fmaxf(lm, 2.f * F[c] * ((fl + fr) * ih2));
        }
        block_max_to_f(&d.sc[i].lam[LAM], lm);
    }
    if (!grid_barrier(d.g)) return false;
    stage_schedule(d, SLOT, LAM, true);
    if (!grid_barrier(d.g)) return false;
    const int M = *(volatile int *)&d.g->P[SLOT];
    for (int m = 1; m <= M; m++) {
        for (int t = blockIdx.x; t < nch; t += gridDim.x) {
            int c0, c1;
            const int i = chunk_range(d, t, c0, c1);
            const int P = d.Pi[SLOT * d.ninst + i];
            if (m > 2 * P - 2) continue;
            const DevParams &p = d.prm[i];
            const FFP &f = d.ffp[i];
            const size_t n = (size_t)p.n;
            float *F = scr_f(d, i);
            const float *V = F, *a1 = F + n, *a2 = F + 2 * n, *u0 = F + 3 * n, *w0 = F + 4 * n;
            const float *uin = m == 1 ? u0 : (((m - 1) & 1) ? F + 5 * n : F + 6 * n);
            const float *win = m == 1 ? w0 : (((m - 1) & 1) ? F + 7 * n : F + 8 * n);
            float *uo = (m & 1) ? F + 5 * n : F + 6 * n;
            float *wo = (m & 1) ? F + 7 * n : F + 8 * n;
            const size_t o = ((size_t)SLOT * d.ninst + i) * 2 * PMAX + (m - 1);
            const float tb = d.tbf[o], rd = d.rdf[o], tauf = d.dtf[i];
            const float ih2 = AXIS == 0 ? f.idx2 : f.idy2;
            const float mu0 = f.mu[0], mu1 = f.mu[1];
            auto mu_of = [&](int cc) { return a1[cc] * mu0 + a2[cc] * mu1; };
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                const Nb nb = neighbours(p, c);
                const int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
                const float mc = mu_of(c);
                const float mm = cm >= 0 ? 0.5f * (mu_of(cm) + mc) : 0.f;
                const float mp = cp >= 0 ? 0.5f * (mc + mu_of(cp)) : 0.f;
                const float uc = uin[c], wc = win[c];
                const float Lu = (cp >= 0 ? 4.f / 3.f * mp * (uin[cp] - uc) * ih2 : 0.f) -
                                 (cm >= 0 ? 4.f / 3.f * mm * (uc - uin[cm]) * ih2 : 0.f);
                const float Lw =
                    (cp >= 0 ? mp * (win[cp] - wc) * ih2 : 0.f) - (cm >= 0 ? mm * (wc - win[cm]) * ih2 : 0.f);
                uo[c] = (u0[c] + tb * uc + tauf * V[c] * Lu) * rd;
                wo[c] = (w0[c] + tb * wc + tauf * V[c] * Lw) * rd;
            }
        }
        if (!grid_barrier(d.g)) return false;
    }
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)p.n;
        const int P = d.Pi[SLOT * d.ninst + i];
        float2 *U = d.U + 8 * d.off[i];
        const float *F = scr_f(d, i);
        const float *a1 = F + n, *a2 = F + 2 * n;
        const int last = 2 * P - 2;
        const float *uin = last == 0 ? F + 3 * n : ((last & 1) ? F + 5 * n : F + 6 * n);
        const float *win = last == 0 ? F + 4 * n : ((last & 1) ? F + 7 * n : F + 8 * n);
        const float ih = AXIS == 0 ? f.idx : f.idy;
        const float ti = d.dtf[i] * ih;
        const float mu0 = f.mu[0], mu1 = f.mu[1];
        auto mu_of = [&](int cc) { return a1[cc] * mu0 + a2[cc] * mu1; };
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const Nb nb = neighbours(p, c);
            const int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
            const float mc = mu_of(c);
            float Fn[2], Ft[2], W[2], aF1[2], aF2[2];
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int cl = sd == 0 ? cm : c, cr = sd == 0 ? c : cp;
                if ((sd == 0 ? cm : cp) < 0) {
                    Fn[sd] = Ft[sd] = W[sd] = aF1[sd] = aF2[sd] = 0.f;
                    continue;
                }
                const float lmf = 0.5f * ((sd == 0 ? mu_of(cm) : mc) + (sd == 0 ? mc : mu_of(cp)));
                Fn[sd] = 4.f / 3.f * lmf * (uin[cr] - uin[cl]) * ih;
                Ft[sd] = lmf * (win[cr] - win[cl]) * ih;
                W[sd] = 0.5f * (uin[cl] + uin[cr]) * Fn[sd] + 0.5f * (win[cl] + win[cr]) * Ft[sd];
                aF1[sd] = 0.5f * (a1[cl] + a1[cr]);
                aF2[sd] = 0.5f * (a2[cl] + a2[cr]);
            }
            const float uh = uin[c], wh = win[c];
            ff q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = ld_ff(U, k * n + c);
            q[QN] = ff_add_f(q[QN], ti * (Fn[1] - Fn[0]));
            q[QT] = ff_add_f(q[QT], ti * (Ft[1] - Ft[0]));
            q[6] = ff_add_f(q[6], ti * (W[1] - W[0]));
            q[4] = ff_add_f(q[4], ti * ((aF1[1] * W[1] - aF1[0] * W[0]) - (uh * (aF1[1] * Fn[1] - aF1[0] * Fn[0]) +
                                                                        wh * (aF1[1] * Ft[1] - aF1[0] * Ft[0]))));
            q[5] = ff_add_f(q[5], ti * ((aF2[1] * W[1] - aF2[0] * W[0]) - (uh * (aF2[1] * Fn[1] - aF2[0] * Fn[0]) +
                                                                        wh * (aF2[1] * Ft[1] - aF2[0] * Ft[0]))));
            if (relax) {
                const unsigned r = ff_prelax(f, q);
                if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
                st |= r & DIM_ST_NAN;
            }
#pragma unroll
            for (int k = 2; k < NQ; k++) st_ff(U, k * n + c, q[k]);
        }
        flag(&d.sc[i], st);
    }
    return grid_barrier(d.g);
}

// temperature relaxation + heat conduction for all instances (Sec. 3.4), FP32
// bulk, one Algorithm-1 iteration; scratch per instance (FP32 planes): T0, V,
// L, va, vb, Ia
__device__ bool stage_heat(const BatchDev &d)
{
    constexpr int SLOT = 2;
    const int nch = d.ch[d.ninst];
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)d.prm[i].n;
        float2 *U = d.U + 8 * d.off[i];
        float *F = scr_f(d, i);
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const ff M1 = ld_ff(U, c), M2 = ld_ff(U, n + c);
            const float m1 = ff_f(M1), m2 = ff_f(M2);
            ff E1 = ld_ff(U, 4 * n + c), E2 = ld_ff(U, 5 * n + c);
            float T;
            ff a2;
            const unsigned r = ff_equilibrium(f, M1, M2, ff_add(E1, E2), T, a2, E1, E2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            st_ff(U, 4 * n + c, E1);
            st_ff(U, 5 * n + c, E2);
            st_ff(U, 7 * n + c, a2);
            F[c] = T;
            float V, L;
            ff_heat_coeffs(f, m1, m2, T, a2, V, L);
            F[n + c] = V;
            F[2 * n + c] = L;
            F[5 * n + c] = ff_f(ff_sub(ff_one(), a2)) * f.src[0] + ff_f(a2) * f.src[1];
        }
        flag(&d.sc[i], st);
    }
    if (!grid_barrier(d.g)) return false;
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)p.n;
        const float *F = scr_f(d, i);
        float lm = 0.f;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x)
            lm = fmaxf(lm, gershf(p, neighbours(p, c), c, F + n, F + 2 * n, f.idx2, f.idy2));
        block_max_to_f(&d.sc[i].lam[0], lm);
    }
    if (!grid_barrier(d.g)) return false;
    stage_schedule(d, SLOT, 0, false);
    if (!grid_barrier(d.g)) return false;
    const int M = *(volatile int *)&d.g->P[SLOT];
    for (int m = 1; m <= M; m++) {
        for (int t = blockIdx.x; t < nch; t += gridDim.x) {
            int c0, c1;
            const int i = chunk_range(d, t, c0, c1);
            const int P = d.Pi[SLOT * d.ninst + i];
            if (m > 2 * P - 2) continue;
            const DevParams &p = d.prm[i];
            const FFP &f = d.ffp[i];
            const size_t n = (size_t)p.n;
            float *F = scr_f(d, i);
            const float *T0 = F, *V = F + n, *L = F + 2 * n, *Ia = F + 5 * n;
            const float *vin = m == 1 ? T0 : (((m - 1) & 1) ? F + 3 * n : F + 4 * n);
            float *vout = (m & 1) ? F + 3 * n : F + 4 * n;
            const size_t o = ((size_t)SLOT * d.ninst + i) * 2 * PMAX + (m - 1);
            const float tb = d.tbf[o], rd = d.rdf[o], tauf = d.dtf[i];
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                const float Lv = lapf(p, neighbours(p, c), c, vin, L, f.idx2, f.idy2);
                vout[c] = (T0[c] + tb * vin[c] + tauf * V[c] * (Lv + Ia[c])) * rd;
            }
        }
        if (!grid_barrier(d.g)) return false;
    }
    for (int t = blockIdx.x; t < nch; t += gridDim.x) {
        int c0, c1;
        const int i = chunk_range(d, t, c0, c1);
        const DevParams &p = d.prm[i];
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)p.n;
        const int P = d.Pi[SLOT * d.ninst + i];
        float2 *U = d.U + 8 * d.off[i];
        const float *F = scr_f(d, i);
        const int last = 2 * P - 2;
        const float *vin = last == 0 ? F : ((last & 1) ? F + 3 * n : F + 4 * n);
        const float *L = F + 2 * n;
        const float tauf = d.dtf[i];
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const float dq = tauf * (lapf(p, neighbours(p, c), c, vin, L, f.idx2, f.idy2) + F[5 * n + c]);
            ff q[NQ];
            q[0] = ld_ff(U, c);
            q[1] = ld_ff(U, n + c);
            q[2] = q[3] = ff_of(0.f);
            float T;
            const unsigned r = ff_equilibrium(f, q[0], q[1], ff_add_f(ff_add(ld_ff(U, 4 * n + c), ld_ff(U, 5 * n + c)), dq),
                                              T, q[7], q[4], q[5]);
            q[6] = ff_add_f(ld_ff(U, 6 * n + c), dq);
            st_ff(U, 4 * n + c, q[4]);
            st_ff(U, 5 * n + c, q[5]);
            st_ff(U, 6 * n + c, q[6]);
            st_ff(U, 7 * n + c, q[7]);
            st |= ff_check(f, q) | (r & DIM_ST_NAN);
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
        const int i = chunk_range(d, t, c0, c1);
        const FFP &f = d.ffp[i];
        const size_t n = (size_t)d.prm[i].n;
        float2 *U = d.U + 8 * d.off[i];
        unsigned st = 0;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            ff q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = ld_ff(U, k * n + c);
            float T;
            const unsigned r = ff_equilibrium(f, q[0], q[1], ff_add(q[4], q[5]), T, q[7], q[4], q[5]);
            st_ff(U, 4 * n + c, q[4]);
            st_ff(U, 5 * n + c, q[5]);
            st_ff(U, 7 * n + c, q[7]);
            st |= ff_check(f, q) | (r & DIM_ST_NAN);
        }
        flag(&d.sc[i], st);
    }
}

template <int TNX, int TLX, int TNY, int TLY>
__global__ void __launch_bounds__(256) k_batch_step(BatchDev d)
{
    extern __shared__ float4 smem_b[];
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
    stage_dt(d);
    if (!grid_barrier(d.g)) return;
    stage_sweep<0, TNX, TLX>(d, d.U, d.U2, smem_b);
    if (!grid_barrier(d.g)) return;
    stage_sweep<1, TNY, TLY>(d, d.U2, d.U, smem_b);
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
            sweepff_smem(a, b) > sweepff_smem(c, e) ? sweepff_smem(a, b) : sweepff_smem(c, e)}

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
FFP ffp_of(const DevParams &p);
cudaError_t launch_ff_in(const double *U, float2 *F, size_t m, cudaStream_t s);
cudaError_t launch_ff_out(const float2 *F, double *U, size_t m, cudaStream_t s);
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
    dimk::FFP *ffp;
    long long *off;
    int *ch;
    int *tx[dimk::kNumVariants], *ty[dimk::kNumVariants];
    Scalars *sc, *g;
    double *bs, *S, *beta;
    float *tbf, *rdf, *dtf;
    float2 *Uf, *Uf2;  // float-float state planes (packed) while steps run
    int *Pi;
    int viscous, heat, trelax;
    int nsm, maxb[dimk::kNumVariants];
    int variant, blocks;
    cudaGraphExec_t gexec;
    int gvariant, gblocks;
};

static void batch_free(dim_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->prm);
    cudaFree(b->ffp);
    cudaFree(b->off);
    cudaFree(b->ch);
    for (int v = 0; v < dimk::kNumVariants; v++) {
        cudaFree(b->tx[v]);
        cudaFree(b->ty[v]);
    }
    cudaFree(b->sc);
    cudaFree(b->g);
    cudaFree(b->bs);
    cudaFree(b->tbf);
    cudaFree(b->rdf);
    cudaFree(b->dtf);
    cudaFree(b->Uf);
    cudaFree(b->Uf2);
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

static dimk::BatchDev batch_dev(const dim_batch *b)
{
    dimk::BatchDev d;
    d.prm = b->prm;
    d.ffp = b->ffp;
    d.off = b->off;
    d.tx = b->tx[b->variant];
    d.ty = b->ty[b->variant];
    d.ch = b->ch;
    d.sc = b->sc;
    d.g = b->g;
    d.bs = b->bs;
    d.tbf = b->tbf;
    d.rdf = b->rdf;
    d.dtf = b->dtf;
    d.Pi = b->Pi;
    d.U = b->Uf;
    d.U2 = b->Uf2;
    d.S = b->S;
    d.ninst = b->ninst;
    d.viscous = b->viscous;
    d.heat = b->heat;
    d.trelax = b->trelax;
    return d;
}

// one step of the FF state on the internal stream (no graph)
static cudaError_t batch_step_direct(dim_batch *b, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->g, 0, offsetof(Scalars, status), s);
    if (e != cudaSuccess) return e;
    return dimk::batch_launch(b->variant, b->blocks, batch_dev(b), s);
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
    if (r == DIM_OK && hp->n_outer != 1) r = DIM_EINVAL;  // batches run one Algorithm-1 iteration
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
    dimk::FFP *ffp_h = (dimk::FFP *)calloc(ninst, sizeof(dimk::FFP));
    ok = ok && ffp_h;
    for (int i = 0; ok && i < ninst; i++) ffp_h[i] = dimk::ffp_of(b->prm_h[i]);
    ok = ok && cudaMalloc(&b->ffp, sizeof(dimk::FFP) * ninst) == cudaSuccess &&
         cudaMemcpy(b->ffp, ffp_h, sizeof(dimk::FFP) * ninst, cudaMemcpyHostToDevice) == cudaSuccess;
    free(ffp_h);
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
         cudaMalloc(&b->tbf, sizeof(float) * 3 * ninst * 2 * dimk::PMAX) == cudaSuccess &&
         cudaMalloc(&b->rdf, sizeof(float) * 3 * ninst * 2 * dimk::PMAX) == cudaSuccess &&
         cudaMalloc(&b->dtf, sizeof(float) * ninst) == cudaSuccess &&
         cudaMalloc(&b->Pi, sizeof(int) * 3 * ninst) == cudaSuccess &&
         cudaMalloc(&b->Uf, sizeof(float2) * 8 * N) == cudaSuccess &&
         cudaMalloc(&b->Uf2, sizeof(float2) * 8 * N) == cudaSuccess &&
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

// the caller's stream -> internal stream (state to FF planes, steps, back) ->
// the caller's stream
static int batch_run(dim_batch *b, double *U, int nsteps, bool use_graph)
{
    const size_t m = 8 * (size_t)b->ncell;
    if (cudaEventRecord(b->ev_in, b->user) != cudaSuccess || cudaStreamWaitEvent(b->own, b->ev_in, 0) != cudaSuccess)
        return DIM_ECUDA;
    if (nsteps > 0 && dimk::launch_ff_in(U, b->Uf, m, b->own) != cudaSuccess) return DIM_ECUDA;
    if (use_graph && nsteps > 0) {
        if (!b->gexec || b->gvariant != b->variant || b->gblocks != b->blocks) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DIM_ECUDA;
            cudaError_t e = batch_step_direct(b, b->own);
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
            b->gvariant = b->variant;
            b->gblocks = b->blocks;
        }
        for (int s = 0; s < nsteps; s++)
            if (cudaGraphLaunch(b->gexec, b->own) != cudaSuccess) return DIM_ECUDA;
    } else {
        for (int s = 0; s < nsteps; s++)
            if (batch_step_direct(b, b->own) != cudaSuccess) return DIM_ECUDA;
    }
    if (nsteps > 0 && dimk::launch_ff_out(b->Uf, U, m, b->own) != cudaSuccess) return DIM_ECUDA;
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
    const size_t m = 8 * (size_t)b->ncell;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaStreamSynchronize(b->user) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return DIM_ECUDA;
    }
    float best = 1e30f;
    int bv = 0, bb = b->maxb[0] * b->nsm;
    int rc = DIM_OK;
    // every trial starts from the caller's state converted into the FF planes
    // (the caller's U is only read)
    for (int v = 0; v < dimk::kNumVariants && rc == DIM_OK; v++) {
        for (int per = 1; per <= b->maxb[v] && rc == DIM_OK; per++) {
            if (per != 1 && per != b->maxb[v]) continue;
            b->variant = v;
            b->blocks = per * b->nsm;
            if (dimk::launch_ff_in(U, b->Uf, m, b->own) != cudaSuccess || batch_step_direct(b, b->own) != cudaSuccess ||
                cudaEventRecord(e0, b->own) != cudaSuccess || batch_step_direct(b, b->own) != cudaSuccess ||
                batch_step_direct(b, b->own) != cudaSuccess || cudaEventRecord(e1, b->own) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
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

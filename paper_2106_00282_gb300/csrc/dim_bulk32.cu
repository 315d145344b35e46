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
#include "dim_bulk32.cuh"

namespace dimk {
template <int AXIS, int TN, int TL>
__global__ void __launch_bounds__(TN *TL) k_sweep32(const DevParams p, const double *__restrict__ Uin,
                                                    double *__restrict__ Uout, double dt_host, Scalars *sc, int relax,
                                                    int check)
{
    extern __shared__ double smem[];
    const double dt = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    sweep32_tile<AXIS, TN, TL>(p, Uin, Uout, dt, sc, relax, check, blockIdx.x * TN, blockIdx.y * TL, smem);
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
        float p1 = (float)sg_p<true>(p, 0, q[4], a1), p2 = (float)sg_p<true>(p, 1, q[5], a2);
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

__global__ void __launch_bounds__(256) k_heat32(const DevParams p, double *U, HeatScratch32 s,
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
            unsigned r = equilibrium<true>(p, m1, m2, E1 + E2, T, a2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            U[4 * n + c] = m1 * p.cv[0] * T + (1.0 - a2) * p.pinf[0];
            U[5 * n + c] = m2 * p.cv[1] * T + a2 * p.pinf[1];
            U[7 * n + c] = a2;
        } else {
            T = mixture_T<true>(p, m1, m2, E1, E2, a2);
        }
        s.T0[c] = (float)T;
        float V, L;
        heat_coeffs_f(p, m1, m2, T, a2, V, L);
        s.V[c] = V;
        s.L[c] = L;
        s.Ia[c] = (float)((1.0 - a2) * p.src[0] + a2 * p.src[1]);
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
                vout[c] = (s.T0[c] + tb * vin[c] + tauf * s.V[c] * (Lv + s.Ia[c])) * rden;
            }
            if (!grid_barrier(sc)) return;
            vin = vout;
        }
        if (it == nout - 1) {
            for (int c = t0; c < n; c += nt) {
                double q = (double)lapf(p, neighbours(p, c), c, vin, s.L, idx2, idy2) + (double)s.Ia[c];
                double m1 = U[c], m2 = U[n + c];
                double rhoe = U[4 * n + c] + U[5 * n + c] + tau * q;
                double T, a2;
                unsigned r = equilibrium<true>(p, m1, m2, rhoe, T, a2);
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
                double q = (double)lapf(p, neighbours(p, c), c, vin, s.L, idx2, idy2) + (double)s.Ia[c];
                double T, a2;
                unsigned r = equilibrium<true>(p, U[c], U[n + c], U[4 * n + c] + U[5 * n + c] + tau * q, T, a2);
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
                s.Ia[c] = (float)((1.0 - s.Ai[c]) * p.src[0] + s.Ai[c] * p.src[1]);
            }
        }
    }
    flag(sc, st);
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_visc32(const DevParams p, double *U, ViscScratch32 s,
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
            unsigned r = prelax<true>(p, q);
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

static int g_heat32_blocks = 0, g_visc32_blocks[2] = {0, 0};

// the FP32 sweep kernels' shared-memory limit (once per device)
cudaError_t sweep32_setup()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep32<0, SX32_TN, SX32_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep32_smem(SX32_TN, SX32_TL));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep32<1, SY32_TN, SY32_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep32_smem(SY32_TN, SY32_TL));
}

cudaError_t bulk32_setup(int nsm)
{
    cudaError_t e = sweep32_setup();
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
    HeatScratch32 hs{F, F + n, F + 2 * n, F + 3 * n, F + 4 * n, F + 5 * n, F + 6 * n, S};
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

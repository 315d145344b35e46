// dim_parabolic.cu -- parabolic stages by the Chebyshev local-iteration method
// (Sec. 3.2, Eqs. LIM, LIM_last) as persistent cooperative kernels (sm_103a).
//
// The number of Chebyshev parameters P depends on lambda_max, a grid-wide
// reduction, so it is only known on the device.  One cooperative launch per
// stage runs: coefficients -> barrier -> lambda_max reduction -> barrier ->
// schedule b_m (per block, in shared memory) -> 2P-2 predictor sweeps, each
// followed by a barrier -> the conservative last sweep and the stage's
// pointwise epilogue.  No host round trip, any P up to PMAX.
//
// k_heat   Sec. 3.4.2 / Algorithm 1 (optionally preceded by the temperature
//          relaxation of Sec. 3.4.1 in the same launch).
// k_visc   Sec. 3.2 along one axis, optionally followed by the pressure
//          relaxation of Sec. 3.3.
#include <cooperative_groups.h>

#include "dim_device.cuh"

namespace dimk {


// (L_h v)_c = Fx_{+} - Fx_{-} + Fy_{+} - Fy_{-}, F = Lam_f (v_R - v_L) / h^2,
// Lam_f = mean of the two cells (Eq. qk_dis in flux-difference form), read from
// the face planes Lfx, Lfy (the face after each cell; the face before a cell is
// the face after its predecessor)
__device__ __forceinline__ double lap(const DevParams &p, const Nb &nb, int c, const double *v, const double *Lfx,
                                      const double *Lfy)
{
    double r = 0.0;
    double vc = v[c];
    if (p.nx > 1) {
        double fl = nb.xm >= 0 ? Lfx[nb.xm] * (vc - v[nb.xm]) * p.idx2 : 0.0;
        double fr = nb.xp >= 0 ? Lfx[c] * (v[nb.xp] - vc) * p.idx2 : 0.0;
        r += fr - fl;
    }
    if (p.ny > 1) {
        double fl = nb.ym >= 0 ? Lfy[nb.ym] * (vc - v[nb.ym]) * p.idy2 : 0.0;
        double fr = nb.yp >= 0 ? Lfy[c] * (v[nb.yp] - vc) * p.idy2 : 0.0;
        r += fr - fl;
    }
    return r;
}

// the face means 0.5 (Lam_c + Lam_next) after cell c along x and y (unused at a wall)
__device__ __forceinline__ void face_means(const DevParams &p, const Nb &nb, int c, const double *L, double *Lfx,
                                           double *Lfy)
{
    const double Lc = L[c];
    if (p.nx > 1 && nb.xp >= 0) Lfx[c] = 0.5 * (Lc + L[nb.xp]);
    if (p.ny > 1 && nb.yp >= 0) Lfy[c] = 0.5 * (Lc + L[nb.yp]);
}

// Gershgorin row bound 2 V_c sum_f Lam_f / h_f^2 of A = -V L_h
__device__ __forceinline__ double gersh(const DevParams &p, const Nb &nb, int c, const double *V, const double *L)
{
    double Lc = L[c];
    double s = 0.0;
    if (p.nx > 1) {
        double fl = nb.xm >= 0 ? 0.5 * (L[nb.xm] + Lc) : 0.0;
        double fr = nb.xp >= 0 ? 0.5 * (Lc + L[nb.xp]) : 0.0;
        s += (fl + fr) * p.idx2;
    }
    if (p.ny > 1) {
        double fl = nb.ym >= 0 ? 0.5 * (L[nb.ym] + Lc) : 0.0;
        double fr = nb.yp >= 0 ? 0.5 * (Lc + L[nb.yp]) : 0.0;
        s += (fl + fr) * p.idy2;
    }
    return 2.0 * V[c] * s;
}

// ---------------------------------------------------------------------------
// heat conduction (Algorithm 1 with the LIM)
// ---------------------------------------------------------------------------
// VARIANTS: compiled with the paper's midpoint temperature relaxation and the
// linear (T, alpha) update (chosen by p.trelax / p.heat_alpha); the default
// instantiation holds only the equilibrium relaxation and projection.
template <bool VARIANTS>
__global__ void __launch_bounds__(256) k_heat(const DevParams p, double *U, HeatScratch s,
                                              Scalars *sc, double dt_host, int trelax_first, int check)
{
    __shared__ double s_b[2 * PMAX];
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const double tau = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const int nout = p.n_outer < 1 ? 1 : (p.n_outer > 8 ? 8 : p.n_outer);
    unsigned st = 0;

    // A. (temperature relaxation,) temperature and frozen coefficients
    for (int c = t0; c < n; c += nt) {
        double m1 = U[c], m2 = U[n + c], E1 = U[4 * n + c], E2 = U[5 * n + c], a2 = U[7 * n + c];
        double T;
        if (trelax_first) {
            unsigned r = VARIANTS ? trelax_cell(p, m1, m2, E1, E2, a2, T, a2) : equilibrium(p, m1, m2, E1 + E2, T, a2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            U[4 * n + c] = m1 * p.cv[0] * T + (1.0 - a2) * p.pinf[0];
            U[5 * n + c] = m2 * p.cv[1] * T + a2 * p.pinf[1];
            U[7 * n + c] = a2;
            // temperature of the relaxed energies, as a later heat stage would read it
            T = mixture_T(p, m1, m2, U[4 * n + c], U[5 * n + c], a2);
        } else {
            T = mixture_T(p, m1, m2, E1, E2, a2);
        }
        s.T0[c] = T;
        double V, L;
        heat_coeffs(p, m1, m2, T, a2, V, L);
        s.V[c] = V;
        s.L[c] = L;
        const double Ia = (1.0 - a2) * p.src[0] + a2 * p.src[1];
        s.Ia[c] = Ia;
        s.tV[c] = tau * V;
        s.tf[c] = tau * (V * Ia);
    }

    size_t hoff = 0;  // history planes used by the earlier outer iterations
    for (int it = 0; it < nout; it++) {
        if (!grid_barrier(sc)) return;
        // B. face means of Lam and lambda_max (Gershgorin) of this iteration's
        //    frozen operator
        {
            double lm = 0.0;
            for (int c = t0; c < n; c += nt) {
                const Nb nb = neighbours(p, c);
                face_means(p, nb, c, s.L, s.Lfx, s.Lfy);
                if (!p.frozen) lm = fmax(lm, gersh(p, nb, c, s.V, s.L));
            }
            if (!p.frozen) block_max_to(&sc->lam[it], lm);
        }
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
        if (s.hist) {
            for (int c = t0; c < n; c += nt) {
                s.hist[hoff * n + c] = it == 0 ? s.T0[c] : s.Ti[c];
                s.hist[(hoff + 1) * n + c] = it == 0 ? U[7 * n + c] : s.Ai[c];
            }
        }
        // C. the 2P-2 predictor sweeps from v^(0) = T^n
        const double *vin = s.T0;
        for (int m = 1; m <= 2 * P - 2; m++) {
            double *vout = s.hist ? s.hist + (hoff + 1 + m) * n : ((m & 1) ? s.va : s.vb);
            const double bm = s_b[m - 1];
            const double rden = 1.0 / (1.0 + tau * bm);
            for (int c = t0; c < n; c += nt) {
                double Lv = lap(p, neighbours(p, c), c, vin, s.Lfx, s.Lfy);
                vout[c] = (s.T0[c] + tau * bm * vin[c] + s.tV[c] * Lv + s.tf[c]) * rden;
            }
            if (!grid_barrier(sc)) return;
            vin = vout;
        }
        hoff += 2 * (size_t)P;
        // D. last (explicit, b = 0) sweep in conservative form on the energy and
        //    the projection onto the p,T-equilibrium manifold (or the linear
        //    update T = T^n + tau V q, a = a^n + tau U q of Eqs. ht_eq2_ht, ht_eq3_ht
        //    with the V, U this iteration froze)
        const bool linear = VARIANTS && p.heat_alpha == DIM_HEAT_ALPHA_LINEAR;
        if (it == nout - 1) {
            for (int c = t0; c < n; c += nt) {
                double q = lap(p, neighbours(p, c), c, vin, s.Lfx, s.Lfy) + s.Ia[c];
                double m1 = U[c], m2 = U[n + c];
                double rhoe = U[4 * n + c] + U[5 * n + c] + tau * q;
                double T, a2;
                unsigned r = 0;
                if (linear) {
                    const double Tit = it == 0 ? s.T0[c] : s.Ti[c], ait = it == 0 ? U[7 * n + c] : s.Ai[c];
                    const double Uc = heat_U(p, m1, m2, Tit, ait, s.V[c]);
                    T = s.T0[c] + tau * s.V[c] * q;
                    a2 = U[7 * n + c] + tau * Uc * q;
                    if (!(gt0_i(a2) && lt_i(a2, 1.0) && gt0_i(T))) r |= DIM_ST_NONPHYS;
                    if (nan_i(a2) || nan_i(T)) r |= DIM_ST_NAN;
                } else {
                    r = equilibrium(p, m1, m2, rhoe, T, a2);
                }
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
                double q = lap(p, neighbours(p, c), c, vin, s.Lfx, s.Lfy) + s.Ia[c];
                double T, a2;
                if (linear) {
                    const double Tit = it == 0 ? s.T0[c] : s.Ti[c], ait = it == 0 ? U[7 * n + c] : s.Ai[c];
                    const double Uc = heat_U(p, U[c], U[n + c], Tit, ait, s.V[c]);
                    T = s.T0[c] + tau * s.V[c] * q;
                    a2 = U[7 * n + c] + tau * Uc * q;
                } else {
                    unsigned r = equilibrium(p, U[c], U[n + c], U[4 * n + c] + U[5 * n + c] + tau * q, T, a2);
                    if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
                }
                // every thread reads and writes only its own cells here
                s.Ti[c] = T;
                s.Ai[c] = a2;
            }
            if (!grid_barrier(sc)) return;
            for (int c = t0; c < n; c += nt) {
                double V, L;
                heat_coeffs(p, U[c], U[n + c], s.Ti[c], s.Ai[c], V, L);
                s.V[c] = V;
                s.L[c] = L;
                const double Ia = (1.0 - s.Ai[c]) * p.src[0] + s.Ai[c] * p.src[1];
                s.Ia[c] = Ia;
                s.tV[c] = tau * V;
                s.tf[c] = tau * (V * Ia);
            }
        }
    }
    flag(sc, st);
}

// ---------------------------------------------------------------------------
// viscous step along one axis (Sec. 3.2)
// ---------------------------------------------------------------------------
// rho du_n/dt = d(4/3 mu du_n/dh)/dh, rho du_t/dt = d(mu du_t/dh)/dh by the LIM
// with V = 1/rho; conservative last sweep on rho u; rho E and E_k from the
// face fluxes with two-cell face means and u_hat_i in place of u_i.
template <int AXIS>
__device__ __forceinline__ void visc_nb(const DevParams &p, int c, int &cm, int &cp)
{
    Nb nb = neighbours(p, c);
    cm = AXIS == 0 ? nb.xm : nb.ym;
    cp = AXIS == 0 ? nb.xp : nb.yp;
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_visc(const DevParams p, double *U, ViscScratch s, Scalars *sc,
                                              double dt_host, int relax, int check)
{
    __shared__ double s_b[2 * PMAX];
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    constexpr int SLOT = AXIS == 0 ? LAM_VX : LAM_VY;
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const double tau = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const double ih2 = AXIS == 0 ? p.idx2 : p.idy2;
    const double ih = AXIS == 0 ? 1.0 / p.dx : 1.0 / p.dy;
    unsigned st = 0;

    // mixture viscosity of a cell from alpha_2 (U is not written before phase D)
    auto mu_of = [&](int c) {
        double a2 = U[7 * n + c];
        return (1.0 - a2) * p.mu[0] + a2 * p.mu[1];
    };
    // A. velocities, V = 1/rho, alpha_2 snapshot; face coefficients 4/3 mu_f
    //    and mu_f (two-cell means) at the face after each cell
    for (int c = t0; c < n; c += nt) {
        double rho = U[c] + U[n + c];
        const double V = 1.0 / rho;
        s.V[c] = V;
        s.tV[c] = tau * V;
        s.A2[c] = U[7 * n + c];
        s.u0[c] = U[QN * n + c] / rho;
        s.w0[c] = U[QT * n + c] / rho;
        int cm, cp;
        visc_nb<AXIS>(p, c, cm, cp);
        if (cp >= 0) {
            const double mc = mu_of(c), mr = mu_of(cp);
            s.LN[c] = 0.5 * (4.0 / 3.0 * mc + 4.0 / 3.0 * mr);
            s.LM[c] = 0.5 * (mc + mr);
        }
    }
    if (!grid_barrier(sc)) return;
    // B. lambda_max with the normal coefficient 4/3 mu (bounds the tangential one too)
    if (!p.frozen) {
        double lm = 0.0;
        for (int c = t0; c < n; c += nt) {
            int cm, cp;
            visc_nb<AXIS>(p, c, cm, cp);
            double fl = cm >= 0 ? s.LN[cm] : 0.0;
            double fr = cp >= 0 ? s.LN[c] : 0.0;
            lm = fmax(lm, 2.0 * s.V[c] * ((fl + fr) * ih2));
        }
        block_max_to(&sc->lam[SLOT], lm);
    }
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
    // C. predictor sweeps on u_n (4/3 mu) and u_t (mu)
    const double *uin = s.u0, *win = s.w0;
    const size_t M = 2 * (size_t)P - 2;
    for (int m = 1; m <= 2 * P - 2; m++) {
        double *uo = s.hist ? s.hist + (size_t)(m - 1) * n : ((m & 1) ? s.ua : s.ub);
        double *wo = s.hist ? s.hist + (M + m - 1) * n : ((m & 1) ? s.wa : s.wb);
        const double bm = s_b[m - 1];
        const double rden = 1.0 / (1.0 + tau * bm);
        for (int c = t0; c < n; c += nt) {
            int cm, cp;
            visc_nb<AXIS>(p, c, cm, cp);
            double uc = uin[c], wc = win[c];
            double Lu = (cp >= 0 ? s.LN[c] * (uin[cp] - uc) * ih2 : 0.0) -
                        (cm >= 0 ? s.LN[cm] * (uc - uin[cm]) * ih2 : 0.0);
            double Lw = (cp >= 0 ? s.LM[c] * (win[cp] - wc) * ih2 : 0.0) -
                        (cm >= 0 ? s.LM[cm] * (wc - win[cm]) * ih2 : 0.0);
            uo[c] = (s.u0[c] + tau * bm * uc + s.tV[c] * Lu) * rden;
            wo[c] = (s.w0[c] + tau * bm * wc + s.tV[c] * Lw) * rden;
        }
        if (!grid_barrier(sc)) return;
        uin = uo;
        win = wo;
    }
    // D1. the face values of the conservative last sweep, once per face (the
    //     face after cell c, between c and its successor)
    const size_t fn = (size_t)n;
    for (int c = t0; c < n; c += nt) {
        int cm, cp;
        visc_nb<AXIS>(p, c, cm, cp);
        if (cp < 0) continue;
        const int cl = c, cr = cp;
        double Fn = s.LN[c] * (uin[cr] - uin[cl]) * ih;
        double Ft = s.LM[c] * (win[cr] - win[cl]) * ih;
        double ubar = 0.5 * (uin[cl] + uin[cr]);
        double wbar = 0.5 * (win[cl] + win[cr]);
        double W = ubar * Fn + wbar * Ft;
        double a2l = s.A2[cl], a2r = s.A2[cr];
        double aF2 = 0.5 * (a2l + a2r);
        double aF1 = 0.5 * ((1.0 - a2l) + (1.0 - a2r));
        s.F[VF_FN * fn + c] = Fn;
        s.F[VF_FT * fn + c] = Ft;
        s.F[VF_W * fn + c] = W;
        s.F[VF_A1W * fn + c] = aF1 * W;
        s.F[VF_A1FN * fn + c] = aF1 * Fn;
        s.F[VF_A1FT * fn + c] = aF1 * Ft;
        s.F[VF_A2W * fn + c] = aF2 * W;
        s.F[VF_A2FN * fn + c] = aF2 * Fn;
        s.F[VF_A2FT * fn + c] = aF2 * Ft;
    }
    if (!grid_barrier(sc)) return;
    // D2. conservative update and energies of each cell from its two faces
    for (int c = t0; c < n; c += nt) {
        int cm, cp;
        visc_nb<AXIS>(p, c, cm, cp);
        double f[2][VF_N];
#pragma unroll
        for (int k = 0; k < VF_N; k++) {
            f[0][k] = cm >= 0 ? s.F[k * fn + cm] : 0.0;
            f[1][k] = cp >= 0 ? s.F[k * fn + c] : 0.0;
        }
        double uh = uin[c], wh = win[c];
        double q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
        q[QN] = q[QN] + tau * (f[1][VF_FN] - f[0][VF_FN]) * ih;
        q[QT] = q[QT] + tau * (f[1][VF_FT] - f[0][VF_FT]) * ih;
        q[6] = q[6] + tau * (f[1][VF_W] - f[0][VF_W]) * ih;
        q[4] = q[4] + tau * (f[1][VF_A1W] - f[0][VF_A1W]) * ih -
               tau * (uh * (f[1][VF_A1FN] - f[0][VF_A1FN]) + wh * (f[1][VF_A1FT] - f[0][VF_A1FT])) * ih;
        q[5] = q[5] + tau * (f[1][VF_A2W] - f[0][VF_A2W]) * ih -
               tau * (uh * (f[1][VF_A2FN] - f[0][VF_A2FN]) + wh * (f[1][VF_A2FT] - f[0][VF_A2FT])) * ih;
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
static int g_heat_blocks[2] = {0, 0}, g_visc_blocks[2] = {0, 0};

cudaError_t parabolic_setup(int nsm)
{
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_heat<false>, 256, 0);
    if (e != cudaSuccess) return e;
    g_heat_blocks[0] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_heat<true>, 256, 0);
    if (e != cudaSuccess) return e;
    g_heat_blocks[1] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_visc<0>, 256, 0);
    if (e != cudaSuccess) return e;
    g_visc_blocks[0] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_visc<1>, 256, 0);
    if (e != cudaSuccess) return e;
    g_visc_blocks[1] = b * nsm;
    return cudaSuccess;
}

static int coop_grid(int maxb, int n)
{
    int need = (n + 255) / 256;
    return need < maxb ? need : maxb;
}

cudaError_t launch_heat(const DevParams &p, double *U, const HeatScratch &s, Scalars *sc, double dt_host,
                        int trelax_first, int check, cudaStream_t st)
{
    DevParams pp = p;
    HeatScratch ss = s;
    void *args[] = {(void *)&pp, (void *)&U, (void *)&ss, (void *)&sc, (void *)&dt_host, (void *)&trelax_first,
                    (void *)&check};
    const int var = p.trelax == DIM_TRELAX_MIDPOINT || p.heat_alpha == DIM_HEAT_ALPHA_LINEAR;
    const void *f = var ? (const void *)k_heat<true> : (const void *)k_heat<false>;
    return cudaLaunchCooperativeKernel(f, dim3(coop_grid(g_heat_blocks[var], p.n)), dim3(256), args, 0, st);
}

cudaError_t launch_visc(const DevParams &p, int axis, double *U, const ViscScratch &s, Scalars *sc, double dt_host,
                        int relax, int check, cudaStream_t st)
{
    DevParams pp = p;
    ViscScratch ss = s;
    void *args[] = {(void *)&pp, (void *)&U, (void *)&ss, (void *)&sc, (void *)&dt_host, (void *)&relax,
                    (void *)&check};
    const void *f = axis == 0 ? (const void *)k_visc<0> : (const void *)k_visc<1>;
    return cudaLaunchCooperativeKernel(f, dim3(coop_grid(g_visc_blocks[axis], p.n)), dim3(256), args, 0, st);
}

}  // namespace dimk

// dim_sweep.cu -- hyperbolic directional sweep and pointwise kernels (sm_103a).
//
// k_sweep<AXIS>: one Godunov/HLLC sweep of the six-equation system (Sec. 3.1,
// Eq. vectorForm) with PVT-consistent minmod MUSCL reconstruction (Sec. 3.6)
// and, fused into the epilogue, the pressure relaxation of Sec. 3.3.
//
// Tiling: a block owns TN cells along the sweep axis times TL lines.  It stages
// the 8 conserved planes of its TN+4 cells per line (2 ghosts per side) in
// shared memory with coalesced loads (the x-sweep walks along rows; the
// y-sweep loads TL adjacent columns per row so each warp reads contiguous
// x), converts them to primitives once, computes the TN+1 face fluxes per line
// from shared memory, and writes the TN updated cells.  Out of place: Uin ->
// Uout (neighbouring tiles read the old state).
#include "dim_device.cuh"

namespace dimk {

// primitive W = (alpha_2, m1, m2, u_n, u_t, p1, p2) from a line-local state
// (m1, m2, rho u_n, rho u_t, E1, E2, rho E, alpha_2)
__device__ __forceinline__ void prims(const DevParams &p, const double *q, double *w)
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

struct Face {
    double a2, un, ut, rho, p, c;
    double q[NQ];
};

__device__ __forceinline__ void face_state(const DevParams &p, const double *w, Face &s)
{
    double a2 = w[0], a1 = 1.0 - a2;
    double m1 = w[1], m2 = w[2], un = w[3], ut = w[4], p1 = w[5], p2 = w[6];
    double rho = m1 + m2;
    double E1 = sg_E(p, 0, p1, a1), E2 = sg_E(p, 1, p2, a2);
    s.a2 = a2;
    s.un = un;
    s.ut = ut;
    s.rho = rho;
    s.p = a1 * p1 + a2 * p2;
    s.c = mix_c(p, a1, p1, a2, p2, rho);
    s.q[0] = m1;
    s.q[1] = m2;
    s.q[2] = rho * un;
    s.q[3] = rho * ut;
    s.q[4] = E1;
    s.q[5] = E2;
    s.q[6] = E1 + E2 + 0.5 * rho * (un * un + ut * ut);
    s.q[7] = a2;
}

// HLLC state at x/t = 0 and its flux F = u* U* + p* D(u*), D = [0 0 1 0 0 0 u* 0];
// Davis bounds; phase masses and energies scale like rho across the acoustic
// waves, alpha_2 is continuous there (exact isolated contacts, Sec. 3.5)
__device__ __forceinline__ void hllc(const Face &L, const Face &R, double *F)
{
    double SL = fmin(L.un - L.c, R.un - R.c);
    double SR = fmax(L.un + L.c, R.un + R.c);
    double Ss = (R.p - L.p + L.rho * L.un * (SL - L.un) - R.rho * R.un * (SR - R.un)) /
                (L.rho * (SL - L.un) - R.rho * (SR - R.un));
    double q[NQ], us, ps;
    const bool starL = ge0_i(Ss);
    if (ge0_i(SL)) {
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = L.q[k];
        us = L.un;
        ps = L.p;
    } else if (ge0_i(SR)) {
        const Face &K = starL ? L : R;
        double SK = starL ? SL : SR;
        double chi = (SK - K.un) / (SK - Ss);
        q[0] = chi * K.q[0];
        q[1] = chi * K.q[1];
        q[2] = chi * K.rho * Ss;
        q[3] = chi * K.rho * K.ut;
        q[4] = chi * K.q[4];
        q[5] = chi * K.q[5];
        q[6] = chi * (K.q[6] + (Ss - K.un) * (K.rho * Ss + K.p / (SK - K.un)));
        q[7] = K.a2;
        us = Ss;
        ps = K.p + K.rho * (SK - K.un) * (Ss - K.un);
    } else {
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = R.q[k];
        us = R.un;
        ps = R.p;
    }
    F[0] = us * q[0];
    F[1] = us * q[1];
    F[2] = us * q[2] + ps;
    F[3] = us * q[3];
    F[4] = us * q[4];
    F[5] = us * q[5];
    F[6] = us * (q[6] + ps);
    F[7] = us * q[7];
    F[8] = us;
}

__device__ __forceinline__ int bc_map(int a, int len, int bc)
{
    if (a >= 0 && a < len) return a;
    if (bc == DIM_BC_PERIODIC) return ((a % len) + len) % len;
    return a < 0 ? 0 : len - 1;
}

// minimum resident blocks per SM the register allocation must allow: 3 (80
// registers) keeps 24 warps per SM on the 256-thread tiles, 1-2 % faster than
// the unconstrained 92-96 registers (timed on the GPU); a build may override it
#ifndef DIM_SX_MINB
#define DIM_SX_MINB 3
#endif
#ifndef DIM_SY_MINB
#define DIM_SY_MINB 3
#endif

template <int AXIS, int TN, int TL>
__global__ void __launch_bounds__(TN *TL, AXIS == 0 ? DIM_SX_MINB : DIM_SY_MINB)
    k_sweep(const DevParams p, const double *__restrict__ Uin,
                                                  double *__restrict__ Uout, double dt_host, Scalars *sc, int relax,
                                                  int check)
{
    extern __shared__ double smem[];
    constexpr int NE = TN + 4;  // cells per line with ghosts
    constexpr int NL = NE * TL;
    constexpr int NFL = TN + 1;  // faces per line
    constexpr int NF = NFL * TL;
    double *sU = smem;         // [8][NL]
    double *sW = sU + NQ * NL;  // [7][NL]
    double *sF = sW + 7 * NL;   // [9][NF]
    double *sS = sF + 9 * NF;   // [7][NL] limited slopes (twice minmod for Overbee on alpha_2, m1, m2)
    const int n = p.n;
    const int len = AXIS == 0 ? p.nx : p.ny;
    const int ntr = AXIS == 0 ? p.ny : p.nx;
    const int a0 = blockIdx.x * TN;
    const int t0 = blockIdx.y * TL;
    const double dt = dt_host > 0.0 ? dt_host : p.cfl / dmax_bits(sc->smax);
    const double dtdx = dt / (AXIS == 0 ? p.dx : p.dy);
    // global plane of line-local component k: normal and tangential momentum swap for y
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;

    // smem index of cell e of line l; x-sweep: e fastest, y-sweep: l fastest
    auto cidx = [&](int e, int l) { return AXIS == 0 ? l * NE + e : e * TL + l; };
    auto fidx = [&](int f, int l) { return AXIS == 0 ? l * NFL + f : f * TL + l; };

    // 1. stage U and primitives of the tile and its ghosts
    for (int li = threadIdx.x; li < NL; li += blockDim.x) {
        int e, l;
        if (AXIS == 0) { l = li / NE; e = li - l * NE; }
        else { e = li / TL; l = li - e * TL; }
        int tr = min(t0 + l, ntr - 1);
        int al = bc_map(a0 - 2 + e, len, p.bc[AXIS]);
        int x = AXIS == 0 ? al : tr, y = AXIS == 0 ? tr : al;
        int c = y * p.nx + x;
        double q[NQ];
        q[0] = Uin[0 * n + c];
        q[1] = Uin[1 * n + c];
        q[2] = Uin[QN * n + c];
        q[3] = Uin[QT * n + c];
        q[4] = Uin[4 * n + c];
        q[5] = Uin[5 * n + c];
        q[6] = Uin[6 * n + c];
        q[7] = Uin[7 * n + c];
        double w[7];
        prims(p, q, w);
#pragma unroll
        for (int k = 0; k < NQ; k++) sU[k * NL + li] = q[k];
#pragma unroll
        for (int k = 0; k < 7; k++) sW[k * NL + li] = w[k];
    }
    __syncthreads();

    // 1b. the limited slope of every cell with both neighbours in the tile, once
    //     per cell (each is used by the faces on both sides)
    const bool lim = p.limiter != DIM_LIMITER_NONE, ob = p.limiter == DIM_LIMITER_OVERBEE;
    if (lim) {
        for (int li = threadIdx.x; li < NL; li += blockDim.x) {
            int e, l;
            if (AXIS == 0) { l = li / NE; e = li - l * NE; }
            else { e = li / TL; l = li - e * TL; }
            if (e < 1 || e > NE - 2) continue;
            const int im = cidx(e - 1, l), ip = cidx(e + 1, l);
#pragma unroll
            for (int k = 0; k < 7; k++) {
                const double *Wk = sW + k * NL;
                double sl = minmod(Wk[li] - Wk[im], Wk[ip] - Wk[li]);
                if (ob && k <= 2) sl = 2.0 * sl;  // Overbee on alpha_2, m1, m2: twice the minmod slope
                sS[k * NL + li] = sl;
            }
        }
        __syncthreads();
    }

    // 2. face fluxes: face f of line l lies between cells e = f+1 and e = f+2
    for (int fi = threadIdx.x; fi < NF; fi += blockDim.x) {
        int f, l;
        if (AXIS == 0) { l = fi / NFL; f = fi - l * NFL; }
        else { f = fi / TL; l = fi - f * TL; }
        const int iL = cidx(f + 1, l), iR = cidx(f + 2, l);
        double wl[7], wr[7];
        if (lim) {
#pragma unroll
            for (int k = 0; k < 7; k++) {
                const double *Wk = sW + k * NL;
                wl[k] = Wk[iL] + 0.5 * sS[k * NL + iL];
                wr[k] = Wk[iR] - 0.5 * sS[k * NL + iR];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 7; k++) {
                wl[k] = sW[k * NL + iL];
                wr[k] = sW[k * NL + iR];
            }
        }
        Face L, R;
        face_state(p, wl, L);
        face_state(p, wr, R);
        double F[9];
        hllc(L, R, F);
#pragma unroll
        for (int k = 0; k < 9; k++) sF[k * NF + fi] = F[k];
    }
    __syncthreads();

    // 3. conservative update with the non-conservative term
    //    U_i -= dt/dx (F_{i+1/2} - F_{i-1/2}) + dt/dx R(U_i^n)(u*_{i+1/2} - u*_{i-1/2}),
    //    R = [0 0 0 0 a1p1 a2p2 0 -a2]; then the pressure relaxation
    unsigned st = 0;
    for (int oi = threadIdx.x; oi < TN * TL; oi += blockDim.x) {
        int i, l;
        if (AXIS == 0) { l = oi / TN; i = oi - l * TN; }
        else { i = oi / TL; l = oi - i * TL; }
        int al = a0 + i, tr = t0 + l;
        if (al >= len || tr >= ntr) continue;
        const int ci = cidx(i + 2, l), fm = fidx(i, l), fp = fidx(i + 1, l);
        double a2 = sW[0 * NL + ci], a1 = 1.0 - a2;
        double Rv[NQ] = {0.0, 0.0, 0.0, 0.0, a1 * sW[5 * NL + ci], a2 * sW[6 * NL + ci], 0.0, -a2};
        double du = sF[8 * NF + fp] - sF[8 * NF + fm];
        double qo[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            qo[k] = sU[k * NL + ci] - dtdx * (sF[k * NF + fp] - sF[k * NF + fm]);
            if (k == 4 || k == 5 || k == 7) qo[k] = qo[k] - dtdx * Rv[k] * du;  // the rows R is nonzero in
        }
        // back to the global plane order
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

// ---------------------------------------------------------------------------
// pointwise kernels
// ---------------------------------------------------------------------------
__global__ void k_from_primitive(const DevParams p, const double *__restrict__ prim, double *__restrict__ U,
                                 Scalars *sc)
{
    const int n = p.n;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double a2 = prim[c], pr = prim[n + c], T = prim[2 * n + c], u = prim[3 * n + c], v = prim[4 * n + c];
        double a1 = 1.0 - a2;
        // Eq. eos_stiffened2: rho_k = (p + pinf_k) / ((gamma_k - 1) Cv_k T)
        double r1 = (pr + p.pinf[0]) / (p.gm1[0] * p.cv[0] * T);
        double r2 = (pr + p.pinf[1]) / (p.gm1[1] * p.cv[1] * T);
        double m1 = a1 * r1, m2 = a2 * r2, rho = m1 + m2;
        double E1 = sg_E(p, 0, pr, a1), E2 = sg_E(p, 1, pr, a2);
        U[c] = m1;
        U[n + c] = m2;
        U[2 * n + c] = rho * u;
        U[3 * n + c] = rho * v;
        U[4 * n + c] = E1;
        U[5 * n + c] = E2;
        U[6 * n + c] = E1 + E2 + 0.5 * rho * (u * u + v * v);
        U[7 * n + c] = a2;
        if (!(gt0_i(a2) && lt_i(a2, 1.0) && gt0_i(T) && gt0_i(pr + p.pinf[0]) && gt0_i(pr + p.pinf[1])))
            st |= DIM_ST_NONPHYS;
    }
    flag(sc, st);
}

// max over cells of (|u_axis| + c) / h_axis, active axes only; also checks that
// the state entering the step is admissible
__global__ void k_wave_max(const DevParams p, const double *__restrict__ U, Scalars *sc)
{
    const int n = p.n;
    double m = 0.0;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
        st |= check_state(p, q);
        double rho = q[0] + q[1];
        double cs = cell_c(p, q[0], q[1], q[4], q[5], q[7]);
        if (p.nx > 1) {
            double s = (fabs(q[2] / rho) + cs) * p.idx;
            if (lt_i(m, s)) m = s;
            if (nan_i(s)) st |= DIM_ST_NAN;
        }
        if (p.ny > 1) {
            double s = (fabs(q[3] / rho) + cs) * p.idy;
            if (lt_i(m, s)) m = s;
            if (nan_i(s)) st |= DIM_ST_NAN;
        }
    }
    block_max_to(&sc->smax, m);
    flag(sc, st);
}

// pointwise relaxation in place: which = DIM_RELAX_PRESSURE or DIM_RELAX_TEMPERATURE
__global__ void k_relax(const DevParams p, double *__restrict__ U, Scalars *sc, int which, int check)
{
    const int n = p.n;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = U[k * n + c];
        unsigned s;
        if (which == DIM_RELAX_PRESSURE) {
            s = prelax(p, q);
            U[4 * n + c] = q[4];
            U[5 * n + c] = q[5];
            U[7 * n + c] = q[7];
        } else {
            double T, a;
            s = trelax_cell(p, q[0], q[1], q[4], q[5], q[7], T, a);
            q[4] = q[0] * p.cv[0] * T + (1.0 - a) * p.pinf[0];
            q[5] = q[1] * p.cv[1] * T + a * p.pinf[1];
            q[7] = a;
            U[4 * n + c] = q[4];
            U[5 * n + c] = q[5];
            U[7 * n + c] = q[7];
        }
        if (check) st |= check_state(p, q) | (s & DIM_ST_NAN);
        else if (s & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
    }
    flag(sc, st);
}

// ---------------------------------------------------------------------------
// host-side launchers (called from dim_api.cu)
// ---------------------------------------------------------------------------
// tile shapes (cells along the sweep x lines); a build may override them
#ifndef DIM_SX_TN
#define DIM_SX_TN 256
#define DIM_SX_TL 1
#endif
#ifndef DIM_SY_TN
#define DIM_SY_TN 32
#define DIM_SY_TL 8
#endif
constexpr int SX_TN = DIM_SX_TN, SX_TL = DIM_SX_TL;
constexpr int SY_TN = DIM_SY_TN, SY_TL = DIM_SY_TL;

static size_t sweep_smem(int TN, int TL) { return sizeof(double) * ((TN + 4) * TL * (NQ + 7 + 7) + (TN + 1) * TL * 9); }

cudaError_t sweep_setup()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep<0, SX_TN, SX_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep_smem(SX_TN, SX_TL));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep<1, SY_TN, SY_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_smem(SY_TN, SY_TL));
}

cudaError_t launch_sweep(const DevParams &p, int axis, const double *Uin, double *Uout, double dt_host, Scalars *sc,
                         int relax, int check, cudaStream_t s)
{
    if (axis == 0) {
        dim3 grid((p.nx + SX_TN - 1) / SX_TN, (p.ny + SX_TL - 1) / SX_TL);
        k_sweep<0, SX_TN, SX_TL><<<grid, SX_TN * SX_TL, sweep_smem(SX_TN, SX_TL), s>>>(p, Uin, Uout, dt_host, sc,
                                                                                       relax, check);
    } else {
        dim3 grid((p.ny + SY_TN - 1) / SY_TN, (p.nx + SY_TL - 1) / SY_TL);
        k_sweep<1, SY_TN, SY_TL><<<grid, SY_TN * SY_TL, sweep_smem(SY_TN, SY_TL), s>>>(p, Uin, Uout, dt_host, sc,
                                                                                       relax, check);
    }
    return cudaGetLastError();
}

static int pw_grid(int n) { return (n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16; }

cudaError_t launch_from_primitive(const DevParams &p, const double *prim, double *U, Scalars *sc, cudaStream_t s)
{
    k_from_primitive<<<pw_grid(p.n), 256, 0, s>>>(p, prim, U, sc);
    return cudaGetLastError();
}

// one thread waits, bounded, on a word nothing writes (the failure path of the
// grid barriers' wait, exercised without stopping any other work)
__global__ void k_wait_selftest(Scalars *sc, const unsigned *word, long long limit)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!wait_while_equal(word, ld_acquire_u32(word), limit)) atomicOr(&sc->status, DIM_ST_TIMEOUT);
    }
}

cudaError_t launch_wait_selftest(Scalars *sc, const unsigned *word, long long limit, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(sc, word, limit);
    return cudaGetLastError();
}

cudaError_t launch_wave_max(const DevParams &p, const double *U, Scalars *sc, cudaStream_t s)
{
    k_wave_max<<<pw_grid(p.n), 256, 0, s>>>(p, U, sc);
    return cudaGetLastError();
}

cudaError_t launch_relax(const DevParams &p, double *U, Scalars *sc, int which, int check, cudaStream_t s)
{
    k_relax<<<pw_grid(p.n), 256, 0, s>>>(p, U, sc, which, check);
    return cudaGetLastError();
}

}  // namespace dimk

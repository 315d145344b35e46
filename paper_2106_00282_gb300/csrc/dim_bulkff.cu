// dim_bulkff.cu -- the FP32-bulk form of the split step (sm_103a): the same
// stages and launch structure as the FP64 kernels (dim_sweep.cu,
// dim_parabolic.cu) on a float-float copy of the state (dim_ff.cuh), with no
// FP64 instruction inside a step:
//   FF:   the conserved state and its accumulation; the phase pressures' E_k /
//         a_k - cold_k; the volume fraction, its reconstruction and flux, and
//         the cold energies it carries; the kinetic energy in the relaxations;
//   FP32: MUSCL reconstruction of m_k, u_n, u_t, p_k; face states, sound
//         speeds, HLLC; the relaxation roots (in the phase-pressure form of
//         dim_ff.cuh); viscous and heat coefficients; every Chebyshev sweep.
// The Chebyshev parameters b_m come from the FP64 root table once per block.
#include <cudaTypedefs.h>

#include "dim_ff.cuh"

namespace dimk {

// ---------------------------------------------------------------------------
// FP64 <-> FF planes
// ---------------------------------------------------------------------------
__global__ void k_ff_in(const double *__restrict__ U, float2 *__restrict__ F, size_t m)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        const ff a = ff_from_d(U[i]);
        F[i] = make_float2(a.h, a.l);
    }
}

// may run in place (F and U the same memory): each element is read before it is written
__global__ void k_ff_out(const float2 *F, double *U, size_t m)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = F[i];
        U[i] = ff_to_d(ff{v.x, v.y});
    }
}

// per-block time step: dt_host if positive, else the step's cfl / S published
// by the CFL kernel
__device__ __forceinline__ float block_dt(const Scalars *sc, double dt_host)
{
    __shared__ float s_dt;
    if (threadIdx.x == 0) s_dt = dt_host > 0.0 ? (float)dt_host : *(volatile const float *)&sc->dt32;
    __syncthreads();
    return s_dt;
}

// L2 prefetch of elements [i0, i1) of a plane (one thread; a bulk prefetch,
// fire and forget).  The range is widened to 16-byte boundaries, which stays
// inside the allocation: every plane set here (the FF state, the scratch) ends
// on a 16-byte boundary or is followed by another plane.
template <class T>
__device__ __forceinline__ void l2_prefetch(const T *plane, size_t i0, size_t i1)
{
    if (i1 <= i0) return;
    const size_t a = (size_t)(plane + i0) & ~(size_t)15, e = ((size_t)(plane + i1) + 15) & ~(size_t)15;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// CFL bound (Sec. 3.1) and input check.  FROM_D: the state is read from the
// caller's FP64 planes Ud and written to the FF planes U on the way (the first
// step of a call), instead of a separate conversion pass.
template <bool FROM_D>
__global__ void __launch_bounds__(256) k_wave_ff(const DevParams p, const FFP f, float2 *U, const double *Ud,
                                                 Scalars *sc)
{
    const int n = p.n;
    float m = 0.f;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        ff q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            if constexpr (FROM_D) {
                q[k] = ff_from_d(Ud[k * (size_t)n + c]);
                st_ff(U, k * (size_t)n + c, q[k]);
            } else {
                q[k] = ld_ff(U, k * (size_t)n + c);
            }
        }
        st |= ff_check(f, q);
        m = fmaxf(m, ff_wave_speed(p, f, q, st));
    }
    block_max_to_f(&sc->smax, m);
    flag(sc, st);
    // the last block to finish publishes dt = cfl / S as a float, once per step
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&sc->wave_blocks, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        sc->dt32 = (float)(p.cfl / read_acc(&sc->smax));
        sc->wave_blocks = 0;
    }
}

template <int AXIS, int TN, int TL, bool BOUND>
// one thread per staged cell (TN + 4 along the sweep): the load phase takes one
// cell per thread
__global__ void __launch_bounds__((TN + 4) * TL) k_sweepff(const DevParams p, const FFP f, const float2 *__restrict__ Uin,
                                                    float2 *__restrict__ Uout, double dt_host, Scalars *sc,
                                                    int relax, int check)
{
    extern __shared__ float4 smem_ff[];
    const float dtdx = block_dt(sc, dt_host) * (AXIS == 0 ? f.idx : f.idy);
    sweepff_tile<AXIS, TN, TL, BOUND>(p, f, Uin, Uout, dtdx, sc, relax, check, blockIdx.x * TN, blockIdx.y * TL,
                                      smem_ff);
}

// pointwise relaxation in place: DIM_RELAX_PRESSURE (Sec. 3.3) or
// DIM_RELAX_TEMPERATURE (Sec. 3.4.1 equilibrium), optionally with the
// end-of-step check
__global__ void __launch_bounds__(256) k_relaxff(const DevParams p, const FFP f, float2 *U, Scalars *sc, int which,
                                                 int check)
{
    const int n = p.n;
    unsigned st = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        ff q[NQ];
#pragma unroll
        for (int k = 0; k < NQ; k++) q[k] = ld_ff(U, k * (size_t)n + c);
        unsigned r;
        if (which == DIM_RELAX_PRESSURE) {
            r = ff_prelax(f, q);
        } else {
            float T;
            r = ff_equilibrium(f, q[0], q[1], ff_add(q[4], q[5]), T, q[7], q[4], q[5]);
        }
        if (check) st |= ff_check(f, q) | (r & DIM_ST_NAN);
        else st |= r & (DIM_ST_NAN | DIM_ST_NONPHYS | DIM_ST_NOROOT);
        st_ff(U, 4 * (size_t)n + c, q[4]);
        st_ff(U, 5 * (size_t)n + c, q[5]);
        st_ff(U, 7 * (size_t)n + c, q[7]);
    }
    flag(sc, st);
}

// Chebyshev parameters of one solve for the whole block: P (thread 0), then
// b_m, tau b_m and 1/(1 + tau b_m) per position (Sec. 3.2, Eq. LIM)
__device__ __forceinline__ int block_schedule(const DevParams &p, double tau, double lam, bool viscous, float *s_tb,
                                              float *s_rd, unsigned &capped)
{
    __shared__ int s_P;
    __shared__ unsigned s_cap;
    __shared__ double s_b[2 * PMAX];
    if (threadIdx.x == 0) {
        unsigned cp;
        s_P = viscous ? cheb_P_visc(p, tau, lam, cp) : cheb_P(p, tau, lam, cp);
        s_cap = cp;
    }
    __syncthreads();
    const int P = s_P;
    cheb_schedule_block(p, P, lam, s_b);
    __syncthreads();
    for (int s = threadIdx.x; s < 2 * P - 1; s += blockDim.x) {
        s_tb[s] = (float)(tau * s_b[s]);
        s_rd[s] = (float)(1.0 / (1.0 + tau * s_b[s]));
    }
    __syncthreads();
    capped = s_cap;
    return P;
}

// FP32 scratch of the heat stage (planes of n floats) and the FF volume
// fraction of an outer iteration
struct HeatFF {
    float *T0, *V, *L, *va, *vb, *Ti, *Ia;
    float2 *Ai;
    float *C0, *tV;  // T0 + tau V Ia and tau V: the constant terms of a predictor sweep
};


// The cells of the grid as (i, j, c), without an integer division per cell:
// row chunks of blockDim.x cells, one chunk per block iteration (grids at
// least one block wide), else a grid-stride loop.
// pf(c0, c1), when given, runs on thread 0 at the start of each chunk with the
// cells [c0, c1) of the block's next chunk (for L2 prefetches).
struct NoPf {
    __device__ void operator()(int, int) const {}
};
template <class F, class PF = NoPf>
__device__ __forceinline__ void for_cells(const DevParams &p, F &&fn, PF pf = PF())
{
    if (p.nx >= (int)blockDim.x) {
        const int nch = (p.nx + blockDim.x - 1) / blockDim.x;
        const int nw = p.ny * nch;
        for (int w = blockIdx.x; w < nw; w += gridDim.x) {
            if (threadIdx.x == 0 && w + (int)gridDim.x < nw) {
                const int wn = w + gridDim.x, jn = wn / nch, in = (wn - jn * nch) * blockDim.x;
                pf(jn * p.nx + in, jn * p.nx + min(in + (int)blockDim.x, p.nx));
            }
            const int j = w / nch, i = (w - j * nch) * blockDim.x + threadIdx.x;
            if (i < p.nx) fn(i, j, j * p.nx + i);
        }
    } else {
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < p.n; c += gridDim.x * blockDim.x) {
            if (threadIdx.x == 0) {
                const int cn = c + gridDim.x * blockDim.x;
                if (cn < p.n) pf(cn, min(cn + (int)blockDim.x, p.n));
            }
            const int j = c / p.nx;
            fn(c - j * p.nx, j, c);
        }
    }
}

// neighbours of cell c = (i, j) (-1: no neighbour across a transmissive wall)
__device__ __forceinline__ Nb nb_of(const DevParams &p, int i, int j, int c)
{
    Nb r;
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

// Temporally blocked predictor sweeps of Eq. (LIM) for the heat stage.  A
// round of up to HB sweeps loads each tile of the grid with a halo of HB
// cells -- the starting iterate, C0 = T0 + tau V Ia, tau V and Lam -- into
// shared memory, forms the face coefficients Lam_f / h^2 (zero across a
// transmissive wall), sweeps there, and writes the tile's cells of the last
// iterate back.  After j sweeps the cells at least j cells inside the region
// are exact (their inputs were), so the tile's cells (HB inside) are exact
// after HB sweeps.  One grid barrier per round instead of one per sweep; the
// halo is swept redundantly.  Rounds alternate between the two iterate
// planes, so no block overwrites a plane another block may still read in the
// same round.
//
// Two forms:
//  - lim_rounds: thread loads (periodic walls wrap).  2D grids: regions of
//    RX x RY cells swept by a block's 512 threads as 64 x 8; 1D grids: a line
//    of RB cells.
//  - lim_rounds_tma: 2D grids with transmissive walls and rows of a multiple
//    of 4 floats.  Regions of TX x TY = 128 x 34 cells arrive by four 2D bulk
//    tensor copies onto an mbarrier (cells outside the grid as zeros), two
//    region buffers, the next tile's copies issued before the current tile is
//    swept.  A block of 1024 threads: warp w sweeps region row w + 1, each
//    lane 4 adjacent cells with 16-byte shared loads, the x neighbours across
//    lanes by warp shuffles; sweep j updates the rows j .. TY - 1 - j only.
constexpr int HB = 4, RX = 64, RY = 36, RB = RX * RY;
// region planes: iterate, C0, tau V, Lam, the second iterate, the x and y faces
constexpr size_t LIM_SMEM = sizeof(float) * RB * 7;
constexpr int HEAT_THREADS = 512;
static_assert(HEAT_THREADS == RX * 8, "the 2D sweep maps the block as 64 x 8 threads");

constexpr int TX = 128, TY = 34, TB = TX * TY;
constexpr int NPL = 4;  // planes of a TMA region: iterate, C0, tau V, Lam
// two TMA region buffers and the second iterate
constexpr size_t LIM_SMEM_TMA = sizeof(float) * TB * (2 * NPL + 1) + 128;  // + the alignment slack
constexpr int HEAT_THREADS_TMA = 1024;
static_assert(HEAT_THREADS_TMA / 32 == TY - 2 && TX == 32 * 4, "one warp per inner region row, 4 cells per lane");
static_assert((TX - 2 * HB) % 4 == 0 && HB % 4 == 0, "TMA region starts must be multiples of 4 floats");
static_assert((TB * sizeof(float)) % 128 == 0, "region planes keep the 128-byte alignment of TMA destinations");
// clock cycles an mbarrier wait polls before it gives up (~0.25 s at 2 GHz; each
// try_wait may suspend the thread, so the bound is on time, not on polls)
constexpr long long kTmaWaitClocks = 500000000LL;

__device__ __forceinline__ bool lim_rounds(const DevParams &p, const FFP &f, const HeatFF &s, Scalars *sc, int M,
                                           const float *s_tb, const float *s_rd, float *sm, const float *&vlast)
{
    float *sv = sm, *sC = sv + RB, *stV = sC + RB, *sL = stV + RB, *vb = sL + RB, *sLx = vb + RB, *sLy = sLx + RB;
    const bool ax = p.nx > 1, ay = p.ny > 1, two = ax && ay;
    const int wx = two ? RX : (ax ? RB : 1), wy = two ? RY : (ay ? RB : 1);  // region
    const int hx = ax ? HB : 0, hy = ay ? HB : 0;
    const int tx = wx - 2 * hx, ty = wy - 2 * hy;  // tile
    const int ntx = (p.nx + tx - 1) / tx, nty = (p.ny + ty - 1) / ty, ntiles = ntx * nty;
    const int lx = threadIdx.x & (RX - 1), ly = threadIdx.x >> 6;
    const bool per_x = p.bc[0] == DIM_BC_PERIODIC, per_y = p.bc[1] == DIM_BC_PERIODIC;
    const float *vin = s.T0;
    int m0 = 0, r = 0;
    while (m0 < M) {
        const int kk = min(HB, M - m0);
        float *vout = (r & 1) ? s.vb : s.va;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int tj = t / ntx, ti = t - tj * ntx;
            const int gx0 = ti * tx - hx, gy0 = tj * ty - hy;
            auto load = [&](int sx, int sy) {
                const int e = sy * wx + sx;
                int gx = gx0 + sx, gy = gy0 + sy;
                bool in = true;
                if (gx < 0 || gx >= p.nx) {
                    if (per_x) gx = (gx % p.nx + p.nx) % p.nx;
                    else in = false;
                }
                if (gy < 0 || gy >= p.ny) {
                    if (per_y) gy = (gy % p.ny + p.ny) % p.ny;
                    else in = false;
                }
                if (in) {
                    const int c = gy * p.nx + gx;
                    sv[e] = vin[c];
                    sC[e] = s.C0[c];
                    stV[e] = s.tV[c];
                    sL[e] = s.L[c];
                } else {  // outside a transmissive wall: no cell (its faces are zero)
                    sv[e] = sC[e] = stV[e] = sL[e] = 0.f;
                }
            };
            if (two) {
                for (int sy = ly; sy < RY; sy += 8) load(lx, sy);
            } else {
                for (int e = threadIdx.x; e < RB; e += blockDim.x) load(ax ? e : 0, ax ? 0 : e);
            }
            __syncthreads();
            // face coefficients after each cell; zero where either cell lies
            // beyond a transmissive wall
            auto inside_x = [&](int sx) { const int g = gx0 + sx; return per_x || (g >= 0 && g < p.nx); };
            auto inside_y = [&](int sy) { const int g = gy0 + sy; return per_y || (g >= 0 && g < p.ny); };
            auto faces = [&](int sx, int sy) {
                const int e = sy * wx + sx;
                const float Lc = sL[e];
                const bool in = inside_x(sx) && inside_y(sy);
                float fx = 0.f, fy = 0.f;
                if (ax && sx + 1 < wx && in && inside_x(sx + 1)) fx = 0.5f * (Lc + sL[e + 1]) * f.idx2;
                if (ay && sy + 1 < wy && in && inside_y(sy + 1)) fy = 0.5f * (Lc + sL[e + wx]) * f.idy2;
                sLx[e] = fx;
                sLy[e] = fy;
            };
            if (two) {
                for (int sy = ly; sy < RY; sy += 8) faces(lx, sy);
            } else {
                for (int e = threadIdx.x; e < RB; e += blockDim.x) faces(ax ? e : 0, ax ? 0 : e);
            }
            __syncthreads();
            float *a = sv, *b = vb;
            for (int j = 1; j <= kk; j++) {
                const float tb = s_tb[m0 + j - 1], rd = s_rd[m0 + j - 1];
                auto cell = [&](int q) {
                    const float vc = a[q];
                    float lap = 0.f;
                    if (ax) lap += sLx[q] * (a[q + 1] - vc) - sLx[q - 1] * (vc - a[q - 1]);
                    if (ay) lap += sLy[q] * (a[q + wx] - vc) - sLy[q - wx] * (vc - a[q - wx]);
                    b[q] = (sC[q] + tb * vc + stV[q] * lap) * rd;
                };
                if (two) {
                    if (lx >= 1 && lx < RX - 1)
                        for (int sy = 1 + ly; sy < RY - 1; sy += 8) cell(sy * RX + lx);
                } else {
                    for (int e = 1 + threadIdx.x; e < RB - 1; e += blockDim.x) cell(e);
                }
                __syncthreads();
                float *tmp = a;
                a = b;
                b = tmp;
            }
            if (two) {
                const int gx = ti * tx + lx - HB;
                if (lx >= HB && lx < RX - HB && gx < p.nx)
                    for (int sy = HB + ly; sy < RY - HB; sy += 8) {
                        const int gy = tj * ty + sy - HB;
                        if (gy < p.ny) vout[gy * p.nx + gx] = a[sy * RX + lx];
                    }
            } else {
                for (int e = threadIdx.x; e < (ax ? tx : ty); e += blockDim.x) {
                    const int g = (ax ? ti * tx : tj * ty) + e;
                    if (g < (ax ? p.nx : p.ny)) vout[g] = a[e + HB];
                }
            }
            __syncthreads();  // the region buffers are refilled for the block's next tile
        }
        if (!grid_barrier(sc)) return false;
        vin = vout;
        m0 += kk;
        r++;
    }
    vlast = vin;
    return true;
}

__device__ __forceinline__ unsigned smem_u32(const void *q) { return (unsigned)__cvta_generic_to_shared(q); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity to complete
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_test(b, parity))
        if (clock64() - t0 > kTmaWaitClocks) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, unsigned long long *b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(smem_u32(b))
        : "memory");
}

// bulk copy of `bytes` (a multiple of 16) from global src to shared dst, both
// 16-byte aligned, completing on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

// the descriptors of the planes a round reads (addresses in the kernel's
// parameter space)
struct LimMapPtrs {
    const CUtensorMap *va, *vb, *T0, *C0, *tV, *L;
};

__device__ __forceinline__ float4 lds4(const float *q) { return *reinterpret_cast<const float4 *>(q); }
__device__ __forceinline__ void sts4(float *q, float4 v) { *reinterpret_cast<float4 *>(q) = v; }

__device__ __forceinline__ bool lim_rounds_tma(const DevParams &p, const FFP &f, const HeatFF &s, LimMapPtrs tm,
                                               Scalars *sc, int M, const float *s_tb, const float *s_rd, float *sm,
                                               const float *&vlast)
{
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int s_fail;
    constexpr unsigned FULL = 0xffffffffu;
    // region buffers (v, C0, tau V, Lam) at base and base + NPL TB.  Bulk tensor
    // copies write 128-byte aligned shared destinations: base is the first such
    // address of the dynamic array, formed as an element offset so that every
    // region pointer stays derived from the shared array (the accesses compile
    // to shared-memory instructions)
    float *const base = sm + ((128u - (smem_u32(sm) & 127u)) & 127u) / sizeof(float);
    float *const vb = base + 2 * NPL * TB;
    constexpr int tx = TX - 2 * HB, ty = TY - 2 * HB;  // tile
    const int ntx = (p.nx + tx - 1) / tx, nty = (p.ny + ty - 1) / ty, ntiles = ntx * nty;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cx = 4 * lane;  // the lane's first column in the region
    const float idx2 = f.idx2, idy2 = f.idy2;
    unsigned use0 = 0u, use1 = 0u;  // completed loads per buffer (the mbarrier phase parity)
    if (smem_u32(base) & 127u) {  // not expected: flag and leave before any copy
        if (threadIdx.x == 0) atomicOr(&sc->status, DIM_ST_TIMEOUT);
        return false;
    }
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const float *vin = s.T0;
    int m0 = 0, r = 0;
    while (m0 < M) {
        const int kk = min(HB, M - m0);
        float *vout = (r & 1) ? s.vb : s.va;
        const CUtensorMap *vmap = r == 0 ? tm.T0 : ((r & 1) ? tm.va : tm.vb);  // the plane vin is
        auto issue = [&](int t, int buf) {  // one thread: the four bulk copies of tile t
            const int tj = t / ntx, ti = t - tj * ntx;
            const int x0 = ti * tx - HB, y0 = tj * ty - HB;
            float *d = base + buf * NPL * TB;
            unsigned long long *bar = buf ? &s_bar[1] : &s_bar[0];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, (unsigned)(NPL * TB * sizeof(float)));
            tma_load_2d(d, vmap, x0, y0, bar);
            tma_load_2d(d + TB, tm.C0, x0, y0, bar);
            tma_load_2d(d + 2 * TB, tm.tV, x0, y0, bar);
            tma_load_2d(d + 3 * TB, tm.L, x0, y0, bar);
        };
        if (threadIdx.x == 0) {
            // the other blocks' iterate writes (ordered by the grid barrier) before
            // this round's bulk copies read them
            asm volatile("fence.proxy.async.global;" ::: "memory");
            if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        }
        int k = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, k++) {
            const int tj = t / ntx, ti = t - tj * ntx;
            const int gx0 = ti * tx - HB, gy0 = tj * ty - HB;
            const int buf = k & 1;
            float *const sv = base + buf * NPL * TB, *const sC = sv + TB, *const stV = sv + 2 * TB,
                         *const sL = sv + 3 * TB;
            {
                const unsigned ub = buf ? use1 : use0, uo = buf ? use0 : use1;
                if (threadIdx.x == 0) {
                    const int tn = t + gridDim.x;
                    s_fail = 0;
                    if (tn < ntiles) issue(tn, buf ^ 1);  // streams while this tile is swept
                    if (!mbar_wait(buf ? &s_bar[1] : &s_bar[0], ub & 1u)) s_fail = 1;
                }
                __syncthreads();
                if (s_fail) {
                    // give up: flag, let the other buffer's copies land (bounded), leave
                    if (threadIdx.x == 0) {
                        atomicOr(&sc->status, DIM_ST_TIMEOUT);
                        if (t + gridDim.x < ntiles) mbar_wait(buf ? &s_bar[0] : &s_bar[1], uo & 1u);
                    }
                    return false;
                }
                if (buf) use1++;
                else use0++;
            }
            // Warp w owns region row ry = w + 1 for all sweeps of the tile: its face
            // coefficients (x faces after each of its cells, the y faces above and
            // below), C0, tau V and its current iterate stay in registers, so a
            // sweep reads only the rows above and below from shared memory and
            // writes its own row.  Faces are zero where either cell lies beyond a
            // transmissive wall.
            const int ry = w + 1, q = ry * TX + cx;
            float4 Lx, Ly, Lu;  // faces: x (after each cell), y below, y above, times 1/h^2
            {
                const float4 Lc = lds4(sL + q), Ld = lds4(sL + q + TX), La = lds4(sL + q - TX);
                const float Le = __shfl_down_sync(FULL, Lc.x, 1);
                Lx = make_float4(0.5f * (Lc.x + Lc.y) * idx2, 0.5f * (Lc.y + Lc.z) * idx2, 0.5f * (Lc.z + Lc.w) * idx2,
                                 lane < 31 ? 0.5f * (Lc.w + Le) * idx2 : 0.f);
                Ly = make_float4(0.5f * (Lc.x + Ld.x) * idy2, 0.5f * (Lc.y + Ld.y) * idy2, 0.5f * (Lc.z + Ld.z) * idy2,
                                 0.5f * (Lc.w + Ld.w) * idy2);
                Lu = make_float4(0.5f * (La.x + Lc.x) * idy2, 0.5f * (La.y + Lc.y) * idy2, 0.5f * (La.z + Lc.z) * idy2,
                                 0.5f * (La.w + Lc.w) * idy2);
                if (gx0 < 0 || gy0 < 0 || gx0 + TX > p.nx || gy0 + TY > p.ny) {  // a region that crosses a wall
                    const int gy = gy0 + ry, gx = gx0 + cx;
                    auto in_x = [&](int g) { return g >= 0 && g < p.nx; };
                    auto in_y = [&](int g) { return g >= 0 && g < p.ny; };
                    const bool row_in = in_y(gy);
                    if (!(row_in && in_x(gx) && in_x(gx + 1))) Lx.x = 0.f;
                    if (!(row_in && in_x(gx + 1) && in_x(gx + 2))) Lx.y = 0.f;
                    if (!(row_in && in_x(gx + 2) && in_x(gx + 3))) Lx.z = 0.f;
                    if (!(row_in && in_x(gx + 3) && in_x(gx + 4))) Lx.w = 0.f;
                    if (!(row_in && in_y(gy + 1))) Ly = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (!(row_in && in_y(gy - 1))) Lu = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (!in_x(gx)) Ly.x = Lu.x = 0.f;
                    if (!in_x(gx + 1)) Ly.y = Lu.y = 0.f;
                    if (!in_x(gx + 2)) Ly.z = Lu.z = 0.f;
                    if (!in_x(gx + 3)) Ly.w = Lu.w = 0.f;
                }
            }
            // the west face of the lane's first cell (every lane takes part in the
            // shuffle; the region's column 0 is never exact, so lane 0 takes 0)
            const float fwl = __shfl_up_sync(FULL, Lx.w, 1);
            const float fw = lane > 0 ? fwl : 0.f;
            const float4 C = lds4(sC + q), V = lds4(stV + q);
            float *const p0 = sv + q, *const p1 = vb + q;  // the row in the two iterate planes
            float4 c = lds4(p0);
#pragma unroll
            for (int j = 1; j <= HB; j++) {
                if (j <= kk) {  // block-uniform
                    const float *const src = (j & 1) ? p0 : p1;
                    float *const dst = (j & 1) ? p1 : p0;
                    if (ry >= j && ry <= TY - 1 - j) {  // warp-uniform
                        const float tb = s_tb[m0 + j - 1], rd = s_rd[m0 + j - 1];
                        // x neighbours of the lane's first and last cells (lanes 0 and
                        // 31 take any finite value: columns 0 and TX - 1 are never exact)
                        const float aw = __shfl_up_sync(FULL, c.w, 1), ae = __shfl_down_sync(FULL, c.x, 1);
                        float4 l;  // the Laplacian: x faces, the face above, the face below
                        l.x = Lx.x * (c.y - c.x) - fw * (c.x - aw);
                        l.y = Lx.y * (c.z - c.y) - Lx.x * (c.y - c.x);
                        l.z = Lx.z * (c.w - c.z) - Lx.y * (c.z - c.y);
                        l.w = Lx.w * (ae - c.w) - Lx.z * (c.w - c.z);
                        {
                            const float4 u = lds4(src - TX);
                            l.x -= Lu.x * (c.x - u.x);
                            l.y -= Lu.y * (c.y - u.y);
                            l.z -= Lu.z * (c.z - u.z);
                            l.w -= Lu.w * (c.w - u.w);
                        }
                        {
                            const float4 d = lds4(src + TX);
                            l.x += Ly.x * (d.x - c.x);
                            l.y += Ly.y * (d.y - c.y);
                            l.z += Ly.z * (d.z - c.z);
                            l.w += Ly.w * (d.w - c.w);
                        }
                        c.x = (C.x + tb * c.x + V.x * l.x) * rd;
                        c.y = (C.y + tb * c.y + V.y * l.y) * rd;
                        c.z = (C.z + tb * c.z + V.z * l.z) * rd;
                        c.w = (C.w + tb * c.w + V.w * l.w) * rd;
                        if (j < kk) sts4(dst, c);  // the last sweep's rows leave from registers
                    }
                    if (j < kk) __syncthreads();
                }
            }
            // the tile: rows HB .. TY - 1 - HB, columns HB .. TX - 1 - HB (lanes 1..30),
            // updated by every sweep of the round
            if (ry >= HB && ry < TY - HB && lane >= 1 && lane < 31) {
                const int gx = gx0 + cx, gy = gy0 + ry;
                if (gx < p.nx && gy < p.ny) *reinterpret_cast<float4 *>(vout + (size_t)gy * p.nx + gx) = c;
            }
            __syncthreads();  // the region buffers are refilled for the block's next tiles
        }
        if (!grid_barrier(sc)) return false;
        vin = vout;
        m0 += kk;
        r++;
    }
    vlast = vin;
    return true;
}

// temperature relaxation + heat conduction by the local-iteration method
// (Sec. 3.4, Algorithm 1), cooperative: coefficients -> lambda_max -> P, b_m
// -> 2P - 2 predictor sweeps (temporally blocked) -> conservative last sweep
// + projection
// Ud (may be null): the end state is written there as FP64 planes (all 8)
// instead of to the FF planes -- the last step of a call, which then needs no
// separate conversion pass
// TMA: the rounds of lim_rounds_tma (blocks of HEAT_THREADS_TMA threads), else
// those of lim_rounds (HEAT_THREADS)
// CFL: the kernel also forms the next step's CFL maximum and time step (a step
// inside a multi-step call); a separate instantiation, so that the others keep
// their code
template <bool TMA, bool CFL>
__global__ void __launch_bounds__(TMA ? HEAT_THREADS_TMA : HEAT_THREADS)
    k_heatff(const DevParams p, const FFP f, float2 *U, HeatFF s, Scalars *sc, double dt_host, int trelax_first,
             int check, double *Ud, const __grid_constant__ LimMaps tm)
{
    extern __shared__ float smem_lim[];
    __shared__ float s_tb[2 * PMAX], s_rd[2 * PMAX];
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    __shared__ double s_tau;
    if (threadIdx.x == 0) s_tau = dt_host > 0.0 ? dt_host : p.cfl / read_acc(&sc->smax);
    __syncthreads();
    const double tau = s_tau;
    const float tauf = (float)tau;
    const int nout = p.n_outer < 1 ? 1 : (p.n_outer > 8 ? 8 : p.n_outer);
    unsigned st = 0;

    for (int c = t0; c < n; c += nt) {
        if (threadIdx.x == 0 && c + nt < n) {  // the block's next chunk of the planes read here
            const size_t c0 = (size_t)c + nt, c1 = min(c0 + blockDim.x, (size_t)n);
            l2_prefetch(U, c0, c1);
            l2_prefetch(U + n, c0, c1);
            l2_prefetch(U + 4 * (size_t)n, c0, c1);
            l2_prefetch(U + 5 * (size_t)n, c0, c1);
            l2_prefetch(U + 7 * (size_t)n, c0, c1);
        }
        const ff M1 = ld_ff(U, c), M2 = ld_ff(U, n + (size_t)c);
        const float m1 = ff_f(M1), m2 = ff_f(M2);
        ff E1 = ld_ff(U, 4 * (size_t)n + c), E2 = ld_ff(U, 5 * (size_t)n + c), a2 = ld_ff(U, 7 * (size_t)n + c);
        float T;
        if (trelax_first) {
            const unsigned r = ff_equilibrium(f, M1, M2, ff_add(E1, E2), T, a2, E1, E2);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
            st_ff(U, 4 * (size_t)n + c, E1);
            st_ff(U, 5 * (size_t)n + c, E2);
            st_ff(U, 7 * (size_t)n + c, a2);
        } else {
            T = ff_mixture_T(f, m1, m2, E1, E2, a2);
        }
        s.T0[c] = T;
        float V, L;
        ff_heat_coeffs(f, m1, m2, T, a2, V, L);
        s.V[c] = V;
        s.L[c] = L;
        const float a2f = ff_f(a2);
        const float Ia = ff_f(ff_sub(ff_one(), a2)) * f.src[0] + a2f * f.src[1];
        s.Ia[c] = Ia;
        s.tV[c] = tauf * V;
        s.C0[c] = T + tauf * V * Ia;
    }
    float mcfl = 0.f;  // CFL: the next step's CFL maximum over this block's cells
    for (int it = 0; it < nout; it++) {
        if (!grid_barrier(sc)) return;
        float lm = 0.f;
        for_cells(p, [&](int i, int j, int c) { lm = fmaxf(lm, gershf(p, nb_of(p, i, j, c), c, s.V, s.L, f.idx2, f.idy2)); });
        block_max_to_f(&sc->lam[it], lm);
        if (!grid_barrier(sc)) return;
        unsigned capped;
        const int P = block_schedule(p, tau, read_acc(&sc->lam[it]), false, s_tb, s_rd, capped);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicMax(&sc->P[0], P);
            if (capped) st |= capped;
        }
        const float *vin = s.T0;
        if constexpr (TMA) {
            const LimMapPtrs mp{&tm.va, &tm.vb, &tm.T0, &tm.C0, &tm.tV, &tm.L};
            if (!lim_rounds_tma(p, f, s, mp, sc, 2 * P - 2, s_tb, s_rd, smem_lim, vin)) return;
        } else {
            if (!lim_rounds(p, f, s, sc, 2 * P - 2, s_tb, s_rd, smem_lim, vin)) return;
        }
        const bool last = it == nout - 1;
        for_cells(p, [&](int i, int j, int c) {
            const float dq = tauf * (lapf(p, nb_of(p, i, j, c), c, vin, s.L, f.idx2, f.idy2) + s.Ia[c]);
            const ff M1 = ld_ff(U, c), M2 = ld_ff(U, n + (size_t)c);
            const ff E1 = ld_ff(U, 4 * (size_t)n + c), E2 = ld_ff(U, 5 * (size_t)n + c);
            float T;
            ff a2, E1n, E2n;
            const unsigned r = ff_equilibrium(f, M1, M2, ff_add_f(ff_add(E1, E2), dq), T, a2, E1n, E2n);
            if (last) {
                ff q[NQ];
                q[0] = M1;
                q[1] = M2;
                q[2] = q[3] = ff_of(0.f);
                q[4] = E1n;
                q[5] = E2n;
                q[6] = ff_add_f(ld_ff(U, 6 * (size_t)n + c), dq);
                q[7] = a2;
                if (Ud || CFL) {
                    q[2] = ld_ff(U, 2 * (size_t)n + c);
                    q[3] = ld_ff(U, 3 * (size_t)n + c);
                }
                if constexpr (CFL) mcfl = fmaxf(mcfl, ff_wave_speed(p, f, q, st));
                if (Ud) {
#pragma unroll
                    for (int k = 0; k < NQ; k++) Ud[k * (size_t)n + c] = ff_to_d(q[k]);
                } else {
                    st_ff(U, 4 * (size_t)n + c, q[4]);
                    st_ff(U, 5 * (size_t)n + c, q[5]);
                    st_ff(U, 6 * (size_t)n + c, q[6]);
                    st_ff(U, 7 * (size_t)n + c, q[7]);
                }
                if (check) st |= ff_check(f, q) | (r & DIM_ST_NAN);
                else if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            } else {
                if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
                s.Ti[c] = T;
                st_ff(s.Ai, c, a2);
            }
        }, [&](int c0, int c1) {  // the planes of the block's next chunk
            l2_prefetch(U, c0, c1);
            l2_prefetch(U + n, c0, c1);
            l2_prefetch(U + 4 * (size_t)n, c0, c1);
            l2_prefetch(U + 5 * (size_t)n, c0, c1);
            l2_prefetch(U + 6 * (size_t)n, c0, c1);
            if (last && (Ud || CFL)) {
                l2_prefetch(U + 2 * (size_t)n, c0, c1);
                l2_prefetch(U + 3 * (size_t)n, c0, c1);
            }
            l2_prefetch(s.Ia, c0, c1);
            l2_prefetch(vin, c0, c1);
            l2_prefetch(s.L, c0, c1);
        });
        if (CFL && last) {
            // the next step's maximum (Sec. 3.1) from this step's end state; the last
            // block to finish publishes it and dt = cfl / S for the next step (every
            // block read this step's time step at its start)
            block_max_to_f(&sc->smax_next, mcfl);
            __shared__ bool s_last_h;
            if (threadIdx.x == 0) {
                __threadfence();
                s_last_h = atomicAdd(&sc->heat_blocks, 1u) == gridDim.x - 1;
            }
            __syncthreads();
            if (s_last_h && threadIdx.x == 0) {
                __threadfence();
                sc->smax = *(volatile unsigned long long *)&sc->smax_next;
                sc->dt32 = (float)(p.cfl / read_acc(&sc->smax));
                sc->smax_next = 0ull;
                sc->heat_blocks = 0u;
                __threadfence();
            }
        }
        if (!last) {
            if (!grid_barrier(sc)) return;
            for (int c = t0; c < n; c += nt) {
                const float m1 = ff_f(ld_ff(U, c)), m2 = ff_f(ld_ff(U, n + (size_t)c));
                const ff a2 = ld_ff(s.Ai, c);
                float V, L;
                ff_heat_coeffs(f, m1, m2, s.Ti[c], a2, V, L);
                s.V[c] = V;
                s.L[c] = L;
                const float Ia = ff_f(ff_sub(ff_one(), a2)) * f.src[0] + ff_f(a2) * f.src[1];
                s.Ia[c] = Ia;
                s.tV[c] = tauf * V;
                s.C0[c] = s.T0[c] + tauf * V * Ia;
            }
        }
    }
    flag(sc, st);
}

// FP32 scratch of the viscous stage (planes of n floats)
struct ViscFF {
    float *V, *a1, *a2, *u0, *w0, *ua, *ub, *wa, *wb;
};

// viscous step along AXIS (Sec. 3.2), cooperative: lambda_max from the state
// -> P, b_m -> (P > 1: velocities, 1/rho and the volume fractions in scratch
// planes -> 2P - 2 predictor sweeps on u_n with 4/3 mu and u_t with mu) ->
// conservative last sweep with the energy updates (+ pressure relaxation).
// With P = 1 (no predictor sweep, u_hat = u^n) the last sweep reads the state
// directly and no scratch plane is written.  Out of place: the stage reads U
// and writes all 8 planes of Uo (the last sweep reads neighbours' momenta).
// staged conservative sweep of the viscous kernels: chunk of VB cells (the
// block size), window capacity VW cells (the chunk, 2 either side, rounding to
// even bounds), two buffers of NQ planes
constexpr int VB = 256, VW = VB + 8;
constexpr size_t VISC_SMEM = sizeof(float2) * 2 * NQ * VW;

template <int AXIS>
__global__ void __launch_bounds__(256) k_viscff(const DevParams p, const FFP f, const float2 *__restrict__ U,
                                                float2 *__restrict__ Uo, ViscFF s, Scalars *sc, double dt_host,
                                                int relax, int check, int lam_mode)
{
    extern __shared__ float4 smem_visc[];
    __shared__ float s_tb[2 * PMAX], s_rd[2 * PMAX];
    constexpr int QN = AXIS == 0 ? 2 : 3, QT = AXIS == 0 ? 3 : 2;
    constexpr int SLOT = AXIS == 0 ? LAM_VX : LAM_VY;
    const int n = p.n;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    __shared__ double s_tau;
    if (threadIdx.x == 0) s_tau = dt_host > 0.0 ? dt_host : p.cfl / read_acc(&sc->smax);
    __syncthreads();
    const double tau = s_tau;
    const float tauf = (float)tau;
    const float ih2 = AXIS == 0 ? f.idx2 : f.idy2;
    const float ih = AXIS == 0 ? f.idx : f.idy;
    const float mu0 = f.mu[0], mu1 = f.mu[1];
    unsigned st = 0;

    // cell quantities from the float-float state
    auto rho_at = [&](int c) { return ff_f(ld_ff(U, c)) + ff_f(ld_ff(U, n + (size_t)c)); };
    auto alpha_at = [&](int c, float &a1, float &a2) {
        const ff a = ld_ff(U, 7 * (size_t)n + c);
        a2 = ff_f(a);
        a1 = ff_f(ff_sub(ff_one(), a));
    };
    auto mu_at = [&](int c) {
        float a1, a2;
        alpha_at(c, a1, a2);
        return a1 * mu0 + a2 * mu1;
    };
    auto nbs = [&](int c, int &cm, int &cp) {
        const Nb nb = neighbours(p, c);
        cm = AXIS == 0 ? nb.xm : nb.ym;
        cp = AXIS == 0 ? nb.xp : nb.yp;
    };
    // lam_mode 3: sc->vbound holds the minimum density of this state (the step's
    // last sweep).  The mixture viscosity a_1 mu_1 + a_2 mu_2 is at most max(mu_1,
    // mu_2), every face coefficient at most 4/3 of that, so lambda_max of either
    // axis is at most 16/3 max(mu_k) / rho_min max(1/h^2); when twice that still
    // gives P = 1, both solves have P = 1, whose one Chebyshev coefficient is 0
    // whatever lambda_max is: the lambda pass is skipped (the accumulators stay 0,
    // from which P = 1 follows here and in the other axis's kernel).
    bool certified = false;
    if (lam_mode == 3 && sc->vbound != 0u) {
        const double rmin = (double)__uint_as_float(0x7f800000u - sc->vbound);
        const double ih2max = fmax(p.nx > 1 ? (double)f.idx2 : 0.0, p.ny > 1 ? (double)f.idy2 : 0.0);
        const double lb = 2.0 * (16.0 / 3.0) * fmax((double)f.mu[0], (double)f.mu[1]) / rmin * ih2max;
        unsigned cp;
        certified = rmin > 0.0 && isfinite(lb) && cheb_P_visc(p, tau, lb, cp) == 1;
    }
    if (lam_mode != 2 && !certified) {
        // lambda_max of this axis; lam_mode 1 or 3: also that of the other axis,
        // whose solve follows on a state with the same densities and fractions
        constexpr int OSLOT = AXIS == 0 ? LAM_VY : LAM_VX;
        const float ih2o = AXIS == 0 ? f.idy2 : f.idx2;
        float lm = 0.f, lmo = 0.f;
        for (int c = t0; c < n; c += nt) {
            if (threadIdx.x == 0 && c + nt < n) {  // the block's next chunk of m_1, m_2, alpha_2
                const size_t c0 = (size_t)c + nt, c1 = min(c0 + blockDim.x, (size_t)n);
                l2_prefetch(U, c0, c1);
                l2_prefetch(U + n, c0, c1);
                l2_prefetch(U + 7 * (size_t)n, c0, c1);
            }
            const Nb nb = neighbours(p, c);
            const int cm = AXIS == 0 ? nb.xm : nb.ym, cp = AXIS == 0 ? nb.xp : nb.yp;
            const float lc = 4.f / 3.f * mu_at(c);
            const float ir = __fdividef(1.f, rho_at(c));
            const float fl = cm >= 0 ? 0.5f * (4.f / 3.f * mu_at(cm) + lc) : 0.f;
            const float fr = cp >= 0 ? 0.5f * (lc + 4.f / 3.f * mu_at(cp)) : 0.f;
            lm = fmaxf(lm, 2.f * ir * ((fl + fr) * ih2));
            if (lam_mode != 0) {
                const int om = AXIS == 0 ? nb.ym : nb.xm, op = AXIS == 0 ? nb.yp : nb.xp;
                const float gl = om >= 0 ? 0.5f * (4.f / 3.f * mu_at(om) + lc) : 0.f;
                const float gr = op >= 0 ? 0.5f * (lc + 4.f / 3.f * mu_at(op)) : 0.f;
                lmo = fmaxf(lmo, 2.f * ir * ((gl + gr) * ih2o));
            }
        }
        block_max_to_f(&sc->lam[SLOT], lm);
        if (lam_mode != 0) block_max_to_f(&sc->lam[OSLOT], lmo);
        if (!grid_barrier(sc)) return;
    }
    unsigned capped;
    const int P = block_schedule(p, tau, read_acc(&sc->lam[SLOT]), true, s_tb, s_rd, capped);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicMax(&sc->P[1 + AXIS], P);
        if (capped) st |= capped;
    }
    const float *uin = s.u0, *win = s.w0;
    if (P > 1) {
        for (int c = t0; c < n; c += nt) {
            const float rho = rho_at(c);
            s.V[c] = __fdividef(1.f, rho);
            alpha_at(c, s.a1[c], s.a2[c]);
            s.u0[c] = __fdividef(ff_f(ld_ff(U, QN * (size_t)n + c)), rho);
            s.w0[c] = __fdividef(ff_f(ld_ff(U, QT * (size_t)n + c)), rho);
        }
        if (!grid_barrier(sc)) return;
        auto mu_of = [&](int c) { return s.a1[c] * mu0 + s.a2[c] * mu1; };
        for (int m = 1; m <= 2 * P - 2; m++) {
            float *uo = (m & 1) ? s.ua : s.ub;
            float *wo = (m & 1) ? s.wa : s.wb;
            const float tb = s_tb[m - 1], rd = s_rd[m - 1];
            for (int c = t0; c < n; c += nt) {
                int cm, cp;
                nbs(c, cm, cp);
                const float mc = mu_of(c);
                const float mm = cm >= 0 ? 0.5f * (mu_of(cm) + mc) : 0.f;
                const float mp = cp >= 0 ? 0.5f * (mc + mu_of(cp)) : 0.f;
                const float uc = uin[c], wc = win[c];
                const float Lu = (cp >= 0 ? 4.f / 3.f * mp * (uin[cp] - uc) * ih2 : 0.f) -
                                 (cm >= 0 ? 4.f / 3.f * mm * (uc - uin[cm]) * ih2 : 0.f);
                const float Lw =
                    (cp >= 0 ? mp * (win[cp] - wc) * ih2 : 0.f) - (cm >= 0 ? mm * (wc - win[cm]) * ih2 : 0.f);
                uo[c] = (s.u0[c] + tb * uc + tauf * s.V[c] * Lu) * rd;
                wo[c] = (s.w0[c] + tb * wc + tauf * s.V[c] * Lw) * rd;
            }
            if (!grid_barrier(sc)) return;
            uin = uo;
            win = wo;
        }
    }
    // the predicted velocities and volume fractions of a cell: from the planes
    // (P > 1) or the state (P = 1)
    auto cell = [&](int c, float &u, float &w, float &a1, float &a2) {
        if (P > 1) {
            u = uin[c];
            w = win[c];
            a1 = s.a1[c];
            a2 = s.a2[c];
        } else {
            const float rho = rho_at(c);
            u = __fdividef(ff_f(ld_ff(U, QN * (size_t)n + c)), rho);
            w = __fdividef(ff_f(ld_ff(U, QT * (size_t)n + c)), rho);
            alpha_at(c, a1, a2);
        }
    };
    // the conservative last sweep of cell c, whose 8 planes are in q[]; nb(cn,
    // u, w, a1, a2) gives a neighbour's velocities and fractions
    auto last_sweep = [&](int c, ff *q, auto &&nb) {
        int cm, cp;
        nbs(c, cm, cp);
        float uc, wc, a1c, a2c;
        if (P > 1) {
            cell(c, uc, wc, a1c, a2c);
        } else {
            const float rho = ff_f(q[0]) + ff_f(q[1]);
            uc = __fdividef(ff_f(q[QN]), rho);
            wc = __fdividef(ff_f(q[QT]), rho);
            a2c = ff_f(q[7]);
            a1c = ff_f(ff_sub(ff_one(), q[7]));
        }
        const float mc = a1c * mu0 + a2c * mu1;
        float Fn[2], Ft[2], W[2], aF1[2], aF2[2];
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            const int cn = sd == 0 ? cm : cp;
            if (cn < 0) {
                Fn[sd] = Ft[sd] = W[sd] = aF1[sd] = aF2[sd] = 0.f;
                continue;
            }
            float un, wn, a1n, a2n;
            nb(cn, un, wn, a1n, a2n);
            const float lmf = 0.5f * (mc + (a1n * mu0 + a2n * mu1));
            // face between cl and cr: cl = cn, cr = c on the minus side
            const float du = sd == 0 ? uc - un : un - uc, dw = sd == 0 ? wc - wn : wn - wc;
            Fn[sd] = 4.f / 3.f * lmf * du * ih;
            Ft[sd] = lmf * dw * ih;
            W[sd] = 0.5f * (un + uc) * Fn[sd] + 0.5f * (wn + wc) * Ft[sd];
            aF1[sd] = 0.5f * (a1n + a1c);
            aF2[sd] = 0.5f * (a2n + a2c);
        }
        const float ti = tauf * ih;
        q[QN] = ff_add_f(q[QN], ti * (Fn[1] - Fn[0]));
        q[QT] = ff_add_f(q[QT], ti * (Ft[1] - Ft[0]));
        q[6] = ff_add_f(q[6], ti * (W[1] - W[0]));
        q[4] = ff_add_f(q[4], ti * ((aF1[1] * W[1] - aF1[0] * W[0]) -
                                    (uc * (aF1[1] * Fn[1] - aF1[0] * Fn[0]) + wc * (aF1[1] * Ft[1] - aF1[0] * Ft[0]))));
        q[5] = ff_add_f(q[5], ti * ((aF2[1] * W[1] - aF2[0] * W[0]) -
                                    (uc * (aF2[1] * Fn[1] - aF2[0] * Fn[0]) + wc * (aF2[1] * Ft[1] - aF2[0] * Ft[0]))));
        if (relax) {
            const unsigned r = ff_prelax(f, q);
            if (r & (DIM_ST_NONPHYS | DIM_ST_NOROOT)) st |= DIM_ST_TRANSIENT;
            st |= r & DIM_ST_NAN;
        }
        if (check) st |= ff_check(f, q);
#pragma unroll
        for (int k = 0; k < NQ; k++) st_ff(Uo, k * (size_t)n + c, q[k]);
    };
    // P = 1 with an even cell count: the state arrives in shared memory by bulk
    // copies, one chunk of VB cells (with 2 cells either side) per block
    // iteration, two buffers, the next chunk's copies issued before the current
    // one is swept; neighbours outside the window (across rows) are read from
    // global memory.  Otherwise the loop reads the planes directly.
    float2 *const vbuf = reinterpret_cast<float2 *>(smem_visc);
    if (P == 1 && (n & 1) == 0 && (smem_u32(vbuf) & 15u) == 0) {
        __shared__ __align__(8) unsigned long long v_bar[2];
        __shared__ int v_fail;
        const int nch = (n + VB - 1) / VB;
        auto window = [&](int ch, int &w0, int &w1) {  // even bounds: 16-byte aligned copies
            const int c0 = ch * VB;
            w0 = max(c0 - 2, 0) & ~1;
            w1 = min(c0 + VB + 2, n);
            w1 = (w1 + 1) & ~1;  // <= n (n even)
        };
        auto issue = [&](int ch, int buf) {  // one thread
            int w0, w1;
            window(ch, w0, w1);
            const unsigned bytes = (unsigned)(w1 - w0) * (unsigned)sizeof(float2);
            unsigned long long *bar = buf ? &v_bar[1] : &v_bar[0];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, NQ * bytes);
#pragma unroll
            for (int k = 0; k < NQ; k++)
                bulk_load(vbuf + (buf * NQ + k) * VW, U + k * (size_t)n + w0, bytes, bar);
        };
        if (threadIdx.x == 0) {
            mbar_init(&v_bar[0], 1);
            mbar_init(&v_bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if ((int)blockIdx.x < nch) issue(blockIdx.x, 0);
        }
        __syncthreads();
        unsigned use0 = 0u, use1 = 0u;
        int k = 0;
        for (int ch = blockIdx.x; ch < nch; ch += gridDim.x, k++) {
            const int buf = k & 1;
            const unsigned ub = buf ? use1 : use0, uo = buf ? use0 : use1;
            if (threadIdx.x == 0) {
                v_fail = 0;
                if (ch + (int)gridDim.x < nch) issue(ch + gridDim.x, buf ^ 1);
                if (!mbar_wait(buf ? &v_bar[1] : &v_bar[0], ub & 1u)) v_fail = 1;
            }
            __syncthreads();
            if (v_fail) {  // give up: flag, let the other buffer's copies land (bounded), leave
                if (threadIdx.x == 0) {
                    atomicOr(&sc->status, DIM_ST_TIMEOUT);
                    if (ch + (int)gridDim.x < nch) mbar_wait(buf ? &v_bar[0] : &v_bar[1], uo & 1u);
                }
                return;
            }
            if (buf) use1++;
            else use0++;
            int w0, w1;
            window(ch, w0, w1);
            const float2 *const sb = vbuf + buf * NQ * VW;
            const int c = ch * VB + threadIdx.x;
            if (c < n) {
                ff q[NQ];
#pragma unroll
                for (int kq = 0; kq < NQ; kq++) {
                    const float2 v = sb[kq * VW + (c - w0)];
                    q[kq] = ff{v.x, v.y};
                }
                last_sweep(c, q, [&](int cn, float &u, float &w, float &a1, float &a2) {
                    if (cn >= w0 && cn < w1) {  // the same arithmetic as cell()
                        const float2 *e = sb + (cn - w0);
                        const float rho = ff_f(ff{e[0].x, e[0].y}) + ff_f(ff{e[VW].x, e[VW].y});
                        u = __fdividef(ff_f(ff{e[QN * VW].x, e[QN * VW].y}), rho);
                        w = __fdividef(ff_f(ff{e[QT * VW].x, e[QT * VW].y}), rho);
                        const ff a{e[7 * VW].x, e[7 * VW].y};
                        a2 = ff_f(a);
                        a1 = ff_f(ff_sub(ff_one(), a));
                    } else {
                        cell(cn, u, w, a1, a2);
                    }
                });
            }
            __syncthreads();  // the buffer is refilled for the block's chunk after next
        }
    } else {
        for (int c = t0; c < n; c += nt) {
            if (threadIdx.x == 0 && c + nt < n) {  // the block's next chunk of the state
                const size_t c0 = (size_t)c + nt, c1 = min(c0 + blockDim.x, (size_t)n);
#pragma unroll
                for (int k = 0; k < NQ; k++) l2_prefetch(U + k * (size_t)n, c0, c1);
            }
            // the cell's state first (one round trip), its velocities and fractions from it
            ff q[NQ];
#pragma unroll
            for (int k = 0; k < NQ; k++) q[k] = ld_ff(U, k * (size_t)n + c);
            last_sweep(c, q, cell);
        }
    }
    flag(sc, st);
}

// ---------------------------------------------------------------------------
// host side: constants, set-up, launchers
// ---------------------------------------------------------------------------
// sweep tiles: TN cells along the sweep, TL lines; a block has (TN + 4) TL
// threads, one per staged cell (128 along x, 256 along y)
constexpr int SXF_TN = 124, SXF_TL = 1;
constexpr int SYF_TN = 28, SYF_TL = 8;

static int g_heatff_blocks[2] = {0, 0}, g_viscff_blocks[2] = {0, 0};

static ff host_split(double x)
{
    const float h = (float)x;
    return ff{h, (float)(x - (double)h)};
}

FFP ffp_of(const DevParams &p)
{
    FFP f;
    memset(&f, 0, sizeof(f));
    for (int k = 0; k < 2; k++) {
        f.g[k] = (float)p.g[k];
        f.gm1[k] = (float)p.gm1[k];
        f.igm1[k] = (float)p.inv_gm1[k];
        f.pinf[k] = (float)p.pinf[k];
        f.gpinf[k] = (float)p.gpinf[k];
        f.cv[k] = (float)p.cv[k];
        f.mu[k] = (float)p.mu[k];
        f.k0[k] = (float)p.k0[k];
        f.src[k] = (float)p.src[k];
        f.cold[k] = host_split(p.gpinf[k] * p.inv_gm1[k]);
        f.pinf_ff[k] = host_split(p.pinf[k]);
        f.g_ff[k] = host_split(p.g[k]);
        f.gm1_ff[k] = host_split(p.gm1[k]);
        f.cv_ff[k] = host_split(p.cv[k]);
        f.gcv_ff[k] = host_split(p.gm1[k] * p.cv[k]);
    }
    f.B1_ff = host_split(p.pinf[0] - p.pinf[1]);
    f.dcold = host_split(p.gpinf[0] * p.inv_gm1[0] - p.gpinf[1] * p.inv_gm1[1]);
    f.B1 = (float)(p.pinf[0] - p.pinf[1]);
    f.cfl = (float)p.cfl;
    f.idx = (float)p.idx;
    f.idy = (float)p.idy;
    f.idx2 = (float)p.idx2;
    f.idy2 = (float)p.idy2;
    f.inv_Tref = (float)p.inv_Tref;
    f.k_exp = (float)p.k_exp;
    f.k_pow = p.k_pow;
    return f;
}

// the sweep kernels' shared-memory limit (once per device)
cudaError_t sweepff_setup()
{
    const int smx = (int)sweepff_smem(SXF_TN, SXF_TL), smy = (int)sweepff_smem(SYF_TN, SYF_TL);
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_sweepff<0, SXF_TN, SXF_TL, false>, at, smx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweepff<0, SXF_TN, SXF_TL, true>, at, smx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweepff<1, SYF_TN, SYF_TL, false>, at, smy);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweepff<1, SYF_TN, SYF_TL, true>, at, smy);
    return e;
}

// co-resident blocks of a heat kernel: the smaller of its two CFL instantiations
template <bool TMA>
static cudaError_t heat_blocks_per_sm(int *b)
{
    const int threads = TMA ? HEAT_THREADS_TMA : HEAT_THREADS;
    const size_t smem = TMA ? LIM_SMEM_TMA : LIM_SMEM;
    int b0 = 0, b1 = 0;
    cudaError_t e = cudaFuncSetAttribute(k_heatff<TMA, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_heatff<TMA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_heatff<TMA, false>, threads, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_heatff<TMA, true>, threads, smem);
    *b = b0 < b1 ? b0 : b1;
    return e;
}

cudaError_t bulkff_setup(int nsm)
{
    cudaError_t e = sweepff_setup();
    if (e != cudaSuccess) return e;
    int b = 0;
    e = heat_blocks_per_sm<false>(&b);
    if (e != cudaSuccess) return e;
    g_heatff_blocks[0] = b * nsm;
    e = heat_blocks_per_sm<true>(&b);
    if (e != cudaSuccess) return e;
    g_heatff_blocks[1] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_viscff<0>, 256, VISC_SMEM);
    if (e != cudaSuccess) return e;
    g_viscff_blocks[0] = b * nsm;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_viscff<1>, 256, VISC_SMEM);
    if (e != cudaSuccess) return e;
    g_viscff_blocks[1] = b * nsm;
    return cudaSuccess;
}

static int elementwise_grid(size_t m)
{
    size_t g = (m + 255) / 256;
    return g < 152 * 16 ? (int)g : 152 * 16;
}

cudaError_t launch_ff_in(const double *U, float2 *F, size_t m, cudaStream_t s)
{
    k_ff_in<<<elementwise_grid(m), 256, 0, s>>>(U, F, m);
    return cudaGetLastError();
}

cudaError_t launch_ff_out(const float2 *F, double *U, size_t m, cudaStream_t s)
{
    k_ff_out<<<elementwise_grid(m), 256, 0, s>>>(F, U, m);
    return cudaGetLastError();
}

cudaError_t launch_wave_ff(const DevParams &p, const FFP &f, const float2 *U, Scalars *sc, cudaStream_t s)
{
    k_wave_ff<false><<<elementwise_grid((size_t)p.n), 256, 0, s>>>(p, f, (float2 *)U, nullptr, sc);
    return cudaGetLastError();
}

// the CFL kernel that also converts the caller's FP64 state Ud into the FF planes U
cudaError_t launch_wave_ff_in(const DevParams &p, const FFP &f, const double *Ud, float2 *U, Scalars *sc,
                              cudaStream_t s)
{
    k_wave_ff<true><<<elementwise_grid((size_t)p.n), 256, 0, s>>>(p, f, U, Ud, sc);
    return cudaGetLastError();
}

cudaError_t launch_sweep_ff_bound(const DevParams &p, const FFP &f, int axis, const float2 *Uin, float2 *Uout,
                                  double dt_host, Scalars *sc, int relax, int check, int bound, cudaStream_t s)
{
    const size_t smx = sweepff_smem(SXF_TN, SXF_TL), smy = sweepff_smem(SYF_TN, SYF_TL);
    if (axis == 0) {
        dim3 grid((p.nx + SXF_TN - 1) / SXF_TN, (p.ny + SXF_TL - 1) / SXF_TL);
        if (bound)
            k_sweepff<0, SXF_TN, SXF_TL, true><<<grid, (SXF_TN + 4) * SXF_TL, smx, s>>>(p, f, Uin, Uout, dt_host, sc,
                                                                                      relax, check);
        else
            k_sweepff<0, SXF_TN, SXF_TL, false><<<grid, (SXF_TN + 4) * SXF_TL, smx, s>>>(p, f, Uin, Uout, dt_host,
                                                                                       sc, relax, check);
    } else {
        dim3 grid((p.ny + SYF_TN - 1) / SYF_TN, (p.nx + SYF_TL - 1) / SYF_TL);
        if (bound)
            k_sweepff<1, SYF_TN, SYF_TL, true><<<grid, (SYF_TN + 4) * SYF_TL, smy, s>>>(p, f, Uin, Uout, dt_host, sc,
                                                                                      relax, check);
        else
            k_sweepff<1, SYF_TN, SYF_TL, false><<<grid, (SYF_TN + 4) * SYF_TL, smy, s>>>(p, f, Uin, Uout, dt_host,
                                                                                       sc, relax, check);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_ff(const DevParams &p, const FFP &f, int axis, const float2 *Uin, float2 *Uout,
                            double dt_host, Scalars *sc, int relax, int check, cudaStream_t s)
{
    return launch_sweep_ff_bound(p, f, axis, Uin, Uout, dt_host, sc, relax, check, 0, s);
}

cudaError_t launch_relax_ff(const DevParams &p, const FFP &f, float2 *U, Scalars *sc, int which, int check,
                            cudaStream_t s)
{
    k_relaxff<<<elementwise_grid((size_t)p.n), 256, 0, s>>>(p, f, U, sc, which, check);
    return cudaGetLastError();
}

static int coop_grid(int maxb, int n)
{
    const int need = (n + 255) / 256;
    return need < maxb ? need : maxb;
}

// the heat stage's FP32 planes alias the context's FP64 scratch planes S (two
// floats per double): T0, V, Lam, the two iterates, T_it, Ia, -, alpha_it (a
// float pair), C0, tau V
static HeatFF heat_planes(const DevParams &p, double *S)
{
    const size_t n = (size_t)p.n;
    float *F = (float *)S;
    return HeatFF{F,         F + n,     F + 2 * n, F + 3 * n, F + 4 * n, F + 5 * n,
                  F + 6 * n, (float2 *)(F + 8 * n), F + 10 * n, F + 11 * n};
}

// TMA descriptors of the heat planes when the grid allows them: 2D, both walls
// transmissive (a region beyond a wall arrives as zeros), rows of a multiple
// of 4 floats (16-byte strides; the regions start at multiples of 4 floats).
// Returns 1 with the maps filled, 0 when the threads load the regions instead.
int heat_tma_setup(const DevParams &p, double *S, LimMaps *m)
{
    if (p.nx < 2 || p.ny < 2 || p.bc[0] != DIM_BC_TRANSMISSIVE || p.bc[1] != DIM_BC_TRANSMISSIVE || p.nx % 4 != 0)
        return 0;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return 0;
    auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    const HeatFF h = heat_planes(p, S);
    const cuuint64_t dim[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny};
    const cuuint64_t stride[1] = {(cuuint64_t)p.nx * sizeof(float)};
    const cuuint32_t box[2] = {TX, TY}, estr[2] = {1, 1};
    float *planes[6] = {h.va, h.vb, h.T0, h.C0, h.tV, h.L};
    CUtensorMap *maps[6] = {&m->va, &m->vb, &m->T0, &m->C0, &m->tV, &m->L};
    for (int i = 0; i < 6; i++)
        if (encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, planes[i], dim, stride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return 0;
    return 1;
}

cudaError_t launch_heat_ff(const DevParams &p, const FFP &f, float2 *U, double *S, Scalars *sc, double dt_host,
                           int trelax_first, int check, cudaStream_t st, double *Ud, const LimMaps *tm, int use_tma,
                           int cfl_next)
{
    HeatFF hs = heat_planes(p, S);
    DevParams pp = p;
    FFP ff_ = f;
    LimMaps maps;
    if (use_tma) maps = *tm;
    else memset(&maps, 0, sizeof(maps));
    void *args[] = {(void *)&pp,      (void *)&ff_,          (void *)&U,     (void *)&hs, (void *)&sc,
                    (void *)&dt_host, (void *)&trelax_first, (void *)&check, (void *)&Ud, (void *)&maps};
    const int threads = use_tma ? HEAT_THREADS_TMA : HEAT_THREADS, maxb = g_heatff_blocks[use_tma ? 1 : 0];
    const int need = (p.n + threads - 1) / threads;
    // the grid fits both CFL instantiations (the smaller occupancy of the two)
    const void *fn = use_tma ? (cfl_next ? (const void *)k_heatff<true, true> : (const void *)k_heatff<true, false>)
                             : (cfl_next ? (const void *)k_heatff<false, true> : (const void *)k_heatff<false, false>);
    return cudaLaunchCooperativeKernel(fn,
                                       dim3(need < maxb ? need : maxb), dim3(threads), args,
                                       use_tma ? LIM_SMEM_TMA : LIM_SMEM, st);
}

cudaError_t launch_visc_ff(const DevParams &p, const FFP &f, int axis, const float2 *U, float2 *Uo, double *S,
                           Scalars *sc, double dt_host, int relax, int check, int lam_mode, cudaStream_t st)
{
    const size_t n = (size_t)p.n;
    float *F = (float *)S;
    ViscFF vs{F, F + n, F + 2 * n, F + 3 * n, F + 4 * n, F + 5 * n, F + 6 * n, F + 7 * n, F + 8 * n};
    DevParams pp = p;
    FFP ff_ = f;
    void *args[] = {(void *)&pp,      (void *)&ff_,   (void *)&U,     (void *)&Uo,      (void *)&vs,
                    (void *)&sc,      (void *)&dt_host, (void *)&relax, (void *)&check, (void *)&lam_mode};
    const void *fn = axis == 0 ? (const void *)k_viscff<0> : (const void *)k_viscff<1>;
    return cudaLaunchCooperativeKernel(fn, dim3(coop_grid(g_viscff_blocks[axis], p.n)), dim3(256), args, VISC_SMEM,
                                       st);
}

}  // namespace dimk

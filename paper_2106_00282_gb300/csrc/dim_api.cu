// dim_api.cu -- host side of the C ABI declared in include/dim.h.
//
// Owns the context (parameters, grid, stream, scratch planes, device scalars)
// and sequences the stage kernels of one split step (Sec. 3): CFL reduction,
// x sweep, y sweep (each with the pressure relaxation fused in its epilogue),
// viscous steps, temperature relaxation fused into the heat-conduction
// launch.  Every call is stream-ordered on the context stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include "dim_ctx.h"

using namespace dimctx;

static const char *const kKernelNames[K_NKERNELS] = {"sweep_x", "sweep_y", "heat",  "viscous_x", "viscous_y",
                                                     "wave_max", "relax",   "copy", "convert"};

static bool g_setup_done[64];


static bool viscous_on(const dim_params &h) { return h.mu[0] > 0.0 || h.mu[1] > 0.0; }
static bool heat_on(const dim_params &h)
{
    return h.trelax != DIM_TRELAX_OFF &&
           (h.k0[0] > 0.0 || h.k0[1] > 0.0 || h.src[0] > 0.0 || h.src[1] > 0.0);
}

static cudaError_t prof_begin(dim_ctx *c, int kid, int *slot)
{
    *slot = -1;
    if (!c->prof) return cudaSuccess;
    if (c->nrec == c->caprec) {
        int nc = c->caprec ? 2 * c->caprec : 256;
        ProfRec *r = (ProfRec *)realloc(c->recs, sizeof(ProfRec) * nc);
        if (!r) return cudaErrorMemoryAllocation;
        for (int i = c->caprec; i < nc; i++) {
            r[i].a = r[i].b = nullptr;
        }
        c->recs = r;
        c->caprec = nc;
    }
    ProfRec &r = c->recs[c->nrec];
    if (!r.a) {
        cudaError_t e = cudaEventCreate(&r.a);
        if (e != cudaSuccess) return e;
        e = cudaEventCreate(&r.b);
        if (e != cudaSuccess) return e;
    }
    r.kid = kid;
    *slot = c->nrec++;
    return cudaEventRecord(r.a, c->stream);
}

static cudaError_t prof_end(dim_ctx *c, int slot)
{
    if (slot < 0) return cudaSuccess;
    return cudaEventRecord(c->recs[slot].b, c->stream);
}

static cudaError_t reset_accumulators(dim_ctx *c)
{
    return cudaMemsetAsync(c->sc, 0, offsetof(Scalars, status), c->stream);
}

static dimk::HeatScratch heat_scratch(dim_ctx *c)
{
    size_t n = (size_t)c->p.n;
    double *S = c->S;
    return dimk::HeatScratch{S,         S + n,     S + 2 * n, S + 3 * n,  S + 4 * n,  S + 5 * n,
                             S + 6 * n, S + 7 * n, nullptr,   S + 8 * n,  S + 9 * n,  S + 10 * n,
                             S + 11 * n};
}

static dimk::ViscScratch visc_scratch(dim_ctx *c)
{
    size_t n = (size_t)c->p.n;
    double *S = c->S;
    return dimk::ViscScratch{S,         S + n,     S + 2 * n, S + 3 * n, S + 4 * n,  S + 5 * n,
                             S + 6 * n, S + 7 * n, nullptr,   S + 8 * n, S + 9 * n, S + 10 * n,
                             S + (10 + dimk::VF_N) * n};
}

static bool fp32(const dim_ctx *c) { return c->p.precision == DIM_PRECISION_FP32_BULK; }

// FP64 stage launchers
static cudaError_t run_sweep(dim_ctx *c, int axis, const double *Uin, double *Uout, double dt, int relax, int check)
{
    return dimk::launch_sweep(c->p, axis, Uin, Uout, dt, c->sc, relax, check, c->stream);
}
static cudaError_t run_wave(dim_ctx *c, const double *U) { return dimk::launch_wave_max(c->p, U, c->sc, c->stream); }
static cudaError_t run_heat(dim_ctx *c, double *U, double dt, int trelax_first, int check)
{
    return dimk::launch_heat(c->p, U, heat_scratch(c), c->sc, dt, trelax_first, check, c->stream);
}
static cudaError_t run_visc(dim_ctx *c, int axis, double *U, double dt, int relax, int check)
{
    return dimk::launch_visc(c->p, axis, U, visc_scratch(c), c->sc, dt, relax, check, c->stream);
}

// FP32 bulk: the second float-float buffer of the sweeps (the context's U2)
static float2 *ff_other(dim_ctx *c) { return (float2 *)c->U2; }
static size_t state_len(const dim_ctx *c) { return 8 * (size_t)c->p.n; }

#define TIMED(c, kid, launch)                      \
    do {                                           \
        int slot_;                                 \
        TRY(prof_begin((c), (kid), &slot_));       \
        TRY(launch);                               \
        TRY(prof_end((c), slot_));                 \
    } while (0)

extern "C" {

const char *dim_strerror(int code)
{
    switch (code) {
    case DIM_OK: return "ok";
    case DIM_EINVAL: return "invalid argument";
    case DIM_ECUDA: return "CUDA error";
    case DIM_ENONPHYS: return "non-physical state (alpha, density or pressure out of range, or NaN)";
    case DIM_ENOROOT: return "relaxation quadratic without real root";
    case DIM_ETIMEOUT: return "grid barrier wait timed out";
    case DIM_ENOTIMPL: return "not implemented";
    case DIM_ETOOLARGE: return "grid larger than the fixed scratch of the no-allocation entry point";
    default: return "unknown error";
    }
}

}  // extern "C"

// Validate a parameter set and a grid and fill the kernels' parameter block.
// No CUDA call, no allocation.  Shared by dim_init and the no-allocation entry
// point.
int dim_host_params(const dim_params *hp, int nx, int ny, double dx, double dy, DevParams *out)
{
    if (!hp || !out) return DIM_EINVAL;
    if (nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 27) || !(dx > 0.0) || !(dy > 0.0)) return DIM_EINVAL;
    if (nx == 1 && ny == 1) return DIM_EINVAL; /* no active axis: no CFL time scale */
    for (int k = 0; k < 2; k++) {
        if (!(hp->gamma[k] > 1.0) || !(hp->cv[k] > 0.0) || !(hp->pinf[k] >= 0.0) || !(hp->k0[k] >= 0.0) ||
            !(hp->mu[k] >= 0.0))
            return DIM_EINVAL;
        if (hp->bc[k] != DIM_BC_TRANSMISSIVE && hp->bc[k] != DIM_BC_PERIODIC) return DIM_EINVAL;
    }
    if (!(hp->cfl > 0.0) || !(hp->T_ref > 0.0)) return DIM_EINVAL;
    if (hp->limiter != DIM_LIMITER_NONE && hp->limiter != DIM_LIMITER_MINMOD && hp->limiter != DIM_LIMITER_OVERBEE)
        return DIM_EINVAL;
    if (!(hp->src[0] >= 0.0) || !(hp->src[1] >= 0.0)) return DIM_EINVAL;
    if (hp->trelax != DIM_TRELAX_OFF && hp->trelax != DIM_TRELAX_EQUILIBRIUM && hp->trelax != DIM_TRELAX_MIDPOINT)
        return DIM_EINVAL;
    if (hp->trelax == DIM_TRELAX_MIDPOINT && (hp->trelax_iters < 1 || hp->trelax_iters > 1000)) return DIM_EINVAL;
    if (hp->heat_alpha != DIM_HEAT_ALPHA_PROJECTION && hp->heat_alpha != DIM_HEAT_ALPHA_LINEAR) return DIM_EINVAL;
    // the paper's variants are FP64 kernels only
    if ((hp->trelax == DIM_TRELAX_MIDPOINT || hp->heat_alpha == DIM_HEAT_ALPHA_LINEAR) &&
        hp->precision != DIM_PRECISION_FP64)
        return DIM_EINVAL;
    if (hp->n_outer < 1 || hp->n_outer > 8) return DIM_EINVAL;
    if (hp->p_policy < DIM_P_FORMULA || hp->p_policy > DIM_P_CLAMP) return DIM_EINVAL;
    if (hp->p_max < 1 || hp->p_max > dimk::PMAX) return DIM_EINVAL;
    if (hp->p_policy == DIM_P_FIXED && (hp->p_fixed < 1 || hp->p_fixed > dimk::PMAX)) return DIM_EINVAL;
    if (hp->p_policy == DIM_P_CLAMP && (hp->p_min < 1 || hp->p_min > hp->p_max)) return DIM_EINVAL;
    if (hp->precision != DIM_PRECISION_FP64 && hp->precision != DIM_PRECISION_FP32_BULK) return DIM_EINVAL;
    DevParams p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < 2; k++) {
        p.g[k] = hp->gamma[k];
        p.pinf[k] = hp->pinf[k];
        p.cv[k] = hp->cv[k];
        p.gm1[k] = hp->gamma[k] - 1.0;
        p.inv_gm1[k] = 1.0 / (hp->gamma[k] - 1.0);
        p.gpinf[k] = hp->gamma[k] * hp->pinf[k];
        p.k0[k] = hp->k0[k];
        p.mu[k] = hp->mu[k];
        p.bc[k] = hp->bc[k];
        p.src[k] = hp->src[k];
    }
    p.k_exp = hp->k_exp;
    p.T_ref = hp->T_ref;
    p.inv_Tref = 1.0 / hp->T_ref;
    {
        double e = hp->k_exp;
        p.k_pow = e == 0.0 ? 0 : ((e == floor(e) && e > 0.0 && e <= 8.0) ? (int)e : -1);
    }
    p.cfl = hp->cfl;
    p.dx = dx;
    p.dy = dy;
    p.idx = 1.0 / dx;
    p.idy = 1.0 / dy;
    p.idx2 = 1.0 / (dx * dx);
    p.idy2 = 1.0 / (dy * dy);
    p.nx = nx;
    p.ny = ny;
    p.n = nx * ny;
    p.limiter = hp->limiter;
    p.trelax = hp->trelax;
    p.trelax_iters = hp->trelax == DIM_TRELAX_MIDPOINT ? hp->trelax_iters : 0;
    p.heat_alpha = hp->heat_alpha;
    p.n_outer = hp->n_outer;
    p.p_policy = hp->p_policy;
    p.p_fixed = hp->p_fixed;
    p.p_min = hp->p_min;
    p.p_max = hp->p_max;
    p.precision = hp->precision;
    p.beta = nullptr;
    *out = p;
    return DIM_OK;
}

extern "C" {

int dim_init(dim_ctx **out, const dim_params *hp, int nx, int ny, double dx, double dy, void *cuda_stream)
{
    if (!out || !hp) return DIM_EINVAL;
    *out = nullptr;
    DevParams pv;
    int r = dim_host_params(hp, nx, ny, dx, dy, &pv);
    if (r != DIM_OK) return r;
    dim_ctx *c = (dim_ctx *)calloc(1, sizeof(dim_ctx));
    if (!c) return DIM_ECUDA;
    c->hp = *hp;
    DevParams &p = c->p;
    p = pv;
    c->stream = (cudaStream_t)cuda_stream;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { free(c); return DIM_ECUDA; }
    c->device = dev;
    if (dev < 64 && !g_setup_done[dev]) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            dimk::sweep_setup() != cudaSuccess || dimk::parabolic_setup(nsm) != cudaSuccess ||
            dimk::bulkff_setup(nsm) != cudaSuccess) {
            free(c);
            return DIM_ECUDA;
        }
        g_setup_done[dev] = true;
    }
    size_t plane = sizeof(double) * (size_t)p.n;
    if (cudaMalloc(&c->U2, 8 * plane) != cudaSuccess || cudaMalloc(&c->S, dimk::SCRATCH_PLANES * plane) != cudaSuccess ||
        cudaMalloc(&c->sc, sizeof(Scalars)) != cudaSuccess || cudaMemset(c->sc, 0, sizeof(Scalars)) != cudaSuccess ||
        cudaMalloc(&c->beta, sizeof(double) * dimk::PMAX * dimk::PMAX) != cudaSuccess ||
        (p.precision == DIM_PRECISION_FP32_BULK && cudaMalloc(&c->Uf, 8 * plane) != cudaSuccess)) {
        dim_destroy(c);
        return DIM_ECUDA;
    }
    c->ffp = dimk::ffp_of(p);
    c->lim_tma = p.precision == DIM_PRECISION_FP32_BULK ? dimk::heat_tma_setup(p, c->S, &c->lim) : 0;
    {
        // roots of the Chebyshev polynomials T_P, P = 1..PMAX, in decreasing order
        const double pi = 3.14159265358979323846;
        double *tab = (double *)calloc((size_t)dimk::PMAX * dimk::PMAX, sizeof(double));
        if (!tab) { dim_destroy(c); return DIM_ECUDA; }
        for (int P = 1; P <= dimk::PMAX; P++)
            for (int m = 1; m <= P; m++) tab[(P - 1) * dimk::PMAX + (m - 1)] = cos((2.0 * m - 1.0) * pi / (2.0 * P));
        cudaError_t e = cudaMemcpy(c->beta, tab, sizeof(double) * dimk::PMAX * dimk::PMAX, cudaMemcpyHostToDevice);
        free(tab);
        if (e != cudaSuccess) { dim_destroy(c); return DIM_ECUDA; }
        p.beta = c->beta;
    }
    *out = c;
    return DIM_OK;
}

void dim_destroy(dim_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    grad_free(c);
    cudaFree(c->U2);
    cudaFree(c->Uf);
    cudaFree(c->S);
    cudaFree(c->Uh);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
        cudaEventDestroy(c->ev_mass);
        cudaEventDestroy(c->ev_mom);
    }
    cudaFree(c->sc);
    cudaFree(c->beta);
    for (int i = 0; i < c->caprec; i++) {
        if (c->recs[i].a) cudaEventDestroy(c->recs[i].a);
        if (c->recs[i].b) cudaEventDestroy(c->recs[i].b);
    }
    free(c->recs);
    free(c);
}

int dim_from_primitive(dim_ctx *c, const double *prim, double *U)
{
    if (!c || !prim || !U) return DIM_EINVAL;
    TRY(dimk::launch_from_primitive(c->p, prim, U, c->sc, c->stream));
    return DIM_OK;
}

int dim_cfl_dt(dim_ctx *c, const double *U, double *dt)
{
    if (!c || !U || !dt) return DIM_EINVAL;
    TRY(reset_accumulators(c));
    if (fp32(c)) {
        TIMED(c, K_CONVERT, dimk::launch_ff_in(U, c->Uf, state_len(c), c->stream));
        TIMED(c, K_WAVE, dimk::launch_wave_ff(c->p, c->ffp, c->Uf, c->sc, c->stream));
    } else {
        TIMED(c, K_WAVE, run_wave(c, U));
    }
    unsigned long long bits = 0;
    TRY(cudaMemcpyAsync(&bits, &c->sc->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    double smax;
    memcpy(&smax, &bits, sizeof(smax));
    *dt = c->p.cfl / smax;
    return DIM_OK;
}

static int status_to_code(unsigned st)
{
    if (st & DIM_ST_TIMEOUT) return DIM_ETIMEOUT;
    if (st & (DIM_ST_NONPHYS | DIM_ST_NAN)) return DIM_ENONPHYS;
    if (st & DIM_ST_NOROOT) return DIM_ENOROOT;
    return DIM_OK;
}

// Where the planes of the state are final within a step: the masses m1, m2
// (planes 0, 1) after the last sweep, the momenta (planes 2, 3) after the last
// viscous stage (else the last sweep); the later stages write planes 4-7 only.
struct StepMarks {
    double *mass_buf, *mom_buf;  // the buffer holding the final planes at that point
};

// one split step on U (device); stages in the order of Sec. 3.  mk (may be
// null): record c->ev_mass and c->ev_mom on the stream at the points above
static int step_once(dim_ctx *c, double *U, StepMarks *mk = nullptr)
{
    const dim_params &h = c->hp;
    const DevParams &p = c->p;
    const bool vis = viscous_on(h), heat = heat_on(h), trx = h.trelax != DIM_TRELAX_OFF;
    const bool sx = p.nx > 1, sy = p.ny > 1;
    // the kernel that ends the step also checks the end-of-step state
    enum { LAST_SX, LAST_SY, LAST_VX, LAST_VY, LAST_TR, LAST_HEAT } last;
    if (heat) last = LAST_HEAT;
    else if (trx) last = LAST_TR;
    else if (vis) last = sy ? LAST_VY : LAST_VX;
    else last = sy ? LAST_SY : LAST_SX;

    TRY(reset_accumulators(c));
    TIMED(c, K_WAVE, run_wave(c, U));
    double *cur = U, *oth = c->U2;
    if (sx) {
        TIMED(c, K_SWEEP_X, run_sweep(c, 0, cur, oth, 0.0, 1, last == LAST_SX));
        double *t = cur; cur = oth; oth = t;
    }
    if (sy) {
        TIMED(c, K_SWEEP_Y, run_sweep(c, 1, cur, oth, 0.0, 1, last == LAST_SY));
        double *t = cur; cur = oth; oth = t;
    }
    if (mk) {
        TRY(cudaEventRecord(c->ev_mass, c->stream));
        mk->mass_buf = cur;
    }
    if (vis) {
        if (sx) TIMED(c, K_VISC_X, run_visc(c, 0, cur, 0.0, !sy, last == LAST_VX));
        if (sy) TIMED(c, K_VISC_Y, run_visc(c, 1, cur, 0.0, 1, last == LAST_VY));
    }
    if (mk) {
        TRY(cudaEventRecord(c->ev_mom, c->stream));
        mk->mom_buf = cur;
    }
    if (heat) {
        TIMED(c, K_HEAT, run_heat(c, cur, 0.0, 1, 1));
    } else if (trx) {
        TIMED(c, K_RELAX, dimk::launch_relax(p, cur, c->sc, DIM_RELAX_TEMPERATURE, 1, c->stream));
    }
    if (cur != U) TIMED(c, K_COPY, cudaMemcpyAsync(U, cur, sizeof(double) * 8 * (size_t)p.n, cudaMemcpyDeviceToDevice, c->stream));
    return DIM_OK;
}

// FP32 bulk: one split step on the float-float state *cur, the sweeps
// alternating between the two FF buffers (same stages as step_once).  Ud_in
// (may be null): the CFL kernel converts this FP64 state into *cur first.
// Ud_out (may be null): the heat kernel, if the step ends with it, writes the
// end state there in FP64; *out_done tells whether it did.
// cfl_ready: the previous step's heat kernel formed this step's CFL maximum and
// time step (no CFL kernel); *cfl_formed: this step's heat kernel forms the
// next one's (requested by cfl_next)
static int step_once_ff(dim_ctx *c, float2 *&cur, float2 *&oth, const double *Ud_in, double *Ud_out, bool *out_done,
                        bool cfl_ready, bool cfl_next, bool *cfl_formed)
{
    const dim_params &h = c->hp;
    const DevParams &p = c->p;
    const dimk::FFP &f = c->ffp;
    const bool vis = viscous_on(h), heat = heat_on(h), trx = h.trelax != DIM_TRELAX_OFF;
    const bool sx = p.nx > 1, sy = p.ny > 1;
    enum { LAST_SX, LAST_SY, LAST_VX, LAST_VY, LAST_TR, LAST_HEAT } last;
    if (heat) last = LAST_HEAT;
    else if (trx) last = LAST_TR;
    else if (vis) last = sy ? LAST_VY : LAST_VX;
    else last = sy ? LAST_SY : LAST_SX;

    *cfl_formed = false;
    if (cfl_ready && !Ud_in) {
        // this step's smax and dt32 are in place: clear the other accumulators only
        if (cudaMemsetAsync(c->sc->lam, 0, offsetof(Scalars, dt32) - offsetof(Scalars, lam), c->stream) !=
            cudaSuccess)
            return DIM_ECUDA;
    } else {
        TRY(reset_accumulators(c));
        if (Ud_in) TIMED(c, K_WAVE, dimk::launch_wave_ff_in(p, f, Ud_in, cur, c->sc, c->stream));
        else TIMED(c, K_WAVE, dimk::launch_wave_ff(p, f, cur, c->sc, c->stream));
    }
    *out_done = false;
    // the last hyperbolic sweep of a step with a viscous stage also records max
    // 1/rho and max mu, from which the viscous kernel that follows may certify
    // P = 1 without its lambda pass
    if (sx) {
        TIMED(c, K_SWEEP_X, dimk::launch_sweep_ff_bound(p, f, 0, cur, oth, 0.0, c->sc, 1, last == LAST_SX,
                                                        vis && !sy, c->stream));
        float2 *t = cur; cur = oth; oth = t;
    }
    if (sy) {
        TIMED(c, K_SWEEP_Y,
              dimk::launch_sweep_ff_bound(p, f, 1, cur, oth, 0.0, c->sc, 1, last == LAST_SY, vis, c->stream));
        float2 *t = cur; cur = oth; oth = t;
    }
    if (vis) {
        if (sx) {
            TIMED(c, K_VISC_X,
                  dimk::launch_visc_ff(p, f, 0, cur, oth, c->S, c->sc, 0.0, !sy, last == LAST_VX, 3, c->stream));
            float2 *t = cur; cur = oth; oth = t;
        }
        if (sy) {
            TIMED(c, K_VISC_Y, dimk::launch_visc_ff(p, f, 1, cur, oth, c->S, c->sc, 0.0, 1, last == LAST_VY,
                                                    sx ? 2 : 3, c->stream));
            float2 *t = cur; cur = oth; oth = t;
        }
    }
    if (heat) {
        TIMED(c, K_HEAT, dimk::launch_heat_ff(p, f, cur, c->S, c->sc, 0.0, 1, 1, c->stream, Ud_out, &c->lim,
                                              c->lim_tma, cfl_next ? 1 : 0));
        *cfl_formed = cfl_next;
        *out_done = Ud_out != nullptr;
    } else if (trx) {
        TIMED(c, K_RELAX, dimk::launch_relax_ff(p, f, cur, c->sc, DIM_RELAX_TEMPERATURE, 1, c->stream));
    }
    return DIM_OK;
}

// FP32 bulk: nsteps (>= 1) steps of the device state U through the FF planes:
// the first step's CFL kernel converts U in, the last step's heat kernel (or a
// conversion pass, when the step does not end with the heat stage) writes it
// back
static int steps_ff(dim_ctx *c, double *U, int nsteps)
{
    float2 *cur = c->Uf, *oth = ff_other(c);
    bool out_done = false, ready = false;
    for (int s = 0; s < nsteps; s++) {
        bool formed = false;
        int r = step_once_ff(c, cur, oth, s == 0 ? U : nullptr, s == nsteps - 1 ? U : nullptr, &out_done, ready,
                             s < nsteps - 1, &formed);
        if (r != DIM_OK) return r;
        ready = formed;
    }
    if (!out_done) TIMED(c, K_CONVERT, dimk::launch_ff_out(cur, U, state_len(c), c->stream));
    return DIM_OK;
}

// After a timed-out grid barrier the barrier counters may hold arrivals of
// blocks that left: clear them so that the next cooperative launch starts
// from a consistent barrier.
static cudaError_t clear_barrier_if_timeout(dim_ctx *c, unsigned st)
{
    if (!(st & DIM_ST_TIMEOUT)) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(&c->sc->bar_count, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->sc->bar_gen, 0, sizeof(unsigned), c->stream);
    // and the FP32-bulk heat kernel's next-step CFL accumulator and block count
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->sc->smax_next, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->sc->heat_blocks, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

static int read_back(dim_ctx *c, double *dt_last)
{
    unsigned long long bits = 0;
    unsigned st = 0;
    TRY(cudaMemcpyAsync(&bits, &c->sc->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaMemcpyAsync(&st, &c->sc->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    TRY(clear_barrier_if_timeout(c, st));
    if (dt_last) {
        double smax;
        memcpy(&smax, &bits, sizeof(smax));
        *dt_last = c->p.cfl / smax;
    }
    return status_to_code(st);
}

int dim_step(dim_ctx *c, double *U, int nsteps, double *dt_last)
{
    if (!c || !U || nsteps < 0) return DIM_EINVAL;
    if (fp32(c)) {
        if (nsteps > 0) {
            int r = steps_ff(c, U, nsteps);
            if (r != DIM_OK) return r;
        }
    } else {
        for (int s = 0; s < nsteps; s++) {
            int r = step_once(c, U);
            if (r != DIM_OK) return r;
        }
    }
    if (dt_last && nsteps > 0) return read_back(c, dt_last);
    return DIM_OK;
}

int dim_step_host(dim_ctx *c, double *U_host, int nsteps, double *dt_last)
{
    if (!c || !U_host || nsteps < 0) return DIM_EINVAL;
    const size_t n = (size_t)c->p.n, bytes = sizeof(double) * 8 * n, two = sizeof(double) * 2 * n;
    if (!c->Uh && cudaMalloc(&c->Uh, bytes) != cudaSuccess) return DIM_ECUDA;
    if (!c->side) {
        // the two events first, the stream last: c->side is set only once all
        // three exist, and a failure destroys whatever was created
        cudaEvent_t em = nullptr, eo = nullptr;
        cudaStream_t sd = nullptr;
        if (cudaEventCreateWithFlags(&em, cudaEventDisableTiming) != cudaSuccess) em = nullptr;
        if (em && cudaEventCreateWithFlags(&eo, cudaEventDisableTiming) != cudaSuccess) eo = nullptr;
        if (eo && cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking) != cudaSuccess) sd = nullptr;
        if (!sd) {
            if (eo) cudaEventDestroy(eo);
            if (em) cudaEventDestroy(em);
            return DIM_ECUDA;
        }
        c->ev_mass = em;
        c->ev_mom = eo;
        c->side = sd;
    }
    TRY(cudaMemcpyAsync(c->Uh, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
    if (fp32(c) && nsteps > 0) {
        int r = steps_ff(c, c->Uh, nsteps);
        if (r != DIM_OK) return r;
        TRY(cudaMemcpyAsync(U_host, c->Uh, bytes, cudaMemcpyDeviceToHost, c->stream));
    } else if (nsteps == 0) {
        TRY(cudaMemcpyAsync(U_host, c->Uh, bytes, cudaMemcpyDeviceToHost, c->stream));
    } else {
        for (int s = 0; s + 1 < nsteps; s++) {
            int r = step_once(c, c->Uh);
            if (r != DIM_OK) return r;
        }
        // the last step: planes 0-3 go back to the host on the side stream as
        // soon as they are final, overlapping the remaining stages
        StepMarks mk;
        int r = step_once(c, c->Uh, &mk);
        if (r != DIM_OK) return r;
        TRY(cudaStreamWaitEvent(c->side, c->ev_mass, 0));
        TRY(cudaMemcpyAsync(U_host, mk.mass_buf, two, cudaMemcpyDeviceToHost, c->side));
        TRY(cudaStreamWaitEvent(c->side, c->ev_mom, 0));
        TRY(cudaMemcpyAsync(U_host + 2 * n, mk.mom_buf + 2 * n, two, cudaMemcpyDeviceToHost, c->side));
        TRY(cudaMemcpyAsync(U_host + 4 * n, c->Uh + 4 * n, 2 * two, cudaMemcpyDeviceToHost, c->stream));
        TRY(cudaStreamSynchronize(c->side));
    }
    double dtl = 0.0;
    int r = read_back(c, &dtl);
    if (dt_last) *dt_last = dtl;
    return r;
}

int dim_hllc_sweep(dim_ctx *c, double *U, int axis, double dt, int relax)
{
    if (!c || !U || (axis != 0 && axis != 1) || !(dt > 0.0)) return DIM_EINVAL;
    TRY(reset_accumulators(c));
    if (fp32(c)) {
        TIMED(c, K_CONVERT, dimk::launch_ff_in(U, c->Uf, state_len(c), c->stream));
        TIMED(c, axis == 0 ? K_SWEEP_X : K_SWEEP_Y,
              dimk::launch_sweep_ff(c->p, c->ffp, axis, c->Uf, ff_other(c), dt, c->sc, relax, 0, c->stream));
        TIMED(c, K_CONVERT, dimk::launch_ff_out(ff_other(c), U, state_len(c), c->stream));
        return DIM_OK;
    }
    TIMED(c, axis == 0 ? K_SWEEP_X : K_SWEEP_Y, run_sweep(c, axis, U, c->U2, dt, relax, 0));
    TIMED(c, K_COPY, cudaMemcpyAsync(U, c->U2, sizeof(double) * 8 * (size_t)c->p.n, cudaMemcpyDeviceToDevice, c->stream));
    return DIM_OK;
}

int dim_relax(dim_ctx *c, double *U, int which)
{
    if (!c || !U || (which != DIM_RELAX_PRESSURE && which != DIM_RELAX_TEMPERATURE)) return DIM_EINVAL;
    if (fp32(c)) {
        TIMED(c, K_CONVERT, dimk::launch_ff_in(U, c->Uf, state_len(c), c->stream));
        TIMED(c, K_RELAX, dimk::launch_relax_ff(c->p, c->ffp, c->Uf, c->sc, which, 0, c->stream));
        TIMED(c, K_CONVERT, dimk::launch_ff_out(c->Uf, U, state_len(c), c->stream));
        return DIM_OK;
    }
    TIMED(c, K_RELAX, dimk::launch_relax(c->p, U, c->sc, which, 0, c->stream));
    return DIM_OK;
}

int dim_cheb_parabolic(dim_ctx *c, double *U, int kind, double dt, int *P_used)
{
    if (!c || !U || !(dt > 0.0)) return DIM_EINVAL;
    TRY(reset_accumulators(c));
    int slot = 0;
    const bool f32 = fp32(c);
    if (kind == DIM_PARABOLIC_HEAT) {
        if (f32) {
            TIMED(c, K_CONVERT, dimk::launch_ff_in(U, c->Uf, state_len(c), c->stream));
            TIMED(c, K_HEAT, dimk::launch_heat_ff(c->p, c->ffp, c->Uf, c->S, c->sc, dt, 0, 0, c->stream, nullptr,
                                                  &c->lim, c->lim_tma, 0));
            TIMED(c, K_CONVERT, dimk::launch_ff_out(c->Uf, U, state_len(c), c->stream));
        } else {
            TIMED(c, K_HEAT, run_heat(c, U, dt, 0, 0));
        }
        slot = 0;
    } else if (kind == DIM_PARABOLIC_VISCOUS_X || kind == DIM_PARABOLIC_VISCOUS_Y) {
        int axis = kind == DIM_PARABOLIC_VISCOUS_X ? 0 : 1;
        if ((axis == 0 ? c->p.nx : c->p.ny) < 2) {
            if (P_used) *P_used = 0;
            return DIM_OK;
        }
        if (f32) {
            TIMED(c, K_CONVERT, dimk::launch_ff_in(U, c->Uf, state_len(c), c->stream));
            TIMED(c, axis == 0 ? K_VISC_X : K_VISC_Y,
                  dimk::launch_visc_ff(c->p, c->ffp, axis, c->Uf, ff_other(c), c->S, c->sc, dt, 0, 0, 0, c->stream));
            TIMED(c, K_CONVERT, dimk::launch_ff_out(ff_other(c), U, state_len(c), c->stream));
        } else {
            TIMED(c, axis == 0 ? K_VISC_X : K_VISC_Y, run_visc(c, axis, U, dt, 0, 0));
        }
        slot = 1 + axis;
    } else {
        return DIM_EINVAL;
    }
    if (P_used) {
        int P = 0;
        unsigned st = 0;
        TRY(cudaMemcpyAsync(&P, &c->sc->P[slot], sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        TRY(cudaMemcpyAsync(&st, &c->sc->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
        TRY(cudaStreamSynchronize(c->stream));
        *P_used = P;
        if (st & DIM_ST_TIMEOUT) return DIM_ETIMEOUT;
    }
    return DIM_OK;
}

int dim_status(dim_ctx *c, unsigned *flags, int reset)
{
    if (!c || !flags) return DIM_EINVAL;
    TRY(cudaMemcpyAsync(flags, &c->sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    if (reset) TRY(cudaMemsetAsync(&c->sc->status, 0, sizeof(unsigned), c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    TRY(clear_barrier_if_timeout(c, *flags));
    return DIM_OK;
}

int dim_wait_selftest(dim_ctx *c, double seconds)
{
    if (!c || !(seconds > 0.0) || seconds > 1.0) return DIM_EINVAL;
    int khz = 0;
    TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device));
    const long long limit = (long long)(seconds * 1e3 * (double)khz);
    // a word of the context scalars that no kernel writes: the spare P slots
    TRY(cudaMemsetAsync(&c->sc->P[11], 0, sizeof(int), c->stream));
    TRY(dimk::launch_wait_selftest(c->sc, (const unsigned *)&c->sc->P[11], limit, c->stream));
    unsigned st = 0;
    TRY(cudaMemcpyAsync(&st, &c->sc->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    TRY(cudaMemsetAsync(&c->sc->status, 0, sizeof(unsigned), c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    return (st & DIM_ST_TIMEOUT) ? DIM_ETIMEOUT : DIM_OK;
}

int dim_profile(dim_ctx *c, int enable, int reset)
{
    if (!c) return DIM_EINVAL;
    if (reset) {
        TRY(cudaStreamSynchronize(c->stream));
        c->nrec = 0;
    }
    c->prof = enable != 0;
    return DIM_OK;
}

int dim_kernel_time(dim_ctx *c, const char *name, int *launches, double *ms)
{
    if (!c || !name || !launches || !ms) return DIM_EINVAL;
    int kid = -1;
    for (int k = 0; k < K_NKERNELS; k++)
        if (strcmp(name, kKernelNames[k]) == 0) kid = k;
    if (kid < 0) return DIM_EINVAL;
    TRY(cudaStreamSynchronize(c->stream));
    int cnt = 0;
    double tot = 0.0;
    for (int i = 0; i < c->nrec; i++) {
        if (c->recs[i].kid != kid) continue;
        float t = 0.0f;
        TRY(cudaEventElapsedTime(&t, c->recs[i].a, c->recs[i].b));
        tot += t;
        cnt++;
    }
    *launches = cnt;
    *ms = tot;
    return DIM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// helpers for the gradient driver (dim_grad.cu)
// ---------------------------------------------------------------------------
int ctx_step_once(dim_ctx *c, double *U) { return step_once(c, U); }
cudaError_t ctx_reset_scalars(dim_ctx *c) { return reset_accumulators(c); }
dimk::HeatScratch ctx_heat_scratch(dim_ctx *c) { return heat_scratch(c); }
dimk::ViscScratch ctx_visc_scratch(dim_ctx *c) { return visc_scratch(c); }
bool ctx_viscous_on(const dim_params &h) { return viscous_on(h); }
bool ctx_heat_on(const dim_params &h) { return heat_on(h); }
int ctx_status_code(dim_ctx *c)
{
    unsigned st = 0;
    TRY(cudaMemcpyAsync(&st, &c->sc->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    return status_to_code(st);
}

// dim_grad.cu -- schedule record / replay and the reverse-mode gradient of
// nsteps split steps (dim_step_sched, dim_grad, dim_from_primitive_vjp).
//
// dim_grad: a forward pass records the schedule of every step (CFL maximum S,
// every LIM lambda_max) and keeps the state every ckpt_every steps.  The
// reverse pass walks the segments backwards: it replays the segment from its
// checkpoint stage by stage with the recorded schedule (the forward kernels,
// same arithmetic as dim_step, so the same states), keeping every stage's
// input and every Chebyshev iterate of the segment, then applies the stages'
// adjoint kernels in reverse order (dim_adjoint.cu).  When a segment's stage
// states do not fit in half of the free device memory, it keeps only the
// segment's step states and replays each step a second time, stage by stage,
// just before reversing it.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "dim_ctx.h"

namespace dimk {
cudaError_t adj_prelax(const DevParams &p, const double *Uin, double *G, cudaStream_t s);
cudaError_t adj_trelax(const DevParams &p, const double *Uin, double *G, cudaStream_t s);
cudaError_t adj_sweep(const DevParams &p, int axis, const double *Uin, const double *Gout, double *Gin, double dtdx,
                      double *fw, cudaStream_t s);
int adj_face_planes();
cudaError_t adj_visc(const DevParams &p, int axis, const double *Uin, const double *hist, int M, const double *b,
                     double tau, const double *G, double *Gin, double *work, double *pbar, cudaStream_t s);
cudaError_t adj_heat(const DevParams &p, const double *Uin, const double *hist, int N, const int *Ms,
                     const double *bs, double tau, const double *G, double *Gin, double *work, double *pbar,
                     cudaStream_t s);
cudaError_t adj_from_primitive(const DevParams &p, const double *prim, const double *Ub, double *pb, cudaStream_t s);
int adj_visc_work_planes();
int adj_heat_work_planes();
}  // namespace dimk

namespace {

enum StageKind { ST_SWEEP, ST_PRELAX, ST_VISC, ST_TRELAX, ST_HEAT };
struct Stage {
    int kind, axis;
};
constexpr int MAX_STAGES = 10;

// the stages of one step in the order of step_once (Sec. 3): sweeps x, y each
// followed by the pressure relaxation; viscous x, y and the pressure
// relaxation; temperature relaxation; heat conduction
int stage_list(const dim_ctx *c, Stage *s)
{
    const bool sx = c->p.nx > 1, sy = c->p.ny > 1;
    int k = 0;
    if (sx) { s[k++] = {ST_SWEEP, 0}; s[k++] = {ST_PRELAX, 0}; }
    if (sy) { s[k++] = {ST_SWEEP, 1}; s[k++] = {ST_PRELAX, 0}; }
    if (ctx_viscous_on(c->hp)) {
        if (sx) s[k++] = {ST_VISC, 0};
        if (sy) s[k++] = {ST_VISC, 1};
        s[k++] = {ST_PRELAX, 0};
    }
    if (ctx_heat_on(c->hp)) {
        s[k++] = {ST_TRELAX, 0};
        s[k++] = {ST_HEAT, 0};
    } else if (c->hp.trelax != DIM_TRELAX_OFF) {
        s[k++] = {ST_TRELAX, 0};
    }
    return k;
}

// Chebyshev parameter count and b_1..b_{2P-2} of a solve, as the kernels
// derive them from (tau, lambda_max) (cheb_P / cheb_P_visc, cheb_schedule_block)
int host_P_formula(double tau, double lam) { return (int)ceil(3.14159265358979323846 / 4.0 * sqrt(tau * lam + 1.0)); }
int host_P_heat(const DevParams &p, double tau, double lam)
{
    int pf = host_P_formula(tau, lam);
    if (p.p_policy == DIM_P_FIXED) return p.p_fixed;
    int P = pf;
    if (p.p_policy == DIM_P_CLAMP && P < p.p_min) P = p.p_min;
    if (P > p.p_max) P = p.p_max;
    return P;
}
int host_P_visc(const DevParams &p, double tau, double lam)
{
    int pf = host_P_formula(tau, lam);
    return pf > p.p_max ? p.p_max : pf;
}
void host_b(int P, double lam, const double *beta_tab, std::vector<double> &b)
{
    const double *beta = beta_tab + (size_t)(P - 1) * dimk::PMAX;
    const double beta1 = beta[0];
    for (int s = 0; s < 2 * P - 2; s++) {
        int m = s < P - 1 ? P - s : 2 * P - 1 - s;
        b.push_back(lam * (beta1 - beta[m - 1]) / (1.0 + beta1));
    }
}

}  // namespace

struct GradWork {
    size_t cap[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // doubles per buffer
    double *buf[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<double> beta;  // host copy of the Chebyshev roots table
};
enum { GW_CK, GW_SEG, GW_STG, GW_HH, GW_HVX, GW_HVY, GW_G, GW_WORK, GW_SMALL };

void grad_free(dim_ctx *c)
{
    if (!c || !c->gw) return;
    for (int i = 0; i < 9; i++) cudaFree(c->gw->buf[i]);
    delete c->gw;
    c->gw = nullptr;
}

static cudaError_t ensure(GradWork *w, int i, size_t doubles)
{
    if (doubles == 0) doubles = 1;
    if (w->cap[i] >= doubles) return cudaSuccess;
    cudaFree(w->buf[i]);
    w->buf[i] = nullptr;
    w->cap[i] = 0;
    cudaError_t e = cudaMalloc(&w->buf[i], doubles * sizeof(double));
    if (e == cudaSuccess) w->cap[i] = doubles;
    return e;
}

// start a replayed step: clear the scalars, then load the step's record
static cudaError_t replay_begin(dim_ctx *c, const double *rec)
{
    cudaError_t e = ctx_reset_scalars(c);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(c->sc, rec, DIM_SCHED * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

// One replayed step.  stg == nullptr: X is advanced in place.  Otherwise X is
// only read: stg[k] (k = 0..nst) receives the input of stage k (stg[0] = X;
// X may be stg itself) and stg[nst] the step's result; hist_* (may be null)
// receive the Chebyshev iterates.
static int run_step(dim_ctx *c, const double *rec, double *X, double *stg, double *hist_h, double *hist_v0,
                    double *hist_v1)
{
    Stage st[MAX_STAGES];
    const int nst = stage_list(c, st);
    DevParams pf = c->p;
    pf.frozen = 1;
    const size_t sb = sizeof(double) * 8 * (size_t)c->p.n, n8 = 8 * (size_t)c->p.n;
    cudaStream_t s = c->stream;
    TRY(replay_begin(c, rec));
    if (stg && stg != X) TRY(cudaMemcpyAsync(stg, X, sb, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < nst; k++) {
        double *in = stg ? stg + k * n8 : X;
        double *out = stg ? stg + (k + 1) * n8 : X;
        if (st[k].kind == ST_SWEEP) {
            double *tgt = stg ? out : c->U2;
            TRY(dimk::launch_sweep(pf, st[k].axis, in, tgt, 0.0, c->sc, 0, 0, s));
            if (!stg) TRY(cudaMemcpyAsync(X, c->U2, sb, cudaMemcpyDeviceToDevice, s));
            continue;
        }
        if (stg) TRY(cudaMemcpyAsync(out, in, sb, cudaMemcpyDeviceToDevice, s));
        switch (st[k].kind) {
        case ST_PRELAX: TRY(dimk::launch_relax(pf, out, c->sc, DIM_RELAX_PRESSURE, 0, s)); break;
        case ST_TRELAX: TRY(dimk::launch_relax(pf, out, c->sc, DIM_RELAX_TEMPERATURE, 0, s)); break;
        case ST_VISC: {
            dimk::ViscScratch vs = ctx_visc_scratch(c);
            vs.hist = st[k].axis == 0 ? hist_v0 : hist_v1;
            TRY(dimk::launch_visc(pf, st[k].axis, out, vs, c->sc, 0.0, 0, 0, s));
            break;
        }
        case ST_HEAT: {
            dimk::HeatScratch hs = ctx_heat_scratch(c);
            hs.hist = hist_h;
            TRY(dimk::launch_heat(pf, out, hs, c->sc, 0.0, 0, 0, s));
            break;
        }
        }
    }
    return DIM_OK;
}

extern "C" {

int dim_step_sched(dim_ctx *c, double *U, int nsteps, double *sched, int replay)
{
    if (!c || !U || !sched || nsteps < 0) return DIM_EINVAL;
    if (c->p.precision != DIM_PRECISION_FP64) return DIM_EINVAL;
    for (int s = 0; s < nsteps; s++) {
        double *rec = sched + (size_t)DIM_SCHED * s;
        if (replay) {
            int r = run_step(c, rec, U, nullptr, nullptr, nullptr, nullptr);
            if (r != DIM_OK) return r;
        } else {
            int r = ctx_step_once(c, U);
            if (r != DIM_OK) return r;
            TRY(cudaMemcpyAsync(rec, c->sc, DIM_SCHED * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    return DIM_OK;
}

int dim_grad(dim_ctx *c, const double *U0, int nsteps, int ckpt_every, const double *dJ_dUT, double *dJ_dU0,
             double *dJ_dparams)
{
    if (!c || !U0 || !dJ_dUT || !dJ_dU0 || nsteps < 0 || ckpt_every < 1) return DIM_EINVAL;
    if (c->p.precision != DIM_PRECISION_FP64) return DIM_EINVAL;
    // the reverse stages differentiate the equilibrium relaxation and projection
    if (c->hp.trelax == DIM_TRELAX_MIDPOINT || c->hp.heat_alpha != DIM_HEAT_ALPHA_PROJECTION) return DIM_EINVAL;
    const DevParams &p = c->p;
    cudaStream_t s = c->stream;
    const size_t n = (size_t)p.n, n8 = 8 * n, sb = n8 * sizeof(double);
    if (!c->gw) c->gw = new GradWork();
    GradWork *w = c->gw;
    if (w->beta.empty()) {
        w->beta.resize((size_t)dimk::PMAX * dimk::PMAX);
        TRY(cudaMemcpy(w->beta.data(), c->beta, w->beta.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    const int K = ckpt_every < nsteps ? ckpt_every : (nsteps > 0 ? nsteps : 1);
    const int nck = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    Stage st[MAX_STAGES];
    const int nst = stage_list(c, st);
    // small: pbar (8 doubles) + the schedule record
    TRY(ensure(w, GW_SMALL, 8 + (size_t)DIM_SCHED * (nsteps > 0 ? nsteps : 1)));
    double *pbar = w->buf[GW_SMALL], *sched = w->buf[GW_SMALL] + 8;
    TRY(ensure(w, GW_CK, n8 * (nck > 0 ? nck : 1)));
    TRY(ensure(w, GW_G, 2 * n8));
    const int wp = dimk::adj_visc_work_planes() > dimk::adj_heat_work_planes() ? dimk::adj_visc_work_planes()
                                                                               : dimk::adj_heat_work_planes();
    // work planes of the parabolic adjoints, then the per-face adjoints of the sweeps
    const size_t nfmax = n + (size_t)(p.nx > p.ny ? p.nx : p.ny);
    const size_t nwork = n * (size_t)wp > nfmax * dimk::adj_face_planes() ? n * (size_t)wp
                                                                          : nfmax * dimk::adj_face_planes();
    TRY(ensure(w, GW_WORK, nwork));
    double *ck = w->buf[GW_CK];
    double *G = w->buf[GW_G], *G2 = w->buf[GW_G] + n8, *work = w->buf[GW_WORK];
    TRY(ensure(w, GW_SEG, n8));
    double *seg = w->buf[GW_SEG];

    // forward pass: record the schedule, keep the checkpoints
    TRY(cudaMemcpyAsync(seg, U0, sb, cudaMemcpyDeviceToDevice, s));
    for (int t = 0; t < nsteps; t++) {
        if (t % K == 0) TRY(cudaMemcpyAsync(ck + (size_t)(t / K) * n8, seg, sb, cudaMemcpyDeviceToDevice, s));
        int r = ctx_step_once(c, seg);
        if (r != DIM_OK) return r;
        TRY(cudaMemcpyAsync(sched + (size_t)DIM_SCHED * t, c->sc, DIM_SCHED * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    }
    {
        int r = ctx_status_code(c);
        if (r != DIM_OK) return r;
    }
    std::vector<double> rec((size_t)DIM_SCHED * (nsteps > 0 ? nsteps : 1));
    TRY(cudaMemcpyAsync(rec.data(), sched, sizeof(double) * DIM_SCHED * nsteps, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));

    // per step: tau, Chebyshev counts; the largest histories
    const int nout = p.n_outer < 1 ? 1 : (p.n_outer > 8 ? 8 : p.n_outer);
    size_t hh = 0, hv[2] = {0, 0};
    for (int t = 0; t < nsteps; t++) {
        const double *r = rec.data() + (size_t)DIM_SCHED * t;
        const double tau = p.cfl / r[0];
        size_t h = 0;
        for (int it = 0; it < nout; it++) h += 2 * (size_t)host_P_heat(p, tau, r[1 + it]);
        if (h > hh) hh = h;
        for (int a = 0; a < 2; a++) {
            size_t v = 2 * (2 * (size_t)host_P_visc(p, tau, r[9 + a]) - 2);
            if (v > hv[a]) hv[a] = v;
        }
    }
    bool heat = false, visc[2] = {false, false};
    for (int k = 0; k < nst; k++) {
        if (st[k].kind == ST_HEAT) heat = true;
        if (st[k].kind == ST_VISC) visc[st[k].axis] = true;
    }
    if (!heat) hh = 0;
    if (!visc[0]) hv[0] = 0;
    if (!visc[1]) hv[1] = 0;
    // Segment storage: when one segment's stage states (K nst + 1 states, the
    // output of each step being the input of the next) and Chebyshev iterates
    // fit in half of the free device memory, the reverse pass replays each
    // segment once, keeping everything; otherwise it keeps the segment's step
    // states only and replays each step a second time, stage by stage.
    const size_t per_step_hist = n * (hh + hv[0] + hv[1]);
    size_t fr = 0, tot = 0;
    TRY(cudaMemGetInfo(&fr, &tot));
    const size_t seg_doubles = (size_t)K * ((size_t)nst * n8 + per_step_hist) + n8;
    const size_t have = w->cap[GW_STG] + w->cap[GW_HH] + w->cap[GW_HVX] + w->cap[GW_HVY] + w->cap[GW_SEG];
    const char *force = getenv("DIM_GRAD_KEEP_SEGMENT");  // "0": always the two-replay form
    const bool keep = !(force && force[0] == '0') && seg_doubles * sizeof(double) < (fr + have * sizeof(double)) / 2;
    const size_t Ks = keep ? (size_t)K : 1;  // steps whose stage states and iterates are kept
    if (keep) {
        TRY(ensure(w, GW_STG, (size_t)K * nst * n8 + n8));
    } else {
        TRY(ensure(w, GW_SEG, n8 * (size_t)K));
        TRY(ensure(w, GW_STG, n8 * (size_t)(nst + 1)));
    }
    seg = w->buf[GW_SEG];
    double *stg = w->buf[GW_STG];
    TRY(ensure(w, GW_HH, Ks * n * hh));
    TRY(ensure(w, GW_HVX, Ks * n * hv[0]));
    TRY(ensure(w, GW_HVY, Ks * n * hv[1]));

    // reverse pass
    TRY(cudaMemcpyAsync(G, dJ_dUT, sb, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemsetAsync(pbar, 0, 8 * sizeof(double), s));
    DevParams pf = p;
    pf.frozen = 1;
    std::vector<double> b;
    std::vector<int> Ms;
    // Chebyshev iterates of step t of the current segment (slot 0 when only one step is kept)
    auto hist_of = [&](int buf, size_t planes, int slot) -> double * {
        return planes ? w->buf[buf] + (size_t)slot * n * planes : nullptr;
    };
    for (int sg = nck - 1; sg >= 0; sg--) {
        const int t0 = sg * K, t1 = t0 + K < nsteps ? t0 + K : nsteps;
        if (keep) {
            // replay the segment once, keeping every stage state and iterate
            TRY(cudaMemcpyAsync(stg, ck + (size_t)sg * n8, sb, cudaMemcpyDeviceToDevice, s));
            for (int t = t0; t < t1; t++) {
                const int j = t - t0;
                double *sj = stg + (size_t)j * nst * n8;
                int r = run_step(c, sched + (size_t)DIM_SCHED * t, sj, sj, hist_of(GW_HH, hh, j),
                                 hist_of(GW_HVX, hv[0], j), hist_of(GW_HVY, hv[1], j));
                if (r != DIM_OK) return r;
            }
        } else {
            TRY(cudaMemcpyAsync(seg, ck + (size_t)sg * n8, sb, cudaMemcpyDeviceToDevice, s));
            for (int t = t0; t + 1 < t1; t++) {
                double *nx = seg + (size_t)(t - t0 + 1) * n8;
                TRY(cudaMemcpyAsync(nx, seg + (size_t)(t - t0) * n8, sb, cudaMemcpyDeviceToDevice, s));
                int r = run_step(c, sched + (size_t)DIM_SCHED * t, nx, nullptr, nullptr, nullptr, nullptr);
                if (r != DIM_OK) return r;
            }
        }
        for (int t = t1 - 1; t >= t0; t--) {
            const double *r = rec.data() + (size_t)DIM_SCHED * t;
            const double tau = p.cfl / r[0];
            const int slot = keep ? t - t0 : 0;
            double *hist_h = hist_of(GW_HH, hh, slot);
            double *hist_v[2] = {hist_of(GW_HVX, hv[0], slot), hist_of(GW_HVY, hv[1], slot)};
            const double *sg_stg = keep ? stg + (size_t)slot * nst * n8 : stg;
            if (!keep) {
                // the step's stage inputs and Chebyshev iterates
                int rr = run_step(c, sched + (size_t)DIM_SCHED * t, seg + (size_t)(t - t0) * n8, stg, hist_h,
                                  hist_v[0], hist_v[1]);
                if (rr != DIM_OK) return rr;
            }
            for (int k = nst - 1; k >= 0; k--) {
                const double *in = sg_stg + (size_t)k * n8;
                switch (st[k].kind) {
                case ST_PRELAX: TRY(dimk::adj_prelax(pf, in, G, s)); break;
                case ST_TRELAX: TRY(dimk::adj_trelax(pf, in, G, s)); break;
                case ST_SWEEP: {
                    const double dtdx = tau / (st[k].axis == 0 ? p.dx : p.dy);
                    TRY(dimk::adj_sweep(pf, st[k].axis, in, G, G2, dtdx, work, s));
                    double *tmp = G; G = G2; G2 = tmp;
                    break;
                }
                case ST_VISC: {
                    const int a = st[k].axis;
                    const int P = host_P_visc(p, tau, r[9 + a]);
                    b.clear();
                    host_b(P, r[9 + a], w->beta.data(), b);
                    TRY(dimk::adj_visc(pf, a, in, hist_v[a], 2 * P - 2, b.data(), tau, G, G2, work, pbar, s));
                    double *tmp = G; G = G2; G2 = tmp;
                    break;
                }
                case ST_HEAT: {
                    b.clear();
                    Ms.clear();
                    for (int it = 0; it < nout; it++) {
                        const int P = host_P_heat(p, tau, r[1 + it]);
                        Ms.push_back(2 * P - 2);
                        host_b(P, r[1 + it], w->beta.data(), b);
                    }
                    TRY(dimk::adj_heat(pf, in, hist_h, nout, Ms.data(), b.data(), tau, G, G2, work, pbar, s));
                    double *tmp = G; G = G2; G2 = tmp;
                    break;
                }
                }
            }
            // the host-side b and Ms are read by the launches above only
            // through kernel arguments, so they can be reused at once
        }
    }
    TRY(cudaMemcpyAsync(dJ_dU0, G, sb, cudaMemcpyDeviceToDevice, s));
    double pb[8];
    TRY(cudaMemcpyAsync(pb, pbar, sizeof(pb), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (dJ_dparams) memcpy(dJ_dparams, pb, sizeof(double) * DIM_GRAD_NPARAMS);
    return ctx_status_code(c);
}

int dim_from_primitive_vjp(dim_ctx *c, const double *prim, const double *Ubar, double *primbar)
{
    if (!c || !prim || !Ubar || !primbar) return DIM_EINVAL;
    TRY(dimk::adj_from_primitive(c->p, prim, Ubar, primbar, c->stream));
    return DIM_OK;
}

}  // extern "C"

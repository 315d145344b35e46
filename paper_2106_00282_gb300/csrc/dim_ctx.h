// dim_ctx.h -- the library context and the stage launchers, shared by the
// host-side translation units of the C ABI (dim_api.cu, dim_grad.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/dim.h"
#include "dim_ff.cuh"

namespace dimk {
cudaError_t sweep_setup();
cudaError_t parabolic_setup(int nsm);
cudaError_t launch_sweep(const DevParams &p, int axis, const double *Uin, double *Uout, double dt_host, Scalars *sc,
                         int relax, int check, cudaStream_t s);
cudaError_t launch_from_primitive(const DevParams &p, const double *prim, double *U, Scalars *sc, cudaStream_t s);
cudaError_t launch_wave_max(const DevParams &p, const double *U, Scalars *sc, cudaStream_t s);
cudaError_t launch_relax(const DevParams &p, double *U, Scalars *sc, int which, int check, cudaStream_t s);
cudaError_t launch_wait_selftest(Scalars *sc, const unsigned *word, long long limit, cudaStream_t s);
cudaError_t launch_heat(const DevParams &p, double *U, const HeatScratch &s, Scalars *sc, double dt_host,
                        int trelax_first, int check, cudaStream_t st);
cudaError_t launch_visc(const DevParams &p, int axis, double *U, const ViscScratch &s, Scalars *sc, double dt_host,
                        int relax, int check, cudaStream_t st);
// FP32-bulk form on float-float state planes (dim_bulkff.cu)
cudaError_t bulkff_setup(int nsm);
FFP ffp_of(const DevParams &p);
cudaError_t launch_ff_in(const double *U, float2 *F, size_t m, cudaStream_t s);
cudaError_t launch_ff_out(const float2 *F, double *U, size_t m, cudaStream_t s);
cudaError_t launch_wave_ff(const DevParams &p, const FFP &f, const float2 *U, Scalars *sc, cudaStream_t s);
cudaError_t launch_wave_ff_in(const DevParams &p, const FFP &f, const double *Ud, float2 *U, Scalars *sc,
                              cudaStream_t s);
cudaError_t launch_sweep_ff(const DevParams &p, const FFP &f, int axis, const float2 *Uin, float2 *Uout,
                            double dt_host, Scalars *sc, int relax, int check, cudaStream_t s);
cudaError_t launch_sweep_ff_bound(const DevParams &p, const FFP &f, int axis, const float2 *Uin, float2 *Uout,
                                  double dt_host, Scalars *sc, int relax, int check, int bound, cudaStream_t s);
cudaError_t launch_relax_ff(const DevParams &p, const FFP &f, float2 *U, Scalars *sc, int which, int check,
                            cudaStream_t s);
int heat_tma_setup(const DevParams &p, double *S, LimMaps *m);
cudaError_t launch_heat_ff(const DevParams &p, const FFP &f, float2 *U, double *S, Scalars *sc, double dt_host,
                           int trelax_first, int check, cudaStream_t st, double *Ud, const LimMaps *tm, int use_tma,
                           int cfl_next);
cudaError_t launch_visc_ff(const DevParams &p, const FFP &f, int axis, const float2 *U, float2 *Uo, double *S,
                           Scalars *sc, double dt_host, int relax, int check, int lam_mode, cudaStream_t st);
}  // namespace dimk

using dimk::DevParams;
using dimk::Scalars;

namespace dimctx {

enum KernelId { K_SWEEP_X, K_SWEEP_Y, K_HEAT, K_VISC_X, K_VISC_Y, K_WAVE, K_RELAX, K_COPY, K_CONVERT, K_NKERNELS };

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

}  // namespace dimctx
using dimctx::ProfRec;

struct GradWork;  // workspace of dim_grad (dim_grad.cu), allocated on first use

struct dim_ctx {
    dim_params hp;
    DevParams p;
    cudaStream_t stream;
    double *U2;   // 8 planes: out-of-place target of the sweeps
    double *S;    // dimk::SCRATCH_PLANES scratch planes for the parabolic stages
    double *Uh;   // 8 planes: device copy of a host state (dim_step_host), lazily allocated
    // dim_step_host: a second stream that copies the planes a step has finished
    // (masses after the sweeps, momenta after the viscous stage) back to the
    // host while the later stages run; events marking those points (lazily created)
    cudaStream_t side;
    cudaEvent_t ev_mass, ev_mom;
    double *beta; // Chebyshev roots table (PMAX x PMAX)
    // FP32 bulk: the state as float-float planes (8 planes of n float2) while
    // steps run; U2 holds the other buffer of the sweeps' ping-pong
    float2 *Uf;
    dimk::FFP ffp;
    dimk::LimMaps lim;  // TMA descriptors of the heat stage's planes (lim_tma != 0)
    int lim_tma;
    Scalars *sc;
    int device;
    // profiling
    int prof;
    ProfRec *recs;
    int nrec, caprec;
    GradWork *gw;
};

void grad_free(dim_ctx *c);  // releases c->gw (dim_grad.cu)

// helpers of dim_api.cu used by dim_grad.cu
int ctx_step_once(dim_ctx *c, double *U);  // one split step, stream-ordered
cudaError_t ctx_reset_scalars(dim_ctx *c);  // clear the per-step scalars (S, lambda_max, P)
dimk::HeatScratch ctx_heat_scratch(dim_ctx *c);
dimk::ViscScratch ctx_visc_scratch(dim_ctx *c);
bool ctx_viscous_on(const dim_params &h);
bool ctx_heat_on(const dim_params &h);
int ctx_status_code(dim_ctx *c);  // synchronizes; DIM_* code of the status word

#define TRY(x)                                     \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return DIM_ECUDA;   \
    } while (0)



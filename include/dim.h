/*
 * dim.h -- C ABI of the GB300 (sm_103a) split time step of the reduced
 * two-temperature Baer-Nunziato model (Zhang, Menshov, Wang & Shen,
 * arXiv:2106.00282): a diffuse-interface model of two compressible phases with
 * phase masses, phase internal energies, mixture momentum, mixture total
 * energy and volume fraction, stiffened-gas EOS, viscosity and heat conduction.
 *
 * Conventions
 * -----------
 *  - State U: 8 planes of nx*ny doubles in DEVICE memory, row-major, cell
 *    (i, j) at j*nx + i, plane q at q*nx*ny:
 *      0 m1 = alpha_1 rho_1   1 m2 = alpha_2 rho_2   2 rho u   3 rho v
 *      4 E1 = alpha_1 rho_1 e_1   5 E2 = alpha_2 rho_2 e_2   6 rho E   7 alpha_2
 *    (the conservative vector of Sec. 3.1, Eq. vectorForm).  Phase 1 is the
 *    dense phase (liquid/solid), phase 2 the gas.  The caller owns U; it must
 *    be 256-byte aligned (any cudaMalloc / torch allocation is).
 *  - Every call is stream-ordered on the stream given to dim_init and does not
 *    synchronize unless it returns a host value (dt_last, P_used, status).
 *  - Return value: 0 on success, a negative DIM_E* code otherwise.  After an
 *    error U is unspecified; restore it from a copy.
 *  - The library owns only the scratch it allocates in dim_init (about
 *    16 planes of nx*ny doubles plus a few device scalars).
 */
#ifndef DIM_H
#define DIM_H

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define DIM_OK 0
#define DIM_EINVAL (-1)   /* bad parameter, size or pointer */
#define DIM_ECUDA (-2)    /* a CUDA call failed (launch, allocation, copy) */
#define DIM_ENONPHYS (-3) /* the end-of-step state is not admissible: alpha_2 outside (0,1),
                             m_k <= 0, p + pinf_k <= 0, or a NaN */
#define DIM_ENOROOT (-4)  /* a relaxation quadratic had no real root */
#define DIM_ETIMEOUT (-5) /* a bounded grid-wide wait inside a kernel gave up */
#define DIM_ENOTIMPL (-6) /* entry point not implemented by this library */
#define DIM_ETOOLARGE (-7) /* grid larger than the fixed scratch of dim_hllc_sweep_noalloc */

/* device status word bits (dim_status) */
#define DIM_ST_NONPHYS 1u   /* end-of-step state inadmissible */
#define DIM_ST_NAN 2u       /* NaN met */
#define DIM_ST_NOROOT 4u    /* negative discriminant in a relaxation quadratic */
#define DIM_ST_TRANSIENT 8u /* an intermediate stage met an inadmissible phase state that a later
                               stage of the same step repaired (informational) */
#define DIM_ST_PCAP 16u     /* the P formula exceeded p_max; P = p_max was used (informational) */
#define DIM_ST_TIMEOUT 32u  /* a grid barrier wait gave up */

/* flag values of dim_params */
#define DIM_LIMITER_NONE 0   /* first-order Godunov */
#define DIM_LIMITER_MINMOD 1 /* PVT-consistent MUSCL, Sec. 3.6 */
#define DIM_LIMITER_OVERBEE 2 /* interface sharpening (cited in Sec. 4.1): slope 2 minmod on alpha_2 and
                                 alpha_k rho_k, minmod on u and p_k */
#define DIM_BC_TRANSMISSIVE 0
#define DIM_BC_PERIODIC 1
#define DIM_TRELAX_OFF 0         /* no temperature relaxation and no conduction */
#define DIM_TRELAX_EQUILIBRIUM 1 /* exact p,T equilibrium, Sec. 3.4.1 */
#define DIM_TRELAX_MIDPOINT 2    /* the implicit scheme of Eqs. ht_eq2_TR_dis, ht_eq3_TR_dis with B2 (Eq. B2_2,
                                    sign that keeps dp1 = dp2) at the averages, trelax_iters simple iterations
                                    from T' = Eq. Taverage, alpha' = alpha^0 (FP64 only) */
#define DIM_HEAT_ALPHA_PROJECTION 0 /* heat stage: (T, alpha) = p,T equilibrium of the updated rho e */
#define DIM_HEAT_ALPHA_LINEAR 1     /* heat stage: T += tau V (L_h u_hat + I), alpha += tau U (L_h u_hat + I) with
                                       the frozen V, U of Eqs. ht_eq2_ht, ht_eq3_ht (FP64 only) */
#define DIM_P_FORMULA 0          /* P = ceil(pi/4 sqrt(tau lambda_max + 1)), capped at p_max */
#define DIM_P_FIXED 1            /* P = p_fixed */
#define DIM_P_CLAMP 2            /* P = clamp(formula, p_min, p_max) */

#define DIM_PRECISION_FP64 0      /* every operation in FP64 */
#define DIM_PRECISION_FP32_BULK 1 /* no FP64 arithmetic inside a step: the state is carried as
                                     float-float pairs (47 bits), which hold the accumulation, the phase
                                     pressures' cancellation against the stiffened-gas cold energy, the
                                     volume fraction and its transport, and one Newton correction of each
                                     relaxation root; flux, relaxation and stencil arithmetic in FP32.  The
                                     caller's state stays FP64; each call converts it once in and out */

#define DIM_RELAX_PRESSURE 0    /* dim_relax: Sec. 3.3 three-step pressure relaxation */
#define DIM_RELAX_TEMPERATURE 1 /* dim_relax: Sec. 3.4.1 temperature relaxation */

#define DIM_PARABOLIC_HEAT 0      /* dim_cheb_parabolic: Sec. 3.4.2 heat conduction, Algorithm 1 */
#define DIM_PARABOLIC_VISCOUS_X 1 /* dim_cheb_parabolic: Sec. 3.2 viscous step along x */
#define DIM_PARABOLIC_VISCOUS_Y 2 /* dim_cheb_parabolic: Sec. 3.2 viscous step along y */

/* Phase and solver parameters.  Stiffened-gas EOS per phase k (Eqs.
 * eos_stiffened, eos_stiffened2, q_k = 0):
 *   rho_k e_k = (p_k + gamma_k pinf_k)/(gamma_k - 1) = rho_k Cv_k T_k + pinf_k.
 * Conductivity lambda_k(T) = k0_k (T/T_ref)^k_exp; viscosity mu_k constant;
 * mixture coefficients are volume-fraction means (Sec. 4.2). */
typedef struct dim_params {
    double gamma[2], pinf[2], cv[2];
    double k0[2], k_exp, T_ref;
    double mu[2];
    double cfl;
    int limiter;
    int bc[2]; /* per axis (x, y) */
    int trelax;
    int n_outer; /* outer iterations of Algorithm 1 (>= 1) */
    int p_policy, p_fixed, p_min, p_max;
    int precision; /* DIM_PRECISION_FP64 or DIM_PRECISION_FP32_BULK */
    double src[2]; /* external heat source I_k >= 0 per unit volume of phase k: I_k = alpha_k I_k (Eq. I),
                      deposited in the heat-conduction stage */
    int heat_alpha;   /* DIM_HEAT_ALPHA_PROJECTION or DIM_HEAT_ALPHA_LINEAR */
    int trelax_iters; /* simple iterations of DIM_TRELAX_MIDPOINT, 1..1000 (read only in that mode) */
} dim_params;

typedef struct dim_ctx dim_ctx; /* opaque: parameters, grid, stream, scratch */

/* Create a context for an nx x ny grid of spacing (dx, dy) and allocate its
 * scratch.  A 1D problem is ny = 1 (or nx = 1); an axis of extent 1 is inactive.
 * cuda_stream is a cudaStream_t (NULL: legacy default stream).
 * Errors: DIM_EINVAL for non-positive sizes/spacings, nx * ny above 2^27 cells
 * (134,217,728: the 32-bit cell-plane indexing of the kernels), a 1 x 1 grid
 * (no axis, hence no CFL time scale), gamma_k <= 1, Cv_k <= 0,
 * cfl <= 0, unknown flags, p_max outside [1, 64], DIM_TRELAX_MIDPOINT with
 * trelax_iters outside [1, 1000], DIM_TRELAX_MIDPOINT or DIM_HEAT_ALPHA_LINEAR
 * with a precision other than FP64; DIM_ECUDA on allocation
 * failure.  The paper's parameters: Sec. 2 (EOS), Sec. 3 (scheme). */
int dim_init(dim_ctx **out, const dim_params *p, int nx, int ny, double dx, double dy, void *cuda_stream);

/* Release the scratch and the context (synchronizes its stream). */
void dim_destroy(dim_ctx *c);

/* Fill U from primitive fields prim (device, 5 planes of nx*ny doubles:
 * alpha_2, p, T, u, v) with both phases at the cell's (p, T): rho_k from Eq.
 * eos_stiffened2, E_k = alpha_k (p + gamma_k pinf_k)/(gamma_k - 1) from Eq.
 * eos_stiffened, rho E = E1 + E2 + rho |u|^2 / 2.  prim and U must not overlap. */
int dim_from_primitive(dim_ctx *c, const double *prim, double *U);

/* Time step of the CFL condition (Sec. 3.1 mixture sound speed
 * c^2 = Y1 c1^2 + Y2 c2^2): dt = cfl / max_cells max_axis (|u_axis| + c)/h_axis.
 * Writes the host double *dt (synchronizes). */
int dim_cfl_dt(dim_ctx *c, const double *U, double *dt);

/* nsteps split steps in place on U (Sec. 3): per step dt from the CFL
 * condition; hyperbolic sweep along x then y (MUSCL + HLLC + non-conservative
 * term, Sec. 3.1/3.6), each followed by pressure relaxation (Sec. 3.3);
 * viscous steps along x and y (Sec. 3.2, only if some mu_k > 0) and pressure
 * relaxation; temperature relaxation (Sec. 3.4.1) and heat conduction
 * (Sec. 3.4.2, Algorithm 1; only if some k0_k > 0), unless trelax is OFF.
 * dt_last: host out (may be NULL).  If dt_last is non-NULL the call
 * synchronizes and also returns DIM_ENONPHYS / DIM_ENOROOT / DIM_ETIMEOUT when
 * the status word says so; with dt_last NULL it is fully asynchronous (check
 * dim_status later). */
int dim_step(dim_ctx *c, double *U, int nsteps, double *dt_last);

/* The same nsteps split steps on a HOST state U_host (8 planes as above, any
 * alignment; page-locked memory lets the copies run asynchronously): copies it
 * to a context-owned device buffer, steps, copies it back -- the masses and
 * momenta of the last step on a second stream as soon as they are final,
 * overlapping the remaining stages; synchronizes; returns the status like
 * dim_step with dt_last. */
int dim_step_host(dim_ctx *c, double *U_host, int nsteps, double *dt_last);

/* One hyperbolic sweep along axis (0 = x, 1 = y) with time step dt (> 0),
 * followed by the pressure relaxation of Sec. 3.3 when relax != 0; in place on
 * U (the sweep itself is computed out of place into scratch). */
int dim_hllc_sweep(dim_ctx *c, double *U, int axis, double dt, int relax);

/* Pointwise relaxation in place: DIM_RELAX_PRESSURE (Sec. 3.3, steps 1-3) or
 * DIM_RELAX_TEMPERATURE (Sec. 3.4.1, exact p,T equilibrium). */
int dim_relax(dim_ctx *c, double *U, int which);

/* Parabolic stage by the Chebyshev local-iteration method (Sec. 3.2, Eqs. LIM,
 * LIM_last) with time step dt: DIM_PARABOLIC_HEAT (Sec. 3.4.2; the input must be
 * in p,T equilibrium, e.g. after dim_relax(TEMPERATURE)) or
 * DIM_PARABOLIC_VISCOUS_X / _Y (Sec. 3.2, no pressure relaxation).  P_used: host
 * out, the number of Chebyshev parameters used (may be NULL; non-NULL
 * synchronizes). */
int dim_cheb_parabolic(dim_ctx *c, double *U, int kind, double dt, int *P_used);

/* Schedule record of one step: DIM_SCHED doubles, [0] S = max_cells max_axis
 * (|u_axis| + c)/h_axis (dt = cfl / S, Sec. 3.1), [1..8] the Gershgorin
 * lambda_max of the heat-conduction solve of outer iterations 0..7 of Algorithm
 * 1, [9] / [10] that of the viscous solve along x / y (Sec. 3.2); slots of
 * stages that did not run are 0.  The Chebyshev parameter count P and the b_m
 * of each solve follow from (dt, lambda_max). */
#define DIM_SCHED 11
/* Parameters a gradient is taken with respect to (dJ_dparams of dim_grad):
 * k0_1, k0_2 (conductivity coefficients), mu_1, mu_2 (viscosities), I_1, I_2
 * (external heat-source intensities, Eq. I). */
#define DIM_GRAD_NPARAMS 6

/* nsteps split steps as dim_step (FP64 precision only), recording (replay = 0)
 * or replaying (replay != 0) the schedule: sched is a DEVICE array of
 * nsteps * DIM_SCHED doubles, written per step, or read per step in place of
 * the CFL reduction and of every LIM lambda_max reduction.  Replaying the
 * record of a run on that run's initial state reproduces it bit for bit;
 * replaying it on a perturbed state gives the map with the time steps and
 * Chebyshev parameters held fixed, the map dim_grad differentiates.
 * Asynchronous.  Errors: DIM_EINVAL (null pointers, nsteps < 0, FP32-bulk
 * precision), DIM_ECUDA. */
int dim_step_sched(dim_ctx *c, double *U, int nsteps, double *sched, int replay);

/* Reverse-mode gradient (adjoint) of the map U0 -> U_T = nsteps split steps,
 * FP64 precision, with the schedule of the run from U0 held fixed: the time
 * step of every step (Sec. 3.1) and the lambda_max, hence P and b_m, of every
 * LIM solve (Sec. 3.2), and every value-decided branch (limiter operand,
 * Davis bounds, HLLC wave region) taken as in that run.  Given the adjoint
 * dJ_dUT = dJ/dU_T of an objective J, returns dJ_dU0 = (dU_T/dU0)^T dJ_dUT and,
 * when dJ_dparams != NULL, dJ/d(k0_1, k0_2, mu_1, mu_2, I_1, I_2).
 *  - U0, dJ_dUT, dJ_dU0: DEVICE arrays of 8 planes (the state layout);
 *    dJ_dU0 may alias dJ_dUT; U0 is not modified.
 *  - dJ_dparams: HOST array of DIM_GRAD_NPARAMS doubles, or NULL.
 *  - ckpt_every >= 1: the forward states are kept every ckpt_every steps and
 *    each segment is replayed once from its checkpoint in the reverse sweep,
 *    keeping its stage states and Chebyshev iterates: device memory ~
 *    nsteps/ckpt_every + ckpt_every x (stages per step, <= 9) states plus
 *    ckpt_every steps' iterates, allocated on the first call and reused.  If
 *    that exceeds half of the free device memory (or the environment variable
 *    DIM_GRAD_KEEP_SEGMENT is "0"), each step is replayed a second time instead
 *    and ~ (nsteps/ckpt_every + ckpt_every + 10) states plus one step's iterates
 *    suffice.  Both forms give the same gradient bit for bit.
 * Synchronizes.  Errors: DIM_EINVAL (null pointers, nsteps < 0, ckpt_every < 1,
 * FP32-bulk precision, DIM_TRELAX_MIDPOINT, DIM_HEAT_ALPHA_LINEAR: the adjoint
 * differentiates the equilibrium projection), DIM_ENONPHYS / DIM_ENOROOT / DIM_ETIMEOUT when the
 * forward run meets them, DIM_ECUDA. */
int dim_grad(dim_ctx *c, const double *U0, int nsteps, int ckpt_every, const double *dJ_dUT, double *dJ_dU0,
             double *dJ_dparams);

/* Failure-detection self-test of the bounded waits: one thread waits, for at
 * most `seconds` (0 < seconds <= 1) of SM clock, on a context word that nothing
 * writes, through the same bounded-wait routine the grid barriers of the
 * cooperative kernels use.  The wait runs out and the call returns DIM_ETIMEOUT
 * (the status bit is cleared again); the context stays usable.  DIM_EINVAL for
 * a null context or seconds outside (0, 1], DIM_ECUDA on a CUDA error.
 * Synchronizes.  (Any call that reports DIM_ETIMEOUT through the status word
 * also clears the grid-barrier counters, so later cooperative launches start
 * from a consistent barrier.) */
int dim_wait_selftest(dim_ctx *c, double seconds);

/* Vector-Jacobian product of dim_from_primitive: primbar (DEVICE, 5 planes:
 * alpha_2, p, T, u, v) = (dU/dprim)^T Ubar at the primitive state prim (DEVICE,
 * 5 planes); Ubar DEVICE, 8 planes.  For chaining an initial-condition
 * parametrisation to dim_grad.  Asynchronous.  Errors: DIM_EINVAL, DIM_ECUDA. */
int dim_from_primitive_vjp(dim_ctx *c, const double *prim, const double *Ubar, double *primbar);

/* The sweep of dim_hllc_sweep without a context and without any allocation,
 * in the precision p->precision selects (the FP64 or the FP32-bulk sweep
 * kernel, as dim_hllc_sweep picks them).
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory -- applications whose own pool
 * allocator owns all device memory, programs with a device-memory budget fixed
 * at load time, and loops that cannot afford the device-wide synchronization of
 * cudaMalloc/cudaFree.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its scratch (an out-of-place copy of the state and the status
 * scalars) is a fixed array compiled into the library, DIM_NOALLOC_MAX_CELLS
 * cells x 8 doubles + 512 B (4 MiB), held by every GPU that loads the library
 * until the process exits.
 *  - p, nx, ny, dx, dy: as for dim_init (validated the same way); U: device
 *    state as everywhere (8 planes, caller-owned), updated in place; axis 0 = x,
 *    1 = y; dt > 0; relax != 0 applies the pressure relaxation of
 *    dim_relax(DIM_RELAX_PRESSURE) after the sweep; cuda_stream: a
 *    cudaStream_t (NULL: legacy default stream).
 *  - Returns DIM_ETOOLARGE if nx * ny > DIM_NOALLOC_MAX_CELLS, DIM_EINVAL for
 *    invalid arguments, DIM_ECUDA if a CUDA call fails.  Asynchronous.
 *  - The first call on a device sets that device up (looks up the array's
 *    device address, sets the kernels' shared-memory limit); make that first
 *    call before any stream capture.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents (the status scalars are cleared at every call): calls that
 *    overlap on the GPU (different streams, or different host threads) race and
 *    give wrong results; serialise them.
 *  - The sweep's status bits (NaN met, a relaxation quadratic without an
 *    admissible root) go to status scalars inside the fixed array, which no
 *    entry point reads: this entry point cannot report them.  A caller that
 *    needs them uses dim_hllc_sweep and dim_status. */
#define DIM_NOALLOC_MAX_CELLS 65536
int dim_hllc_sweep_noalloc(const dim_params *p, int nx, int ny, double dx, double dy, double *U, int axis, double dt,
                           int relax, void *cuda_stream);

/* ---- Batches: many independent grids advanced together (FP32 bulk) ----
 * A batch of ninst independent problems with the same phase parameters and
 * flags p (p->precision must be DIM_PRECISION_FP32_BULK) on grids nx[i] x ny[i]
 * (both >= 2) of spacing dx[i], dy[i].  Each instance has its own CFL time
 * step, lambda_max and Chebyshev parameter count (Sec. 3 per instance).  The
 * states are packed: instance i occupies 8 planes of nx[i]*ny[i] doubles at
 * U + 8 * offsets[i] (offsets from dim_batch_layout), the layout of dim_step
 * within that window.  One split step of every instance is one persistent
 * cooperative kernel launch; dim_batch_step captures it once into a CUDA graph
 * (per state pointer and launch configuration) and replays it.  Calls are
 * ordered on cuda_stream (the graph runs on a library stream joined to it with
 * events).  The paper's method per instance; batching has no counterpart in
 * the paper. */
typedef struct dim_batch dim_batch;
int dim_batch_init(dim_batch **out, const dim_params *p, int ninst, const int *nx, const int *ny, const double *dx,
                   const double *dy, void *cuda_stream);
void dim_batch_destroy(dim_batch *b);
/* offsets[0..ninst]: cell offset of each instance; offsets[ninst] = total cells */
int dim_batch_layout(const dim_batch *b, long long *offsets);
/* prim: 5 planes per instance (alpha_2, p, T, u, v) at prim + 5 * offsets[i] */
int dim_batch_from_primitive(dim_batch *b, const double *prim, double *U);
/* nsteps split steps of every instance, in place, asynchronous */
int dim_batch_step(dim_batch *b, double *U, int nsteps);
/* time every compiled tile-shape variant and block count on a copy of U and
 * keep the fastest; config (may be NULL) receives {variant, blocks, x-sweep
 * tile cells, x-sweep tile lines, y-sweep tile cells, y-sweep tile lines};
 * allocates a temporary copy of the state; synchronizes */
int dim_batch_autotune(dim_batch *b, const double *U, int *config);
/* per-instance status words (flags may be NULL) and their OR; synchronizes */
int dim_batch_status(dim_batch *b, unsigned *flags, unsigned *any);

/* Read (and clear if reset != 0) the device status word (DIM_ST_* bits);
 * synchronizes. */
int dim_status(dim_ctx *c, unsigned *flags, int reset);

/* Per-kernel timing with CUDA events on the context stream.  enable != 0 turns
 * it on (events around every launch), 0 off.  dim_kernel_time returns the
 * accumulated launches and milliseconds of kernel `name` ("sweep_x",
 * "sweep_y", "heat", "viscous_x", "viscous_y", "wave_max", "relax", "copy",
 * "convert": the FP64 <-> float-float state conversions of the FP32-bulk form)
 * since the last reset; synchronizes. */
int dim_profile(dim_ctx *c, int enable, int reset);
int dim_kernel_time(dim_ctx *c, const char *name, int *launches, double *ms);

/* Message of a return code. */
const char *dim_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* DIM_H */

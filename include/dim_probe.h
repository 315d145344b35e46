/*
 * dim_probe.h -- measurement and self-check entry points of libdim.so.
 *
 * The paper has no counterpart to anything in this header: these calls measure
 * the arithmetic rates of the GPU that the roofline of the split step is
 * quoted against, and expose the FP64 <-> float-float state conversion of the
 * FP32-bulk form for an elementwise check.
 * They use no dim_ctx.  Return codes are those of dim.h.
 */
#ifndef DIM_PROBE_H
#define DIM_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* probe kinds of dim_probe_rate */
#define DIM_PROBE_DFMA 0     /* FP64 fused multiply-add chains: 2 FLOP per operation */
#define DIM_PROBE_DADDMUL 1  /* FP64 add and multiply, alternating, never contracted: 1 FLOP each */
#define DIM_PROBE_DDIV 2     /* IEEE FP64 division (the compiler's correctly rounded sequence): 1 op each */
#define DIM_PROBE_DSQRT 3    /* IEEE FP64 square root: 1 op each */
#define DIM_PROBE_FFMA 4     /* FP32 fused multiply-add chains: 2 FLOP per operation */

/* Throughput of one kind of arithmetic: launches a kernel of `blocks` blocks of
 * 256 threads (blocks <= 0: 8 per SM), each thread running independent
 * dependency chains of the operation `iters` times (iters >= 1), on
 * cuda_stream (a cudaStream_t, NULL: legacy default stream), timed with CUDA
 * events on that stream.  Writes the device time in milliseconds to *ms and
 * the number of operations performed to *ops (FLOP for DFMA, DADDMUL, FFMA;
 * divisions / square roots for DDIV, DSQRT; each square root comes with one
 * multiply); rate = *ops / (*ms * 1e-3).
 * Synchronizes.  Errors: DIM_EINVAL (unknown kind, iters < 1, null outputs),
 * DIM_ECUDA. */
int dim_probe_rate(int kind, int blocks, int iters, void *cuda_stream, double *ms, double *ops);

/* Elementwise, n >= 0 elements of DEVICE arrays: y[i] = the FP64 value of the
 * float-float pair the FP32-bulk form converts x[i] to (the round trip of its
 * state conversion: a pair of floats holding the double's leading 47 bits,
 * formed and read back with integer operations).  Asynchronous on
 * cuda_stream.  Errors: DIM_EINVAL (n < 0, null pointers), DIM_ECUDA. */
int dim_probe_ff_roundtrip(const double *x, double *y, int n, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DIM_PROBE_H */

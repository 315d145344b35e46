// dim_probe.cu -- arithmetic-rate probes and the elementwise check of the
// FP32-bulk form's FP64 <-> float-float state conversion (include/dim_probe.h).
//
// A probe kernel runs, in every thread, NCH independent dependency chains of
// one operation (enough independent work per warp to cover the pipeline
// latency at 8 blocks of 256 threads per SM), so its duration is set by the
// issue rate of that operation's pipe.  Each thread writes the sum of its
// chains, which keeps the compiler from removing them.
#include <cuda_runtime.h>

#include "../../include/dim.h"
#include "../../include/dim_probe.h"
#include "dim_ff.cuh"

namespace {

constexpr int NCH = 8;
constexpr int TPB = 256;

template <int KIND>
__global__ void __launch_bounds__(TPB) k_probe(int iters, double a, double b, double *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == DIM_PROBE_FFMA) {
        float x[NCH];
        const float af = (float)a, bf = (float)b;
#pragma unroll
        for (int k = 0; k < NCH; k++) x[k] = 1.0f + 1e-3f * (float)(k + (t & 7));
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int k = 0; k < NCH; k++) x[k] = fmaf(x[k], af, bf);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < NCH; k++) s += x[k];
        out[t] = (double)s;
    } else {
        double x[NCH];
#pragma unroll
        for (int k = 0; k < NCH; k++) x[k] = 1.0 + 1e-3 * (double)(k + (t & 7));
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int k = 0; k < NCH; k++) {
                if constexpr (KIND == DIM_PROBE_DFMA) x[k] = fma(x[k], a, b);
                else if constexpr (KIND == DIM_PROBE_DADDMUL) x[k] = __dadd_rn(__dmul_rn(x[k], a), b);
                else if constexpr (KIND == DIM_PROBE_DDIV) x[k] = a / x[k];  // alternates between x0 and a/x0
                else x[k] = sqrt(x[k]) * a;  // DIM_PROBE_DSQRT: converges to a^2
            }
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NCH; k++) s += x[k];
        out[t] = s;
    }
}

__global__ void k_ff_roundtrip(const double *__restrict__ x, double *__restrict__ y, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = dimk::ff_to_d(dimk::ff_from_d(x[i]));
}

}  // namespace

extern "C" int dim_probe_rate(int kind, int blocks, int iters, void *cuda_stream, double *ms, double *ops)
{
    if (kind < DIM_PROBE_DFMA || kind > DIM_PROBE_FFMA || iters < 1 || !ms || !ops) return DIM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return DIM_ECUDA;
    if (blocks <= 0) blocks = 8 * nsm;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DIM_ECUDA;
    // operands: a contraction for the FMA chains (fixed point 1), a value for
    // the division and square-root chains that keeps them in the normal range
    double a = 0.999999, b = 1e-6;
    if (kind == DIM_PROBE_DDIV) a = 1.7;
    if (kind == DIM_PROBE_DSQRT) a = 1.3;
    if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * TPB) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaError_t e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            switch (kind) {
            case DIM_PROBE_DFMA: k_probe<DIM_PROBE_DFMA><<<blocks, TPB, 0, s>>>(iters, a, b, out); break;
            case DIM_PROBE_DADDMUL: k_probe<DIM_PROBE_DADDMUL><<<blocks, TPB, 0, s>>>(iters, a, b, out); break;
            case DIM_PROBE_DDIV: k_probe<DIM_PROBE_DDIV><<<blocks, TPB, 0, s>>>(iters, a, b, out); break;
            case DIM_PROBE_DSQRT: k_probe<DIM_PROBE_DSQRT><<<blocks, TPB, 0, s>>>(iters, a, b, out); break;
            default: k_probe<DIM_PROBE_FFMA><<<blocks, TPB, 0, s>>>(iters, a, b, out); break;
            }
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) {
            const double per_op = (kind == DIM_PROBE_DFMA || kind == DIM_PROBE_FFMA) ? 2.0 : 1.0;
            const double nop = kind == DIM_PROBE_DADDMUL ? 2.0 : 1.0;  // an add and a multiply per step
            *ms = (double)t;
            *ops = (double)blocks * TPB * (double)iters * NCH * nop * per_op;
            rc = DIM_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}

extern "C" int dim_probe_ff_roundtrip(const double *x, double *y, int n, void *cuda_stream)
{
    if (n < 0 || !x || !y) return DIM_EINVAL;
    if (n == 0) return DIM_OK;
    int g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_ff_roundtrip<<<g, 256, 0, (cudaStream_t)cuda_stream>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? DIM_OK : DIM_ECUDA;
}

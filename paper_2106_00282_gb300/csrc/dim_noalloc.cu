// dim_noalloc.cu -- a hyperbolic sweep that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// all device memory to their own pool allocator and forbid any other
// allocation, programs whose device-memory budget is fixed when they load, and
// loops for which the implicit device-wide synchronization of cudaMalloc /
// cudaFree is not acceptable.  dim_hllc_sweep needs a context from dim_init,
// which allocates its scratch.  dim_hllc_sweep_noalloc runs the same sweep
// kernel (same results) with its scratch -- the out-of-place copy of the state
// and the device status scalars -- in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/dim.h"
#include "dim_ff.cuh"

namespace dimk {
cudaError_t sweep_setup();
cudaError_t sweepff_setup();
cudaError_t launch_sweep(const DevParams &p, int axis, const double *Uin, double *Uout, double dt_host, Scalars *sc,
                         int relax, int check, cudaStream_t s);
FFP ffp_of(const DevParams &p);
cudaError_t launch_ff_in(const double *U, float2 *F, size_t m, cudaStream_t s);
cudaError_t launch_ff_out(const float2 *F, double *U, size_t m, cudaStream_t s);
cudaError_t launch_sweep_ff(const DevParams &p, const FFP &f, int axis, const float2 *Uin, float2 *Uout,
                            double dt_host, Scalars *sc, int relax, int check, cudaStream_t s);
}  // namespace dimk
int dim_host_params(const dim_params *hp, int nx, int ny, double dx, double dy, dimk::DevParams *out);

namespace {

// 8 planes of DIM_NOALLOC_MAX_CELLS doubles (the out-of-place sweep target)
// followed by the status scalars: 4 MiB + 512 B per device.
constexpr size_t kPlaneDoubles = (size_t)DIM_NOALLOC_MAX_CELLS;
constexpr size_t kScalarDoubles = 64;
static_assert(sizeof(dimk::Scalars) <= kScalarDoubles * sizeof(double), "scalar block too small");

static __device__ __align__(256) double g_noalloc_scratch[8 * kPlaneDoubles + kScalarDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
bool g_ready[kMaxDevices];

// once per device, with that device current: the device address of the array
// (the host-side name is only a stand-in) and the shared-memory attribute of
// the sweep kernels of both precisions
int setup_current_device(double **scratch)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DIM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return DIM_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_ready[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return DIM_ECUDA;
        if (dimk::sweep_setup() != cudaSuccess || dimk::sweepff_setup() != cudaSuccess) return DIM_ECUDA;
        g_scratch_ptr[dev] = (double *)ptr;
        g_ready[dev] = true;
    }
    *scratch = g_scratch_ptr[dev];
    return DIM_OK;
}

}  // namespace

extern "C" int dim_hllc_sweep_noalloc(const dim_params *p, int nx, int ny, double dx, double dy, double *U, int axis,
                                      double dt, int relax, void *cuda_stream)
{
    if (!p || !U || (axis != 0 && axis != 1) || !(dt > 0.0)) return DIM_EINVAL;
    dimk::DevParams dp;
    int r = dim_host_params(p, nx, ny, dx, dy, &dp);
    if (r != DIM_OK) return r;
    if ((size_t)nx * (size_t)ny > kPlaneDoubles) return DIM_ETOOLARGE;
    double *scratch = nullptr;
    r = setup_current_device(&scratch);
    if (r != DIM_OK) return r;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *Uout = scratch;
    dimk::Scalars *sc = (dimk::Scalars *)(scratch + 8 * kPlaneDoubles);
    // the array keeps the previous call's contents: the status scalars start at zero
    if (cudaMemsetAsync(sc, 0, sizeof(dimk::Scalars), s) != cudaSuccess) return DIM_ECUDA;
    const size_t m = 8 * (size_t)dp.n;
    if (dp.precision == DIM_PRECISION_FP32_BULK) {
        // the FP32-bulk sweep of dim_hllc_sweep: the state converted to
        // float-float planes in the array, swept into U's own memory (8 planes
        // of float pairs take the bytes of 8 planes of doubles), converted back
        // in place
        float2 *F = (float2 *)scratch;
        const dimk::FFP f = dimk::ffp_of(dp);
        if (dimk::launch_ff_in(U, F, m, s) != cudaSuccess ||
            dimk::launch_sweep_ff(dp, f, axis, F, (float2 *)U, dt, sc, relax, 0, s) != cudaSuccess ||
            dimk::launch_ff_out((const float2 *)U, U, m, s) != cudaSuccess)
            return DIM_ECUDA;
        return DIM_OK;
    }
    if (dimk::launch_sweep(dp, axis, U, Uout, dt, sc, relax, 0, s) != cudaSuccess) return DIM_ECUDA;
    if (cudaMemcpyAsync(U, Uout, sizeof(double) * m, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return DIM_ECUDA;
    return DIM_OK;
}

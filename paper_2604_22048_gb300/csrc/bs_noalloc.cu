// bs_shear_loglike_noalloc: the shear likelihood for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs under a fixed device-memory budget owned by another framework,
// real-time loops that must not allocate between iterations, or a sampler
// embedded in a host program with no allocator of its own.  This entry point
// runs the same kernels as bs_shear_loglike, but keeps their scratch -- four
// FP64 partials (value, d/dg1, d/dg2, sum of weighted |eps|^2) per thread
// block of the reduction -- in a file-scope device array instead of a
// caller workspace.
//
// The array is static device data of this library: every GPU that loads the
// library holds it (64 KB) until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device looks up
// the address with cudaGetSymbolAddress (with that device current) and caches
// it for the life of the process; make that first call before any stream
// capture.  A cudaDeviceReset unloads the library's device data, so the
// cached address does not survive it: the entry point must not be called on
// a device after its reset.  Every call shares the array and it keeps the
// last call's contents: each launch writes every slot it later reads, so
// nothing has to start at zero, but calls that overlap on the GPU (on
// different streams, or from different host threads without ordering) race
// on it.
#include <mutex>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace {

constexpr int kNoAllocBlocks = 2048;                       // partial slots
constexpr int kNoAllocDoubles = kNoAllocBlocks * 4 + 4;   // + the 4 finalize outputs
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
bs_status scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return bs::set_error(BS_ERR_CUDA, "bs_shear_loglike_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return bs::set_error(BS_ERR_UNSUPPORTED, "bs_shear_loglike_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return bs::set_error(BS_ERR_CUDA, "bs_shear_loglike_noalloc: cudaGetSymbolAddress: %s",
                                 cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return BS_OK;
}

}  // namespace

extern "C" bs_status bs_shear_loglike_noalloc(const bs_shear_data *data, double g1, double g2,
                                              double alpha, double *out, void *stream)
{
    bs::ShearLaunch L;
    double add[4], alpha_scale = 1.0;
    bs_status st = bs::shear_prepare(data, g1, g2, alpha, L, add, alpha_scale, "bs_shear_loglike_noalloc");
    if (st != BS_OK) return st;
    if (!out) return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_loglike_noalloc: NULL out");
    const int grid = bs::shear_grid_blocks();
    if (grid > kNoAllocBlocks)
        return bs::set_error(BS_ERR_UNSUPPORTED,
                             "bs_shear_loglike_noalloc: this device needs %d partial slots, the static "
                             "scratch holds %d; use bs_shear_loglike with a workspace",
                             grid, kNoAllocBlocks);
    double *scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != BS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (data->n_gal > 0) {
        L.partials = scratch;
        e = bs::launch_shear(L, grid, s);
        if (e != cudaSuccess)
            return bs::set_error(BS_ERR_CUDA, "bs_shear_loglike_noalloc: launch: %s", cudaGetErrorString(e));
        bs::count_launches(1);
    }
    e = bs::launch_shear_finalize(scratch, data->n_gal > 0 ? grid : 0, add[0], add[1], add[2], add[3],
                                  alpha_scale, out, s);
    if (e != cudaSuccess)
        return bs::set_error(BS_ERR_CUDA, "bs_shear_loglike_noalloc: finalize: %s", cudaGetErrorString(e));
    bs::count_launches(1);
    return BS_OK;
}

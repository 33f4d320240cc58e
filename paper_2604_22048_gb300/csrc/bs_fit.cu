// Launches of the image-sampling kernels of bs_fit_impl.cuh: the instance is
// chosen by the column slots per lane of the largest stamp (smaller stamps of
// the same launch see zero-padded columns), the register budget and the
// galaxy profile.  The exponential instances live here; the Spergel and
// Gaussian ones (Appendix B) in bs_fit_prof.cu, compiled in parallel.
#include "bs_fit_impl.cuh"

namespace bs {

namespace {

using FitKernel = void (*)(const FitParams);

#define BS_FIT_NC_SWITCH(KERNEL)                 \
    switch ((max_side + 31) / 32) {              \
        case 1: return KERNEL<1, 0>;             \
        case 2: return KERNEL<2, 0>;             \
        case 3: return KERNEL<3, 0>;             \
        default: return KERNEL<4, 0>;            \
    }

// Register budget of a launch (128, 96 or 80; 96 only for blocks of up to 4
// chains); 0 takes 128.  The library is built without implicit multiply-add
// contraction, so the three instances round alike and give the same chains.
FitKernel fit_kernel_for(int max_side, int regs, int n_chains)
{
    if (regs != 128 && regs != 96 && regs != 80) regs = 128;
    if (regs == 96 && n_chains > 4) regs = 128;
    if (regs == 80) BS_FIT_NC_SWITCH(fit_kernel_r80)
    if (regs == 96) BS_FIT_NC_SWITCH(fit_kernel_r96)
    BS_FIT_NC_SWITCH(fit_kernel_r128)
}

#undef BS_FIT_NC_SWITCH

}  // namespace

size_t fit_smem_bytes(int max_side, int n_chains)
{
    const int h = (max_side + 1) / 2;
    const int npad = 32 * ((max_side + 31) / 32);
    return (size_t)h * row_floats(npad) * sizeof(float) +
           (size_t)scratch_float2(max_side, h, n_chains) * sizeof(float2) + (size_t)(h + 1) * sizeof(float2);
}

int fit_blocks_per_sm(int n_chains, int max_side, int regs, int profile)
{
    if (profile != 0) return fit_blocks_per_sm_profile(profile, n_chains, max_side);
    int nb = 0;
    const size_t smem = fit_smem_bytes(max_side, n_chains);
    FitKernel k = fit_kernel_for(max_side, regs, n_chains);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * n_chains, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_fit(const FitParams &p, int grid, cudaStream_t stream)
{
    if (p.profile != 0) return launch_fit_profile(p, grid, stream);
    const int cc = cta_chains(p);
    const size_t smem = fit_smem_bytes(p.max_side, cc);
    FitKernel k = fit_kernel_for(p.max_side, p.regs, cc);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * cc, smem, stream>>>(p);
    bs::count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_logpost_points(const FitParams &p, int n_points, const int32_t *gal_index,
                                  const float *theta, double *logp, float *grad,
                                  cudaStream_t stream)
{
    if (p.profile != 0) return launch_logpost_points_profile(p, n_points, gal_index, theta, logp, grad, stream);
    const size_t smem = fit_smem_bytes(p.max_side, 1);
    cudaError_t e = cudaFuncSetAttribute(logpost_points_kernel<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n_points < 4096 ? n_points : 4096;
    if (grid <= 0) return cudaSuccess;
    logpost_points_kernel<0><<<grid, 32, smem, stream>>>(p, n_points, gal_index, theta, logp, grad);
    bs::count_launches(1);
    return cudaGetLastError();
}

}  // namespace bs

// Spergel and Gaussian galaxy profiles of the image-sampling kernels
// (Appendix B: the forward model with a Spergel profile of fixed index nu, or
// a Gaussian), compiled apart from the exponential instances of bs_fit.cu.
#include <cmath>

#include "bs_fit_impl.cuh"

namespace bs {

namespace {

using FitKernel = void (*)(const FitParams);
using PointsKernel = void (*)(const FitParams, int, const int32_t *, const float *, double *, float *);

template <int PROF>
FitKernel prof_kernel(int max_side)
{
    switch ((max_side + 31) / 32) {
        case 1: return fit_kernel_r128<1, PROF>;
        case 2: return fit_kernel_r128<2, PROF>;
        case 3: return fit_kernel_r128<3, PROF>;
        default: return fit_kernel_r128<4, PROF>;
    }
}

// Per-pixel weights (profile 3), exponential: stamps of at most 63 px, two chains
// per CTA of eight warps, the transforms on the tensor cores.
FitKernel pix_kernel(int max_side)
{
    return max_side <= 31 ? fit_kernel_pix<1> : fit_kernel_pix<2>;
}

constexpr int kPixThreads = tc::kThreads;

bool is_pix(int profile) { return profile == 3; }

FitKernel kernel_for(int profile, int max_side)
{
    if (profile == 3) return pix_kernel(max_side);
    if (profile == 4) return fit_kernel_r128<1, 4>;   // a dense covariance: at most 31 px
    return profile == BS_PROFILE_SPERGEL ? prof_kernel<1>(max_side) : prof_kernel<2>(max_side);
}

PointsKernel points_for(int profile, int max_side)
{
    if (is_pix(profile)) return max_side <= 31 ? logpost_points_pix_kernel<1> : logpost_points_pix_kernel<2>;
    if (profile == 4) return logpost_points_kernel<4>;
    return profile == BS_PROFILE_SPERGEL ? logpost_points_kernel<1> : logpost_points_kernel<2>;
}

// Dynamic shared memory of a launch: the pixel-weight path adds the transforms'
// region after the row table, the dense-covariance path its twiddles and
// per-chain scratch.
size_t smem_for(int profile, int max_side, int n_chains)
{
    if (is_pix(profile)) {
        const int h = (max_side + 1) / 2, npad = 32 * ((max_side + 31) / 32);
        return fit_smem_bytes(max_side, 2) + 16 + pix_tc_bytes(max_side, h, npad);
    }
    size_t b = fit_smem_bytes(max_side, n_chains);
    if (profile == 4) {
        const int h = (max_side + 1) / 2, npad = 32 * ((max_side + 31) / 32);
        b += 16 + dense_region_bytes(h, npad, max_side, n_chains);
    }
    return b;
}

int threads_for(int profile, int n_chains) { return is_pix(profile) ? kPixThreads : 32 * n_chains; }

// K_mu(x) = int_0^inf exp(-x cosh t) cosh(mu t) dt by the trapezoidal rule
// (step 1/64; the integrand falls off doubly exponentially).
double bessel_k(double mu, double x)
{
    const double h = 1.0 / 64.0;
    double sum = 0.5 * std::exp(-x);
    for (int j = 1; j < 4096; ++j) {
        const double t = j * h;
        const double term = std::exp(-x * std::cosh(t)) * std::cosh(mu * t);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum * h;
}

}  // namespace

double profile_hlr_over_r0(int profile, double nu)
{
    if (profile == BS_PROFILE_GAUSSIAN) return std::sqrt(2.0 * std::log(2.0));
    if (profile != BS_PROFILE_SPERGEL) return 1.6783469900166608;
    // enclosed flux of the Spergel profile, 1 - x^(1+nu) K_(1+nu)(x) / (2^nu Gamma(1+nu)),
    // increases from 0 to 1: bisect for 1/2
    const double norm = std::pow(2.0, nu) * std::tgamma(1.0 + nu);
    auto enclosed = [&](double x) { return 1.0 - std::pow(x, 1.0 + nu) * bessel_k(1.0 + nu, x) / norm; };
    double lo = 1e-6, hi = 50.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (enclosed(mid) < 0.5) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

int fit_blocks_per_sm_profile(int profile, int n_chains, int max_side)
{
    int nb = 0;
    const size_t smem = smem_for(profile, max_side, n_chains);
    FitKernel k = kernel_for(profile, max_side);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads_for(profile, n_chains), smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_fit_profile(const FitParams &p, int grid, cudaStream_t stream)
{
    const int cc = cta_chains(p);
    const size_t smem = smem_for(p.profile, p.max_side, cc);
    FitKernel k = kernel_for(p.profile, p.max_side);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads_for(p.profile, cc), smem, stream>>>(p);
    bs::count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_logpost_points_profile(const FitParams &p, int n_points, const int32_t *gal_index,
                                          const float *theta, double *logp, float *grad, cudaStream_t stream)
{
    const size_t smem = smem_for(p.profile, p.max_side, 1);
    PointsKernel k = points_for(p.profile, p.max_side);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n_points < 4096 ? n_points : 4096;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, is_pix(p.profile) ? kPixThreads : 32, smem, stream>>>(p, n_points, gal_index, theta, logp, grad);
    bs::count_launches(1);
    return cudaGetLastError();
}

}  // namespace bs

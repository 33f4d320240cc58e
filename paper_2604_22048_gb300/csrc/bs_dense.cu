// Appendix C with a general pixel covariance Sigma (Eq. covar-pixel-likelihood):
// the fit needs its inverse, the precision P = Sigma^-1, once per galaxy.
// One CTA per galaxy computes it in FP64 in a scratch of its own:
//   L = chol(Sigma)           right-looking, one column per step;
//   W = L^-1                  one thread per column, forward substitution;
//   P = W^T W                 one thread per entry of the lower triangle;
// and stores P (symmetric, both triangles) as FP32 in the galaxy's block.
// About n^3 / 2 FP64 multiply-adds for n = N^2 pixels: tens of milliseconds
// per galaxy at 31 px, once per fit.
#include <cmath>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace bs {

namespace {

constexpr int kDenseThreads = 256;

__global__ void __launch_bounds__(kDenseThreads) dense_precision_kernel(int n_gal, const int32_t *side,
                                                                        int max_side, const float *cov,
                                                                        const int64_t *offs,
                                                                        float *prec, int32_t *status,
                                                                        double *scratch, size_t scratch_per_cta)
{
    __shared__ double col[kDenseMaxSide * kDenseMaxSide];   // the pivot column below the diagonal
    double *A = scratch + (size_t)blockIdx.x * scratch_per_cta;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarp = nth >> 5;
    for (int gal = blockIdx.x; gal < n_gal; gal += gridDim.x) {
        const int N = side[gal];
        if (N < 3 || N > max_side || !(N & 1)) {      // the scratch holds max_side only
            if (tid == 0 && status) status[gal] = 2;
            continue;
        }
        const int n = N * N;
        double *Wm = A + (size_t)n * n;
        const float *S = cov + offs[gal];
        float *Pout = prec + offs[gal];
        for (size_t i = tid; i < (size_t)n * n; i += nth) A[i] = (double)S[i];
        __syncthreads();
        // Cholesky of the lower triangle of A (row-major), one column per step
        bool bad = false;
        for (int j = 0; j < n; ++j) {
            const double d = A[(size_t)j * n + j];       // the same value in every thread
            if (!(d > 0.0)) {
                bad = true;
                break;
            }
            const double rd = 1.0 / sqrt(d);
            for (int i = j + 1 + tid; i < n; i += nth) col[i] = A[(size_t)i * n + j] * rd;
            __syncthreads();
            if (tid == 0) A[(size_t)j * n + j] = d * rd;
            for (int i = j + 1 + tid; i < n; i += nth) A[(size_t)i * n + j] = col[i];
            // trailing update: rows i > j over warps, columns j < k <= i over lanes
            for (int i = j + 1 + warp; i < n; i += nwarp) {
                const double ci = col[i];
                double *row = A + (size_t)i * n;
                for (int k = j + 1 + lane; k <= i; k += 32) row[k] -= ci * col[k];
            }
            __syncthreads();
        }
        if (bad) {
            if (tid == 0 && status) status[gal] = 3;
            for (size_t i = tid; i < (size_t)n * n; i += nth) Pout[i] = 0.0f;
            __syncthreads();
            continue;
        }
        // W = L^-1, column c by thread c:
        //   W[i][c] = (delta_ic - sum_{c <= k < i} L[i][k] W[k][c]) / L[i][i]
        for (int c = tid; c < n; c += nth) {
            for (int i = 0; i < c; ++i) Wm[(size_t)i * n + c] = 0.0;
            for (int i = c; i < n; ++i) {
                double s = i == c ? 1.0 : 0.0;
                const double *Li = A + (size_t)i * n;
                for (int k = c; k < i; ++k) s -= Li[k] * Wm[(size_t)k * n + c];
                Wm[(size_t)i * n + c] = s / Li[i];
            }
        }
        __syncthreads();
        // P = W^T W: P[a][b] = sum_{k >= a} W[k][a] W[k][b] for b <= a (W lower
        // triangular), rows a over warps, columns b over lanes
        for (int a = warp; a < n; a += nwarp) {
            for (int b = lane; b <= a; b += 32) {
                double s = 0.0;
                for (int k = a; k < n; ++k) s += Wm[(size_t)k * n + a] * Wm[(size_t)k * n + b];
                Pout[(size_t)a * n + b] = (float)s;
                Pout[(size_t)b * n + a] = (float)s;
            }
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace bs

extern "C" {

size_t bs_dense_precision_workspace_bytes(int32_t max_side)
{
    if (max_side < 3 || max_side > bs::kDenseMaxSide || !(max_side & 1)) return 0;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t n = (size_t)max_side * max_side;
    return (size_t)sms * 2 * n * n * sizeof(double);
}

bs_status bs_dense_precision(int32_t n_gal, const int32_t *side, int32_t max_side, const float *cov,
                             const int64_t *cov_offsets, float *prec, int32_t *status, void *workspace,
                             size_t workspace_bytes, void *stream)
{
    if (n_gal < 0) return bs::set_error(BS_ERR_INVALID_ARG, "bs_dense_precision: n_gal < 0");
    if (n_gal == 0) return BS_OK;
    if (!side || !cov || !cov_offsets || !prec)
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_dense_precision: NULL input or output");
    if (max_side < 3 || max_side > bs::kDenseMaxSide || !(max_side & 1))
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_dense_precision: max_side must be odd, 3..%d",
                             bs::kDenseMaxSide);
    const size_t need = bs_dense_precision_workspace_bytes(max_side);
    if (!workspace || workspace_bytes < need)
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_dense_precision: workspace of %zu bytes needed", need);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_gal < sms ? n_gal : sms;
    const size_t n = (size_t)max_side * max_side;
    bs::dense_precision_kernel<<<grid, bs::kDenseThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_gal, side, max_side, cov, cov_offsets, prec, status, static_cast<double *>(workspace), 2 * n * n);
    bs::count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return bs::set_error(BS_ERR_CUDA, "bs_dense_precision: launch: %s", cudaGetErrorString(e));
    return BS_OK;
}

}  // extern "C"

// Chain diagnostics on sm_103a (Sec. 4.1): per galaxy and parameter, the
// classic potential scale reduction R-hat (Gelman & Rubin 1992) and the
// multi-chain effective sample size with Geyer's initial monotone positive
// sequence (Gelman et al., BDA3 Sec. 11.5):
//   var+ = (n-1)/n W + B/n,  rho_t = 1 - (W - mean_c acov_c(t)) / var+,
//   tau = -1 + 2 sum_k P_k (P_k = rho_2k + rho_2k+1 while positive, made
//   monotone), ESS = m n / tau with tau >= 1 / log10(m n).
// One warp per (galaxy, parameter); autocovariances by direct lane-parallel
// sums, computed pairwise only until the sequence stops.
#include <cmath>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace bs {

namespace {

__global__ void __launch_bounds__(128) ess_kernel(const float *samples, int n_gal, int C, int S,
                                                  float *ess, float *rhat)
{
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)n_gal * 6) return;
    const int gal = (int)(wid / 6), k = (int)(wid % 6);
    const float *x = samples + (((size_t)k * n_gal + gal) * C) * S;
    float mean[kMaxChains];
    float wsum = 0.f, mbar = 0.f;
    for (int c = 0; c < C; ++c) {
        const float *xc = x + (size_t)c * S;
        float s = 0.f;
        for (int i = lane; i < S; i += 32) s += xc[i];
        s = warp_sum(s) / (float)S;
        float v = 0.f;
        for (int i = lane; i < S; i += 32) {
            const float d = xc[i] - s;
            v = fmaf(d, d, v);
        }
        v = warp_sum(v) / (float)(S - 1);
        mean[c] = s;
        wsum += v;
        mbar += s;
    }
    const float W = wsum / C;
    mbar /= C;
    float bn = 0.f;
    if (C > 1) {
        for (int c = 0; c < C; ++c) bn += (mean[c] - mbar) * (mean[c] - mbar);
        bn /= (C - 1);
    }
    const float vp = (S - 1.0f) / S * W + bn;
    auto rho = [&](int t) -> float {
        float a = 0.f;
        for (int c = 0; c < C; ++c) {
            const float *xc = x + (size_t)c * S;
            float s = 0.f;
            for (int i = lane; i + t < S; i += 32) s = fmaf(xc[i] - mean[c], xc[i + t] - mean[c], s);
            a += warp_sum(s) / (float)S;
        }
        a /= C;
        return 1.0f - (W - a) / vp;
    };
    float sum = 0.f, prev = INFINITY;
    for (int kk = 0; 2 * kk + 1 < S; ++kk) {
        const float r0 = (kk == 0) ? 1.0f : rho(2 * kk);
        const float P = r0 + rho(2 * kk + 1);
        if (!(P > 0.f)) break;
        const float Pm = P > prev ? prev : P;
        sum += Pm;
        prev = Pm;
    }
    float tau = -1.0f + 2.0f * sum;
    const float tmin = 1.0f / log10f((float)C * S);
    if (tau < tmin) tau = tmin;
    if (lane == 0) {
        ess[(size_t)gal * 6 + k] = (float)C * S / tau;
        if (rhat) rhat[(size_t)gal * 6 + k] = sqrtf(vp / W);
    }
}

}  // namespace

cudaError_t launch_chain_ess(const float *samples, int n_gal, int n_chains, int n_samples,
                             float *ess, float *rhat, cudaStream_t stream)
{
    const long long warps = (long long)n_gal * 6;
    if (warps == 0) return cudaSuccess;
    const long long blocks = (warps + 3) / 4;
    ess_kernel<<<(unsigned)blocks, 128, 0, stream>>>(samples, n_gal, n_chains, n_samples, ess, rhat);
    return cudaGetLastError();
}

}  // namespace bs

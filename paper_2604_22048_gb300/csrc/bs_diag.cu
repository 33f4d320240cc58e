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

// FP32 FMA throughput: eight independent chains per thread of x = x a + b on
// float pairs, as scalar FFMA or as packed FFMA2 (16 FMAs per iteration either
// way); the sum is stored so the chains are not removed.
template <bool PACKED>
__global__ void __launch_bounds__(256) ffma_kernel(float *out, int iters, float a, float b)
{
    float2 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float2(1e-3f * (float)threadIdx.x + (float)i, 0.5f * (float)i);
    const float2 av = make_float2(a, a), bv = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (PACKED) {
                x[i] = __ffma2_rn(x[i], av, bv);
            } else {
                x[i].x = fmaf(x[i].x, a, b);
                x[i].y = fmaf(x[i].y, a, b);
            }
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += x[i].x + x[i].y;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// FP64 FMA throughput: sixteen independent DFMA chains per thread.
__global__ void __launch_bounds__(256) dfma_kernel(float *out, int iters, double a, double b)
{
    double x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = 1e-3 * (double)threadIdx.x + (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = fma(x[i], a, b);
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) sum += x[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (float)sum;
}

}  // namespace

cudaError_t measure_fma_peak(int kind, double &tflops, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = sms * 8, block = 256, iters = kind == 2 ? 512 : 16384;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMallocAsync(&out, sizeof(float) * (size_t)grid * block, stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, stream);
        if (kind == 1)
            ffma_kernel<true><<<grid, block, 0, stream>>>(out, iters, 1.0000001f, 1e-7f);
        else if (kind == 2)
            dfma_kernel<<<grid, block, 0, stream>>>(out, iters, 1.0000000001, 1e-10);
        else
            ffma_kernel<false><<<grid, block, 0, stream>>>(out, iters, 1.0000001f, 1e-7f);
        count_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (out) cudaFreeAsync(out, stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 16.0 * (double)iters * grid * block;
    tflops = flops / (best * 1e-3) / 1e12;
    return cudaStreamSynchronize(stream);
}

cudaError_t launch_chain_ess(const float *samples, int n_gal, int n_chains, int n_samples,
                             float *ess, float *rhat, cudaStream_t stream)
{
    const long long warps = (long long)n_gal * 6;
    if (warps == 0) return cudaSuccess;
    const long long blocks = (warps + 3) / 4;
    ess_kernel<<<(unsigned)blocks, 128, 0, stream>>>(samples, n_gal, n_chains, n_samples, ess, rhat);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bs

// Shear sampling phase on sm_103a (Sec. 3.2): one streaming pass over the
// interim samples evaluates Eq. likelihood-shear and its gradient.
//
// Per sample, with eps = (eps' - g)/(1 - g* eps') (inverse of
// Eq. shear-transform), U = |1 - g* eps'|^2, Q = |eps|^2 = |eps' - g|^2 / U and
// the identity 1 - |eps|^2 = (1 - |g|^2)(1 - |eps'|^2) / U, the log weight
// log p_e(eps | alpha) + log|d eps/d eps'| - log P0_e(eps') + b splits into a
// per-galaxy constant and
//   x = -kappa ln U - Q / (2 alpha^2) + |eps'|^2 / (2 sigma_e0^2)
//       [- 2 ln(1 - |eps'|^2) for the truncated Gaussian] + b,
// kappa = 4 for the (1-|e|^2)^2 exp(-|e|^2/2 alpha^2) family (2 from that
// factor, 2 from the Jacobian (1-|g|^2)^2 / U^2 of
// Eq. true-prior-jacobian-shear) and 2 for the truncated Gaussian.  Its
// derivatives are dx/dg_i = (-2/U) [du_i (Q/(2 alpha^2) - kappa) - n_i/(2 alpha^2)]
// with du_1 = ur e1 - vi e2, du_2 = ur e2 + vi e1, n = eps' - g, and
// dx/dalpha = Q / alpha^3.
//
// Each galaxy's K samples are read by a group of 8 lanes (float4 loads when
// the rows are 16-byte aligned, one chunk ahead of the arithmetic), x is kept in log2 units for the MUFU exp2, and the group keeps
// an online log-sum-exp (running max, sum of weights and weighted derivative
// sums), merged with shuffles.  Per-galaxy totals are
// accumulated in FP64 and written as per-block partials; a one-block kernel
// sums the partials in a fixed order (deterministic) and adds the
// per-galaxy constants.
#include <cmath>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace bs {

namespace {

constexpr int kGroup = 8;          // lanes per galaxy
constexpr int kShearThreads = 256;

// Hardware approximations with denormal flushing.  Their arguments here are
// normal numbers (U in (0, 4], 1 - |eps'|^2 >= 2^-24, sums of weights >= 1),
// or, for ex2, non-positive differences whose flushed results are weights
// below 2^-126 of the largest; so no range fix-ups are needed around them.
__device__ __forceinline__ float ex2_ftz(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_ftz(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per sample: log2 weight x and the factors of its derivatives,
//   dx/dg_i = -2 rU c_i,  c_i = du_i (Q/(2 alpha^2) - kappa) - n_i/(2 alpha^2),
// returned as (rU, c1, c2, Q); the -2 is applied once per galaxy.
template <int FAMILY, bool HAS_B>
__device__ __forceinline__ void sample_terms(const ShearLaunch &s, float a_nat, float e1, float e2,
                                             float bv, float &x2, float &ru, float &c1, float &c2,
                                             float &q)
{
    const float ur = fmaf(-s.g1, e1, fmaf(-s.g2, e2, 1.0f));
    const float vi = fmaf(s.g1, e2, -s.g2 * e1);
    const float U = fmaf(ur, ur, vi * vi);
    const float n1 = e1 - s.g1, n2 = e2 - s.g2;
    const float Nn = fmaf(n1, n1, n2 * n2);
    const float rU = rcp_ftz(U);
    const float Q = Nn * rU;
    const float Ep = fmaf(e1, e1, e2 * e2);
    float x = fmaf(s.c0, Ep, fmaf(-s.kappa, lg2_ftz(U), -s.a2 * Q));
    if (FAMILY == BS_EPRIOR_TRUNC_GAUSS) {
        x = fmaf(-2.0f, lg2_ftz(1.0f - Ep), x);
        if (!(Q < s.r2)) x = -INFINITY;
    }
    if (HAS_B) x = fmaf(kLog2e, bv, x);
    const float aqk = fmaf(a_nat, Q, -s.kappa);
    const float du1 = fmaf(ur, e1, -vi * e2);
    const float du2 = fmaf(ur, e2, vi * e1);
    c1 = fmaf(du1, aqk, -a_nat * n1);
    c2 = fmaf(du2, aqk, -a_nat * n2);
    ru = rU;
    q = Q;
    x2 = x;
}

// Loads of one chunk (4 consecutive samples of this lane).
template <bool HAS_B, bool VEC>
__device__ __forceinline__ void load_chunk(const ShearLaunch &s, long long base, int k0, int K, float (&ex)[4],
                                           float (&ey)[4], float (&eb)[4], bool (&valid)[4])
{
    if (VEC) {
        if (k0 < K) {
            const float4 v1 = __ldg(reinterpret_cast<const float4 *>(s.e1 + base + k0));
            const float4 v2 = __ldg(reinterpret_cast<const float4 *>(s.e2 + base + k0));
            ex[0] = v1.x; ex[1] = v1.y; ex[2] = v1.z; ex[3] = v1.w;
            ey[0] = v2.x; ey[1] = v2.y; ey[2] = v2.z; ey[3] = v2.w;
            if (HAS_B) {
                const float4 vb = __ldg(reinterpret_cast<const float4 *>(s.b + base + k0));
                eb[0] = vb.x; eb[1] = vb.y; eb[2] = vb.z; eb[3] = vb.w;
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) valid[r] = k0 < K;
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            valid[r] = k0 + r < K;
            if (valid[r]) {
                const long long j = base + k0 + r;
                ex[r] = __ldg(s.e1 + j);
                ey[r] = __ldg(s.e2 + j);
                eb[r] = HAS_B ? __ldg(s.b + j) : 0.f;
            }
        }
    }
}

template <int FAMILY, bool HAS_B, bool VEC>
__global__ void __launch_bounds__(kShearThreads, 4) shear_kernel(const ShearLaunch s)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kGroup - 1);
    const unsigned gmask = 0xFFu << (lane & ~(kGroup - 1));
    const long long group = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    const long long ngroups = (long long)gridDim.x * blockDim.x / kGroup;
    const float a_nat = s.a2 * kLn2;    // 1 / (2 alpha^2)
    const int K = s.K;
    double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;

    for (long long n = group; n < s.n_gal; n += ngroups) {
        const long long base = n * (long long)K;
        float m = -1e30f, sw = 0.f, t1 = 0.f, t2 = 0.f, tq = 0.f;
        // software pipelined: the next chunk's loads are in flight while the
        // current chunk is evaluated
        float ex[4] = {0.f, 0.f, 0.f, 0.f}, ey[4] = {0.f, 0.f, 0.f, 0.f}, eb[4] = {0.f, 0.f, 0.f, 0.f};
        bool valid[4];
        int k0 = 4 * sub;
        load_chunk<HAS_B, VEC>(s, base, k0, K, ex, ey, eb, valid);
        while (k0 < K) {
            float cx[4], cy[4], cb[4];
            bool cv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cx[r] = ex[r];
                cy[r] = ey[r];
                cb[r] = eb[r];
                cv[r] = valid[r];
            }
            k0 += 4 * kGroup;
            load_chunk<HAS_B, VEC>(s, base, k0, K, ex, ey, eb, valid);
            float x[4], ru[4], c1[4], c2[4], qq[4];
            float mloc = m;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sample_terms<FAMILY, HAS_B>(s, a_nat, cx[r], cy[r], HAS_B ? cb[r] : 0.f, x[r], ru[r], c1[r],
                                            c2[r], qq[r]);
                if (!cv[r]) x[r] = -INFINITY;
                mloc = fmaxf(mloc, x[r]);
            }
            if (mloc > m) {          // rescale only when the running maximum rises
                const float sc = ex2_ftz(m - mloc);
                sw *= sc;
                t1 *= sc;
                t2 *= sc;
                tq *= sc;
                m = mloc;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float e = ex2_ftz(x[r] - m);
                const float er = e * ru[r];
                sw += e;
                t1 = fmaf(er, c1[r], t1);
                t2 = fmaf(er, c2[r], t2);
                tq = fmaf(e, qq[r], tq);
            }
        }
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) {
            const float mo = __shfl_xor_sync(gmask, m, o, kGroup);
            const float so = __shfl_xor_sync(gmask, sw, o, kGroup);
            const float o1 = __shfl_xor_sync(gmask, t1, o, kGroup);
            const float o2 = __shfl_xor_sync(gmask, t2, o, kGroup);
            const float oq = __shfl_xor_sync(gmask, tq, o, kGroup);
            const float mn = fmaxf(m, mo);
            const float ca = ex2_ftz(m - mn), cb = ex2_ftz(mo - mn);
            sw = sw * ca + so * cb;
            t1 = t1 * ca + o1 * cb;
            t2 = t2 * ca + o2 * cb;
            tq = tq * ca + oq * cb;
            m = mn;
        }
        if (sub == 0) {
            if (sw > 0.f) {
                const float inv = 1.0f / sw;
                av += (double)m + (double)__log2f(sw);
                a1 += (double)(-2.0f * t1 * inv);
                a2 += (double)(-2.0f * t2 * inv);
                aq += (double)(tq * inv);
            } else {
                av = -INFINITY;
            }
        }
    }
    // block reduction in FP64
    __shared__ double red[kShearThreads / 32][4];
    av = warp_sum_d(av);
    a1 = warp_sum_d(a1);
    a2 = warp_sum_d(a2);
    aq = warp_sum_d(aq);
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        red[w][0] = av;
        red[w][1] = a1;
        red[w][2] = a2;
        red[w][3] = aq;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int i = 0; i < kShearThreads / 32; ++i) t += red[i][threadIdx.x];
        s.partials[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) shear_finalize_kernel(const double *partials, int n_part,
                                                              double add_value, double add_g1,
                                                              double add_g2, double add_alpha,
                                                              double alpha_scale, double *out)
{
    __shared__ double red[256][4];
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n_part; i += blockDim.x)
        for (int k = 0; k < 4; ++k) t[k] += partials[(size_t)i * 4 + k];
    for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = t[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + o][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0] * 0.6931471805599453 + add_value;
        out[1] = red[0][1] + add_g1;
        out[2] = red[0][2] + add_g2;
        out[3] = red[0][3] * alpha_scale + add_alpha;
    }
}

template <int FAMILY, bool HAS_B>
cudaError_t launch_fb(const ShearLaunch &s, int grid, bool vec, cudaStream_t st)
{
    if (vec)
        shear_kernel<FAMILY, HAS_B, true><<<grid, kShearThreads, 0, st>>>(s);
    else
        shear_kernel<FAMILY, HAS_B, false><<<grid, kShearThreads, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace

int shear_grid_blocks()
{
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, shear_kernel<BS_EPRIOR_BA14, false, true>,
                                                  kShearThreads, 0);
    if (sms <= 0) sms = 1;
    if (nb <= 0) nb = 1;
    return sms * nb;
}

cudaError_t launch_shear(const ShearLaunch &s, int grid, cudaStream_t stream)
{
    const bool vec = (s.K % 4 == 0) && ((reinterpret_cast<uintptr_t>(s.e1) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.e2) & 15) == 0) &&
                     (s.b == nullptr || (reinterpret_cast<uintptr_t>(s.b) & 15) == 0);
    const bool hb = s.b != nullptr;
    if (s.family == BS_EPRIOR_BA14)
        return hb ? launch_fb<BS_EPRIOR_BA14, true>(s, grid, vec, stream)
                  : launch_fb<BS_EPRIOR_BA14, false>(s, grid, vec, stream);
    return hb ? launch_fb<BS_EPRIOR_TRUNC_GAUSS, true>(s, grid, vec, stream)
              : launch_fb<BS_EPRIOR_TRUNC_GAUSS, false>(s, grid, vec, stream);
}

cudaError_t launch_shear_finalize(const double *partials, int n_part, double add_value,
                                  double add_g1, double add_g2, double add_alpha,
                                  double alpha_scale, double *out, cudaStream_t stream)
{
    shear_finalize_kernel<<<1, 256, 0, stream>>>(partials, n_part, add_value, add_g1, add_g2,
                                                 add_alpha, alpha_scale, out);
    return cudaGetLastError();
}

}  // namespace bs

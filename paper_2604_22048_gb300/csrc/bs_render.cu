// Forward model on sm_103a (Sec. 3.3): analytic k-space model of an
// exponential galaxy sheared in the reduced-shear convention
// (Eq. shear-transform), convolved with a known PSF and the pixel response,
// drawn on the stamp's periodic grid by a separable inverse DFT.
//
// One CTA per stamp: the half-plane spectrum M(u, v), u = 0..c, is formed in
// shared memory; the column pass A[u][iy] = sum_v M(u,v) exp(+2 pi i v (iy-c)/N)
// and the row pass m[iy][ix] = (1/N^2) sum_u w_u Re(A[u][iy] exp(+2 pi i u
// (ix-c)/N)) (w_0 = 1, w_u = 2: the other half plane is the conjugate) use an
// N-entry twiddle table indexed by exact integer phase reduction.
#include "bs_device.cuh"
#include "bs_internal.h"

namespace bs {

namespace {

__device__ float r_half_x_pow_knu(float nu, float x)
{
    const float lx = logf(0.5f * x);
    const float h = 0.25f;
    float sum = 0.5f * expf(-x + nu * lx);
    for (int j = 1; j < 400; ++j) {
        const float t = j * h;
        const float ch = coshf(t);
        const float a = -x * ch;
        const float term = 0.5f * (expf(a + nu * (lx + t)) + expf(a + nu * (lx - t)));
        sum += term;
        if (x * ch > nu * t + 40.f && term <= 1e-9f * sum) break;
    }
    return sum * h;
}

__device__ float r_psf_transfer(const bs_psf &ps, float k)
{
    if (ps.kind == BS_PSF_GAUSSIAN) {
        const float s = ps.fwhm * (1.0f / 2.3548200450309493f);
        return expf(-0.5f * k * k * s * s);
    }
    const float beta = ps.beta;
    const float rd = ps.fwhm / (2.0f * sqrtf(exp2f(1.0f / beta) - 1.0f));
    const float x = k * rd;
    if (x == 0.0f) return 1.0f;
    const float nu = beta - 1.0f;
    return 2.0f / tgammaf(nu) * r_half_x_pow_knu(nu, x);
}

__device__ __forceinline__ float r_sincpi(float x)
{
    return x == 0.0f ? 1.0f : sinpif(x) / (3.14159265358979f * x);
}

__global__ void __launch_bounds__(256) render_kernel(int n, const float *theta, const float *shear,
                                                     const int64_t *offsets, const int32_t *side,
                                                     int max_side, const bs_psf *psf, int n_psf,
                                                     float p, float *out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int hm = (max_side + 1) / 2;
    float2 *M = reinterpret_cast<float2 *>(smem_raw);        // [hm][max_side]
    float2 *A = M + (size_t)hm * max_side;                    // [hm][max_side]
    float2 *tw = A + (size_t)hm * max_side;                   // [max_side]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int N = side[i];
        if (N < 3 || N > max_side || !(N & 1)) continue;   // uniform per CTA; stamp left untouched
        const int c = (N - 1) / 2, H = c + 1;
        const float *th = theta + (size_t)i * 6;
        const float F = exp10f(th[0]);
        const float r0 = exp10f(th[1]) * (1.0f / kHlrOverR0);
        float e1 = th[2], e2 = th[3];
        if (shear) {
            // eps' = (eps + g) / (1 + conj(g) eps)
            const float g1 = shear[2 * i], g2 = shear[2 * i + 1];
            const float nr = e1 + g1, ni = e2 + g2;
            const float dr = 1.0f + g1 * e1 + g2 * e2, di = g1 * e2 - g2 * e1;
            const float inv = 1.0f / (dr * dr + di * di);
            e1 = (nr * dr + ni * di) * inv;
            e2 = (ni * dr - nr * di) * inv;
        }
        const float E = e1 * e1 + e2 * e2;
        const float Pq = 1.0f / (1.0f - E);
        const float r02 = r0 * r0;
        const float al = r02 * (1.0f + E + 2.0f * e1) * Pq;
        const float be = r02 * (1.0f + E - 2.0f * e1) * Pq;
        const float ga = r02 * 4.0f * e2 * Pq;
        const float dk = 6.283185307179586f / ((float)N * p);
        const float invN = 1.0f / (float)N;
        const bs_psf ps = psf[n_psf == 1 ? 0 : i];
        for (int m = tid; m < N; m += nth) {
            float s, co;
            sincospif(2.0f * (float)m * invN, &s, &co);
            tw[m] = make_float2(co, s);
        }
        for (int o = tid; o < H * N; o += nth) {
            const int u = o / N, vi = o - u * N;
            const int v = vi - c;
            const float kx = u * dk, ky = v * dk;
            const float s = 1.0f + al * kx * kx + be * ky * ky + ga * kx * ky;
            const float rs = rsqrtf(s);
            const float amp = F * rs * rs * rs * r_psf_transfer(ps, sqrtf(kx * kx + ky * ky)) *
                              r_sincpi((float)u * invN) * r_sincpi((float)v * invN);
            float sn, co;
            sincospif(-2.0f * ((float)u * th[4] + (float)v * th[5]) * invN, &sn, &co);
            M[u * N + vi] = make_float2(amp * co, amp * sn);
        }
        __syncthreads();
        // column pass: A[u][iy] = sum_v M(u, v) exp(+2 pi i v (iy - c) / N)
        for (int o = tid; o < H * N; o += nth) {
            const int u = o / N, iy = o - u * N;
            const int dy = ((iy - c) % N + N) % N;
            int idx = (int)(((long long)(N - c) * dy) % N);   // v = -c
            float re = 0.f, im = 0.f;
            for (int vi = 0; vi < N; ++vi) {
                const float2 mv = M[u * N + vi];
                const float2 t = tw[idx];
                re = fmaf(mv.x, t.x, fmaf(-mv.y, t.y, re));
                im = fmaf(mv.x, t.y, fmaf(mv.y, t.x, im));
                idx += dy;
                if (idx >= N) idx -= N;
            }
            A[u * N + iy] = make_float2(re, im);
        }
        __syncthreads();
        // row pass
        float *img = out + offsets[i];
        const float norm = invN * invN;
        for (int o = tid; o < N * N; o += nth) {
            const int iy = o / N, ix = o - iy * N;
            const int dx = ((ix - c) % N + N) % N;
            int idx = 0;
            float acc = A[iy].x;   // u = 0, weight 1
            for (int u = 1; u < H; ++u) {
                idx += dx;
                if (idx >= N) idx -= N;
                const float2 av = A[u * N + iy];
                const float2 t = tw[idx];
                acc = fmaf(2.0f * av.x, t.x, fmaf(-2.0f * av.y, t.y, acc));
            }
            img[o] = acc * norm;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_render(int n, const float *theta, const float *shear, const int64_t *offsets,
                          const int32_t *side, int max_side, const bs_psf *psf, int n_psf,
                          float pixel_scale, float *out, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const int hm = (max_side + 1) / 2;
    const size_t smem = (size_t)(2 * hm * max_side + max_side) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n < 65535 ? n : 65535;
    render_kernel<<<grid, 256, smem, stream>>>(n, theta, shear, offsets, side, max_side, psf, n_psf,
                                              pixel_scale, out);
    bs::count_launches(1);
    return cudaGetLastError();
}

}  // namespace bs

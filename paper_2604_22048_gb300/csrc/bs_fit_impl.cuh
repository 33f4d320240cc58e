#pragma once
// Image sampling phase on sm_103a: per-galaxy HMC on the interim posterior
// (Sec. 3.3; Eq. interim-post = Eq. likelihood-pixels x Eq. interim-prior).
//
// Layout.  A persistent CTA takes one galaxy at a time from an atomic work
// queue and runs its n_chains chains, one warp per chain.  Per galaxy the CTA
// stages in shared memory, once:
//   Dt[u][v] = (sqrt(w_u)/N) DFT(d)(u, v)          (data spectrum)
//   Tt[u][v] = (sqrt(w_u)/N) PSF(|k|) sinc(kx p/2) sinc(ky p/2)
// on the half plane u = 0..c (c = (N-1)/2), v = -c..c, with w_0 = 1 and
// w_u = 2 for u > 0 (the other half is the complex conjugate: d and the
// model are real).  Lane l owns the columns v = l + 32 j - c, j < NC.
//
// Evaluation.  The model spectrum M(k) (Sec. 3.3 forward model: exponential
// profile (1 + r0^2 k^T S^2 k)^{-3/2}, PSF and pixel transfer, centroid
// phase) is formed point by point; since the model image is the inverse DFT
// of M on the stamp's periodic grid, Parseval gives
//   chi^2 = sum_pixels (d - m)^2 = sum_half |Dt - Mt|^2,
//   d chi^2/d theta = -2 sum_half Re[conj(Dt - Mt) dMt/dtheta],
// i.e. the residual's adjoint DFT is Dt - Mt exactly, and the per-evaluation
// cost is one pass over the half plane instead of two O(N^3) transforms.
// The gradient needs seven sums: six are accumulated per lane in FP32 (five
// per point, three of them per column and weighted by ky once at the end)
// and reduced with an xor butterfly (identical bits in all lanes, so
// warp-uniform decisions stay uniform), and the seventh follows from them;
// chi^2 (only on the last step of a trajectory) is accumulated per lane in
// FP32 as F^2 |Dt - Mt|^2 from the terms the gradient already forms (positive
// terms, each accumulator ~14 rows long) and finished in FP64 at the warp total.
//
// Chain state.  Lane i < 6 owns parameter i of the chain (position hi/lo,
// momentum, gradient, inverse metric, Welford moments) as scalars; the six
// positions are gathered with shuffles before each evaluation.  Energies are
// butterfly sums, so accept and divergence decisions are warp-uniform.
//
// Sampler (same algorithm as the oracle, written independently): Philox4x64-10
// keyed by (seed, galaxy_id * n_chains + chain); fixed-L or random-L HMC with
// a diagonal metric; dual averaging of the step size (Hoffman & Gelman 2014,
// gamma 0.05, t0 10, kappa 0.75); Stan-style windowed metric adaptation; a
// doubling/halving step-size search at the start and after each window.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "bs_device.cuh"
#include "bs_internal.h"
#include "bs_pix_tc.cuh"

namespace bs {

namespace {

struct GalCtx {
    int N, H, c, NC;
    float dk;      // 2 pi / (N p)
    float p;       // pixel scale
    float invN;
    float inv_b;   // 1 / sigma^2 (1 when the exposures are folded into the table)
};

// chi^2 of the galaxy's exposures minus that of its folded table (a constant
// of the galaxy, 0 for one exposure with white noise); in shared memory, so
// that it takes no register in the chains' loop.
__shared__ double s_chi2_off;

// Row layout of the staged tables for NCT = npad / 32 column slots per lane
// (3 * npad floats per row u).  Slots are paired, (2p, 2p+1), so that a lane
// loads both slots of a pair with one 8-byte access and the pair is processed
// with packed FP32x2 arithmetic:
//   pair p:      [Dx pairs: 64][Dy pairs: 64][T pairs: 64]   (float2 per lane)
//   odd slot:    [D (x, y): 64][T: 32]                        (last slot, NCT odd)
__host__ __device__ __forceinline__ int row_floats(int npad) { return 3 * npad; }

// Per-chain phase tables X(u) = exp(-2 pi i u dx / N) of one evaluation, in
// the setup scratch (free once the galaxy is staged), extended when the
// chains need more than it holds.
// Entry u of a table is (Re X(u), Im X(u), -Im X(u), 0), one 16-byte load.
// Per-chain stride of the phase tables, in entries (even).
__host__ __device__ __forceinline__ int phase_stride(int h_max) { return (h_max + 1) & ~1; }

// float2 slots of the scratch: the setup's three rows, or the chains' phase
// tables if larger; even, so that the (kx, kx^2) table after it stays 16-byte
// aligned.
__host__ __device__ __forceinline__ int scratch_float2(int max_side, int h_max, int n_chains)
{
    const int setup = 3 * max_side + 4;
    const int phase = 2 * n_chains * phase_stride(h_max);
    const int n = setup > phase ? setup : phase;
    return (n + 1) & ~1;
}

struct SmemView {
    float *tab;    // [h_max][3 npad] data spectrum and transfer, paired layout
    float2 *G;     // [max_side], setup scratch (one frequency row)
    float2 *tw;    // [max_side]
    float2 *Gc;    // [max_side], setup scratch (a row of the noise correlation's transform)
    float4 *xph;   // [n_chains][phase_stride(h_max)] phase tables (aliases G, tw after setup)
    float2 *kxr;   // [h_max]: (kx, kx^2) of row u
};

__device__ __forceinline__ SmemView smem_view(unsigned char *base, int h_max, int npad, int max_side, int n_chains)
{
    SmemView v;
    v.tab = reinterpret_cast<float *>(base);
    v.G = reinterpret_cast<float2 *>(v.tab + (size_t)h_max * row_floats(npad));
    v.tw = v.G + (size_t)max_side;
    v.Gc = v.tw + (size_t)max_side;
    v.xph = reinterpret_cast<float4 *>(v.G);
    v.kxr = v.G + (size_t)scratch_float2(max_side, h_max, n_chains);
    return v;
}

// Positions of slot j of lane l within a row: Dx, Dy, T.
__device__ __forceinline__ void slot_offsets(int npad, int j, int l, int &ox, int &oy, int &ot)
{
    const int nct = npad >> 5, npair = nct >> 1;
    const int p = j >> 1;
    if (p < npair) {
        const int base = p * 192, h = j & 1;
        ox = base + 2 * l + h;
        oy = base + 64 + 2 * l + h;
        ot = base + 128 + 2 * l + h;
    } else {
        const int base = npair * 192;
        ox = base + 2 * l;
        oy = base + 2 * l + 1;
        ot = base + 64 + l;
    }
}

// (x/2)^nu K_nu(x) from K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the
// trapezoidal rule (step 1/4); the factor (x/2)^nu is folded into the
// exponent so the integrand stays bounded for small x.
__device__ float half_x_pow_knu(float nu, float x)
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

// Transform of the unit-flux PSF at |k| (1/arcsec).
__device__ float psf_transfer(const bs_psf &ps, float k)
{
    if (ps.kind == BS_PSF_GAUSSIAN) {
        const float s = ps.fwhm * (1.0f / 2.3548200450309493f);
        return expf(-0.5f * k * k * s * s);
    }
    // Moffat: (2 / Gamma(beta - 1)) (x/2)^(beta-1) K_(beta-1)(x), x = k rd
    const float beta = ps.beta;
    const float rd = ps.fwhm / (2.0f * sqrtf(exp2f(1.0f / beta) - 1.0f));
    const float x = k * rd;
    if (x == 0.0f) return 1.0f;
    const float nu = beta - 1.0f;
    return 2.0f / tgammaf(nu) * half_x_pow_knu(nu, x);
}

// sin(pi x) / (pi x)
__device__ __forceinline__ float sincpi(float x)
{
    return x == 0.0f ? 1.0f : sinpif(x) / (3.14159265358979f * x);
}

__device__ __forceinline__ float load_pix(const void *data, int f64, int64_t idx)
{
    return f64 ? (float)__ldg(static_cast<const double *>(data) + idx)
               : __ldg(static_cast<const float *>(data) + idx);
}

// A stamp side the shared-memory layout of this launch can hold.
__device__ __forceinline__ bool side_ok(const FitParams &P, int N)
{
    return N >= 3 && N <= P.max_side && (N & 1);
}

// G[iy] = sum_ix img[iy][ix] exp(-2 pi i u (ix - c) / N): the x transform of
// the N x N image at `off`, frequency u (threads of the CTA over rows).
__device__ __forceinline__ void row_dft(const void *img, int f64, int64_t off, int N, int c, int u,
                                        const float2 *tw, float2 *G)
{
    for (int iy = threadIdx.x; iy < N; iy += blockDim.x) {
        int idx = (int)(((long long)(N - u) * c) % N);   // -u c mod N
        float re = 0.f, im = 0.f;
        const int64_t rowoff = off + (int64_t)iy * N;
        for (int ix = 0; ix < N; ++ix) {
            const float d = load_pix(img, f64, rowoff + ix);
            const float2 t = tw[idx];
            re = fmaf(d, t.x, re);
            im = fmaf(-d, t.y, im);
            idx += u;
            if (idx >= N) idx -= N;
        }
        G[iy] = make_float2(re, im);
    }
}

// sum_iy G[iy] exp(-2 pi i v (iy - c) / N): the y transform at frequency v.
__device__ __forceinline__ float2 col_dft(const float2 *G, int N, int c, int v, const float2 *tw)
{
    const int vm = ((v % N) + N) % N;
    int idx = (int)(((long long)(N - vm) * c) % N);   // -v c mod N
    float re = 0.f, im = 0.f;
    for (int iy = 0; iy < N; ++iy) {
        const float2 gv = G[iy];
        const float2 t = tw[idx];
        // gv * conj(t)
        re = fmaf(gv.x, t.x, fmaf(gv.y, t.y, re));
        im = fmaf(gv.y, t.x, fmaf(-gv.x, t.y, im));
        idx += vm;
        if (idx >= N) idx -= N;
    }
    return make_float2(re, im);
}

// scale x the PSF x pixel transfer of psf `ps` at grid point (u, v).
__device__ __forceinline__ float transfer_at(const bs_psf &ps, const GalCtx &gc, int u, int v, float scale)
{
    const float kx = u * gc.dk, ky = v * gc.dk;
    return scale * psf_transfer(ps, sqrtf(kx * kx + ky * ky)) * sincpi((float)u * gc.invN) *
           sincpi((float)v * gc.invN);
}

// Sum over the CTA of one double per thread, in a fixed order.
__device__ double block_sum_d(double v)
{
    __shared__ double part[32];
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) part[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += part[i];
    __syncthreads();
    return t;
}

// Appendix C: the galaxy's J exposures on one grid, exposure j with its own
// transfer T_j and noise covariance sigma_j^2 C_j, C_j circulant with
// spectrum lambda_j(k) (the transform of the correlation at lag).  Each
// Gaussian term is diagonal in k,
//   r_j^T Sigma_j^-1 r_j = (1/N^2) sum_k |D_j - T_j G|^2 / (sigma_j^2 lambda_j),
// with G the galaxy's (PSF-free) spectrum, and the sum over exposures is one
// term of the single-exposure form plus a constant:
//   sum_j W_j |D_j - T_j G|^2 = S |C/S - G|^2 + (E - |C|^2/S),
//   W_j = 1/(sigma_j^2 lambda_j), S = sum_j W_j T_j^2, C = sum_j W_j T_j D_j,
//   E = sum_j W_j |D_j|^2.
// So the table holds T' = sqrt(S) and D' = C/sqrt(S) (with inv_b = 1) and the
// fit kernel runs unchanged; the constant goes to chi2_off so that the
// log posterior is that of the exposures.  Returns false (uniform across the
// CTA) when some lambda_j is not positive.
__device__ bool setup_folded(const FitParams &P, int gal, const SmemView &sm, GalCtx &gc)
{
    const int N = gc.N, c = gc.c, H = gc.H, J = P.n_exp;
    const int npad = P.npad, rowf = row_floats(npad);
    const int tid = threadIdx.x, nth = blockDim.x;
    const float sqrt2 = 1.41421356237309515f;
    const int64_t off0 = P.offsets[gal];
    const int64_t NN = (int64_t)N * N;
    double cacc = 0.0;
    bool bad = false;
    for (int u = 0; u < H; ++u) {
        float *row = sm.tab + (size_t)u * rowf;
        const float scale = (u == 0 ? 1.0f : sqrt2) * gc.invN;
        const double s2 = (double)scale * scale;
        for (int j = 0; j < J; ++j) {
            const int64_t off = off0 + (int64_t)j * NN;
            row_dft(P.data, P.data_f64, off, N, c, u, sm.tw, sm.G);
            if (P.noise_corr) row_dft(P.noise_corr, 0, off, N, c, u, sm.tw, sm.Gc);
            __syncthreads();
            const bs_psf ps = P.psf[P.n_psf == 1 ? 0 : (int64_t)gal * J + j];
            const float sig = P.sigma[(int64_t)gal * J + j];
            for (int vi = tid; vi < npad; vi += nth) {
                float Cx = 0.f, Cy = 0.f, S = 0.f;
                if (vi < N) {
                    const int v = vi - c;
                    const float2 D = col_dft(sm.G, N, c, v, sm.tw);
                    float lam = P.noise_corr ? col_dft(sm.Gc, N, c, v, sm.tw).x : 1.0f;
                    if (!(lam > 0.f)) {
                        bad = true;
                        lam = 1.0f;
                    }
                    const float Wj = 1.0f / (sig * sig * lam);
                    const float T = transfer_at(ps, gc, u, v, 1.0f);
                    const float WT = Wj * T;
                    Cx = WT * D.x;
                    Cy = WT * D.y;
                    S = WT * T;
                    cacc += s2 * (double)Wj * ((double)D.x * D.x + (double)D.y * D.y);
                }
                int ox, oy, ot;
                slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
                if (j == 0) {
                    row[ox] = Cx;
                    row[oy] = Cy;
                    row[ot] = S;
                } else {
                    row[ox] += Cx;
                    row[oy] += Cy;
                    row[ot] += S;
                }
            }
            __syncthreads();   // G and Gc are rewritten by the next exposure
        }
        // (C, S) -> (D', T'), each thread on the columns it accumulated
        for (int vi = tid; vi < N; vi += nth) {
            int ox, oy, ot;
            slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
            const float Cx = row[ox], Cy = row[oy], S = row[ot];
            float Dx = 0.f, Dy = 0.f, T = 0.f;
            if (S > 0.f) {
                const float rs = rsqrtf(S);
                T = scale * S * rs;
                Dx = scale * Cx * rs;
                Dy = scale * Cy * rs;
                cacc -= s2 * ((double)Cx * Cx + (double)Cy * Cy) / (double)S;
            }
            row[ox] = Dx;
            row[oy] = Dy;
            row[ot] = T;
        }
    }
    gc.inv_b = 1.0f;
    const double off = block_sum_d(cacc);
    if (tid == 0) s_chi2_off = off;
    return __syncthreads_or(bad) == 0;
}

// Stage the galaxy's data spectrum and transfer table (all threads of the CTA).
// The caller has checked side_ok.  Returns false, uniformly, when the galaxy
// cannot be fitted (a noise correlation without a positive spectrum).
__device__ bool setup_galaxy(const FitParams &P, int gal, const SmemView &sm, GalCtx &gc)
{
    const int N = P.side[gal];
    const int c = (N - 1) / 2;
    const int H = c + 1;
    const int npad = P.npad;
    const int tid = threadIdx.x, nth = blockDim.x;
    gc.N = N;
    gc.H = H;
    gc.c = c;
    gc.NC = (N + 31) / 32;
    gc.p = P.pixel_scale;
    gc.dk = 6.283185307179586f / ((float)N * P.pixel_scale);
    gc.invN = 1.0f / (float)N;
    if (tid == 0) s_chi2_off = 0.0;

    for (int m = tid; m < N; m += nth) {
        float s, co;
        sincospif(2.0f * (float)m / (float)N, &s, &co);
        sm.tw[m] = make_float2(co, s);   // exp(+2 pi i m / N)
    }
    for (int u = tid; u < H; u += nth) {
        const float kx = (float)u * gc.dk;
        sm.kxr[u] = make_float2(kx, kx * kx);
    }
    __syncthreads();
    if (P.n_exp > 1 || P.noise_corr) return setup_folded(P, gal, sm, gc);

    const float sig = P.sigma[gal];
    gc.inv_b = P.pix_prec ? 1.0f : 1.0f / (sig * sig);   // a covariance carries the noise level
    const int64_t off = P.offsets[gal];
    const bs_psf ps = P.psf[P.n_psf == 1 ? 0 : gal];
    const float sqrt2 = 1.41421356237309515f;
    const int rowf = row_floats(npad);
    // one frequency row u at a time, so the scratch is a single column G[iy]
    for (int u = 0; u < H; ++u) {
        row_dft(P.data, P.data_f64, off, N, c, u, sm.tw, sm.G);
        __syncthreads();
        // D(u, v) = sum_iy G[iy] exp(-2 pi i v (iy - c) / N), scaled; transfer T(u, v)
        float *row = sm.tab + (size_t)u * rowf;
        const float scale = (u == 0 ? 1.0f : sqrt2) * gc.invN;
        for (int vi = tid; vi < npad; vi += nth) {
            float2 Dv = make_float2(0.f, 0.f);
            float Tv = 0.f;
            if (vi < N) {
                const int v = vi - c;
                const float2 D = col_dft(sm.G, N, c, v, sm.tw);
                Dv = make_float2(D.x * scale, D.y * scale);
                Tv = transfer_at(ps, gc, u, v, scale);
            }
            int ox, oy, ot;
            slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
            row[ox] = Dv.x;
            row[oy] = Dv.y;
            row[ot] = Tv;
        }
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ bool in_support(const FitParams &P, const float th[6])
{
    const float E = th[2] * th[2] + th[3] * th[3];
    return th[0] > P.lf_lo && th[0] < P.lf_hi && th[1] > P.ls_lo && th[1] < P.ls_hi && E < 1.0f;
}

// 1/sqrt(s) for s >= 1 (the profile argument 1 + r0^2 q(k)): the hardware
// approximation with denormal flushing, which cannot occur here, so no
// range fix-ups are issued around it.
__device__ __forceinline__ float rsqrt_ge1(float s)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
    return r;
}

// 1/s for s >= 1 on the special-function unit: squaring the reciprocal
// square root would cost the FMA pipe, which bounds the fit kernels, one
// more packed multiply per point pair.
__device__ __forceinline__ float rcp_ge1(float s)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
    return r;
}

// sin(pi x) and cos(pi x) for the per-evaluation phase factors, on the
// special-function unit: x - 2 rint(x / 2) reduces x to [-1, 1] without
// rounding error, so the hardware approximation sees an angle in [-pi, pi],
// where its absolute error is about 2^-21 (the library's sincospif spends a
// polynomial on the FMA pipe per call for its last bits).
__device__ __forceinline__ void sincospi_sfu(float x, float *s, float *c)
{
    const float r = fmaf(-2.0f, rintf(0.5f * x), x);
    __sincosf(3.14159265358979f * r, s, c);
}

// Packed FP32x2 helpers (two column slots of a lane in one instruction; each
// half is rounded exactly like the scalar operation).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Per-lane partial sums of one evaluation: slot pairs packed, odd slot scalar.
template <int NCT>
struct Sums {
    static constexpr int NP = NCT / 2 > 0 ? NCT / 2 : 1;
    float2 Swkx2, Sbkx;                     // sum w kx^2, sum b kx (both halves)
    float2 Wc[NP], Wkx[NP], Bc[NP];         // per slot: sum w, sum w kx, sum b
    float sWc, sWkx, sBc;                   // odd slot
    float2 chi0, chi1;                      // F^2 sum |Dt - Mt|^2, even and odd rows
};

// Per-lane, per-slot constants of one evaluation.
template <int NCT>
struct SlotConst {
    static constexpr int NP = NCT / 2 > 0 ? NCT / 2 : 1;
    float2 Yr[NP], Yi[NP], nYr[NP], cst[NP], gky[NP];   // F exp(-i ky p dy) (and -Re), 1 + be ky^2, ga ky
    float sYr, sYi, scst, sgky;
};

// Model-data terms of one row u for all column slots of this lane.
// Profile amplitude f(s) of the model at s = 1 + r0^2 q(k) (PSF, flux and phase
// apart) and the weight psi(s) of the gradient sums (d log f / ds = -c psi):
//   exponential (PROF 0)  f = s^-3/2,                     psi = 1/s;
//   Spergel     (PROF 1)  f = s^-(1+nu), npow = -(1+nu),   psi = 1/s;
//   Gaussian    (PROF 2)  f = exp(-(s - 1)/2),             psi = 1.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <int PROF>
__device__ __forceinline__ void profile_amp(float2 s, float npow, float2 &f, float2 &psi)
{
    if (PROF == 0) {
        const float2 rs = make_float2(rsqrt_ge1(s.x), rsqrt_ge1(s.y));
        psi = mul2(rs, rs);
        f = mul2(psi, rs);
    } else if (PROF == 1) {
        const float lx = lg2_approx(s.x), ly = lg2_approx(s.y);
        psi = make_float2(ex2_approx(-lx), ex2_approx(-ly));
        f = make_float2(ex2_approx(npow * lx), ex2_approx(npow * ly));
    } else {
        const float h = 0.72134752044448170f;   // log2(e) / 2
        f = make_float2(ex2_approx(fmaf(-h, s.x, h)), ex2_approx(fmaf(-h, s.y, h)));
        psi = f2(1.0f);
    }
}
template <int PROF>
__device__ __forceinline__ void profile_amp1(float s, float npow, float &f, float &psi)
{
    float2 ff, pp;
    profile_amp<PROF>(make_float2(s, s), npow, ff, pp);
    f = ff.x;
    psi = pp.x;
}

// The phase of the model at (u, v) is P = X(u) Y(v) with X(u) = exp(-2 pi i u dx / N)
// (row, in the warp's phase table as (Re, Im, -Im)) and Y(v) = F exp(-2 pi i v dy / N)
// (column, in registers).  The point needs z = conj(D) P = (conj(D) Y) X: the column
// factor first, whose negated real part is a register, then the row factor, whose
// negated imaginary part the table holds, so that both complex products are two
// multiplies and two multiply-adds.  With c = Re z - A F^2 (the real part of
// conj(D - M) P, M = A P), the residual is |D - M|^2 = (c^2 + (Im z)^2) / F^2, since
// |P| = F; the log-likelihood pass accumulates c^2 + (Im z)^2 and scales once.
template <int NCT, bool LL, int PROF>
__device__ __forceinline__ void row_terms(Sums<NCT> &S, float2 &chi, const SlotConst<NCT> &K,
                                          const float *__restrict__ row, float kx, float kx2, float al,
                                          float4 X, float F2, float npow)
{
    constexpr int NPAIR = NCT / 2;
    const int lane = threadIdx.x & 31;
    const float2 kxv = f2(kx), kx2v = f2(kx2), alv = f2(al), Xrv = f2(X.x), Xiv = f2(X.y), nXiv = f2(X.z);
    const float2 nF2v = f2(-F2);
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const float *b = row + p * 192 + 2 * lane;
        const float2 Dx = *reinterpret_cast<const float2 *>(b);
        const float2 Dy = *reinterpret_cast<const float2 *>(b + 64);
        const float2 T = *reinterpret_cast<const float2 *>(b + 128);
        const float2 s = fma2(fma2(alv, kxv, K.gky[p]), kxv, K.cst[p]);   // 1 + r0^2 q(k), Horner in kx
        float2 A, rs2;                                                   // |M| / F and psi
        if (PROF == 0) {
            const float2 rs = make_float2(rsqrt_ge1(s.x), rsqrt_ge1(s.y));
            rs2 = make_float2(rcp_ge1(s.x), rcp_ge1(s.y));
            A = mul2(mul2(T, rs2), rs);
        } else {
            float2 fa;
            profile_amp<PROF>(s, npow, fa, rs2);
            A = mul2(T, fa);
        }
        const float2 Er = fma2(Dx, K.Yr[p], mul2(Dy, K.Yi[p]));         // conj(D) Y
        const float2 Ei = fma2(Dx, K.Yi[p], mul2(Dy, K.nYr[p]));
        const float2 zr = fma2(Er, Xrv, mul2(Ei, nXiv));                 // z = conj(D) Y X
        const float2 zi = fma2(Er, Xiv, mul2(Ei, Xrv));
        const float2 c = fma2(A, nF2v, zr);                             // Re conj(D - M) P
        const float2 a = mul2(A, c);                                    // Re conj(D - M) M
        const float2 bb = mul2(A, zi);                                  // Im conj(D - M) M
        const float2 w = mul2(a, rs2);                                  // a / s
        S.Wc[p] = add2(S.Wc[p], w);
        S.Wkx[p] = fma2(w, kxv, S.Wkx[p]);
        S.Swkx2 = fma2(w, kx2v, S.Swkx2);
        S.Bc[p] = add2(S.Bc[p], bb);
        S.Sbkx = fma2(bb, kxv, S.Sbkx);
        if (LL) chi = fma2(c, c, fma2(zi, zi, chi));
    }
    if (NCT & 1) {
        const float *b = row + NPAIR * 192;
        const float2 D = *reinterpret_cast<const float2 *>(b + 2 * lane);
        const float T = b[64 + lane];
        const float s = fmaf(fmaf(al, kx, K.sgky), kx, K.scst);
        float A, rs2;
        if (PROF == 0) {
            const float rs = rsqrt_ge1(s);
            rs2 = rs * rs;
            A = T * rs2 * rs;
        } else {
            float fa;
            profile_amp1<PROF>(s, npow, fa, rs2);
            A = T * fa;
        }
        const float Er = fmaf(D.x, K.sYr, D.y * K.sYi);
        const float Ei = fmaf(D.x, K.sYi, -(D.y * K.sYr));
        const float zr = fmaf(Er, X.x, Ei * X.z);
        const float zi = fmaf(Er, X.y, Ei * X.x);
        const float c = fmaf(A, -F2, zr);
        const float a = A * c;
        const float bb = A * zi;
        const float w = a * rs2;
        S.sWc += w;
        S.sWkx = fmaf(w, kx, S.sWkx);
        S.Swkx2.x = fmaf(w, kx2, S.Swkx2.x);
        S.sBc += bb;
        S.Sbkx.x = fmaf(bb, kx, S.Sbkx.x);
        if (LL) chi.x = fmaf(c, c, fmaf(zi, zi, chi.x));
    }
}

// Half-plane pass, two rows per iteration (four with at most one pair of slots per
// row); each row reads its (kx, kx^2) from the galaxy's row table and X(u) from the
// warp's phase table.
template <int NCT, bool LL, int PROF>
__device__ __forceinline__ void half_plane(Sums<NCT> &S, const SlotConst<NCT> &K,
                                           const float *__restrict__ tab, const float2 *__restrict__ kxr,
                                           const float4 *__restrict__ xph, int H, float al, float F2, float npow)
{
    constexpr int ROWF = 96 * NCT;
    const float *row = tab;
    int u = 0;
    if constexpr (NCT <= 2) {
        // one pair of column slots (or one slot) per row: four rows in flight (10^4
        // galaxies at 53 px 244.6 -> 237.2 ms, at 25 px 138.2 -> 116.7 ms; with two
        // pairs per row, 65-95 px, it was slower: 477.6 -> 484.6 ms at 75 px)
        for (; u + 3 < H; u += 4) {
            const float4 k01 = *reinterpret_cast<const float4 *>(kxr + u);
            const float4 k23 = *reinterpret_cast<const float4 *>(kxr + u + 2);
            row_terms<NCT, LL, PROF>(S, S.chi0, K, row, k01.x, k01.y, al, xph[u], F2, npow);
            row_terms<NCT, LL, PROF>(S, S.chi1, K, row + ROWF, k01.z, k01.w, al, xph[u + 1], F2, npow);
            row_terms<NCT, LL, PROF>(S, S.chi0, K, row + 2 * ROWF, k23.x, k23.y, al, xph[u + 2], F2, npow);
            row_terms<NCT, LL, PROF>(S, S.chi1, K, row + 3 * ROWF, k23.z, k23.w, al, xph[u + 3], F2, npow);
            row += 4 * ROWF;
        }
    }
    for (; u + 1 < H; u += 2) {
        const float4 k01 = *reinterpret_cast<const float4 *>(kxr + u);   // (kx, kx^2) of rows u, u+1
        row_terms<NCT, LL, PROF>(S, S.chi0, K, row, k01.x, k01.y, al, xph[u], F2, npow);
        row_terms<NCT, LL, PROF>(S, S.chi1, K, row + ROWF, k01.z, k01.w, al, xph[u + 1], F2, npow);
        row += 2 * ROWF;
    }
    if (u < H) {
        const float2 k0 = kxr[u];
        row_terms<NCT, LL, PROF>(S, S.chi0, K, row, k0.x, k0.y, al, xph[u], F2, npow);
    }
}

// Sums over the warp of NV <= 8 per-lane values, returned in every lane with
// identical bits.  Recursive halving: at each xor distance a lane keeps half
// of its values and receives the partner's partial sums of them, so after
// distances 16, 8, 4 lane l holds value (l >> 2) & 7 summed over 8 lanes; two
// butterfly steps finish it (commutative adds, so the 4 lanes of a group
// agree) and one shuffle per value broadcasts it from lane 4 j.
template <int NV>
__device__ __forceinline__ void warp_sum_n(float (&v)[NV])
{
    static_assert(NV >= 5 && NV <= 8, "four values per half at the first step");
    const int lane = threadIdx.x & 31;
    float r4[4];
    const bool h16 = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float lo = v[k], hi = k + 4 < NV ? v[k + 4] : 0.0f;
        const float keep = h16 ? hi : lo, send = h16 ? lo : hi;
        r4[k] = keep + __shfl_xor_sync(BS_FULL_MASK, send, 16);
    }
    float r2[2];
    const bool h8 = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float keep = h8 ? r4[k + 2] : r4[k], send = h8 ? r4[k] : r4[k + 2];
        r2[k] = keep + __shfl_xor_sync(BS_FULL_MASK, send, 8);
    }
    const bool h4 = lane & 4;
    float r = (h4 ? r2[1] : r2[0]) + __shfl_xor_sync(BS_FULL_MASK, h4 ? r2[0] : r2[1], 4);
    r += __shfl_xor_sync(BS_FULL_MASK, r, 2);
    r += __shfl_xor_sync(BS_FULL_MASK, r, 1);
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = __shfl_sync(BS_FULL_MASK, r, 4 * j);
}

// The model's shape at th (Sec. 3.3 forward model): flux, r0^2 and the coefficients
// of the sheared quadratic form r0^2 q(k) = al kx^2 + be ky^2 + ga kx ky.
struct Shape {
    float F, r02, e1, e2, E, Pq, al, be, ga;
};
template <int PROF>
__device__ __forceinline__ Shape model_shape(const FitParams &P, const float th[6])
{
    Shape m;
    m.F = exp10f(th[0]);
    const float r0 = exp10f(th[1]) * (PROF == 0 ? 1.0f / kHlrOverR0 : P.inv_hlr_r0);
    m.r02 = r0 * r0;
    m.e1 = th[2];
    m.e2 = th[3];
    m.E = m.e1 * m.e1 + m.e2 * m.e2;
    m.Pq = 1.0f / (1.0f - m.E);
    m.al = m.r02 * (1.0f + m.E + 2.0f * m.e1) * m.Pq;   // coefficient of kx^2 in r0^2 q
    m.be = m.r02 * (1.0f + m.E - 2.0f * m.e1) * m.Pq;   // ky^2
    m.ga = m.r02 * 4.0f * m.e2 * m.Pq;                  // kx ky
    return m;
}

// The half-plane pass over rows [u0, u1) (warp-cooperative; u0 even): the warp's
// phase table X(u) = exp(-2 pi i u dx / N) for those rows, then the six sums of the
// gradient, reduced over the warp into sums[] (identical in all lanes): sum w,
// sum w kx^2, sum w ky^2, sum w kx ky, sum b kx, sum b ky; and, if LL, this lane's
// part of F^2 chi^2 as a compensated pair (hi, lo).
template <int NC, bool LL, int PROF>
__device__ __forceinline__ void spectral_sums(const FitParams &P, const GalCtx &gc, const Shape &m,
                                              const float *__restrict__ tab, const float2 *__restrict__ kxr,
                                              float4 *__restrict__ xph, const float vcol[NC], const float th[6],
                                              int u0, int u1, float (&sums)[6], float &chi_hi, float &chi_lo)
{
    const float F2 = m.F * m.F;
    const float dk = gc.dk;
    {
        const int lane = threadIdx.x & 31;
        for (int u = u0 + lane; u < u1; u += 32) {
            float sx, cx;
            sincospi_sfu(-2.0f * th[4] * (float)u * gc.invN, &sx, &cx);
            xph[u] = make_float4(cx, sx, -sx, 0.0f);
        }
        __syncwarp();
    }
    float Yr[NC], Yi[NC], cst[NC], gky[NC], ky[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        float s, co;
        sincospi_sfu(-2.0f * th[5] * vcol[j] * gc.invN, &s, &co);   // exp(-2 pi i v dy / N)
        Yr[j] = m.F * co;
        Yi[j] = m.F * s;
        ky[j] = vcol[j] * dk;
        cst[j] = fmaf(m.be * ky[j], ky[j], 1.0f);
        gky[j] = m.ga * ky[j];
    }
    SlotConst<NC> K;
    Sums<NC> S;
    constexpr int NPAIR = NC / 2;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        K.Yr[p] = make_float2(Yr[2 * p], Yr[2 * p + 1]);
        K.Yi[p] = make_float2(Yi[2 * p], Yi[2 * p + 1]);
        K.nYr[p] = make_float2(-Yr[2 * p], -Yr[2 * p + 1]);
        K.cst[p] = make_float2(cst[2 * p], cst[2 * p + 1]);
        K.gky[p] = make_float2(gky[2 * p], gky[2 * p + 1]);
        S.Wc[p] = f2(0.f);
        S.Wkx[p] = f2(0.f);
        S.Bc[p] = f2(0.f);
    }
    if (NC & 1) {
        K.sYr = Yr[NC - 1];
        K.sYi = Yi[NC - 1];
        K.scst = cst[NC - 1];
        K.sgky = gky[NC - 1];
    }
    S.Swkx2 = f2(0.f);
    S.Sbkx = f2(0.f);
    S.sWc = 0.f;
    S.sWkx = 0.f;
    S.sBc = 0.f;
    S.chi0 = f2(0.f);
    S.chi1 = f2(0.f);
    if (u1 > u0)
        half_plane<NC, LL, PROF>(S, K, tab + (size_t)u0 * row_floats(P.npad), kxr + u0, xph + u0, u1 - u0, m.al,
                                 F2, P.prof_npow);
    __syncwarp();   // the table is rewritten by the next evaluation

    float Swkx2 = S.Swkx2.x + S.Swkx2.y, Sbkx = S.Sbkx.x + S.Sbkx.y;
    float Sw = 0.f, Swky2 = 0.f, Swkxky = 0.f, Sbky = 0.f;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        float wc, wkx, bc;
        if (j < 2 * NPAIR) {
            const int p = j >> 1;
            wc = (j & 1) ? S.Wc[p].y : S.Wc[p].x;
            wkx = (j & 1) ? S.Wkx[p].y : S.Wkx[p].x;
            bc = (j & 1) ? S.Bc[p].y : S.Bc[p].x;
        } else {
            wc = S.sWc;
            wkx = S.sWkx;
            bc = S.sBc;
        }
        Sw += wc;
        Swky2 = fmaf(ky[j] * ky[j], wc, Swky2);
        Swkxky = fmaf(ky[j], wkx, Swkxky);
        Sbky = fmaf(ky[j], bc, Sbky);
    }
    sums[0] = Sw;
    sums[1] = Swkx2;
    sums[2] = Swky2;
    sums[3] = Swkxky;
    sums[4] = Sbkx;
    sums[5] = Sbky;
    warp_sum_n(sums);
    if (LL) {
        // the lane's residual sums (positive terms, each at most ~14 rows long)
        const float2 t = add2(S.chi0, S.chi1);
        two_sum(t.x, t.y, chi_hi, chi_lo);
    }
}

// The gradient of the log posterior from the six sums of the half-plane pass (the
// likelihood's part, over sigma^2) and the interim prior's part.
template <int PROF>
__device__ __forceinline__ void spectral_grad(const FitParams &P, const GalCtx &gc, const Shape &m,
                                              const float (&sums)[6], const float th[6], float g[6])
{
    const float Sw = sums[0], Swkx2 = sums[1], Swky2 = sums[2], Swkxky = sums[3], Sbkx = sums[4], Sbky = sums[5];
    const float al = m.al, be = m.be, ga = m.ga, r02 = m.r02, e1 = m.e1, e2 = m.e2, E = m.E, Pq = m.Pq;
    // sum of w (s - 1) = al sum w kx^2 + be sum w ky^2 + ga sum w kx ky.  With
    // psi = 1/s (exponential, Spergel) a = w s, so sum a = sum w + that; with
    // psi = 1 (Gaussian) a = w.  The sum of a is therefore not accumulated.
    const float st = al * Swkx2 + be * Swky2 + ga * Swkxky;
    const float Sa = PROF == 2 ? Sw : Sw + st;

    const float ib = gc.inv_b;
    const float P2 = Pq * Pq;
    // derivatives of the quadratic-form coefficients with respect to e1, e2
    const float da1 = r02 * ((2.0f * e1 + 2.0f) * Pq + (1.0f + E + 2.0f * e1) * 2.0f * e1 * P2);
    const float da2 = r02 * (2.0f * e2 * Pq + (1.0f + E + 2.0f * e1) * 2.0f * e2 * P2);
    const float db1 = r02 * ((2.0f * e1 - 2.0f) * Pq + (1.0f + E - 2.0f * e1) * 2.0f * e1 * P2);
    const float db2 = r02 * (2.0f * e2 * Pq + (1.0f + E - 2.0f * e1) * 2.0f * e2 * P2);
    const float dg1 = r02 * 8.0f * e1 * e2 * P2;
    const float dg2 = r02 * (4.0f * Pq + 8.0f * e2 * e2 * P2);
    g[0] = kLn10 * Sa * ib;
    if (PROF == 0) {
        g[1] = -3.0f * kLn10 * st * ib;
        g[2] = -1.5f * (da1 * Swkx2 + db1 * Swky2 + dg1 * Swkxky) * ib - 4.0f * e1 * Pq - e1 * P.inv_se2;
        g[3] = -1.5f * (da2 * Swkx2 + db2 * Swky2 + dg2 * Swkxky) * ib - 4.0f * e2 * Pq - e2 * P.inv_se2;
    } else {
        // d M / d log10 hlr = -2 c ln10 psi (s - 1) M, and the sum of
        // a psi (s - 1) = w (s - 1) is st for both profiles
        const float c = P.prof_c;
        g[1] = -2.0f * c * kLn10 * st * ib;
        g[2] = -c * (da1 * Swkx2 + db1 * Swky2 + dg1 * Swkxky) * ib - 4.0f * e1 * Pq - e1 * P.inv_se2;
        g[3] = -c * (da2 * Swkx2 + db2 * Swky2 + dg2 * Swkxky) * ib - 4.0f * e2 * Pq - e2 * P.inv_se2;
    }
    g[4] = gc.p * Sbkx * ib - th[4] * P.inv_sxy2;
    g[5] = gc.p * Sbky * ib - th[5] * P.inv_sxy2;
}

// Component i of the same gradient, each lane its own parameter's: the flux and size
// components are multiples of (al, be, ga) on the shape sums, the ellipticity
// components take the derivatives of those coefficients with respect to e_i, the
// position components the b sums; the lane picks its coefficients and forms one dot
// product (instead of all six components in every lane).
template <int PROF>
__device__ __forceinline__ float spectral_grad_at(const FitParams &P, const GalCtx &gc, const Shape &m,
                                                  const float (&sums)[6], const float th[6], int i)
{
    const float e1 = m.e1, e2 = m.e2, E = m.E, Pq = m.Pq, r02 = m.r02;
    const bool ell = i == 2 || i == 3;
    const float ei = i == 2 ? e1 : e2;
    const float P2 = Pq * Pq;
    const float tei = 2.0f * ei;
    const float dl = i == 2 ? 2.0f : 0.0f;
    const float da = r02 * ((tei + dl) * Pq + (1.0f + E + 2.0f * e1) * tei * P2);
    const float db = r02 * ((tei - dl) * Pq + (1.0f + E - 2.0f * e1) * tei * P2);
    const float dg = r02 * (8.0f * ei * e2 * P2 + (i == 3 ? 4.0f * Pq : 0.0f));
    // d log f / d s = -ce / s on the shape sums; the size scale enters s as r0^2
    const float ce = PROF == 0 ? 1.5f : P.prof_c;
    const float kq = i == 0 ? (PROF == 2 ? 0.0f : kLn10) : -2.0f * ce * kLn10;
    const float cx = ell ? -ce * da : kq * m.al;
    const float cy = ell ? -ce * db : kq * m.be;
    const float cxy = ell ? -ce * dg : kq * m.ga;
    const float cw = i == 0 ? kLn10 : 0.0f;
    const bool pos = i >= 4;
    const float sb = i == 4 ? sums[4] : sums[5];
    const float lik = pos ? gc.p * sb : fmaf(cw, sums[0], fmaf(cx, sums[1], fmaf(cy, sums[2], cxy * sums[3])));
    const float tp = i == 4 ? th[4] : th[5];
    const float pri = pos ? -tp * P.inv_sxy2 : (ell ? -4.0f * ei * Pq - ei * P.inv_se2 : 0.0f);
    return lik * gc.inv_b + pri;
}

// Log posterior (if want_ll) and gradient at th, warp-cooperative.
// gi receives the gradient's component for this lane's parameter, min(lane, 5).
template <int NC, int PROF>
__device__ __forceinline__ double eval_logpost(const FitParams &P, const GalCtx &gc,
                                               const float *__restrict__ tab, const float2 *__restrict__ kxr,
                                               float4 *__restrict__ xph, const float vcol[NC], const float th[6],
                                               float &gi, bool want_ll)
{
    const Shape m = model_shape<PROF>(P, th);
    float sums[6];
    float chi_hi = 0.f, chi_lo = 0.f;
    if (want_ll)
        spectral_sums<NC, true, PROF>(P, gc, m, tab, kxr, xph, vcol, th, 0, gc.H, sums, chi_hi, chi_lo);
    else
        spectral_sums<NC, false, PROF>(P, gc, m, tab, kxr, xph, vcol, th, 0, gc.H, sums, chi_hi, chi_lo);
    const int lane = threadIdx.x & 31;
    gi = spectral_grad_at<PROF>(P, gc, m, sums, th, lane < 6 ? lane : 5);
    if (!want_ll) return 0.0;
    // then the warp
    const double chi2 = warp_sum_comp(chi_hi, chi_lo) / ((double)m.F * (double)m.F);
    const float E = m.E;
    const float lprior = P.prior_const - 0.5f * (th[4] * th[4] + th[5] * th[5]) * P.inv_sxy2 +
                         2.0f * log1pf(-E) - 0.5f * E * P.inv_se2;
    return -0.5 * (chi2 + s_chi2_off) * (double)gc.inv_b + (double)lprior;
}

#include "bs_fit_pixel.cuh"

__device__ __forceinline__ float pick6(const float (&v)[6], int i)
{
    float r = v[0];
#pragma unroll
    for (int k = 1; k < 6; ++k)
        if (i == k) r = v[k];
    return r;
}

// 1/2 sum_i m_i p_i^2 over the six parameter lanes (identical in all lanes).
__device__ __forceinline__ double kinetic(float pm, float im, bool own)
{
    return 0.5 * (double)warp_sum(own ? im * pm * pm : 0.0f);
}

enum { MODE_INIT = 0, MODE_SEARCH = 1, MODE_STEP = 2 };

// One trajectory of nst leapfrog steps from (tp, tpl, gp, pm) (updated in
// place); lpp receives the log posterior at its end; returns false when it
// leaves the prior support.  The warp of the CTA's `slot` uses that slot's
// phase table.
template <int NC, int PROF>
__device__ __forceinline__ bool trajectory(const FitParams &P, const GalCtx &gc, const SmemView &sm, int gal,
                                        int slot, float eps_use, int nst, float im, float &tp, float &tpl,
                                        float &gp, float &pm, double &lpp, int &ngrad)
{
    const int lane = threadIdx.x & 31;
    const int pi = lane < 6 ? lane : 5;
    float vcol[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) vcol[j] = (float)(lane + 32 * j - gc.c);
    float4 *xph_c = sm.xph + (size_t)slot * phase_stride(P.h_max);   // this warp's phase table
    for (int l = 0; l < nst; ++l) {
        const float he = 0.5f * eps_use;
        pm = fmaf(he, gp, pm);
        {
            // compensated position update (hi, lo) += eps m p
            const float d = fmaf(eps_use * im, pm, tpl);
            float s, e;
            two_sum(tp, d, s, e);
            tp = s;
            tpl = e;
        }
        float x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = __shfl_sync(BS_FULL_MASK, tp, k);
        if (!in_support(P, x)) return false;
        double v;
        if constexpr (PROF == 3) {
            float gg[6];
            v = eval_pix<NC>(P, gc, sm, gal, xph_c, vcol, x, gg, l == nst - 1, nullptr);
            gp = pick6(gg, pi);
        } else if constexpr (PROF == 4) {
            v = eval_dense<NC>(P, gc, dense_view(sm.kxr, P.h_max, P.npad, P.max_side, slot), gal, sm.kxr, xph_c,
                               vcol, x, gp, l == nst - 1);
        } else {
            v = eval_logpost<NC, PROF>(P, gc, sm.tab, sm.kxr, xph_c, vcol, x, gp, l == nst - 1);
        }
        ++ngrad;
        if (l == nst - 1) lpp = v;
        pm = fmaf(he, gp, pm);
    }
    return true;
}

// The state of a chain that changes only between trajectories, in shared memory (one
// slot per warp of the CTA: the pixel path's four warps of a chain keep a copy each),
// so that it holds no registers while the trajectory's evaluations run: the warp's
// scalars (step size, dual-averaging and window state, search and transition
// counters, log posterior, the trajectory's start energy and accept uniform) and each
// parameter's position, gradient and window moments, written by the parameter's lane
// (lanes 6.. read parameter 5's slot; their copies of the chain's per-parameter values
// are never used: only lanes 0-5 feed the gathers, the energies and the outputs).
struct ChainScalars {
    double lp, H0;
    uint64_t key;
    float eps, da_mu, da_hbar, da_lebar, s_eps, asum, lu6;
    int da_m, wn, wi, s_idx, s_t, s_dir, it, ndiv, mode, u_base;
};
struct ChainLanes {
    float th[8], thl[8], g[8], wmean[8], wm2[8];
};
__shared__ ChainScalars s_chain_scal[kMaxChains];
__shared__ ChainLanes s_chain_lanes[kMaxChains];

// Chain `chain` of galaxy gal, run by the warp of the CTA's `slot`.
template <int NC, int PROF>
__device__ void run_chain(const FitParams &P, const GalCtx &gc, const SmemView &sm, int gal,
                          int chain, int slot)
{
    const int lane = threadIdx.x & 31;
    const int pi = lane < 6 ? lane : 5;     // parameter of this lane (lanes 6.. shadow parameter 5)
    const bool own = lane < 6;
    // the pixel path's groups of four warps run one chain each: their first warp writes
    const bool wr = PROF != 3 || (threadIdx.x & 127) < 32;
    const int C = P.n_chains, W = P.n_warmup, S = P.n_samples, L = P.n_leapfrog;
    ChainScalars &cs = s_chain_scal[threadIdx.x >> 5];
    ChainLanes &cl = s_chain_lanes[threadIdx.x >> 5];
    const uint64_t gid = P.gal_id ? P.gal_id[gal] : (uint64_t)gal;
    cs.key = gid * (uint64_t)C + (uint64_t)chain;

    const size_t ci0 = (size_t)gal * C + chain;
    // this lane's parameter: position (hi, lo), gradient, inverse metric
    if (own) cl.th[pi] = P.init[ci0 * 6 + pi];
    if (own) cl.thl[pi] = 0.f;
    if (own) cl.g[pi] = 0.f;
    float im = P.init_im ? P.init_im[ci0 * 6 + pi] : 1.f;
    if (own) cl.wmean[pi] = 0.f;
    if (own) cl.wm2[pi] = 0.f;
    cs.lp = -INFINITY;
    cs.eps = P.init_step ? P.init_step[ci0] : 1.0f;
    cs.da_mu = 0.f;
    cs.da_hbar = 0.f;
    cs.da_lebar = 0.f;
    cs.da_m = 0;
    cs.wn = 0;
    cs.wi = 0;
    cs.s_idx = 0;
    cs.s_t = 0;
    cs.s_dir = 0;
    cs.s_eps = 1.0f;
    cs.it = 0;
    cs.asum = 0.f;
    cs.ndiv = 0;
    int ngrad = 0;
    cs.mode = MODE_INIT;
    const double thr_search = -0.22314355131420976;   // ln 0.8
    const size_t chain_row = ci0 * (size_t)S;
    const size_t plane = (size_t)P.n_gal * C * S;
    // the uniforms of four transitions at a time: lane 8 j + k holds uniform k of
    // transition u_base + j (the lanes run four Philox blocks side by side, in the
    // time of one; a transition gathers its eight with shuffles)
    float u_cache = 0.f;
    cs.u_base = -4;

    if (W + S == 0) cs.mode = -1;
    while (cs.mode >= 0) {
        float u[8];
        float eps_use = 0.f;
        int nst = 1;
        if (cs.mode == MODE_SEARCH) {
            uniforms8(P.seed, cs.key, (uint64_t)cs.s_idx, 1ull, (uint64_t)cs.s_t, u);
            eps_use = cs.s_eps;
        } else if (cs.mode == MODE_STEP) {
            if (cs.it - cs.u_base >= 4) {   // transitions run in order, each once
                cs.u_base = cs.it;
                u_cache = uniform_of8(P.seed, cs.key, (uint64_t)(cs.it + (lane >> 3)), 0ull, 0ull, lane & 7);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = __shfl_sync(BS_FULL_MASK, u_cache, 8 * (cs.it - cs.u_base) + q);
            eps_use = cs.eps;
            cs.lu6 = logf(u[6]);
            if (P.random_steps) {
                // L_i = 1 + floor(u7 L), in integers: u7 = (2j + 1) 2^-25
                const unsigned twoj1 = (unsigned)(u[7] * 33554432.0f);
                nst = 1 + (int)(((unsigned long long)twoj1 * (unsigned)L) >> 25);
            } else {
                nst = L;
                eps_use = cs.eps * (1.0f + P.jitter * (2.0f * u[7] - 1.0f));
            }
        }
        // momentum of this lane's parameter: Box-Muller on the pair (u_2j, u_2j+1)
        float pm = 0.f;
        if (cs.mode != MODE_INIT) {
            const int j = pi >> 1;
            const float ua = j == 0 ? u[0] : (j == 1 ? u[2] : u[4]);
            const float ub = j == 0 ? u[1] : (j == 1 ? u[3] : u[5]);
            const float r = sqrtf(-2.0f * logf(ua));
            float sn, cs;
            sincospif(2.0f * ub, &sn, &cs);
            pm = ((pi & 1) ? r * sn : r * cs) / sqrtf(im);
        }
        cs.H0 = -cs.lp + kinetic(pm, im, own);
        float tp = cl.th[pi], tpl = cl.thl[pi], gp = cl.g[pi];
        double lpp = cs.lp;
        bool ok = trajectory<NC, PROF>(P, gc, sm, gal, slot, eps_use, nst, im, tp, tpl, gp, pm, lpp, ngrad);
        if (cs.mode == MODE_INIT) {
            if (own) cl.th[pi] = tp;
            if (own) cl.thl[pi] = tpl;
            if (own) cl.g[pi] = gp;
            cs.lp = ok ? lpp : -INFINITY;
            if (!isfinite(cs.lp) && wr && lane == 0 && P.status) P.status[gal] = 1;
            if (P.init_step) {
                // resume with the given step size: no search, dual averaging from it
                cs.da_mu = logf(10.0f * cs.eps);
                cs.mode = MODE_STEP;
            } else {
                cs.mode = MODE_SEARCH;
                cs.s_idx = 0;
                cs.s_t = 0;
                cs.s_eps = 1.0f;
            }
            continue;
        }
        double dH = INFINITY;
        if (ok) {
            dH = (-lpp + kinetic(pm, im, own)) - cs.H0;
            if (!isfinite(dH) || dH > 1000.0) ok = false;
        }
        if (cs.mode == MODE_SEARCH) {
            const double la = ok ? -dH : -INFINITY;
            const bool good = la > thr_search;
            bool done = false;
            if (cs.s_t == 0)
                cs.s_dir = good ? 1 : -1;
            else if ((cs.s_dir > 0 && !good) || (cs.s_dir < 0 && good))
                done = true;
            if (cs.s_t == 60) done = true;
            if (!done) {
                ++cs.s_t;
                cs.s_eps = cs.s_dir > 0 ? 2.0f * cs.s_eps : 0.5f * cs.s_eps;
                continue;
            }
            cs.eps = cs.s_eps;
            cs.da_mu = logf(10.0f * cs.eps);
            cs.da_hbar = 0.f;
            cs.da_lebar = 0.f;
            cs.da_m = 0;
            cs.mode = MODE_STEP;
            if (cs.it >= W + S) cs.mode = -1;
            continue;
        }
        // ---- transition at iteration `it`
        const float a = ok ? (dH < 0.0 ? 1.0f : expf((float)-dH)) : 0.0f;
        const bool acc = ok && ((double)cs.lu6 < -dH);
        if (acc) {
            if (own) cl.th[pi] = tp;
            if (own) cl.thl[pi] = tpl;
            if (own) cl.g[pi] = gp;
            cs.lp = lpp;
        }
        if (cs.it < W) {
            if (wr && lane == 7) {
                const size_t wi0 = ci0 * (size_t)W + cs.it;
                if (P.warm_accepted) P.warm_accepted[wi0] = acc ? 1 : 0;
                if (P.warm_stat) P.warm_stat[wi0] = a;
                if (P.warm_step) P.warm_step[wi0] = cs.eps;
            }
            // dual averaging
            cs.da_m += 1;
            const float m = (float)cs.da_m;
            const float eta = 1.0f / (m + 10.0f);
            cs.da_hbar = (1.0f - eta) * cs.da_hbar + eta * (P.target_accept - a);
            const float le = cs.da_mu - sqrtf(m) * 20.0f * cs.da_hbar;
            const float xe = powf(m, -0.75f);
            cs.da_lebar = xe * le + (1.0f - xe) * cs.da_lebar;
            cs.eps = expf(le);
            if (cs.wi < P.n_windows && cs.it >= P.win_start[cs.wi] && cs.it < P.win_end[cs.wi]) {
                ++cs.wn;
                const float x = cl.th[pi] + cl.thl[pi];
                const float d = x - cl.wmean[pi];
                if (own) cl.wmean[pi] = fmaf(d, 1.0f / (float)cs.wn, cl.wmean[pi]);
                if (own) cl.wm2[pi] = fmaf(d, x - cl.wmean[pi], cl.wm2[pi]);
            }
            if (cs.wi < P.n_windows && cs.it == P.win_end[cs.wi] - 1) {
                const float n = (float)cs.wn;
                const float var = cl.wm2[pi] / (n - 1.0f);
                im = (n / (n + 5.0f)) * var + 1e-3f * (5.0f / (n + 5.0f));
                if (own) cl.wmean[pi] = 0.f;
                if (own) cl.wm2[pi] = 0.f;
                cs.wn = 0;
                cs.mode = MODE_SEARCH;
                cs.s_idx = cs.wi + 1;
                cs.s_t = 0;
                cs.s_eps = cs.eps;
                ++cs.wi;
            }
            if (cs.it == W - 1) cs.eps = expf(cs.da_lebar);
        } else {
            const int s = cs.it - W;
            cs.asum += a;
            cs.ndiv += ok ? 0 : 1;
            if (wr) {
                if (own) P.samples[(size_t)pi * plane + chain_row + s] = cl.th[pi] + cl.thl[pi];
                if (lane == 6 && P.logp) P.logp[chain_row + s] = (float)cs.lp;
                if (lane == 7 && P.accepted) P.accepted[chain_row + s] = acc ? 1 : 0;
            }
        }
        ++cs.it;
        if (cs.it >= W + S && cs.mode == MODE_STEP) cs.mode = -1;
    }
    if (wr && lane == 0) {
        if (P.accept_rate) P.accept_rate[ci0] = S > 0 ? cs.asum / (float)S : 0.f;
        if (P.step_size) P.step_size[ci0] = cs.eps;
        if (P.n_div) P.n_div[ci0] = cs.ndiv;
        if (P.n_grad) P.n_grad[ci0] = ngrad;
    }
    if (wr && P.inv_mass && own) P.inv_mass[ci0 * 6 + pi] = im;
}

// Serving: copy n elements at src (this CTA's galaxy's outputs) to the
// pinned mirror, src + pub_shift.
template <typename T>
__device__ __forceinline__ void publish_range(const T *src, size_t n, long long shift)
{
    if (!src) return;
    T *dst = reinterpret_cast<T *>(reinterpret_cast<char *>(const_cast<T *>(src)) + shift);
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// All threads of the CTA, after the galaxy's chains have finished: its
// outputs go to the host mirror, then done[gal] is raised.  Each thread
// fences its own stores at system scope before the barrier, so the host that
// sees the flag sees every result.
__device__ void publish_galaxy(const FitParams &P, int gal)
{
    const size_t C = P.n_chains, cs = C * P.n_samples;
    const size_t plane = (size_t)P.n_gal * cs;
    const long long sh = P.pub_shift;
    for (int k = 0; k < 6; ++k) publish_range(P.samples + k * plane + gal * cs, cs, sh);
    if (P.logp) publish_range(P.logp + gal * cs, cs, sh);
    if (P.accepted) publish_range(P.accepted + gal * cs, cs, sh);
    if (P.accept_rate) publish_range(P.accept_rate + gal * C, C, sh);
    if (P.step_size) publish_range(P.step_size + gal * C, C, sh);
    if (P.inv_mass) publish_range(P.inv_mass + gal * C * 6, C * 6, sh);
    if (P.n_div) publish_range(P.n_div + gal * C, C, sh);
    if (P.n_grad) publish_range(P.n_grad + gal * C, C, sh);
    if (P.status) publish_range(P.status + gal, 1, sh);
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence_system();
        *reinterpret_cast<volatile uint32_t *>(P.done + gal) = 1u;
    }
}

// The persistent fit loop of one CTA (all threads).
template <int NC, int PROF>
__device__ __forceinline__ void fit_loop(const FitParams &P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_gal, s_grp;
    const int cc = cta_chains(P);              // chains of this CTA
    const int groups = cta_groups(P);          // CTAs a galaxy's chains are split over
    // the pixel path: two chains per CTA, each run by a group of four warps (a phase
    // table per group)
    const SmemView sm = smem_view(smem_raw, P.h_max, P.npad, P.max_side, PROF == 3 ? 2 : cc);
    const int warp = threadIdx.x >> 5;
    if constexpr (PROF == 3) pix_tc_begin(pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side));
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0) {
            s_grp = 0;
            if (P.done) {
                // serving: galaxy blockIdx.x only, so that nothing of the
                // launch's memory is touched after its completion flag
                s_gal = first ? (int)blockIdx.x : -1;
            } else {
                // items (position in the work list, chain group), or galaxy
                // indices when there is no list
                const int q = (int)atomicAdd(P.queue, 1u);
                const int wq = q / groups;
                s_gal = q < P.n_work * groups ? (P.work ? P.work[wq] : wq) : -1;
                s_grp = q - wq * groups;
            }
        }
        first = false;
        __syncthreads();
        const int gal = s_gal;
        if (gal < 0 || gal >= P.n_gal) break;
        if (!side_ok(P, P.side[gal])) {     // uniform across the CTA
            if (threadIdx.x == 0 && P.status) P.status[gal] = 2;
            __syncthreads();
            if (P.done) publish_galaxy(P, gal);
            continue;
        }
        GalCtx gc;
        if (!setup_galaxy(P, gal, sm, gc)) {
            if (threadIdx.x == 0 && P.status) P.status[gal] = 3;
            __syncthreads();
            if (P.done) publish_galaxy(P, gal);
            continue;
        }
        if constexpr (PROF == 3) {
            const PixTc px = pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side);
            if (threadIdx.x == 0) px.done[0] = px.done[1] = 0;
            pix_tc_setup(P, gc, sm, px, gal);
            const int grp = warp >> 2, chain = 2 * s_grp + grp;
            float vcol[NC];
#pragma unroll
            for (int j = 0; j < NC; ++j) vcol[j] = (float)((threadIdx.x & 31) + 32 * j - gc.c);
            float4 *xph = sm.xph + (size_t)grp * phase_stride(P.h_max);
            if (chain < P.n_chains) run_chain<NC, PROF>(P, gc, sm, gal, chain, grp);
            pix_drain<NC>(P, gc, sm, gal, xph, vcol);
            __syncthreads();
            if (threadIdx.x == 0 && *px.abort && P.status) P.status[gal] = 4;
        } else {
            if constexpr (PROF == 4) dense_setup(P, gc, sm, cc);
            if (warp < cc) run_chain<NC, PROF>(P, gc, sm, gal, s_grp * cc + warp, warp);
        }
        __syncthreads();
        if (P.done) publish_galaxy(P, gal);
    }
    if constexpr (PROF == 3) pix_tc_end(pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side));
}

// Register budgets of the kernel instances (the launch bounds give ptxas the
// occupancy target): 128 registers, 4 CTAs of 4 chains per SM, no spills;
// at most 102 (5 CTAs; blocks of up to 4 chains only); at most 85 (6 CTAs,
// a few spills outside the half-plane loop).
template <int NC, int PROF>
__global__ void __launch_bounds__(256, 2) fit_kernel_r128(const FitParams P) { fit_loop<NC, PROF>(P); }
template <int NC, int PROF>
__global__ void __launch_bounds__(128, 5) fit_kernel_r96(const FitParams P) { fit_loop<NC, PROF>(P); }
template <int NC, int PROF>
__global__ void __launch_bounds__(256, 3) fit_kernel_r80(const FitParams P) { fit_loop<NC, PROF>(P); }
// The pixel path: two chains per CTA of eight warps; its tensor memory (the transforms'
// constants and accumulator: all 512 columns) allows one CTA per SM.
template <int NC>
__global__ void __launch_bounds__(tc::kThreads, 1) fit_kernel_pix(const FitParams P) { fit_loop<NC, 3>(P); }

// One CTA of 32 threads per point: stage the galaxy, then evaluate.
template <int NC, int PROF>
__device__ void point_eval(const FitParams &P, const GalCtx &gc, const SmemView &sm, int gal,
                           const float *theta, double *logp, float *grad)
{
    const int lane = threadIdx.x & 31;
    float vcol[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) vcol[j] = (float)(lane + 32 * j - gc.c);
    float th[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) th[i] = theta[i];
    double v = -INFINITY;
    float gl = NAN;   // the gradient's component for this lane's parameter (lanes < 6)
    if (in_support(P, th)) {
        if constexpr (PROF == 3) {
            float g[6];
            v = eval_pix<NC>(P, gc, sm, gal, sm.xph, vcol, th, g, true, nullptr);
            gl = pick6(g, lane < 6 ? lane : 5);
        } else if constexpr (PROF == 4) {
            v = eval_dense<NC>(P, gc, dense_view(sm.kxr, P.h_max, P.npad, P.max_side, 0), gal, sm.kxr, sm.xph, vcol,
                               th, gl, true);
        } else {
            v = eval_logpost<NC, PROF>(P, gc, sm.tab, sm.kxr, sm.xph, vcol, th, gl, true);
        }
    }
    if (threadIdx.x >= 32) return;   // the pixel path's other warps hold the same values
    if (lane == 0 && logp) *logp = v;
    if (grad && lane < 6) grad[lane] = gl;
}

template <int PROF>
__global__ void __launch_bounds__(32) logpost_points_kernel(const FitParams P, int n_points,
                                                            const int32_t *gal_index,
                                                            const float *theta, double *logp,
                                                            float *grad)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemView sm = smem_view(smem_raw, P.h_max, P.npad, P.max_side, 1);
    for (int i = blockIdx.x; i < n_points; i += gridDim.x) {
        const int gal = gal_index[i];
        if (gal < 0 || gal >= P.n_gal || !side_ok(P, P.side[gal])) {
            if (threadIdx.x == 0 && logp) logp[i] = NAN;
            if (grad && threadIdx.x < 6) grad[(size_t)i * 6 + threadIdx.x] = NAN;
            continue;
        }
        GalCtx gc;
        if (!setup_galaxy(P, gal, sm, gc)) {
            if (threadIdx.x == 0 && logp) logp[i] = NAN;
            if (grad && threadIdx.x < 6) grad[(size_t)i * 6 + threadIdx.x] = NAN;
            continue;
        }
        if constexpr (PROF == 4) dense_setup(P, gc, sm, 1);
        const float *th = theta + (size_t)i * 6;
        double *lp = logp ? logp + i : nullptr;
        float *gr = grad ? grad + (size_t)i * 6 : nullptr;
        switch (P.npad >> 5) {     // the table layout follows the launch's slot count
            case 1: point_eval<1, PROF>(P, gc, sm, gal, th, lp, gr); break;
            case 2: point_eval<2, PROF>(P, gc, sm, gal, th, lp, gr); break;
            case 3: point_eval<3, PROF>(P, gc, sm, gal, th, lp, gr); break;
            default: point_eval<4, PROF>(P, gc, sm, gal, th, lp, gr); break;
        }
        __syncthreads();
    }
}

// The pixel path's points: one CTA of eight warps per point; the first group of four
// warps evaluates it, the second joins with a skip flag.
template <int NC>
__global__ void __launch_bounds__(tc::kThreads, 1) logpost_points_pix_kernel(const FitParams P, int n_points,
                                                                            const int32_t *gal_index, const float *theta,
                                                                            double *logp, float *grad)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemView sm = smem_view(smem_raw, P.h_max, P.npad, P.max_side, 2);
    const PixTc px = pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side);
    pix_tc_begin(px);
    const int grp = threadIdx.x >> 7, lane = threadIdx.x & 31;
    for (int i = blockIdx.x; i < n_points; i += gridDim.x) {
        const int gal = gal_index[i];
        GalCtx gc;
        const bool ok = gal >= 0 && gal < P.n_gal && side_ok(P, P.side[gal]) && setup_galaxy(P, gal, sm, gc);
        if (!ok) {
            if (threadIdx.x == 0 && logp) logp[i] = NAN;
            if (grad && threadIdx.x < 6) grad[(size_t)i * 6 + threadIdx.x] = NAN;
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) px.done[0] = px.done[1] = 0;
        pix_tc_setup(P, gc, sm, px, gal);
        float vcol[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) vcol[j] = (float)(lane + 32 * j - gc.c);
        float4 *xph = sm.xph + (size_t)grp * phase_stride(P.h_max);
        if (grp == 0) {
            const float *th = theta + (size_t)i * 6;
            float t[6], g[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) t[k] = th[k];
            double v = -INFINITY;
            if (in_support(P, t)) {
                v = eval_pix<NC>(P, gc, sm, gal, xph, vcol, t, g, true, nullptr);
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) g[k] = NAN;
            }
            if (threadIdx.x == 0 && logp) logp[i] = v;
            if (grad && threadIdx.x < 6) grad[(size_t)i * 6 + threadIdx.x] = pick6(g, threadIdx.x);
        }
        pix_drain<NC>(P, gc, sm, gal, xph, vcol);
        __syncthreads();
    }
    pix_tc_end(px);
}

}  // namespace

}  // namespace bs

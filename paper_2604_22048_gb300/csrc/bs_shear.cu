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
// Each galaxy's K samples are read by a group of lanes: when K % 4 == 0 and the
// rows are 16-byte aligned, 4 lanes per galaxy read 12-sample chunks from tiles
// of 64 galaxies x 48 samples that the tensor memory accelerator streams into
// shared memory (without b), or from a per-lane cp.async ring (with b); otherwise
// 8 lanes per galaxy with scalar loads one chunk ahead.  The
// arithmetic runs on pairs of samples in packed FP32x2 instructions, x is
// kept in log2 units for the MUFU exp2, and the group keeps
// an online log-sum-exp (a reference log weight that may lag the running
// maximum by up to 32, sum of weights and weighted derivative sums), merged
// with shuffles.  Per-galaxy totals are
// accumulated in FP64 and written as per-block partials; a one-block kernel
// sums the partials in a fixed order (deterministic) and adds the
// per-galaxy constants.
#include <cmath>

#include <cuda.h>            // CUtensorMap and its enums (types only: the encoder is looked up at run time)
#include <cudaTypedefs.h>    // PFN_cuTensorMapEncodeTiled

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

// log2 of a galaxy's sum of weights (a normal positive float), once per galaxy:
// the exponent exactly and the mantissa's logarithm, in [-1, 0), to about
// 6e-8 by the accurate log2f.  The hardware approximation's absolute error
// (about 2^-22, the same sign for sums of the same size) would add up over
// 10^6 galaxies to a shift of the total of a few tenths of a nat.
__device__ __forceinline__ double log2_total(float x)
{
    int e;
    const float m = frexpf(x, &e);      // x = m 2^e, m in [0.5, 1)
    return (double)e + (double)log2f(m);
}

// Packed FP32x2 arithmetic: two samples per instruction, each half rounded
// like the scalar operation.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Per-launch constants in registers.
struct ShearConst {
    float2 g1, g2, ng1, ng2;         // g, -g
    float2 a2n, an, nan, nk;         // -a2 (log2 units), a = 1/(2 alpha^2), -a, -kappa
    float2 c0;                       // log2(e)/(2 sigma_e0^2)
    float2 gg, m2;                   // |g|^2, -2
    float r2;
};

__device__ __forceinline__ ShearConst shear_const(const ShearLaunch &s)
{
    ShearConst c;
    const float a = s.a2 * kLn2;
    c.g1 = f2(s.g1);
    c.g2 = f2(s.g2);
    c.ng1 = f2(-s.g1);
    c.ng2 = f2(-s.g2);
    c.a2n = f2(-s.a2);
    c.an = f2(a);
    c.nan = f2(-a);
    c.nk = f2(-s.kappa);
    c.c0 = f2(s.c0);
    c.gg = f2(s.g1 * s.g1 + s.g2 * s.g2);
    c.m2 = f2(-2.0f);
    c.r2 = s.r2;
    return c;
}

// Two samples: the weight split as exp2(x) f, with x = c0 |eps'|^2 -
// a2 Q (+ b log2 e) the exponent and f the power of U the log term stands for:
//   BA14:               -4 log2 U                    -> f = (1/U)^4
//   truncated Gaussian: -2 log2 U - 2 log2(1 - |eps'|^2) -> f = (1/(U (1 - |eps'|^2)))^2
// (f lies in about [0.004, 16], so it cannot overflow a weight; no logarithm
// per sample), and the factors of the derivatives,
//   dx/dg_i = -2 rU c_i,  c_i = du_i (a Q - kappa) - a n_i,  n = eps' - g,
//   du_i = eps'_i - g_i |eps'|^2  (-1/2 dU/dg_i),
// regrouped as c_i = eps'_i p - g_i r with p = a Q - kappa - a and
// r = |eps'|^2 (a Q - kappa) - a, so that a galaxy's weighted sum of c_i is
// sum(w rU p eps'_i) - g_i sum(w rU r): three running sums instead of two
// per-sample factors c_i (2 fewer packed operations per pair of samples);
// the -2 is applied once per galaxy.  U = |1 - conj(g) eps'|^2 is taken in the
// Lagrange form 1 - 2 g.eps' + |g|^2 |eps'|^2 (U is near 1: no cancellation);
// n is formed explicitly (not expanded through |eps'|^2 - 2 g.eps' + |g|^2,
// which cancels when eps' is near g).
template <int FAMILY, bool HAS_B>
__device__ __forceinline__ void pair_terms(const ShearConst &c, float2 e1, float2 e2, float2 bv, float2 &x,
                                           float2 &fw, float2 &ru, float2 &pp, float2 &rr, float2 &q)
{
    const float2 Ep = fma2(e1, e1, mul2(e2, e2));
    const float2 ge = fma2(c.g1, e1, mul2(c.g2, e2));            // g.eps'
    const float2 U = fma2(c.gg, Ep, fma2(c.m2, ge, f2(1.0f)));
    const float2 n1 = sub2(e1, c.g1), n2 = sub2(e2, c.g2);
    const float2 Nn = fma2(n1, n1, mul2(n2, n2));
    float2 rU, f;
    if (FAMILY == BS_EPRIOR_TRUNC_GAUSS) {
        const float2 om = sub2(f2(1.0f), Ep);
        const float2 uo = mul2(U, om);
        const float2 r = make_float2(rcp_ftz(uo.x), rcp_ftz(uo.y));   // 1 / (U (1 - |eps'|^2))
        rU = mul2(r, om);
        f = mul2(r, r);
    } else {
        rU = make_float2(rcp_ftz(U.x), rcp_ftz(U.y));
        const float2 r2 = mul2(rU, rU);
        f = mul2(r2, r2);
    }
    const float2 Q = mul2(Nn, rU);
    float2 xx = fma2(c.c0, Ep, mul2(c.a2n, Q));
    if (FAMILY == BS_EPRIOR_TRUNC_GAUSS) {
        if (!(Q.x < c.r2)) xx.x = -INFINITY;
        if (!(Q.y < c.r2)) xx.y = -INFINITY;
    }
    if (HAS_B) xx = fma2(f2(kLog2e), bv, xx);
    const float2 aqk = fma2(c.an, Q, c.nk);
    pp = add2(aqk, c.nan);
    rr = fma2(Ep, aqk, c.nan);
    fw = f;
    ru = rU;
    q = Q;
    x = xx;
}

// One chunk: 4 consecutive samples of this lane.
struct Chunk {
    float4 e1, e2, b;
    bool full;     // all four samples exist
    int nvalid;
};

// Scalar loads of one chunk (any K, any alignment); missing samples are zero.
template <bool HAS_B>
__device__ __forceinline__ void load_chunk(const ShearLaunch &s, long long base, int k0, int K, Chunk &ch)
{
    ch.nvalid = k0 < K ? min(4, K - k0) : 0;
    ch.full = ch.nvalid == 4;
    float t1[4] = {0.f, 0.f, 0.f, 0.f}, t2[4] = {0.f, 0.f, 0.f, 0.f}, tb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (r < ch.nvalid) {
            const long long j = base + k0 + r;
            t1[r] = __ldg(s.e1 + j);
            t2[r] = __ldg(s.e2 + j);
            if (HAS_B) tb[r] = __ldg(s.b + j);
        }
    }
    ch.e1 = make_float4(t1[0], t1[1], t1[2], t1[3]);
    ch.e2 = make_float4(t2[0], t2[1], t2[2], t2[3]);
    ch.b = make_float4(tb[0], tb[1], tb[2], tb[3]);
}

// Online log-sum-exp state of one lane (both halves share the maximum).
struct Lse {
    float m;
    float2 sw, t1, t2, tq;   // t_i: sum of weight rU p eps'_i
    float2 tr;               // sum of weight rU r
};

// Samples missing from a chunk (past K) get log weight -inf.
__device__ __forceinline__ void mask_missing(const Chunk &ch, float2 (&x)[2])
{
    if (ch.nvalid < 4) x[1].y = -INFINITY;
    if (ch.nvalid < 3) x[1].x = -INFINITY;
    if (ch.nvalid < 2) x[0].y = -INFINITY;
    if (ch.nvalid < 1) x[0].x = -INFINITY;
}

template <int FAMILY, bool HAS_B>
__device__ __forceinline__ void eval_chunk(const ShearConst &c, const Chunk &ch, Lse &L)
{
    float2 x[2], fw[2], ru[2], pp[2], rr[2], qq[2];
    const float2 e1[2] = {make_float2(ch.e1.x, ch.e1.y), make_float2(ch.e1.z, ch.e1.w)};
    const float2 e2[2] = {make_float2(ch.e2.x, ch.e2.y), make_float2(ch.e2.z, ch.e2.w)};
    const float2 bb[2] = {make_float2(ch.b.x, ch.b.y), make_float2(ch.b.z, ch.b.w)};
#pragma unroll
    for (int h = 0; h < 2; ++h)
        pair_terms<FAMILY, HAS_B>(c, e1[h], e2[h], bb[h], x[h], fw[h], ru[h], pp[h], rr[h], qq[h]);
    if (!ch.full) mask_missing(ch, x);
    // The weights are taken against the lane's reference L.m, which may lag the
    // largest log2 weight seen by up to 32 (weights below 2^32 f, so sums of any
    // realistic K stay finite), so that the exponentials need not wait for this
    // chunk's maximum; only a larger jump (the first chunk of a galaxy, whose
    // reference starts at -1e30) rescales the sums and recomputes the chunk's
    // weights (from the samples: the first pass's exponents are not kept).
    const float2 nm = f2(-L.m);
    float2 ew[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 d = add2(x[h], nm);
        ew[h] = mul2(make_float2(ex2_ftz(d.x), ex2_ftz(d.y)), fw[h]);
    }
    const float mloc = fmaxf(fmaxf(x[0].x, x[0].y), fmaxf(x[1].x, x[1].y));
    if (mloc - L.m > 32.0f) {
        const float2 sc = f2(ex2_ftz(L.m - mloc));
        L.sw = mul2(L.sw, sc);
        L.t1 = mul2(L.t1, sc);
        L.t2 = mul2(L.t2, sc);
        L.tq = mul2(L.tq, sc);
        L.tr = mul2(L.tr, sc);
        L.m = mloc;
        float2 x2[2], f2w[2], u0, u1, u2, u3;
#pragma unroll
        for (int h = 0; h < 2; ++h) pair_terms<FAMILY, HAS_B>(c, e1[h], e2[h], bb[h], x2[h], f2w[h], u0, u1, u2, u3);
        if (!ch.full) mask_missing(ch, x2);
        const float2 nl = f2(-mloc);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 d = add2(x2[h], nl);
            ew[h] = mul2(make_float2(ex2_ftz(d.x), ex2_ftz(d.y)), f2w[h]);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 e = ew[h];
        const float2 er = mul2(e, ru[h]);
        const float2 erp = mul2(er, pp[h]);
        L.sw = add2(L.sw, e);
        L.t1 = fma2(erp, e1[h], L.t1);
        L.t2 = fma2(erp, e2[h], L.t2);
        L.tr = fma2(er, rr[h], L.tr);
        L.tq = fma2(e, qq[h], L.tq);
    }
}

// Merge the lanes of a galaxy's group and add the galaxy's log-sum-exp and
// softmax-weighted derivative sums, times the galaxy's weight w[n] (1 when w
// is NULL; a zero weight drops the galaxy), to the lane-0 accumulators; (g1, g2)
// is the shear of the evaluation.
template <int G = kGroup>
__device__ __forceinline__ void finish_galaxy(const Lse &L, float g1, float g2, unsigned gmask, int sub,
                                              const float *w, long long n, double &av, double &a1, double &a2,
                                              double &aq)
{
    float m = L.m;
    const float tr = L.tr.x + L.tr.y;
    float sw = L.sw.x + L.sw.y, tq = L.tq.x + L.tq.y;
    float t1 = fmaf(-g1, tr, L.t1.x + L.t1.y), t2 = fmaf(-g2, tr, L.t2.x + L.t2.y);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float mo = __shfl_xor_sync(gmask, m, o, G);
        const float so = __shfl_xor_sync(gmask, sw, o, G);
        const float o1 = __shfl_xor_sync(gmask, t1, o, G);
        const float o2 = __shfl_xor_sync(gmask, t2, o, G);
        const float oq = __shfl_xor_sync(gmask, tq, o, G);
        const float mn = fmaxf(m, mo);
        const float ca = ex2_ftz(m - mn), cb = ex2_ftz(mo - mn);
        sw = sw * ca + so * cb;
        t1 = t1 * ca + o1 * cb;
        t2 = t2 * ca + o2 * cb;
        tq = tq * ca + oq * cb;
        m = mn;
    }
    if (sub == 0) {
        const double wn = w ? (double)__ldg(w + n) : 1.0;
        if (wn == 0.0) return;
        if (sw > 0.f) {
            const float inv = 1.0f / sw;
            av += wn * ((double)m + log2_total(sw));
            a1 += wn * (double)(-2.0f * t1 * inv);
            a2 += wn * (double)(-2.0f * t2 * inv);
            aq += wn * (double)(tq * inv);
        } else {
            av = -INFINITY;
        }
    }
}

__device__ __forceinline__ void lse_reset(Lse &L)
{
    L.m = -1e30f;
    L.sw = L.t1 = L.t2 = L.tq = L.tr = f2(0.f);
}

// Block reduction of the four FP64 accumulators into this block's partials.
__device__ __forceinline__ void block_partials(const ShearLaunch &s, double av, double a1, double a2, double aq)
{
    __shared__ double red[kShearThreads / 32][4];
    const int lane = threadIdx.x & 31;
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

// Any K and alignment: scalar loads into two register buffers in turn (the
// next chunk's loads in flight while the current one is evaluated).
template <int FAMILY, bool HAS_B>
__global__ void __launch_bounds__(kShearThreads, 3) shear_kernel(const ShearLaunch s)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kGroup - 1);
    const unsigned gmask = 0xFFu << (lane & ~(kGroup - 1));
    const long long group = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    const long long ngroups = (long long)gridDim.x * blockDim.x / kGroup;
    const ShearConst c = shear_const(s);
    const int K = s.K;
    double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;

    for (long long n = group; n < s.n_gal; n += ngroups) {
        const long long base = n * (long long)K;
        Lse L;
        lse_reset(L);
        Chunk A, B;
        int k0 = 4 * sub;
        load_chunk<HAS_B>(s, base, k0, K, A);
        for (;;) {
            if (k0 >= K) break;
            load_chunk<HAS_B>(s, base, k0 + 4 * kGroup, K, B);
            eval_chunk<FAMILY, HAS_B>(c, A, L);
            k0 += 4 * kGroup;
            if (k0 >= K) break;
            load_chunk<HAS_B>(s, base, k0 + 4 * kGroup, K, A);
            eval_chunk<FAMILY, HAS_B>(c, B, L);
            k0 += 4 * kGroup;
        }
        finish_galaxy(L, s.g1, s.g2, gmask, sub, s.w, n, av, a1, a2, aq);
    }
    block_partials(s, av, a1, a2, aq);
}

// Asynchronous 16-byte global -> shared copies (L2 only), grouped per chunk.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 4 lanes per galaxy and 12-sample chunks: a group spans 48 samples per step
// (336 slots for K = 300), the ring's per-chunk bookkeeping is shared by 12
// samples per lane.  Launch bounds for 3 CTAs (24 warps) per SM leave 80
// registers, so that the chunk's exponentials and sums are not serialised for
// lack of them (measured with the tile-streamed kernel below: 2,080 passes/s
// against 1,993 at 4 CTAs and 64 registers and 1,934 at 2 CTAs).  Measured on
// one GPU for this kernel at 4 CTAs: 8 lanes x 8 samples x 3 stages (3 CTAs)
// 1,793 passes/s, 4 x 16 x 2 (3 CTAs) 1,864, 4 x 8 x 2 1,883, 4 x 12 x 2 1,904.
constexpr int kAGroup = 4;     // lanes per galaxy
constexpr int kStages = 2;     // chunks per lane in flight, this one included
constexpr int kAsyncBlocks = 3;   // CTAs per SM the launch bounds target (80 registers)
constexpr int kChunk = 12;     // samples per lane per chunk (kChunk / 4 16-byte copies per array)
constexpr int kQuads = kChunk / 4;

__host__ __device__ constexpr size_t async_smem_bytes(bool has_b)
{
    return (size_t)kStages * (has_b ? 3 : 2) * kQuads * kShearThreads * sizeof(float4);
}

// K % 4 == 0 and 16-byte aligned rows: each lane streams its 12-sample chunks
// through a kStages-deep ring of its own shared-memory slots with cp.async,
// over the flattened sequence (galaxy, chunk) of its group, so the pipeline
// does not drain between galaxies.  A lane only reads the slots it filled,
// after cp.async.wait_group; no barrier is needed.
template <int FAMILY, bool HAS_B>
__global__ void __launch_bounds__(kShearThreads, HAS_B ? 3 : kAsyncBlocks) shear_kernel_async(const ShearLaunch s)
{
    extern __shared__ float4 sbuf[];
    constexpr int NV = HAS_B ? 3 : 2;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int sub = lane & (kAGroup - 1);
    const unsigned gmask = ((1u << kAGroup) - 1u) << (lane & ~(kAGroup - 1));
    const long long group = ((long long)blockIdx.x * blockDim.x + tid) / kAGroup;
    const long long ngroups = (long long)gridDim.x * blockDim.x / kAGroup;
    const ShearConst c = shear_const(s);
    const int K = s.K;
    constexpr int span = kChunk * kAGroup;                   // samples of a group per chunk step
    const int cpg = (K + span - 1) / span;                   // chunks per galaxy per lane
    const long long my_gal = group < s.n_gal ? (s.n_gal - 1 - group) / ngroups + 1 : 0;
    const long long n_items = my_gal * cpg;
    double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;
    // slot (stage, array, half) of this thread
    auto slot = [&](int st, int arr, int q) -> float4 * {
        return &sbuf[((st * NV + arr) * kQuads + q) * kShearThreads + tid];
    };

    // issuer position: galaxy, chunk, ring slot
    long long in = group;
    int ic = 0, ist = 0;
    auto issue = [&]() {
        if (in < s.n_gal) {
            const int k0 = kChunk * sub + span * ic;
            const long long off = in * (long long)K + k0;
#pragma unroll
            for (int h = 0; h < kQuads; ++h) {
                if (k0 + 4 * h < K) {
                    cp_async16(slot(ist, 0, h), s.e1 + off + 4 * h);
                    cp_async16(slot(ist, 1, h), s.e2 + off + 4 * h);
                    if (HAS_B) cp_async16(slot(ist, 2, h), s.b + off + 4 * h);
                }
            }
            if (++ic == cpg) {
                ic = 0;
                in += ngroups;
            }
        }
        cp_async_commit();
        ist = ist + 1 == kStages ? 0 : ist + 1;
    };
#pragma unroll
    for (int t = 0; t < kStages - 1; ++t) issue();

    Lse L;
    lse_reset(L);
    int cc = 0, cst = 0;     // consumer: chunk within the galaxy, ring slot
    long long cn = group;    // consumer galaxy
    for (long long t = 0; t < n_items; ++t) {
        issue();
        cp_async_wait<kStages - 1>();
        const int k0 = kChunk * sub + span * cc;
#pragma unroll
        for (int h = 0; h < kQuads; ++h) {
            Chunk ch;
            ch.nvalid = k0 + 4 * h < K ? 4 : 0;
            ch.full = ch.nvalid == 4;
            if (ch.full) {
                ch.e1 = *slot(cst, 0, h);
                ch.e2 = *slot(cst, 1, h);
                ch.b = HAS_B ? *slot(cst, 2, h) : make_float4(0.f, 0.f, 0.f, 0.f);
                eval_chunk<FAMILY, HAS_B>(c, ch, L);
            }
        }
        cst = cst + 1 == kStages ? 0 : cst + 1;
        if (++cc == cpg) {
            cc = 0;
            finish_galaxy<kAGroup>(L, s.g1, s.g2, gmask, sub, s.w, cn, av, a1, a2, aq);
            cn += ngroups;
            lse_reset(L);
        }
    }
    cp_async_wait<0>();
    block_partials(s, av, a1, a2, aq);
}

// ---- Tensor-memory-accelerator tiles (no b): a CTA streams tiles of kTileG
// consecutive galaxies x kTileK samples of e1 and e2 with 2-D
// cp.async.bulk.tensor loads into a kTmaStages-deep ring; one thread issues both
// loads of a stage and arms the stage's mbarrier with their byte count, and the
// others wait on it.  Thread t serves galaxy t / 4 of the tile and its samples
// [12 (t mod 4), + 12) of each chunk (the cp.async kernel's group of 4 lanes and
// 12-sample chunks).  Galaxies past n_gal and samples past K arrive zero-filled and
// are masked by index.  A wait gives up after two seconds: the CTA then writes NaN
// partials, so that the pass's value is NaN.
constexpr int kTileG = kShearThreads / kAGroup;   // 64 galaxies per tile
constexpr int kTileK = kChunk * kAGroup;          // 48 samples per chunk
constexpr int kTmaStages = 3;
constexpr int kTileFloats = kTileG * kTileK;      // one array's box, 12 KB

__host__ __device__ constexpr size_t tma_smem_bytes()
{
    return (size_t)kTmaStages * 2 * kTileFloats * sizeof(float) + 128;   // + alignment of the ring
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait for the phase of the given parity.  Each try_wait may suspend the warp
// in hardware for up to 20 us until the phase completes (no busy loop taking
// issue slots from the computing warps); the limit is checked between tries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t t0)
{
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) return false;
    }
}

// The CTA's ring of kTmaStages stages, each one tile-chunk of e1 and e2, with a
// "full" mbarrier per stage (armed by the producer with the stage's byte count) and an
// "empty" one (one arrival per warp once the warp has read the stage).  Thread 0 is
// the producer: it issues item i (tile blockIdx.x + t gridDim.x, chunk c) after the
// stage's previous item has been released.  Every wait gives up after two seconds.
struct TmaRing {
    float *ring;
    uint64_t *full, *empty;
    int cpg, n_items;
    // producer state (thread 0): next item to load, its tile and chunk
    int p_item = 0, p_chunk = 0;
    long long p_tile;
    bool p_ok = true;

    __device__ void init(unsigned char *raw, uint64_t *f, uint64_t *e, long long n_gal, int K)
    {
        constexpr int kWarps = kShearThreads / 32;
        ring = reinterpret_cast<float *>(raw + ((128u - (smem_u32(raw) & 127u)) & 127u));
        full = f;
        empty = e;
        cpg = (K + kTileK - 1) / kTileK;   // chunks per tile
        const long long n_tiles = (n_gal + kTileG - 1) / kTileG;
        const int my_tiles = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
        n_items = my_tiles * cpg;
        p_tile = blockIdx.x;
        if (threadIdx.x == 0) {
            for (int st = 0; st < kTmaStages; ++st) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[st])), "r"(kWarps)
                             : "memory");
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    __device__ void issue(const CUtensorMap *m1, const CUtensorMap *m2)
    {
        if (p_item >= n_items || !p_ok) return;
        const int st = p_item % kTmaStages;
        if (p_item >= kTmaStages) {   // the stage's previous item has been read by every warp
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)((p_item / kTmaStages - 1) & 1), t0)) {
                p_ok = false;
                return;
            }
        }
        const uint32_t bar = smem_u32(&full[st]);
        const uint32_t d1 = smem_u32(ring + (size_t)st * 2 * kTileFloats), d2 = d1 + kTileFloats * 4;
        const int x = p_chunk * kTileK, y = (int)(p_tile * kTileG);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)(2 * kTileFloats * 4))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                "r"(d1),
            "l"(m1), "r"(x), "r"(y), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                "r"(d2),
            "l"(m2), "r"(x), "r"(y), "r"(bar)
            : "memory");
        ++p_item;
        if (++p_chunk == cpg) {
            p_chunk = 0;
            p_tile += gridDim.x;
        }
    }
    // all threads: wait until item's stage has landed (false, in every lane, on a timeout)
    __device__ bool wait_full(int item) const
    {
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        return __all_sync(BS_FULL_MASK,
                          mbar_wait(smem_u32(&full[item % kTmaStages]), (uint32_t)((item / kTmaStages) & 1), t0));
    }
    // all threads of a warp, after reading item's stage
    __device__ void release(int item) const
    {
        __syncwarp();
        if ((threadIdx.x & 31) == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[item % kTmaStages]))
                         : "memory");
    }
    // all threads, at the end: loads still in flight land in the ring (waited for, with the limit)
    __device__ void drain() const
    {
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            for (int it = p_item - kTmaStages; it < p_item; ++it)
                if (it >= 0) mbar_wait(smem_u32(&full[it % kTmaStages]), (uint32_t)((it / kTmaStages) & 1), t1);
        }
    }
};

// Quad h (4 consecutive samples) of this thread's part of chunk `chunk` of its
// galaxy (4 lanes per galaxy, 12 samples each) in item's stage; false past K.
__device__ __forceinline__ bool tma_quad(const TmaRing &R, int item, int K, int chunk, int h, Chunk &ch)
{
    const int tid = threadIdx.x, sub = tid & (kAGroup - 1), gl = tid / kAGroup;
    if (chunk * kTileK + kChunk * sub + 4 * h >= K) return false;
    const float *r1 = R.ring + (size_t)(item % kTmaStages) * 2 * kTileFloats + gl * kTileK + kChunk * sub + 4 * h;
    ch.nvalid = 4;
    ch.full = true;
    ch.e1 = *reinterpret_cast<const float4 *>(r1);
    ch.e2 = *reinterpret_cast<const float4 *>(r1 + kTileFloats);
    ch.b = make_float4(0.f, 0.f, 0.f, 0.f);
    return true;
}

template <int FAMILY>
__global__ void __launch_bounds__(kShearThreads, kAsyncBlocks)
    shear_kernel_tma(const ShearLaunch s, const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap m2)
{
    extern __shared__ __align__(128) unsigned char tma_raw[];
    __shared__ __align__(8) uint64_t full[kTmaStages], empty[kTmaStages];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int sub = tid & (kAGroup - 1), gl = tid / kAGroup;
    const unsigned gmask = ((1u << kAGroup) - 1u) << (lane & ~(kAGroup - 1));
    const ShearConst c = shear_const(s);
    const int K = s.K;
    TmaRing R;
    R.init(tma_raw, full, empty, s.n_gal, K);
    if (tid == 0)
        for (int t = 0; t < kTmaStages - 1; ++t) R.issue(&m1, &m2);
    double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;
    Lse L;
    lse_reset(L);
    bool failed = false;
    int chunk = 0;
    long long tile = blockIdx.x;
    for (int item = 0; item < R.n_items; ++item) {
        if (tid == 0) R.issue(&m1, &m2);
        if (!R.wait_full(item)) {
            failed = true;
            break;
        }
        const long long n = tile * kTileG + gl;
        if (n < s.n_gal) {
#pragma unroll
            for (int h = 0; h < kQuads; ++h) {
                Chunk ch;
                if (tma_quad(R, item, K, chunk, h, ch)) eval_chunk<FAMILY, false>(c, ch, L);
            }
        }
        R.release(item);
        if (++chunk == R.cpg) {
            if (n < s.n_gal) finish_galaxy<kAGroup>(L, s.g1, s.g2, gmask, sub, s.w, n, av, a1, a2, aq);
            lse_reset(L);
            chunk = 0;
            tile += gridDim.x;
        }
    }
    if (failed || (tid == 0 && !R.p_ok)) av = a1 = a2 = aq = NAN;
    R.drain();
    block_partials(s, av, a1, a2, aq);
}

// The tensor-map encoder of the driver, looked up once through the runtime
// (no link to the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// A [n_gal][K] FP32 row-major array as a 2-D tensor map with kTileK x kTileG boxes.
bool make_sample_map(CUtensorMap &m, const float *base, long long n_gal, int K)
{
    auto enc = tensor_map_encoder();
    if (!enc || n_gal <= 0 || n_gal > 0xFFFFFFFFll) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n_gal};
    const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileG};
    const cuuint32_t estr[2] = {1, 1};
    return enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

// ---- all properties free ----------------------------------------------------

// log Phi(t) and the inverse Mills ratio phi(t)/Phi(t) of the standard normal,
// through erfcx on the left tail so that neither underflows.
__device__ __forceinline__ void log_ndtr_mills(float t, float &lphi, float &r)
{
    if (t < 0.0f) {
        const float u = -t * 0.70710678118654752f;
        const float ex = erfcxf(u);                 // exp(u^2) erfc(u)
        lphi = logf(0.5f * ex) - u * u;
        r = 0.79788456080286536f / ex;              // sqrt(2/pi) / erfcx
    } else {
        const float q = 0.5f * erfcf(t * 0.70710678118654752f);   // 1 - Phi(t)
        lphi = log1pf(-q);
        r = 0.39894228040143268f * expf(-0.5f * t * t) / (1.0f - q);
    }
}

struct FullAcc {
    float m, sw, t1, t2, tq, h[5];
};

// One sample: log2 weight of the ellipticity part (as pair_terms, scalar) plus
// the flux/size log prior ratio up to per-galaxy constants,
//   -z^2/2 + log Phi(a z) - y^2/2,  z = (lf - mu_f)/sigma_f, y = (ls - mu_s)/sigma_s,
// and the factors of its derivatives (times sigma where that is constant):
//   (z - a r), z (z - a r), r z, y, y^2,  r = phi(a z)/Phi(a z).
template <int FAMILY>
__device__ __forceinline__ void full_sample(const ShearFullLaunch &f, float an, float e1, float e2, float lf,
                                            float ls, bool valid, FullAcc &A)
{
    const ShearLaunch &s = f.s;
    const float Ep = fmaf(e1, e1, e2 * e2);
    const float ge = fmaf(s.g1, e1, s.g2 * e2);
    const float U = fmaf(s.g1 * s.g1 + s.g2 * s.g2, Ep, fmaf(-2.0f, ge, 1.0f));   // Lagrange form
    const float n1 = e1 - s.g1, n2 = e2 - s.g2;
    const float rU = rcp_ftz(U);
    const float Q = fmaf(n1, n1, n2 * n2) * rU;
    const float larg = FAMILY == BS_EPRIOR_TRUNC_GAUSS ? U * (1.0f - Ep) : U;
    const float lgk = FAMILY == BS_EPRIOR_TRUNC_GAUSS ? -2.0f : -s.kappa;
    float x = fmaf(s.c0, Ep, fmaf(lgk, lg2_ftz(larg), -s.a2 * Q));
    if (FAMILY == BS_EPRIOR_TRUNC_GAUSS && !(Q < s.r2)) x = -INFINITY;
    const float aqk = fmaf(an, Q, -s.kappa);
    const float du1 = fmaf(-s.g1, Ep, e1);
    const float du2 = fmaf(-s.g2, Ep, e2);
    const float c1 = fmaf(du1, aqk, -an * n1);
    const float c2 = fmaf(du2, aqk, -an * n2);
    const float z = (lf - f.mu_f) * f.inv_sf;
    const float y = (ls - f.mu_s) * f.inv_ss;
    float lphi, r;
    log_ndtr_mills(f.a_f * z, lphi, r);
    x = fmaf(kLog2e, lphi - 0.5f * fmaf(z, z, y * y), x);
    if (!valid) x = -INFINITY;
    if (x > A.m) {
        const float sc = ex2_ftz(A.m - x);
        A.sw *= sc;
        A.t1 *= sc;
        A.t2 *= sc;
        A.tq *= sc;
#pragma unroll
        for (int i = 0; i < 5; ++i) A.h[i] *= sc;
        A.m = x;
    }
    const float e = ex2_ftz(x - A.m);
    const float er = e * rU;
    const float h0 = fmaf(-f.a_f, r, z);
    A.sw += e;
    A.t1 = fmaf(er, c1, A.t1);
    A.t2 = fmaf(er, c2, A.t2);
    A.tq = fmaf(e, Q, A.tq);
    A.h[0] = fmaf(e, h0, A.h[0]);
    A.h[1] = fmaf(e, z * h0, A.h[1]);
    A.h[2] = fmaf(e, r * z, A.h[2]);
    A.h[3] = fmaf(e, y, A.h[3]);
    A.h[4] = fmaf(e, y * y, A.h[4]);
}

template <int FAMILY>
__global__ void __launch_bounds__(kShearThreads, 2) shear_full_kernel(const ShearFullLaunch f)
{
    const ShearLaunch &s = f.s;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kGroup - 1);
    const unsigned gmask = 0xFFu << (lane & ~(kGroup - 1));
    const long long group = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    const long long ngroups = (long long)gridDim.x * blockDim.x / kGroup;
    const float an = s.a2 * kLn2;
    const int K = s.K;
    double acc[kShearFullOut];
#pragma unroll
    for (int i = 0; i < kShearFullOut; ++i) acc[i] = 0.0;

    for (long long n = group; n < s.n_gal; n += ngroups) {
        const long long base = n * (long long)K;
        FullAcc A;
        A.m = -1e30f;
        A.sw = A.t1 = A.t2 = A.tq = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) A.h[i] = 0.f;
        for (int k = sub; k < K; k += kGroup) {
            const long long j = base + k;
            full_sample<FAMILY>(f, an, __ldg(s.e1 + j), __ldg(s.e2 + j), __ldg(f.lf + j), __ldg(f.ls + j), true, A);
        }
        // merge the 8 lanes of the group
        float v[10] = {A.m, A.sw, A.t1, A.t2, A.tq, A.h[0], A.h[1], A.h[2], A.h[3], A.h[4]};
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) {
            float w[10];
#pragma unroll
            for (int i = 0; i < 10; ++i) w[i] = __shfl_xor_sync(gmask, v[i], o, kGroup);
            const float mn = fmaxf(v[0], w[0]);
            const float ca = ex2_ftz(v[0] - mn), cb = ex2_ftz(w[0] - mn);
#pragma unroll
            for (int i = 1; i < 10; ++i) v[i] = v[i] * ca + w[i] * cb;
            v[0] = mn;
        }
        const double wn = sub == 0 && s.w ? (double)__ldg(s.w + n) : 1.0;
        if (sub == 0 && wn != 0.0) {
            if (v[1] > 0.f) {
                const float inv = 1.0f / v[1];
                acc[0] += wn * ((double)v[0] + log2_total(v[1]));
                acc[1] += wn * (double)(-2.0f * v[2] * inv);
                acc[2] += wn * (double)(-2.0f * v[3] * inv);
                acc[3] += wn * (double)(v[4] * inv);
#pragma unroll
                for (int i = 0; i < 5; ++i) acc[4 + i] += wn * (double)(v[5 + i] * inv);
            } else {
                acc[0] = -INFINITY;
            }
        }
    }
    __shared__ double red[kShearThreads / 32][kShearFullOut];
#pragma unroll
    for (int i = 0; i < kShearFullOut; ++i) acc[i] = warp_sum_d(acc[i]);
    const int w = threadIdx.x >> 5;
    if (lane == 0)
        for (int i = 0; i < kShearFullOut; ++i) red[w][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < kShearFullOut) {
        double t = 0.0;
        for (int i = 0; i < kShearThreads / 32; ++i) t += red[i][threadIdx.x];
        s.partials[(size_t)blockIdx.x * kShearFullOut + threadIdx.x] = t;
    }
}

struct FinalizeN {
    double scale[kShearFullOut], add[kShearFullOut];
};

__global__ void __launch_bounds__(256) shear_finalize_n_kernel(const double *partials, int n_part, int n_out,
                                                                FinalizeN c, double *out)
{
    __shared__ double red[256];
    for (int k = 0; k < n_out; ++k) {
        double t = 0.0;
        for (int i = threadIdx.x; i < n_part; i += blockDim.x) t += partials[(size_t)i * n_out + k];
        red[threadIdx.x] = t;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = red[0] * c.scale[k] + c.add[k];
        __syncthreads();
    }
}

template <int FAMILY, bool HAS_B>
cudaError_t launch_fb(const ShearLaunch &s, int grid, bool vec, cudaStream_t st)
{
    if (vec && !HAS_B) {
        // e1, e2 as tensor maps, streamed in tiles by the tensor memory accelerator
        CUtensorMap m1, m2;
        if (make_sample_map(m1, s.e1, s.n_gal, s.K) && make_sample_map(m2, s.e2, s.n_gal, s.K)) {
            const cudaError_t e = cudaFuncSetAttribute(shear_kernel_tma<FAMILY>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)tma_smem_bytes());
            if (e != cudaSuccess) return e;
            shear_kernel_tma<FAMILY><<<grid, kShearThreads, tma_smem_bytes(), st>>>(s, m1, m2);
            return cudaGetLastError();
        }
    }
    if (vec) {
        // the ring (48 KB, 72 KB with b) plus the static reduction buffer is
        // above the default dynamic shared-memory limit
        const cudaError_t e = cudaFuncSetAttribute(shear_kernel_async<FAMILY, HAS_B>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)async_smem_bytes(HAS_B));
        if (e != cudaSuccess) return e;
        shear_kernel_async<FAMILY, HAS_B><<<grid, kShearThreads, async_smem_bytes(HAS_B), st>>>(s);
    } else
        shear_kernel<FAMILY, HAS_B><<<grid, kShearThreads, 0, st>>>(s);
    return cudaGetLastError();
}

// ---- Several points per pass.  One read of the samples serves up to
// kMultiPoints (g1, g2, alpha) points: each sample's weight and derivative
// factors are formed for every point (the same per-sample arithmetic as
// shear_kernel), so the pass turns from HBM-bound into ALU-bound; the shear
// estimate's batches (central differences of its Hessian, Gauss-Hermite nodes)
// then cost about their arithmetic alone.  A galaxy group's FP64 totals go to
// its own shared-memory slot (one writer), summed over the block in a fixed
// order; partials are laid out per point so that each point is finalized as
// a single-point pass.
__device__ __forceinline__ ShearConst shear_const_point(const ShearMultiLaunch &m, int p)
{
    ShearLaunch s = m.s;
    s.g1 = m.g1[p];
    s.g2 = m.g2[p];
    s.a2 = m.a2[p];
    return shear_const(s);
}

template <int FAMILY>
__global__ void __launch_bounds__(kShearThreads, 2) shear_kernel_multi(const ShearMultiLaunch m)
{
    constexpr int NP = kMultiPoints;
    constexpr int kGroups = kShearThreads / kGroup;
    __shared__ double acc[kGroups][NP][4];
    const ShearLaunch &s = m.s;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kGroup - 1);
    const int gi = threadIdx.x / kGroup;
    const unsigned gmask = 0xFFu << (lane & ~(kGroup - 1));
    const long long group = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    const long long ngroups = (long long)gridDim.x * blockDim.x / kGroup;
    const int K = s.K;
    if (sub == 0)
        for (int p = 0; p < NP; ++p)
            for (int i = 0; i < 4; ++i) acc[gi][p][i] = 0.0;

    for (long long n = group; n < s.n_gal; n += ngroups) {
        const long long base = n * (long long)K;
        Lse L[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) lse_reset(L[p]);
        Chunk A, B;
        int k0 = 4 * sub;
        auto eval_all = [&](const Chunk &ch) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
                if (p < m.n_points) eval_chunk<FAMILY, false>(shear_const_point(m, p), ch, L[p]);
        };
        load_chunk<false>(s, base, k0, K, A);
        for (;;) {
            if (k0 >= K) break;
            load_chunk<false>(s, base, k0 + 4 * kGroup, K, B);
            eval_all(A);
            k0 += 4 * kGroup;
            if (k0 >= K) break;
            load_chunk<false>(s, base, k0 + 4 * kGroup, K, A);
            eval_all(B);
            k0 += 4 * kGroup;
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (p < m.n_points) {
                double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;
                finish_galaxy(L[p], m.g1[p], m.g2[p], gmask, sub, s.w, n, av, a1, a2, aq);
                if (sub == 0) {
                    acc[gi][p][0] += av;
                    acc[gi][p][1] += a1;
                    acc[gi][p][2] += a2;
                    acc[gi][p][3] += aq;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < NP * 4) {
        const int p = threadIdx.x >> 2, i = threadIdx.x & 3;
        double t = 0.0;
        for (int k = 0; k < kGroups; ++k) t += acc[k][p][i];
        m.partials[((size_t)p * gridDim.x + blockIdx.x) * 4 + i] = t;
    }
}

}  // namespace

int shear_grid_blocks()
{
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(shear_kernel_async<BS_EPRIOR_BA14, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)async_smem_bytes(false));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, shear_kernel_async<BS_EPRIOR_BA14, false>, kShearThreads,
                                                  async_smem_bytes(false));
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

int shear_full_grid_blocks()
{
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, shear_full_kernel<BS_EPRIOR_BA14>, kShearThreads, 0);
    if (sms <= 0) sms = 1;
    if (nb <= 0) nb = 1;
    return sms * nb;
}

cudaError_t launch_shear_full(const ShearFullLaunch &f, int grid, cudaStream_t stream)
{
    if (f.s.family == BS_EPRIOR_BA14)
        shear_full_kernel<BS_EPRIOR_BA14><<<grid, kShearThreads, 0, stream>>>(f);
    else
        shear_full_kernel<BS_EPRIOR_TRUNC_GAUSS><<<grid, kShearThreads, 0, stream>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_shear_finalize_n(const double *partials, int n_part, int n_out, const double *scale,
                                    const double *add, double *out, cudaStream_t stream)
{
    if (n_out < 1 || n_out > kShearFullOut) return cudaErrorInvalidValue;
    FinalizeN c;
    for (int i = 0; i < kShearFullOut; ++i) {
        c.scale[i] = i < n_out ? scale[i] : 0.0;
        c.add[i] = i < n_out ? add[i] : 0.0;
    }
    shear_finalize_n_kernel<<<1, 256, 0, stream>>>(partials, n_part, n_out, c, out);
    return cudaGetLastError();
}

int shear_multi_grid_blocks()
{
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, shear_kernel_multi<BS_EPRIOR_BA14>, kShearThreads, 0);
    if (sms <= 0) sms = 1;
    if (nb <= 0) nb = 1;
    return sms * nb;
}

// Several points per pass with the samples streamed in tiles (K a multiple of 4,
// 16-byte aligned rows, no b): the one-point tile kernel's ring and lane layout, each
// quad of samples evaluated for every point, each point keeping its own log-sum-exp
// state; a galaxy's 4 lanes put their FP64 totals per point in their own shared-memory
// slot, summed over the block in a fixed order.  On a wait that gives up, the block's
// partials are NaN.
template <int FAMILY>
__global__ void __launch_bounds__(kShearThreads, 2)
    shear_kernel_tma_multi(const ShearMultiLaunch m, const __grid_constant__ CUtensorMap m1,
                           const __grid_constant__ CUtensorMap m2)
{
    constexpr int NP = kMultiPoints;
    extern __shared__ __align__(128) unsigned char tma_raw[];
    __shared__ __align__(8) uint64_t full[kTmaStages], empty[kTmaStages];
    __shared__ double acc[kTileG][NP][4];
    __shared__ int s_fail;
    const ShearLaunch &s = m.s;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int sub = tid & (kAGroup - 1), gl = tid / kAGroup;
    const unsigned gmask = ((1u << kAGroup) - 1u) << (lane & ~(kAGroup - 1));
    const int K = s.K;
    if (sub == 0)
        for (int p = 0; p < NP; ++p)
            for (int i = 0; i < 4; ++i) acc[gl][p][i] = 0.0;
    if (tid == 0) s_fail = 0;
    TmaRing R;
    R.init(tma_raw, full, empty, s.n_gal, K);   // (its barrier also orders the resets above)
    if (tid == 0)
        for (int t = 0; t < kTmaStages - 1; ++t) R.issue(&m1, &m2);
    Lse L[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) lse_reset(L[p]);
    bool failed = false;
    int chunk = 0;
    long long tile = blockIdx.x;
    for (int item = 0; item < R.n_items; ++item) {
        if (tid == 0) R.issue(&m1, &m2);
        if (!R.wait_full(item)) {
            failed = true;
            break;
        }
        const long long n = tile * kTileG + gl;
        if (n < s.n_gal) {
#pragma unroll
            for (int h = 0; h < kQuads; ++h) {
                Chunk ch;
                if (tma_quad(R, item, K, chunk, h, ch)) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        if (p < m.n_points) eval_chunk<FAMILY, false>(shear_const_point(m, p), ch, L[p]);
                }
            }
        }
        R.release(item);
        if (++chunk == R.cpg) {
            if (n < s.n_gal) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (p < m.n_points) {
                        double av = 0.0, a1 = 0.0, a2 = 0.0, aq = 0.0;
                        finish_galaxy<kAGroup>(L[p], m.g1[p], m.g2[p], gmask, sub, s.w, n, av, a1, a2, aq);
                        if (sub == 0) {
                            acc[gl][p][0] += av;
                            acc[gl][p][1] += a1;
                            acc[gl][p][2] += a2;
                            acc[gl][p][3] += aq;
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) lse_reset(L[p]);
            chunk = 0;
            tile += gridDim.x;
        }
    }
    if (failed || (tid == 0 && !R.p_ok)) s_fail = 1;
    R.drain();
    __syncthreads();
    if (tid < NP * 4) {
        const int p = tid >> 2, i = tid & 3;
        double t = 0.0;
        for (int k = 0; k < kTileG; ++k) t += acc[k][p][i];
        m.partials[((size_t)p * gridDim.x + blockIdx.x) * 4 + i] = s_fail ? NAN : t;
    }
}

cudaError_t launch_shear_multi(const ShearMultiLaunch &m, int grid, cudaStream_t stream)
{
    const ShearLaunch &s = m.s;
    const bool vec = (s.K % 4 == 0) && ((reinterpret_cast<uintptr_t>(s.e1) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(s.e2) & 15) == 0) && s.b == nullptr;
    CUtensorMap m1, m2;
    if (vec && make_sample_map(m1, s.e1, s.n_gal, s.K) && make_sample_map(m2, s.e2, s.n_gal, s.K)) {
        auto k = s.family == BS_EPRIOR_BA14 ? shear_kernel_tma_multi<BS_EPRIOR_BA14>
                                            : shear_kernel_tma_multi<BS_EPRIOR_TRUNC_GAUSS>;
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tma_smem_bytes());
        if (e != cudaSuccess) return e;
        k<<<grid, kShearThreads, tma_smem_bytes(), stream>>>(m, m1, m2);
        return cudaGetLastError();
    }
    if (m.s.family == BS_EPRIOR_BA14)
        shear_kernel_multi<BS_EPRIOR_BA14><<<grid, kShearThreads, 0, stream>>>(m);
    else
        shear_kernel_multi<BS_EPRIOR_TRUNC_GAUSS><<<grid, kShearThreads, 0, stream>>>(m);
    return cudaGetLastError();
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

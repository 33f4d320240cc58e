// Pixel-space evaluations of the log posterior and its gradient (Appendix C): per-pixel
// weights on the tensor cores, a dense covariance on the CUDA cores.  Included by
// bs_fit_impl.cuh inside namespace bs::(anonymous), after the spectral evaluation
// (eval_logpost) and the table layout it reuses.
#pragma once

// ---- Spatially variable noise (Appendix C): log L = -1/2 sum_x w(x) (d - m)^2 / sigma^2.
// Parseval no longer makes this a sum over k, but the gradient is still sum_k
// Re[conj(R_k) dM_k / dtheta] / (sigma^2 N^2) with R = DFT(w (d - m)), so the half-plane
// pass of eval_logpost gives it when its data spectrum is replaced by the effective
// D' = M + R (scaled as the table).  The transforms run on the tensor cores (the layout
// and operand split are described with PixTc); one CTA of eight warps evaluates two chains.

// Per galaxy (all threads): the A operands of the four products for this side into
// tensor memory (warp w writes lanes 32 (w mod 4) .. + 31, the high parts for w < 4 and
// the low parts otherwise), the second chain's copy of the table, and the stamp and
// its weights in shared memory.
__device__ void pix_tc_setup(const FitParams &P, const GalCtx &gc, const SmemView &sm, const PixTc &px, int gal)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = gc.N, c = gc.c, H = gc.H;
    const int row = 32 * (warp & 3) + lane;      // the TMEM lane this thread writes
    const bool lo = warp >= 4;
    const uint32_t tl = *px.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    auto part = [&](float x) { const float h = tc::tf32_rn(x); return lo ? tc::tf32_rn(x - h) : h; };
    // [[C, -S], [S, C]]: row r = (p, a), column k = (q, b): p = q gives C, else -S (p = 0) or S
    const int p = row >> 6, a = row & 63;
    for (int k0 = 0; k0 < 128; k0 += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j, q = k >> 6, b = k & 63;
            float co = 0.f, sn = 0.f;
            if (a < N && b < N) {
                int m = ((a - c) * (b - c)) % N;   // exact reduction of the phase index
                if (m < 0) m += N;
                sincospif(2.0f * (float)m / (float)N, &sn, &co);
            }
            v[j] = part(p == q ? co : (p == 0 ? -sn : sn));
        }
        tc::st8(tl + (lo ? tc::kColAFlo : tc::kColAF) + k0, v);
    }
    // the complex-to-real constant: rows ix < 64, K (re, u | im, u):
    // (w_u / N^2) (cos, -sin)(2 pi u (ix - c) / N); rows 64.. zero
    const float wn = 1.0f / ((float)N * (float)N);
    for (int k0 = 0; k0 < 64; k0 += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j, q = k >> 5, u = k & 31;
            float co = 0.f, sn = 0.f;
            if (row < N && u < H) {
                int m = (u * (row - c)) % N;
                if (m < 0) m += N;
                sincospif(2.0f * (float)m / (float)N, &sn, &co);
                const float wu = u ? 2.0f * wn : wn;
                co *= wu;
                sn *= wu;
            }
            v[j] = part(q ? -sn : co);
        }
        tc::st8(tl + (lo ? tc::kColA2lo : tc::kColA2) + k0, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    const int nrow = gc.H * row_floats(P.npad);
    for (int i = tid; i < nrow; i += blockDim.x) px.tab1[i] = sm.tab[i];
    const int64_t off = P.offsets[gal];
    const int n = N * N;
    for (int i = tid; i < n; i += blockDim.x) {
        px.dimg[i] = load_pix(P.data, P.data_f64, off + i);
        px.wimg[i] = __ldg(P.pix_w + off + i);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// One 3xTF32 product into TMEM columns [0, N) (all threads; thread 0 issues and
// commits, everyone waits for the given parity).  K runs over n_q halves of nk steps
// of 8: step (q, k) reads A at TMEM column a + q a_q + 8 k (its low part a_lo columns
// further) and B at b + q b_q + 288 k bytes (the data operand: leading offset 144 B,
// row groups sbo_b apart).  Returns false (for every thread) if the wait gave up; the
// CTA is then aborted with that parity pending.
struct TcGemm {
    uint32_t a, a_q, a_lo, b, b_q, sbo_b, id;
    int n_q, nk;
};
__device__ __forceinline__ bool tc_run(const PixTc &px, const TcGemm &G, uint32_t parity)
{
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    const uint32_t bar = tc::saddr(px.bar);
    if (threadIdx.x == 0) {
        tc::fence_after();
        const uint32_t tmem = *px.tmem;
        const uint32_t b_lo = tc::kBopFloats * 4;
        for (int q = 0; q < G.n_q; ++q) {
            // a k-step advances the B descriptor's start-address field (bytes / 16, the
            // low 14 bits; every address stays below 256 KB, so the field does not carry)
            uint32_t a = tmem + G.a + q * G.a_q;
            const uint32_t b0 = G.b + q * G.b_q;
            uint64_t bh = tc::sdesc(b0, tc::kLboB, G.sbo_b), bl = tc::sdesc(b0 + b_lo, tc::kLboB, G.sbo_b);
            for (int k = 0; k < G.nk; ++k) {
                tc::mma_ta(tmem, a, bl, G.id, (q | k) ? 1u : 0u);
                tc::mma_ta(tmem, a + G.a_lo, bh, G.id, 1u);
                tc::mma_ta(tmem, a, bh, G.id, 1u);
                a += 8;
                bh += 288 / 16;
                bl += 288 / 16;
            }
        }
        tc::commit(bar);
    }
    const bool ok = tc::wait_parity(bar, parity);
    const bool bad = __syncthreads_or(!ok);
    if (bad) {
        if (threadIdx.x == 0) *px.abort = 2 + (int)parity;
        return false;
    }
    tc::fence_after();
    return true;
}

__device__ __forceinline__ double pix_nan(float g[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = NAN;
    return NAN;
}

// The gradient of the log posterior of this group's chain from the half-plane pass on
// its effective spectrum, with the rows split over the group's four warps: warp j of
// the group sums the terms of its rows u in [r j, r (j + 1)), r even (the pass reads
// rows in pairs); the four warp sums meet in shared memory, where every thread of the
// group adds them in warp order and forms the gradient (the sums and the gradient of
// eval_logpost, exponential profile, no chi^2).
template <int NC>
__device__ void pix_grad(const FitParams &P, const GalCtx &gc, const float *tab, const float2 *kxr, const PixTc &px,
                         float4 *xph, const float vcol[NC], const float th[6], float g[6])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp >> 2, wj = warp & 3;
    const int per = 2 * ((gc.H + 7) >> 3);
    const int u0 = min(gc.H, wj * per), u1 = min(gc.H, u0 + per);
    const Shape m = model_shape<0>(P, th);
    float sums[6], chi_hi = 0.f, chi_lo = 0.f;
    spectral_sums<NC, false, 0>(P, gc, m, tab, kxr, xph, vcol, th, u0, u1, sums, chi_hi, chi_lo);
    float *gs = px.gsum + grp * 24;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) gs[6 * wj + k] = sums[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; ++k) sums[k] = ((gs[k] + gs[6 + k]) + gs[12 + k]) + gs[18 + k];
    spectral_grad<0>(P, gc, m, sums, th, g);
}

// One evaluation of both chains of the CTA (all threads; each group passes its own
// chain's th; a group with skip set passes any finite th and ignores the results).
// Returns the log posterior of the caller's chain if want_ll (the caller's group's
// flag), else 0; *all_done is set when both groups have raised their done flags (the
// evaluation then does nothing).
template <int NC>
__device__ double eval_pix(const FitParams &P, const GalCtx &gc, const SmemView &sm, int gal, float4 *xph,
                           const float vcol[NC], const float th[6], float g[6], bool want_ll, bool *all_done)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp >> 2;                        // the chain of this thread's group
    const int L = 32 * (warp & 3) + lane;             // this thread's TMEM lane
    const int tg = tid & 127;                         // thread within the group
    const PixTc px = pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side);
    const int N = gc.N, H = gc.H, c = gc.c, npad = P.npad;
    const int rowf = row_floats(npad);
    float *tab = grp ? px.tab1 : sm.tab;
    __syncthreads();   // the previous evaluation's readers of the tables and buffers are done
    if (all_done) *all_done = px.done[0] && px.done[1];
    if (px.done[0] && px.done[1]) return 0.0;
    if (*px.abort) return pix_nan(g);
    const float F = exp10f(th[0]);
    const float r0 = exp10f(th[1]) * (1.0f / kHlrOverR0);
    const float r02 = r0 * r0;
    const float e1 = th[2], e2 = th[3];
    const float E = e1 * e1 + e2 * e2;
    const float Pq = 1.0f / (1.0f - E);
    const float al = r02 * (1.0f + E + 2.0f * e1) * Pq;
    const float be = r02 * (1.0f + E - 2.0f * e1) * Pq;
    const float ga = r02 * 4.0f * e2 * Pq;
    const float sqrt2 = 1.41421356237309515f;
    float2 *xs = px.xs + 32 * grp, *ys = px.ys + 64 * grp;
    if (tg < 32) {
        float sx = 0.f, cx = 0.f;
        if (tg < H) sincospi_sfu(-2.0f * th[4] * (float)tg * gc.invN, &sx, &cx);
        xs[tg] = make_float2(cx, sx);
    } else if (tg < 96) {
        const int vi = tg - 32;
        float sy = 0.f, cy = 0.f;
        if (vi < N) sincospi_sfu(-2.0f * th[5] * (float)(vi - c) * gc.invN, &sy, &cy);
        ys[vi] = make_float2(F * cy, F * sy);
    }
    __syncthreads();
    float *bh = px.bop, *bl = px.bop + tc::kBopFloats;
    constexpr int kLb = tc::kLboB / 4;
    // (a) the model's half spectrum Mt into the chain's table D slots, and M = Mt /
    // scale_u as the operand of (1): rows (chain, u < 32), K (re, vi | im, vi); thread
    // tg of the group takes column vi = tg mod 64 and the rows u = tg / 64 + 2 i
    {
        const int vi = tg & 63, u0 = tg >> 6;
        const bool col = vi < N;
        int ox = 0, oy = 0, ot = 0;
        if (col) slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
        const float ky = (float)(vi - c) * gc.dk;
        const float cst = fmaf(be * ky, ky, 1.0f), gky = ga * ky;
        const float2 Y = ys[vi];
        const float sN = (float)N, sN2 = (float)N * 0.70710678118654752f;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int u = u0 + 2 * i;
            float Mr = 0.f, Mi = 0.f;
            if (col && u < H) {
                float *row = tab + (size_t)u * rowf;
                const float kx = sm.kxr[u].x;
                const float s = fmaf(fmaf(al, kx, gky), kx, cst);
                const float rs = rsqrtf(s);
                const float A = row[ot] * rs * rs * rs;
                const float2 X = xs[u];
                const float mr = A * (X.x * Y.x - X.y * Y.y), mi = A * (X.x * Y.y + X.y * Y.x);
                row[ox] = mr;
                row[oy] = mi;
                const float inv_scale = u == 0 ? sN : sN2;
                Mr = mr * inv_scale;
                Mi = mi * inv_scale;
            }
            tc::split_store(bh, bl, tc::op_index(32 * grp + u, vi, 128, kLb), Mr);
            tc::split_store(bh, bl, tc::op_index(32 * grp + u, 64 + vi, 128, kLb), Mi);
        }
    }
    const uint32_t bop = tc::saddr(px.bop);
    const int ks = (N + 7) >> 3;   // k-steps of 8 covering the side
    const uint32_t tl = *px.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    constexpr uint32_t aflo = tc::kColAFlo - tc::kColAF, a2lo = tc::kColA2lo - tc::kColA2;
    // (1) G = M E for both chains: rows (re, iy | im, iy), columns (chain, u)
    if (!tc_run(px, TcGemm{tc::kColAF, 64u, aflo, bop, 16u * 144, 32u * 144, tc::idesc(128, 64), 2, ks}, 0))
        return pix_nan(g);
    // (1) -> operand of (2): row (chain, iy), K (re, u | im, u), G as it is (the weights
    // are in the constant); this thread's lane (p, iy), its chain's 32 columns
    {
        float v[32];
        tc::ld32(tl + 32 * grp, v);
        const int p = L >> 6, iy = L & 63;
        const int e0 = tc::op_index(64 * grp + iy, p * 32, 64, kLb);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            tc::split_store4(bh, bl, e0 + m * kLb, v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
    }
    // (2) m = W G: rows ix, columns (chain, iy)
    if (!tc_run(px, TcGemm{tc::kColA2, 32u, a2lo, bop, 8u * 144, 16u * 144, tc::idesc(128, 128), 2,
                           (H + 7) >> 3},
                1))
        return pix_nan(g);
    // the residual, chi^2 (compensated FP32 per thread, FP64 across threads) and the
    // operand of (3): rows (chain, iy), K ix; lanes ix < 64 of the group's warps 0 and
    // 1, the chain's 64 columns iy
    double chi = 0.0;
    if ((warp & 3) < 2) {
        const int ix = L;
        float c_hi = 0.f, c_lo = 0.f;
        const int eb = (ix >> 2) * kLb + (ix & 3);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float m[32];
            tc::ld32(tl + 64 * grp + 32 * h, m);
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const int iy = 32 * h + t;
                float r = 0.f;
                if (ix < N && iy < N) {
                    const int e = iy * N + ix;
                    const float res = px.dimg[e] - m[t];
                    r = px.wimg[e] * res;
                    if (want_ll) {
                        float t_hi, t_lo;
                        two_sum(c_hi, r * res, t_hi, t_lo);
                        c_hi = t_hi;
                        c_lo += t_lo;
                    }
                }
                const int rr = 64 * grp + iy;
                tc::split_store(bh, bl, eb + (rr >> 3) * 16 * kLb + ((rr & 7) << 2), r);
            }
        }
        chi = (double)c_hi + (double)c_lo;
    }
    if (want_ll) {
        const double cw = warp_sum_d(chi);
        if (lane == 0) px.chi[warp] = cw;
    }
    // (3) conj Q = [C; S] r: rows (re, a | im, a), columns (chain, iy)
    if (!tc_run(px, TcGemm{tc::kColAF, 0u, aflo, bop, 0u, 16u * 144, tc::idesc(128, 128), 1, ks}, 0))
        return pix_nan(g);
    // (3) -> operand of (4): row (chain, u = a - c < 32), K (re, iy | im, iy); this
    // thread's lane (q, a), its chain's 64 columns iy
    {
        const int q = L >> 6, u = (L & 63) - c;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::ld32(tl + 64 * grp + 32 * h, v);
            if (u >= 0 && u < 32) {
                const int e0 = tc::op_index(32 * grp + u, q * 64 + 32 * h, 128, kLb);
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    tc::split_store4(bh, bl, e0 + m * kLb, v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
            }
        }
    }
    // (4) conj R = E conj Q: rows (re, vi | im, vi), columns (chain, u)
    if (!tc_run(px, TcGemm{tc::kColAF, 64u, aflo, bop, 16u * 144, 32u * 144, tc::idesc(128, 64), 2, ks}, 1))
        return pix_nan(g);
    // D' = Mt + scale_u R in the chain's table D slots; this thread's lane (p, vi), its
    // chain's 32 columns u
    {
        const int p = L >> 6, vi = L & 63;
        float v[32];
        tc::ld32(tl + 32 * grp, v);
        if (vi < N) {
            int ox, oy, ot;
            slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
            const int os = p ? oy : ox;
            const float sg = p ? -gc.invN : gc.invN;
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                if (u < H) {
                    float *slot = tab + (size_t)u * rowf + os;
                    *slot = fmaf((u ? sqrt2 : 1.0f) * sg, v[u], *slot);
                }
            }
        }
    }
    __syncthreads();
    // the gradient from the half-plane pass on the chain's effective spectrum, its rows
    // over the group's four warps
    pix_grad<NC>(P, gc, tab, sm.kxr, px, xph, vcol, th, g);
    if (!want_ll) return 0.0;
    const double chi2 = px.chi[4 * grp] + px.chi[4 * grp + 1];
    const float lprior = P.prior_const - 0.5f * (th[4] * th[4] + th[5] * th[5]) * P.inv_sxy2 +
                         2.0f * log1pf(-E) - 0.5f * E * P.inv_se2;
    return -0.5 * chi2 * (double)gc.inv_b + (double)lprior;
}

// A group whose chain has no further evaluations (all threads of the group): raise
// its done flag, then join the other group's evaluations until both are done.
template <int NC>
__device__ void pix_drain(const FitParams &P, const GalCtx &gc, const SmemView &sm, int gal, float4 *xph,
                          const float vcol[NC])
{
    const PixTc px = pix_tc_view(sm.kxr, P.h_max, P.npad, P.max_side);
    if ((threadIdx.x & 127) == 0) px.done[threadIdx.x >> 7] = 1;
    const float th[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // any finite point: the results are not used
    float g[6];
    for (;;) {
        bool all = false;
        eval_pix<NC>(P, gc, sm, gal, xph, vcol, th, g, false, &all);
        if (all) break;
    }
}

// ---- A general dense pixel covariance (Appendix C, Eq. covar-pixel-likelihood):
// log L = -1/2 (d - m)^T P (d - m) with the precision P = Sigma^-1.  Its cost is the
// product y = P (d - m), N^4 multiply-adds per evaluation reading P from L2, beside
// which the two separable transforms are small; and P amplifies rounding errors of
// the rendered model m, so the transforms stay in FP32 on the CUDA cores (kernel
// instance PROF 4, one warp per chain).  The gradient is the half-plane pass on the
// effective spectrum D' = M + DFT(y) (scaled as the table).
//
// After the shared region: the twiddles exp(+2 pi i m / N) (max_side float2) and,
// per chain, a private copy of the table ([h_max][3 npad]: the D slots hold the
// evaluation's effective spectrum, the T slots the transfer), the half-transformed
// image ([h_max][max_side] float2), the residual image and its product with the
// precision (max_side^2 floats each).  Sizes in floats, each chain's block a multiple
// of 4 floats.
__host__ __device__ __forceinline__ int dense_chain_floats(int h_max, int npad, int max_side)
{
    const int n = h_max * row_floats(npad) + 2 * h_max * max_side + 2 * max_side * max_side;
    return (n + 3) & ~3;
}
__host__ __device__ __forceinline__ size_t dense_region_bytes(int h_max, int npad, int max_side, int n_chains)
{
    return ((size_t)2 * ((max_side + 1) & ~1) + (size_t)n_chains * dense_chain_floats(h_max, npad, max_side)) *
           sizeof(float);
}
struct DenseView {
    float2 *tw;    // [max_side] exp(+2 pi i m / N)
    float *tab;    // this chain's table
    float2 *G;     // [h_max][max_side]
    float *rb;     // [max_side^2] residual d - m
    float *yb;     // [max_side^2] precision x residual
};
// kxr ends at h_max + 1 float2 after its start; the region follows, 16-byte aligned.
__device__ __forceinline__ DenseView dense_view(float2 *kxr, int h_max, int npad, int max_side, int chain)
{
    float *base = reinterpret_cast<float *>(kxr + ((h_max + 2) & ~1));
    DenseView v;
    v.tw = reinterpret_cast<float2 *>(base);
    float *c0 = base + 2 * ((max_side + 1) & ~1) + (size_t)chain * dense_chain_floats(h_max, npad, max_side);
    v.tab = c0;
    v.G = reinterpret_cast<float2 *>(c0 + (size_t)h_max * row_floats(npad));
    v.rb = reinterpret_cast<float *>(v.G + (size_t)h_max * max_side);
    v.yb = v.rb + max_side * max_side;
    return v;
}

// Per-galaxy set-up of the dense path (all threads): the twiddles, and each
// chain's private table from the staged one (transfer, zero spectrum).
__device__ void dense_setup(const FitParams &P, const GalCtx &gc, const SmemView &sm, int n_tables)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const DenseView p0 = dense_view(sm.kxr, P.h_max, P.npad, P.max_side, 0);
    for (int m = tid; m < gc.N; m += nth) {
        float s, co;
        sincospif(2.0f * (float)m * gc.invN, &s, &co);
        p0.tw[m] = make_float2(co, s);
    }
    const int rowf = row_floats(P.npad);
    const int nrow = gc.H * rowf;
    for (int t = 0; t < n_tables; ++t) {
        float *dst = dense_view(sm.kxr, P.h_max, P.npad, P.max_side, t).tab;
        for (int i = tid; i < nrow; i += nth) dst[i] = sm.tab[i];
    }
    __syncthreads();
}

template <int NC>
__device__ double eval_dense(const FitParams &P, const GalCtx &gc, const DenseView &pv, int gal,
                           const float2 *__restrict__ kxr, float4 *__restrict__ xph, const float vcol[NC],
                           const float th[6], float &gi, bool want_ll)
{
    const int lane = threadIdx.x & 31;
    const int N = gc.N, H = gc.H, c = gc.c, npad = P.npad;
    const int rowf = row_floats(npad);
    const float F = exp10f(th[0]);
    const float r0 = exp10f(th[1]) * (1.0f / kHlrOverR0);
    const float r02 = r0 * r0;
    const float e1 = th[2], e2 = th[3];
    const float E = e1 * e1 + e2 * e2;
    const float Pq = 1.0f / (1.0f - E);
    const float al = r02 * (1.0f + E + 2.0f * e1) * Pq;
    const float be = r02 * (1.0f + E - 2.0f * e1) * Pq;
    const float ga = r02 * 4.0f * e2 * Pq;
    const float sqrt2 = 1.41421356237309515f;
    for (int u = lane; u < H; u += 32) {
        float sx, cx;
        sincospi_sfu(-2.0f * th[4] * (float)u * gc.invN, &sx, &cx);
        xph[u] = make_float4(cx, sx, -sx, 0.0f);
    }
    __syncwarp();
    // (a) the model's half spectrum Mt = Tt F f(s) X(u) Y(v) into the D slots
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int vi = lane + 32 * j;
        float sy, cy;
        sincospi_sfu(-2.0f * th[5] * vcol[j] * gc.invN, &sy, &cy);
        const float Yr = F * cy, Yi = F * sy;
        const float ky = vcol[j] * gc.dk;
        const float cst = fmaf(be * ky, ky, 1.0f), gky = ga * ky;
        int ox, oy, ot;
        slot_offsets(npad, j, lane, ox, oy, ot);
        for (int u = 0; u < H; ++u) {
            float *row = pv.tab + (size_t)u * rowf;
            const float kx = kxr[u].x;
            const float s = fmaf(fmaf(al, kx, gky), kx, cst);
            const float rs = rsqrtf(s);
            const float A = row[ot] * rs * rs * rs;
            const float4 X = xph[u];
            const float Pr = X.x * Yr - X.y * Yi, Pi = X.x * Yi + X.y * Yr;
            const float mr = vi < N ? A * Pr : 0.0f, mi = vi < N ? A * Pi : 0.0f;
            row[ox] = mr;
            row[oy] = mi;
            // unscaled M(u, v) = Mt / scale_u, contiguous, for the inverse transform
            const float inv_scale = (float)N * (u == 0 ? 1.0f : 0.70710678118654752f);
            if (vi < N) pv.G[(size_t)u * N + vi] = make_float2(mr * inv_scale, mi * inv_scale);
        }
    }
    __syncwarp();
    // (b1) G(u, iy) = sum_v M(u, v) exp(+2 pi i v (iy - c) / N), in place row by
    // row (a row's outputs need only that row's M; lanes over iy, at most 2 each)
    for (int u = 0; u < H; ++u) {
        float2 *grow = pv.G + (size_t)u * N;
        float2 res[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int iy = lane + 32 * r;
            if (iy < N) {
                const int step = iy - c;
                float re = 0.f, im = 0.f;
                int k = ((-c * step) % N + N) % N;
                const int dk = (step % N + N) % N;
                for (int vi = 0; vi < N; ++vi) {
                    const float2 mv = grow[vi];
                    const float2 t = pv.tw[k];
                    re = fmaf(mv.x, t.x, fmaf(-mv.y, t.y, re));
                    im = fmaf(mv.x, t.y, fmaf(mv.y, t.x, im));
                    k += dk;
                    if (k >= N) k -= N;
                }
                res[r] = make_float2(re, im);
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (lane + 32 * r < N) grow[lane + 32 * r] = res[r];
        __syncwarp();
    }
    // (b2) per pixel row: m(ix, iy) and the residual r = d - m; y = P r needs every row of r
    const int64_t off = P.offsets[gal];
    const float invN2 = gc.invN * gc.invN;
    double chi = 0.0;
    for (int iy = 0; iy < N; ++iy) {
        for (int ix = lane; ix < N; ix += 32) {
            const int dk = ((ix - c) % N + N) % N;      // u (ix - c) mod N, advanced per u
            int k = dk;
            float acc = pv.G[iy].x;                     // u = 0 (real)
            for (int u = 1; u < H; ++u) {
                const float2 gv = pv.G[(size_t)u * N + iy];
                const float2 t = pv.tw[k];
                acc = fmaf(2.0f * gv.x, t.x, fmaf(-2.0f * gv.y, t.y, acc));
                k += dk;
                if (k >= N) k -= N;
            }
            pv.rb[iy * N + ix] = load_pix(P.data, P.data_f64, off + (int64_t)iy * N + ix) - acc * invN2;
        }
    }
    __syncwarp();
    {
        // y = Sigma^-1 r: the precision is symmetric, so y_a = sum_b P[b][a] r_b with
        // lanes over a reads each row b of it coalesced (from L2: tens of
        // evaluations of the galaxy's chains share it); chi^2 = r.y
        constexpr int kSlots = (kDenseMaxSide * kDenseMaxSide + 31) / 32;
        const int n = N * N;
        const float *Pg = P.pix_prec + P.prec_offs[gal];
        float yv[kSlots];
#pragma unroll
        for (int j = 0; j < kSlots; ++j) yv[j] = 0.f;
        for (int b = 0; b < n; ++b) {
            const float rb = pv.rb[b];
            const float *prow = Pg + (size_t)b * n;
#pragma unroll
            for (int j = 0; j < kSlots; ++j) {
                const int a = lane + 32 * j;
                if (a < n) yv[j] = fmaf(__ldg(prow + a), rb, yv[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kSlots; ++j) {
            const int a = lane + 32 * j;
            if (a < n) {
                pv.yb[a] = yv[j];
                chi += (double)pv.rb[a] * (double)yv[j];
            }
        }
        __syncwarp();
        // Q(u, iy) = sum_ix y(ix, iy) exp(-2 pi i u (ix - c) / N), one row iy at a time
        for (int iy = 0; iy < N; ++iy) {
            const float *yrow = pv.yb + iy * N;
            for (int u = lane; u < H; u += 32) {
                float re = 0.f, im = 0.f;
                int k = ((u * c) % N + N) % N;           // -u (ix - c) at ix = 0
                const int dk = (N - u % N) % N;
                for (int ix = 0; ix < N; ++ix) {
                    const float r = yrow[ix];
                    const float2 t = pv.tw[k];
                    re = fmaf(r, t.x, re);
                    im = fmaf(r, t.y, im);
                    k += dk;
                    if (k >= N) k -= N;
                }
                pv.G[(size_t)u * N + iy] = make_float2(re, im);
            }
        }
        __syncwarp();
    }
    // (b3) D' = Mt + scale_u R(u, v), R(u, v) = sum_iy Q(u, iy) exp(-2 pi i v (iy - c) / N);
    // the H x N (u, v) outputs spread over the lanes
    for (int t = lane; t < H * N; t += 32) {
        const int u = t / N, vi = t - u * N, v = vi - c;
        const int dk = ((-v) % N + N) % N;
        int k = ((v * c) % N + N) % N;                  // -v (iy - c) at iy = 0
        const float2 *qrow = pv.G + (size_t)u * N;
        float re = 0.f, im = 0.f;
        for (int iy = 0; iy < N; ++iy) {
            const float2 q = qrow[iy];
            const float2 tw = pv.tw[k];
            re = fmaf(q.x, tw.x, fmaf(-q.y, tw.y, re));
            im = fmaf(q.x, tw.y, fmaf(q.y, tw.x, im));
            k += dk;
            if (k >= N) k -= N;
        }
        int ox, oy, ot;
        slot_offsets(npad, vi >> 5, vi & 31, ox, oy, ot);
        const float scale = (u == 0 ? 1.0f : sqrt2) * gc.invN;
        float *row = pv.tab + (size_t)u * rowf;
        row[ox] = fmaf(scale, re, row[ox]);
        row[oy] = fmaf(scale, im, row[oy]);
    }
    __syncwarp();
    // (c) the gradient from the half-plane pass on the effective spectrum
    eval_logpost<NC, 0>(P, gc, pv.tab, kxr, xph, vcol, th, gi, false);
    if (!want_ll) return 0.0;
    const double chi2 = warp_sum_d(chi);
    const float lprior = P.prior_const - 0.5f * (th[4] * th[4] + th[5] * th[5]) * P.inv_sxy2 +
                         2.0f * log1pf(-E) - 0.5f * E * P.inv_se2;
    return -0.5 * chi2 * (double)gc.inv_b + (double)lprior;
}


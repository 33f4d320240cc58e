#pragma once
// Pixel-space evaluation of the log posterior and its gradient on the 5th-generation
// tensor cores (Appendix C: per-pixel weights w, log L = -1/2 sum_x w (d - m)^2 / sigma^2).
//
// Parseval does not diagonalise these likelihoods, so each evaluation renders the
// model image m from its half spectrum M and transforms the weighted residual back:
//   G(u, iy) = sum_v M(u, v) e^{+2 pi i v (iy - c) / N}                 (1: complex, along y)
//   m(ix, iy) = N^-2 sum_u w_u Re[G(u, iy) e^{+2 pi i u (ix - c) / N}]  (2: complex to real, along x)
//   r = w (d - m)
//   Q(u, iy) = sum_ix r(ix, iy) e^{-2 pi i u (ix - c) / N}             (3: real to complex, along x)
//   R(u, v) = sum_iy Q(u, iy) e^{-2 pi i v (iy - c) / N}               (4: complex, along y)
// (w_0 = 1, w_u = 2 for u > 0, v = vi - c centred), and the gradient is the spectral
// half-plane pass on the effective spectrum D' = Mt + (sqrt(w_u) / N) R.
//
// With centred indices every transform is a product with one matrix built from
// C[a][b] = cos(2 pi (a - c)(b - c) / N) and S[a][b] = sin(...), zero-padded to 64 x 64:
//   (1)  rows (re, iy | im, iy) x K (re, v | im, v): A = [[C, -S], [S, C]];
//   (2)  rows ix x K (re, u | im, u): its own complex-to-real constant with the weights
//        w_u / N^2 folded in, so that the operand is G as the first product leaves it;
//   (3)  rows (re, u + c | im, u + c) x K ix: the first half [C; S] of (1)'s A (the
//        imaginary output is -Q_i: conj Q);
//   (4)  conj R = transform (1) of conj Q.
// These A operands live in tensor memory (lane = row, column = K index), high and
// low TF32 parts: 384 of the CTA's 512 columns, the accumulator the other 128.  Each
// transform is a tcgen05.mma of kind::tf32 (M = 128, N = 64 or 128, K = 8 per
// instruction; B, the data, in shared memory without swizzle) in three terms,
// A_hi B_hi + A_hi B_lo + A_lo B_hi with x = hi + lo split by round-to-nearest TF32
// (3xTF32): the operand rounding of plain TF32 would miss the log-likelihood
// tolerance by a factor of several.
//
// One CTA of eight warps runs two chains in lockstep: warps 0-3 the first, 4-7 the
// second (each group's warps run the same chain logic and make the same decisions,
// from the same numbers).  Every step of a chain is one evaluation, so the two meet
// at each one; every product carries both chains' data (B rows (chain, u) or (chain,
// iy)), so each barrier and MMA round trip serves two evaluations.  Thread t reads TMEM
// lane 32 (w mod 4) + (t mod 32) and its chain's columns (w / 4), the group's warps
// split the spectral gradient pass by rows, and thread 0 issues the MMAs.  A chain that
// has finished, or has no evaluation at a step, joins with a skip flag until both are
// done.  Each evaluation commits four MMA groups to one mbarrier, so the parities it
// waits on are 0, 1, 0, 1 in every evaluation.  A wait gives up after two seconds: the
// CTA then marks its galaxy (status 4), issues no further MMA, and its evaluations
// return NaN until the chains end.
#include <cstdint>

namespace bs {

namespace {

namespace tc {

constexpr int kLboB = 144;                     // data operands: 16-byte pad per core matrix (column
                                               // stores of a warp fall in 32 distinct banks)
constexpr int kBopFloats = 16 * 16 * (kLboB / 4);   // one data operand: 128 rows x 64 K or 64 x 128
constexpr uint64_t kWaitNs = 2000000000ull;    // limit of one MMA wait

// Element (row, k) of an operand of kt K-elements per row (no swizzle, K-major):
// core matrices of 8 rows x 4 elements (16 bytes a row), lbo_f floats apart along
// K, row groups of 8 (kt / 4) lbo_f floats apart.
__host__ __device__ __forceinline__ int op_index(int row, int k, int kt, int lbo_f)
{
    return (row >> 3) * (kt >> 2) * lbo_f + (k >> 2) * lbo_f + ((row & 7) << 2) + (k & 3);
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (row-group) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Round a finite float to the nearest TF32 value, ties away from zero (the
// rounding of cvt.rna.tf32.f32): add half a unit of the 13 dropped bits to the
// magnitude's bit pattern and clear them.
__device__ __forceinline__ float tf32_rn(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// x = hi + lo (hi exact in TF32; lo rounded to TF32, error ~2^-22 |x|)
__device__ __forceinline__ void split_store(float *hi, float *lo, int i, float x)
{
    const float h = tf32_rn(x);
    hi[i] = h;
    lo[i] = tf32_rn(x - h);
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared stores made visible to the tensor cores' (async) proxy
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete; false after kWaitNs.  Each
// try_wait may suspend the warp in hardware for up to 20 us until the phase
// completes; the limit is checked between tries.
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = now_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

// 32 consecutive TMEM columns of this thread's lane (the warp's 32 lanes).
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Four consecutive K-elements (one core-matrix row) as high and low TF32 parts.
__device__ __forceinline__ void split_store4(float *hi, float *lo, int i, float a, float b, float c, float d)
{
    float4 h, l;
    h.x = tf32_rn(a);
    h.y = tf32_rn(b);
    h.z = tf32_rn(c);
    h.w = tf32_rn(d);
    l.x = tf32_rn(a - h.x);
    l.y = tf32_rn(b - h.y);
    l.z = tf32_rn(c - h.z);
    l.w = tf32_rn(d - h.w);
    *reinterpret_cast<float4 *>(hi + i) = h;
    *reinterpret_cast<float4 *>(lo + i) = l;
}

// TMEM columns of the CTA: the accumulator, then the A operands (high, low).
constexpr int kTmemCols = 512;
constexpr int kColAF = 128;                    // [[C, -S], [S, C]], 128 columns: K (re, v | im, v)
constexpr int kColAFlo = 256;
constexpr int kColA2 = 384;                    // the complex-to-real constant, 64 columns: K (re, u | im, u)
constexpr int kColA2lo = 448;
constexpr int kThreads = 256;                  // eight warps: lane quadrant w % 4, chain w / 4

__device__ __forceinline__ void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t id, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(id), "r"(accumulate));
}

// Eight consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

}  // namespace tc

// Shared memory of the tensor-core pixel path, after the (kx, kx^2) table.
struct PixTc {
    double *chi;      // [8] per-warp partial chi^2 of the evaluation
    uint64_t *bar;    // MMA completion barrier
    uint32_t *tmem;   // TMEM base of the CTA (512 columns)
    int *abort;       // 2 + the pending parity once a wait gave up, else 0
    int *done;        // [2] a chain group has no more evaluations
    float2 *xs;       // [2][32] per chain: exp(-2 pi i u dx / N)
    float2 *ys;       // [2][64] per chain: F exp(-2 pi i v dy / N), v = vi - c
    float *gsum;      // [2][4][6] per chain and warp of its group: the six gradient sums
    float *bop;       // [2][kBopFloats] the data operand of the current transform, high then low
    float *tab1;      // [h_max][3 npad] the second chain's table (the first's is the staged one)
    float *dimg;      // [max_side^2] the stamp
    float *wimg;      // [max_side^2] the weights
};

__host__ __device__ __forceinline__ int pix_tc_img_floats(int max_side) { return (max_side * max_side + 3) & ~3; }

// Floats of the region: 16 (chi) + 2 (barrier) + 1 (TMEM address) + 1 (abort) + 2
// (done) + 2 (pad) + 128 (xs) + 256 (ys) + 48 (gradient sums) + operand + table + two
// images.
__host__ __device__ __forceinline__ size_t pix_tc_bytes(int max_side, int h_max, int npad)
{
    return ((size_t)456 + 2 * tc::kBopFloats + (size_t)h_max * 3 * npad + 2 * (size_t)pix_tc_img_floats(max_side)) *
           sizeof(float);
}

// The region starts after the (kx, kx^2) table (h_max + 1 float2), 16-byte aligned.
__device__ __forceinline__ PixTc pix_tc_view(float2 *kxr, int h_max, int npad, int max_side)
{
    float *base = reinterpret_cast<float *>(kxr + ((h_max + 2) & ~1));
    PixTc v;
    v.chi = reinterpret_cast<double *>(base);
    v.bar = reinterpret_cast<uint64_t *>(base + 16);
    v.tmem = reinterpret_cast<uint32_t *>(base + 18);
    v.abort = reinterpret_cast<int *>(base + 19);
    v.done = reinterpret_cast<int *>(base + 20);
    v.xs = reinterpret_cast<float2 *>(base + 24);
    v.ys = reinterpret_cast<float2 *>(base + 152);
    v.gsum = base + 408;
    v.bop = base + 456;
    v.tab1 = v.bop + 2 * tc::kBopFloats;
    v.dimg = v.tab1 + (size_t)h_max * 3 * npad;
    v.wimg = v.dimg + pix_tc_img_floats(max_side);
    return v;
}

// Once per CTA, before its first galaxy (all threads): TMEM columns, the barrier.
__device__ void pix_tc_begin(const PixTc &px)
{
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(px.tmem)),
                     "r"(tc::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(px.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *px.abort = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// Once per CTA, after its last galaxy (all threads).  After a wait that gave up,
// the MMAs still in flight are waited for once more (again with the limit) before
// the columns are freed.
__device__ void pix_tc_end(const PixTc &px)
{
    __syncthreads();
    if (threadIdx.x == 0 && *px.abort) {
        const int pend = *px.abort - 2;
        if (pend >= 0) tc::wait_parity(tc::saddr(px.bar), (uint32_t)pend);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*px.tmem), "r"(tc::kTmemCols)
                     : "memory");
}

}  // namespace

}  // namespace bs

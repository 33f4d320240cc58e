// Device helpers shared by the bpshear kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bpshear.h"

#define BS_FULL_MASK 0xffffffffu

namespace bs {

constexpr float kLn10 = 2.302585092994046f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
// half-light radius of the exponential profile in units of its scale length:
// the root of 1 - (1 + x) exp(-x) = 1/2
constexpr float kHlrOverR0 = 1.6783469900166608f;

// ---------------------------------------------------------------------------
// Philox4x64 with 10 rounds (Salmon et al., SC'11): per round the counter
// words 0 and 2 are multiplied by two fixed odd 64-bit constants, the
// high/low product halves are permuted across the words and the high halves
// are xored with the other counter words and the key; the key is bumped by
// two Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct Philox4x64 {
    uint64_t w[4];
};

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ Philox4x64 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                            uint64_t c3, uint64_t k0, uint64_t k1)
{
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    const uint64_t w0 = 0x9E3779B97F4A7C15ull, w1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0hi = mulhi64(m0, c0), p0lo = m0 * c0;
        const uint64_t p1hi = mulhi64(m1, c2), p1lo = m1 * c2;
        const uint64_t n0 = p1hi ^ c1 ^ k0;
        const uint64_t n2 = p0hi ^ c3 ^ k1;
        c0 = n0;
        c1 = p1lo;
        c2 = n2;
        c3 = p0lo;
        k0 += w0;
        k1 += w1;
    }
    Philox4x64 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

// Eight uniforms in (0, 1) from one block: the top 24 bits of each 32-bit half,
// centred in their bins, (j + 1/2) 2^-24 (exact in FP32).
__device__ __forceinline__ void uniforms8(uint64_t seed, uint64_t key, uint64_t c0, uint64_t c1,
                                          uint64_t c2, float u[8])
{
    const Philox4x64 r = philox4x64_10(c0, c1, c2, 0ull, seed, key);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t hi = (uint32_t)(r.w[j] >> 32), lo = (uint32_t)r.w[j];
        u[2 * j] = ((float)(hi >> 8) + 0.5f) * 5.9604644775390625e-08f;
        u[2 * j + 1] = ((float)(lo >> 8) + 0.5f) * 5.9604644775390625e-08f;
    }
}

// Uniform k (0..7) of the block uniforms8 draws for the same counter.
__device__ __forceinline__ float uniform_of8(uint64_t seed, uint64_t key, uint64_t c0, uint64_t c1, uint64_t c2,
                                             int k)
{
    const Philox4x64 r = philox4x64_10(c0, c1, c2, 0ull, seed, key);
    const int j = k >> 1;
    uint64_t w = r.w[0];
    if (j == 1) w = r.w[1];
    if (j == 2) w = r.w[2];
    if (j == 3) w = r.w[3];
    const uint32_t h = (k & 1) ? (uint32_t)w : (uint32_t)(w >> 32);
    return ((float)(h >> 8) + 0.5f) * 5.9604644775390625e-08f;
}

// ---------------------------------------------------------------------------
// Warp reductions.  The xor butterfly leaves the same bits in every lane
// (each step adds the same two operands in both partner lanes), which keeps
// warp-replicated chain state identical across lanes.
// ---------------------------------------------------------------------------
template <int WIDTH = 32>
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = WIDTH / 2; o > 0; o >>= 1) v += __shfl_xor_sync(BS_FULL_MASK, v, o, WIDTH);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(BS_FULL_MASK, v, o);
    return v;
}

// Error-free sum a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    const float ap = s - bp;
    e = (a - ap) + (b - bp);
}

// Warp-wide sum of compensated pairs, finished in double on return.
__device__ __forceinline__ double warp_sum_comp(float hi, float lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(BS_FULL_MASK, hi, o);
        const float ol = __shfl_xor_sync(BS_FULL_MASK, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        hi = s;
        lo = lo + ol + e;
    }
    return (double)hi + (double)lo;
}

}  // namespace bs

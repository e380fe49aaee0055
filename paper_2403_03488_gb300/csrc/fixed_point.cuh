// Exact fixed-point aggregation terms shared by the BM3D filtering kernels
// (FP32 SIMT and tensor-core paths): every contribution is converted to a
// 64-bit integer in units of 2^-36 and added with integer atomics, so the
// sums do not depend on the order in which groups are aggregated.
#pragma once

#include "f32x2.cuh"

namespace dn {
namespace {

// num(x) = sum over (group g, patch q of g) of w_g kai(x - q) v_{g,q}(x - q) is
// accumulated per pixel; den(x) = sum_q kai(x - q) W(q), W(q) = the sum of the
// weights of the groups that hold patch q, is accumulated per patch position
// (one addition per patch) and correlated with the Kaiser window when
// normalising.  Both sums are fixed point with 36 fraction bits (exact whenever
// the FP32 term is >= 2^-13 in magnitude) added with integer atomics, so they
// are bitwise reproducible whatever the order of the groups.  Weights are used
// scaled by sigma^2 (1/N_har, 1/sum w^2, or sigma^2 for an all-zero group),
// which leaves num/den unchanged.
//
// A term c with |c| < 512 (all of them, in practice) is added to the 64-bit
// main plane as round(c 2^36) < 2^45; any other c (a heavy weight or a large
// value) is clamped to |c| <= 2^40 and split as c 2^36 = hi 2^32 + lo,
// 0 <= lo <= 2^32: lo goes to the main plane, hi to a high-word plane.  With at
// most 2^14 terms per sum neither plane can overflow, and the value is
// main + hi 2^32.

// round(c 2^36) (ties to even) for |c| < 512, on the FP32 and integer pipes:
// t = c 2^13 is split into its nearest integer A (magic-number rounding, valid
// for |t| < 2^22) and the exact remainder r, |r| <= 1/2; then
// round(c 2^36) = A 2^23 + round(r 2^23).
__device__ __forceinline__ long long fix_fast(float c)
{
    const float M = 12582912.0f;  // 1.5 * 2^23
    const float t = c * 8192.0f;
    const float ta = t + M;
    const int A = __float_as_int(ta) - 0x4B400000;
    const float r = t - (ta - M);
    const int Bq = __float_as_int(fmaf(r, 8388608.0f, M)) - 0x4B400000;
    return (long long)A * 8388608ll + Bq;
}

// fix_fast on the two lanes of a packed pair t = c 2^13 (the caller folds the
// exact power-of-two scale into its own multiplier): the same operations, so
// the same bits.  Valid for |t| < 2^22.
__device__ __forceinline__ void fix_t2(f2 t, long long &x0, long long &x1)
{
    const f2 M = f2_pack(12582912.0f, 12582912.0f);
    const f2 ta = f2_add(t, M);
    const f2 r = f2_sub(t, f2_sub(ta, M));
    const f2 u = f2_fma(r, f2_pack(8388608.0f, 8388608.0f), M);
    x0 = (long long)(__float_as_int(f2_lo(ta)) - 0x4B400000) * 8388608ll + (__float_as_int(f2_lo(u)) - 0x4B400000);
    x1 = (long long)(__float_as_int(f2_hi(ta)) - 0x4B400000) * 8388608ll + (__float_as_int(f2_hi(u)) - 0x4B400000);
}

// fix_fast on the two lanes of a packed pair.
__device__ __forceinline__ void fix_fast2(f2 c, long long &x0, long long &x1)
{
    fix_t2(f2_mul(c, f2_pack(8192.0f, 8192.0f)), x0, x1);
}

// Adds a 64-bit fixed-point term to a sum in shared memory with two 32-bit
// atomics (a 64-bit shared-memory atomic costs several times as much): the
// low word's atomic returns its previous value, which gives the carry out of
// bit 31 exactly, and the high word then gets (x >> 32) + carry (nothing when
// that is 0).  Every carry is counted once, by the addition that produced it,
// so once all additions are done the word holds the exact sum (mod 2^64)
// whatever their order.  A word is updated this way only (never by a 64-bit
// atomic at the same time).  split_lo / split_hi are the two halves, for
// callers that issue a batch of low-word atomics before their high words.
__device__ __forceinline__ unsigned split_lo(unsigned long long *p, long long x)
{
    return atomicAdd(reinterpret_cast<unsigned *>(p), (unsigned)x);
}

__device__ __forceinline__ void split_hi(unsigned long long *p, long long x, unsigned old)
{
    const unsigned l = (unsigned)x;
    const int d = (int)(x >> 32) + (old + l < l ? 1 : 0);
    if (d != 0) atomicAdd(reinterpret_cast<unsigned *>(p) + 1, (unsigned)d);
}

__device__ __forceinline__ void split_add(unsigned long long *p, long long x)
{
    split_hi(p, x, split_lo(p, x));
}

struct Fix {
    unsigned long long lo;  // main-plane part
    long long hi;           // high-word part (0 on the fast path)
};

__device__ __forceinline__ Fix to_fixed(float c)
{
    Fix f;
    if (fabsf(c) < 512.0f) {
        f.lo = (unsigned long long)fix_fast(c);
        f.hi = 0;
    } else {
        const float s = fminf(fmaxf(c, -1099511627776.0f), 1099511627776.0f) * 16.0f;  // |c| <= 2^40, times 2^4
        const float fl = floorf(s);
        f.hi = (long long)fl;
        f.lo = (unsigned long long)__float2ll_rn((s - fl) * 4294967296.0f);
    }
    return f;
}

}  // namespace
}  // namespace dn

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

// ---- the shared-memory num window of a filtering CTA ----
//
// There a pixel's sum is kept in units of 2^-F (F <= 36) as two 32-bit
// integer planes, the low and high words of its 64-bit slot: a term
// x = round(c 2^F) is split as x = h 2^s + l with 0 <= l < 2^s, l goes to the
// low plane and h to the high plane, each with a plain 32-bit atomic (no
// returned value, no carry), and the pixel's sum is H 2^s + L once the window
// is complete (win_value, which also rescales it to the global planes' 2^-36).
// With at most 2^m terms per pixel and window, s = 32 - m keeps L below 2^32,
// and terms with |x| < 2^(62 - 2m) keep |H| below 2^31 (|h| <= 2^(30 - m) + 1),
// so neither plane can overflow and the sum is exact; F = min(36, 54 - 2m)
// lets every term with |c| < 256 in (the rounding to 2^-F is then at most
// 2^-35 for m <= 10 and 2^-33 for m = 11), and a larger term goes to the
// global planes directly.  A term is formed as t = c 2^(F - 23) (an exact
// power-of-two scale folded into its weight), x = round(t 2^23).  (A 64-bit
// shared-memory atomic costs several times as much as a 32-bit one.)
struct WinFmt {
    int s;         // bits of the low plane: 32 - m, m >= 9
    int sh;        // 36 - F
    float tscale;  // 2^(F - 23)
    float tlim;    // the window takes terms with |t| < tlim = 2^(39 - 2m)
};

// The format for windows whose pixels receive at most max_terms terms.
inline WinFmt win_format(long long max_terms)
{
    int m = 9;
    while ((1ll << m) < max_terms) ++m;
    const int F = 54 - 2 * m < 36 ? 54 - 2 * m : 36;
    WinFmt f;
    f.s = 32 - m;
    f.sh = 36 - F;
    f.tscale = ldexpf(1.0f, F - 23);
    f.tlim = ldexpf(1.0f, 39 - 2 * m);
    return f;
}

// fix_t2's steps on both lanes of t (|t| < 2^22), stopped before the 64-bit
// composition: A = round(t), B = round((t - A) 2^23), so that
// round(t 2^23) = A 2^23 + B with |B| <= 2^22.
__device__ __forceinline__ void fix_parts2(f2 t, int (&A)[2], int (&B)[2])
{
    const f2 M = f2_pack(12582912.0f, 12582912.0f);
    const f2 ta = f2_add(t, M);
    const f2 r = f2_sub(t, f2_sub(ta, M));
    const f2 u = f2_fma(r, f2_pack(8388608.0f, 8388608.0f), M);
    A[0] = __float_as_int(f2_lo(ta)) - 0x4B400000;
    A[1] = __float_as_int(f2_hi(ta)) - 0x4B400000;
    B[0] = __float_as_int(f2_lo(u)) - 0x4B400000;
    B[1] = __float_as_int(f2_hi(u)) - 0x4B400000;
}

// Adds A 2^23 + B to a window slot: l = B mod 2^s, h = A 2^(23 - s) + floor(B / 2^s).
__device__ __forceinline__ void win_add(unsigned long long *p, int A, int B, int s)
{
    unsigned *w = reinterpret_cast<unsigned *>(p);
    atomicAdd(w, (unsigned)B & ((1u << s) - 1u));
    atomicAdd(w + 1, ((unsigned)A << (23 - s)) + (unsigned)(B >> s));
}

// Adds one term t (|t| < tlim) to a window slot.
__device__ __forceinline__ void win_add1(unsigned long long *p, float t, int s)
{
    int A[2], B[2];
    fix_parts2(f2_pack(t, 0.0f), A, B);
    win_add(p, A[0], B[0], s);
}

// The sum held by a window slot, in units of 2^-36.
__device__ __forceinline__ long long win_value(unsigned long long v, const WinFmt &f)
{
    const long long x = (long long)(int)(unsigned)(v >> 32) * (1ll << f.s) + (long long)(unsigned)(v & 0xFFFFFFFFull);
    return x * (1ll << f.sh);
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

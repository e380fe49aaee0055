// Exact fixed-point aggregation terms shared by the BM3D filtering kernels
// (FP32 SIMT, tensor-core and larger-patch paths): every contribution is
// rounded once to a fixed-point grid and added as an integer, so the sums do
// not depend on the order in which groups are aggregated.
#pragma once

#include "f32x2.cuh"

namespace dn {
namespace {

// num(x) = sum over (group g, patch q of g) of w_g kai(x - q) v_{g,q}(x - q) is
// accumulated per pixel; den(x) = sum_q kai(x - q) W(q), W(q) = the sum of the
// weights of the groups that hold patch q, is accumulated per patch position
// (one addition per patch) and correlated with the Kaiser window when
// normalising.  Both global sums are 64-bit fixed point with 36 fraction bits
// added with integer atomics, so they are bitwise reproducible whatever the
// order of the groups.  A weight goes there directly (rounded to 2^-36: exact
// whenever the FP32 value is >= 2^-13 in magnitude); a num term goes first to
// its CTA's shared window (below), rounded to that window's grid.  Weights are
// used scaled by sigma^2 (1/N_har, 1/sum w^2, or sigma^2 for an all-zero
// group), which leaves num/den unchanged.
//
// A term c added to a global plane directly with |c| < 512 goes to the
// 64-bit main plane as round(c 2^36) < 2^45; any other c (a heavy weight or a
// large value) is clamped to |c| <= 2^40 and split as c 2^36 = hi 2^32 + lo,
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

// ---- the shared-memory num window of a filtering CTA ----
//
// There a pixel's sum is kept in units of 2^-F (F <= 36) as two 32-bit
// integer planes (separate arrays, so that the 32 lanes of one atomic
// instruction, on 4 window rows of 8 consecutive pixels, hit 32 banks): a term
// x = round(c 2^F) is split as x = h 2^s + l with h = round(x / 2^s) and
// |l| <= 2^(s - 1), l goes to the low plane and h to the high plane, each with
// a plain 32-bit atomic (no returned value, no carry), and the pixel's sum is
// H 2^s + L once the window is complete (win_value, which also rescales it to
// the global planes' 2^-36).  With at most 2^m terms per pixel and window,
// s = 31 - m keeps |L| <= 2^30, and terms with |x| < 2^(61 - 2m) keep |H|
// below 2^31 (|h| < 2^(30 - m) + 1/2), so neither plane can overflow and the
// sum is exact; F = min(36, 53 - 2m) lets every term with |c| < 256 in (its
// rounding to 2^-F is at most 2^-34 for m <= 10 and 2^-32 for m = 11), and a
// larger term goes to the global planes directly.  A term is formed as
// t = c 2^(F - 23) (an exact power-of-two scale folded into its weight),
// x = round(t 2^23).  (A 64-bit shared-memory atomic costs several times as
// much as a 32-bit one, and the carry of a two-word sum needs the atomic's
// returned value.)
struct WinFmt {
    int s;         // 31 - m, m >= 9
    int sh;        // 36 - F
    float tscale;  // 2^(F - 23)
    float tlim;    // the window takes terms with |t| < tlim = 2^(38 - 2m)
};

// The format for windows whose pixels receive at most max_terms terms.
inline WinFmt win_format(long long max_terms)
{
    int m = 9;
    while ((1ll << m) < max_terms) ++m;
    const int F = 53 - 2 * m < 36 ? 53 - 2 * m : 36;
    WinFmt f;
    f.s = 31 - m;
    f.sh = 36 - F;
    f.tscale = ldexpf(1.0f, F - 23);
    f.tlim = ldexpf(1.0f, 38 - 2 * m);
    return f;
}

// round(t 2^23) = h 2^s + l with h = round(t 2^(23 - s)) and |l| <= 2^(s - 1),
// on both lanes of t (|t| < tlim).
__device__ __forceinline__ void win_parts2(f2 t, int s, int (&h)[2], int (&l)[2])
{
    const f2 M = f2_pack(12582912.0f, 12582912.0f);
    const float hs = __int_as_float((150 - s) << 23), ls = __int_as_float((104 + s) << 23);  // 2^(23-s), -2^(s-23)
    const f2 hf = f2_fma(t, f2_pack(hs, hs), M);
    const f2 r = f2_fma(f2_sub(hf, M), f2_pack(-ls, -ls), t);
    const f2 u = f2_fma(r, f2_pack(8388608.0f, 8388608.0f), M);
    h[0] = __float_as_int(f2_lo(hf)) - 0x4B400000;
    h[1] = __float_as_int(f2_hi(hf)) - 0x4B400000;
    l[0] = __float_as_int(f2_lo(u)) - 0x4B400000;
    l[1] = __float_as_int(f2_hi(u)) - 0x4B400000;
}

// Adds h 2^s + l to a window pixel (p in the low plane, the high plane
// `plane` words further).
__device__ __forceinline__ void win_red(unsigned *p, int plane, int h, int l)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"((unsigned)l) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + 4u * plane), "r"((unsigned)h) : "memory");
}

// Adds one term t (|t| < tlim) to a window pixel.
__device__ __forceinline__ void win_add1(unsigned *p, int plane, float t, int s)
{
    int h[2], l[2];
    win_parts2(f2_pack(t, 0.0f), s, h, l);
    win_red(p, plane, h[0], l[0]);
}

// The sum held by a window pixel (low and high plane words), in units of 2^-36.
__device__ __forceinline__ long long win_value(unsigned lo, unsigned hi, const WinFmt &f)
{
    return (long long)(((unsigned long long)(long long)(int)hi << (f.s + f.sh)) + ((unsigned long long)(long long)(int)lo << f.sh));
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

// Exact FP32 block-matching distance and the warp-per-reference exhaustive
// matcher shared by the matching kernels (internal header).
//
// Every path that ranks candidates with an FP32 distance evaluates
// d = ||P - Q||^2 / 64 with one fixed association, so equal pixel sets give
// bit-equal distances and the paths agree bit for bit.  With e_j the rounded
// differences of a patch row, the row sum is
//     (fma(e2, e2, fma(e1, e1, e0 e0)) + fma(e5, e5, fma(e4, e4, e3 e3)))
//         + fma(e7, e7, e6 e6)
// (the 3 + 3 + 2 split of ((e0^2 + e1^2) + e2^2) + ((e3^2 + e4^2) + e5^2) +
// (e6^2 + e7^2) with every "sum + e^2" a single fused multiply-add), and the
// 8 row sums are added as (((h0 + h1) + h2) + ((h3 + h4) + h5)) + (h6 + h7).
// The 3 + 3 + 2 split matches the reference grid step of 3, which lets the
// tiled kernel share partial sums between neighbouring references.  The
// fused multiply-adds are written out: left to itself the compiler fuses a
// product into a following sum in some kernels and not in others (measured
// for the packed FP32x2 instructions), which would break the bit equality.
#pragma once

#include "common.cuh"
#include "f32x2.cuh"

namespace dn {
namespace {

__device__ __forceinline__ float tree8(float a0, float a1, float a2, float a3, float a4, float a5, float a6, float a7)
{
    const float t0 = __fadd_rn(__fadd_rn(a0, a1), a2);
    const float t1 = __fadd_rn(__fadd_rn(a3, a4), a5);
    return __fadd_rn(__fadd_rn(t0, t1), __fadd_rn(a6, a7));
}

// Row sum of squares of 8 rounded differences in the fixed association.
__device__ __forceinline__ float row_sumsq(float e0, float e1, float e2, float e3, float e4, float e5, float e6,
                                           float e7)
{
    const float t0 = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
    const float t1 = __fmaf_rn(e5, e5, __fmaf_rn(e4, e4, __fmul_rn(e3, e3)));
    return __fadd_rn(__fadd_rn(t0, t1), __fmaf_rn(e7, e7, __fmul_rn(e6, e6)));
}

__device__ __forceinline__ f2 f2_tree8(f2 a0, f2 a1, f2 a2, f2 a3, f2 a4, f2 a5, f2 a6, f2 a7)
{
    const f2 t0 = f2_add(f2_add(a0, a1), a2);
    const f2 t1 = f2_add(f2_add(a3, a4), a5);
    return f2_add(f2_add(t0, t1), f2_add(a6, a7));
}

// ||P - Q||^2 for P = ref (row-major registers), Q read through q(i, j).
template <typename Q>
__device__ __forceinline__ float canon_d64(const float (&ref)[64], Q q)
{
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e[j] = __fsub_rn(ref[i * 8 + j], q(i, j));
        h[i] = row_sumsq(e[0], e[1], e[2], e[3], e[4], e[5], e[6], e[7]);
    }
    return tree8(h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7]);
}

// insert_sorted restricted to slots [S, L): valid when d >= bd[S - 1] (the
// candidate lands at or after slot S, so the slots before it do not move).
template <int L, int S>
__device__ __forceinline__ void insert_sorted_tail(float (&bd)[L], int (&bi)[L], float d, int id)
{
    bool after = d < bd[L - 1];
#pragma unroll
    for (int j = L - 1; j > S; --j) {
        const bool before_prev = d < bd[j - 1];
        bd[j] = before_prev ? bd[j - 1] : (after ? d : bd[j]);
        bi[j] = before_prev ? bi[j - 1] : (after ? id : bi[j]);
        after = before_prev;
    }
    if (after) {
        bd[S] = d;
        bi[S] = id;
    }
}

// Sorted insertion; candidates arrive in increasing index order, so a strict
// comparison keeps equal distances in index order.
template <int L>
__device__ __forceinline__ void insert_sorted(float (&bd)[L], int (&bi)[L], float d, int id)
{
    // slot j takes slot j-1 if d precedes it, else d if d precedes the old slot j
    bool after = d < bd[L - 1];
#pragma unroll
    for (int j = L - 1; j > 0; --j) {
        const bool before_prev = d < bd[j - 1];
        bd[j] = before_prev ? bd[j - 1] : (after ? d : bd[j]);
        bi[j] = before_prev ? bi[j - 1] : (after ? id : bi[j]);
        after = before_prev;
    }
    if (after) {
        bd[0] = d;
        bi[0] = id;
    }
}

// Group size from the number of kept candidates (reference excluded).
__device__ __forceinline__ int group_size(int kept, int n2)
{
    const int tot = min(kept + 1, n2);
    int n = 1;
    while (n * 2 <= tot) n *= 2;
    return n;
}

// Exhaustive exact matching of reference (rx, ry) of image g by one warp:
// lanes take every 32nd candidate of the window in row-major order, keep
// their own sorted top list, and the warp merges the 32 lists by repeated
// (d, index) minimum.  Writes out[0..n2) and *nout.  L = n2 - 1 (>= 1).
template <int L>
__device__ void match_ref_warp(const float *g, int H, int W, int step, int hs, float tau, int n2, int rx, int ry,
                               int *out, int *nout)
{
    const int lane = threadIdx.x & 31;
    const int x0 = min(rx * step, W - 8), y0 = min(ry * step, H - 8);
    float ref[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) ref[i * 8 + j] = g[(size_t)(y0 + i) * W + x0 + j];
    const int xs = max(0, x0 - hs), xe = min(W - 8, x0 + hs);
    const int ys = max(0, y0 - hs), ye = min(H - 8, y0 + hs);
    const int ww = xe - xs + 1, cnt = (ye - ys + 1) * ww;
    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);
        bi[j] = 0x7fffffff;
    }
    int kept = 0;
    for (int e = lane; e < cnt; e += 32) {
        const int y = ys + e / ww, x = xs + e % ww;
        if (y == y0 && x == x0) continue;
        const float *q = g + (size_t)y * W + x;
        const float d = __fmul_rn(canon_d64(ref, [&](int i, int j) { return q[(size_t)i * W + j]; }), 0.015625f);
        if (d <= tau) {
            ++kept;
            if (d < bd[L - 1]) insert_sorted<L>(bd, bi, d, y * W + x);
        }
    }
    kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0) out[0] = y0 * W + x0;
    int head = 0;
    for (int k = 0; k < L; ++k) {
        // lane's current head (lists are sorted; exhausted lists give +inf)
        float hd = __int_as_float(0x7f800000);
        int hi = 0x7fffffff;
#pragma unroll
        for (int j = 0; j < L; ++j)
            if (j == head) {
                hd = bd[j];
                hi = bi[j];
            }
        float md = hd;
        int mi = hi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, md, o);
            const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
            if (od < md || (od == md && oi < mi)) {
                md = od;
                mi = oi;
            }
        }
        if (hd == md && hi == mi && head < L) ++head;  // the winning lane pops its head
        if (lane == 0 && 1 + k < n2) out[1 + k] = (mi == 0x7fffffff) ? -1 : mi;
    }
    if (lane == 0) *nout = group_size(kept, n2);
}

}  // namespace
}  // namespace dn

// BM3D collaborative filtering and aggregation, FP32 SIMT path.
//
// First pass (hard thresholding), per group of n patches (n a power of 2):
//   Z = H_n (G T2D^T): 2D orthonormal DCT-II of every 8x8 patch, then the
//   normalised Walsh-Hadamard transform along the group; zero |Z| <= lambda
//   sigma; N_har = #kept; invert both; group weight 1/(sigma^2 N_har)
//   (1 when N_har = 0).
// Second pass (empirical Wiener), per group: the same 3D transform of the
//   basic-estimate group B and of the noisy group Y (same positions); gains
//   w = B^2 / (B^2 + sigma^2); estimate T3D^-1(w Y); weight 1/(sigma^2 sum w^2)
//   (1 when the sum is 0).
// Aggregation: every estimate pixel adds weight * kaiser(i) kaiser(j) * value to
// num and weight * kaiser(i) kaiser(j) to den; the output is num / den.  The
// sums are exact (fixed point, see fixed_point.cuh), so the result does not
// depend on the order in which groups are aggregated; den is formed from the
// per-position weight sums (see the aggregation section).
//
// Layout: a CTA owns a tile of reference positions, reads its patches from an
// image window staged in shared memory, and aggregates its groups into a
// shared-memory num window first (one global add per window pixel instead of
// one per contribution).  A warp filters one group at a time (in the first
// pass, two groups of at most 16 patches at once): lane k owns patch k,
// holds it in registers and computes its 8x8 DCT with an even/odd fast DCT,
// two 1D transforms per packed FP32x2 instruction (row pairs, then column
// pairs), and writes the spectrum to its row of a per-warp transpose buffer
// (rows of 65 floats, conflict-free both ways); for the group transform each
// lane owns two coefficient positions across all patches and runs the
// Walsh-Hadamard butterflies for both in packed registers (in the second
// pass the Wiener gains of the basic group wait in the warp's TMEM columns,
// 64 per lane, while the noisy group is transformed); the inverse goes back
// the same way, and the warp then aggregates in chunks of patches with its
// lanes spread over the 64 pixels (into the two 32-bit planes of the shared
// window, see WinFmt).
#include <cmath>

#include "common.cuh"
#include "f32x2.cuh"
#include "fixed_point.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kTS = 65;    // transpose buffer row stride (floats)
constexpr int kNMax = 32;

struct FilterArgs {
    const float *img;    // [b][C][H][W]: noisy (pass 2) or the image to filter (pass 1)
    const float *basic;  // pass 2 only
    const int *idx;
    const int *n;
    unsigned long long *num, *wsum;        // fixed-point sums per pixel / per patch position, layout of img
    unsigned long long *num_hi, *wsum_hi;  // their high words (signed, units of 2^32)
    int C, H, W, R, Rx, Ry, n2, step, hs;
    float lambda;
    WinFmt wf;  // format of the shared num window
    float sig[kChunk * 3];
    float kai[64];  // Kaiser outer product
};

// ---- 8-point orthonormal DCT-II and its inverse (even/odd decomposition), ----
// ---- two independent transforms per packed FP32x2 instruction            ----

// The DCT constants broadcast to both lanes (and negated where subtracted).
struct DctK2 {
    f2 h1, h2, h3, h5, h6, h7, r8, nh1, nh2, nh5, nh7;
};

// h_k = cos(k pi / 16) / 2 for k = 1..7 (h_4 = 1/sqrt(8)) and r8 = 1/sqrt(8),
// rounded to FP32: the constants of the orthonormal 8-point DCT with the 1/2
// scale folded in; as compile-time literals the packed pairs can be
// rematerialised instead of occupying registers.
constexpr float kH1 = 0.490392625f, kH2 = 0.461939752f, kH3 = 0.415734798f, kH5 = 0.277785122f,
                kH6 = 0.191341713f, kH7 = 0.0975451618f, kR8 = 0.353553385f;

__device__ __forceinline__ DctK2 pack_dct()
{
    DctK2 P;
    P.h1 = f2_pack(kH1, kH1);
    P.h2 = f2_pack(kH2, kH2);
    P.h3 = f2_pack(kH3, kH3);
    P.h5 = f2_pack(kH5, kH5);
    P.h6 = f2_pack(kH6, kH6);
    P.h7 = f2_pack(kH7, kH7);
    P.r8 = f2_pack(kR8, kR8);
    P.nh1 = f2_pack(-kH1, -kH1);
    P.nh2 = f2_pack(-kH2, -kH2);
    P.nh5 = f2_pack(-kH5, -kH5);
    P.nh7 = f2_pack(-kH7, -kH7);
    return P;
}

// The 8-point DCT and its inverse, on two vectors at once:
//   forward X[u] = a_u sum_m x[m] cos(pi (2m+1) u / 16),
//   inverse x[m] = sum_u a_u X[u] cos(pi (2m+1) u / 16).
__device__ __forceinline__ void dct8_2(f2 (&v)[8], const DctK2 &K)
{
    const f2 s0 = f2_add(v[0], v[7]), d0 = f2_sub(v[0], v[7]);
    const f2 s1 = f2_add(v[1], v[6]), d1 = f2_sub(v[1], v[6]);
    const f2 s2 = f2_add(v[2], v[5]), d2 = f2_sub(v[2], v[5]);
    const f2 s3 = f2_add(v[3], v[4]), d3 = f2_sub(v[3], v[4]);
    const f2 e0 = f2_add(s0, s3), e1 = f2_add(s1, s2), f0 = f2_sub(s0, s3), f1 = f2_sub(s1, s2);
    v[0] = f2_mul(K.r8, f2_add(e0, e1));
    v[4] = f2_mul(K.r8, f2_sub(e0, e1));
    v[2] = f2_fma(K.h2, f0, f2_mul(K.h6, f1));
    v[6] = f2_fma(K.h6, f0, f2_mul(K.nh2, f1));
    v[1] = f2_fma(K.h1, d0, f2_fma(K.h3, d1, f2_fma(K.h5, d2, f2_mul(K.h7, d3))));
    v[3] = f2_fma(K.h3, d0, f2_fma(K.nh7, d1, f2_fma(K.nh1, d2, f2_mul(K.nh5, d3))));
    v[5] = f2_fma(K.h5, d0, f2_fma(K.nh1, d1, f2_fma(K.h7, d2, f2_mul(K.h3, d3))));
    v[7] = f2_fma(K.h7, d0, f2_fma(K.nh5, d1, f2_fma(K.h3, d2, f2_mul(K.nh1, d3))));
}

__device__ __forceinline__ void idct8_2(f2 (&v)[8], const DctK2 &K)
{
    const f2 a = f2_mul(K.r8, f2_add(v[0], v[4])), b = f2_mul(K.r8, f2_sub(v[0], v[4]));
    const f2 p = f2_fma(K.h2, v[2], f2_mul(K.h6, v[6])), q = f2_fma(K.h6, v[2], f2_mul(K.nh2, v[6]));
    const f2 e0 = f2_add(a, p), e3 = f2_sub(a, p), e1 = f2_add(b, q), e2 = f2_sub(b, q);
    const f2 o0 = f2_fma(K.h1, v[1], f2_fma(K.h3, v[3], f2_fma(K.h5, v[5], f2_mul(K.h7, v[7]))));
    const f2 o1 = f2_fma(K.h3, v[1], f2_fma(K.nh7, v[3], f2_fma(K.nh1, v[5], f2_mul(K.nh5, v[7]))));
    const f2 o2 = f2_fma(K.h5, v[1], f2_fma(K.nh1, v[3], f2_fma(K.h7, v[5], f2_mul(K.h3, v[7]))));
    const f2 o3 = f2_fma(K.h7, v[1], f2_fma(K.nh5, v[3], f2_fma(K.h3, v[5], f2_mul(K.nh1, v[7]))));
    v[0] = f2_add(e0, o0);
    v[7] = f2_sub(e0, o0);
    v[1] = f2_add(e1, o1);
    v[6] = f2_sub(e1, o1);
    v[2] = f2_add(e2, o2);
    v[5] = f2_sub(e2, o2);
    v[3] = f2_add(e3, o3);
    v[4] = f2_sub(e3, o3);
}

// ---- group transform along the patches (one coefficient column) -------------

template <int N>
__device__ __forceinline__ float sqrt_n()
{
    return N == 1 ? 1.0f : N == 2 ? 1.41421356237309505f : N == 4 ? 2.0f : N == 8 ? 2.82842712474619010f
         : N == 16 ? 4.0f : 5.65685424949238019f;
}

// The group transform runs unnormalised: fwht twice multiplies by N, so the
// thresholds and gains below are expressed on the unscaled coefficients
// (|c| / sqrt(N) > thr  <=>  |c| > thr sqrt(N);  B^2 / N / (B^2 / N + s2) =
// B^2 / (B^2 + N s2)) and the exact power-of-two factor 1/N is applied to the
// aggregation weight of the estimate instead.

template <int N>
__device__ __forceinline__ void fwht2(f2 (&v)[N])
{
#pragma unroll
    for (int h = 1; h < N; h <<= 1)
#pragma unroll
        for (int i = 0; i < N; i += 2 * h)
#pragma unroll
            for (int j = i; j < i + h; ++j) {
                const f2 x = v[j], y = v[j + h];
                v[j] = f2_add(x, y);
                v[j + h] = f2_sub(x, y);
            }
}

// The lane's two coefficient columns (lane, lane + 32) of rows [0, N) of T,
// packed: column lane in the low half, column lane + 32 in the high half.
template <int N>
__device__ __forceinline__ void load_cols(const float *T, int lane, f2 (&v)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = f2_pack(T[k * kTS + lane], T[k * kTS + lane + 32]);
}

template <int N>
__device__ __forceinline__ void store_cols(float *T, int lane, const f2 (&v)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
        T[k * kTS + lane] = f2_lo(v[k]);
        T[k * kTS + lane + 32] = f2_hi(v[k]);
    }
}

// Hard threshold of the lane's two coefficient columns of an N-patch group in
// T; returns the number of kept coefficients.
template <int N>
__device__ __forceinline__ int hard_cols(float *T, int lane, float thr)
{
    f2 v[N];
    load_cols<N>(T, lane, v);
    fwht2<N>(v);
    const float thr_n = thr * sqrt_n<N>();
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float lo = f2_lo(v[k]), hi = f2_hi(v[k]);
        const bool klo = fabsf(lo) > thr_n, khi = fabsf(hi) > thr_n;
        cnt += (klo ? 1 : 0) + (khi ? 1 : 0);
        v[k] = f2_pack(klo ? lo : 0.0f, khi ? hi : 0.0f);
    }
    fwht2<N>(v);
    store_cols<N>(T, lane, v);
    return cnt;
}

// Wiener gains of the lane's two coefficient columns of the basic-estimate
// group in T, kept in registers (om); returns their sum of squares.
template <int N>
__device__ __forceinline__ float wiener_gains(const float *T, int lane, float s2, f2 (&om)[N])
{
    f2 v[N];
    load_cols<N>(T, lane, v);
    fwht2<N>(v);
    const float s2n = s2 * (float)N;
    const f2 s2n2 = f2_pack(s2n, s2n);
    f2 wsq = f2_pack(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const f2 b2 = f2_mul(v[k], v[k]);
        const f2 den = f2_add(b2, s2n2);  // >= sigma^2 > 0
        om[k] = f2_pack(__fdividef(f2_lo(b2), f2_lo(den)), __fdividef(f2_hi(b2), f2_hi(den)));
        wsq = f2_fma(om[k], om[k], wsq);
    }
    return f2_lo(wsq) + f2_hi(wsq);
}

// hard_cols<16> on two 16-patch groups at once (rows 0-15 and 16-31 of T):
// two independent chains for the scheduler to interleave.
__device__ __forceinline__ int2 hard_cols_pair16(float *T, int lane, float thr)
{
    f2 va[16], vb[16];
    load_cols<16>(T, lane, va);
    load_cols<16>(T + 16 * kTS, lane, vb);
    fwht2<16>(va);
    fwht2<16>(vb);
    const float thr_n = thr * sqrt_n<16>();
    int ca = 0, cb = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float alo = f2_lo(va[k]), ahi = f2_hi(va[k]), blo = f2_lo(vb[k]), bhi = f2_hi(vb[k]);
        const bool kalo = fabsf(alo) > thr_n, kahi = fabsf(ahi) > thr_n;
        const bool kblo = fabsf(blo) > thr_n, kbhi = fabsf(bhi) > thr_n;
        ca += (kalo ? 1 : 0) + (kahi ? 1 : 0);
        cb += (kblo ? 1 : 0) + (kbhi ? 1 : 0);
        va[k] = f2_pack(kalo ? alo : 0.0f, kahi ? ahi : 0.0f);
        vb[k] = f2_pack(kblo ? blo : 0.0f, kbhi ? bhi : 0.0f);
    }
    fwht2<16>(va);
    fwht2<16>(vb);
    store_cols<16>(T, lane, va);
    store_cols<16>(T + 16 * kTS, lane, vb);
    return make_int2(ca, cb);
}

__device__ __forceinline__ int hard_columns(float *T, int n, int lane, float thr)
{
    switch (n) {
        case 1: return hard_cols<1>(T, lane, thr);
        case 2: return hard_cols<2>(T, lane, thr);
        case 4: return hard_cols<4>(T, lane, thr);
        case 8: return hard_cols<8>(T, lane, thr);
        case 16: return hard_cols<16>(T, lane, thr);
        default: return hard_cols<32>(T, lane, thr);
    }
}

// Shared-memory state of one CTA for the current channel: the num window over
// pixels [Y0, Y0+RH) x [X0, X0+RW) (two planes of 32-bit words, row stride
// RS = 8 mod 32 words, so that four rows of 8 consecutive words fill all 32
// banks) and the image windows the patches are read from (row stride RW).
struct Window {
    unsigned *num;            // [2][RH][RS]: low and high planes (WinFmt)
    int plane;                // RH * RS
    const float *img;         // [RH][RW]: the image to filter (noisy in pass 2)
    const float *basic;       // [RH][RW]: pass 2 only
    int X0, Y0, RH, RW, RS;
};

// Loads a group's positions into lanes [base, base+n) (lane base+k gets patch
// k; other lanes keep theirs).  Returns n, 0 if the list is invalid (the group
// is skipped), or -n if it does not fit below row 32 (nothing loaded).
// The same from the group's size n and this lane's list entry rid (entry
// lane - base, loaded ahead by the caller).
__device__ __forceinline__ int decode_group(const FilterArgs &a, int n, int rid, int lane, int base, int &py, int &px)
{
    if (n < 1 || n > a.n2 || n > kNMax || (n & (n - 1)) != 0) return 0;
    if (base + n > 32) return -n;
    const bool mine = lane >= base && lane < base + n;
    const int id = mine ? rid : 0;
    const int y = id / a.W, x = id - (id / a.W) * a.W;
    const bool bad = mine && (id < 0 || y > a.H - 8 || x > a.W - 8);
    if (__any_sync(0xffffffffu, bad)) return 0;
    if (mine) {
        py = y;
        px = x;
    }
    return n;
}

__device__ __forceinline__ int load_group(const FilterArgs &a, int b, int r, int lane, int base, int &py, int &px)
{
    const size_t gr = (size_t)b * a.R + r;
    const int n = a.n[gr];
    if (n < 1 || n > a.n2 || n > kNMax || (n & (n - 1)) != 0) return 0;
    if (base + n > 32) return -n;
    const bool mine = lane >= base && lane < base + n;
    const int id = mine ? a.idx[gr * a.n2 + lane - base] : 0;
    const int y = id / a.W, x = id - (id / a.W) * a.W;
    const bool bad = mine && (id < 0 || y > a.H - 8 || x > a.W - 8);
    if (__any_sync(0xffffffffu, bad)) return 0;
    if (mine) {
        py = y;
        px = x;
    }
    return n;
}

__device__ __forceinline__ bool in_window(const Window &win, int py, int px)
{
    return py >= win.Y0 && py + 8 <= win.Y0 + win.RH && px >= win.X0 && px + 8 <= win.X0 + win.RW;
}

// Forward 2D DCT of the valid lanes' patches kept in registers: row pairs
// (r, r+1) packed for the row pass, column pairs (j, j+1) for the column pass;
// the result goes to row `lane` of T.
__device__ __forceinline__ void dct_reg(float *T, const Window &win, const float *wimg, const float *gimg, int W,
                                        bool valid, int lane, int py, int px, const DctK2 &K)
{
    const bool all_in = __all_sync(0xffffffffu, !valid || in_window(win, py, px));
    if (valid) {
        const float *src = all_in ? wimg + (py - win.Y0) * win.RW + (px - win.X0) : gimg + (size_t)py * W + px;
        const int stride = all_in ? win.RW : W;
        f2 x[4][8];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[r2][j] = f2_pack(src[2 * r2 * stride + j], src[(2 * r2 + 1) * stride + j]);
            dct8_2(x[r2], K);
        }
        float *row = T + lane * kTS;
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            f2 y[8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
                y[r] = (r & 1) ? f2_pack(f2_hi(x[r >> 1][j]), f2_hi(x[r >> 1][j + 1]))
                               : f2_pack(f2_lo(x[r >> 1][j]), f2_lo(x[r >> 1][j + 1]));
            dct8_2(y, K);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                row[r * 8 + j] = f2_lo(y[r]);
                row[r * 8 + j + 1] = f2_hi(y[r]);
            }
        }
    }
}

// Inverse 2D DCT of row `lane` of T in place, the patch kept in registers
// between the column pass and the row pass.
__device__ __forceinline__ void idct_reg(float *T, bool valid, int lane, const DctK2 &K)
{
    if (valid) {
        float *row = T + lane * kTS;
        f2 y[4][8];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
#pragma unroll
            for (int r = 0; r < 8; ++r) y[j2][r] = f2_pack(row[r * 8 + 2 * j2], row[r * 8 + 2 * j2 + 1]);
            idct8_2(y[j2], K);
        }
#pragma unroll
        for (int r = 0; r < 8; r += 2) {
            f2 x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                x[j] = (j & 1) ? f2_pack(f2_hi(y[j >> 1][r]), f2_hi(y[j >> 1][r + 1]))
                               : f2_pack(f2_lo(y[j >> 1][r]), f2_lo(y[j >> 1][r + 1]));
            idct8_2(x, K);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                row[r * 8 + j] = f2_lo(x[j]);
                row[(r + 1) * 8 + j] = f2_hi(x[j]);
            }
        }
    }
}

// The lane's gains om[0, N) to its TMEM lane, columns tm .. tm + 2N.
template <int N>
__device__ __forceinline__ void gains_to_tmem(uint32_t tm, const f2 (&om)[N])
{
    if constexpr (N >= 4) {
#pragma unroll
        for (int k = 0; k < N; k += 4) {
            const uint32_t r[8] = {(uint32_t)om[k].v, (uint32_t)(om[k].v >> 32), (uint32_t)om[k + 1].v,
                                   (uint32_t)(om[k + 1].v >> 32), (uint32_t)om[k + 2].v, (uint32_t)(om[k + 2].v >> 32),
                                   (uint32_t)om[k + 3].v, (uint32_t)(om[k + 3].v >> 32)};
            tc::tmem_st8(tm + 2 * k, r);
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) tc::tmem_st2(tm + 2 * k, (uint32_t)om[k].v, (uint32_t)(om[k].v >> 32));
    }
    tc::tmem_wait_st();
}

// Applies the gains kept in TMEM to the lane's two coefficient columns of the
// noisy group in T (in place), both columns per packed instruction.
template <int N>
__device__ __forceinline__ void wiener_apply_tm(float *T, int lane, uint32_t tm)
{
    f2 v[N];
    load_cols<N>(T, lane, v);
    fwht2<N>(v);
    if constexpr (N >= 8) {
#pragma unroll
        for (int k = 0; k < N; k += 8) {
            uint32_t r[16];
            tc::tmem_ld16(tm + 2 * k, r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                f2 g;
                g.v = (unsigned long long)r[2 * q] | ((unsigned long long)r[2 * q + 1] << 32);
                v[k + q] = f2_mul(v[k + q], g);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            uint32_t r0, r1;
            tc::tmem_ld2(tm + 2 * k, r0, r1);
            tc::tmem_wait_ld();
            f2 g;
            g.v = (unsigned long long)r0 | ((unsigned long long)r1 << 32);
            v[k] = f2_mul(v[k], g);
        }
    }
    fwht2<N>(v);
    store_cols<N>(T, lane, v);
}

// Wiener transform of one group of N patches (rows [0, N) of T): gains from
// the basic-estimate group, parked in the warp's TMEM columns while the noisy
// patches are transformed, then applied to the noisy group; T is left holding
// the filtered spectra of the noisy patches.
template <int N>
__device__ __forceinline__ float wiener_group(const FilterArgs &a, const Window &win, float *T, size_t cbase,
                                              int lane, int py, int px, float s2, const DctK2 &K, uint32_t tm)
{
    dct_reg(T, win, win.basic, a.basic + cbase, a.W, lane < N, lane, py, px, K);
    __syncwarp();
    float wsq;
    {
        f2 om[N];
        wsq = wiener_gains<N>(T, lane, s2, om);
        gains_to_tmem<N>(tm, om);
    }
    __syncwarp();
    dct_reg(T, win, win.img, a.img + cbase, a.W, lane < N, lane, py, px, K);
    __syncwarp();
    wiener_apply_tm<N>(T, lane, tm);
    return wsq;
}

// Aggregation of the estimates in rows [s, s+n) of T (one group, weight w).
// The weight goes to the patch positions (lane k adds it for row k); for num
// the warp walks the patches and its lanes cover the 64 pixels of each (lane
// l: pixels l and l+32), so the window atomics of one instruction hit 4 rows
// of 8 consecutive words (no bank conflict).  When every patch of the group
// lies inside the window (always, for lists from this library's matcher) the
// patches go in chunks of up to 8: the chunk's terms are formed first and
// one warp vote picks the branch-free fast path for the whole chunk, so the
// chunk's conversions and atomics are independent and overlap.

// Terms of patches [k0, k0+K) scaled by 2^(F - 23) (wk carries the exact factor),
// then their exact fixed-point additions to the window (or, for a chunk with
// a term beyond the window's bound, to the global planes); wo = the window
// offset of the lane's own patch, poff = the lane's pixel offset.
template <int K>
__device__ __forceinline__ void agg_chunk(const FilterArgs &a, const Window &win, const float *T, size_t cbase, int k0,
                                          int lane, f2 wk, int wo, int poff, int gpos, int pg)
{
    f2 t[K];
    bool fast = true;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int k = k0 + q;
        t[q] = f2_mul(wk, f2_pack(T[k * kTS + lane], T[k * kTS + lane + 32]));
        fast = fast && fabsf(f2_lo(t[q])) < a.wf.tlim && fabsf(f2_hi(t[q])) < a.wf.tlim;
    }
    if (__all_sync(0xffffffffu, fast)) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int o = __shfl_sync(0xffffffffu, wo, k0 + q) + poff;
            int h[2], l[2];
            win_parts2(t[q], a.wf.s, h, l);
            win_red(win.num + o, win.plane, h[0], l[0]);
            win_red(win.num + o + 4 * win.RS, win.plane, h[1], l[1]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const size_t g = cbase + (size_t)__shfl_sync(0xffffffffu, gpos, k0 + q) + pg;
            const float ri = 1.0f / a.wf.tscale;  // exact: a power of two
            const Fix f0 = to_fixed(f2_lo(t[q]) * ri), f1 = to_fixed(f2_hi(t[q]) * ri);
            atomicAdd(a.num + g, f0.lo);
            atomicAdd(a.num + g + 4 * (size_t)a.W, f1.lo);
            if (f0.hi != 0) atomicAdd(a.num_hi + g, (unsigned long long)f0.hi);
            if (f1.hi != 0) atomicAdd(a.num_hi + g + 4 * (size_t)a.W, (unsigned long long)f1.hi);
        }
    }
}

__device__ __forceinline__ void aggregate(const FilterArgs &a, const Window &win, const float *T, size_t cbase, int s,
                                          int n, int lane, int py, int px, float w, const float (&ka)[2])
{
    const float vs = 1.0f / (float)n;  // the unnormalised group transform's factor n (exact power of two)
    const bool mine = lane >= s && lane < s + n;
    if (mine) {
        const Fix fw = to_fixed(w);
        const size_t q = cbase + (size_t)py * a.W + px;
        atomicAdd(a.wsum + q, fw.lo);
        if (fw.hi != 0) atomicAdd(a.wsum_hi + q, (unsigned long long)fw.hi);
    }
    const int i0 = lane >> 3, j = lane & 7;
    const int ly = py - win.Y0, lx = px - win.X0;
    const bool in = ly >= 0 && ly + 8 <= win.RH && lx >= 0 && lx + 8 <= win.RW;
    const unsigned gm = n == 32 ? 0xffffffffu : ((1u << n) - 1u) << s;
    if ((__ballot_sync(0xffffffffu, in && mine) & gm) == gm) {
        // w kai / n times the window's scale (exact powers of two)
        const f2 wk = f2_pack(w * ka[0] * vs * a.wf.tscale, w * ka[1] * vs * a.wf.tscale);
        const int wo = ly * win.RS + lx, poff = i0 * win.RS + j, gpos = py * a.W + px, pg = i0 * a.W + j;
        switch (n) {
            case 1: agg_chunk<1>(a, win, T, cbase, s, lane, wk, wo, poff, gpos, pg); break;
            case 2: agg_chunk<2>(a, win, T, cbase, s, lane, wk, wo, poff, gpos, pg); break;
            case 4: agg_chunk<4>(a, win, T, cbase, s, lane, wk, wo, poff, gpos, pg); break;
            case 16:  // the common first-pass size, unrolled (4.48 -> 4.42 ms; 32 unrolled was slower)
                agg_chunk<8>(a, win, T, cbase, s, lane, wk, wo, poff, gpos, pg);
                agg_chunk<8>(a, win, T, cbase, s + 8, lane, wk, wo, poff, gpos, pg);
                break;
            default:
                for (int k0 = s; k0 < s + n; k0 += 8) agg_chunk<8>(a, win, T, cbase, k0, lane, wk, wo, poff, gpos, pg);
                break;
        }
        return;
    }
    const f2 wk = f2_pack(w * ka[0] * vs, w * ka[1] * vs);
#pragma unroll 2
    for (int k = s; k < s + n; ++k) {
        const int yk = __shfl_sync(0xffffffffu, py, k), xk = __shfl_sync(0xffffffffu, px, k);
        const int ly0 = yk - win.Y0, lx0 = xk - win.X0;
        const bool inside = ly0 >= 0 && ly0 + 8 <= win.RH && lx0 >= 0 && lx0 + 8 <= win.RW;
        // the lane's two pixels (rows i0 and i0 + 4 of the patch, column j)
        const f2 c = f2_mul(wk, f2_pack(T[k * kTS + lane], T[k * kTS + lane + 32]));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + 4 * h;
            const float ch = h ? f2_hi(c) : f2_lo(c);
            if (inside && fabsf(ch) * a.wf.tscale < a.wf.tlim) {
                win_add1(win.num + (ly0 + i) * win.RS + lx0 + j, win.plane, ch * a.wf.tscale, a.wf.s);
            } else {
                const Fix f = to_fixed(ch);
                atomicAdd(a.num + cbase + (size_t)(yk + i) * a.W + xk + j, f.lo);
                if (f.hi != 0)
                    atomicAdd(a.num_hi + cbase + (size_t)(yk + i) * a.W + xk + j, (unsigned long long)f.hi);
            }
        }
    }
}

// First pass on one batch of at most two groups: group A in rows [0, nA),
// group B (nB may be 0) in rows [16, 16+nB).  Positions are already loaded.
__device__ __forceinline__ void hard_batch(const FilterArgs &a, const Window &win, float *T, size_t cbase, float sig,
                                           int nA, int nB, int lane, int py, int px, const float (&ka)[2])
{
    const bool valid = lane < nA || (lane >= 16 && lane < 16 + nB);
    dct_reg(T, win, win.img, a.img + cbase, a.W, valid, lane, py, px, pack_dct());
    __syncwarp();
    const float thr = a.lambda * sig;
    int nharA, nharB;
    if (nA == 16 && nB == 16) {
        const int2 cc = hard_cols_pair16(T, lane, thr);
        nharA = __reduce_add_sync(0xffffffffu, cc.x);
        nharB = __reduce_add_sync(0xffffffffu, cc.y);
    } else {
        nharA = __reduce_add_sync(0xffffffffu, hard_columns(T, nA, lane, thr));
        nharB = nB ? __reduce_add_sync(0xffffffffu, hard_columns(T + 16 * kTS, nB, lane, thr)) : 0;
    }
    // 1/(sigma^2 N_har), or 1 when nothing survives, both times sigma^2
    const float wA = nharA > 0 ? 1.0f / (float)nharA : sig * sig;
    const float wB = nharB > 0 ? 1.0f / (float)nharB : sig * sig;
    __syncwarp();
    idct_reg(T, valid, lane, pack_dct());
    __syncwarp();
    aggregate(a, win, T, cbase, 0, nA, lane, py, px, wA, ka);
    if (nB) aggregate(a, win, T, cbase, 16, nB, lane, py, px, wB, ka);
    __syncwarp();
}

// Second pass on one group of n patches (rows [0, n)).
__device__ __forceinline__ void wiener_one(const FilterArgs &a, const Window &win, float *T, size_t cbase, float sig,
                                           int n, int lane, int py, int px, const float (&ka)[2], uint32_t tm)
{
    const float s2 = sig * sig;
    float wsq;
    switch (n) {
        case 1: wsq = wiener_group<1>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
        case 2: wsq = wiener_group<2>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
        case 4: wsq = wiener_group<4>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
        case 8: wsq = wiener_group<8>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
        case 16: wsq = wiener_group<16>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
        default: wsq = wiener_group<32>(a, win, T, cbase, lane, py, px, s2, pack_dct(), tm); break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsq += __shfl_xor_sync(0xffffffffu, wsq, o);
    const float w = wsq > 0.0f ? 1.0f / wsq : s2;  // 1/(sigma^2 sum w^2) or 1, times sigma^2
    __syncwarp();
    idct_reg(T, lane < n, lane, pack_dct());
    __syncwarp();
    aggregate(a, win, T, cbase, 0, n, lane, py, px, w, ka);
    __syncwarp();
}

// A CTA owns a TR x TR tile of reference positions; per channel it stages the
// image window covering every patch its groups can hold (tile + search radius
// + patch) in shared memory, its warps filter the tile's groups and add num
// into a shared window, and the window is then added once to the global plane.
// In the first pass a warp takes the tile's references two at a time and
// filters both groups together when each has at most 16 patches.
template <bool WIENER>
__global__ void __launch_bounds__(512) k_filter(FilterArgs a, int TR, int RH, int RW, int RS)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    const int nw = blockDim.x >> 5;
    Window win;
    win.num = reinterpret_cast<unsigned *>(dsm_raw);
    win.plane = RH * RS;
    win.RH = RH;
    win.RW = RW;
    win.RS = RS;
    float *simg = reinterpret_cast<float *>(win.num + 2 * (size_t)RH * RS);  // [1 or 2][RH][RW]
    float *tbufs = simg + (size_t)(WIENER ? 2 : 1) * RH * RW;            // [nw][32][65]
    win.img = simg;
    win.basic = WIENER ? simg + (size_t)RH * RW : nullptr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z;
    const int rx0 = blockIdx.x * TR, ry0 = blockIdx.y * TR;
    const int Rx = a.Rx, Ry = a.Ry;
    const int gx0 = min(rx0 * a.step, a.W - 8), gy0 = min(ry0 * a.step, a.H - 8);
    win.X0 = max(0, gx0 - a.hs);
    win.Y0 = max(0, gy0 - a.hs);
    const float ka[2] = {a.kai[lane], a.kai[lane + 32]};
    // Wiener pass: 64 TMEM columns per warp (its lane quarter) park the gains
    __shared__ uint32_t s_tmem;
    if (WIENER) {
        if (warp == 0) tc::tmem_alloc(&s_tmem, 256);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    const uint32_t tm = WIENER ? s_tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(warp >> 2) * 64 : 0u;

    float *T = tbufs + (size_t)warp * 32 * kTS;
    const int tw = min(TR, Rx - rx0), th = min(TR, Ry - ry0), cnt = tw * th;
    const size_t HW = (size_t)a.H * a.W;
    const int rh = min(RH, a.H - win.Y0), rw = min(RW, a.W - win.X0);
    auto ref_of = [&](int q) { return (ry0 + q / tw) * Rx + rx0 + q % tw; };

    __shared__ int s_next[2];
    for (int c = 0; c < a.C; ++c) {
        const size_t cbase = ((size_t)b * a.C + c) * HW;
        const float sig = a.sig[b * 3 + c];
        if (threadIdx.x == 0) s_next[c & 1] = 0;
        for (int i = threadIdx.x; i < (2 * RH * RS) / 4; i += blockDim.x)
            reinterpret_cast<uint4 *>(win.num)[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int ly = warp; ly < rh; ly += nw) {
            const float *gi = a.img + cbase + (size_t)(win.Y0 + ly) * a.W + win.X0;
            const float *gb = WIENER ? a.basic + cbase + (size_t)(win.Y0 + ly) * a.W + win.X0 : nullptr;
            for (int lx = lane; lx < rw; lx += 32) {
                tc::cp_async4(tc::smem_u32(simg + ly * RW + lx), gi + lx);
                if (WIENER) tc::cp_async4(tc::smem_u32(simg + (size_t)RH * RW + ly * RW + lx), gb + lx);
            }
        }
        tc::cp_async_commit();
        tc::cp_async_wait<0>();
        __syncthreads();
        // the next group's list is loaded while the current one is filtered
        auto grab = [&](int per) {
            int q = 0;
            if (lane == 0) q = per * atomicAdd(&s_next[c & 1], 1);
            return __shfl_sync(0xffffffffu, q, 0);
        };
        auto raw = [&](int q, int base, int &n, int &rid) {
            const size_t gr = (size_t)b * a.R + ref_of(q);
            n = a.n[gr];
            if (lane >= base && lane - base < a.n2) rid = a.idx[gr * a.n2 + lane - base];
        };
        if (WIENER) {
            int q = grab(1), rn = 0, rid = 0;
            if (q < cnt) raw(q, 0, rn, rid);
            while (q < cnt) {
                const int qn = grab(1);
                int nn = 0, nid = 0;
                if (qn < cnt) raw(qn, 0, nn, nid);
                int py = 0, px = 0;
                const int n = decode_group(a, rn, rid, lane, 0, py, px);
                if (n > 0) wiener_one(a, win, T, cbase, sig, n, lane, py, px, ka, tm);
                q = qn;
                rn = nn;
                rid = nid;
            }
        } else if (a.n2 <= 16) {
            // group pairs: lanes 0-15 hold the first group's entries, lanes 16-31 the second's
            int q = grab(2), rnA = 0, rnB = 0, rid = 0;
            if (q < cnt) raw(q, 0, rnA, rid);
            if (q + 1 < cnt) raw(q + 1, 16, rnB, rid);
            while (q < cnt) {
                const int qn = grab(2);
                int nA_ = 0, nB_ = 0, nid = 0;
                if (qn < cnt) raw(qn, 0, nA_, nid);
                if (qn + 1 < cnt) raw(qn + 1, 16, nB_, nid);
                int py = 0, px = 0;
                const int nA = decode_group(a, rnA, rid, lane, 0, py, px);
                int nB = 0;
                if (q + 1 < cnt) {
                    nB = nA > 0 ? decode_group(a, rnB, rid, lane, 16, py, px) : -1;
                    if (nB < 0) nB = -1;  // filtered on its own below
                }
                if (nA > 0) hard_batch(a, win, T, cbase, sig, nA, nB > 0 ? nB : 0, lane, py, px, ka);
                if (nB < 0) {
                    const int n = load_group(a, b, ref_of(q + 1), lane, 0, py, px);
                    if (n > 0) hard_batch(a, win, T, cbase, sig, n, 0, lane, py, px, ka);
                }
                q = qn;
                rnA = nA_;
                rnB = nB_;
                rid = nid;
            }
        } else {
            for (;;) {
                int q = 0;
                if (lane == 0) q = 2 * atomicAdd(&s_next[c & 1], 1);
                q = __shfl_sync(0xffffffffu, q, 0);
                if (q >= cnt) break;
                int py = 0, px = 0;
                const int nA = load_group(a, b, ref_of(q), lane, 0, py, px);
                int nB = 0;
                if (q + 1 < cnt) {
                    nB = nA > 0 && nA <= 16 ? load_group(a, b, ref_of(q + 1), lane, 16, py, px) : -1;
                    if (nB < 0 || nB > 16) nB = -1;  // filtered on its own below
                }
                if (nA > 0) hard_batch(a, win, T, cbase, sig, nA, nB > 0 ? nB : 0, lane, py, px, ka);
                if (nB < 0) {
                    const int n = load_group(a, b, ref_of(q + 1), lane, 0, py, px);
                    if (n > 0) hard_batch(a, win, T, cbase, sig, n, 0, lane, py, px, ka);
                }
            }
        }
        __syncthreads();
        for (int ly = warp; ly < rh; ly += nw) {
            unsigned long long *gn = a.num + cbase + (size_t)(win.Y0 + ly) * a.W + win.X0;
            for (int lx = lane; lx < rw; lx += 32) {
                const long long v = win_value(win.num[ly * RS + lx], win.num[win.plane + ly * RS + lx], a.wf);
                if (v != 0) atomicAdd(gn + lx, (unsigned long long)v);
            }
        }
        __syncthreads();  // the windows are refilled for the next channel
    }
    if (WIENER) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            tc::fence_after_sync();
            tc::tmem_dealloc(s_tmem, 256);
        }
    }
}

// A fixed-point sum (main + hi 2^32, in units of 2^-36) as an FP32 value in
// the same units, from 32-bit halves (the int64 -> FP64 path would run on the
// narrow FP64 unit): relative error <= 2^-23.
__device__ __forceinline__ float fixed_to_float(long long main, long long hi)
{
    const float m = fmaf((float)(int)(main >> 32), 4294967296.0f, (float)(unsigned)(main & 0xFFFFFFFFll));
    if (hi == 0) return m;
    const float h = fmaf((float)(int)(hi >> 32), 4294967296.0f, (float)(unsigned)(hi & 0xFFFFFFFFll));
    return fmaf(h, 4294967296.0f, m);
}

// out = num / den, den(y, x) = sum_{i,j} k_i k_j W(y - i, x - j) over patch
// positions (i, j < K, the patch side), evaluated separably in FP32 (fixed
// order, so reproducible) from the exact weight sums.  One CTA per 32 x 32
// output tile of one plane.
constexpr int kNT = 32;

struct Kaiser1 {
    float k[16];
};

template <int K>
__global__ void __launch_bounds__(256) k_normalize(const long long *num, const long long *wsum,
                                                   const long long *num_hi, const long long *wsum_hi, float *out,
                                                   int H, int W, Kaiser1 kw)
{
    __shared__ float sw[kNT + K - 1][kNT + K];  // W at positions (y0-K+1.., x0-K+1..)
    __shared__ float sr[kNT + K - 1][kNT + 1];  // row pass
    const size_t base = (size_t)blockIdx.z * H * W;
    const int y0 = blockIdx.y * kNT, x0 = blockIdx.x * kNT;
    for (int e = threadIdx.x; e < (kNT + K - 1) * (kNT + K - 1); e += blockDim.x) {
        const int r = e / (kNT + K - 1), cc = e - r * (kNT + K - 1);
        const int y = y0 - (K - 1) + r, x = x0 - (K - 1) + cc;
        float v = 0.0f;
        if (y >= 0 && y < H && x >= 0 && x < W) {
            const size_t i = base + (size_t)y * W + x;
            v = fixed_to_float(wsum[i], wsum_hi[i]);
        }
        sw[r][cc] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (kNT + K - 1) * kNT; e += blockDim.x) {
        const int r = e / kNT, cc = e - r * kNT;
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(kw.k[j], sw[r][cc + K - 1 - j], acc);
        sr[r][cc] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNT * kNT; e += blockDim.x) {
        const int r = e / kNT, cc = e - r * kNT;
        const int y = y0 + r, x = x0 + cc;
        if (y >= H || x >= W) continue;
        float den = 0.0f;
#pragma unroll
        for (int i = 0; i < K; ++i) den = fmaf(kw.k[i], sr[r + K - 1 - i][cc], den);
        const size_t o = base + (size_t)y * W + x;
        out[o] = fixed_to_float(num[o], num_hi[o]) / den;  // the 2^36 scale cancels
    }
}

dn_status filter_common(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B,
                        int C, int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    FilterArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.R = a.Ry * a.Rx;
    a.n2 = p.n2;
    a.step = p.step;
    a.hs = p.search / 2;
    a.lambda = p.lambda3d;
    Tables t;
    make_tables(p.beta, &t);
    for (int i = 0; i < 64; ++i) a.kai[i] = t.kai[i];
    const size_t HW = (size_t)H * W, N = (size_t)B * C * HW;
    // tile of references per CTA and its aggregation window
    const int nwarps = 16;
    const int nimg = wiener ? 2 : 1;
    const size_t per_warp = (size_t)32 * kTS * sizeof(float);
    int TR = 16;
    int RH = 0, RW = 0, RS = 0;
    size_t smem = 0;
    for (; TR >= 1; TR /= 2) {
        RH = (TR - 1) * p.step + 2 * a.hs + 8;
        RW = RH;
        RS = RW + ((8 - RW % 32) + 32) % 32;  // row stride = 8 (mod 32) words
        smem = (size_t)nwarps * per_warp + (size_t)RH * RS * sizeof(unsigned long long) +
               (size_t)nimg * RH * RW * sizeof(float);
        if (smem <= 225 * 1024) break;
    }
    if (TR < 1) return DN_EUNSUPPORTED;
    a.wf = win_format((long long)TR * TR * p.n2);  // a pixel gets at most one term per patch of each group
    const void *fn = wiener ? (const void *)k_filter<true> : (const void *)k_filter<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        const size_t off = (size_t)b0 * C * HW;
        a.img = img + off;
        a.basic = basic ? basic + off : nullptr;
        a.idx = idx + (size_t)b0 * a.R * p.n2;
        a.n = n + (size_t)b0 * a.R;
        unsigned long long *fx = reinterpret_cast<unsigned long long *>(acc);
        a.num = fx + off;
        a.wsum = fx + N + off;
        a.num_hi = fx + 2 * N + off;
        a.wsum_hi = fx + 3 * N + off;
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < 3; ++c) a.sig[i * 3 + c] = c < C ? sig[(size_t)(b0 + i) * C + c] : 0.0f;
        dim3 grid((a.Rx + TR - 1) / TR, (a.Ry + TR - 1) / TR, nb);
        dn_status st = wiener ? launch("bm3d_filter_wiener_fp32", s,
                                       [&] { k_filter<true><<<grid, nwarps * 32, smem, s>>>(a, TR, RH, RW, RS); })
                              : launch("bm3d_filter_hard_fp32", s,
                                       [&] { k_filter<false><<<grid, nwarps * 32, smem, s>>>(a, TR, RH, RW, RS); });
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace

dn_status filter_hard_fp32(const float *img, const int *idx, const int *n, int B, int C, int H, int W,
                           const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    return filter_common(false, img, nullptr, idx, n, B, C, H, W, sig, p, acc, s);
}

dn_status filter_wiener_fp32(const float *noisy, const float *basic, const int *idx, const int *n, int B, int C,
                             int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    return filter_common(true, noisy, basic, idx, n, B, C, H, W, sig, p, acc, s);
}

dn_status normalize(const float *acc, float *out, int B, int C, int H, int W, float beta, cudaStream_t s, int K)
{
    const size_t N = (size_t)B * C * H * W;
    Kaiser1 kw;
    if (K == 8) {
        Tables t;
        make_tables(beta, &t);
        for (int i = 0; i < 8; ++i) kw.k[i] = t.kai1[i];
    } else if (K == 11 || K == 12) {
        make_kaiser(K, beta, kw.k);
    } else {
        return DN_EUNSUPPORTED;
    }
    const dim3 grid((W + kNT - 1) / kNT, (H + kNT - 1) / kNT, B * C);
    return launch("bm3d_normalize", s, [&] {
        const long long *fx = reinterpret_cast<const long long *>(acc);
        if (K == 8) k_normalize<8><<<grid, 256, 0, s>>>(fx, fx + N, fx + 2 * N, fx + 3 * N, out, H, W, kw);
        else if (K == 11) k_normalize<11><<<grid, 256, 0, s>>>(fx, fx + N, fx + 2 * N, fx + 3 * N, out, H, W, kw);
        else k_normalize<12><<<grid, 256, 0, s>>>(fx, fx + N, fx + 2 * N, fx + 3 * N, out, H, W, kw);
    });
}

}  // namespace dn

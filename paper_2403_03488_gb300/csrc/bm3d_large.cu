// BM3D with larger patches: the high-noise profile's 12 x 12 first pass and
// 11 x 11 second pass (patch sides 11 and 12), FP32 SIMT.
//
// The definitions are those of the 8 x 8 kernels with the patch side K a
// template parameter:
//   matching     d(P, Q) = ||P - Q||^2 / K^2 on pixels, or ||Y(P) - Y(Q)||^2 / K^2
//                on 2D-prethresholded K-point DCT-II coefficients (first pass
//                at high noise); the reference first, then ascending
//                (d, y W + x) among the candidates with d <= tau; group size
//                the largest power of two <= min(#kept, n2);
//   filtering    orthonormal K x K DCT-II of every patch, normalised
//                Walsh-Hadamard transform along the group, hard threshold
//                lambda sigma with group weight 1/(sigma^2 N_har) (pass 1) or
//                empirical Wiener gains B^2/(B^2 + sigma^2) of the basic
//                estimate's group with weight 1/(sigma^2 sum gains^2) (pass 2),
//                inverse transforms, Kaiser(K) x Kaiser(K) window;
//   aggregation  the exact 64-bit fixed-point sums of fixed_point.cuh (num per
//                pixel, group weights per patch position), divided by
//                normalize() with the same K.
//
// k_match_k: a CTA owns 16 x 8 references and stages the union of their
// search windows in shared memory; a thread owns one reference and walks its
// window in chunks of 8 horizontally adjacent candidates: per patch row it
// loads the reference row and the K + 7 candidate pixels once and forms the 8
// row sums of squares (16 K + 7 loads per 8 K^2 differences).
// k_match_pre_k: the prethresholded distance with the row-by-row structure of
// the 8 x 8 kernel (a ring of K row transforms, the column transforms of one
// candidate row staged in shared memory, the reference's K^2 coefficients in
// registers); K a multiple of 4 and n2 <= 16 (the first pass's group size).
// k_filter_k: a CTA owns a tile of references and shared-memory windows of the
// image (and basic estimate) and of the num plane covering every patch its
// groups can hold; a warp filters one group at a time: the group's patches are
// gathered from the window into a per-warp buffer (odd row and patch strides),
// the 2D transforms run as K-point matrix products with the DCT matrix in the
// kernel parameters, the lanes spread over (patch, row) and then (patch,
// column) jobs; lanes then own coefficient columns for the Walsh-Hadamard
// stage, the inverse goes back the same way, and the warp aggregates patch by
// patch with its lanes spread over the K^2 pixels.
#include <cmath>

#include "common.cuh"
#include "fixed_point.cuh"
#include "tc.cuh"
#include "match_exact.cuh"

namespace dn {

namespace {

constexpr int kKMax = 16;

// K-point orthonormal DCT-II matrix C[u][m] = a_u cos(pi (2m+1) u / (2K)) and
// the Kaiser window of length K, built on the host from their definitions.
struct LargeTables {
    float C[kKMax * kKMax];
    float kai[kKMax];
};

void make_large_tables(int K, float beta, LargeTables *t)
{
    const double pi = 3.14159265358979323846;
    for (int u = 0; u < K; ++u)
        for (int m = 0; m < K; ++m) {
            const double au = u == 0 ? std::sqrt(1.0 / K) : std::sqrt(2.0 / K);
            t->C[u * K + m] = (float)(au * std::cos(pi * (2 * m + 1) * u / (2.0 * K)));
        }
    make_kaiser(K, beta, t->kai);
}

// ---- pixel-domain matching ---------------------------------------------------

constexpr int kMX = 16, kMY = 8, kMT = kMX * kMY;

struct MatchKArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, pitch;
    float tau[kChunk];
    int *idx;
    int *n;
    int n2;
};

template <int K, int L>
__global__ void __launch_bounds__(kMT) k_match_k(const __grid_constant__ MatchKArgs a)
{
    extern __shared__ float sm[];
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W;
    const int rx0 = blockIdx.x * kMX, ry0 = blockIdx.y * kMY;
    const int rx = rx0 + threadIdx.x % kMX, ry = ry0 + threadIdx.x / kMX;

    const int gx_first = min(rx0 * a.step, W - K);
    const int gx_last = min(min(rx0 + kMX - 1, a.Rx - 1) * a.step, W - K);
    const int gy_first = min(ry0 * a.step, H - K);
    const int gy_last = min(min(ry0 + kMY - 1, a.Ry - 1) * a.step, H - K);
    const int X0 = max(0, gx_first - a.hs), X1 = min(W - 1, gx_last + a.hs + K - 1);
    const int Y0 = max(0, gy_first - a.hs), Y1 = min(H - 1, gy_last + a.hs + K - 1);
    const int rw = X1 - X0 + 1, rh = Y1 - Y0 + 1;
    for (int i = threadIdx.x; i < rh * rw; i += kMT) {
        const int yy = i / rw, xx = i - yy * rw;
        sm[yy * a.pitch + xx] = g[(size_t)(Y0 + yy) * W + X0 + xx];
    }
    // slack columns read by the last (partially valid) chunk of a row
    for (int i = threadIdx.x; i < rh * 8; i += kMT) sm[(i >> 3) * a.pitch + rw + (i & 7)] = 0.0f;
    __syncthreads();
    if (rx >= a.Rx || ry >= a.Ry) return;

    const int x0 = min(rx * a.step, W - K), y0 = min(ry * a.step, H - K);
    const float *refp = sm + (y0 - Y0) * a.pitch + (x0 - X0);
    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);  // +inf
        bi[j] = -1;
    }
    const float tau = a.tau[b], k2 = (float)(K * K);
    int kept = 0;
    const int xs = max(0, x0 - a.hs), xe = min(W - K, x0 + a.hs);
    const int ys = max(0, y0 - a.hs), ye = min(H - K, y0 + a.hs);
    for (int y = ys; y <= ye; ++y) {
        const float *rowbase = sm + (y - Y0) * a.pitch - X0;
        for (int xc = xs; xc <= xe; xc += 8) {
            // acc[c] = sum over patch rows i of (sum over j of (ref - cand)^2, left to right)
            float acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
#pragma unroll 2
            for (int i = 0; i < K; ++i) {
                const float *row = rowbase + i * a.pitch + xc;
                const float *rr = refp + i * a.pitch;
                float r[K], s[K + 7];
#pragma unroll
                for (int j = 0; j < K; ++j) r[j] = rr[j];
#pragma unroll
                for (int q = 0; q < K + 7; ++q) s[q] = row[q];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float e0 = __fsub_rn(r[0], s[c]);
                    float h = __fmul_rn(e0, e0);
#pragma unroll
                    for (int j = 1; j < K; ++j) {
                        const float e = __fsub_rn(r[j], s[c + j]);
                        h = __fmaf_rn(e, e, h);
                    }
                    acc[c] = __fadd_rn(acc[c], h);
                }
            }
            unsigned ins = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int x = xc + c;
                acc[c] = __fdiv_rn(acc[c], k2);
                if (x <= xe && !(x == x0 && y == y0) && acc[c] <= tau) {
                    ++kept;
                    if (acc[c] < bd[L - 1]) ins |= 1u << c;
                }
            }
            // insertions after the chunk's 8 distances, in index order
            while (ins) {
                const int c = __ffs(ins) - 1;
                ins &= ins - 1;
                float d = acc[0];
#pragma unroll
                for (int j = 1; j < 8; ++j) d = c == j ? acc[j] : d;
                insert_sorted<L>(bd, bi, d, y * W + xc + c);
            }
        }
    }
    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    int *out = a.idx + r * a.n2;
    out[0] = y0 * W + x0;
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (1 + j < a.n2) out[1 + j] = bi[j];
    a.n[r] = group_size(kept, a.n2);
}

// ---- matching on 2D-prethresholded patches ---------------------------------------

constexpr int kQX = 16, kQY = 16, kQT = kQX * kQY;  // 8 warps share the staged rows (measured: 8 rows of
                                                    // references, 4 warps per SM, were latency-bound)
constexpr int kQF = 2;  // pixels of the next row prefetched per thread

struct PreKArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, ncol_max;
    int spad;  // floats of padding after every `step` staged vectors (0 or 4)
    float tau[kChunk];
    float thr[kChunk];
    LargeTables t;
    int *idx;
    int *n;
    int n2;
};

template <int K>
struct PreShape {
    static constexpr int kCS = K * K + 4;  // staged floats per candidate vector (16-byte rows)
    static constexpr int kLoads = K * K / 4;  // 16-byte loads per vector
};

template <int K>
__device__ __forceinline__ float dct_at(const float *C, int v, const float *p)
{
    float s = __fmul_rn(C[v * K], p[0]);
#pragma unroll
    for (int j = 1; j < K; ++j) s = __fmaf_rn(C[v * K + j], p[j], s);
    return s;
}

__device__ __forceinline__ float keep_above_k(float c, float thr) { return fabsf(c) > thr ? c : 0.0f; }

template <int K, int L>
__global__ void __launch_bounds__(kQT) k_match_pre_k(const __grid_constant__ PreKArgs a)
{
    static_assert(K % 4 == 0, "vector loads of 4 coefficients, 4 partial sums");
    using S_ = PreShape<K>;
    constexpr int kCS = S_::kCS, NL = S_::kLoads;
    extern __shared__ __align__(16) float sm[];
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W, tid = threadIdx.x, nc = a.ncol_max;
    const float *C = a.t.C;
    float *ring = sm;                  // [K][nc][K]: row transforms of pixel rows y (slot y % K)
    float *S = ring + K * K * nc;      // thresholded vectors of the current candidate row (see soff)
    float *prow = S + kCS * nc + (nc / a.step + 1) * a.spad;  // [nc + K]: one pixel row of the CTA's window
    // Vector of candidate column x at S + soff(x): kCS floats each, plus spad after every `step`
    // of them.  The lanes of a quarter warp hold references `step` apart, so their candidates sit
    // step apart too; in 16-byte units their vectors start l (step kCS/4 + spad/4) + const apart,
    // an odd multiple when spad makes it one: the eight 16-byte loads hit distinct bank groups.
    auto soff = [&](int x) { return x * kCS + (x / a.step) * a.spad; };

    const int rx0 = blockIdx.x * kQX, ry0 = blockIdx.y * kQY;
    const int rx = rx0 + tid % kQX, ry = ry0 + tid / kQX;
    const bool active = rx < a.Rx && ry < a.Ry;
    const int gx_first = min(rx0 * a.step, W - K), gx_last = min(min(rx0 + kQX - 1, a.Rx - 1) * a.step, W - K);
    const int gy_first = min(ry0 * a.step, H - K), gy_last = min(min(ry0 + kQY - 1, a.Ry - 1) * a.step, H - K);
    const int X0 = max(0, gx_first - a.hs), X1 = min(W - K, gx_last + a.hs);
    const int Y0 = max(0, gy_first - a.hs), Y1 = min(H - K, gy_last + a.hs);
    const int ncol = X1 - X0 + 1, npx = ncol + K - 1;  // X0 + npx - 1 = X1 + K - 1 <= W - 1
    const float thr = a.thr[b], tau = a.tau[b];

    // the thread's reference vector (inactive threads take the last reference; they write nothing)
    const int x0 = min(min(rx, a.Rx - 1) * a.step, W - K), y0 = min(min(ry, a.Ry - 1) * a.step, H - K);
    // the same operations as the row and column transforms below: coefficient (u, v) =
    // C[u][0] t[0][v] then + C[u][i] t[i][v] for i = 1 .. K-1, t[i] = row i's transform;
    // accumulated row by row so that only one row transform is live
    f2 rr[K * K / 2];
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
        float p[K], t[K];
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = g[(size_t)(y0 + i) * W + x0 + j];
#pragma unroll
        for (int v = 0; v < K; ++v) t[v] = dct_at<K>(C, v, p);
#pragma unroll
        for (int u = 0; u < K; ++u)
#pragma unroll
            for (int v = 0; v < K; v += 2) {
                const f2 cu = f2_pack(C[u * K + i], C[u * K + i]), tv = f2_pack(t[v], t[v + 1]);
                f2 &acc = rr[(u * K + v) / 2];
                acc = i == 0 ? f2_mul(cu, tv) : f2_fma(cu, tv, acc);
            }
    }
#pragma unroll
    for (int q = 0; q < K * K / 2; ++q) rr[q] = f2_pack(keep_above_k(f2_lo(rr[q]), thr), keep_above_k(f2_hi(rr[q]), thr));

    auto load_row = [&](int y) {
        for (int i = tid; i < npx; i += kQT) prow[i] = g[(size_t)y * W + X0 + i];
    };
    float nxt[kQF];  // the next pixel row, in flight while a row is matched (npx <= kQT kQF: host check)
    auto fetch_row = [&](int y) {
#pragma unroll
        for (int j = 0; j < kQF; ++j) {
            const int i = tid + j * kQT;
            nxt[j] = (y < H && i < npx) ? g[(size_t)y * W + X0 + i] : 0.0f;
        }
    };
    auto store_row = [&]() {
#pragma unroll
        for (int j = 0; j < kQF; ++j)
            if (tid + j * kQT < npx) prow[tid + j * kQT] = nxt[j];
    };
    auto row_transform = [&](int y) {
        float *dst = ring + (y % K) * nc * K;
        for (int o = tid; o < ncol * K; o += kQT) dst[o] = dct_at<K>(C, o % K, prow + o / K);
    };
    for (int r = 0; r < K - 1; ++r) {
        __syncthreads();
        load_row(Y0 + r);
        __syncthreads();
        row_transform(Y0 + r);
    }

    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);  // +inf
        bi[j] = -1;
    }
    int kept = 0;
    const int xs = max(0, x0 - a.hs), xe = min(W - K, x0 + a.hs);
    const int ys = max(0, y0 - a.hs), ye = min(H - K, y0 + a.hs);

    fetch_row(Y0 + K - 1);
    for (int yy = Y0; yy <= Y1; ++yy) {
        __syncthreads();  // the previous row's readers of prow and S are done
        store_row();      // pixel row yy + K - 1
        __syncthreads();
        row_transform(yy + K - 1);
        __syncthreads();
        // column transforms: one (x, v) job gives the K coefficients (u, v) of candidate x
        for (int o = tid; o < ncol * K; o += kQT) {
            const int x = o / K, v = o % K;
            float t[K];
#pragma unroll
            for (int i = 0; i < K; ++i) t[i] = ring[((yy + i) % K) * nc * K + x * K + v];
#pragma unroll
            for (int u = 0; u < K; ++u) {
                float c = __fmul_rn(C[u * K], t[0]);
#pragma unroll
                for (int i = 1; i < K; ++i) c = __fmaf_rn(C[u * K + i], t[i], c);
                S[soff(x) + u * K + v] = keep_above_k(c, thr);
            }
        }
        __syncthreads();
        if (yy < Y1) fetch_row(yy + K);
        if (!active || yy < ys || yy > ye) continue;
        // insertions deferred over groups of 4 candidates, made in index order (65.2 -> 63.3 ms per
        // 16 x 1024^2 launch)
        for (int xg = xs; xg <= xe; xg += 4) {
          float dk[4];
          unsigned ins = 0;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int x = xg + kk;
            dk[kk] = 0.0f;
            if (x > xe || (x == x0 && yy == y0)) continue;
            const ulonglong2 *q4 = reinterpret_cast<const ulonglong2 *>(S + soff(x - X0));
            // partial sum j takes loads j NL/4 .. (j+1) NL/4 - 1 in order (load l holds pairs 2l, 2l+1)
            f2 acc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = f2_pack(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < NL / 4; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int l = j * (NL / 4) + k;
                    const ulonglong2 v = q4[l];
                    f2 qa, qb;
                    qa.v = v.x;
                    qb.v = v.y;
                    f2 e = f2_sub(rr[2 * l], qa);
                    acc[j] = f2_fma(e, e, acc[j]);
                    e = f2_sub(rr[2 * l + 1], qb);
                    acc[j] = f2_fma(e, e, acc[j]);
                }
            const float h01 = __fadd_rn(__fadd_rn(f2_lo(acc[0]), f2_hi(acc[0])), __fadd_rn(f2_lo(acc[1]), f2_hi(acc[1])));
            const float h23 = __fadd_rn(__fadd_rn(f2_lo(acc[2]), f2_hi(acc[2])), __fadd_rn(f2_lo(acc[3]), f2_hi(acc[3])));
            const float d = __fdiv_rn(__fadd_rn(h01, h23), (float)(K * K));
            dk[kk] = d;
            if (d <= tau) {
                ++kept;
                if (d < bd[L - 1]) ins |= 1u << kk;
            }
          }
          while (ins) {
            const int k = __ffs(ins) - 1;
            ins &= ins - 1;
            float d = dk[0];
#pragma unroll
            for (int j = 1; j < 4; ++j) d = k == j ? dk[j] : d;
            insert_sorted<L>(bd, bi, d, yy * W + xg + k);
          }
        }
    }

    if (!active) return;
    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    int *out = a.idx + r * a.n2;
    out[0] = y0 * W + x0;
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (1 + j < a.n2) out[1 + j] = bi[j];
    a.n[r] = group_size(kept, a.n2);
}

// ---- collaborative filtering -----------------------------------------------------

constexpr int kFW = 4;  // warps per CTA

struct FilterKArgs {
    const float *img;    // [b][C][H][W]: noisy (pass 2) or the image to filter (pass 1)
    const float *basic;  // pass 2 only
    const int *idx;
    const int *n;
    unsigned long long *num, *wsum;        // fixed-point sums per pixel / per patch position
    unsigned long long *num_hi, *wsum_hi;  // their high words (signed, units of 2^32)
    int C, H, W, R, Rx, Ry, n2, step, hs;
    int TR, RH, RW, RS;                    // reference tile side and window (rows, columns, num stride)
    float lambda;
    WinFmt wf;                             // format of the shared num window
    float sig[kChunk * 3];
    LargeTables t;
};

// Patch buffers: row i of patch t at t KS + i RSP; both strides odd, so the
// lanes of a warp, spread over (patch, row) jobs, over (patch, column) jobs
// or over coefficients, fall in distinct banks or nearly.
template <int K>
struct FShape {
    static constexpr int RSP = K | 1;
    static constexpr int KS = (K * RSP) | 1;
    static constexpr int NE = (K * K + 31) / 32;  // pixels of a patch per lane
};

// The K-point transform (INV: its transpose) of every row (COLS: column) of
// the n patches in T, the warp's lanes over the (patch, row) jobs.
template <int K, bool COLS, bool INV>
__device__ __forceinline__ void dct_pass(float *T, int n, int lane, const float *C)
{
    using F = FShape<K>;
    for (int j = lane; j < n * K; j += 32) {
        const int t = j / K, r = j - t * K;
        float *v = T + t * F::KS + (COLS ? r : r * F::RSP);
        constexpr int st = COLS ? F::RSP : 1;
        float x[K];
#pragma unroll
        for (int q = 0; q < K; ++q) x[q] = v[q * st];
#pragma unroll
        for (int o = 0; o < K; ++o) {
            // forward: sum_q C[o][q] x[q]; inverse: sum_q C[q][o] x[q]
            float s = (INV ? C[o] : C[o * K]) * x[0];
#pragma unroll
            for (int q = 1; q < K; ++q) s = fmaf(INV ? C[q * K + o] : C[o * K + q], x[q], s);
            v[o * st] = s;
        }
    }
}

template <int K>
__device__ __forceinline__ void dct2_fwd_warp(float *T, int n, int lane, const float *C)
{
    dct_pass<K, false, false>(T, n, lane, C);  // rows
    __syncwarp();
    dct_pass<K, true, false>(T, n, lane, C);   // columns
}

template <int K>
__device__ __forceinline__ void dct2_inv_warp(float *T, int n, int lane, const float *C)
{
    dct_pass<K, true, true>(T, n, lane, C);    // columns
    __syncwarp();
    dct_pass<K, false, true>(T, n, lane, C);   // rows
}

template <int N>
__device__ __forceinline__ void fwht_k(float (&v)[N])
{
#pragma unroll
    for (int h = 1; h < N; h <<= 1)
#pragma unroll
        for (int i = 0; i < N; i += 2 * h)
#pragma unroll
            for (int j = i; j < i + h; ++j) {
                const float x = v[j], y = v[j + h];
                v[j] = x + y;
                v[j + h] = x - y;
            }
}

// The group transform runs unnormalised (fwht twice multiplies by N): the
// threshold becomes lambda sigma sqrt(N), the Wiener gain B^2/(B^2 + N sigma^2),
// and the factor 1/N goes to the aggregation weight.

// Hard threshold of the lane's coefficient columns of an N-patch group in T;
// returns the number of kept coefficients.
template <int K, int N>
__device__ __forceinline__ int hard_cols_k(float *T, int lane, float thr_n)
{
    using F = FShape<K>;
    int cnt = 0;
    for (int c = lane; c < K * K; c += 32) {
        const int off = (c / K) * F::RSP + c % K;
        float v[N];
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = T[k * F::KS + off];
        fwht_k<N>(v);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const bool keep = fabsf(v[k]) > thr_n;
            cnt += keep ? 1 : 0;
            v[k] = keep ? v[k] : 0.0f;
        }
        fwht_k<N>(v);
#pragma unroll
        for (int k = 0; k < N; ++k) T[k * F::KS + off] = v[k];
    }
    return cnt;
}

// Wiener gains from the basic group's spectra (Tb) applied to the noisy
// group's (Ty, left holding the filtered spectra); returns the lane's part of
// the sum of squared gains.
template <int K, int N>
__device__ __forceinline__ float wiener_cols_k(const float *Tb, float *Ty, int lane, float s2n)
{
    using F = FShape<K>;
    float wsq = 0.0f;
    for (int c = lane; c < K * K; c += 32) {
        const int off = (c / K) * F::RSP + c % K;
        float vb[N], vy[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            vb[k] = Tb[k * F::KS + off];
            vy[k] = Ty[k * F::KS + off];
        }
        fwht_k<N>(vb);
        fwht_k<N>(vy);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float b2 = vb[k] * vb[k];
            const float om = __fdividef(b2, b2 + s2n);  // s2n >= sigma^2 > 0
            wsq = fmaf(om, om, wsq);
            vy[k] *= om;
        }
        fwht_k<N>(vy);
#pragma unroll
        for (int k = 0; k < N; ++k) Ty[k * F::KS + off] = vy[k];
    }
    return wsq;
}

template <int K>
__device__ __forceinline__ int cols_dispatch_hard(float *T, int n, int lane, float thr)
{
    switch (n) {
        case 1: return hard_cols_k<K, 1>(T, lane, thr);
        case 2: return hard_cols_k<K, 2>(T, lane, thr * 1.41421356237309505f);
        case 4: return hard_cols_k<K, 4>(T, lane, thr * 2.0f);
        case 8: return hard_cols_k<K, 8>(T, lane, thr * 2.82842712474619010f);
        case 16: return hard_cols_k<K, 16>(T, lane, thr * 4.0f);
        default: return hard_cols_k<K, 32>(T, lane, thr * 5.65685424949238019f);
    }
}

template <int K>
__device__ __forceinline__ float cols_dispatch_wiener(const float *Tb, float *Ty, int n, int lane, float s2)
{
    switch (n) {
        case 1: return wiener_cols_k<K, 1>(Tb, Ty, lane, s2);
        case 2: return wiener_cols_k<K, 2>(Tb, Ty, lane, 2.0f * s2);
        case 4: return wiener_cols_k<K, 4>(Tb, Ty, lane, 4.0f * s2);
        case 8: return wiener_cols_k<K, 8>(Tb, Ty, lane, 8.0f * s2);
        case 16: return wiener_cols_k<K, 16>(Tb, Ty, lane, 16.0f * s2);
        default: return wiener_cols_k<K, 32>(Tb, Ty, lane, 32.0f * s2);
    }
}

// A CTA owns a TR x TR tile of references; per channel it stages the image
// window covering every patch its groups can hold (tile + search radius +
// patch; for the second pass also the basic estimate's) and a num window of
// the same extent in shared memory, its warps filter the tile's groups one
// each at a time, and the num window is then added once to the global plane.
template <int K, bool WIENER>
__global__ void __launch_bounds__(kFW * 32) k_filter_k(const __grid_constant__ FilterKArgs a)
{
    using F = FShape<K>;
    constexpr int KS = F::KS, RSP = F::RSP, NE = F::NE;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    unsigned *win = reinterpret_cast<unsigned *>(fsm_raw);              // [2][RH][RS] (WinFmt)
    float *simg = reinterpret_cast<float *>(win + 2 * (size_t)a.RH * a.RS);  // [RH][RW]
    float *sbas = simg + (size_t)a.RH * a.RW;                                    // pass 2: [RH][RW]
    float *bufs = sbas + (WIENER ? (size_t)a.RH * a.RW : 0);                     // [kFW][1 or 2][n2][KS]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *T = bufs + (size_t)warp * (WIENER ? 2 : 1) * a.n2 * KS;  // the filtered group
    float *Tb = T + (size_t)a.n2 * KS;                               // pass 2: the basic estimate's group
    const int b = blockIdx.z, W = a.W, H = a.H;
    const int rx0 = blockIdx.x * a.TR, ry0 = blockIdx.y * a.TR;
    const int X0 = max(0, min(rx0 * a.step, W - K) - a.hs), Y0 = max(0, min(ry0 * a.step, H - K) - a.hs);
    const int tw = min(a.TR, a.Rx - rx0), th = min(a.TR, a.Ry - ry0), cnt = tw * th;
    const int rh = min(a.RH, H - Y0), rw = min(a.RW, W - X0);
    const size_t HW = (size_t)H * W;
    const float *C = a.t.C;
    // the lane's pixels of a patch (e = lane + 32 m < K^2): row, column and window weight
    int ei[NE], ej[NE];
    float kk[NE];
#pragma unroll
    for (int m = 0; m < NE; ++m) {
        const int e = lane + 32 * m;
        ei[m] = e < K * K ? e / K : 0;
        ej[m] = e < K * K ? e % K : 0;
        kk[m] = a.t.kai[ei[m]] * a.t.kai[ej[m]];
    }

    for (int c = 0; c < a.C; ++c) {
        const size_t cbase = ((size_t)b * a.C + c) * HW;
        const float sig = a.sig[b * 3 + c];
        for (int i = threadIdx.x; i < 2 * a.RH * a.RS; i += blockDim.x) win[i] = 0u;
        for (int i = threadIdx.x; i < rh * rw; i += blockDim.x) {
            const int ly = i / rw, lx = i - ly * rw;
            const size_t g = cbase + (size_t)(Y0 + ly) * W + X0 + lx;
            tc::cp_async4(tc::smem_u32(simg + ly * a.RW + lx), a.img + g);
            if (WIENER) tc::cp_async4(tc::smem_u32(sbas + ly * a.RW + lx), a.basic + g);
        }
        tc::cp_async_commit();
        tc::cp_async_wait<0>();
        __syncthreads();
        for (int q = warp; q < cnt; q += kFW) {
            const size_t r = (size_t)b * a.R + (size_t)(ry0 + q / tw) * a.Rx + rx0 + q % tw;
            const int n = a.n[r];
            if (n <= 0) continue;
            const int pos = lane < n ? a.idx[r * a.n2 + lane] : 0;
            const int py = pos / W, px = pos - (pos / W) * W;
            // gather patch t into T (and Tb), from the staged window (from the planes for a patch
            // outside it, only possible for match lists not produced by this library's matcher)
            for (int t = 0; t < n; ++t) {
                const int yt = __shfl_sync(0xffffffffu, py, t), xt = __shfl_sync(0xffffffffu, px, t);
                const int ly = yt - Y0, lx = xt - X0;
                const bool inside = ly >= 0 && ly + K <= rh && lx >= 0 && lx + K <= rw;
#pragma unroll
                for (int m = 0; m < NE; ++m) {
                    const int e = lane + 32 * m;
                    if (e < K * K) {
                        const int o = t * KS + ei[m] * RSP + ej[m];
                        if (inside) {
                            const int wo = (ly + ei[m]) * a.RW + lx + ej[m];
                            T[o] = simg[wo];
                            if (WIENER) Tb[o] = sbas[wo];
                        } else {
                            const size_t gi = cbase + (size_t)(yt + ei[m]) * W + xt + ej[m];
                            T[o] = a.img[gi];
                            if (WIENER) Tb[o] = a.basic[gi];
                        }
                    }
                }
            }
            __syncwarp();
            dct2_fwd_warp<K>(T, n, lane, C);
            if (WIENER) {
                __syncwarp();
                dct2_fwd_warp<K>(Tb, n, lane, C);
            }
            __syncwarp();
            float w;
            if (WIENER) {
                float wsq = cols_dispatch_wiener<K>(Tb, T, n, lane, sig * sig);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wsq += __shfl_xor_sync(0xffffffffu, wsq, o);
                w = wsq > 0.0f ? 1.0f / wsq : sig * sig;  // 1/(sigma^2 sum w^2) or 1, times sigma^2
            } else {
                const int nhar = __reduce_add_sync(0xffffffffu, cols_dispatch_hard<K>(T, n, lane, a.lambda * sig));
                w = nhar > 0 ? 1.0f / (float)nhar : sig * sig;  // 1/(sigma^2 N_har) or 1, times sigma^2
            }
            __syncwarp();
            dct2_inv_warp<K>(T, n, lane, C);
            __syncwarp();
            // aggregation: the group weight per patch position, w kai kai / n times the estimate per pixel
            if (lane < n) {
                const Fix fw = to_fixed(w);
                const size_t gq = cbase + (size_t)py * W + px;
                atomicAdd(a.wsum + gq, fw.lo);
                if (fw.hi != 0) atomicAdd(a.wsum_hi + gq, (unsigned long long)fw.hi);
            }
            const float wn = w / (float)n;  // exact: n is a power of two
            for (int t = 0; t < n; ++t) {
                const int yt = __shfl_sync(0xffffffffu, py, t), xt = __shfl_sync(0xffffffffu, px, t);
                const int ly = yt - Y0, lx = xt - X0;
                const bool inside = ly >= 0 && ly + K <= a.RH && lx >= 0 && lx + K <= a.RW;
#pragma unroll
                for (int m = 0; m < NE; ++m) {
                    const int e = lane + 32 * m;
                    if (e < K * K) {
                        const float c = wn * kk[m] * T[t * KS + ei[m] * RSP + ej[m]];
                        if (inside && fabsf(c) * a.wf.tscale < a.wf.tlim) {
                            win_add1(win + (ly + ei[m]) * a.RS + lx + ej[m], a.RH * a.RS, c * a.wf.tscale, a.wf.s);
                        } else {
                            const Fix f = to_fixed(c);
                            const size_t g = cbase + (size_t)(yt + ei[m]) * W + xt + ej[m];
                            atomicAdd(a.num + g, f.lo);
                            if (f.hi != 0) atomicAdd(a.num_hi + g, (unsigned long long)f.hi);
                        }
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < rh * rw; i += blockDim.x) {
            const int ly = i / rw, lx = i - ly * rw;
            const long long v = win_value(win[ly * a.RS + lx], win[a.RH * a.RS + ly * a.RS + lx], a.wf);
            if (v != 0) atomicAdd(a.num + cbase + (size_t)(Y0 + ly) * W + X0 + lx, (unsigned long long)v);
        }
        __syncthreads();  // the windows are refilled for the next channel
    }
}

// ---- host side -------------------------------------------------------------------

template <int K, int L>
dn_status launch_match_k(MatchKArgs &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match_k<K, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    dim3 grid((a.Rx + kMX - 1) / kMX, (a.Ry + kMY - 1) / kMY, B);
    return launch("bm3d_match_large_fp32", s, [&] { k_match_k<K, L><<<grid, kMT, smem, s>>>(a); });
}

template <int K>
dn_status match_k_n2(MatchKArgs &a, int B, cudaStream_t s, size_t smem)
{
    switch (a.n2) {
        case 1: return launch_match_k<K, 1>(a, B, s, smem);  // slot unused (n2 = 1)
        case 2: return launch_match_k<K, 1>(a, B, s, smem);
        case 4: return launch_match_k<K, 3>(a, B, s, smem);
        case 8: return launch_match_k<K, 7>(a, B, s, smem);
        case 16: return launch_match_k<K, 15>(a, B, s, smem);
        case 32: return launch_match_k<K, 31>(a, B, s, smem);
        default: return DN_EINVAL;
    }
}

template <int K, int L>
dn_status launch_pre_k(PreKArgs &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match_pre_k<K, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DN_ECUDA;
    dim3 grid((a.Rx + kQX - 1) / kQX, (a.Ry + kQY - 1) / kQY, B);
    return launch("bm3d_match_pre_large", s, [&] { k_match_pre_k<K, L><<<grid, kQT, smem, s>>>(a); });
}

template <int K>
dn_status pre_k_n2(PreKArgs &a, int B, cudaStream_t s, size_t smem)
{
    switch (a.n2) {
        case 1: return launch_pre_k<K, 1>(a, B, s, smem);
        case 2: return launch_pre_k<K, 1>(a, B, s, smem);
        case 4: return launch_pre_k<K, 3>(a, B, s, smem);
        case 8: return launch_pre_k<K, 7>(a, B, s, smem);
        case 16: return launch_pre_k<K, 15>(a, B, s, smem);
        default: return DN_EUNSUPPORTED;  // n2 = 32 would keep 62 list registers beside the 144 of the vector
    }
}

template <int K>
size_t filter_k_smem(bool wiener, int TR, int step, int hs, int n2, int *RH, int *RS)
{
    *RH = (TR - 1) * step + 2 * hs + K;
    *RS = *RH | 1;  // odd stride of 64-bit words
    return (size_t)*RH * *RS * sizeof(unsigned long long) + (size_t)(wiener ? 2 : 1) * *RH * *RH * sizeof(float) +
           (size_t)kFW * (wiener ? 2 : 1) * n2 * FShape<K>::KS * sizeof(float);
}

template <int K>
dn_status filter_k_impl(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B, int C,
                        int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    FilterKArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.Ry = grid_count(H, K, p.step);
    a.Rx = grid_count(W, K, p.step);
    a.R = a.Ry * a.Rx;
    a.n2 = p.n2;
    a.step = p.step;
    a.hs = p.search / 2;
    a.lambda = p.lambda3d;
    make_large_tables(K, p.beta, &a.t);
    // the largest tile of at most 4 x 4 references whose windows and buffers fit
    size_t smem = 0;
    int TR = 4;
    for (; TR >= 1; TR /= 2) {
        smem = filter_k_smem<K>(wiener, TR, p.step, a.hs, p.n2, &a.RH, &a.RS);
        if (smem <= 225 * 1024) break;
    }
    if (TR < 1) return DN_EUNSUPPORTED;
    a.TR = TR;
    a.RW = a.RH;
    a.wf = win_format((long long)TR * TR * p.n2);  // a pixel gets at most one term per patch of each group
    const void *fn = wiener ? (const void *)k_filter_k<K, true> : (const void *)k_filter_k<K, false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    const size_t HW = (size_t)H * W, N = (size_t)B * C * HW;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
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
        dn_status st = wiener ? launch("bm3d_filter_wiener_large_fp32", s,
                                       [&] { k_filter_k<K, true><<<grid, kFW * 32, smem, s>>>(a); })
                              : launch("bm3d_filter_hard_large_fp32", s,
                                       [&] { k_filter_k<K, false><<<grid, kFW * 32, smem, s>>>(a); });
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace

bool large_patch_supported(int K) { return K == 11 || K == 12; }

bool large_prethresh_supported(int K) { return K == 12; }

dn_status match_large(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p, const float *tau,
                      int *idx, int *n, cudaStream_t s)
{
    const int K = p.patch;
    if (!large_patch_supported(K)) return DN_EUNSUPPORTED;
    MatchKArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, K, p.step);
    a.Rx = grid_count(W, K, p.step);
    a.n2 = p.n2;
    a.plane = plane;
    const int width = (kMX - 1) * p.step + 2 * a.hs + K;
    const int height = (kMY - 1) * p.step + 2 * a.hs + K;
    int pitch = width + 8;
    pitch += ((16 - pitch % 32) + 32) % 32;  // pitch = 16 (mod 32)
    a.pitch = pitch;
    const size_t smem = (size_t)height * pitch * sizeof(float);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) a.tau[i] = tau[b0 + i];
        const size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        DN_TRY(K == 11 ? match_k_n2<11>(a, nb, s, smem) : match_k_n2<12>(a, nb, s, smem));
    }
    return DN_OK;
}

// Padding (floats) after every `step` staged vectors: makes step kCS/4 + spad/4 odd.
int pre_spad(int K, int step) { return ((step * ((K * K + 4) / 4)) % 2 == 0) ? 4 : 0; }

size_t match_pre_large_smem_bytes(int W, const dn_bm3d_pass &p)
{
    const int K = p.patch;
    int nc = (kQX - 1) * p.step + 2 * (p.search / 2) + 1;
    if (nc > W - K + 1) nc = W - K + 1;
    return (size_t)(K * K * nc + (K * K + 4) * nc + (nc / p.step + 1) * pre_spad(K, p.step) + nc + K) *
           sizeof(float);
}

dn_status match_prethresh_large(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                                const float *tau, const float *thr, int *idx, int *n, cudaStream_t s)
{
    const int K = p.patch;
    if (!large_prethresh_supported(K)) return DN_EUNSUPPORTED;
    PreKArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, K, p.step);
    a.Rx = grid_count(W, K, p.step);
    a.ncol_max = (kQX - 1) * p.step + 2 * a.hs + 1;
    if (a.ncol_max > W - K + 1) a.ncol_max = W - K + 1;
    a.n2 = p.n2;
    a.plane = plane;
    a.spad = pre_spad(K, p.step);
    make_large_tables(K, p.beta, &a.t);
    const size_t smem = match_pre_large_smem_bytes(W, p);
    // (about 1.2 KB per staged column: the 200 KB bound keeps a row's K - 1 + columns far below
    // the kQT kQF pixels the prefetch registers hold)
    if (smem > 200 * 1024 || a.ncol_max + K - 1 > kQT * kQF) return DN_EUNSUPPORTED;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) {
            a.tau[i] = tau[b0 + i];
            a.thr[i] = thr[b0 + i];
        }
        const size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        DN_TRY(pre_k_n2<12>(a, nb, s, smem));
    }
    return DN_OK;
}

dn_status filter_large(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B, int C,
                       int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    switch (p.patch) {
        case 11: return filter_k_impl<11>(wiener, img, basic, idx, n, B, C, H, W, sig, p, acc, s);
        case 12: return filter_k_impl<12>(wiener, img, basic, idx, n, B, C, H, W, sig, p, acc, s);
        default: return DN_EUNSUPPORTED;
    }
}

}  // namespace dn

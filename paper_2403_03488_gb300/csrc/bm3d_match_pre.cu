// Block matching on 2D-prethresholded patches: BM3D's first-pass distance at
// high noise.  Every patch P is replaced by Y(P), its orthonormal 2D DCT-II
// with every coefficient of magnitude <= thr set to zero, and
//     d(P, Q) = ||Y(P) - Y(Q)||^2 / 64;
// window, ordering (the reference first, then ascending (d, y*W + x) among
// d <= tau) and group size are those of the pixel-domain matcher.  With
// thr = 0 the distance equals the pixel-domain one up to rounding (the
// transform is orthonormal).
//
// k_match_pre: a CTA owns kPX x kPY grid references and walks the union of
// their search windows one candidate row at a time.  The 2D transform is
// separable: the 8-point transforms of every 8-pixel row segment,
//     t[r][x][v] = sum_j C[v][j] p[r][x + j],
// are kept in shared memory for the last 8 pixel rows (a ring), so moving
// down one candidate row transforms one new pixel row; the column transforms
//     c[u][v] = sum_i C[u][i] t[y + i][x][v]
// then give the thresholded coefficient vectors of the row's candidates,
// staged with a 68-float stride (the 16-byte loads of a quarter warp, whose
// lanes hold references `step` apart, fall in distinct banks for step 3);
// the next pixel row is loaded into registers while the current row is
// matched.  Each thread forms its own reference's vector with the same
// operations in the same order, so equal patches give equal vectors, and
// accumulates (r - q)^2 with packed FP32x2 operations in four interleaved
// partial sums.  No coefficient buffer: the transforms cost about an eighth of
// the distance arithmetic.  The kernel is bound by shared-memory bandwidth
// (each pair reads the candidate's 256-byte vector; lanes read different
// candidates).
#include <cmath>

#include "common.cuh"
#include "f32x2.cuh"
#include "match_exact.cuh"

namespace dn {

namespace {

constexpr int kPX = 32;            // references per CTA along x
constexpr int kPY = 4;             // references per CTA along y
constexpr int kPT = kPX * kPY;
constexpr int kCS = 68;            // staged floats per candidate vector (64 + 4 pad, 16-byte rows)
constexpr int kPF = 2;             // pixels of the next row prefetched per thread (kPT * kPF >= nc + 7)

struct PreArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, ncol_max;
    float tau[kChunk];
    float thr[kChunk];
    float C[64];  // C[v][j] = a_v cos(pi (2 j + 1) v / 16), orthonormal DCT-II
    int *idx;
    int *n;
    int n2;
};

// 8-point transform of 8 consecutive values: sum_j C[v][j] p[j], fixed order.
__device__ __forceinline__ float dct8_at(const float *C, int v, const float *p)
{
    float s = __fmul_rn(C[v * 8], p[0]);
#pragma unroll
    for (int j = 1; j < 8; ++j) s = __fmaf_rn(C[v * 8 + j], p[j], s);
    return s;
}

__device__ __forceinline__ float keep_above(float c, float thr) { return fabsf(c) > thr ? c : 0.0f; }

template <int L>
__global__ void __launch_bounds__(kPT) k_match_pre(PreArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W, tid = threadIdx.x, nc = a.ncol_max;
    float *ring = sm;             // [8][nc][8]: row transforms of pixel rows y (slot y & 7)
    float *S = ring + 64 * nc;    // [nc][kCS]: thresholded vectors of the current candidate row
    float *prow = S + kCS * nc;   // [nc + 8]: one pixel row of the CTA's window

    const int rx0 = blockIdx.x * kPX, ry0 = blockIdx.y * kPY;
    const int rx = rx0 + tid % kPX, ry = ry0 + tid / kPX;
    const bool active = rx < a.Rx && ry < a.Ry;
    const int gx_first = min(rx0 * a.step, W - 8), gx_last = min(min(rx0 + kPX - 1, a.Rx - 1) * a.step, W - 8);
    const int gy_first = min(ry0 * a.step, H - 8), gy_last = min(min(ry0 + kPY - 1, a.Ry - 1) * a.step, H - 8);
    const int X0 = max(0, gx_first - a.hs), X1 = min(W - 8, gx_last + a.hs);
    const int Y0 = max(0, gy_first - a.hs), Y1 = min(H - 8, gy_last + a.hs);
    const int ncol = X1 - X0 + 1, npx = ncol + 7;  // npx <= nc + 7, X0 + npx - 1 = X1 + 7 <= W - 1
    const float thr = a.thr[b], tau = a.tau[b];

    // the thread's reference vector (inactive threads take the last reference; they write nothing)
    const int x0 = min(min(rx, a.Rx - 1) * a.step, W - 8), y0 = min(min(ry, a.Ry - 1) * a.step, H - 8);
    f2 rr[32];
    {
        float t[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float p[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) p[j] = g[(size_t)(y0 + i) * W + x0 + j];
#pragma unroll
            for (int v = 0; v < 8; ++v) t[i][v] = dct8_at(a.C, v, p);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 8; v += 2) {
                float c0 = __fmul_rn(a.C[u * 8], t[0][v]), c1 = __fmul_rn(a.C[u * 8], t[0][v + 1]);
#pragma unroll
                for (int i = 1; i < 8; ++i) {
                    c0 = __fmaf_rn(a.C[u * 8 + i], t[i][v], c0);
                    c1 = __fmaf_rn(a.C[u * 8 + i], t[i][v + 1], c1);
                }
                rr[(u * 8 + v) / 2] = f2_pack(keep_above(c0, thr), keep_above(c1, thr));
            }
    }

    auto load_row = [&](int y) {
        for (int i = tid; i < npx; i += kPT) prow[i] = g[(size_t)y * W + X0 + i];
    };
    float nxt[kPF];  // the next pixel row, in flight while a row is matched
    auto fetch_row = [&](int y) {
#pragma unroll
        for (int j = 0; j < kPF; ++j) {
            const int i = tid + j * kPT;
            nxt[j] = (y < H && i < npx) ? g[(size_t)y * W + X0 + i] : 0.0f;
        }
    };
    auto store_row = [&]() {
#pragma unroll
        for (int j = 0; j < kPF; ++j)
            if (tid + j * kPT < npx) prow[tid + j * kPT] = nxt[j];
    };
    auto row_transform = [&](int y) {
        float *dst = ring + (y & 7) * nc * 8;
        for (int o = tid; o < ncol * 8; o += kPT) dst[o] = dct8_at(a.C, o & 7, prow + (o >> 3));
    };
    for (int r = 0; r < 7; ++r) {
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
    const int xs = max(0, x0 - a.hs), xe = min(W - 8, x0 + a.hs);
    const int ys = max(0, y0 - a.hs), ye = min(H - 8, y0 + a.hs);

    const bool prefetch = npx <= kPT * kPF;  // else (wide windows) rows are loaded directly
    if (prefetch) fetch_row(Y0 + 7);
    for (int yy = Y0; yy <= Y1; ++yy) {
        __syncthreads();  // the previous row's readers of prow and S are done
        if (prefetch) store_row();  // pixel row yy + 7
        else load_row(yy + 7);
        __syncthreads();
        row_transform(yy + 7);
        __syncthreads();
        // column transforms: one (x, v) job gives the 8 coefficients (u, v) of candidate x
        for (int o = tid; o < ncol * 8; o += kPT) {
            const int x = o >> 3, v = o & 7;
            float t[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] = ring[((yy + i) & 7) * nc * 8 + x * 8 + v];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float c = __fmul_rn(a.C[u * 8], t[0]);
#pragma unroll
                for (int i = 1; i < 8; ++i) c = __fmaf_rn(a.C[u * 8 + i], t[i], c);
                S[x * kCS + u * 8 + v] = keep_above(c, thr);
            }
        }
        __syncthreads();
        if (prefetch && yy < Y1) fetch_row(yy + 8);
        if (!active || yy < ys || yy > ye) continue;
        // insertions deferred over groups of 8 candidates and then made in index order, one loop
        // trip per inserting candidate (26.60 -> 25.95 ms per 16 x 1024^2 launch)
        for (int xg = xs; xg <= xe; xg += 8) {
          float dk[8];
          unsigned ins = 0;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const int x = xg + kk;
            dk[kk] = 0.0f;
            if (x > xe || (x == x0 && yy == y0)) continue;
            // 16-byte loads straight into two packed pairs (no repacking of float4 lanes)
            const ulonglong2 *q4 = reinterpret_cast<const ulonglong2 *>(S + (x - X0) * kCS);
            f2 acc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = f2_pack(0.0f, 0.0f);
            // partial sum j takes coefficient pairs 8 j .. 8 j + 7 in order (load 4 j + k holds pairs
            // 8 j + 2 k and 8 j + 2 k + 1)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const ulonglong2 v = q4[4 * j + k];
                    f2 qa, qb;
                    qa.v = v.x;
                    qb.v = v.y;
                    f2 e = f2_sub(rr[8 * j + 2 * k], qa);
                    acc[j] = f2_fma(e, e, acc[j]);
                    e = f2_sub(rr[8 * j + 2 * k + 1], qb);
                    acc[j] = f2_fma(e, e, acc[j]);
                }
            const f2 s0 = acc[0], s1 = acc[1], s2 = acc[2], s3 = acc[3];
            const float h01 = __fadd_rn(__fadd_rn(f2_lo(s0), f2_hi(s0)), __fadd_rn(f2_lo(s1), f2_hi(s1)));
            const float h23 = __fadd_rn(__fadd_rn(f2_lo(s2), f2_hi(s2)), __fadd_rn(f2_lo(s3), f2_hi(s3)));
            const float d = __fmul_rn(__fadd_rn(h01, h23), 0.015625f);  // / 64, exact
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
            for (int j = 1; j < 8; ++j) d = k == j ? dk[j] : d;
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

template <int L>
dn_status launch_pre(PreArgs &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match_pre<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    dim3 grid((a.Rx + kPX - 1) / kPX, (a.Ry + kPY - 1) / kPY, B);
    return launch("bm3d_match_pre", s, [&] { k_match_pre<L><<<grid, kPT, smem, s>>>(a); });
}

}  // namespace

size_t match_pre_smem_bytes(int W, const dn_bm3d_pass &p)
{
    int nc = (kPX - 1) * p.step + 2 * (p.search / 2) + 1;
    if (nc > W - 7) nc = W - 7;
    return (size_t)(64 * nc + kCS * nc + nc + 8) * sizeof(float);
}

dn_status match_prethresh(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                          const float *tau, const float *thr, int *idx, int *n, cudaStream_t s)
{
    PreArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.ncol_max = (kPX - 1) * p.step + 2 * a.hs + 1;
    if (a.ncol_max > W - 7) a.ncol_max = W - 7;
    a.n2 = p.n2;
    a.plane = plane;
    const double pi = 3.14159265358979323846;
    for (int v = 0; v < 8; ++v)
        for (int j = 0; j < 8; ++j)
            a.C[v * 8 + j] = (float)((v == 0 ? std::sqrt(0.125) : 0.5) * std::cos(pi * (2 * j + 1) * v / 16.0));
    const size_t smem = match_pre_smem_bytes(W, p);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
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
        dn_status st;
        switch (p.n2) {
            case 1: st = launch_pre<1>(a, nb, s, smem); break;  // slot unused (n2 = 1)
            case 2: st = launch_pre<1>(a, nb, s, smem); break;
            case 4: st = launch_pre<3>(a, nb, s, smem); break;
            case 8: st = launch_pre<7>(a, nb, s, smem); break;
            case 16: st = launch_pre<15>(a, nb, s, smem); break;
            case 32: st = launch_pre<31>(a, nb, s, smem); break;
            default: return DN_EINVAL;
        }
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace dn

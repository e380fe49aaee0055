// Exhaustive FP32 block matching (the BM3D grouping step).
//
// For every reference patch P on the grid (0, step, ... plus L-8 on each axis)
// and every candidate Q whose top-left corner lies in the search window
// centred on P's corner (clipped to the image):
//     d(P, Q) = ||P - Q||^2 / 64.
// The reference is group member 0; the other candidates with d <= tau follow
// in ascending (d, y*W + x) order; the group size is
// n = min(n2, largest power of two <= #kept).
//
// Design: one CTA owns a 16 x 8 tile of reference positions and stages the
// union of their search windows in shared memory (one coalesced load).  One
// thread per reference keeps its patch in 64 registers and scans candidate
// rows in chunks of 8 horizontally adjacent candidates: each of the 8 patch
// rows loads 15 consecutive pixels once and feeds 8 accumulators, so shared
// loads are 15 per 64 subtract-FMA pairs.  The per-candidate sum runs in the
// same (row, column) order for every candidate, so equal pixel sets give
// bit-equal distances and ties resolve by index exactly as in the definition.
// The sorted top list lives in registers and is updated by a branch-free
// insertion network (static register indices).  The smem row pitch is
// 16 mod 32 floats: lanes hold references 3 pixels apart in two rows, which
// then hit 32 distinct banks.
#include "common.cuh"

namespace dn {

namespace {

constexpr int kTX = 16;     // references per CTA along x
constexpr int kTY = 8;      // references per CTA along y
constexpr int kThreads = kTX * kTY;

struct MatchArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, pitch;
    float tau[kChunk];
    int *idx;
    int *n;
    int n2;
};

template <int L>
__device__ __forceinline__ void insert_sorted(float (&bd)[L], int (&bi)[L], float d, int id)
{
    // Keep bd ascending; equal distances keep scan (= index) order.
#pragma unroll
    for (int j = L - 1; j > 0; --j) {
        bool before_prev = d < bd[j - 1];
        bool before_this = d < bd[j];
        float nd = before_prev ? bd[j - 1] : (before_this ? d : bd[j]);
        int ni = before_prev ? bi[j - 1] : (before_this ? id : bi[j]);
        bd[j] = nd;
        bi[j] = ni;
    }
    if (d < bd[0]) {
        bd[0] = d;
        bi[0] = id;
    }
}

// L = n2 - 1 list slots after the reference.
template <int L>
__global__ void __launch_bounds__(kThreads) k_match_fp32(MatchArgs a)
{
    extern __shared__ float sm[];
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W;
    const int rx0 = blockIdx.x * kTX, ry0 = blockIdx.y * kTY;
    const int rx = rx0 + threadIdx.x % kTX, ry = ry0 + threadIdx.x / kTX;

    const int gx_first = min(rx0 * a.step, W - 8);
    const int gx_last = min(min(rx0 + kTX - 1, a.Rx - 1) * a.step, W - 8);
    const int gy_first = min(ry0 * a.step, H - 8);
    const int gy_last = min(min(ry0 + kTY - 1, a.Ry - 1) * a.step, H - 8);
    const int X0 = max(0, gx_first - a.hs), X1 = min(W - 1, gx_last + a.hs + 7);
    const int Y0 = max(0, gy_first - a.hs), Y1 = min(H - 1, gy_last + a.hs + 7);
    const int rw = X1 - X0 + 1, rh = Y1 - Y0 + 1;

    for (int i = threadIdx.x; i < rh * rw; i += kThreads) {
        int yy = i / rw, xx = i - yy * rw;
        sm[yy * a.pitch + xx] = g[(size_t)(Y0 + yy) * W + X0 + xx];
    }
    // slack columns read by the last (partially valid) chunk of a row
    for (int i = threadIdx.x; i < rh * 8; i += kThreads) sm[(i >> 3) * a.pitch + rw + (i & 7)] = 0.0f;
    __syncthreads();
    if (rx >= a.Rx || ry >= a.Ry) return;

    const int x0 = min(rx * a.step, W - 8), y0 = min(ry * a.step, H - 8);
    float ref[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) ref[i * 8 + j] = sm[(y0 - Y0 + i) * a.pitch + (x0 - X0 + j)];

    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);  // +inf
        bi[j] = -1;
    }
    const float tau = a.tau[b];
    int kept = 0;
    const int xs = max(0, x0 - a.hs), xe = min(W - 8, x0 + a.hs);
    const int ys = max(0, y0 - a.hs), ye = min(H - 8, y0 + a.hs);

    for (int y = ys; y <= ye; ++y) {
        const float *rowbase = sm + (y - Y0) * a.pitch - X0;
        for (int xc = xs; xc <= xe; xc += 8) {
            float acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float *row = rowbase + i * a.pitch + xc;
                float s[15];
#pragma unroll
                for (int k = 0; k < 15; ++k) s[k] = row[k];
#pragma unroll
                for (int c = 0; c < 8; ++c)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float e = ref[i * 8 + j] - s[c + j];
                        acc[c] = fmaf(e, e, acc[c]);
                    }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int x = xc + c;
                const float d = acc[c] * 0.015625f;  // / 64, exact
                const bool valid = (x <= xe) && !(x == x0 && y == y0) && (d <= tau);
                if (valid) {
                    ++kept;
                    if (d < bd[L - 1]) insert_sorted<L>(bd, bi, d, y * W + x);
                }
            }
        }
    }

    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    int *out = a.idx + r * a.n2;
    out[0] = y0 * W + x0;
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (1 + j < a.n2) out[1 + j] = bi[j];
    int total = min(kept + 1, a.n2);
    int n = 1;
    while (n * 2 <= total) n *= 2;
    a.n[r] = n;
}

template <int L>
dn_status launch_match(MatchArgs &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match_fp32<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DN_ECUDA;
    dim3 grid((a.Rx + kTX - 1) / kTX, (a.Ry + kTY - 1) / kTY, B);
    return launch("bm3d_match_fp32", s, [&] { k_match_fp32<L><<<grid, kThreads, smem, s>>>(a); });
}

}  // namespace

dn_status match_fp32(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                     const float *tau, int *idx, int *n, cudaStream_t s)
{
    MatchArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.n2 = p.n2;
    a.plane = plane;
    int width = (kTX - 1) * p.step + 2 * a.hs + 8;
    int height = (kTY - 1) * p.step + 2 * a.hs + 8;
    int pitch = width + 8;
    pitch += ((16 - pitch % 32) + 32) % 32;  // pitch = 16 (mod 32)
    a.pitch = pitch;
    size_t smem = (size_t)height * pitch * sizeof(float);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) a.tau[i] = tau[b0 + i];
        size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        dn_status st;
        switch (p.n2) {
            case 1: st = launch_match<1>(a, nb, s, smem); break;  // slot unused (n2 = 1)
            case 2: st = launch_match<1>(a, nb, s, smem); break;
            case 4: st = launch_match<3>(a, nb, s, smem); break;
            case 8: st = launch_match<7>(a, nb, s, smem); break;
            case 16: st = launch_match<15>(a, nb, s, smem); break;
            case 32: st = launch_match<31>(a, nb, s, smem); break;
            default: return DN_EINVAL;
        }
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace dn

// Pixel-wise NL-means (the NLM prefilter of Sec. IV-A), FP32.
//
// For every pixel p and every offset delta of the search window with
// q = p + delta inside the image:
//     d2(p, q) = mean over the patch x patch neighbourhood of (g(p+t) - g(q+t))^2
//                (guide channel g, half-sample symmetric reflection),
//     w        = exp(-max(d2 - 2 sigma^2, 0) / h^2),
// out_c(p) = sum_q w y_c(q) / sum_q w for every channel c.
//
// Design: offset-major box filtering.  A CTA owns a 32 x 16 output tile and
// stages the reflected guide (tile + patch and search halos) and the other
// channels in shared memory once.  For each pair of horizontally adjacent
// offsets (dx, dx + 1) it forms the two squared-difference images over tile +
// patch halo in the two lanes of packed FP32x2 values, sums them vertically
// then horizontally (2 * patch adds per pixel instead of patch^2; each sum in
// the same sequential order as a scalar loop), and each thread folds its
// pixel's two weights into register accumulators.  Threads map to rows and
// columns of the difference image directly (no index division).
#include "common.cuh"
#include "f32x2.cuh"

namespace dn {

namespace {

constexpr int kTX = 32, kTY = 16, kThreads = kTX * kTY;

struct NlmArgs {
    const float *in;
    float *out;
    int C, H, W, r, hs;
    float inv_np;
    float two_s2[kChunk];
    float inv_h2[kChunk];
};

__device__ __forceinline__ int reflect_hs(int i, int L, int r)
{
    // clamp to [-r, L-1+r], then half-sample symmetric reflection
    i = max(-r, min(L - 1 + r, i));
    if (i < 0) i = -i - 1;
    if (i >= L) i = 2 * L - i - 1;
    return max(0, min(L - 1, i));
}

// RT > 0: patch radius fixed at compile time (unrolled box sums, constant
// strides); RT = 0: the radius from the arguments.
template <int RT>
__global__ void __launch_bounds__(kThreads) k_nlm(NlmArgs a)
{
    extern __shared__ float sm[];
    const int r = RT > 0 ? RT : a.r, hs = a.hs, P = 2 * r + 1;
    const int GW = kTX + 2 * r + 2 * hs, GH = kTY + 2 * r + 2 * hs;  // guide region
    const int DW = kTX + 2 * r, DH = kTY + 2 * r;                    // difference image
    const int VW = kTX + 2 * hs, VH = kTY + 2 * hs;                  // value regions (other channels)
    float *S = sm;                                                   // [GH][GW]
    f2 *D = reinterpret_cast<f2 *>(S + ((GH * GW + 1) & ~1));        // [DH][DW] offset pairs
    f2 *V = D + DH * DW;                                             // [kTY][DW]
    float *Y = reinterpret_cast<float *>(V + kTY * DW);              // [C-1][VH][VW]

    const int b = blockIdx.z;
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const float *g = a.in + (size_t)b * a.C * HW;

    for (int i = threadIdx.x; i < GH * GW; i += kThreads) {
        int yy = i / GW, xx = i - yy * GW;
        int sy = reflect_hs(Y0 - r - hs + yy, H, r), sx = reflect_hs(X0 - r - hs + xx, W, r);
        S[i] = g[(size_t)sy * W + sx];
    }
    for (int c = 1; c < a.C; ++c)
        for (int i = threadIdx.x; i < VH * VW; i += kThreads) {
            int yy = i / VW, xx = i - yy * VW;
            int sy = max(0, min(H - 1, Y0 - hs + yy)), sx = max(0, min(W - 1, X0 - hs + xx));
            Y[(c - 1) * VH * VW + i] = g[c * HW + (size_t)sy * W + sx];
        }
    __syncthreads();

    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int px = X0 + tx, py = Y0 + ty;
    const float two_s2 = a.two_s2[b], inv_h2 = a.inv_h2[b];
    const f2 inv_np = f2_pack(a.inv_np, a.inv_np);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    float wsum = 0.0f;

    // this thread's elements of the difference image (at most 2 x 2): the
    // reference pixel does not depend on the offset
    constexpr int kMaxR = RT > 0 ? RT : 7;
    constexpr int kEY = (kTY + 2 * kMaxR + kTY - 1) / kTY, kEX = (kTX + 2 * kMaxR + kTX - 1) / kTX;
    float s0[kEY][kEX];
#pragma unroll
    for (int ey = 0; ey < kEY; ++ey)
#pragma unroll
        for (int ex = 0; ex < kEX; ++ex) {
            const int yy = ty + ey * kTY, xx = tx + ex * kTX;
            s0[ey][ex] = (yy < DH && xx < DW) ? S[(yy + hs) * GW + xx + hs] : 0.0f;
        }

    for (int dy = -hs; dy <= hs; ++dy)
        for (int dx = -hs; dx <= hs; dx += 2) {
            // squared differences for offsets dx (low lane) and dx + 1 (high lane)
#pragma unroll
            for (int ey = 0; ey < kEY; ++ey)
#pragma unroll
                for (int ex = 0; ex < kEX; ++ex) {
                    const int yy = ty + ey * kTY, xx = tx + ex * kTX;
                    if (yy < DH && xx < DW) {
                        const float *q = S + (yy + hs + dy) * GW + xx + hs + dx;
                        D[yy * DW + xx] = f2_sqd(f2_pack(s0[ey][ex], s0[ey][ex]), f2_pack(q[0], q[1]));
                    }
                }
            __syncthreads();
#pragma unroll
            for (int ex = 0; ex < kEX; ++ex) {
                const int xx = tx + ex * kTX;
                if (xx < DW) {
                    const f2 *d = D + ty * DW + xx;
                    f2 v = d[0];
#pragma unroll
                    for (int t = 1; t < (RT > 0 ? 2 * RT + 1 : 1); ++t) v = f2_add(v, d[t * DW]);
                    if (RT == 0)
                        for (int t = 1; t < P; ++t) v = f2_add(v, d[t * DW]);
                    V[ty * DW + xx] = v;
                }
            }
            __syncthreads();
            const f2 *vr = V + ty * DW + tx;
            f2 d2 = vr[0];
#pragma unroll
            for (int t = 1; t < (RT > 0 ? 2 * RT + 1 : 1); ++t) d2 = f2_add(d2, vr[t]);
            if (RT == 0)
                for (int t = 1; t < P; ++t) d2 = f2_add(d2, vr[t]);
            d2 = f2_mul(d2, inv_np);
            const int qy = py + dy;
            if (qy >= 0 && qy < H) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ox = dx + e, qx = px + ox;
                    if (ox <= hs && qx >= 0 && qx < W) {
                        const float ee = fmaxf((e ? f2_hi(d2) : f2_lo(d2)) - two_s2, 0.0f);
                        const float w = __expf(-ee * inv_h2);
                        acc[0] = fmaf(w, S[(ty + r + hs + dy) * GW + tx + r + hs + ox], acc[0]);
#pragma unroll
                        for (int c = 1; c < 3; ++c)
                            if (c < a.C)
                                acc[c] = fmaf(w, Y[(c - 1) * VH * VW + (ty + hs + dy) * VW + tx + hs + ox], acc[c]);
                        wsum += w;
                    }
                }
            }
        }
    if (px < W && py < H) {
        float *o = a.out + (size_t)b * a.C * HW + (size_t)py * W + px;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c < a.C) o[c * HW] = acc[c] / wsum;
    }
}

}  // namespace

dn_status nlm_launch(const float *in, float *out, int B, int C, int H, int W, const float *sig_guide,
                     const dn_nlm_params &p, cudaStream_t s)
{
    NlmArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.r = p.patch / 2;
    a.hs = p.search / 2;
    a.inv_np = 1.0f / (float)(p.patch * p.patch);
    const int GW = kTX + 2 * a.r + 2 * a.hs, GH = kTY + 2 * a.r + 2 * a.hs;
    const int DW = kTX + 2 * a.r, DH = kTY + 2 * a.r;
    const int VW = kTX + 2 * a.hs, VH = kTY + 2 * a.hs;
    size_t smem = sizeof(float) * ((size_t)((GH * GW + 1) & ~1) + 2 * (size_t)DH * DW + 2 * (size_t)kTY * DW +
                                   (size_t)(C - 1) * VH * VW);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    void (*kern)(NlmArgs) = a.r == 1 ? k_nlm<1> : a.r == 2 ? k_nlm<2> : a.r == 3 ? k_nlm<3> : a.r == 4 ? k_nlm<4>
                          : a.r == 5 ? k_nlm<5> : k_nlm<0>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.in = in + (size_t)b0 * C * H * W;
        a.out = out + (size_t)b0 * C * H * W;
        for (int i = 0; i < nb; ++i) {
            float sg = sig_guide[b0 + i], h = p.h_over_sigma * sg;
            a.two_s2[i] = 2.0f * sg * sg;
            a.inv_h2[i] = 1.0f / (h * h);
        }
        dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, nb);
        DN_TRY(launch("nlm_fp32", s, [&] { kern<<<grid, kThreads, smem, s>>>(a); }));
    }
    return DN_OK;
}

}  // namespace dn

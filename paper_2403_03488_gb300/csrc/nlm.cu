// Pixel-wise NL-means (the NLM prefilter of Sec. IV-A), FP32.
//
// For every pixel p and every offset delta of the search window with
// q = p + delta inside the image:
//     d2(p, q) = mean over the patch x patch neighbourhood of (g(p+t) - g(q+t))^2
//                (guide channel g, half-sample symmetric reflection),
//     w        = exp(-max(d2 - 2 sigma^2, 0) / h^2),
// out_c(p) = sum_q w y_c(q) / sum_q w for every channel c.
//
// Design: offset-major box filtering.  A CTA owns a 32 x 8 output tile and
// stages the reflected guide (tile + patch and search halos) and the other
// channels in shared memory once.  For each offset it forms the squared
// difference image over tile + patch halo, sums it vertically then
// horizontally (2 * patch adds per pixel instead of patch^2), and each thread
// folds its pixel's weight into register accumulators.
#include "common.cuh"

namespace dn {

namespace {

constexpr int kTX = 32, kTY = 8, kThreads = kTX * kTY;

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

__global__ void __launch_bounds__(kThreads) k_nlm(NlmArgs a)
{
    extern __shared__ float sm[];
    const int r = a.r, hs = a.hs, P = 2 * r + 1;
    const int GW = kTX + 2 * r + 2 * hs, GH = kTY + 2 * r + 2 * hs;  // guide region
    const int DW = kTX + 2 * r, DH = kTY + 2 * r;                    // difference image
    const int VW = kTX + 2 * hs, VH = kTY + 2 * hs;                  // value regions (other channels)
    float *S = sm;                    // [GH][GW]
    float *D = S + GH * GW;           // [DH][DW]
    float *V = D + DH * DW;           // [kTY][DW]
    float *Y = V + kTY * DW;          // [C-1][VH][VW]

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
    float acc[3] = {0.0f, 0.0f, 0.0f};
    float wsum = 0.0f;

    for (int dy = -hs; dy <= hs; ++dy)
        for (int dx = -hs; dx <= hs; ++dx) {
            for (int i = threadIdx.x; i < DH * DW; i += kThreads) {
                int yy = i / DW, xx = i - yy * DW;
                float e = S[(yy + hs) * GW + xx + hs] - S[(yy + hs + dy) * GW + xx + hs + dx];
                D[i] = e * e;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < kTY * DW; i += kThreads) {
                int yy = i / DW, xx = i - yy * DW;
                float s = 0.0f;
                for (int t = 0; t < P; ++t) s += D[(yy + t) * DW + xx];
                V[i] = s;
            }
            __syncthreads();
            float d2 = 0.0f;
            for (int t = 0; t < P; ++t) d2 += V[ty * DW + tx + t];
            d2 *= a.inv_np;
            const int qy = py + dy, qx = px + dx;
            if (qy >= 0 && qy < H && qx >= 0 && qx < W) {
                float e = fmaxf(d2 - two_s2, 0.0f);
                float w = __expf(-e * inv_h2);
                acc[0] = fmaf(w, S[(ty + r + hs + dy) * GW + tx + r + hs + dx], acc[0]);
#pragma unroll
                for (int c = 1; c < 3; ++c)
                    if (c < a.C) acc[c] = fmaf(w, Y[(c - 1) * VH * VW + (ty + hs + dy) * VW + tx + hs + dx], acc[c]);
                wsum += w;
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
    size_t smem = sizeof(float) * ((size_t)GH * GW + (size_t)DH * DW + (size_t)kTY * DW + (size_t)(C - 1) * VH * VW);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    if (cudaFuncSetAttribute(k_nlm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
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
        DN_TRY(launch("nlm_fp32", s, [&] { k_nlm<<<grid, kThreads, smem, s>>>(a); }));
    }
    return DN_OK;
}

}  // namespace dn

// Layers of the flexible lightweight network of Sec. III ("Ours-FL": a U-Net
// of depthwise-separable 3x3 convolutions with stride-2 downsampling, 2x2
// transposed-convolution upsampling and additive skips, fed the noise level
// as an extra input plane), FP32, forward and backward, NCHW.
//
//   depthwise 3x3   y[n][c][yo][xo] = b[c] + sum_{i,j} w[c][i][j] x[n][c][s yo + i - 1][s xo + j - 1]
//                   (zero padding 1, stride s = 1 or 2, Ho = ceil(H / s))
//   pointwise       y[n][co][p] = b[co] + sum_ci w[co][ci] x[n][ci][p]
//   transposed 2x2  y[n][co][2i + a][2j + c] = b[co] + skip[...] + sum_ci w[ci][co][a][c] x[n][ci][i][j]
//
// Forward kernels map one thread to one output pixel (and a block of output
// channels in registers); data gradients map one thread to one input pixel
// (gathers, no atomics); weight gradients reduce over all pixels in a fixed
// order (per-thread partial sums, then a block tree), so every result is
// deterministic.
#include "common.cuh"

namespace dn {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float relu_if(float v, int relu) { return relu ? fmaxf(v, 0.0f) : v; }

// ---- depthwise 3x3 ----------------------------------------------------------------

__global__ void k_dw_fwd(const float *x, const float *w, const float *b, float *y, int N, int C, int H, int W,
                         int s, int Ho, int Wo, int relu)
{
    const size_t total = (size_t)N * C * Ho * Wo;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int xo = (int)(e % Wo);
        const int yo = (int)((e / Wo) % Ho);
        const size_t nc = e / ((size_t)Wo * Ho);
        const int c = (int)(nc % C);
        const float *xp = x + nc * H * W;
        const float *wc = w + c * 9;
        float acc = b ? b[c] : 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int yy = s * yo + i - 1;
            if (yy < 0 || yy >= H) continue;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int xx = s * xo + j - 1;
                if (xx >= 0 && xx < W) acc = fmaf(wc[i * 3 + j], xp[(size_t)yy * W + xx], acc);
            }
        }
        y[e] = relu_if(acc, relu);
    }
}

// dx[n][c][yy][xx] = sum over the outputs that read (yy, xx) of g * w.
__global__ void k_dw_bwd_data(const float *g, const float *w, float *dx, int N, int C, int H, int W, int s, int Ho,
                              int Wo)
{
    const size_t total = (size_t)N * C * H * W;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int xx = (int)(e % W);
        const int yy = (int)((e / W) % H);
        const size_t nc = e / ((size_t)W * H);
        const int c = (int)(nc % C);
        const float *gp = g + nc * Ho * Wo;
        const float *wc = w + c * 9;
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int t = yy + 1 - i;  // = s yo
            if (t < 0 || t % s) continue;
            const int yo = t / s;
            if (yo >= Ho) continue;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int u = xx + 1 - j;
                if (u < 0 || u % s) continue;
                const int xo = u / s;
                if (xo < Wo) acc = fmaf(wc[i * 3 + j], gp[(size_t)yo * Wo + xo], acc);
            }
        }
        dx[e] = acc;
    }
}

// Block reduction of V per-thread partial sums (fixed tree: deterministic).
template <int V>
__device__ __forceinline__ void block_sum(float (&v)[V], float *out)
{
    __shared__ float red[kT / 32][V];
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < V; ++k) red[wp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < V) {
        float s = 0.0f;
        for (int q = 0; q < kT / 32; ++q) s += red[q][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// One block per channel: dw[c][9] and db[c] summed over every (n, yo, xo).
__global__ void __launch_bounds__(kT) k_dw_bwd_weight(const float *x, const float *g, float *dw, float *db, int N,
                                                      int C, int H, int W, int s, int Ho, int Wo)
{
    const int c = blockIdx.x;
    float v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = 0.0f;
    const size_t per = (size_t)Ho * Wo;
    for (int n = 0; n < N; ++n) {
        const float *xp = x + ((size_t)n * C + c) * H * W;
        const float *gp = g + ((size_t)n * C + c) * per;
        for (size_t q = threadIdx.x; q < per; q += kT) {
            const int yo = (int)(q / Wo), xo = (int)(q % Wo);
            const float gv = gp[q];
            v[9] += gv;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int yy = s * yo + i - 1;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int xx = s * xo + j - 1;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W) v[i * 3 + j] = fmaf(gv, xp[(size_t)yy * W + xx], v[i * 3 + j]);
                }
            }
        }
    }
    __shared__ float out[10];
    block_sum<10>(v, out);
    __syncthreads();
    if (threadIdx.x < 9) dw[c * 9 + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x == 9 && db) db[c] = out[9];
}

// ---- pointwise ----------------------------------------------------------------------

constexpr int kPC = 16;  // output channels per thread

// y[n][co][p] = b[co] + sum_ci W(co, ci) x[n][ci][p], W(co, ci) = w[co * wso + ci * wsi]
// (wso = Cin, wsi = 1 for the forward pass; wso = 1, wsi = Cout for the data
// gradient, which multiplies by the transposed weights).
__global__ void k_pw(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                     int wso, int wsi, int relu)
{
    const int cg = blockIdx.y;  // block of kPC output channels
    const size_t total = (size_t)N * HW;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t n = e / HW, p = e % HW;
        const float *xp = x + n * Cin * HW + p;
        float acc[kPC];
#pragma unroll
        for (int k = 0; k < kPC; ++k) {
            const int co = cg * kPC + k;
            acc[k] = (b && co < Cout) ? b[co] : 0.0f;
        }
        for (int ci = 0; ci < Cin; ++ci) {
            const float xv = xp[(size_t)ci * HW];
#pragma unroll
            for (int k = 0; k < kPC; ++k) {
                const int co = cg * kPC + k;
                if (co < Cout) acc[k] = fmaf(__ldg(w + (size_t)co * wso + (size_t)ci * wsi), xv, acc[k]);
            }
        }
        float *yp = y + n * Cout * HW + p;
#pragma unroll
        for (int k = 0; k < kPC; ++k) {
            const int co = cg * kPC + k;
            if (co < Cout) yp[(size_t)co * HW] = relu_if(acc[k], relu);
        }
    }
}

constexpr int kWC = 16;  // input channels per block in the weight gradient

// Block (co, block of kWC input channels): dw[co][ci] = sum_{n,p} g[n][co][p] x[n][ci][p],
// and db[co] = sum g (from the first channel block).
__global__ void __launch_bounds__(kT) k_pw_bwd_weight(const float *x, const float *g, float *dw, float *db, int N,
                                                      int Cin, int Cout, int HW)
{
    const int co = blockIdx.x, c0 = blockIdx.y * kWC;
    float v[kWC + 1];
#pragma unroll
    for (int k = 0; k <= kWC; ++k) v[k] = 0.0f;
    for (int n = 0; n < N; ++n) {
        const float *gp = g + ((size_t)n * Cout + co) * HW;
        const float *xp = x + (size_t)n * Cin * HW;
        for (int p = threadIdx.x; p < HW; p += kT) {
            const float gv = gp[p];
            v[kWC] += gv;
#pragma unroll
            for (int k = 0; k < kWC; ++k)
                if (c0 + k < Cin) v[k] = fmaf(gv, xp[(size_t)(c0 + k) * HW + p], v[k]);
        }
    }
    __shared__ float out[kWC + 1];
    block_sum<kWC + 1>(v, out);
    __syncthreads();
    if (threadIdx.x < kWC && c0 + threadIdx.x < Cin) dw[(size_t)co * Cin + c0 + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x == kWC && blockIdx.y == 0 && db) db[co] = out[kWC];
}

// ---- transposed 2x2, stride 2 ----------------------------------------------------------

constexpr int kDC = 8;  // output channels per thread

// One thread per input pixel (n, i, j) and block of kDC output channels: the
// 2 x 2 output pixels it feeds.
__global__ void k_deconv_fwd(const float *x, const float *w, const float *b, const float *skip, float *y, int N,
                             int Cin, int Cout, int H, int W)
{
    const int cg = blockIdx.y;
    const size_t HW = (size_t)H * W, total = (size_t)N * HW;
    const int W2 = 2 * W;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t n = e / HW, q = e % HW;
        const int i = (int)(q / W), j = (int)(q % W);
        float acc[kDC][4];
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            const int co = cg * kDC + k;
            const float bb = (b && co < Cout) ? b[co] : 0.0f;
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[k][t] = bb;
        }
        const float *xp = x + n * Cin * HW + q;
        for (int ci = 0; ci < Cin; ++ci) {
            const float xv = xp[(size_t)ci * HW];
#pragma unroll
            for (int k = 0; k < kDC; ++k) {
                const int co = cg * kDC + k;
                if (co < Cout) {
                    const float4 w4 = __ldg(reinterpret_cast<const float4 *>(w + ((size_t)ci * Cout + co) * 4));
                    acc[k][0] = fmaf(w4.x, xv, acc[k][0]);
                    acc[k][1] = fmaf(w4.y, xv, acc[k][1]);
                    acc[k][2] = fmaf(w4.z, xv, acc[k][2]);
                    acc[k][3] = fmaf(w4.w, xv, acc[k][3]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            const int co = cg * kDC + k;
            if (co >= Cout) continue;
            const size_t base = ((n * Cout + co) * (2 * H) + 2 * i) * (size_t)W2 + 2 * j;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const size_t o = base + (size_t)(t >> 1) * W2 + (t & 1);
                y[o] = acc[k][t] + (skip ? skip[o] : 0.0f);
            }
        }
    }
}

// dx[n][ci][i][j] = sum_{co, a, c} w[ci][co][a][c] g[n][co][2i + a][2j + c]; one
// thread per input pixel and block of kDC input channels.
__global__ void k_deconv_bwd_data(const float *g, const float *w, float *dx, int N, int Cin, int Cout, int H, int W)
{
    const int cg = blockIdx.y;
    const size_t HW = (size_t)H * W, total = (size_t)N * HW;
    const int W2 = 2 * W;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t n = e / HW, q = e % HW;
        const int i = (int)(q / W), j = (int)(q % W);
        float acc[kDC];
#pragma unroll
        for (int k = 0; k < kDC; ++k) acc[k] = 0.0f;
        for (int co = 0; co < Cout; ++co) {
            const size_t base = ((n * Cout + co) * (2 * H) + 2 * i) * (size_t)W2 + 2 * j;
            const float g0 = g[base], g1 = g[base + 1], g2 = g[base + W2], g3 = g[base + W2 + 1];
#pragma unroll
            for (int k = 0; k < kDC; ++k) {
                const int ci = cg * kDC + k;
                if (ci < Cin) {
                    const float4 w4 = __ldg(reinterpret_cast<const float4 *>(w + ((size_t)ci * Cout + co) * 4));
                    acc[k] = fmaf(w4.x, g0, fmaf(w4.y, g1, fmaf(w4.z, g2, fmaf(w4.w, g3, acc[k]))));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            const int ci = cg * kDC + k;
            if (ci < Cin) dx[(n * Cin + ci) * HW + q] = acc[k];
        }
    }
}

// Block (ci, co): dw[ci][co][a][c] = sum_{n,i,j} x[n][ci][i][j] g[n][co][2i+a][2j+c];
// db[co] = sum g from the blocks with ci = 0.
__global__ void __launch_bounds__(kT) k_deconv_bwd_weight(const float *x, const float *g, float *dw, float *db,
                                                          int N, int Cin, int Cout, int H, int W)
{
    const int ci = blockIdx.x, co = blockIdx.y;
    const size_t HW = (size_t)H * W;
    const int W2 = 2 * W;
    float v[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int n = 0; n < N; ++n) {
        const float *xp = x + ((size_t)n * Cin + ci) * HW;
        const float *gp = g + ((size_t)n * Cout + co) * 4 * HW;
        for (size_t q = threadIdx.x; q < HW; q += kT) {
            const int i = (int)(q / W), j = (int)(q % W);
            const float xv = xp[q];
            const size_t o = (size_t)(2 * i) * W2 + 2 * j;
            const float g0 = gp[o], g1 = gp[o + 1], g2 = gp[o + W2], g3 = gp[o + W2 + 1];
            v[0] = fmaf(xv, g0, v[0]);
            v[1] = fmaf(xv, g1, v[1]);
            v[2] = fmaf(xv, g2, v[2]);
            v[3] = fmaf(xv, g3, v[3]);
            v[4] += (g0 + g1) + (g2 + g3);
        }
    }
    __shared__ float out[5];
    block_sum<5>(v, out);
    __syncthreads();
    if (threadIdx.x < 4) dw[((size_t)ci * Cout + co) * 4 + threadIdx.x] = out[threadIdx.x];
    if (threadIdx.x == 4 && ci == 0 && db) db[co] = out[4];
}

// z [N][3][H][W] = [pre / 255, noisy / 255, sigma_n / 255] (the noise-level map).
struct Sig255 {
    float v[kChunk];
};

__global__ void k_fl_pack_s(const float *pre, const float *noisy, Sig255 sg, float *z, int N, size_t HW)
{
    const size_t total = (size_t)N * HW;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t n = e / HW, p = e % HW;
        float *zp = z + n * 3 * HW + p;
        zp[0] = pre[e] * (1.0f / 255.0f);
        zp[HW] = noisy[e] * (1.0f / 255.0f);
        zp[2 * HW] = sg.v[n];
    }
}

int blocks_for(size_t total)
{
    const size_t b = (total + kT - 1) / kT;
    return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

bool dims_ok(long a, long b, long c, long d) { return a >= 1 && b >= 1 && c >= 1 && d >= 1; }

}  // namespace

}  // namespace dn

using namespace dn;

extern "C" {

dn_status dn_dw3x3_fwd(const float *x, const float *w, const float *b, float *y, int N, int C, int H, int W,
                       int stride, int relu, dn_stream_t stream)
{
    if (!x || !w || !y || !dims_ok(N, C, H, W) || (stride != 1 && stride != 2)) return DN_EINVAL;
    const int Ho = (H + stride - 1) / stride, Wo = (W + stride - 1) / stride;
    const size_t total = (size_t)N * C * Ho * Wo;
    return launch("fl_dw3x3_fwd", (cudaStream_t)stream, [&] {
        k_dw_fwd<<<blocks_for(total), kT, 0, (cudaStream_t)stream>>>(x, w, b, y, N, C, H, W, stride, Ho, Wo, relu);
    });
}

dn_status dn_dw3x3_bwd(const float *x, const float *g, const float *w, float *dx, float *dw, float *db, int N, int C,
                       int H, int W, int stride, dn_stream_t stream)
{
    if (!x || !g || !w || !dw || !dims_ok(N, C, H, W) || (stride != 1 && stride != 2)) return DN_EINVAL;
    const int Ho = (H + stride - 1) / stride, Wo = (W + stride - 1) / stride;
    cudaStream_t s = (cudaStream_t)stream;
    if (dx)
        DN_TRY(launch("fl_dw3x3_bwd_data", s, [&] {
            k_dw_bwd_data<<<blocks_for((size_t)N * C * H * W), kT, 0, s>>>(g, w, dx, N, C, H, W, stride, Ho, Wo);
        }));
    return launch("fl_dw3x3_bwd_weight", s, [&] {
        k_dw_bwd_weight<<<C, kT, 0, s>>>(x, g, dw, db, N, C, H, W, stride, Ho, Wo);
    });
}

dn_status dn_pw_fwd(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                    int relu, int transposed, dn_stream_t stream)
{
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, HW)) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(blocks_for((size_t)N * HW), (Cout + kPC - 1) / kPC);
    const int wso = transposed ? 1 : Cin, wsi = transposed ? Cout : 1;
    return launch("fl_pw_fwd", s, [&] { k_pw<<<grid, kT, 0, s>>>(x, w, b, y, N, Cin, Cout, HW, wso, wsi, relu); });
}

dn_status dn_pw_bwd_weight(const float *x, const float *g, float *dw, float *db, int N, int Cin, int Cout, int HW,
                           dn_stream_t stream)
{
    if (!x || !g || !dw || !dims_ok(N, Cin, Cout, HW)) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(Cout, (Cin + kWC - 1) / kWC);
    return launch("fl_pw_bwd_weight", s, [&] { k_pw_bwd_weight<<<grid, kT, 0, s>>>(x, g, dw, db, N, Cin, Cout, HW); });
}

dn_status dn_deconv2x2_fwd(const float *x, const float *w, const float *b, const float *skip, float *y, int N, int Cin,
                           int Cout, int H, int W, dn_stream_t stream)
{
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, (long)H * W)) return DN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(w) & 15) != 0) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(blocks_for((size_t)N * H * W), (Cout + kDC - 1) / kDC);
    return launch("fl_deconv2x2_fwd", s, [&] { k_deconv_fwd<<<grid, kT, 0, s>>>(x, w, b, skip, y, N, Cin, Cout, H, W); });
}

dn_status dn_deconv2x2_bwd(const float *x, const float *g, const float *w, float *dx, float *dw, float *db, int N,
                           int Cin, int Cout, int H, int W, dn_stream_t stream)
{
    if (!x || !g || !w || !dw || !dims_ok(N, Cin, Cout, (long)H * W)) return DN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(w) & 15) != 0) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (dx) {
        dim3 grid(blocks_for((size_t)N * H * W), (Cin + kDC - 1) / kDC);
        DN_TRY(launch("fl_deconv2x2_bwd_data", s, [&] { k_deconv_bwd_data<<<grid, kT, 0, s>>>(g, w, dx, N, Cin, Cout, H, W); }));
    }
    dim3 gw(Cin, Cout);
    return launch("fl_deconv2x2_bwd_weight", s, [&] { k_deconv_bwd_weight<<<gw, kT, 0, s>>>(x, g, dw, db, N, Cin, Cout, H, W); });
}

dn_status dn_fl_pack_input(const float *pre, const float *noisy, const float *sigma, float *z, int N, int H, int W,
                           dn_stream_t stream)
{
    if (!pre || !noisy || !sigma || !z || !dims_ok(N, H, W, 1)) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t HW = (size_t)H * W;
    for (int n0 = 0; n0 < N; n0 += kChunk) {
        const int nb = N - n0 < kChunk ? N - n0 : kChunk;
        Sig255 sg;
        for (int i = 0; i < nb; ++i) {
            if (!(sigma[n0 + i] >= 0.0f) || !(sigma[n0 + i] <= 255.0f)) return DN_EINVAL;
            sg.v[i] = sigma[n0 + i] / 255.0f;
        }
        const size_t off = (size_t)n0 * HW;
        DN_TRY(launch("fl_pack_input", s, [&] {
            k_fl_pack_s<<<blocks_for((size_t)nb * HW), kT, 0, s>>>(pre + off, noisy + off, sg, z + 3 * off, nb, HW);
        }));
    }
    return DN_OK;
}

}  // extern "C"

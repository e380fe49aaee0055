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
// Forward kernels: the depthwise layer gives each thread 4 adjacent output
// columns and a band of output rows (its whole input window loaded at once
// with 16-byte loads); the pointwise and transposed layers keep a block of
// output channels' weights in shared memory and give each thread 4 pixels x
// a block of output channels in registers, its inputs staged through shared
// memory with per-thread cp.async; scalar forms cover widths that are not
// multiples of 4 (or 8 at stride 2).  Data gradients map one thread to one
// input pixel (gathers, no atomics); weight gradients reduce over all pixels
// in a fixed order (per-thread partial sums, then a block tree), so every
// result is deterministic.
#include "common.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float relu_if(float v, int relu) { return relu ? fmaxf(v, 0.0f) : v; }

// ---- depthwise 3x3 ----------------------------------------------------------------

// Output rows per thread in the depthwise forward: the thread loads the
// S * (rows - 1) + 3 input rows of its 3-column window at once (all loads in
// flight together), then forms the outputs from registers.
template <int S> struct DwRows {
    static constexpr int value = S == 1 ? 16 : 8;
};

// One block per (plane n*C + c, column chunk, band of rows); each thread owns one
// output column of a band.  Threads of a warp hold consecutive columns, so every
// row load is coalesced.  Block shape: cw columns x (kT / cw) bands, cw =
// min(kT, Wo rounded up to 32).  Zero padding outside the image.
template <int S>
__global__ void __launch_bounds__(kT) k_dw_fwd(const float *__restrict__ x, const float *__restrict__ w,
                                               const float *__restrict__ b, float *__restrict__ y, int C, int H, int W,
                                               int Ho, int Wo, int cw, int bands_per_block, int col_chunks, int c0,
                                               int relu)
{
    constexpr int R = DwRows<S>::value, IN = S * (R - 1) + 3;
    const size_t nc = blockIdx.y;
    const int c = (int)((c0 + nc) % C);
    const int chunk = blockIdx.x % col_chunks, band0 = (blockIdx.x / col_chunks) * bands_per_block;
    const int xo = chunk * cw + (int)threadIdx.x % cw;
    const int yo0 = (band0 + (int)threadIdx.x / cw) * R;
    if (xo >= Wo || yo0 >= Ho) return;
    const float *xp = x + nc * H * W;
    const int xc = S * xo, y0 = S * yo0 - 1;
    const bool hl = xc - 1 >= 0, hr = xc + 1 < W;
    float v[IN][3];
#pragma unroll
    for (int r = 0; r < IN; ++r) {
        const int yy = y0 + r;
        if (yy >= 0 && yy < H) {
            const float *rp = xp + (size_t)yy * W + xc;
            v[r][0] = hl ? rp[-1] : 0.0f;
            v[r][1] = rp[0];
            v[r][2] = hr ? rp[1] : 0.0f;
        } else {
            v[r][0] = v[r][1] = v[r][2] = 0.0f;
        }
    }
    float k[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) k[t] = w[c * 9 + t];
    const float bias = b ? b[c] : 0.0f;
    float *yp = y + nc * Ho * Wo + xo;
#pragma unroll
    for (int o = 0; o < R; ++o) {
        if (yo0 + o >= Ho) break;
        float acc = bias;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc = fmaf(k[i * 3 + j], v[S * o + i][j], acc);
        yp[(size_t)(yo0 + o) * Wo] = relu_if(acc, relu);
    }
}

// Vector form for planes whose width is a multiple of 4 (stride 1) or 8
// (stride 2), 16-byte aligned: each thread owns 4 adjacent output columns (one
// float4 store per output row) and DwRows4<S> output rows.  Per input row it
// loads the values under its outputs with 16-byte loads (4 at stride 1, 8 at
// stride 2) plus the edge values beside them: input columns S xo - 1 ..
// S xo + 4 S, where output j takes columns S j .. S j + 2 of that run.
template <int S> struct DwRows4 {
    static constexpr int value = S == 1 ? 8 : 4;
};

template <int S>
__global__ void __launch_bounds__(kT) k_dw_fwd4(const float *__restrict__ x, const float *__restrict__ w,
                                                const float *__restrict__ b, float *__restrict__ y, int C, int H,
                                                int W, int Ho, int Wo, int cw, int bands_per_block, int col_chunks,
                                                int c0, int relu)
{
    constexpr int R = DwRows4<S>::value, IN = S * (R - 1) + 3, NV = S == 1 ? 6 : 9;
    const size_t nc = blockIdx.y;
    const int c = (int)((c0 + nc) % C);
    const int chunk = blockIdx.x % col_chunks, band0 = (blockIdx.x / col_chunks) * bands_per_block;
    const int q = chunk * cw + (int)threadIdx.x % cw;  // output quad: columns 4 q .. 4 q + 3
    const int yo0 = (band0 + (int)threadIdx.x / cw) * R;
    if (4 * q >= Wo || yo0 >= Ho) return;
    const float *xp = x + nc * H * W;
    const int xl = S * 4 * q - 1, y0 = S * yo0 - 1;  // first input column and row of the thread's window
    float v[IN][NV];
#pragma unroll
    for (int r = 0; r < IN; ++r) {
        const int yy = y0 + r;
        if (yy < 0 || yy >= H) {
#pragma unroll
            for (int k = 0; k < NV; ++k) v[r][k] = 0.0f;
            continue;
        }
        const float *rp = xp + (size_t)yy * W;
        v[r][0] = xl >= 0 ? rp[xl] : 0.0f;
        const float4 a = *reinterpret_cast<const float4 *>(rp + xl + 1);
        v[r][1] = a.x, v[r][2] = a.y, v[r][3] = a.z, v[r][4] = a.w;
        if (S == 1) {
            v[r][5] = xl + 5 < W ? rp[xl + 5] : 0.0f;
        } else {  // W % 8 == 0: the second quad ends at column 8 q + 7 <= W - 1
            const float4 e = *reinterpret_cast<const float4 *>(rp + xl + 5);
            v[r][5] = e.x, v[r][6] = e.y, v[r][7] = e.z, v[r][8] = e.w;
        }
    }
    float k[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) k[t] = w[c * 9 + t];
    const float bias = b ? b[c] : 0.0f;
    float *yp = y + nc * Ho * Wo + 4 * q;
#pragma unroll
    for (int o = 0; o < R; ++o) {
        if (yo0 + o >= Ho) break;
        float acc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = bias;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int t = 0; t < 3; ++t) s = fmaf(k[i * 3 + t], v[S * o + i][S * j + t], s);
            acc[j] = relu_if(s, relu);
        }
        *reinterpret_cast<float4 *>(yp + (size_t)(yo0 + o) * Wo) = make_float4(acc[0], acc[1], acc[2], acc[3]);
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

constexpr int kPC = 16;   // output channels per block row (grid.y)
constexpr int kPMax = 256; // largest Cin of the shared-memory weight block

// y[n][co][p] = b[co] + sum_ci W(co, ci) x[n][ci][p], W(co, ci) = w[co * wso + ci * wsi]
// (wso = Cin, wsi = 1 for the forward pass; wso = 1, wsi = Cout for the data
// gradient, which multiplies by the transposed weights).  The block's kPC x Cin
// weights are staged once in shared memory as [ci][kPC] and read with 16-byte
// broadcast loads; each thread owns two pixels (blockDim apart, so loads and
// stores stay coalesced) and kPC accumulators for each.
__global__ void __launch_bounds__(kT) k_pw(const float *__restrict__ x, const float *__restrict__ w,
                                           const float *__restrict__ b, float *__restrict__ y, int N, int Cin,
                                           int Cout, int HW, int wso, int wsi, int relu)
{
    __shared__ __align__(16) float ws[kPMax * kPC];
    __shared__ float bias[kPC];
    // blockIdx.x = output-channel chunk (fastest, so the chunks reading one pixel
    // tile run together and the tile comes from DRAM once), blockIdx.y = pixel tile
    const int co0 = blockIdx.x * kPC;
    for (int i = threadIdx.x; i < Cin * kPC; i += kT) {
        const int ci = i / kPC, k = i % kPC;
        ws[i] = co0 + k < Cout ? w[(size_t)(co0 + k) * wso + (size_t)ci * wsi] : 0.0f;
    }
    if (threadIdx.x < kPC) bias[threadIdx.x] = (b && co0 + threadIdx.x < Cout) ? b[co0 + threadIdx.x] : 0.0f;
    __syncthreads();
    const float4 *w4 = reinterpret_cast<const float4 *>(ws);
    const size_t total = (size_t)N * HW;
    for (size_t e0 = (size_t)blockIdx.y * 2 * kT + threadIdx.x; e0 < total; e0 += (size_t)gridDim.y * 2 * kT) {
        const size_t e1 = e0 + kT;
        const bool has1 = e1 < total;
        const size_t n0 = e0 / HW, p0 = e0 % HW, n1 = has1 ? e1 / HW : n0, p1 = has1 ? e1 % HW : p0;
        const float *xp0 = x + n0 * Cin * HW + p0, *xp1 = x + n1 * Cin * HW + p1;
        float a0[kPC], a1[kPC];
#pragma unroll
        for (int k = 0; k < kPC; ++k) a0[k] = a1[k] = bias[k];
        auto step = [&](int ci, float x0, float x1) {
#pragma unroll
            for (int q = 0; q < kPC / 4; ++q) {
                const float4 wq = w4[ci * (kPC / 4) + q];
                a0[4 * q] = fmaf(wq.x, x0, a0[4 * q]);
                a0[4 * q + 1] = fmaf(wq.y, x0, a0[4 * q + 1]);
                a0[4 * q + 2] = fmaf(wq.z, x0, a0[4 * q + 2]);
                a0[4 * q + 3] = fmaf(wq.w, x0, a0[4 * q + 3]);
                a1[4 * q] = fmaf(wq.x, x1, a1[4 * q]);
                a1[4 * q + 1] = fmaf(wq.y, x1, a1[4 * q + 1]);
                a1[4 * q + 2] = fmaf(wq.z, x1, a1[4 * q + 2]);
                a1[4 * q + 3] = fmaf(wq.w, x1, a1[4 * q + 3]);
            }
        };
        int ci = 0;
        for (; ci + 4 <= Cin; ci += 4) {  // four input channels' loads in flight at once
            float u0[4], u1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u0[q] = xp0[(size_t)(ci + q) * HW];
                u1[q] = xp1[(size_t)(ci + q) * HW];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) step(ci + q, u0[q], u1[q]);
        }
        for (; ci < Cin; ++ci) step(ci, xp0[(size_t)ci * HW], xp1[(size_t)ci * HW]);
        float *yp0 = y + n0 * Cout * HW + p0, *yp1 = y + n1 * Cout * HW + p1;
#pragma unroll
        for (int k = 0; k < kPC; ++k)
            if (co0 + k < Cout) {
                yp0[(size_t)k * HW + (size_t)co0 * HW] = relu_if(a0[k], relu);
                if (has1) yp1[(size_t)k * HW + (size_t)co0 * HW] = relu_if(a1[k], relu);
            }
    }
}

constexpr int kKC = 8;  // input channels per cp.async stage
constexpr size_t kStageBytes = 2 * kKC * kT * sizeof(float4);  // dynamic shared memory of the staged kernels

// Feeds step(ci, v) the float4 xp[ci * stride] of every channel ci < Cin in
// order, through the calling thread's slots of `stage` ([2][kKC][kT] float4):
// the thread copies kKC channels per stage with cp.async, two stages deep (the
// next kKC channels are in flight while the current ones are consumed), and
// reads back only what it copied itself, so no barrier is needed and the loads
// in flight hold no registers.
template <class Step>
__device__ __forceinline__ void staged_channels(const float4 *__restrict__ xp, size_t stride, int Cin, float4 *stage,
                                                int tid, Step &step)
{
    const int nchunk = (Cin + kKC - 1) / kKC;
    auto issue = [&](int c) {  // channels c kKC .. c kKC + kKC - 1 into stage c & 1
#pragma unroll
        for (int t = 0; t < kKC; ++t) {
            const int ci = c * kKC + t;
            if (ci < Cin)
                tc::cp_async16(tc::smem_u32(&stage[((c & 1) * kKC + t) * kT + tid]), xp + (size_t)ci * stride);
        }
        tc::cp_async_commit();
    };
    issue(0);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) issue(c + 1);
        else tc::cp_async_commit();  // an empty group keeps "all but the newest group" meaning chunk c
        tc::cp_async_wait<1>();
#pragma unroll
        for (int t = 0; t < kKC; ++t) {
            const int ci = c * kKC + t;
            if (ci >= Cin) break;
            step(ci, stage[((c & 1) * kKC + t) * kT + tid]);
        }
    }
}

// Vector form of k_pw for HW % 4 == 0 with 16-byte aligned x and y: each thread
// owns four consecutive pixels of one image (one float4 per channel row) and
// kPC output channels; its input float4s arrive through staged_channels.
__global__ void __launch_bounds__(kT) k_pw4(const float *__restrict__ x, const float *__restrict__ w,
                                            const float *__restrict__ b, float *__restrict__ y, int N, int Cin,
                                            int Cout, int HW, int wso, int wsi, int relu)
{
    extern __shared__ __align__(16) float4 stage[];  // [2][kKC][kT]
    __shared__ __align__(16) float ws[kPMax * kPC];
    __shared__ float bias[kPC];
    const int co0 = blockIdx.x * kPC, tid = threadIdx.x;
    for (int i = tid; i < Cin * kPC; i += kT) {
        const int ci = i / kPC, k = i % kPC;
        ws[i] = co0 + k < Cout ? w[(size_t)(co0 + k) * wso + (size_t)ci * wsi] : 0.0f;
    }
    if (tid < kPC) bias[tid] = (b && co0 + tid < Cout) ? b[co0 + tid] : 0.0f;
    __syncthreads();
    const float4 *w4 = reinterpret_cast<const float4 *>(ws);
    const size_t HW4 = (size_t)HW / 4, total = (size_t)N * HW4;
    for (size_t e = (size_t)blockIdx.y * kT + tid; e < total; e += (size_t)gridDim.y * kT) {
        const size_t n = e / HW4, q = e % HW4;
        const float4 *xp = reinterpret_cast<const float4 *>(x) + n * Cin * HW4 + q;
        float a[kPC][4];
#pragma unroll
        for (int k = 0; k < kPC; ++k) a[k][0] = a[k][1] = a[k][2] = a[k][3] = bias[k];
        auto step = [&](int ci, float4 v) {
#pragma unroll
            for (int g = 0; g < kPC / 4; ++g) {
                const float4 wq = w4[ci * (kPC / 4) + g];
                const float wk[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float *ak = a[4 * g + u];
                    ak[0] = fmaf(wk[u], v.x, ak[0]);
                    ak[1] = fmaf(wk[u], v.y, ak[1]);
                    ak[2] = fmaf(wk[u], v.z, ak[2]);
                    ak[3] = fmaf(wk[u], v.w, ak[3]);
                }
            }
        };
        staged_channels(xp, HW4, Cin, stage, tid, step);
        float4 *yp = reinterpret_cast<float4 *>(y) + (n * Cout + co0) * HW4 + q;
#pragma unroll
        for (int k = 0; k < kPC; ++k)
            if (co0 + k < Cout)
                yp[(size_t)k * HW4] = make_float4(relu_if(a[k][0], relu), relu_if(a[k][1], relu),
                                                  relu_if(a[k][2], relu), relu_if(a[k][3], relu));
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
// 2 x 2 output pixels it feeds.  The block's Cin x kDC x 4 weights are staged
// in shared memory ([ci][k][a][c], 16-byte broadcast loads).
__global__ void __launch_bounds__(kT) k_deconv_fwd(const float *x, const float *w, const float *b, const float *skip,
                                                   float *y, int N, int Cin, int Cout, int H, int W)
{
    __shared__ __align__(16) float ws[kPMax * kDC * 4];
    const int co0 = blockIdx.x * kDC;  // output-channel chunk fastest (pixel tile read once from DRAM)
    for (int i = threadIdx.x; i < Cin * kDC * 4; i += kT) {
        const int ci = i / (kDC * 4), k = (i / 4) % kDC, t = i % 4;
        ws[i] = co0 + k < Cout ? w[((size_t)ci * Cout + co0 + k) * 4 + t] : 0.0f;
    }
    __syncthreads();
    const float4 *w4 = reinterpret_cast<const float4 *>(ws);
    const size_t HW = (size_t)H * W, total = (size_t)N * HW;
    const int W2 = 2 * W;
    for (size_t e = (size_t)blockIdx.y * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.y * blockDim.x) {
        const size_t n = e / HW, q = e % HW;
        const int i = (int)(q / W), j = (int)(q % W);
        float acc[kDC][4];
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            const int co = co0 + k;
            const float bb = (b && co < Cout) ? b[co] : 0.0f;
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[k][t] = bb;
        }
        const float *xp = x + n * Cin * HW + q;
        for (int ci = 0; ci < Cin; ++ci) {
            const float xv = xp[(size_t)ci * HW];
#pragma unroll
            for (int k = 0; k < kDC; ++k) {
                const float4 w4v = w4[ci * kDC + k];
                acc[k][0] = fmaf(w4v.x, xv, acc[k][0]);
                acc[k][1] = fmaf(w4v.y, xv, acc[k][1]);
                acc[k][2] = fmaf(w4v.z, xv, acc[k][2]);
                acc[k][3] = fmaf(w4v.w, xv, acc[k][3]);
            }
        }
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            const int co = co0 + k;
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

constexpr int kDC4 = 4;  // output channels per block in the vector transposed conv

// Vector form of k_deconv_fwd for W % 4 == 0 with 16-byte aligned x, y and skip:
// each thread owns four consecutive input pixels of a row (one float4 per
// channel, arriving through staged_channels) and kDC4 output channels, i.e.
// two 8-wide output row segments per channel, stored as float4 pairs.
__global__ void __launch_bounds__(kT, 2) k_deconv_fwd4(const float *__restrict__ x, const float *__restrict__ w,
                                                    const float *__restrict__ b, const float *__restrict__ skip,
                                                    float *__restrict__ y, int N, int Cin, int Cout, int H, int W)
{
    extern __shared__ __align__(16) float4 stage[];  // [2][kKC][kT]: staged_channels
    __shared__ __align__(16) float ws[kPMax * kDC4 * 4];
    const int co0 = blockIdx.x * kDC4;
    for (int i = threadIdx.x; i < Cin * kDC4 * 4; i += kT) {
        const int ci = i / (kDC4 * 4), k = (i / 4) % kDC4, t = i % 4;
        ws[i] = co0 + k < Cout ? w[((size_t)ci * Cout + co0 + k) * 4 + t] : 0.0f;
    }
    __syncthreads();
    const float4 *w4 = reinterpret_cast<const float4 *>(ws);
    const int W4 = W / 4, W2 = 2 * W;
    const size_t HW4 = (size_t)H * W4, total = (size_t)N * HW4;
    for (size_t e = (size_t)blockIdx.y * kT + threadIdx.x; e < total; e += (size_t)gridDim.y * kT) {
        const size_t n = e / HW4, q = e % HW4;
        const int i = (int)(q / W4), j = 4 * (int)(q % W4);
        float acc[kDC4][4][4];  // [co][tap a*2+c][pixel]
#pragma unroll
        for (int k = 0; k < kDC4; ++k) {
            const float bb = (b && co0 + k < Cout) ? b[co0 + k] : 0.0f;
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[k][t][0] = acc[k][t][1] = acc[k][t][2] = acc[k][t][3] = bb;
        }
        const float4 *xp = reinterpret_cast<const float4 *>(x) + n * Cin * HW4 + q;
        auto step = [&](int ci, float4 v) {
#pragma unroll
            for (int k = 0; k < kDC4; ++k) {
                const float4 wq = w4[ci * kDC4 + k];
                const float wt[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[k][t][0] = fmaf(wt[t], v.x, acc[k][t][0]);
                    acc[k][t][1] = fmaf(wt[t], v.y, acc[k][t][1]);
                    acc[k][t][2] = fmaf(wt[t], v.z, acc[k][t][2]);
                    acc[k][t][3] = fmaf(wt[t], v.w, acc[k][t][3]);
                }
            }
        };
        staged_channels(xp, HW4, Cin, stage, (int)threadIdx.x, step);
#pragma unroll
        for (int k = 0; k < kDC4; ++k) {
            if (co0 + k >= Cout) continue;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                // output row 2i + a, columns 2j .. 2j + 7: taps (a, 0), (a, 1) of pixels j .. j + 3
                const size_t o = ((n * Cout + co0 + k) * (2 * (size_t)H) + 2 * i + a) * (size_t)W2 + 2 * j;
                const float *c0 = acc[k][2 * a], *c1 = acc[k][2 * a + 1];
                float4 lo = make_float4(c0[0], c1[0], c0[1], c1[1]), hi = make_float4(c0[2], c1[2], c0[3], c1[3]);
                if (skip) {
                    const float4 s0 = *reinterpret_cast<const float4 *>(skip + o);
                    const float4 s1 = *reinterpret_cast<const float4 *>(skip + o + 4);
                    lo.x += s0.x, lo.y += s0.y, lo.z += s0.z, lo.w += s0.w;
                    hi.x += s1.x, hi.y += s1.y, hi.z += s1.z, hi.w += s1.w;
                }
                *reinterpret_cast<float4 *>(y + o) = lo;
                *reinterpret_cast<float4 *>(y + o + 4) = hi;
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

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

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
    const bool vec = (stride == 1 ? W % 4 == 0 : W % 8 == 0) && aligned16(x) && aligned16(y);
    const int cols = vec ? Wo / 4 : Wo;  // threads along a row: output quads or columns
    const int cw = cols >= kT ? kT : (cols + 31) / 32 * 32, bpb = kT / cw;
    const int R = vec ? (stride == 1 ? DwRows4<1>::value : DwRows4<2>::value)
                      : (stride == 1 ? DwRows<1>::value : DwRows<2>::value);
    const int col_chunks = (cols + cw - 1) / cw, bands = (Ho + R - 1) / R;
    const int gx = col_chunks * ((bands + bpb - 1) / bpb);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t planes = (size_t)N * C, in_plane = (size_t)H * W, out_plane = (size_t)Ho * Wo;
    for (size_t p0 = 0; p0 < planes; p0 += 65535) {  // grid.y = planes of this launch
        const unsigned np = (unsigned)(planes - p0 < 65535 ? planes - p0 : 65535);
        const float *xs = x + p0 * in_plane;
        float *ys = y + p0 * out_plane;
        const int c0 = (int)(p0 % C);  // channel of this launch's first plane
        DN_TRY(launch("fl_dw3x3_fwd", s, [&] {
            const dim3 grid(gx, np);
            if (vec && stride == 1)
                k_dw_fwd4<1><<<grid, kT, 0, s>>>(xs, w, b, ys, C, H, W, Ho, Wo, cw, bpb, col_chunks, c0, relu);
            else if (vec)
                k_dw_fwd4<2><<<grid, kT, 0, s>>>(xs, w, b, ys, C, H, W, Ho, Wo, cw, bpb, col_chunks, c0, relu);
            else if (stride == 1)
                k_dw_fwd<1><<<grid, kT, 0, s>>>(xs, w, b, ys, C, H, W, Ho, Wo, cw, bpb, col_chunks, c0, relu);
            else
                k_dw_fwd<2><<<grid, kT, 0, s>>>(xs, w, b, ys, C, H, W, Ho, Wo, cw, bpb, col_chunks, c0, relu);
        }));
    }
    return DN_OK;
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
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, HW) || Cin > kPMax) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((Cout + kPC - 1) / kPC, blocks_for(((size_t)N * HW + 1) / 2));
    const int wso = transposed ? 1 : Cin, wsi = transposed ? Cout : 1;
    if (HW % 4 == 0 && aligned16(x) && aligned16(y)) {
        if (cudaFuncSetAttribute(k_pw4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes) != cudaSuccess)
            return DN_ECUDA;
        dim3 g4((Cout + kPC - 1) / kPC, blocks_for((size_t)N * HW / 4));
        return launch("fl_pw_fwd", s,
                      [&] { k_pw4<<<g4, kT, kStageBytes, s>>>(x, w, b, y, N, Cin, Cout, HW, wso, wsi, relu); });
    }
    return launch("fl_pw_fwd", s, [&] { k_pw<<<grid, kT, 0, s>>>(x, w, b, y, N, Cin, Cout, HW, wso, wsi, relu); });
}

dn_status dn_pw_fwd_bf16(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                         int relu, int transposed, dn_stream_t stream)
{
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, HW)) return DN_EINVAL;
    if (Cin > 256 || Cout > 256) return DN_EUNSUPPORTED;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    return pw_fwd_tc(x, w, b, y, N, Cin, Cout, HW, relu, transposed, err, (cudaStream_t)stream);
}

dn_status dn_deconv2x2_fwd_bf16(const float *x, const float *w, const float *b, const float *skip, float *y, int N,
                                int Cin, int Cout, int H, int W, dn_stream_t stream)
{
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, (long)H * W)) return DN_EINVAL;
    if (Cin > 256 || Cout > 256) return DN_EUNSUPPORTED;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    return deconv2x2_fwd_tc(x, w, b, skip, y, N, Cin, Cout, H, W, err, (cudaStream_t)stream);
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
    if (!x || !w || !y || !dims_ok(N, Cin, Cout, (long)H * W) || Cin > kPMax) return DN_EINVAL;
    if ((reinterpret_cast<uintptr_t>(w) & 15) != 0) return DN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (W % 4 == 0 && aligned16(x) && aligned16(y) && (!skip || aligned16(skip))) {
        if (cudaFuncSetAttribute(k_deconv_fwd4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes) !=
            cudaSuccess)
            return DN_ECUDA;
        dim3 g4((Cout + kDC4 - 1) / kDC4, blocks_for((size_t)N * H * W / 4));
        return launch("fl_deconv2x2_fwd", s,
                      [&] { k_deconv_fwd4<<<g4, kT, kStageBytes, s>>>(x, w, b, skip, y, N, Cin, Cout, H, W); });
    }
    dim3 grid((Cout + kDC - 1) / kDC, blocks_for((size_t)N * H * W));
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

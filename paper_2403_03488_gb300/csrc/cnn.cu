// Residual CNN of Sec. II (Fig. 1, Eq. 2-3): FP32 SIMT kernels.
//
// Layers are 3x3 cross-correlations with zero padding 1 on NCHW float
// activations, weights [Cout][3][3][Cin].  Forward, data gradient (the same
// kernel reading the weights flipped and transposed), weight gradient,
// the L1 loss gradient of Eq. 2 and Adam.  These kernels are the FP32 plain
// path and the reference of the gradient checks; the BF16 tensor-core
// forward lives in conv_tc.cu.
#include <cmath>

#include "common.cuh"

namespace dn {

namespace {

constexpr int kT = 16;       // output tile side
constexpr int kOG = 8;        // output channels per CTA
constexpr int kHalo = kT + 2;

// y[n][o] = sum_i sum_taps wv(o, i, ky, kx) x[n][i][py + ky - 1][px + kx - 1]
// TRANS: wv(o, i, ky, kx) = w[i][2-ky][2-kx][o] (w of shape [Kin][3][3][Kout]),
//        i.e. the data gradient of a layer whose weights are w.
template <bool TRANS>
__global__ void __launch_bounds__(kT *kT) k_conv3x3(const float *x, const float *w, const float *bias,
                                                    const float *mask, float *y, int Kin, int Kout, int H, int W,
                                                    int relu)
{
    extern __shared__ float sm[];
    float *ws = sm;                   // [kOG][Kin][9]
    float *xs = sm + kOG * Kin * 9;   // [kHalo][kHalo]
    const int groups = (Kout + kOG - 1) / kOG;
    const int n = blockIdx.z / groups, og = blockIdx.z % groups;
    const int o0 = og * kOG;
    const int X0 = blockIdx.x * kT, Y0 = blockIdx.y * kT;
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
    const size_t HW = (size_t)H * W;

    for (int e = threadIdx.x; e < kOG * Kin * 9; e += kT * kT) {
        int oo = e / (Kin * 9), rem = e - oo * Kin * 9, i = rem / 9, t = rem - i * 9;
        int o = o0 + oo;
        float v = 0.0f;
        if (o < Kout) {
            int ky = t / 3, kx = t % 3;
            v = TRANS ? w[((size_t)(i * 3 + (2 - ky)) * 3 + (2 - kx)) * Kout + o]
                      : w[((size_t)(o * 3 + ky) * 3 + kx) * Kin + i];
        }
        ws[e] = v;
    }
    float acc[kOG];
#pragma unroll
    for (int oo = 0; oo < kOG; ++oo) acc[oo] = 0.0f;

    const float *xn = x + (size_t)n * Kin * HW;
    for (int i = 0; i < Kin; ++i) {
        __syncthreads();
        for (int e = threadIdx.x; e < kHalo * kHalo; e += kT * kT) {
            int yy = e / kHalo, xx = e - yy * kHalo;
            int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
            xs[e] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xn[(size_t)i * HW + (size_t)gy * W + gx] : 0.0f;
        }
        __syncthreads();
        float v[9];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) v[ky * 3 + kx] = xs[(ty + ky) * kHalo + tx + kx];
#pragma unroll
        for (int oo = 0; oo < kOG; ++oo) {
            const float *wo = ws + (oo * Kin + i) * 9;
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[oo] = fmaf(wo[t], v[t], acc[oo]);
        }
    }
    const int px = X0 + tx, py = Y0 + ty;
    if (px >= W || py >= H) return;
#pragma unroll
    for (int oo = 0; oo < kOG; ++oo) {
        int o = o0 + oo;
        if (o >= Kout) break;
        size_t at = ((size_t)n * Kout + o) * HW + (size_t)py * W + px;
        float r = acc[oo] + (bias ? bias[o] : 0.0f);
        if (relu) r = fmaxf(r, 0.0f);
        if (mask && !(mask[at] > 0.0f)) r = 0.0f;
        y[at] = r;
    }
}

// dw[co][ky][kx][ci] += sum over one 16x16 tile of dy[co] * x[ci] shifted; db[co] += sum dy[co].
__global__ void __launch_bounds__(kT *kT) k_conv3x3_bwd_w(const float *x, const float *dy, float *dw, float *db,
                                                          int Cin, int Cout, int H, int W)
{
    extern __shared__ float sm[];
    float *ds = sm;                    // [Cout][256]
    float *xs = sm + Cout * kT * kT;   // [Cin][kHalo*kHalo]
    const int n = blockIdx.z;
    const int X0 = blockIdx.x * kT, Y0 = blockIdx.y * kT;
    const size_t HW = (size_t)H * W;
    for (int e = threadIdx.x; e < Cout * kT * kT; e += kT * kT) {
        int co = e / (kT * kT), p = e - co * kT * kT;
        int gy = Y0 + p / kT, gx = X0 + p % kT;
        ds[e] = (gy < H && gx < W) ? dy[((size_t)n * Cout + co) * HW + (size_t)gy * W + gx] : 0.0f;
    }
    for (int e = threadIdx.x; e < Cin * kHalo * kHalo; e += kT * kT) {
        int ci = e / (kHalo * kHalo), p = e - ci * kHalo * kHalo;
        int gy = Y0 - 1 + p / kHalo, gx = X0 - 1 + p % kHalo;
        xs[e] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? x[((size_t)n * Cin + ci) * HW + (size_t)gy * W + gx]
                                                          : 0.0f;
    }
    __syncthreads();
    const int total = Cout * 9 * Cin;
    for (int o = threadIdx.x; o < total; o += kT * kT) {
        int co = o / (9 * Cin), rem = o - co * 9 * Cin, t = rem / Cin, ci = rem - t * Cin;
        int ky = t / 3, kx = t % 3;
        const float *d = ds + co * kT * kT;
        const float *xx = xs + ci * kHalo * kHalo;
        float s = 0.0f;
        for (int py = 0; py < kT; ++py)
#pragma unroll 4
            for (int px = 0; px < kT; ++px) s = fmaf(d[py * kT + px], xx[(py + ky) * kHalo + px + kx], s);
        atomicAdd(dw + o, s);
    }
    for (int co = threadIdx.x; co < Cout; co += kT * kT) {
        float s = 0.0f;
        for (int p = 0; p < kT * kT; ++p) s += ds[co * kT * kT + p];
        atomicAdd(db + co, s);
    }
}

// z[n] = [pre[n] / 255 (cc planes), noisy[n] / 255 (cc planes)]; i runs over
// the N cc HW elements of pre / noisy.
__global__ void k_pack_input(const float *pre, const float *noisy, float *z, size_t HW, int cc, size_t total)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t nc = i / HW, p = i - nc * HW, n = nc / cc, c = nc - n * cc;
        z[(2 * cc * n + c) * HW + p] = pre[i] * (1.0f / 255.0f);
        z[(2 * cc * n + cc + c) * HW + p] = noisy[i] * (1.0f / 255.0f);
    }
}

__global__ void k_residual_out(const float *pre, const float *r, float *out, size_t total)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        out[i] = fmaf(255.0f, r[i], pre[i]);
}

__global__ void k_relu_bwd(const float *g, const float *y, float *out, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = y[i] > 0.0f ? g[i] : 0.0f;
}

__global__ void k_l1_grad(const float *r, const float *pre, const float *clean, float *dr, size_t count,
                          double *loss)
{
    const float g = 255.0f / (float)count;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        float e = fmaf(255.0f, r[i], pre[i]) - clean[i];
        dr[i] = e > 0.0f ? g : (e < 0.0f ? -g : 0.0f);
        s += fabs((double)e);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
        if (loss) atomicAdd(loss, t);
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t count, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi;
        float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

int ew_blocks(size_t n)
{
    size_t b = (n + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

dn_status conv3x3_fwd_fp32(const float *x, const float *w, const float *b, const float *mask, float *y, int N,
                           int Kin, int Kout, int H, int W, int relu, bool trans, cudaStream_t s)
{
    const int groups = (Kout + kOG - 1) / kOG;
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, N * groups);
    size_t smem = sizeof(float) * ((size_t)kOG * Kin * 9 + kHalo * kHalo);
    if (trans) {
        if (cudaFuncSetAttribute(k_conv3x3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DN_ECUDA;
        return launch("conv3x3_bwd_data_fp32", s,
                      [&] { k_conv3x3<true><<<grid, kT * kT, smem, s>>>(x, w, b, mask, y, Kin, Kout, H, W, relu); });
    }
    if (cudaFuncSetAttribute(k_conv3x3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    return launch("conv3x3_fwd_fp32", s,
                  [&] { k_conv3x3<false><<<grid, kT * kT, smem, s>>>(x, w, b, mask, y, Kin, Kout, H, W, relu); });
}

dn_status conv3x3_bwd_weight_fp32(const float *x, const float *dy, float *dw, float *db, int N, int Cin, int Cout,
                                  int H, int W, cudaStream_t s)
{
    if (cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)Cout * 9 * Cin, s) != cudaSuccess) return DN_ECUDA;
    if (cudaMemsetAsync(db, 0, sizeof(float) * (size_t)Cout, s) != cudaSuccess) return DN_ECUDA;
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, N);
    size_t smem = sizeof(float) * ((size_t)Cout * kT * kT + (size_t)Cin * kHalo * kHalo);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    if (cudaFuncSetAttribute(k_conv3x3_bwd_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    return launch("conv3x3_bwd_weight_fp32", s,
                  [&] { k_conv3x3_bwd_w<<<grid, kT * kT, smem, s>>>(x, dy, dw, db, Cin, Cout, H, W); });
}

dn_status pack_input(const float *pre, const float *noisy, float *z, int N, int cc, int H, int W, cudaStream_t s)
{
    size_t HW = (size_t)H * W, total = (size_t)N * cc * HW;
    return launch("cnn_pack_input", s,
                  [&] { k_pack_input<<<ew_blocks(total), 256, 0, s>>>(pre, noisy, z, HW, cc, total); });
}

dn_status residual_out(const float *pre, const float *r, float *out, size_t total, cudaStream_t s)
{
    return launch("cnn_residual_out", s, [&] { k_residual_out<<<ew_blocks(total), 256, 0, s>>>(pre, r, out, total); });
}

dn_status relu_bwd(const float *g, const float *y, float *out, size_t count, cudaStream_t s)
{
    return launch("relu_bwd", s, [&] { k_relu_bwd<<<ew_blocks(count), 256, 0, s>>>(g, y, out, count); });
}

dn_status l1_grad(const float *r, const float *pre, const float *clean, float *dr, size_t count, double *loss,
                  cudaStream_t s)
{
    return launch("l1_residual_grad", s,
                  [&] { k_l1_grad<<<ew_blocks(count), 256, 0, s>>>(r, pre, clean, dr, count, loss); });
}

dn_status adam(float *p, const float *g, float *m, float *v, size_t count, int t, float lr, float b1, float b2,
               float eps, cudaStream_t s)
{
    double c1 = 1.0 / (1.0 - std::pow((double)b1, t)), c2 = 1.0 / (1.0 - std::pow((double)b2, t));
    return launch("adam_step", s, [&] {
        k_adam<<<ew_blocks(count), 256, 0, s>>>(p, g, m, v, count, lr, b1, b2, eps, (float)c1, (float)c2);
    });
}

}  // namespace dn

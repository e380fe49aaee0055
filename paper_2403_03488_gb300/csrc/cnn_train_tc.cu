// Training of the residual CNN (Sec. II, Eq. 2) with BF16 operands on the
// tensor cores and FP32 accumulation / master weights.
//
// One gradient evaluation of the L1 loss of Eq. 2 over a batch:
//   forward   a_0 = ReLU(conv_first(z)), a_l = ReLU(conv_l(a_{l-1})) on tcgen05
//             (l = 1 .. K-2), out = pre + 255 conv_last(a_{K-2}); activations
//             kept as NHWC BF16;
//   loss      dr = 255 sign(out - clean) / count;
//   backward  G_{K-2} = (a_{K-2} > 0) * conv_last^T(dr)                 (CUDA cores)
//             dW_l = sum_px G_l (x) shift(a_{l-1}), db_l = sum_px G_l    (tcgen05 GEMM, K = pixels)
//             G_{l-1} = (a_{l-1} > 0) * conv_l^T(G_l)                   (tcgen05, flipped weights)
//             dW_first = sum_px G_0 (x) shift(z)                         (CUDA cores)
// Every reduction over pixels is a fixed-order sum of per-CTA partials, so
// the gradient is bitwise reproducible.
//
// Weight-gradient GEMM (hidden layers, C = 32): for each output-gradient row
// r and horizontal tap dx, D[m][n] += sum_p A[m][p] B[p][n] with
//   m = dy * 32 + ci (dy = 0..3; dy = 3 is computed and discarded),
//   A[m][p] = a_{l-1}[r + dy - 1][p + dx - 1][ci], B[p][n] = G_l[r][p][n],
// both MN-major straight from the staged rows: a staged row holds 4 channel
// planes of 16-byte pixels (8 channels), so 8 channels x 8 pixels form a core
// matrix, the 4 planes of a row and 4 consecutive rows have one uniform
// stride along M (2080 bytes), and the tap dx is a 16-byte shift of the
// start.  The three dx accumulators (3 x 32 TMEM columns) persist over all the
// work items of a CTA; each CTA writes one partial.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kBwR = 4;                 // output-gradient rows per work item
constexpr int kBwPX = 128;              // pixels per strip (K of one row)
constexpr int kXP = 130;                // staged activation pixels per row (halo of 1)
constexpr int kXRow = kXP * 64;         // bytes of one staged activation row (C = 32)
constexpr int kGRow = kBwPX * 64;       // bytes of one staged gradient row
constexpr int kBwSmem = (kBwR + 3) * kXRow + kBwR * kGRow + 64;
constexpr int kBwCtasPerSm = 2;
constexpr int kPartW = 3 * 32 * 96;     // floats of one weight-gradient partial [dy][ci][dx][co]
// BF16 x BF16 -> F32, M = 128, N = 32, A and B MN-major
constexpr uint32_t kIdescBw = tc::idesc_bf16(128, 32) | (1u << 15) | (1u << 16);

struct BwArgs {
    const uint4 *x;   // a_{l-1}: [N][H][W][32] bf16
    const uint4 *g;   // G_l:     [N][H][W][32] bf16
    float *partial;   // [gridDim.x][kPartW]
    int N, H, W, strips, groups;
    int *err;
};

__global__ void __launch_bounds__(128) k_conv_bwd_w_tc(BwArgs a)
{
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *xs = sm;                              // [kBwR + 3 rows][4 planes][130][16 B]
    uint8_t *gs = sm + (kBwR + 3) * kXRow;         // [kBwR rows][4 planes][128][16 B]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(gs + kBwR * kGRow);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    if (tid == 0) tc::mbar_init(mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool first = true, failed = false;
    const int items = a.N * a.strips * a.groups;
    for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const int grp = it % a.groups, rest = it / a.groups;
        const int strip = rest % a.strips, n = rest / a.strips;
        const int x0 = strip * kBwPX, r0 = grp * kBwR;
        // activation rows r0 - 1 .. r0 + kBwR + 1, pixels x0 - 1 .. x0 + 128 (zeros outside the image)
        for (int i = tid; i < (kBwR + 3) * kXP * 4; i += 128) {
            const int row = i / (kXP * 4), rem = i - row * (kXP * 4), px = rem >> 2, ck = rem & 3;
            const int gy = r0 - 1 + row, gx = x0 - 1 + px;
            uint8_t *dst = xs + row * kXRow + ck * kXP * 16 + px * 16;
            if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                tc::cp_async16(tc::smem_u32(dst), a.x + (((size_t)n * a.H + gy) * a.W + gx) * 4 + ck);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        // gradient rows r0 .. r0 + kBwR - 1, pixels x0 .. x0 + 127
        for (int i = tid; i < kBwR * kBwPX * 4; i += 128) {
            const int row = i / (kBwPX * 4), rem = i - row * (kBwPX * 4), px = rem >> 2, ck = rem & 3;
            const int gy = r0 + row, gx = x0 + px;
            uint8_t *dst = gs + row * kGRow + ck * kBwPX * 16 + px * 16;
            if (gy < a.H && gx < a.W)
                tc::cp_async16(tc::smem_u32(dst), a.g + (((size_t)n * a.H + gy) * a.W + gx) * 4 + ck);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::cp_async_commit();
        tc::cp_async_wait<0>();
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t xb = tc::smem_u32(xs), gb = tc::smem_u32(gs);
            for (int rr = 0; rr < kBwR; ++rr) {
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int k = 0; k < kBwPX / 16; ++k) {
                        const uint64_t ad = tc::sdesc(xb + rr * kXRow + (16 * k + dx) * 16, 128, kXP * 16);
                        const uint64_t bd = tc::sdesc(gb + rr * kGRow + 16 * k * 16, 128, kBwPX * 16);
                        const uint32_t acc = (first && rr == 0 && k == 0) ? 0u : 1u;
                        tc::mma_bf16(tmem + (uint32_t)(32 * dx), ad, bd, kIdescBw, acc);
                    }
            }
            tc::mma_commit(mbar);
        }
        first = false;
        // the staged rows are overwritten by the next item only after these MMAs completed
        const bool ok = tc::mbar_wait(mbar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            if (tid == 0) atomicExch(a.err, 4);
            tc::mbar_wait(mbar, phase ^ 1u);  // bounded: the MMAs in flight finish before TMEM is freed
        }
        tc::fence_after_sync();
    }
    float *part = a.partial + (size_t)blockIdx.x * kPartW;
    if (warp < 3) {
        // lane m = warp * 32 + lane: dy = warp, ci = lane; columns dx * 32 + co
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            uint32_t r[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * dx), r);
            tc::tmem_wait_ld();
            float *dst = part + ((size_t)warp * 32 + lane) * 96 + dx * 32;
#pragma unroll
            for (int co = 0; co < 32; ++co) dst[co] = (first || failed) ? 0.0f : __uint_as_float(r[co]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 128);
    }
}

// dw [32][3][3][32] (= sum over partials, fixed order), db [32] from the bias partials.
__global__ void k_reduce_dw_tc(const float *part, int nparts, const float *bpart, int nb, float *dw, float *db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // dw index (co, dy, dx, ci)
    if (i < 32 * 9 * 32) {
        const int ci = i & 31, t = (i >> 5) % 9, co = i / (9 * 32), dy = t / 3, dx = t % 3;
        const int j = (dy * 32 + ci) * 96 + dx * 32 + co;
        float s = 0.0f;
        for (int p = 0; p < nparts; ++p) s += part[(size_t)p * kPartW + j];
        dw[i] = s;
    } else if (i < 32 * 9 * 32 + 32) {
        const int co = i - 32 * 9 * 32;
        float s = 0.0f;
        for (int p = 0; p < nb; ++p) s += bpart[(size_t)p * 32 + co];
        db[co] = s;
    }
}

// Per-CTA partial sums over 256 pixels of G [N][H][W][32] bf16 per channel.
__global__ void __launch_bounds__(256) k_bias_grad_nhwc(const uint4 *g, size_t npx, float *bpart)
{
    __shared__ float red[8][32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // lane = channel pair index (16 pairs) x 2 pixel parities
    float s = 0.0f;
    const size_t p0 = (size_t)blockIdx.x * 256;
    for (int k = w; k < 256; k += 8) {
        const size_t p = p0 + k;
        if (p < npx) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(g + p * 4);
            const uint32_t u = row[lane >> 1];
            s += (lane & 1) ? tc::bf16_hi(u) : tc::bf16_lo(u);
        }
    }
    red[w][lane] = s;
    __syncthreads();
    if (tid < 32) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += red[k][tid];
        bpart[(size_t)blockIdx.x * 32 + tid] = t;
    }
}

// Last layer (32 -> 1) backward.  dr: [N][H][W] FP32 (dL/dr); a: [N][H][W][32]
// bf16 (its input, a ReLU output).  G[p][ci] = (a[p][ci] > 0) sum_{ky,kx}
// w[ky][kx][ci] dr[py - ky + 1][px - kx + 1], stored as bf16.
__global__ void __launch_bounds__(256) k_last_bwd_data(const float *dr, const uint4 *a, const float *w, uint4 *G,
                                                      int H, int W, size_t npx)
{
    __shared__ float ws[9 * 32];
    for (int i = threadIdx.x; i < 9 * 32; i += 256) ws[i] = w[i];
    __syncthreads();
    const size_t p = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= npx) return;
    const size_t HW = (size_t)H * W;
    const size_t n = p / HW;
    const int rem = (int)(p - n * HW), py = rem / W, px = rem - py * W;
    float d[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int qy = py - ky + 1, qx = px - kx + 1;
            d[ky * 3 + kx] = (qy >= 0 && qy < H && qx >= 0 && qx < W) ? dr[n * HW + (size_t)qy * W + qx] : 0.0f;
        }
    const uint4 *ap = a + p * 4;
    uint4 *gp = G + p * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 u = ap[q];
        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ci = q * 8 + 2 * e + h;
                float s = 0.0f;
#pragma unroll
                for (int t = 0; t < 9; ++t) s = fmaf(ws[t * 32 + ci], d[t], s);
                const float av = h ? tc::bf16_hi(uu[e]) : tc::bf16_lo(uu[e]);
                v[h] = av > 0.0f ? s : 0.0f;
            }
            pk[e] = tc::pack_bf16x2(v[0], v[1]);
        }
        gp[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Weight gradient of the last layer over one 16 x 16 tile: part[blk][t * 32 + ci]
// = sum_p dr[p] a[p + tap - 1][ci] (t = tap), part[blk][288] = sum_p dr[p].
__global__ void __launch_bounds__(320) k_last_bwd_w(const float *dr, const uint4 *a, float *part, int H, int W)
{
    __shared__ float ds[256];
    __shared__ uint4 as[18 * 18 * 4];
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16, tid = threadIdx.x;
    const size_t HW = (size_t)H * W;
    for (int i = tid; i < 256; i += 320) {
        const int y = Y0 + i / 16, x = X0 + i % 16;
        ds[i] = (y < H && x < W) ? dr[n * HW + (size_t)y * W + x] : 0.0f;
    }
    for (int i = tid; i < 18 * 18 * 4; i += 320) {
        const int p = i >> 2, ck = i & 3, yy = p / 18, xx = p % 18, gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        as[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? a[((size_t)n * HW + (size_t)gy * W + gx) * 4 + ck]
                                                         : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const size_t blk = ((size_t)n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (tid < 288) {
        const int t = tid / 32, ci = tid % 32, ky = t / 3, kx = t % 3;
        const int ck = ci >> 3, e = (ci & 7) >> 1, hi = ci & 1;
        float s = 0.0f;
        for (int i = 0; i < 256; ++i) {
            const uint4 u = as[((i / 16 + ky) * 18 + (i % 16) + kx) * 4 + ck];
            const uint32_t uu = e == 0 ? u.x : (e == 1 ? u.y : (e == 2 ? u.z : u.w));
            s = fmaf(ds[i], hi ? tc::bf16_hi(uu) : tc::bf16_lo(uu), s);
        }
        part[blk * 289 + tid] = s;
    } else if (tid == 288) {
        float s = 0.0f;
        for (int i = 0; i < 256; ++i) s += ds[i];
        part[blk * 289 + 288] = s;
    }
}

// Weight gradient of the first layer (2 -> 32) over one 16 x 16 tile:
// part[blk][(co * 9 + t) * 2 + c] = sum_p G[p][co] z_c[p + tap - 1] with
// z = [pre / 255, noisy / 255]; part[blk][576 + co] = sum_p G[p][co].
__global__ void __launch_bounds__(608) k_first_bwd_w(const float *pre, const float *noisy, const uint4 *G, float *part,
                                                     int H, int W)
{
    __shared__ float zs[2][18 * 18];
    __shared__ uint4 gs[256 * 4];
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16, tid = threadIdx.x;
    const size_t HW = (size_t)H * W;
    for (int i = tid; i < 2 * 324; i += 608) {
        const int c = i / 324, p = i % 324, yy = p / 18, xx = p % 18, gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        const float *src = c == 0 ? pre : noisy;
        zs[c][p] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? src[n * HW + (size_t)gy * W + gx] * (1.0f / 255.0f)
                                                           : 0.0f;
    }
    for (int i = tid; i < 256 * 4; i += 608) {
        const int p = i >> 2, ck = i & 3, y = Y0 + p / 16, x = X0 + p % 16;
        gs[i] = (y < H && x < W) ? G[((size_t)n * HW + (size_t)y * W + x) * 4 + ck] : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const size_t blk = ((size_t)n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (tid < 608) {
        const bool bias = tid >= 576;
        const int co = bias ? tid - 576 : tid / 18, t = (tid % 18) / 2, c = tid & 1;
        const int ky = t / 3, kx = t % 3, ck = co >> 3, e = (co & 7) >> 1, hi = co & 1;
        float s = 0.0f;
        for (int i = 0; i < 256; ++i) {
            const uint4 u = gs[i * 4 + ck];
            const uint32_t uu = e == 0 ? u.x : (e == 1 ? u.y : (e == 2 ? u.z : u.w));
            const float gv = hi ? tc::bf16_hi(uu) : tc::bf16_lo(uu);
            s = bias ? s + gv : fmaf(gv, zs[c][(i / 16 + ky) * 18 + (i % 16) + kx], s);
        }
        part[blk * 608 + tid] = s;
    }
}

// out[j] = sum_p part[p * stride + off + j] for j < len (fixed order).
__global__ void k_sum_partials(const float *part, int nparts, int stride, int off, int len, float *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float s = 0.0f;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * stride + off + j];
    out[j] = s;
}

// dL/dout of the L1 loss of Eq. 2: dr = 255 sign(out - clean) / count; loss += sum |out - clean|.
__global__ void k_l1_grad_out(const float *out, const float *clean, float *dr, size_t count, double *loss)
{
    __shared__ double red[8];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < count) {
        const float d = out[i] - clean[i];
        dr[i] = d > 0.0f ? 255.0f / (float)count : (d < 0.0f ? -255.0f / (float)count : 0.0f);
        e = fabs((double)d);
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        atomicAdd(loss, t);
    }
}

struct TrainWs {
    char *act;        // [layers - 1][N][H][W][32] bf16
    char *G[2];       // [N][H][W][32] bf16
    char *wpf, *wpb;  // packed forward / flipped weights of the hidden layers
    float *out, *dr;  // [N][H][W]
    float *partw;     // weight-gradient partials of the tcgen05 kernel
    float *partb;     // bias partials
    float *parts;     // first / last layer partials
    size_t bytes;
};

int bw_grid() { return 152 * kBwCtasPerSm; }

TrainWs train_layout(void *base, int N, int H, int W, int layers)
{
    Carver cv(base);
    TrainWs w;
    const size_t px = (size_t)N * H * W, act = px * 64;
    w.act = cv.take<char>(act * (layers - 1));
    w.G[0] = cv.take<char>(act);
    w.G[1] = cv.take<char>(act);
    const size_t wp = (size_t)9 * 32 * 32 * 2;
    w.wpf = cv.take<char>(wp * (layers - 2));
    w.wpb = cv.take<char>(wp * (layers - 2));
    w.out = cv.take<float>(px);
    w.dr = cv.take<float>(px);
    w.partw = cv.take<float>((size_t)bw_grid() * kPartW);
    w.partb = cv.take<float>((px + 255) / 256 * 32);
    const size_t tiles = (size_t)N * ((H + 15) / 16) * ((W + 15) / 16);
    w.parts = cv.take<float>(tiles * 608);
    w.bytes = cv.off;
    return w;
}

}  // namespace

size_t conv_bwd_w_tc_workspace_bytes(int N, int H, int W)
{
    const size_t px = (size_t)N * H * W;
    return align256((size_t)bw_grid() * kPartW * sizeof(float)) + align256((px + 255) / 256 * 32 * sizeof(float));
}

dn_status conv_bwd_w_tc(const void *x, const void *g, float *dw, float *db, int N, int H, int W, void *ws, int *err,
                        cudaStream_t s)
{
    Carver cv(ws);
    const size_t px = (size_t)N * H * W;
    float *partw = cv.take<float>((size_t)bw_grid() * kPartW);
    float *partb = cv.take<float>((px + 255) / 256 * 32);
    BwArgs b;
    b.x = static_cast<const uint4 *>(x);
    b.g = static_cast<const uint4 *>(g);
    b.N = N;
    b.H = H;
    b.W = W;
    b.strips = (W + kBwPX - 1) / kBwPX;
    b.groups = (H + kBwR - 1) / kBwR;
    b.err = err;
    b.partial = partw;
    const long items = (long)N * b.strips * b.groups;
    const int grid = (int)(items < bw_grid() ? items : bw_grid());
    if (cudaFuncSetAttribute(k_conv_bwd_w_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwSmem) != cudaSuccess)
        return DN_ECUDA;
    const int nbp = (int)((px + 255) / 256);
    DN_TRY(launch("conv3x3_bwd_weight_tc", s, [&] { k_conv_bwd_w_tc<<<grid, 128, kBwSmem, s>>>(b); }));
    DN_TRY(launch("bias_grad_nhwc", s, [&] { k_bias_grad_nhwc<<<nbp, 256, 0, s>>>(b.g, px, partb); }));
    return launch("reduce_dw_tc", s, [&] {
        k_reduce_dw_tc<<<(32 * 9 * 32 + 32 + 255) / 256, 256, 0, s>>>(partw, grid, partb, nbp, dw, db);
    });
}

size_t cnn_grad_tc_workspace_bytes(int N, int H, int W, int layers)
{
    return train_layout(nullptr, N, H, W, layers).bytes;
}

dn_status cnn_grad_tc(const float *noisy, const float *pre, const float *clean, int N, int H, int W, int layers,
                      const float *weights, float *grad, double *loss, void *ws, int *err, cudaStream_t s)
{
    constexpr int C = 32;
    TrainWs w = train_layout(ws, N, H, W, layers);
    const size_t px = (size_t)N * H * W, actb = px * 64;
    auto act = [&](int l) { return w.act + actb * l; };  // output of layer l (0 .. layers - 2)
    // parameter offsets: layer 0 (2 -> C), hidden (C -> C), last (C -> 1)
    const size_t s0 = (size_t)C * 9 * 2 + C, sh = (size_t)C * 9 * C + C;
    auto woff = [&](int l) { return l == 0 ? (size_t)0 : s0 + sh * (l - 1); };
    // forward, keeping every activation
    DN_TRY(conv_first_bf16(pre, noisy, weights, weights + C * 9 * 2, act(0), N, 1, H, W, C, s));
    const size_t wp = (size_t)9 * C * C * 2;
    for (int l = 1; l < layers - 1; ++l) {
        const float *wl = weights + woff(l);
        DN_TRY(pack_w_tc(wl, w.wpf + wp * (l - 1), C, s));
        DN_TRY(pack_w_tc(wl, w.wpb + wp * (l - 1), C, s, true));
        DN_TRY(conv3x3_tc(act(l - 1), act(l), w.wpf + wp * (l - 1), wl + (size_t)C * 9 * C, N, H, W, C, 1, err, s));
    }
    const float *wlast = weights + woff(layers - 1);
    DN_TRY(conv_last_bf16(act(layers - 2), wlast, wlast + 9 * C, pre, w.out, N, 1, H, W, C, s));
    // loss gradient
    DN_TRY(launch("l1_grad_out", s, [&] {
        k_l1_grad_out<<<(unsigned)((px + 255) / 256), 256, 0, s>>>(w.out, clean, w.dr, px, loss);
    }));
    // last layer
    const dim3 tg((W + 15) / 16, (H + 15) / 16, N);
    const int ntiles = (int)(tg.x * tg.y * tg.z);
    float *glast = grad + woff(layers - 1);
    DN_TRY(launch("cnn_last_bwd_w", s, [&] {
        k_last_bwd_w<<<tg, 320, 0, s>>>(w.dr, static_cast<const uint4 *>((const void *)act(layers - 2)), w.parts, H, W);
    }));
    DN_TRY(launch("sum_partials", s, [&] {
        k_sum_partials<<<2, 256, 0, s>>>(w.parts, ntiles, 289, 0, 289, glast);
    }));
    int cur = 0;
    DN_TRY(launch("cnn_last_bwd_data", s, [&] {
        k_last_bwd_data<<<(unsigned)((px + 255) / 256), 256, 0, s>>>(
            w.dr, static_cast<const uint4 *>((const void *)act(layers - 2)), wlast,
            reinterpret_cast<uint4 *>(w.G[cur]), H, W, px);
    }));
    // hidden layers, last to first
    BwArgs b;
    b.N = N;
    b.H = H;
    b.W = W;
    b.strips = (W + kBwPX - 1) / kBwPX;
    b.groups = (H + kBwR - 1) / kBwR;
    b.err = err;
    b.partial = w.partw;
    const long items = (long)N * b.strips * b.groups;
    const int grid = (int)(items < bw_grid() ? items : bw_grid());
    if (cudaFuncSetAttribute(k_conv_bwd_w_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwSmem) != cudaSuccess)
        return DN_ECUDA;
    const int nbp = (int)((px + 255) / 256);
    for (int l = layers - 2; l >= 1; --l) {
        float *gl = grad + woff(l);
        b.x = static_cast<const uint4 *>((const void *)act(l - 1));
        b.g = static_cast<const uint4 *>((const void *)w.G[cur]);
        DN_TRY(launch("conv3x3_bwd_weight_tc", s, [&] { k_conv_bwd_w_tc<<<grid, 128, kBwSmem, s>>>(b); }));
        DN_TRY(launch("bias_grad_nhwc", s, [&] {
            k_bias_grad_nhwc<<<nbp, 256, 0, s>>>(b.g, px, w.partb);
        }));
        DN_TRY(launch("reduce_dw_tc", s, [&] {
            k_reduce_dw_tc<<<(32 * 9 * 32 + 32 + 255) / 256, 256, 0, s>>>(w.partw, grid, w.partb, nbp, gl,
                                                                       gl + (size_t)C * 9 * C);
        }));
        // data gradient through the flipped weights, masked by this layer's input ReLU
        DN_TRY(conv3x3_tc(w.G[cur], w.G[cur ^ 1], w.wpb + wp * (l - 1), nullptr, N, H, W, C, 0, err, s, act(l - 1)));
        cur ^= 1;
    }
    // first layer (weights only: the input needs no gradient)
    DN_TRY(launch("cnn_first_bwd_w", s, [&] {
        k_first_bwd_w<<<tg, 608, 0, s>>>(pre, noisy, reinterpret_cast<const uint4 *>(w.G[cur]), w.parts, H, W);
    }));
    return launch("sum_partials", s, [&] {
        k_sum_partials<<<3, 256, 0, s>>>(w.parts, ntiles, 608, 0, 608, grad);
    });
}

}  // namespace dn

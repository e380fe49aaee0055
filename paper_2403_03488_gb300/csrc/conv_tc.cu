// Residual CNN forward in BF16 on the 5th-generation tensor cores (sm_103a).
//
// Network of Sec. II (Fig. 1, Eq. 2-3): z = [pre/255, noisy/255];
// layer 1 (2 -> 32) and the last layer (32 -> 1, plus out = pre + 255 r) are
// thin and run on CUDA cores; every 32 -> 32 hidden layer is an implicit GEMM
// on tcgen05: M = 128 output pixels (one row segment), N = 32 output channels,
// K = 9 taps x 32 input channels, FP32 accumulation in TMEM, BF16 activations
// in HBM (NHWC, 64 bytes per pixel).
//
// Hidden-layer kernel: a CTA owns a 128-pixel column strip and a run of rows.
// It keeps the packed weights (18 KB) and a ring of three staged input rows
// (130 pixels incl. halo) in shared memory in the K-major core-matrix layout
// [channel chunk of 8][pixel][8 channels], so the A operand of tap (dy, dx) is
// the staged row y+dy-1 shifted by dx pixels: a descriptor offset, no im2col.
// Per output row one thread issues 18 MMAs (9 taps x 2 K-steps of 16), commits
// them to an mbarrier, and all 128 threads (thread = pixel = TMEM lane) read
// the 32 accumulators back, add the bias, apply ReLU and store 64 B of BF16.
// Each input row is read from HBM once per strip.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kPX = 128;                  // output pixels per row tile (MMA M)
constexpr int kP = 130;                   // staged pixels per input row (P = 2 mod 8: conflict-free chunk planes)
constexpr int kCh = 32;                   // hidden channels
constexpr int kRowBytes = kP * kCh * 2;   // 8320
constexpr int kWBytes = 9 * 4 * kCh * 16; // 18432: [tap][chunk][cout][8 ch] bf16
constexpr uint32_t kIdesc = tc::idesc_bf16(128, 32);

struct ConvTcArgs {
    const uint4 *x;       // [N][H][W][32] bf16, 4 x uint4 per pixel
    uint4 *y;             // same layout
    const uint4 *wpack;   // kWBytes
    const float *bias;    // [32]
    int H, W, rows_per_cta, relu;
    int *err;
};

__device__ __forceinline__ void stage_row(const ConvTcArgs &a, uint8_t *slot, int n, int r, int x0, int tid)
{
    for (int i = tid; i < kP * 4; i += 128) {
        const int px = i >> 2, ck = i & 3;
        const int gx = x0 - 1 + px;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r >= 0 && r < a.H && gx >= 0 && gx < a.W) v = a.x[(((size_t)n * a.H + r) * a.W + gx) * 4 + ck];
        *reinterpret_cast<uint4 *>(slot + ck * kP * 16 + px * 16) = v;
    }
}

__global__ void __launch_bounds__(128) k_conv3x3_tc(ConvTcArgs a)
{
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *wsm = sm;
    uint8_t *rows = sm + kWBytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(rows + 3 * kRowBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    float *sbias = reinterpret_cast<float *>(tslot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kPX, n = blockIdx.z;
    const int y_begin = blockIdx.y * a.rows_per_cta;
    const int y_end = min(a.H, y_begin + a.rows_per_cta);
    if (y_begin >= a.H) return;

    for (int i = tid; i < kWBytes / 16; i += 128) reinterpret_cast<uint4 *>(wsm)[i] = a.wpack[i];
    if (tid < kCh) sbias[tid] = a.bias[tid];
    if (warp == 0) tc::tmem_alloc(tslot, 32);
    if (tid == 0) tc::mbar_init(mbar, 1);
    stage_row(a, rows + ((y_begin + 2) % 3) * kRowBytes, n, y_begin - 1, x0, tid);
    stage_row(a, rows + (y_begin % 3) * kRowBytes, n, y_begin, x0, tid);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t wbase = tc::smem_u32(wsm);
    uint32_t phase = 0;
    bool failed = false;

    for (int y = y_begin; y < y_end; ++y) {
        stage_row(a, rows + ((y + 1) % 3) * kRowBytes, n, y + 1, x0, tid);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3, dx = t % 3;
                const uint32_t rb = tc::smem_u32(rows + ((y + 2 + dy) % 3) * kRowBytes);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint64_t ad = tc::sdesc(rb + (2 * k) * kP * 16 + dx * 16, kP * 16, 128);
                    const uint64_t bd = tc::sdesc(wbase + ((t * 4 + 2 * k) * kCh) * 16, kCh * 16, 128);
                    tc::mma_bf16(tmem, ad, bd, kIdesc, (t | k) != 0);
                }
            }
            tc::mma_commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, phase);
        if (__syncthreads_or(!ok)) {  // block-uniform decision
            failed = true;
            if (tid == 0) atomicExch(a.err, 1);
            break;
        }
        phase ^= 1;
        tc::fence_after_sync();
        uint32_t r[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), r);
        tc::tmem_wait_ld();
        const int x = x0 + warp * 32 + lane;
        if (x < a.W) {
            uint32_t pk[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float v0 = __uint_as_float(r[2 * c]) + sbias[2 * c];
                float v1 = __uint_as_float(r[2 * c + 1]) + sbias[2 * c + 1];
                if (a.relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                pk[c] = tc::pack_bf16x2(v0, v1);
            }
            uint4 *dst = a.y + (((size_t)n * a.H + y) * a.W + x) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
        tc::fence_before_sync();
    }
    if (failed) {
        // bounded second wait for MMAs still in flight before the TMEM is freed
        tc::mbar_wait(mbar, phase);
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 32);
    }
}

// W [32][3][3][32] fp32 -> [tap][chunk][cout][8 ch] bf16 (the B operand layout).
__global__ void k_pack_w_tc(const float *w, uint16_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * 4 * kCh * 8) return;
    const int j = i & 7, co = (i >> 3) & 31, ck = (i >> 8) & 3, t = i >> 10;
    const float v = w[(co * 9 + t) * kCh + ck * 8 + j];
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    out[i] = *reinterpret_cast<uint16_t *>(&b);
}

// Layer 1 (2 -> 32) + bias + ReLU: pre/noisy planes (0..255) -> NHWC bf16.
__global__ void __launch_bounds__(256) k_conv_first_bf16(const float *pre, const float *noisy, const float *w,
                                                        const float *b, uint4 *y, int H, int W)
{
    __shared__ float zs[2][18][18];
    __shared__ float ws[kCh * 18];
    __shared__ float bs[kCh];
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < kCh * 18; i += 256) ws[i] = w[i];
    if (threadIdx.x < kCh) bs[threadIdx.x] = b[threadIdx.x];
    for (int i = threadIdx.x; i < 2 * 324; i += 256) {
        const int c = i / 324, p = i % 324, yy = p / 18, xx = p % 18;
        const int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        const float *src = c == 0 ? pre : noisy;
        zs[c][yy][xx] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? src[n * HW + (size_t)gy * W + gx] * (1.0f / 255.0f)
                                                                  : 0.0f;
    }
    __syncthreads();
    const int px = X0 + tx, py = Y0 + ty;
    if (px >= W || py >= H) return;
    float v[18];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        v[2 * t] = zs[0][ty + t / 3][tx + t % 3];
        v[2 * t + 1] = zs[1][ty + t / 3][tx + t % 3];
    }
    uint32_t pk[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        float a0 = bs[2 * c], a1 = bs[2 * c + 1];
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            a0 = fmaf(ws[(2 * c) * 18 + k], v[k], a0);
            a1 = fmaf(ws[(2 * c + 1) * 18 + k], v[k], a1);
        }
        pk[c] = tc::pack_bf16x2(fmaxf(a0, 0.0f), fmaxf(a1, 0.0f));
    }
    uint4 *dst = y + ((size_t)n * HW + (size_t)py * W + px) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
}

// Last layer (32 -> 1) + bias, then out = pre + 255 r (Eq. 2).
__global__ void __launch_bounds__(256) k_conv_last_bf16(const uint4 *x, const float *w, const float *b,
                                                       const float *pre, float *out, int H, int W)
{
    __shared__ uint4 xs[324 * 4];
    __shared__ float ws[9 * kCh];
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < 9 * kCh; i += 256) ws[i] = w[i];
    for (int i = threadIdx.x; i < 324 * 4; i += 256) {
        const int p = i >> 2, ck = i & 3, yy = p / 18, xx = p % 18;
        const int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        xs[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? x[((size_t)n * HW + (size_t)gy * W + gx) * 4 + ck]
                                                         : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int px = X0 + tx, py = Y0 + ty;
    if (px >= W || py >= H) return;
    float acc = b[0];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int p = (ty + t / 3) * 18 + tx + t % 3;
#pragma unroll
        for (int ck = 0; ck < 4; ++ck) {
            const uint4 q = xs[p * 4 + ck];
            const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                acc = fmaf(ws[t * kCh + ck * 8 + 2 * e], tc::bf16_lo(u[e]), acc);
                acc = fmaf(ws[t * kCh + ck * 8 + 2 * e + 1], tc::bf16_hi(u[e]), acc);
            }
        }
    }
    const size_t at = n * HW + (size_t)py * W + px;
    out[at] = fmaf(255.0f, acc, pre[at]);
}

}  // namespace

size_t conv_tc_smem_bytes() { return kWBytes + 3 * kRowBytes + 64 + kCh * 4; }

dn_status pack_w_tc(const float *w, void *out, cudaStream_t s)
{
    return launch("pack_w_tc", s, [&] { k_pack_w_tc<<<(9 * 4 * kCh * 8 + 255) / 256, 256, 0, s>>>(w, (uint16_t *)out); });
}

dn_status conv3x3_tc(const void *x, void *y, const void *wpack, const float *bias, int N, int H, int W, int relu,
                     int *err, cudaStream_t s)
{
    ConvTcArgs a;
    a.x = static_cast<const uint4 *>(x);
    a.y = static_cast<uint4 *>(y);
    a.wpack = static_cast<const uint4 *>(wpack);
    a.bias = bias;
    a.H = H;
    a.W = W;
    a.relu = relu;
    a.err = err;
    const int strips = (W + kPX - 1) / kPX;
    const long target = 152L * 10;
    long chunks = (target + (long)strips * N - 1) / ((long)strips * N);
    if (chunks < 1) chunks = 1;
    int rows = (int)((H + chunks - 1) / chunks);
    if (rows < 4) rows = 4;
    a.rows_per_cta = rows;
    dim3 grid(strips, (H + rows - 1) / rows, N);
    const size_t smem = conv_tc_smem_bytes();
    if (cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    return launch("conv3x3_tc_bf16", s, [&] { k_conv3x3_tc<<<grid, 128, smem, s>>>(a); });
}

dn_status conv_first_bf16(const float *pre, const float *noisy, const float *w, const float *b, void *y, int N,
                          int H, int W, cudaStream_t s)
{
    dim3 grid((W + 15) / 16, (H + 15) / 16, N);
    return launch("conv_first_bf16", s,
                  [&] { k_conv_first_bf16<<<grid, 256, 0, s>>>(pre, noisy, w, b, static_cast<uint4 *>(y), H, W); });
}

dn_status conv_last_bf16(const void *x, const float *w, const float *b, const float *pre, float *out, int N, int H,
                         int W, cudaStream_t s)
{
    dim3 grid((W + 15) / 16, (H + 15) / 16, N);
    return launch("conv_last_bf16", s, [&] {
        k_conv_last_bf16<<<grid, 256, 0, s>>>(static_cast<const uint4 *>(x), w, b, pre, out, H, W);
    });
}

}  // namespace dn

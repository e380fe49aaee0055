// Residual CNN forward in BF16 on the 5th-generation tensor cores (sm_103a).
//
// Network of Sec. II (Fig. 1, Eq. 2-3): z = [pre/255, noisy/255] (cc planes
// each: cc = 1 for the grey network, 3 for a colour-native one); layer 1
// (2 cc -> C) and the last layer (C -> cc, plus out = pre + 255 r) are thin and
// run on CUDA cores; every C -> C hidden layer (C = 32 or 64) is an implicit
// GEMM on tcgen05: M = 128 output pixels (one row segment), N = C output
// channels, K = 9 taps x C input channels, FP32 accumulation in TMEM, BF16
// activations in HBM (NHWC, 2 C bytes per pixel).
//
// Hidden-layer kernel: persistent CTAs take work items of 32 output rows of
// a 128-pixel column strip.  Packed weights (18 KB at C = 32, 72 KB at 64)
// stay in shared memory; input rows (130 pixels incl. halo) are staged in a
// ring of 6 slots in the K-major core-matrix layout [channel chunk of 8]
// [pixel][8 channels], so the A operand of tap (dy, dx) is the staged row
// y+dy-1 shifted by dx pixels: a descriptor offset, no im2col.  Rows are
// fetched with cp.async three rows ahead of use; per output row one thread
// issues 9 C / 16 MMAs (9 taps x C/16 K-steps of 16) into one of two TMEM
// accumulator buffers and commits them to that buffer's mbarrier, and while
// the tensor cores work on row y all 128 threads (thread = pixel = TMEM lane)
// drain row y-1: read C accumulators, add the bias, apply ReLU and store 2 C
// bytes of BF16.  Each input row is read from HBM once per strip and item
// (plus 2 halo rows per 32).
#include <cuda_bf16.h>

#include "common.cuh"
#include "f32x2.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kPX = 128;                  // output pixels per row tile (MMA M)
constexpr int kP = 130;                   // staged pixels per input row (P = 2 mod 8: conflict-free chunk planes)
constexpr int kCh = 32;                   // channels of the default (10 x 32) network
constexpr int kPF = 1;                    // rows in flight beyond the next one
constexpr int kSlots = kPF + 5;           // rows y-2 (last MMA) .. y+2+kPF
constexpr int kItemRows = 32;             // output rows per work item

// Shapes of a C -> C hidden layer (C = 32 or 64 channels).
template <int C>
struct Shape {
    static constexpr int kChunks = C / 8;                   // 16-byte channel chunks per pixel
    static constexpr int kRowBytes = kP * C * 2;            // one staged row
    static constexpr int kWBytes = 9 * kChunks * C * 16;    // [tap][chunk][cout][8 ch] bf16
    static constexpr int kSmem = kWBytes + kSlots * kRowBytes + 32 + C * 4;
    static constexpr int kCtasPerSm = (227 * 1024) / (kSmem + 1024);
    static constexpr uint32_t kIdesc = tc::idesc_bf16(128, C);
};

struct ConvTcArgs {
    const uint4 *x;       // [N][H][W][C] bf16, C / 8 x uint4 per pixel
    uint4 *y;             // same layout
    const uint4 *wpack;   // Shape<C>::kWBytes
    const float *bias;    // [C], or null (no bias)
    const uint4 *mask;    // null, or [N][H][W][C] bf16: outputs where mask <= 0 are zeroed (ReLU backward)
    int N, H, W, strips, chunks, relu;
    int *err;
};

// Row r of image n, pixels x0-1 .. x0+128, into the chunk planes of a ring
// slot: cp.async for pixels inside the image, zeros elsewhere.
template <int C>
__device__ __forceinline__ void issue_row(const ConvTcArgs &a, uint8_t *slot, int n, int r, int x0, int tid)
{
    constexpr int K = Shape<C>::kChunks;
    const bool rin = r >= 0 && r < a.H;
    const uint4 *src = a.x + ((size_t)n * a.H + (rin ? r : 0)) * a.W * K;
    for (int i = tid; i < kP * K; i += 128) {
        const int px = i / K, ck = i % K;
        const int gx = x0 - 1 + px;
        uint8_t *dst = slot + ck * kP * 16 + px * 16;
        if (rin && gx >= 0 && gx < a.W)
            tc::cp_async16(tc::smem_u32(dst), src + (size_t)gx * K + ck);
        else
            *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int C>
__global__ void __launch_bounds__(128) k_conv3x3_tc(ConvTcArgs a)
{
    using S = Shape<C>;
    constexpr int K = S::kChunks;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *wsm = sm;
    uint8_t *ring = sm + S::kWBytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ring + kSlots * S::kRowBytes);  // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    float *sbias = reinterpret_cast<float *>(tslot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < S::kWBytes / 16; i += 128) reinterpret_cast<uint4 *>(wsm)[i] = a.wpack[i];
    for (int i = tid; i < C; i += 128) sbias[i] = a.bias ? a.bias[i] : 0.0f;
    if (warp == 0) tc::tmem_alloc(tslot, 2 * C);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t wbase = tc::smem_u32(wsm);
    uint32_t phases = 0u;  // bit b: parity of the next completion of mbar[b]
    bool failed = false;
    bool fail = false;  // this warp saw a wait time out

    // drains output row yy from TMEM buffer `buf`
    auto epilogue = [&](int n, int x0, int yy, int buf) {
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&mbar[buf], (phases >> buf) & 1u));
        phases ^= 1u << buf;
        if (!ok) {  // warp-uniform: the TMEM load below is a warp-collective
            fail = true;
            return;
        }
        tc::fence_after_sync();
        const int x = x0 + warp * 32 + lane;
        uint4 *dst = a.y + (((size_t)n * a.H + yy) * a.W + x) * K;
#pragma unroll
        for (int h = 0; h < C / 32; ++h) {
            uint32_t r[32];
            tc::tmem_ld32(tmem + (uint32_t)(C * buf + 32 * h) + ((uint32_t)(warp * 32) << 16), r);
            tc::tmem_wait_ld();
            if (x < a.W) {
                uint32_t mk[16];
                if (a.mask) {
                    const uint4 *ms = a.mask + (((size_t)n * a.H + yy) * a.W + x) * K + 4 * h;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 u = ms[q];
                        mk[4 * q] = u.x;
                        mk[4 * q + 1] = u.y;
                        mk[4 * q + 2] = u.z;
                        mk[4 * q + 3] = u.w;
                    }
                }
                uint32_t pk[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float v0 = __uint_as_float(r[2 * c]) + sbias[32 * h + 2 * c];
                    float v1 = __uint_as_float(r[2 * c + 1]) + sbias[32 * h + 2 * c + 1];
                    if (a.relu) {
                        v0 = fmaxf(v0, 0.0f);
                        v1 = fmaxf(v1, 0.0f);
                    }
                    if (a.mask) {  // the layer input's ReLU: pass the gradient where it was positive
                        v0 = tc::bf16_lo(mk[c]) > 0.0f ? v0 : 0.0f;
                        v1 = tc::bf16_hi(mk[c]) > 0.0f ? v1 : 0.0f;
                    }
                    pk[c] = tc::pack_bf16x2(v0, v1);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[4 * h + q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
        }
        tc::fence_before_sync();
    };

    const int items = a.N * a.strips * a.chunks;
    for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const int chunk = it % a.chunks, rest = it / a.chunks;
        const int strip = rest % a.strips, n = rest / a.strips;
        const int x0 = strip * kPX, y0 = chunk * kItemRows, y1 = min(a.H, y0 + kItemRows);
        auto slot = [&](int r) { return ring + ((r - y0 + 1) % kSlots) * S::kRowBytes; };
        for (int r = y0 - 1; r <= y0 + 1 + kPF; ++r) {
            if (r <= y1) issue_row<C>(a, slot(r), n, r, x0, tid);
            tc::cp_async_commit();
        }
        for (int y = y0; y < y1; ++y) {
            const int rn = y + 2 + kPF;
            if (rn <= y1) issue_row<C>(a, slot(rn), n, rn, x0, tid);
            tc::cp_async_commit();
            tc::cp_async_wait<kPF + 1>();  // rows up to y + 1 have landed (this thread's copies)
            tc::fence_proxy_async();
            tc::fence_before_sync();
            if (__syncthreads_or(fail)) {  // block-uniform
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const int buf = (y - y0) & 1;
            if (tid == 0) {
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const int dy = t / 3, dx = t % 3;
                    const uint32_t rb = tc::smem_u32(slot(y - 1 + dy));
#pragma unroll
                    for (int k = 0; k < C / 16; ++k) {
                        const uint64_t ad = tc::sdesc(rb + (2 * k) * kP * 16 + dx * 16, kP * 16, 128);
                        const uint64_t bd = tc::sdesc(wbase + ((t * K + 2 * k) * C) * 16, C * 16, 128);
                        tc::mma_bf16(tmem + (uint32_t)(C * buf), ad, bd, S::kIdesc, (t | k) != 0);
                    }
                }
                tc::mma_commit(&mbar[buf]);
            }
            if (y > y0) epilogue(n, x0, y - 1, buf ^ 1);
        }
        if (!failed) epilogue(n, x0, y1 - 1, (y1 - 1 - y0) & 1);
        tc::cp_async_wait<0>();
        if (__syncthreads_or(fail)) failed = true;
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        // bounded waits for MMAs still in flight before the TMEM is freed
        tc::mbar_wait(&mbar[0], phases & 1u);
        tc::mbar_wait(&mbar[1], (phases >> 1) & 1u);
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 2 * C);
    }
}

// Two hidden C -> C layers (A then B, bias + ReLU each) in one pass: layer A's
// output rows never leave shared memory.  A work item is 32 output rows of a
// strip of kPX - 2 = 126 output pixels: layer A computes 128 pixels (the strip
// plus one on each side, the halo layer B needs) into a ring of kMid rows in
// the operand layout (zero outside the image: layer B's zero padding), and
// layer B reads them like staged input rows.  Layer B runs three rows behind
// layer A, so at every step both layers' MMAs depend only on rows finished in
// earlier steps.  Warp 4 issues them (one thread, descriptors advanced from
// precomputed bases) into one of two TMEM buffer pairs as soon as the 128
// loader / epilogue threads signal on an mbarrier that the step's rows are
// staged; those threads then drain the previous step's two results (A into
// the ring, B to global memory) while the tensor cores work.  Two CTAs per
// SM (measured: one CTA with two more rows of prefetch took 1.76 ms per
// 16 x 1024^2 pair against 1.01 ms).
constexpr int kMid = 4;          // ring rows of layer A's output
constexpr int kPairPF = 0;       // input rows in flight beyond the next one (two CTAs per SM)
constexpr int kPairSlots = kPairPF + 5;
constexpr int kPairOut = kPX - 2;  // output pixels per strip

template <int C>
struct PairShape {
    static constexpr int kChunks = C / 8;
    static constexpr int kRowBytes = kP * C * 2;
    static constexpr int kWBytes = 9 * kChunks * C * 16;
    static constexpr int kSmem = 2 * kWBytes + (kPairSlots + kMid) * kRowBytes + 64 + 2 * C * 4;  // + barriers
    static constexpr int kCtasPerSm = (227 * 1024) / (kSmem + 1024);
    static constexpr uint32_t kIdesc = tc::idesc_bf16(128, C);
};

struct ConvPairArgs {
    const uint4 *x;
    uint4 *y;
    const uint4 *wa, *wb;        // packed weights of layers A and B
    const float *ba, *bb;        // biases
    int N, H, W, strips, chunks;
    int *err;
};

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

template <int C>
__global__ void __launch_bounds__(160, 2) k_conv3x3_tc_pair(ConvPairArgs a)
{
    using S = PairShape<C>;
    constexpr int K = S::kChunks;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *wsa = sm, *wsb = sm + S::kWBytes;
    uint8_t *ring = sm + 2 * S::kWBytes;                      // input rows
    uint8_t *mid = ring + kPairSlots * S::kRowBytes;          // layer A rows
    uint64_t *ready = reinterpret_cast<uint64_t *>(mid + kMid * S::kRowBytes);  // [2]: operands of step staged
    uint64_t *done = ready + 2;                                                  // [2]: MMAs of step complete
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    float *sba = reinterpret_cast<float *>(tslot + 4), *sbb = sba + C;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 4;
    for (int i = tid; i < S::kWBytes / 16; i += 160) {
        reinterpret_cast<uint4 *>(wsa)[i] = a.wa[i];
        reinterpret_cast<uint4 *>(wsb)[i] = a.wb[i];
    }
    for (int i = tid; i < C; i += 160) {
        sba[i] = a.ba[i];
        sbb[i] = a.bb[i];
    }
    // ring pixels 128, 129 of layer A's rows are never computed: zero (layer B's garbage lanes only)
    for (int i = tid; i < kMid * K * 2; i += 160) {
        const int slot = i / (K * 2), rem = i % (K * 2), ck = rem >> 1, px = 128 + (rem & 1);
        *reinterpret_cast<uint4 *>(mid + slot * S::kRowBytes + ck * kP * 16 + px * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) tc::tmem_alloc(tslot, 4 * C);  // [buffer 0: A, B][buffer 1: A, B]
    if (tid == 0) {
        tc::mbar_init(&ready[0], 128);
        tc::mbar_init(&ready[1], 128);
        tc::mbar_init(&done[0], 1);
        tc::mbar_init(&done[1], 1);
        *abort_flag = 0;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    volatile int *abort_v = abort_flag;
    // descriptors: the start-address field (bits 0-13, address >> 4) is advanced by offsets
    const uint64_t wa_d = tc::sdesc(tc::smem_u32(wsa), C * 16, 128), wb_d = tc::sdesc(tc::smem_u32(wsb), C * 16, 128);
    const uint64_t ring_d = tc::sdesc(tc::smem_u32(ring), kP * 16, 128), mid_d = tc::sdesc(tc::smem_u32(mid), kP * 16, 128);
    uint32_t g = 0;  // steps so far (all items): buffer g & 1, barrier parity (g >> 1) & 1

    const int items = a.N * a.strips * a.chunks;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        if (*abort_v) break;
        const int chunk = it % a.chunks, rest = it / a.chunks;
        const int strip = rest % a.strips, n = rest / a.strips;
        const int xo = strip * kPairOut;                    // first output pixel of the strip
        const int x0 = xo - 1;                              // layer A's first pixel
        const int y0 = chunk * kItemRows, y1 = min(a.H, y0 + kItemRows);
        // layer A row of step t: y0 - 1 + t (t < tA); layer B row: y0 - 4 + t (in [y0, y1))
        const int tA = y1 - y0 + 2, tEnd = y1 - y0 + 4;
        auto in_idx = [&](int r) { return (r - (y0 - 2)) % kPairSlots; };
        auto mid_idx = [&](int r) { return (r - (y0 - 1)) % kMid; };
        if (mma_warp) {
            if (lane == 0) {
                for (int t = 0; t < tEnd; ++t, ++g) {
                    const int buf = g & 1;
                    if (!tc::mbar_wait(&ready[buf], (g >> 1) & 1u) || *abort_v) {
                        atomicExch(abort_flag, 1);
                        break;
                    }
                    tc::fence_after_sync();
                    const int rA = y0 - 1 + t, rB = y0 - 4 + t;
                    if (t < tA) {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const uint32_t rowo = (uint32_t)(in_idx(rA - 1 + tap / 3) * S::kRowBytes + (tap % 3) * 16);
#pragma unroll
                            for (int k = 0; k < C / 16; ++k)
                                tc::mma_bf16(tmem + (uint32_t)(2 * C * buf),
                                             ring_d + ((rowo + (uint32_t)(2 * k * kP * 16)) >> 4),
                                             wa_d + ((uint32_t)((tap * K + 2 * k) * C * 16) >> 4), S::kIdesc,
                                             (tap | k) != 0);
                        }
                    }
                    if (rB >= y0 && rB < y1) {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const uint32_t rowo = (uint32_t)(mid_idx(rB - 1 + tap / 3) * S::kRowBytes + (tap % 3) * 16);
#pragma unroll
                            for (int k = 0; k < C / 16; ++k)
                                tc::mma_bf16(tmem + (uint32_t)(2 * C * buf + C),
                                             mid_d + ((rowo + (uint32_t)(2 * k * kP * 16)) >> 4),
                                             wb_d + ((uint32_t)((tap * K + 2 * k) * C * 16) >> 4), S::kIdesc,
                                             (tap | k) != 0);
                        }
                    }
                    tc::mma_commit(&done[buf]);
                }
            }
            g = __shfl_sync(0xffffffffu, g, 0);
            continue;
        }
        // loader / epilogue warps (thread = pixel = TMEM lane)
        for (int r = y0 - 2; r <= y0 + kPairPF; ++r) {
            issue_row<C>(ConvTcArgs{a.x, nullptr, nullptr, nullptr, nullptr, a.N, a.H, a.W, 0, 0, 0, nullptr},
                         ring + in_idx(r) * S::kRowBytes, n, r, x0, tid);
            tc::cp_async_commit();
        }
        bool stop = false;
        for (int t = 0; t <= tEnd; ++t, ++g) {
            const int rA = y0 - 1 + t;
            if (t < tEnd) {
                const int rn = rA + 2 + kPairPF;  // input row of step t + 1 + kPairPF
                if (rn <= y1 + 1)
                    issue_row<C>(ConvTcArgs{a.x, nullptr, nullptr, nullptr, nullptr, a.N, a.H, a.W, 0, 0, 0, nullptr},
                                 ring + in_idx(rn) * S::kRowBytes, n, rn, x0, tid);
                tc::cp_async_commit();
                tc::cp_async_wait<kPairPF + 1>();  // this thread's copies of rows up to rA + 1 have landed
                tc::fence_proxy_async();           // ... and its ring writes of earlier steps are visible
                tc::fence_before_sync();
                mbar_arrive_cta(&ready[g & 1]);
            }
            if (t == 0) continue;
            // drain step t - 1 (buffer (g - 1) & 1)
            const uint32_t pg = g - 1;
            const int pb = pg & 1, prA = rA - 1, prB = y0 - 5 + t;
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&done[pb], (pg >> 1) & 1u));
            if (!ok || *abort_v) {
                atomicExch(abort_flag, 1);
                stop = true;
                ++g;
                break;
            }
            tc::fence_after_sync();
            const int m = warp * 32 + lane;
            if (t - 1 < tA) {
                // layer A row prA, pixel x0 + m, into the ring; zero outside the image
                const int x = x0 + m;
                const bool inside = prA >= 0 && prA < a.H && x >= 0 && x < a.W;
                uint8_t *dst = mid + mid_idx(prA) * S::kRowBytes + m * 16;
#pragma unroll
                for (int h = 0; h < C / 32; ++h) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + (uint32_t)(2 * C * pb + 32 * h) + ((uint32_t)(warp * 32) << 16), r);
                    tc::tmem_wait_ld();
                    uint32_t pk[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float v0 = fmaxf(__uint_as_float(r[2 * c]) + sba[32 * h + 2 * c], 0.0f);
                        const float v1 = fmaxf(__uint_as_float(r[2 * c + 1]) + sba[32 * h + 2 * c + 1], 0.0f);
                        pk[c] = inside ? tc::pack_bf16x2(v0, v1) : 0u;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4 *>(dst + (4 * h + q) * kP * 16) =
                            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                }
            }
            if (prB >= y0 && prB < y1) {
                const int x = xo + m;
                uint4 *dst = a.y + (((size_t)n * a.H + prB) * a.W + x) * K;
#pragma unroll
                for (int h = 0; h < C / 32; ++h) {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + (uint32_t)(2 * C * pb + C + 32 * h) + ((uint32_t)(warp * 32) << 16), r);
                    tc::tmem_wait_ld();
                    if (m < kPairOut && x < a.W) {
                        uint32_t pk[16];
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const float v0 = fmaxf(__uint_as_float(r[2 * c]) + sbb[32 * h + 2 * c], 0.0f);
                            const float v1 = fmaxf(__uint_as_float(r[2 * c + 1]) + sbb[32 * h + 2 * c + 1], 0.0f);
                            pk[c] = tc::pack_bf16x2(v0, v1);
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            dst[4 * h + q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                    }
                }
            }
            tc::fence_before_sync();
        }
        // g counted the tEnd + 1 iterations; the MMA warp counted tEnd steps
        g -= 1;
        tc::cp_async_wait<0>();
        if (stop) break;
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    if (*abort_v) {
        if (tid == 0) atomicExch(a.err, 1);
        // bounded waits for MMAs that may still be in flight before the TMEM is freed
        tc::mbar_wait(&done[0], 0);
        tc::mbar_wait(&done[1], 0);
    }
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 4 * C);
    }
}

// W [C][3][3][C] fp32 -> [tap][chunk][cout][8 ch] bf16 (the B operand layout).
// FLIP packs the data-gradient layer instead: output channel i, input channel
// o, tap (ky, kx) takes W[o][2 - ky][2 - kx][i] (the transposed convolution).
template <int C, bool FLIP>
__global__ void k_pack_w_tc(const float *w, uint16_t *out)
{
    constexpr int K = C / 8;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * K * C * 8) return;
    const int j = i & 7, co = (i >> 3) % C, ck = (i / (8 * C)) % K, t = i / (8 * C * K);
    const float v = FLIP ? w[((ck * 8 + j) * 9 + (8 - t)) * C + co] : w[(co * 9 + t) * C + ck * 8 + j];
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    out[i] = *reinterpret_cast<uint16_t *>(&b);
}

// First layer of any other shape (2 cc -> C, cc = 1 or 3 colour planes):
// z = [pre / 255 (cc planes), noisy / 255 (cc planes)], bias, ReLU, NHWC bf16
// out.  One pixel per thread over a 16 x 16 tile; the C accumulators stay in
// registers and the weights, transposed to [tap][cin][C] in shared memory, are
// read as float4 along the output channel (the 2 -> 32 case has its own
// kernel below).
template <int C>
__global__ void __launch_bounds__(256) k_conv_first_any(const float *pre, const float *noisy, const float *w,
                                                       const float *b, uint4 *y, int cc, int H, int W)
{
    extern __shared__ float4 fsm4[];
    const int cin = 2 * cc;
    float *ws = reinterpret_cast<float *>(fsm4);  // [9][cin][C]
    float *zs = ws + 9 * cin * C;                 // [cin][18][18]
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < C * 9 * cin; i += 256) {
        const int co = i / (9 * cin), rest = i - co * 9 * cin;  // w [co][t][ci], rest = t cin + ci
        ws[rest * C + co] = w[i];
    }
    for (int i = threadIdx.x; i < cin * 324; i += 256) {
        const int c = i / 324, p = i - c * 324, yy = p / 18, xx = p - yy * 18;
        const int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        const float *src = c < cc ? pre + ((size_t)n * cc + c) * HW : noisy + ((size_t)n * cc + c - cc) * HW;
        zs[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? src[(size_t)gy * W + gx] * (1.0f / 255.0f) : 0.0f;
    }
    __syncthreads();
    const int px = X0 + tx, py = Y0 + ty;
    if (px >= W || py >= H) return;
    float acc[C];
#pragma unroll
    for (int co = 0; co < C; ++co) acc[co] = b[co];
    for (int t = 0; t < 9; ++t)
        for (int ci = 0; ci < cin; ++ci) {
            const float z = zs[ci * 324 + (ty + t / 3) * 18 + tx + t % 3];
            const float4 *w4 = reinterpret_cast<const float4 *>(ws + (t * cin + ci) * C);
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                const float4 u = w4[q];
                acc[4 * q] = fmaf(u.x, z, acc[4 * q]);
                acc[4 * q + 1] = fmaf(u.y, z, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(u.z, z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(u.w, z, acc[4 * q + 3]);
            }
        }
    uint4 *dst = y + ((size_t)n * HW + (size_t)py * W + px) * (C / 8);
#pragma unroll
    for (int q = 0; q < C / 8; ++q) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            pk[e] = tc::pack_bf16x2(fmaxf(acc[8 * q + 2 * e], 0.0f), fmaxf(acc[8 * q + 2 * e + 1], 0.0f));
        dst[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Last layer of any other shape (C -> cc) + bias, then out = pre + 255 r per
// colour plane (Eq. 2).  One pixel per thread over a 16 x 16 tile; weights
// transposed to [tap][channel][cc] so each input channel feeds all cc outputs.
template <int C>
__global__ void __launch_bounds__(256) k_conv_last_any(const uint4 *x, const float *w, const float *b,
                                                      const float *pre, float *out, int cc, int H, int W)
{
    extern __shared__ uint4 lsm[];
    constexpr int K = C / 8;
    uint4 *xs = lsm;                                        // [324][K]
    float *ws = reinterpret_cast<float *>(xs + 324 * K);    // [9][C][cc]
    const int n = blockIdx.z, X0 = blockIdx.x * 16, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < cc * 9 * C; i += 256) {
        const int co = i / (9 * C), rest = i - co * 9 * C;  // w [co][t][ci], rest = t C + ci
        ws[rest * cc + co] = w[i];
    }
    for (int i = threadIdx.x; i < 324 * K; i += 256) {
        const int p = i / K, ck = i % K, yy = p / 18, xx = p - yy * 18;
        const int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            tc::cp_async16(tc::smem_u32(&xs[i]), x + ((size_t)n * HW + (size_t)gy * W + gx) * K + ck);
        else
            xs[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::cp_async_commit();
    tc::cp_async_wait<0>();
    __syncthreads();
    const int px = X0 + tx, py = Y0 + ty;
    if (px >= W || py >= H) return;
    float acc[3] = {b[0], cc > 1 ? b[1] : 0.0f, cc > 2 ? b[2] : 0.0f};
    for (int t = 0; t < 9; ++t) {
        const int p = (ty + t / 3) * 18 + tx + t % 3;
#pragma unroll
        for (int ck = 0; ck < K; ++ck) {
            const uint4 q = xs[p * K + ck];
            const uint32_t u[4] = {q.x, q.y, q.z, q.w};
            const float *wt = ws + (t * C + ck * 8) * cc;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float lo = tc::bf16_lo(u[e]), hi = tc::bf16_hi(u[e]);
#pragma unroll
                for (int co = 0; co < 3; ++co)
                    if (co < cc) {
                        acc[co] = fmaf(wt[(2 * e) * cc + co], lo, acc[co]);
                        acc[co] = fmaf(wt[(2 * e + 1) * cc + co], hi, acc[co]);
                    }
            }
        }
    }
#pragma unroll
    for (int co = 0; co < 3; ++co)
        if (co < cc) {
            const size_t at = ((size_t)n * cc + co) * HW + (size_t)py * W + px;
            out[at] = fmaf(255.0f, acc[co], pre[at]);
        }
}

// Layer 1 (2 -> 32) + bias + ReLU: pre/noisy planes (0..255) -> NHWC bf16.
// CTA: 32 x 16 output pixels; thread (tx, ty) computes pixels tx and tx + 16
// of row ty (lanes on consecutive pixels), two output channels per packed
// FP32x2 FMA (weights transposed so a channel pair is one 64-bit load).  The
// two planes' window is staged in 16-byte pieces from column X0 - 4 (aligned),
// scalar loads only where a piece crosses the image border or a row is not
// 16-byte aligned (measured per 16 x 1024^2 launch: 0.58 ms, 0.61 with 4-byte
// pieces, 1,224 copies per CTA).
__global__ void __launch_bounds__(256) k_conv_first_bf16(const float *pre, const float *noisy, const float *w,
                                                        const float *b, uint4 *y, int H, int W)
{
    __shared__ __align__(16) float zs[2][18][48];  // columns X0 - 4 .. X0 + 35; row stride 16 (mod 32)
    __shared__ __align__(16) float ws[18][kCh];    // transposed: the weights of one input tap, channel-contiguous
    __shared__ __align__(8) float bs[kCh];
    const int n = blockIdx.z, X0 = blockIdx.x * 32, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < kCh * 18; i += 256) {
        const int c = i / 18, k = i - c * 18;
        ws[k][c] = w[i];
    }
    if (threadIdx.x < kCh) bs[threadIdx.x] = b[threadIdx.x];
    // raw planes (scaled by 1/255 at use), all copies in flight at once
    for (int i = threadIdx.x; i < 2 * 18 * 10; i += 256) {
        const int c = i / 180, rem = i - c * 180, yy = rem / 10, q = rem - yy * 10;
        const int gy = Y0 - 1 + yy, gx0 = X0 - 4 + 4 * q;
        const float *src = (c == 0 ? pre : noisy) + n * HW + (size_t)gy * W + gx0;
        float *dst = &zs[c][yy][4 * q];
        const bool row_in = gy >= 0 && gy < H;
        if (row_in && gx0 >= 0 && gx0 + 3 < W && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            tc::cp_async16(tc::smem_u32(dst), src);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) dst[e] = (row_in && gx0 + e >= 0 && gx0 + e < W) ? src[e] : 0.0f;
        }
    }
    tc::cp_async_commit();
    tc::cp_async_wait<0>();
    __syncthreads();
    const int py = Y0 + ty;
    if (py >= H || X0 + tx >= W) return;
    // the inputs of the thread's two pixels, each broadcast to both lanes of a packed pair
    f2 v0[18], v1[18];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float a = zs[c][ty + t / 3][tx + 3 + t % 3] * (1.0f / 255.0f);
            const float e = zs[c][ty + t / 3][tx + 19 + t % 3] * (1.0f / 255.0f);
            v0[2 * t + c] = f2_pack(a, a);
            v1[2 * t + c] = f2_pack(e, e);
        }
    uint32_t p0[16], p1[16];
    const float4 *w4 = reinterpret_cast<const float4 *>(&ws[0][0]);
    const f2 *b2 = reinterpret_cast<const f2 *>(bs);
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        // channels (2c, 2c+1) and (2c+2, 2c+3) in the lanes of two packed pairs, one
        // 16-byte weight load per tap, same accumulation order as one channel at a time
        f2 a = b2[c], a2 = b2[c + 1], bb = b2[c], bb2 = b2[c + 1];
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 wq = w4[k * (kCh / 4) + c / 2];
            const f2 wk = f2_pack(wq.x, wq.y), wk2 = f2_pack(wq.z, wq.w);
            a = f2_fma(wk, v0[k], a);
            a2 = f2_fma(wk2, v0[k], a2);
            bb = f2_fma(wk, v1[k], bb);
            bb2 = f2_fma(wk2, v1[k], bb2);
        }
        p0[c] = tc::pack_bf16x2(fmaxf(f2_lo(a), 0.0f), fmaxf(f2_hi(a), 0.0f));
        p0[c + 1] = tc::pack_bf16x2(fmaxf(f2_lo(a2), 0.0f), fmaxf(f2_hi(a2), 0.0f));
        p1[c] = tc::pack_bf16x2(fmaxf(f2_lo(bb), 0.0f), fmaxf(f2_hi(bb), 0.0f));
        p1[c + 1] = tc::pack_bf16x2(fmaxf(f2_lo(bb2), 0.0f), fmaxf(f2_hi(bb2), 0.0f));
    }
    uint4 *dst = y + ((size_t)n * HW + (size_t)py * W + X0 + tx) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(p0[4 * q], p0[4 * q + 1], p0[4 * q + 2], p0[4 * q + 3]);
    if (X0 + tx + 16 < W) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            dst[64 + q] = make_uint4(p1[4 * q], p1[4 * q + 1], p1[4 * q + 2], p1[4 * q + 3]);
    }
}

// Last layer (32 -> 1) + bias, then out = pre + 255 r (Eq. 2).  CTA: 32 x 16
// output pixels; thread (tx, ty) computes pixels tx and tx + 16 of row ty.
// Staged pixels are 80 bytes apart (64 B + 16 B pad), so the 8 lanes of each
// 128-bit load phase hit disjoint banks.
constexpr int kLastPS = 5;  // uint4 per staged pixel

__global__ void __launch_bounds__(256) k_conv_last_bf16(const uint4 *x, const float *w, const float *b,
                                                       const float *pre, float *out, int H, int W)
{
    extern __shared__ uint4 xs_dyn[];  // [18 * 34 * kLastPS] pixels, then 9 x 32 weights
    uint4 *xs = xs_dyn;
    float *ws = reinterpret_cast<float *>(xs_dyn + 18 * 34 * kLastPS);
    const int n = blockIdx.z, X0 = blockIdx.x * 32, Y0 = blockIdx.y * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const size_t HW = (size_t)H * W;
    for (int i = threadIdx.x; i < 9 * kCh; i += 256) ws[i] = w[i];
    for (int i = threadIdx.x; i < 18 * 34 * 4; i += 256) {
        const int p = i >> 2, ck = i & 3, yy = p / 34, xx = p - (p / 34) * 34;
        const int gy = Y0 - 1 + yy, gx = X0 - 1 + xx;
        uint4 *dst = &xs[p * kLastPS + ck];
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            tc::cp_async16(tc::smem_u32(dst), x + ((size_t)n * HW + (size_t)gy * W + gx) * 4 + ck);
        else
            *dst = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::cp_async_commit();
    tc::cp_async_wait<0>();
    __syncthreads();
    const int py = Y0 + ty;
    if (py >= H || X0 + tx >= W) return;
    float acc0 = b[0], acc1 = acc0;
    const float4 *w4 = reinterpret_cast<const float4 *>(ws);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int p = (ty + t / 3) * 34 + tx + t % 3;
#pragma unroll
        for (int ck = 0; ck < 4; ++ck) {
            const uint4 q0 = xs[p * kLastPS + ck], q1 = xs[(p + 16) * kLastPS + ck];
            const float4 wa = w4[(t * kCh + ck * 8) / 4], wb = w4[(t * kCh + ck * 8) / 4 + 1];
            const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
            const uint32_t u0[4] = {q0.x, q0.y, q0.z, q0.w}, u1[4] = {q1.x, q1.y, q1.z, q1.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                acc0 = fmaf(wv[2 * e], tc::bf16_lo(u0[e]), acc0);
                acc0 = fmaf(wv[2 * e + 1], tc::bf16_hi(u0[e]), acc0);
                acc1 = fmaf(wv[2 * e], tc::bf16_lo(u1[e]), acc1);
                acc1 = fmaf(wv[2 * e + 1], tc::bf16_hi(u1[e]), acc1);
            }
        }
    }
    const size_t at = n * HW + (size_t)py * W + X0 + tx;
    out[at] = fmaf(255.0f, acc0, pre[at]);
    if (X0 + tx + 16 < W) out[at + 16] = fmaf(255.0f, acc1, pre[at + 16]);
}

}  // namespace

size_t conv_tc_smem_bytes() { return Shape<kCh>::kSmem; }

dn_status pack_w_tc(const float *w, void *out, int C, cudaStream_t s, bool flip)
{
    if (C == 32)
        return launch("pack_w_tc", s, [&] {
            if (flip)
                k_pack_w_tc<32, true><<<(9 * 4 * 32 * 8 + 255) / 256, 256, 0, s>>>(w, (uint16_t *)out);
            else
                k_pack_w_tc<32, false><<<(9 * 4 * 32 * 8 + 255) / 256, 256, 0, s>>>(w, (uint16_t *)out);
        });
    if (C == 64)
        return launch("pack_w_tc", s, [&] {
            if (flip)
                k_pack_w_tc<64, true><<<(9 * 8 * 64 * 8 + 255) / 256, 256, 0, s>>>(w, (uint16_t *)out);
            else
                k_pack_w_tc<64, false><<<(9 * 8 * 64 * 8 + 255) / 256, 256, 0, s>>>(w, (uint16_t *)out);
        });
    return DN_EUNSUPPORTED;
}

template <int C>
dn_status conv3x3_tc_c(ConvTcArgs &a, cudaStream_t s)
{
    using S = Shape<C>;
    const long items = (long)a.N * a.strips * a.chunks;
    const int grid = (int)(items < 152L * S::kCtasPerSm ? items : 152L * S::kCtasPerSm);
    if (cudaFuncSetAttribute(k_conv3x3_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem) != cudaSuccess)
        return DN_ECUDA;
    return launch(C == 32 ? "conv3x3_tc_bf16" : "conv3x3_tc64_bf16", s,
                  [&] { k_conv3x3_tc<C><<<grid, 128, S::kSmem, s>>>(a); });
}

dn_status conv3x3_tc(const void *x, void *y, const void *wpack, const float *bias, int N, int H, int W, int C,
                     int relu, int *err, cudaStream_t s, const void *mask)
{
    ConvTcArgs a;
    a.x = static_cast<const uint4 *>(x);
    a.y = static_cast<uint4 *>(y);
    a.wpack = static_cast<const uint4 *>(wpack);
    a.bias = bias;
    a.mask = static_cast<const uint4 *>(mask);
    a.N = N;
    a.H = H;
    a.W = W;
    a.relu = relu;
    a.err = err;
    a.strips = (W + kPX - 1) / kPX;
    a.chunks = (H + kItemRows - 1) / kItemRows;
    if (C == 32) return conv3x3_tc_c<32>(a, s);
    if (C == 64) return conv3x3_tc_c<64>(a, s);
    return DN_EUNSUPPORTED;
}

template <int C>
dn_status conv3x3_tc_pair_c(ConvPairArgs &a, cudaStream_t s)
{
    using S = PairShape<C>;
    const long items = (long)a.N * a.strips * a.chunks;
    const long cap = 152L * (S::kCtasPerSm > 0 ? S::kCtasPerSm : 1);
    const int grid = (int)(items < cap ? items : cap);
    if (cudaFuncSetAttribute(k_conv3x3_tc_pair<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem) !=
        cudaSuccess)
        return DN_ECUDA;
    return launch("conv3x3_tc_pair_bf16", s, [&] { k_conv3x3_tc_pair<C><<<grid, 160, S::kSmem, s>>>(a); });
}

dn_status conv3x3_tc_pair(const void *x, void *y, const void *wpa, const float *ba, const void *wpb, const float *bb,
                          int N, int H, int W, int C, int *err, cudaStream_t s)
{
    ConvPairArgs a;
    a.x = static_cast<const uint4 *>(x);
    a.y = static_cast<uint4 *>(y);
    a.wa = static_cast<const uint4 *>(wpa);
    a.wb = static_cast<const uint4 *>(wpb);
    a.ba = ba;
    a.bb = bb;
    a.N = N;
    a.H = H;
    a.W = W;
    a.err = err;
    a.strips = (W + kPairOut - 1) / kPairOut;
    a.chunks = (H + kItemRows - 1) / kItemRows;
    if (C == 32) return conv3x3_tc_pair_c<32>(a, s);
    return DN_EUNSUPPORTED;
}

template <int C>
dn_status conv_first_any(const float *pre, const float *noisy, const float *w, const float *b, void *y, int N, int cc,
                         int H, int W, cudaStream_t s)
{
    const int smem = (int)sizeof(float) * (C * 9 * 2 * cc + 2 * cc * 324);
    if (cudaFuncSetAttribute(k_conv_first_any<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return DN_ECUDA;
    dim3 grid((W + 15) / 16, (H + 15) / 16, N);
    return launch("conv_first_bf16", s, [&] {
        k_conv_first_any<C><<<grid, 256, smem, s>>>(pre, noisy, w, b, static_cast<uint4 *>(y), cc, H, W);
    });
}

template <int C>
dn_status conv_last_any(const void *x, const float *w, const float *b, const float *pre, float *out, int N, int cc,
                        int H, int W, cudaStream_t s)
{
    const int smem = 324 * (C / 8) * 16 + (int)sizeof(float) * cc * 9 * C;
    if (cudaFuncSetAttribute(k_conv_last_any<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return DN_ECUDA;
    dim3 grid((W + 15) / 16, (H + 15) / 16, N);
    return launch("conv_last_bf16", s, [&] {
        k_conv_last_any<C><<<grid, 256, smem, s>>>(static_cast<const uint4 *>(x), w, b, pre, out, cc, H, W);
    });
}

dn_status conv_first_bf16(const float *pre, const float *noisy, const float *w, const float *b, void *y, int N,
                          int cc, int H, int W, int C, cudaStream_t s)
{
    if (cc == 1 && C == 32) {
        dim3 grid((W + 31) / 32, (H + 15) / 16, N);
        return launch("conv_first_bf16", s, [&] {
            k_conv_first_bf16<<<grid, 256, 0, s>>>(pre, noisy, w, b, static_cast<uint4 *>(y), H, W);
        });
    }
    if (C == 32) return conv_first_any<32>(pre, noisy, w, b, y, N, cc, H, W, s);
    if (C == 64) return conv_first_any<64>(pre, noisy, w, b, y, N, cc, H, W, s);
    return DN_EUNSUPPORTED;
}

dn_status conv_last_bf16(const void *x, const float *w, const float *b, const float *pre, float *out, int N, int cc,
                         int H, int W, int C, cudaStream_t s)
{
    if (cc == 1 && C == 32) {
        dim3 grid((W + 31) / 32, (H + 15) / 16, N);
        const int smem = 18 * 34 * kLastPS * 16 + 9 * kCh * 4;
        if (cudaFuncSetAttribute(k_conv_last_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return DN_ECUDA;
        return launch("conv_last_bf16", s, [&] {
            k_conv_last_bf16<<<grid, 256, smem, s>>>(static_cast<const uint4 *>(x), w, b, pre, out, H, W);
        });
    }
    if (C == 32) return conv_last_any<32>(x, w, b, pre, out, N, cc, H, W, s);
    if (C == 64) return conv_last_any<64>(x, w, b, pre, out, N, cc, H, W, s);
    return DN_EUNSUPPORTED;
}

}  // namespace dn

// Contractions of the flexible network (Sec. III, "Ours-FL") on the tensor
// cores: BF16 operands, FP32 accumulation in TMEM, FP32 activations in HBM.
//
// One kernel computes, for every image n and pixel p of an input plane,
//   y[n][co][q(p)] = act(sum_ci w(co, ci) x[n][ci][p] + b[co]) (+ skip[n][co][q(p)])
// with w(co, ci) = w[co * sco + ci * sci + woff] and q(p) = p (pointwise
// layer; its data gradient is the same product with the transposed weights),
// or, for the 2 x 2 transposed convolution (stride 2), the taps (a, 0) and
// (a, 1) of one output row parity a in one launch (two launches cover the
// output): q(p) = (2 i + a) (2 W) + 2 j + c for p = i W + j, the two taps'
// results of a pixel stored together as one 8-byte pair.
//
// GEMM per tile of 128 pixels: M = 128 pixels, N = Cout (padded to 16),
// K = Cin (padded to 16).  A = the pixel tile, MN-major: x is NCHW, so 8
// consecutive pixels of one channel (converted from FP32 to BF16 on the way
// into shared memory) are one 16-byte core-matrix row; B = the weights,
// K-major, packed once per CTA.  Persistent CTAs of 8 warps; two A buffers and
// two TMEM accumulators, so that the next tile's load and MMAs overlap this
// tile's epilogue (thread = pixel = TMEM lane, the two warps of a lane quarter
// splitting the output channels; stores coalesced along the pixels).
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kTP = 128;  // pixels per tile (MMA M)

struct PwTcArgs {
    const float *x;      // [N][Cin][HW]
    const float *w;      // w(co, ci) = w[co * sco + ci * sci + woff]
    const float *b;      // [Cout] or null
    const float *skip;   // same layout as y, or null
    float *y;            // [N][Cout][HW] (mode 0) or [N][Cout][4 HW] (mode 1)
    int N, Cin, Cout, HW, Win;
    int sco, sci, woff;
    int mode, a, relu;
    int Kp, Np;          // padded K and N
    int *err;
};

__device__ __forceinline__ void tmem_ld16_cols(uint32_t taddr, uint32_t (&r)[16]) { tc::tmem_ld16(taddr, r); }

// NT = taps per launch: 1 (pointwise) or 2 (transposed convolution, taps (a, 0) and (a, 1)).
template <int NT>
__global__ void __launch_bounds__(256) k_pw_tc(PwTcArgs a)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const int Kp = a.Kp, Np = a.Np;
    const size_t wbytes = (size_t)Np * Kp * 2;
    uint8_t *ws = sm;                                  // NT x [Np / 8][Kp / 8][8][8] bf16 (K-major B)
    uint8_t *as = sm + NT * wbytes;                    // 2 x [Kp / 8][16][8][8] bf16 (MN-major A)
    const size_t abytes = (size_t)kTP * Kp * 2;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(as + 2 * abytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    float *sb = reinterpret_cast<float *>(tslot + 4);  // [Np] bias

    // 8 warps: warps w and w + 4 read TMEM lane quarter w and split its 16-column blocks
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quarter = warp & 3, half = warp >> 2;
    // weights: element (n, k) at ((n / 8) (Kp / 8) + k / 8) 128 + (n % 8) 16 + (k % 8) 2
    for (int i = tid; i < NT * Np * Kp; i += 256) {
        const int tp = i / (Np * Kp), r = i - tp * (Np * Kp), n = r / Kp, k = r - n * Kp;
        const float v =
            (n < a.Cout && k < a.Cin) ? a.w[(size_t)n * a.sco + (size_t)k * a.sci + a.woff + tp] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(ws + tp * wbytes + ((n >> 3) * (Kp >> 3) + (k >> 3)) * 128 + (n & 7) * 16 +
                                           (k & 7) * 2) = h;
    }
    for (int i = tid; i < Np; i += 256) sb[i] = (a.b && i < a.Cout) ? a.b[i] : 0.0f;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(2 * NT * Np)) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, Np) | (1u << 15);  // A MN-major, B K-major
    const uint64_t bdesc0 = tc::sdesc(tc::smem_u32(ws), 128, (Kp >> 3) * 128);
    const int tiles_per = (a.HW + kTP - 1) / kTP;
    const int items = a.N * tiles_per;

    // stage the A tile of item `it` into buffer `buf`
    auto stage = [&](int it, int buf) {
        const int n = it / tiles_per, p0 = (it - n * tiles_per) * kTP;
        uint8_t *dst = as + buf * abytes;
        const float *xn = a.x + (size_t)n * a.Cin * a.HW;
        const bool vec = (a.HW & 3) == 0;
        for (int i = tid; i < Kp * (kTP / 8); i += 256) {
            const int k = i >> 4, g = i & 15, p = p0 + 8 * g;
            float v[8];
            if (k < a.Cin && vec && p + 8 <= a.HW) {
                const float4 *src = reinterpret_cast<const float4 *>(xn + (size_t)k * a.HW + p);
                const float4 u0 = src[0], u1 = src[1];
                v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
                v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = (k < a.Cin && p + e < a.HW) ? xn[(size_t)k * a.HW + p + e] : 0.0f;
            }
            *reinterpret_cast<uint4 *>(dst + ((k >> 3) * 16 + g) * 128 + (k & 7) * 16) =
                make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]), tc::pack_bf16x2(v[4], v[5]),
                           tc::pack_bf16x2(v[6], v[7]));
        }
    };
    auto issue = [&](int buf) {
        const uint32_t ab = tc::smem_u32(as + buf * abytes);
        for (int tp = 0; tp < NT; ++tp)
            for (int ks = 0; ks < Kp / 16; ++ks) {
                const uint64_t ad = tc::sdesc(ab + 2 * ks * 16 * 128, 16 * 128, 128);
                const uint64_t bd = bdesc0 + (uint64_t)((tp * wbytes + 2 * ks * 128) >> 4);
                tc::mma_bf16(tmem + (uint32_t)((buf * NT + tp) * Np), ad, bd, idesc, ks != 0);
            }
        tc::mma_commit(&mbar[buf]);
    };

    uint32_t phases = 0u;
    bool failed = false;
    int it = blockIdx.x, t = 0;
    if (it < items) {
        stage(it, 0);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) issue(0);
    }
    for (; it < items && !failed; it += gridDim.x, ++t) {
        const int buf = t & 1, nxt = it + gridDim.x;
        if (nxt < items) {
            stage(nxt, buf ^ 1);  // the previous user of this buffer was drained last iteration
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) issue(buf ^ 1);
        }
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&mbar[buf], (phases >> buf) & 1u));
        phases ^= 1u << buf;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        const int n = it / tiles_per, p = (it - n * tiles_per) * kTP + quarter * 32 + lane;
        if (NT == 1) {
            for (int c0 = 16 * half; c0 < Np; c0 += 32) {
                uint32_t r[16];
                tmem_ld16_cols(tmem + (uint32_t)(buf * Np + c0) + ((uint32_t)(quarter * 32) << 16), r);
                tc::tmem_wait_ld();
                if (p < a.HW) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int co = c0 + q;
                        if (co < a.Cout) {
                            const size_t at = ((size_t)n * a.Cout + co) * a.HW + p;
                            float v = __uint_as_float(r[q]) + sb[co];
                            if (a.skip) v += a.skip[at];
                            if (a.relu) v = fmaxf(v, 0.0f);
                            a.y[at] = v;
                        }
                    }
                }
            }
        } else {
            // taps (a, 0) and (a, 1): output pixels (2 i + a, 2 j) and (2 i + a, 2 j + 1), one float2
            const int i = p / a.Win, j = p - (p / a.Win) * a.Win;
            const size_t oplane = (size_t)4 * a.HW, opos = (size_t)(2 * i + a.a) * (2 * a.Win) + 2 * j;
            for (int c0 = 16 * half; c0 < Np; c0 += 32) {
                // the skip pairs are loaded first so that their latency overlaps the TMEM loads
                float2 sk[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int co = c0 + q;
                    sk[q] = (a.skip && p < a.HW && co < a.Cout)
                                ? __ldg(reinterpret_cast<const float2 *>(a.skip + ((size_t)n * a.Cout + co) * oplane +
                                                                         opos))
                                : make_float2(0.0f, 0.0f);
                }
                uint32_t r0[16], r1[16];
                tmem_ld16_cols(tmem + (uint32_t)(2 * buf * Np + c0) + ((uint32_t)(quarter * 32) << 16), r0);
                tmem_ld16_cols(tmem + (uint32_t)((2 * buf + 1) * Np + c0) + ((uint32_t)(quarter * 32) << 16), r1);
                tc::tmem_wait_ld();
                if (p < a.HW) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int co = c0 + q;
                        if (co < a.Cout) {
                            const size_t at = ((size_t)n * a.Cout + co) * oplane + opos;
                            const float2 v = make_float2(__uint_as_float(r0[q]) + sb[co] + sk[q].x,
                                                         __uint_as_float(r1[q]) + sb[co] + sk[q].y);
                            __stcs(reinterpret_cast<float2 *>(a.y + at), v);
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();  // both buffers' users are done before the next iteration stages into one
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 5);
        tc::mbar_wait(&mbar[0], phases & 1u);
        tc::mbar_wait(&mbar[1], (phases >> 1) & 1u);
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

template <int NT>
dn_status launch_pw_tc(PwTcArgs &a, cudaStream_t s, const char *name)
{
    a.Kp = (a.Cin + 15) / 16 * 16;
    a.Np = (a.Cout + 15) / 16 * 16;
    if (NT * a.Np > 256 || a.Kp > 256) return DN_EUNSUPPORTED;
    const size_t smem = NT * (size_t)a.Np * a.Kp * 2 + 2 * (size_t)kTP * a.Kp * 2 + 64 + (size_t)a.Np * 4;
    if (smem > 225 * 1024) return DN_EUNSUPPORTED;
    if (cudaFuncSetAttribute(k_pw_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(2 * NT * a.Np)) ncols <<= 1;
    per_sm = per_sm < (int)(512 / ncols) ? per_sm : (int)(512 / ncols);  // TMEM columns per SM
    if (per_sm < 1) per_sm = 1;
    const long items = (long)a.N * ((a.HW + kTP - 1) / kTP);
    const int grid = (int)(items < 152L * per_sm ? items : 152L * per_sm);
    return launch(name, s, [&] { k_pw_tc<NT><<<grid, 256, smem, s>>>(a); });
}

}  // namespace

dn_status pw_fwd_tc(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                    int relu, int transposed, int *err, cudaStream_t s)
{
    PwTcArgs a{};
    a.x = x;
    a.w = w;
    a.b = b;
    a.skip = nullptr;
    a.y = y;
    a.N = N;
    a.Cin = Cin;
    a.Cout = Cout;
    a.HW = HW;
    a.Win = 1;
    a.sco = transposed ? 1 : Cin;     // transposed: w is [Cin][Cout] of the forward layer
    a.sci = transposed ? Cout : 1;
    a.woff = 0;
    a.mode = 0;
    a.relu = relu;
    a.err = err;
    return launch_pw_tc<1>(a, s, "fl_pw_fwd_tc");
}

dn_status deconv2x2_fwd_tc(const float *x, const float *w, const float *b, const float *skip, float *y, int N,
                           int Cin, int Cout, int H, int W, int *err, cudaStream_t s)
{
    for (int ra = 0; ra < 2; ++ra) {
        PwTcArgs a{};
        a.x = x;
        a.w = w;          // [Cin][Cout][2][2]: tap (ra, c) at offset 2 ra + c
        a.b = b;
        a.skip = skip;
        a.y = y;
        a.N = N;
        a.Cin = Cin;
        a.Cout = Cout;
        a.HW = H * W;
        a.Win = W;
        a.sco = 4;
        a.sci = Cout * 4;
        a.woff = 2 * ra;
        a.mode = 1;
        a.a = ra;
        a.relu = 0;
        a.err = err;
        DN_TRY(launch_pw_tc<2>(a, s, "fl_deconv2x2_fwd_tc"));
    }
    return DN_OK;
}

}  // namespace dn

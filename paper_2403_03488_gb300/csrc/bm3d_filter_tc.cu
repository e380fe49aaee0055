// BM3D collaborative filtering with the 2D patch transforms on the tensor
// cores (tcgen05.mma kind::f16: BF16 operands, FP32 accumulation in TMEM).
//
// The method, reference grid, group weights and exact fixed-point
// aggregation are those of the FP32 SIMT kernels (bm3d_filter.cu).  What
// moves to the tensor cores is the separable 2D DCT-II of every patch and its
// inverse, written as dense 64 x 64 contractions with D = C (x) C (C the
// orthonormal 8-point DCT-II, D rounded to BF16):
//   forward  X [64 coef][N patch] = D [64 coef][64 px] P^T   (P: patches, K-major B operand)
//   inverse  G [64 px][N patch]   = D^T [64 px][64 coef] X'  (X': spectra, MN-major B operand)
// The A operand holds D (or D^T) twice (M = 128), so TMEM lanes u and 64 + u
// carry the same coefficient (or pixel) and the two halves of a warpgroup
// work on different patch columns.
//
// Precision: every patch is centred on its own FP32 mean before it is rounded
// to BF16.  The mean is its 2D DC coefficient / 8 and stays in FP32 through
// the group transform (the DC row of D and DC column of D^T are zero; the
// thread of coefficient 0 takes 8 x mean from shared memory instead of TMEM,
// and the filtered DC value is added back to every pixel before
// aggregation), so flat regions and the dominant DC energy never pass through
// BF16.  The AC coefficients carry the BF16 rounding of the centred pixels
// and of the filtered spectra entering the inverse (relative 2^-9 each) and
// of D itself.
//
// The Walsh-Hadamard transform along the group, the hard threshold (N_har) or
// Wiener gains (sum of squared gains) and the group weights run in FP32 on
// the CUDA cores: the forward result has one coefficient per TMEM lane and
// the patches along the columns, so a thread reads one coefficient of a whole
// group into registers and transforms it there, with two patches per packed
// FP32x2 instruction.
//
// Work split: persistent CTAs (one per SM, 16 warps = 4 independent
// warpgroups) over tiles of TR x TR reference positions.  Per tile and
// channel the CTA stages the image window(s) and a shared num window as the
// SIMT kernel does.  Each warpgroup then takes G groups of at most S patches
// at a time (S = 16 or 32; hard pass: G = 128 / S groups, 128 forward MMA
// columns; Wiener pass: G = 64 / S groups, basic patches in columns 0..63 and
// noisy patches in 64..127):
//   1. gather: thread j loads patch j, subtracts its mean, stores 8 rows of
//      8 BF16 (16 B each) into the warpgroup's shared operand buffer;
//   2. one thread issues the forward MMAs (M 128, N 128, K 64) into the
//      warpgroup's 128 TMEM columns and commits them to an mbarrier;
//   3. thread (coefficient u, half h) reads its groups' columns, transforms,
//      thresholds / applies the gains, transforms back and stores the spectra
//      as BF16 into the same buffer, MN-major (16-byte runs of 8 patches);
//   4. the inverse MMAs (N = G S) overwrite the same TMEM columns; thread
//      (pixel p, half h) adds the FP32 DC value back, weights by
//      w_g kai(p) / n and adds the terms to the num window (exact fixed
//      point); thread j adds the group weight to wsum at patch j's position.
#include <cuda_bf16.h>

#include "common.cuh"
#include "f32x2.cuh"
#include "fixed_point.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kWgs = 4;                  // warpgroups per CTA
constexpr int kThreads = 128 * kWgs;
constexpr int kCols = 128;               // forward MMA columns (N) and TMEM columns per warpgroup
constexpr int kOpBytes = 8 * kCols * 16; // one 128 x 64 BF16 operand (16 KB)
constexpr int kLbo = kCols * 16;         // K-adjacent core-matrix distance of the K-major operands

struct WgMeta {
    int woff[kCols];    // num-window offset of patch column j's top-left pixel, -1 outside the window
    int gpos[kCols];    // y W + x of patch column j (inverse column numbering)
    float mean[kCols];  // FP32 mean of the patch in forward column j
    float dcv[kCols];   // filtered DC value / 8 of inverse column j (group transform unnormalised)
    int gn[8];          // group sizes of the current tile, 0 = skipped
    int inall[8];       // 1 when every patch of the group lies inside the num window
    int cnt[8];         // hard: kept coefficients per group
    float wsq[8][2];    // Wiener: sum of squared gains per group, one partial per coefficient half
};

constexpr int kMetaBytes = (sizeof(WgMeta) + 127) / 128 * 128;
constexpr int kFixedBytes = 2 * kOpBytes + kWgs * kOpBytes + kWgs * 2 * kMetaBytes + 128;

struct TcArgs {
    const float *img;    // [b][C][H][W]: image to filter (pass 1) or noisy (pass 2)
    const float *basic;  // pass 2 only
    const int *idx;
    const int *n;
    unsigned long long *num, *wsum, *num_hi, *wsum_hi;
    int *err;
    int C, H, W, R, Rx, Ry, n2, step, hs, nb;
    int TR, RH, RW, RS, tiles_x, tiles_y;
    float lambda;
    WinFmt wf;  // format of the shared num window
    float sig[kChunk * 3];
    float kai[64];
    float dct[64];  // C[u][m] = a_u cos(pi (2m+1) u / 16)
};

template <int N>
__device__ __forceinline__ constexpr float sqrt_of()
{
    return N == 1 ? 1.0f : N == 2 ? 1.41421356237309505f : N == 4 ? 2.0f : N == 8 ? 2.82842712474619010f
         : N == 16 ? 4.0f : 5.65685424949238019f;
}

// Unnormalised Walsh-Hadamard transform (Sylvester order) of v[0..N), two
// butterflies per packed instruction: pack k holds (v[k], v[k + N/2]), the
// stages on the lower index bits run on the packs and the top-bit stage
// inside each pack.  The stages commute, so the result is the natural-order
// transform.
template <int N, int S>
__device__ __forceinline__ void fwht_n(float (&v)[S])
{
    if constexpr (N >= 2) {
        constexpr int M = N / 2;
        f2 p[M];
#pragma unroll
        for (int k = 0; k < M; ++k) p[k] = f2_pack(v[k], v[k + M]);
#pragma unroll
        for (int h = 1; h < M; h <<= 1)
#pragma unroll
            for (int i = 0; i < M; i += 2 * h)
#pragma unroll
                for (int j = i; j < i + h; ++j) {
                    const f2 x = p[j], y = p[j + h];
                    p[j] = f2_add(x, y);
                    p[j + h] = f2_sub(x, y);
                }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const float lo = f2_lo(p[k]), hi = f2_hi(p[k]);
            v[k] = lo + hi;
            v[k + M] = lo - hi;
        }
    }
}

// Hard threshold of one coefficient across a group of N patches: forward
// transform, keep |c| > lambda sigma (on the unnormalised coefficients:
// |c| > lambda sigma sqrt(N)), inverse transform (the factor N is taken out
// at aggregation).  Returns the number of kept coefficients.
template <int N, int S>
__device__ __forceinline__ int hard_n(float (&v)[S], float thr)
{
    fwht_n<N>(v);
    const float t = thr * sqrt_of<N>();
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const bool keep = fabsf(v[k]) > t;
        cnt += keep ? 1 : 0;
        v[k] = keep ? v[k] : 0.0f;
    }
    fwht_n<N>(v);
    return cnt;
}

template <int S>
__device__ __forceinline__ int hard_any(float (&v)[S], int n, float thr)
{
    switch (n) {
        case 1: return hard_n<1>(v, thr);
        case 2: return hard_n<2>(v, thr);
        case 4: return hard_n<4>(v, thr);
        case 8: return hard_n<8>(v, thr);
        case 16: return hard_n<16>(v, thr);
        default:
            if constexpr (S >= 32) return hard_n<32>(v, thr);
            return 0;
    }
}

// Wiener filtering of one coefficient across a group of N patches: gains
// w = B^2 / (B^2 + sigma^2) from the basic-estimate coefficients b (with the
// unnormalised transform: B^2 / (B^2 + N sigma^2)), applied to the noisy
// coefficients y, which are transformed back in place.  Returns sum w^2.
template <int N, int S>
__device__ __forceinline__ float wiener_n(float (&b)[S], float (&y)[S], float s2)
{
    fwht_n<N>(b);
    const float s2n = s2 * (float)N;
    float wsq = 0.0f;
    if constexpr (N == 1) {
        const float b2 = b[0] * b[0];
        b[0] = __fdividef(b2, b2 + s2n);
        wsq = b[0] * b[0];
    } else {
        constexpr int M = N / 2;
        const f2 s2n2 = f2_pack(s2n, s2n);
        f2 acc = f2_pack(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const f2 bb = f2_pack(b[k], b[k + M]);
            const f2 b2 = f2_mul(bb, bb);
            const f2 den = f2_add(b2, s2n2);  // >= sigma^2 N > 0
            const float w0 = __fdividef(f2_lo(b2), f2_lo(den)), w1 = __fdividef(f2_hi(b2), f2_hi(den));
            b[k] = w0;
            b[k + M] = w1;
            const f2 ww = f2_pack(w0, w1);
            acc = f2_fma(ww, ww, acc);
        }
        wsq = f2_lo(acc) + f2_hi(acc);
    }
    fwht_n<N>(y);
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] *= b[k];
    fwht_n<N>(y);
    return wsq;
}

template <int S>
__device__ __forceinline__ float wiener_any(float (&b)[S], float (&y)[S], int n, float s2)
{
    switch (n) {
        case 1: return wiener_n<1>(b, y, s2);
        case 2: return wiener_n<2>(b, y, s2);
        case 4: return wiener_n<4>(b, y, s2);
        case 8: return wiener_n<8>(b, y, s2);
        case 16: return wiener_n<16>(b, y, s2);
        default:
            if constexpr (S >= 32) return wiener_n<32>(b, y, s2);
            return 0.0f;
    }
}

template <int S>
__device__ __forceinline__ void tmem_ld_slot(uint32_t taddr, float (&v)[S])
{
    if constexpr (S == 16) {
        uint32_t r[16];
        tc::tmem_ld16(taddr, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
    } else {
        uint32_t r[32];
        tc::tmem_ld32(taddr, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
    }
}

// Stores coefficient row u of a group's filtered spectra (columns
// [col0, col0 + S), only the first n used) into the MN-major B operand of
// the inverse: element (u, j) at (u / 8) lbo + (j / 8) 128 + (u % 8) 16 + (j % 8) 2.
template <int S>
__device__ __forceinline__ void store_spectra(uint8_t *op, int lbo, int u, int col0, int n, const float (&v)[S],
                                              bool zero)
{
    uint8_t *row = op + (u >> 3) * lbo + (u & 7) * 16;
#pragma unroll
    for (int q = 0; q < S / 8; ++q)
        if (q * 8 < n) {
            uint4 pk = make_uint4(0u, 0u, 0u, 0u);
            if (!zero)
                pk = make_uint4(tc::pack_bf16x2(v[8 * q], v[8 * q + 1]), tc::pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                                tc::pack_bf16x2(v[8 * q + 4], v[8 * q + 5]),
                                tc::pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
            *reinterpret_cast<uint4 *>(row + ((col0 >> 3) + q) * 128) = pk;
        }
}

// Aggregation of one group's N estimates of pixel p (this thread): term
// t_k = (v_k + dc_k) w kai(p) / n scaled by 2^(F - 23), added to the num window as
// exact fixed point (see WinFmt).  The terms are formed first and one warp
// vote picks the branch-free fast path (every term within the window's bound
// and every patch inside the window, the common case) for the whole group.
template <int N, int S>
__device__ __forceinline__ void agg_n(const float (&v)[S], const WgMeta &mt, int j0, float wk, bool inall,
                                      unsigned *wnum, int poffw, const TcArgs &a, size_t poffg)
{
    float t[N];
    if constexpr (N == 1) {
        t[0] = (v[0] + mt.dcv[j0]) * wk;
    } else {
        const f2 wk2 = f2_pack(wk, wk);
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            const float2 dc = *reinterpret_cast<const float2 *>(&mt.dcv[j0 + k]);
            const f2 c = f2_mul(f2_add(f2_pack(v[k], v[k + 1]), f2_pack(dc.x, dc.y)), wk2);
            t[k] = f2_lo(c);
            t[k + 1] = f2_hi(c);
        }
    }
    bool fast = inall;
#pragma unroll
    for (int k = 0; k < N; ++k) fast = fast && fabsf(t[k]) < a.wf.tlim;
    if (__all_sync(0xffffffffu, fast)) {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            int h[2], l[2];
            win_parts2(f2_pack(t[k], N > 1 ? t[k + (N > 1)] : 0.0f), a.wf.s, h, l);
            if constexpr (N > 1) {
                const int2 wo = *reinterpret_cast<const int2 *>(&mt.woff[j0 + k]);
                win_red(wnum + wo.x + poffw, a.RH * a.RS, h[0], l[0]);
                win_red(wnum + wo.y + poffw, a.RH * a.RS, h[1], l[1]);
            } else {
                win_red(wnum + mt.woff[j0] + poffw, a.RH * a.RS, h[0], l[0]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float c = t[k] * (1.0f / a.wf.tscale);  // exact: a power of two
            const int o = mt.woff[j0 + k];
            const size_t gp = poffg + (size_t)mt.gpos[j0 + k];
            if (o >= 0 && fabsf(t[k]) < a.wf.tlim) {
                win_add1(wnum + o + poffw, a.RH * a.RS, t[k], a.wf.s);
            } else {
                const Fix f = to_fixed(c);
                atomicAdd(a.num + gp, f.lo);
                if (f.hi != 0) atomicAdd(a.num_hi + gp, (unsigned long long)f.hi);
            }
        }
    }
}

// Shared-memory layout of one CTA (dynamic, 1024-byte aligned base):
//   [A_fwd 16 KB][A_inv 16 KB][operand buffer per warpgroup][WgMeta per warpgroup]
//   [mbarriers, TMEM address, failure flag (128 B)][num window 2 x RH x RS u32][image window(s) RH x RW f32]
template <bool WIENER, int S>
__global__ void __launch_bounds__(kThreads, 1) k_filter_tc(TcArgs a)
{
    constexpr int G = (WIENER ? 64 : 128) / S;  // groups per warpgroup tile
    constexpr int NI = G * S;                   // inverse MMA columns
    constexpr int kLboI = (NI / 8) * 128;       // K-adjacent distance of the MN-major spectra
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *afwd = sm, *ainv = sm + kOpBytes;
    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, wq = t >> 5, lane = tid & 31;
    uint8_t *op = sm + 2 * kOpBytes + wg * kOpBytes;
    // two metadata buffers per warpgroup, alternating between its tiles, so that
    // a tile's gather may start while slower warps still aggregate the last one
    uint8_t *meta = sm + (2 + kWgs) * kOpBytes + wg * 2 * kMetaBytes;
    uint8_t *ctl = sm + (2 + kWgs) * kOpBytes + kWgs * 2 * kMetaBytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ctl) + 2 * wg;  // [forward, inverse]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(ctl + 64);
    int *sfail = reinterpret_cast<int *>(ctl + 72);
    unsigned *wnum = reinterpret_cast<unsigned *>(sm + kFixedBytes);             // [2][RH][RS] (WinFmt)
    float *simg = reinterpret_cast<float *>(wnum + 2 * (size_t)a.RH * a.RS);  // [1 or 2][RH][RW]
    const float *wbasic = simg + (size_t)a.RH * a.RW;

    // A operands: D (forward, [coef][px]) and D^T (inverse, [px][coef]), each
    // twice along M, K-major: element (m, k) at (k / 8) kLbo + m 16 + (k % 8) 2.
    for (int e = tid; e < 128 * 64; e += kThreads) {
        const int m = e >> 6, k = e & 63, r = m & 63;
        const int u = k, p = r;  // inverse: row = pixel, k = coefficient
        const float vi = u ? a.dct[(u >> 3) * 8 + (p >> 3)] * a.dct[(u & 7) * 8 + (p & 7)] : 0.0f;
        const float vf = r ? a.dct[(r >> 3) * 8 + (k >> 3)] * a.dct[(r & 7) * 8 + (k & 7)] : 0.0f;
        const int off = (k >> 3) * kLbo + m * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(afwd + off) = __float2bfloat16_rn(vf);
        *reinterpret_cast<__nv_bfloat16 *>(ainv + off) = __float2bfloat16_rn(vi);
    }
    if (tid < 32) tc::tmem_alloc(tslot, kWgs * kCols);
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (tid == 0) *sfail = 0;
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot + (uint32_t)(wg * kCols);
    const uint32_t tlane = (uint32_t)(wq * 32) << 16;
    const uint32_t afwd_s = tc::smem_u32(afwd), ainv_s = tc::smem_u32(ainv), op_s = tc::smem_u32(op);
    constexpr uint32_t kIdF = tc::idesc_bf16(128, kCols);
    constexpr uint32_t kIdI = tc::idesc_bf16(128, NI) | (1u << 16);  // B (spectra) MN-major
    const int bar_id = 1 + wg;
    const int u = (wq & 1) * 32 + lane;  // coefficient (step 3) / pixel (step 4) of this thread
    const int half = wq >> 1;            // which groups of the tile this thread's warp works on
    const float kp = a.kai[u];
    const int pi = u >> 3, pj = u & 7;
    uint32_t phase = 0;  // parity of the next completion of both mbarriers
    uint32_t it = 0;     // tiles of this warpgroup so far (selects the metadata buffer)
    bool failed = false, wait_failed = false;
    // this thread's gather column: forward column t, inverse column jc, group g, member k
    const bool second = WIENER && t >= 64;  // noisy half of the Wiener columns
    const int jc = WIENER ? (t & 63) : t;
    const int gcol = jc / S, kcol = jc % S;

    const int tiles = a.nb * a.tiles_y * a.tiles_x;
    const size_t HW = (size_t)a.H * a.W;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int b = tile / (a.tiles_y * a.tiles_x), rest = tile - b * a.tiles_y * a.tiles_x;
        const int rx0 = (rest % a.tiles_x) * a.TR, ry0 = (rest / a.tiles_x) * a.TR;
        const int gx0 = min(rx0 * a.step, a.W - 8), gy0 = min(ry0 * a.step, a.H - 8);
        const int X0 = max(0, gx0 - a.hs), Y0 = max(0, gy0 - a.hs);
        const int tw = min(a.TR, a.Rx - rx0), th = min(a.TR, a.Ry - ry0), cnt = tw * th;
        const int rh = min(a.RH, a.H - Y0), rw = min(a.RW, a.W - X0);
        for (int c = 0; c < a.C; ++c) {
            const size_t cbase = ((size_t)b * a.C + c) * HW;
            const float sig = a.sig[b * 3 + c];
            for (int i = tid; i < 2 * a.RH * a.RS; i += kThreads) wnum[i] = 0u;
            for (int i = tid; i < rh * rw; i += kThreads) {
                const int ly = i / rw, lx = i - ly * rw;
                const size_t g = cbase + (size_t)(Y0 + ly) * a.W + X0 + lx;
                tc::cp_async4(tc::smem_u32(simg + ly * a.RW + lx), a.img + g);
                if (WIENER) tc::cp_async4(tc::smem_u32(simg + (size_t)a.RH * a.RW + ly * a.RW + lx), a.basic + g);
            }
            tc::cp_async_commit();
            tc::cp_async_wait<0>();
            __syncthreads();
            failed = failed || *sfail != 0;
            // group size and match index of this thread's column in tile gtt (both
            // loads independent, issued one tile ahead of their use)
            auto fetch = [&](int gtt, int &nn, int &id) {
                const int q = gtt * G + gcol;
                nn = 0;
                id = -1;
                if (q < cnt) {
                    const size_t gr = (size_t)b * a.R + (size_t)(ry0 + q / tw) * a.Rx + rx0 + q % tw;
                    nn = a.n[gr];
                    id = a.idx[gr * a.n2 + min(kcol, a.n2 - 1)];
                }
            };
            int n_next, id_next;
            fetch(wg, n_next, id_next);
            for (int gt = wg; !failed && gt * G < cnt; gt += kWgs, ++it) {
                WgMeta &mt = *reinterpret_cast<WgMeta *>(meta + (it & 1) * kMetaBytes);
                // ---- 1. gather: thread t owns forward column t ----------------------
                {
                    const int g = gcol, k = kcol;
                    int n = n_next, py = 0, px = 0;
                    const int id = id_next;
                    fetch(gt + kWgs, n_next, id_next);
                    if (n < 1 || n > a.n2 || n > S || (n & (n - 1)) != 0) n = 0;
                    bool bad = false;
                    if (k < n) {
                        py = id / a.W;
                        px = id - py * a.W;
                        bad = id < 0 || py > a.H - 8 || px > a.W - 8;
                    }
                    // the group's S columns are S consecutive lanes of this warp
                    const unsigned bal = __ballot_sync(0xffffffffu, bad);
                    const unsigned gmask = S == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
                    if (bal & gmask) n = 0;
                    if (k < n) {
                        const bool inside = py >= Y0 && py + 8 <= Y0 + a.RH && px >= X0 && px + 8 <= X0 + a.RW;
                        const float *src;
                        int stride;
                        if (inside) {
                            src = (second || !WIENER ? simg : wbasic) + (py - Y0) * a.RW + (px - X0);
                            stride = a.RW;
                        } else {
                            src = (second || !WIENER ? a.img : a.basic) + cbase + (size_t)py * a.W + px;
                            stride = a.W;
                        }
                        float v[64];
#pragma unroll
                        for (int r = 0; r < 8; ++r)
#pragma unroll
                            for (int cc = 0; cc < 8; ++cc) v[r * 8 + cc] = src[r * stride + cc];
                        f2 s2 = f2_pack(0.0f, 0.0f);
#pragma unroll
                        for (int e = 0; e < 32; ++e) s2 = f2_add(s2, f2_pack(v[e], v[e + 32]));
                        const float mean = (f2_lo(s2) + f2_hi(s2)) * (1.0f / 64.0f);
                        const f2 m2 = f2_pack(mean, mean);
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            uint32_t pk[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const f2 d = f2_sub(f2_pack(v[r * 8 + 2 * e], v[r * 8 + 2 * e + 1]), m2);
                                pk[e] = tc::pack_bf16x2(f2_lo(d), f2_hi(d));
                            }
                            *reinterpret_cast<uint4 *>(op + r * kLbo + t * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                        mt.mean[t] = mean;
                        if (!second) {
                            mt.woff[jc] = inside ? (py - Y0) * a.RS + (px - X0) : -1;
                            mt.gpos[jc] = py * a.W + px;
                        }
                    }
                    const bool outside = k < n && !(py >= Y0 && py + 8 <= Y0 + a.RH && px >= X0 && px + 8 <= X0 + a.RW);
                    const unsigned bout = __ballot_sync(0xffffffffu, outside);
                    if (!second && k == 0) {
                        mt.gn[g] = n;
                        mt.cnt[g] = 0;
                        mt.inall[g] = (bout & gmask) == 0;
                    }
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                tc::bar_sync(bar_id, 128);
                // ---- 2. forward MMAs ------------------------------------------------
                if (t == 0) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        tc::mma_bf16(tmem, tc::sdesc(afwd_s + s * 2 * kLbo, kLbo, 128),
                                     tc::sdesc(op_s + s * 2 * kLbo, kLbo, 128), kIdF, s);
                    tc::mma_commit(&mbar[0]);
                }
                // bounded wait; on a timeout the tile goes on with whatever TMEM holds (the
                // status word reports it and the CTA stops at its next block-wide sync)
                if (!tc::mbar_wait(&mbar[0], phase)) wait_failed = true;
                tc::fence_after_sync();
                // ---- 3. group transform, shrinkage, spectra back to shared memory ----
                {
                    const float sg2 = sig * sig;
#pragma unroll 1
                    for (int gg = 0; gg < G / 2; ++gg) {
                        const int g = half * (G / 2) + gg, n = mt.gn[g];
                        if (n == 0) continue;  // warp-uniform
                        if (!WIENER) {
                            float v[S];
                            tmem_ld_slot<S>(tmem + tlane + (uint32_t)(g * S), v);
                            if (u == 0)
#pragma unroll
                                for (int k = 0; k < S; ++k) v[k] = 8.0f * mt.mean[g * S + k];
                            const int c0 = __reduce_add_sync(0xffffffffu, hard_any<S>(v, n, a.lambda * sig));
                            if (lane == 0) atomicAdd(&mt.cnt[g], c0);
                            store_spectra<S>(op, kLboI, u, g * S, n, v, u == 0);
                            if (u == 0)
#pragma unroll
                                for (int k = 0; k < S; ++k)
                                    if (k < n) mt.dcv[g * S + k] = v[k] * 0.125f;
                        } else {
                            float bv[S], yv[S];
                            tmem_ld_slot<S>(tmem + tlane + (uint32_t)(g * S), bv);
                            tmem_ld_slot<S>(tmem + tlane + (uint32_t)(64 + g * S), yv);
                            if (u == 0)
#pragma unroll
                                for (int k = 0; k < S; ++k) {
                                    bv[k] = 8.0f * mt.mean[g * S + k];
                                    yv[k] = 8.0f * mt.mean[64 + g * S + k];
                                }
                            float wsq = wiener_any<S>(bv, yv, n, sg2);
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) wsq += __shfl_xor_sync(0xffffffffu, wsq, o);
                            if (lane == 0) mt.wsq[g][wq & 1] = wsq;
                            store_spectra<S>(op, kLboI, u, g * S, n, yv, u == 0);
                            if (u == 0)
#pragma unroll
                                for (int k = 0; k < S; ++k)
                                    if (k < n) mt.dcv[g * S + k] = yv[k] * 0.125f;
                        }
                    }
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                tc::bar_sync(bar_id, 128);
                // ---- 4. inverse MMAs, group weights, aggregation -----------------------
                if (t == 0) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        tc::mma_bf16(tmem, tc::sdesc(ainv_s + s * 2 * kLbo, kLbo, 128),
                                     tc::sdesc(op_s + s * 2 * kLboI, kLboI, 128), kIdI, s);
                    tc::mma_commit(&mbar[1]);
                }

                // group weights, scaled by sigma^2: 1/N_har or 1/sum w^2, sigma^2 when 0
                auto weight = [&](int g) {
                    if (WIENER) {
                        const float s = mt.wsq[g][0] + mt.wsq[g][1];
                        return s > 0.0f ? 1.0f / s : sig * sig;
                    }
                    const int c = mt.cnt[g];
                    return c > 0 ? 1.0f / (float)c : sig * sig;
                };
                if (t < NI) {  // wsum at the position of inverse column t
                    const int g = t / S, k = t % S;
                    if (k < mt.gn[g]) {
                        const Fix fw = to_fixed(weight(g));
                        const size_t q = cbase + (size_t)mt.gpos[t];
                        atomicAdd(a.wsum + q, fw.lo);
                        if (fw.hi != 0) atomicAdd(a.wsum_hi + q, (unsigned long long)fw.hi);
                    }
                }
                if (!tc::mbar_wait(&mbar[1], phase)) wait_failed = true;
                phase ^= 1u;
                tc::fence_after_sync();
                {
                    const int poffw = pi * a.RS + pj;
                    const size_t poffg = cbase + (size_t)pi * a.W + pj;
#pragma unroll 1
                    for (int gg = 0; gg < G / 2; ++gg) {
                        const int g = half * (G / 2) + gg, n = mt.gn[g];
                        if (n == 0) continue;  // warp-uniform
                        float v[S];
                        tmem_ld_slot<S>(tmem + tlane + (uint32_t)(g * S), v);
                        // w kai(p) / n with the fixed-point scale 2^13 folded in (powers of two: exact)
                        const float wk = weight(g) * kp * (a.wf.tscale / (float)n);
                        const bool inall = mt.inall[g] != 0;
                        const int j0 = g * S;
                        switch (n) {
                            case 1: agg_n<1>(v, mt, j0, wk, inall, wnum, poffw, a, poffg); break;
                            case 2: agg_n<2>(v, mt, j0, wk, inall, wnum, poffw, a, poffg); break;
                            case 4: agg_n<4>(v, mt, j0, wk, inall, wnum, poffw, a, poffg); break;
                            case 8: agg_n<8>(v, mt, j0, wk, inall, wnum, poffw, a, poffg); break;
                            case 16: agg_n<16>(v, mt, j0, wk, inall, wnum, poffw, a, poffg); break;
                            default:
                                if constexpr (S >= 32) agg_n<32>(v, mt, j0, wk, inall, wnum, poffw, a, poffg);
                                break;
                        }
                    }
                }
                tc::fence_before_sync();
            }
            if (wait_failed) {
                *sfail = 1;
                atomicExch(a.err, 3);
            }
            __syncthreads();
            for (int i = tid; i < rh * rw; i += kThreads) {
                const int ly = i / rw, lx = i - ly * rw;
                const long long v = win_value(wnum[ly * a.RS + lx], wnum[a.RH * a.RS + ly * a.RS + lx], a.wf);
                if (v != 0) atomicAdd(a.num + cbase + (size_t)(Y0 + ly) * a.W + X0 + lx, (unsigned long long)v);
            }
            __syncthreads();  // windows are refilled for the next channel / tile
            failed = failed || *sfail != 0;
        }
        if (failed) break;
    }
    // after a timeout: bounded waits for MMAs that may still be in flight before
    // the TMEM is freed
    if (failed) {
        tc::mbar_wait(&mbar[0], phase ^ 1u);
        tc::mbar_wait(&mbar[1], phase ^ 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(*tslot, kWgs * kCols);
    }
}

}  // namespace

size_t filter_tc_smem_bytes(bool wiener, int step, int search, int *tr)
{
    const int hs = search / 2;
    for (int TR = 8; TR >= 1; TR /= 2) {
        const int RH = (TR - 1) * step + 2 * hs + 8, RW = RH;
        const int RS = RW + ((8 - RW % 32) + 32) % 32;  // row stride = 8 (mod 32) words
        const size_t smem = (size_t)kFixedBytes + (size_t)RH * RS * 8 + (size_t)(wiener ? 2 : 1) * RH * RW * 4;
        if (smem <= 227 * 1024) {
            if (tr) *tr = TR;
            return smem;
        }
    }
    return 0;
}

dn_status filter_tc(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B, int C,
                    int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, int *err, cudaStream_t s)
{
    TcArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.R = a.Ry * a.Rx;
    a.n2 = p.n2;
    a.step = p.step;
    a.hs = p.search / 2;
    a.lambda = p.lambda3d;
    a.err = err;
    Tables tb;
    make_tables(p.beta, &tb);
    for (int i = 0; i < 64; ++i) {
        a.kai[i] = tb.kai[i];
        a.dct[i] = tb.dct[i];
    }
    int TR = 0;
    const size_t smem = filter_tc_smem_bytes(wiener, p.step, p.search, &TR);
    if (!smem) return DN_EUNSUPPORTED;
    a.TR = TR;
    a.RH = (TR - 1) * p.step + 2 * a.hs + 8;
    a.RW = a.RH;
    a.RS = a.RW + ((8 - a.RW % 32) + 32) % 32;
    a.tiles_x = (a.Rx + TR - 1) / TR;
    a.tiles_y = (a.Ry + TR - 1) / TR;
    a.wf = win_format((long long)TR * TR * p.n2);  // a pixel gets at most one term per patch of each group
    const bool s16 = p.n2 <= 16;
    const void *fn = wiener ? (s16 ? (const void *)k_filter_tc<true, 16> : (const void *)k_filter_tc<true, 32>)
                            : (s16 ? (const void *)k_filter_tc<false, 16> : (const void *)k_filter_tc<false, 32>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DN_ECUDA;
    const size_t HW = (size_t)H * W, N = (size_t)B * C * HW;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        const size_t off = (size_t)b0 * C * HW;
        a.nb = nb;
        a.img = img + off;
        a.basic = basic ? basic + off : nullptr;
        a.idx = idx + (size_t)b0 * a.R * p.n2;
        a.n = n + (size_t)b0 * a.R;
        unsigned long long *fx = reinterpret_cast<unsigned long long *>(acc);
        a.num = fx + off;
        a.wsum = fx + N + off;
        a.num_hi = fx + 2 * N + off;
        a.wsum_hi = fx + 3 * N + off;
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < 3; ++c) a.sig[i * 3 + c] = c < C ? sig[(size_t)(b0 + i) * C + c] : 0.0f;
        const int tiles = nb * a.tiles_x * a.tiles_y;
        const int grid = tiles < sms ? tiles : sms;
        dn_status st;
        if (wiener)
            st = launch("bm3d_filter_wiener_bf16", s, [&] {
                if (s16)
                    k_filter_tc<true, 16><<<grid, kThreads, smem, s>>>(a);
                else
                    k_filter_tc<true, 32><<<grid, kThreads, smem, s>>>(a);
            });
        else
            st = launch("bm3d_filter_hard_bf16", s, [&] {
                if (s16)
                    k_filter_tc<false, 16><<<grid, kThreads, smem, s>>>(a);
                else
                    k_filter_tc<false, 32><<<grid, kThreads, smem, s>>>(a);
            });
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace dn

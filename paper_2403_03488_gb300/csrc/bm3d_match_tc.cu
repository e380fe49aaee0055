// Block matching with an FP16 tensor-core prefilter and an exact FP32 re-rank.
//
// Result: the same match lists as the exhaustive FP32 kernels (bm3d_match.cu):
// the reference first, then the candidates with d <= tau in ascending
// (d, index) order, d = ||P - Q||^2 / 64 evaluated in FP32 with the one fixed
// association of match_exact.cuh.
//
// Prefilter.  With a constant m per CTA (the mean of its pixel region) and
// a = P - m, b = Q - m, d = (||a||^2 + ||b||^2 - 2 a.b) / 64 exactly, so for a
// fixed reference the ranking key is v = ||b||^2 - 2 a.b.  The cross terms
// a.b of 128 references (M) against 128 candidate positions (N) are one
// tcgen05 GEMM with K = 64 (four MMAs of K = 16) on FP16-rounded a and b,
// accumulated in FP32 in TMEM.  Each (reference, candidate) pair gets a bound
//   E = 0.0021 |a| |b| + 2^-14 (|a|^2 + |b|^2) + 2^-16 (|a| + |b|) + 1e-3
// on |v_hat - v|: FP16 rounding of both operands (2^-11 each, so 2^-10 of
// sum |a_i b_i| <= |a| |b| per product sum, doubled in v), the FP32
// accumulation (taken as 2^-14 of the same sum, eight times the worst case of
// 64 rounded additions), FP16 subnormals (2^-25 absolute per operand), the
// FP32 evaluation of the norms and of v_hat, and the FP32 rounding of the
// exact re-rank's distance; hence lo = v_hat - E <= v <= hi = v_hat + E.
//
// Selection.  The epilogue keeps the K = (n2 - 1) + kSlack candidates of
// smallest lo (lo below the tau bound, since lo > 64 tau - |a|^2 proves
// d > tau).  With U = max hi over the first n2 - 1 of them (an upper bound of
// the (n2-1)-th smallest exact key), every candidate of the exact result has
// lo <= U, so the list holds the whole result when it never dropped a
// candidate or when its largest lo exceeds U (every dropped candidate has lo
// at least that large).  Certified lists are re-ranked with the exact FP32
// distance; the other references are matched exhaustively by
// k_match_fallback (one warp per reference, same arithmetic).
//
// Operands.  No patch is ever copied per candidate: the CTA stores each row of
// its FP16 pixel region as 64 "segments" of 8 consecutive pixels (16 bytes,
// one core-matrix row), so the K-major B operand of candidate row y and patch
// rows (i, i+1) is the segment rows y+i and y+i+1: the same buffer, the
// descriptor start moved by one row (1 KB) per patch row.
//
// CTA: 8 x 16 references (reference t = TMEM lane t), one CTA per SM:
// warp 8 issues the MMAs (one elected thread), warps 0-7 read the results
// (warp w reads lanes 32 (w % 4) .. +31, warps w and w + 4 take alternate
// chunks of two candidate rows and share their running thresholds), four
// TMEM buffers of 128 columns so that MMAs run ahead of the readers.
#include <cmath>
#include <cuda_fp16.h>

#include "common.cuh"
#include "match_exact.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kTX = 8;             // references per CTA along x
constexpr int kTY = 16;            // references per CTA along y
constexpr int kSegs = 64;          // candidate columns (segments) per region row
constexpr int kNC = 128;           // MMA N: two candidate rows per chunk
constexpr int kBufs = 4;           // TMEM buffers of kNC columns
constexpr int kEpi = 8;            // epilogue warps
constexpr int kThreads = (kEpi + 1) * 32;
constexpr int kSlack = 8;          // list entries beyond n2 - 1
constexpr int kRP = 72;            // FP32 region row pitch (64 + 7 columns used)
constexpr int kMaxChunks = 128;    // chunks of two candidate rows per CTA (at most)
constexpr float kKappa = 0.0021f;  // E = kKappa |a| |b| + ...
constexpr float kRel = 6.103515625e-05f;  // 2^-14
constexpr float kAbs1 = 1.52587890625e-05f;  // 2^-16
// F16 x F16 -> F32, both operands K-major, M = 128, N = kNC
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kNC >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

struct MatchTcArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, n2;
    int seg_rows, cst_rows, img_rows;  // shared-memory extents (rows)
    float tau[kChunk];
    int *idx;
    int *n;
    int *err;
    float *cross;  // test surface: m then the raw cross terms of CTA (cross_tx, cross_ty, 0), or null
    int cross_tx, cross_ty;
    int *fb_count;  // references whose list could not be certified: count and indices
    int *fb_list;
};

struct FallbackArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, n2;
    float tau[kChunk];
    int *idx;
    int *n;
    const int *fb_count;
    const int *fb_list;
};

// Exhaustive exact matching of the deferred references, one warp per
// reference (match_ref_warp: same distance arithmetic as the FP32 kernels).
template <int L>
__global__ void __launch_bounds__(256) k_match_fallback(FallbackArgs a)
{
    const int wglobal = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int total = *a.fb_count;
    const size_t R = (size_t)a.Ry * a.Rx;
    for (int f = wglobal; f < total; f += nwarps) {
        const int r = a.fb_list[f];
        const int b = (int)(r / R);
        const int rr = (int)(r - (size_t)b * R);
        const int ry = rr / a.Rx, rx = rr - ry * a.Rx;
        match_ref_warp<L>(a.g + (size_t)b * a.plane, a.H, a.W, a.step, a.hs, a.tau[b], a.n2, rx, ry,
                          a.idx + (size_t)r * a.n2, a.n + r);
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

// Shared-memory layout of one CTA (byte offsets).
struct Smem {
    size_t seg, rsq, cst, A, img, thr, nrm, red, seq, bar, total, reuse;
};

__host__ __device__ inline Smem smem_layout(int seg_rows, int cst_rows, int img_rows)
{
    Smem s;
    size_t o = 0;
    s.seg = o;                                   // FP16 segments [seg_rows][64][8]
    o += (size_t)seg_rows * kSegs * 16;
    s.rsq = o;                                   // row sums of squares [img_rows][64] f32
    o += (size_t)img_rows * kSegs * 4;
    s.cst = o;                                   // per-candidate (c1, c2) [cst_rows][64] float2
    o += (size_t)cst_rows * kSegs * 8;
    s.reuse = o;                                 // bytes of the region above, reused after the sweep
    o = (o + 1023) & ~(size_t)1023;
    s.A = o;                                     // A operand [8][16][8][8] f16 = 16 KB
    o += 128 * 64 * 2;
    s.img = o;                                   // FP32 region [img_rows][kRP]
    o += (size_t)img_rows * kRP * 4;
    s.thr = o;                                   // running thresholds [8 warps][32]
    o += kEpi * 32 * 4;
    s.nrm = o;                                   // per reference: |a|^2, |a| [2][128]
    o += 2 * 128 * 4;
    s.red = o;                                   // reduction scratch [kThreads / 32][3] + status
    o += 32 * 4;
    s.seq = o;                                   // chunk processing order [kMaxChunks] int
    o += kMaxChunks * 4;
    s.bar = o;                                   // mbarriers: mma_done[4], buf_free[4]; TMEM slot
    o += 2 * kBufs * 8 + 16;
    s.total = o;
    return s;
}

// v[q] for a runtime q in 0..31 (five levels of selects).
__device__ __forceinline__ float select32(const float (&v)[32], int q)
{
    float a[16], b[8], c[4], d[2];
    const bool s4 = (q & 16) != 0, s3 = (q & 8) != 0, s2 = (q & 4) != 0, s1 = (q & 2) != 0, s0 = (q & 1) != 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = s4 ? v[i + 16] : v[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = s3 ? a[i + 8] : a[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = s2 ? b[i + 4] : b[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) d[i] = s1 ? c[i + 2] : c[i];
    return s0 ? d[1] : d[0];
}

// Sorted insertion of (key, slot) into a list of K (ascending key; equal keys
// keep arrival order).
template <int K>
__device__ __forceinline__ void insert_key(float (&kv)[K], int (&ks)[K], float key, int slot)
{
    bool after = key < kv[K - 1];
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        const bool before_prev = key < kv[j - 1];
        kv[j] = before_prev ? kv[j - 1] : (after ? key : kv[j]);
        ks[j] = before_prev ? ks[j - 1] : (after ? slot : ks[j]);
        after = before_prev;
    }
    if (after) {
        kv[0] = key;
        ks[0] = slot;
    }
}

template <int L>
__global__ void __launch_bounds__(kThreads, 1) k_match_tc(MatchTcArgs a)
{
    constexpr int K = L + kSlack;
    extern __shared__ __align__(1024) uint8_t sm[];
    const Smem S = smem_layout(a.seg_rows, a.cst_rows, a.img_rows);
    uint8_t *seg = sm + S.seg;
    float *rsq = reinterpret_cast<float *>(sm + S.rsq);
    float2 *cst = reinterpret_cast<float2 *>(sm + S.cst);
    uint8_t *At = sm + S.A;
    float *img = reinterpret_cast<float *>(sm + S.img);
    volatile float *thr_sh = reinterpret_cast<float *>(sm + S.thr);
    float *nrm = reinterpret_cast<float *>(sm + S.nrm);
    float *red = reinterpret_cast<float *>(sm + S.red);
    int *status = reinterpret_cast<int *>(red + 31);
    int *seq = reinterpret_cast<int *>(sm + S.seq);
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(sm + S.bar);
    uint64_t *buf_free = mma_done + kBufs;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(buf_free + kBufs);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z;
    const int H = a.H, W = a.W, hs = a.hs, step = a.step;
    const float *g = a.g + (size_t)b * a.plane;
    const int rx0 = blockIdx.x * kTX, ry0 = blockIdx.y * kTY;

    // union of the windows: candidate top-left positions [CY0, CY0 + CH) x [CX0, CX0 + CW)
    const int gx_first = min(rx0 * step, W - 8), gx_last = min(min(rx0 + kTX - 1, a.Rx - 1) * step, W - 8);
    const int gy_first = min(ry0 * step, H - 8), gy_last = min(min(ry0 + kTY - 1, a.Ry - 1) * step, H - 8);
    const int CX0 = max(0, gx_first - hs), CX1 = min(W - 8, gx_last + hs);
    const int CY0 = max(0, gy_first - hs), CY1 = min(H - 8, gy_last + hs);
    const int CW = CX1 - CX0 + 1, CH = CY1 - CY0 + 1;
    const int RH = CH + 7;  // pixel rows of the region
    const int nchunks = (CH + 1) / 2;

    if (warp == kEpi) tc::tmem_alloc(tslot, kBufs * kNC);
    if (tid == 0) {
        for (int i = 0; i < kBufs; ++i) {
            tc::mbar_init(&mma_done[i], 1);
            tc::mbar_init(&buf_free[i], 4);
        }
        *status = 0;
        // Processing order of the chunks: blocks of 2 step chunks (the rows one reference row
        // of the tile adds), taken one chunk of every block in turn, so that every row quarter
        // of the tile has work throughout instead of waiting for its part of a top-down sweep.
        const int bs = 2 * step, nblk = (nchunks + bs - 1) / bs;
        int j = 0;
        for (int r = 0; r < bs; ++r)
            for (int k = 0; k < nblk; ++k) {
                const int c = k * bs + r;
                if (c < nchunks) seq[j++] = c;
            }
    }
    // running thresholds start at +inf before any warp can read its partner's
    if (tid < kEpi * 32) thr_sh[tid] = __int_as_float(0x7f800000);

    // ---- prologue: FP32 region, centring constant m ----------------------------------
    float psum = 0.0f, pmax = 0.0f;
    int pcnt = 0;
    for (int i = tid; i < RH * (kSegs + 7); i += kThreads) {
        const int yy = i / (kSegs + 7), xx = i - yy * (kSegs + 7);
        const int y = CY0 + yy, x = CX0 + xx;
        float v = 0.0f;
        if (y < H && x < W) {
            v = g[(size_t)y * W + x];
            psum += v;
            pmax = fmaxf(pmax, fabsf(v));
            if (!(fabsf(v) <= 3.0e4f)) pmax = __int_as_float(0x7fc00000);  // NaN / huge: no FP16 path
            ++pcnt;
        }
        img[yy * kRP + xx] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        psum += __shfl_xor_sync(0xffffffffu, psum, o);
        pcnt += __shfl_xor_sync(0xffffffffu, pcnt, o);
        const float om = __shfl_xor_sync(0xffffffffu, pmax, o);
        pmax = (om != om || pmax != pmax) ? __int_as_float(0x7fc00000) : fmaxf(pmax, om);
    }
    if (lane == 0) {
        red[warp * 3] = psum;
        red[warp * 3 + 1] = (float)pcnt;
        red[warp * 3 + 2] = pmax;
    }
    __syncthreads();
    float m = 0.0f;
    bool fp16_ok = true;
    {
        float s = 0.0f, c = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) {
            s += red[w * 3];
            c += red[w * 3 + 1];
            const float mx = red[w * 3 + 2];
            if (!(mx <= 3.0e4f)) fp16_ok = false;
        }
        m = c > 0.0f ? s / c : 0.0f;
    }

    // ---- segments (FP16 of pixel - m) and row sums of squares ---------------------------
    for (int i = tid; i < a.seg_rows * kSegs; i += kThreads) {
        const int yy = i >> 6, xs = i & 63;
        uint4 pk = make_uint4(0, 0, 0, 0);
        if (yy < RH) {
            float v[8];
            float sq = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = img[yy * kRP + xs + j] - m;
                sq = fmaf(v[j], v[j], sq);
            }
            const __half2 h0 = __floats2half2_rn(v[0], v[1]), h1 = __floats2half2_rn(v[2], v[3]);
            const __half2 h2 = __floats2half2_rn(v[4], v[5]), h3 = __floats2half2_rn(v[6], v[7]);
            pk = make_uint4(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1),
                            *reinterpret_cast<const uint32_t *>(&h2), *reinterpret_cast<const uint32_t *>(&h3));
            rsq[yy * kSegs + xs] = sq;
        }
        *reinterpret_cast<uint4 *>(seg + (size_t)i * 16) = pk;
    }
    __syncthreads();

    // ---- per-candidate constants, A operand, reference norms ----------------------------
    for (int i = tid; i < a.cst_rows * kSegs; i += kThreads) {
        const int row = i >> 6, col = i & 63;
        float2 k = make_float2(__int_as_float(0x7f800000), 0.0f);  // invalid: lo = +inf
        if (row < CH && col < CW) {
            float nq = 0.0f;
#pragma unroll
            for (int r = 0; r < 8; ++r) nq += rsq[(row + r) * kSegs + col];
            const float nb = sqrtf(nq);
            k.x = fmaf(-kRel, nq, nq) - fmaf(kAbs1, nb, 1e-3f);  // |b|^2 (1 - 2^-14) - 2^-16 |b| - 1e-3
            k.y = fmaf(kKappa, nb, kAbs1);                      // kKappa |b| + 2^-16
        }
        cst[i] = k;
    }
    if (tid < 128) {
        const int rx = rx0 + (tid & 7), ry = ry0 + (tid >> 3);
        const bool active = rx < a.Rx && ry < a.Ry;
        const int lx0 = min(rx * step, W - 8) - CX0, ly0 = min(ry * step, H - 8) - CY0;
        float np = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (active) {
                v = *reinterpret_cast<const uint4 *>(seg + ((size_t)(ly0 + i) * kSegs + lx0) * 16);
                np += rsq[(ly0 + i) * kSegs + lx0];
            }
            *reinterpret_cast<uint4 *>(At + ((i * 16 + (tid >> 3)) * 8 + (tid & 7)) * 16) = v;
        }
        nrm[tid] = np;
        nrm[128 + tid] = sqrtf(np);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    const bool dump = a.cross != nullptr && blockIdx.x == a.cross_tx && blockIdx.y == a.cross_ty && b == 0;
    if (dump && tid == 0) a.cross[0] = m;

    if (!fp16_ok) {
        // values outside the FP16 range (or not finite): every reference goes to the exact kernel
        if (tid < 128) {
            const int rx = rx0 + (tid & 7), ry = ry0 + (tid >> 3);
            if (rx < a.Rx && ry < a.Ry) {
                const int slot = atomicAdd(a.fb_count, 1);
                a.fb_list[slot] = (int)(((size_t)b * a.Ry + ry) * a.Rx + rx);
            }
        }
        __syncthreads();
        if (warp == kEpi) tc::tmem_dealloc(tmem, kBufs * kNC);
        return;
    }

    if (warp == kEpi) {
        // ---- producer: one thread issues the MMAs of every chunk --------------------------
        if (lane == 0) {
            const uint32_t abase = tc::smem_u32(At), bbase = tc::smem_u32(seg);
            int issued = 0;
            bool ok = true;
            for (int j = 0; j < nchunks && ok; ++j) {
                const int buf = j & (kBufs - 1), c = seq[j];
                if (j >= kBufs) ok = tc::mbar_wait(&buf_free[buf], ((j >> 2) - 1) & 1);
                if (!ok || *reinterpret_cast<volatile int *>(status)) break;
                tc::fence_after_sync();
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t ad = tc::sdesc(abase + 2 * t * 2048, 2048, 128);
                    const uint64_t bd = tc::sdesc(bbase + (uint32_t)(2 * c + 2 * t) * 1024, 1024, 128);
                    tc::mma_bf16(tmem + (uint32_t)(buf * kNC), ad, bd, kIdesc, t != 0);
                }
                tc::mma_commit(&mma_done[buf]);
                issued = j + 1;
            }
            if (!ok) {
                atomicExch(status, 1);
                atomicExch(a.err, 2);
            }
            // every issued MMA has completed before TMEM is released
            if (issued > 0) {
                const int j = issued - 1;
                if (!tc::mbar_wait(&mma_done[j & (kBufs - 1)], (j >> 2) & 1)) atomicExch(a.err, 2);
            }
        }
        __syncwarp();
    }

    // ---- epilogue: per reference, the K smallest lower bounds --------------------------------
    const int q4 = warp & 3, par = warp >> 2;
    const int t = q4 * 32 + lane;  // reference of this thread = TMEM lane
    const int rx = rx0 + (t & 7), ry = ry0 + (t >> 3);
    const bool active = rx < a.Rx && ry < a.Ry;
    const int x0 = min(rx * step, W - 8), y0 = min(ry * step, H - 8);
    const int lx0 = x0 - CX0, ly0 = y0 - CY0;
    const float np = nrm[t], na = nrm[128 + t];
    const float tau = a.tau[b];
    // key offset: the sweep's key is lo + 2^-14 |a|^2 (that term of E is per reference)
    const float koff = kRel * np;
    const float tlim = fmaf(64.0f * tau, 1.0f + 3.0517578125e-05f, -np * (1.0f - 3.0517578125e-05f)) + 1e-3f + koff;
    float kv[K];
    int ks[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        kv[j] = __int_as_float(0x7f800000);
        ks[j] = -1;
    }
    if (warp < kEpi) {
        const int wx_lo = max(0, lx0 - hs), wx_hi = min(CW - 1, lx0 + hs);
        const int wy_lo = active ? max(0, ly0 - hs) : 1, wy_hi = active ? min(CH - 1, ly0 + hs) : 0;
        // column masks of the two 32-column halves (window columns, minus the reference itself on its row)
        uint32_t cmask0, cmask1;
        {
            const int lo0 = max(wx_lo, 0), hi0 = min(wx_hi, 31);
            const int lo1 = max(wx_lo - 32, 0), hi1 = min(wx_hi - 32, 31);
            cmask0 = lo0 > hi0 ? 0u : ((hi0 - lo0 == 31) ? 0xffffffffu : (((1u << (hi0 - lo0 + 1)) - 1u) << lo0));
            cmask1 = lo1 > hi1 ? 0u : ((hi1 - lo1 == 31) ? 0xffffffffu : (((1u << (hi1 - lo1 + 1)) - 1u) << lo1));
        }
        // chunks any reference of this warp's rows needs (warp-uniform)
        const int yr0 = min((ry0 + 4 * q4) * step, H - 8) - CY0;
        const int yr1 = min(min(ry0 + 4 * q4 + 3, a.Ry - 1) * step, H - 8) - CY0;
        const int c_lo = max(0, yr0 - hs) >> 1, c_hi = min(CH - 1, yr1 + hs) >> 1;
        bool ok = true;
        for (int j = par; j < nchunks; j += 2) {
            const int buf = j & (kBufs - 1), c = seq[j];
            ok = tc::mbar_wait(&mma_done[buf], (j >> 2) & 1);
            if (__any_sync(0xffffffffu, !ok)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const bool need = (c >= c_lo && c <= c_hi) || dump;
            if (!need) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&buf_free[buf]);
                continue;
            }
            float thr = fminf(fminf(kv[K - 1], thr_sh[(warp ^ 4) * 32 + lane]), tlim);
#pragma unroll 1
            for (int grp = 0; grp < 4; ++grp) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * kNC + grp * 32), r);
                tc::tmem_wait_ld();
                if (grp == 3) {
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&buf_free[buf]);
                }
                const int row = 2 * c + (grp >> 1), colb = (grp & 1) * 32;
                if (dump) {
                    const int nch = nchunks;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        a.cross[1 + ((size_t)t * nch + c) * kNC + grp * 32 + q] = __uint_as_float(r[q]);
                    if (c < c_lo || c > c_hi) continue;
                }
                uint32_t cm = (row >= wy_lo && row <= wy_hi) ? ((grp & 1) ? cmask1 : cmask0) : 0u;
                if (row == ly0 && (lx0 >> 5) == (grp & 1)) cm &= ~(1u << (lx0 & 31));
                if (!__any_sync(0xffffffffu, cm != 0u)) continue;
                const float4 *cs = reinterpret_cast<const float4 *>(cst + row * kSegs + colb);
                float lo[32];
                uint32_t m32 = 0;
#pragma unroll
                for (int q = 0; q < 32; q += 2) {
                    const float4 k2 = cs[q >> 1];
                    const float t0 = fmaf(na, -k2.y, k2.x), t1 = fmaf(na, -k2.w, k2.z);
                    lo[q] = fmaf(-2.0f, __uint_as_float(r[q]), t0);
                    lo[q + 1] = fmaf(-2.0f, __uint_as_float(r[q + 1]), t1);
                    m32 |= (lo[q] < thr ? 1u : 0u) << q;
                    m32 |= (lo[q + 1] < thr ? 1u : 0u) << (q + 1);
                }
                m32 &= cm;
                while (m32) {
                    const int q = __ffs(m32) - 1;
                    m32 &= m32 - 1;
                    const float v = select32(lo, q);
                    if (v < kv[K - 1]) {
                        insert_key<K>(kv, ks, v, (row << 6) | (colb + q));
                        thr = fminf(thr, kv[K - 1]);
                    }
                }
            }
            thr_sh[warp * 32 + lane] = kv[K - 1];
        }
        if (!ok) {
            if (lane == 0) {
                atomicExch(status, 1);
                atomicExch(a.err, 2);
            }
        }
    }
    __syncthreads();  // every MMA has completed (each chunk was waited on): the operand buffers are free
    if (warp == kEpi) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kBufs * kNC);
    }
    if (*reinterpret_cast<volatile int *>(status)) return;

    // ---- merge the two lists of every reference, certify, exact re-rank --------------------
    float2 *P = reinterpret_cast<float2 *>(sm + S.seg);                 // partner lists [128][K]
    int *Ml = reinterpret_cast<int *>(P + 128 * K);                     // merged slots [128][K]
    float2 *D = reinterpret_cast<float2 *>(Ml + 128 * K);               // exact (d, index) [128][K]
    int *cert_sh = reinterpret_cast<int *>(D + 128 * K);                // [128]
    if (warp >= 4 && warp < kEpi) {
#pragma unroll
        for (int j = 0; j < K; ++j) P[t * K + j] = make_float2(kv[j], __int_as_float(ks[j]));
    }
    __syncthreads();
    if (warp < 4) {
        // partner entries in ascending order: insert while they beat the current K-th
        for (int j = 0; j < K; ++j) {
            const float2 e = P[t * K + j];
            if (!(e.x < kv[K - 1])) break;
            insert_key<K>(kv, ks, e.x, __float_as_int(e.y));
        }
        int cert = active ? 1 : 0;
        if (active && ks[K - 1] >= 0) {
            // full list: U = max over the first L entries of hi = lo + 2 E
            float U = -__int_as_float(0x7f800000);
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const int sl = ks[j];
                const float2 kc = cst[(sl >> 6) * kSegs + (sl & 63)];
                // E = na c2 + 2^-14 (nq + np) + ... ; nq recovered (over-estimated) from c1
                const float nq = (kc.x + 1e-3f) * (1.0f + 2.0f * kRel) + 1.0f;
                const float E = fmaf(na, kc.y, fmaf(kRel, nq, koff)) + fmaf(kAbs1, sqrtf(nq), 1e-3f);
                U = fmaxf(U, fmaf(2.0f, E, kv[j]));
            }
            cert = kv[K - 1] > U ? 1 : 0;
        }
#pragma unroll
        for (int j = 0; j < K; ++j) Ml[t * K + j] = ks[j];
        cert_sh[t] = cert;
        if (active && !cert) {
            const int slot = atomicAdd(a.fb_count, 1);
            a.fb_list[slot] = (int)(((size_t)b * a.Ry + ry) * a.Rx + rx);
        }
    }
    __syncthreads();
    // exact FP32 distances of the merged entries (warp w: even entries, warp w + 4: odd entries)
    const bool mine = warp < kEpi && active && cert_sh[t];
    if (mine) {
        float ref[64];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) ref[i * 8 + j] = img[(ly0 + i) * kRP + lx0 + j];
        for (int j = par; j < K; j += 2) {
            const int sl = Ml[t * K + j];
            float2 e = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7fffffff));
            if (sl >= 0) {
                const int row = sl >> 6, col = sl & 63;
                const float *q = img + row * kRP + col;
                const float d = __fmul_rn(canon_d64(ref, [&](int i, int jj) { return q[i * kRP + jj]; }), 0.015625f);
                e = make_float2(d, __int_as_float((CY0 + row) * W + CX0 + col));
            }
            D[t * K + j] = e;
        }
    }
    __syncthreads();
    if (mine) {
        // rank of each kept entry by (d, index) among the kept entries; kept = d <= tau
        const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
        int *out = a.idx + r * a.n2;
        int kept = 0;
        for (int i = 0; i < K; ++i) kept += D[t * K + i].x <= tau ? 1 : 0;
        for (int j = par; j < K; j += 2) {
            const float2 e = D[t * K + j];
            if (!(e.x <= tau)) continue;
            const int ei = __float_as_int(e.y);
            int rank = 0;
            for (int i = 0; i < K; ++i) {
                const float2 f = D[t * K + i];
                const int fi = __float_as_int(f.y);
                rank += (f.x < e.x || (f.x == e.x && fi < ei)) ? 1 : 0;
            }
            if (rank < L && 1 + rank < a.n2) out[1 + rank] = ei;
        }
        if (par == 0) {
            out[0] = y0 * W + x0;
            for (int j = 1 + min(kept, L); j < a.n2; ++j) out[j] = -1;
            a.n[r] = group_size(kept, a.n2);
        }
    }
}

template <int L>
dn_status launch_tc(MatchTcArgs &a, int B, size_t smem, cudaStream_t s)
{
    if (cudaFuncSetAttribute(k_match_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    if (cudaMemsetAsync(a.fb_count, 0, sizeof(int), s) != cudaSuccess) return DN_ECUDA;
    dim3 grid((a.Rx + kTX - 1) / kTX, (a.Ry + kTY - 1) / kTY, B);
    DN_TRY(launch("bm3d_match_tc_f16", s, [&] { k_match_tc<L><<<grid, kThreads, smem, s>>>(a); }));
    FallbackArgs f;
    f.g = a.g;
    f.plane = a.plane;
    f.H = a.H;
    f.W = a.W;
    f.Ry = a.Ry;
    f.Rx = a.Rx;
    f.step = a.step;
    f.hs = a.hs;
    f.n2 = a.n2;
    for (int i = 0; i < B; ++i) f.tau[i] = a.tau[i];
    f.idx = a.idx;
    f.n = a.n;
    f.fb_count = a.fb_count;
    f.fb_list = a.fb_list;
    return launch("bm3d_match_fallback", s, [&] { k_match_fallback<L><<<152 * 4, 256, 0, s>>>(f); });
}

// Region extents for the parameters: candidate rows (CH) and pixel rows.
void extents(int step, int search, int *cst_rows, int *seg_rows, int *img_rows)
{
    const int hs = search / 2;
    const int ch = (kTY - 1) * step + 2 * hs + 1;  // largest CH
    *cst_rows = ch + 1;                              // the last chunk may hold one row past CH
    *seg_rows = ch + 1 + 7;                          // rows an MMA of the last chunk reads
    *img_rows = ch + 1 + 7;
}

}  // namespace

size_t match_tc_smem_bytes(int step, int search)
{
    int cr, sr, ir;
    extents(step, search, &cr, &sr, &ir);
    const Smem S = smem_layout(sr, cr, ir);
    return S.total;
}

bool match_tc_supported(const dn_bm3d_pass &p)
{
    if (p.n2 < 2 || p.n2 > 32) return false;
    // candidate columns of a CTA must fit the 64 segments of a region row
    if ((kTX - 1) * p.step + 2 * (p.search / 2) + 1 > kSegs) return false;
    int cr, sr, ir;
    extents(p.step, p.search, &cr, &sr, &ir);
    const Smem S = smem_layout(sr, cr, ir);
    if (S.total > 225 * 1024 || (cr + 1) / 2 > kMaxChunks) return false;
    // merge buffers (partner lists, merged slots: below the constants, read during the
    // certification; exact distances and flags: within the reused region)
    const size_t K = (size_t)(p.n2 - 1 + kSlack);
    return 128 * K * 12 <= S.cst - S.seg && 128 * K * 20 + 512 <= S.reuse;
}

size_t match_tc_workspace_bytes(int B, int H, int W, const dn_bm3d_pass &p)
{
    const size_t R = (size_t)grid_count(H, 8, p.step) * grid_count(W, 8, p.step);
    const size_t b = B < kChunk ? (size_t)B : (size_t)kChunk;
    return align256((64 + b * R) * sizeof(int));
}

dn_status match_tc(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p, const float *tau,
                   int *idx, int *n, int *err, int *fb_ws, cudaStream_t s, float *cross, int cross_tx, int cross_ty)
{
    MatchTcArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.n2 = p.n2;
    a.err = err;
    a.cross = cross;
    a.cross_tx = cross_tx;
    a.cross_ty = cross_ty;
    a.plane = plane;
    extents(p.step, p.search, &a.cst_rows, &a.seg_rows, &a.img_rows);
    if (!match_tc_supported(p)) return DN_EUNSUPPORTED;
    const size_t smem = match_tc_smem_bytes(p.step, p.search);
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) a.tau[i] = tau[b0 + i];
        const size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        a.fb_count = fb_ws;
        a.fb_list = fb_ws + 64;
        dn_status st;
        switch (p.n2) {
            case 2: st = launch_tc<1>(a, nb, smem, s); break;
            case 4: st = launch_tc<3>(a, nb, smem, s); break;
            case 8: st = launch_tc<7>(a, nb, smem, s); break;
            case 16: st = launch_tc<15>(a, nb, smem, s); break;
            case 32: st = launch_tc<31>(a, nb, smem, s); break;
            default: return DN_EUNSUPPORTED;
        }
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace dn

// Block matching with a BF16 tensor-core prefilter and an exact FP32 re-rank.
//
// Result: the same match lists as the exhaustive FP32 kernel (bm3d_match.cu):
// reference first, then the candidates with d <= tau in ascending (d, index)
// order, d = ||P - Q||^2 / 64 evaluated in FP32 with the same association.
//
// Prefilter.  With patch means mu and centred patches P_c = P - mu_P,
//   d = (||P_c||^2 + ||Q_c||^2 - 2 P_c . Q_c) / 64 + (mu_P - mu_Q)^2
//     = A_P + c_Q - P_c . Q_c / 32 - 2 mu_P mu_Q,
//   A_P = ||P_c||^2 / 64 + mu_P^2,  c_Q = ||Q_c||^2 / 64 + mu_Q^2.
// The cross terms of 128 references (M) against a chunk of 256 candidate
// positions (N) are one tcgen05 GEMM with K = 64 pixels on BF16-rounded
// centred patches, accumulated in FP32 in TMEM, so each candidate costs a few
// FP32 operations: d_hat from the TMEM value and per-candidate constants.
// Every pair gets a bound eps >= |d_hat - d| (see pair_eps: BF16 rounding of
// both operands, the FP32 accumulation and the FP32 evaluation of the other
// terms), hence lo = d_hat - eps <= d <= hi = d_hat + eps.
//
// One sweep keeps the K = (n2 - 1) + 8 candidates of smallest lo among those
// with lo <= tau (with their hi).  Let U = min(tau, the (n2-1)-th smallest hi
// of the list), an upper bound of the (n2-1)-th smallest exact d below tau.
// Every candidate of the exact result has lo <= U, so the list holds the
// whole result when it held every lo <= tau candidate or when its largest lo
// exceeds U; it holds every candidate with d <= tau (needed for the group
// size) when it held every lo <= tau candidate or when the exact re-rank
// already finds n2 - 1 of them.  Certified lists are re-ranked with the
// exact FP32 distance; otherwise the reference is scanned exhaustively.
//
// CTA: 128 references (8 x 16 grid positions; thread = reference = TMEM
// lane), the FP32 image region of their union of windows in shared memory,
// candidate positions in rows of 64 slots, 4 rows (256 candidates) per MMA
// chunk.  Warp w holds reference rows 4w..4w+3 and reads back only the chunks
// its windows touch, 8 TMEM columns at a time (the insertion network is
// inlined 8 times, as in the FP32 kernel).
#include <cmath>

#include "common.cuh"
#include "match_exact.cuh"
#include "tc.cuh"

namespace dn {

namespace {

constexpr int kTX = 8;          // references per CTA along x
constexpr int kTY = 16;         // references per CTA along y
constexpr int kRows = 4;        // candidate rows per chunk
constexpr int kCW = 64;         // candidate slots per row
constexpr int kN = kRows * kCW; // 256 candidates per chunk (MMA N)
constexpr int kSlack = 8;       // list entries beyond n2 - 1
constexpr uint32_t kIdesc = tc::idesc_bf16(128, kN);

struct MatchTcArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, n2, RP;  // RP: smem image row pitch (floats)
    float tau[kChunk];
    int *idx;
    int *n;
    int *err;
    float *cross;  // test surface: raw cross terms of CTA (cross_tx, cross_ty, 0), or null
    int cross_tx, cross_ty;
    int *fb_count;  // references whose list could not be certified: count and indices
    int *fb_list;
};

template <int L>
__device__ __forceinline__ void insert_lex(float (&bd)[L], int (&bi)[L], float d, int id);

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

// |d_hat - d| bound for one pair (k1 = 0.0082 sp / 64, k0 = 1.6e-5 np / 64 + 1e-3).
// Cross term: each BF16 product is within (2 * 2^-9 + 2^-18) of the exact one
// and the accumulation adds at most 2^-14 of sum |a_i b_i| <= ||P_c|| ||Q_c||:
// 0.00397 ||P_c|| ||Q_c||, doubled in d and divided by 64 -> 0.0082 sp sq / 64
// with margin.  FP32 evaluation of the norms and of the exact re-rank: 2^-16
// of the magnitudes (c_Q >= ||Q_c||^2 / 64); means in FP32 shift d by at most
// 0.008 |mu_P - mu_Q|; 1e-3 absolute.
__device__ __forceinline__ float pair_eps(float k1, float k0, float sq, float cq, float dmu, float dh)
{
    return fmaf(k1, sq, k0) + 1.6e-5f * cq + 0.01f * fabsf(dmu) + 3.2e-5f * fabsf(dh);
}

template <int K>
__device__ __forceinline__ void insert_lo(float (&lo)[K], float (&hi)[K], int (&sl)[K], float l, float h, int s)
{
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        const bool before_prev = l < lo[j - 1];
        const bool before_this = l < lo[j];
        const float nl = before_prev ? lo[j - 1] : (before_this ? l : lo[j]);
        const float nh = before_prev ? hi[j - 1] : (before_this ? h : hi[j]);
        const int ns = before_prev ? sl[j - 1] : (before_this ? s : sl[j]);
        lo[j] = nl;
        hi[j] = nh;
        sl[j] = ns;
    }
    if (l < lo[0]) {
        lo[0] = l;
        hi[0] = h;
        sl[0] = s;
    }
}

// Sorted insertion by (d, index) (entries arrive in arbitrary index order).
template <int L>
__device__ __forceinline__ void insert_lex(float (&bd)[L], int (&bi)[L], float d, int id)
{
#pragma unroll
    for (int j = L - 1; j > 0; --j) {
        const bool before_prev = d < bd[j - 1] || (d == bd[j - 1] && id < bi[j - 1]);
        const bool before_this = d < bd[j] || (d == bd[j] && id < bi[j]);
        const float nd = before_prev ? bd[j - 1] : (before_this ? d : bd[j]);
        const int ni = before_prev ? bi[j - 1] : (before_this ? id : bi[j]);
        bd[j] = nd;
        bi[j] = ni;
    }
    if (d < bd[0] || (d == bd[0] && id < bi[0])) {
        bd[0] = d;
        bi[0] = id;
    }
}

// Exact FP32 distance, same association as the exhaustive kernels.
__device__ __forceinline__ float exact_d(const float (&ref)[64], const float *img, int RP, int ly, int lx)
{
    const float *q = img + ly * RP + lx;
    return __fmul_rn(canon_d64(ref, [&](int i, int j) { return q[i * RP + j]; }), 0.015625f);
}

template <int L>
__global__ void __launch_bounds__(128) k_match_tc(MatchTcArgs a)
{
    constexpr int K = L + kSlack;
    extern __shared__ __align__(128) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int b = blockIdx.z;
    const int H = a.H, W = a.W, hs = a.hs;
    const float *g = a.g + (size_t)b * a.plane;
    const int rx0 = blockIdx.x * kTX, ry0 = blockIdx.y * kTY;

    // union of the windows: candidate top-left positions [CY0, CY1] x [CX0, CX1]
    const int gx_first = min(rx0 * a.step, W - 8), gx_last = min(min(rx0 + kTX - 1, a.Rx - 1) * a.step, W - 8);
    const int gy_first = min(ry0 * a.step, H - 8), gy_last = min(min(ry0 + kTY - 1, a.Ry - 1) * a.step, H - 8);
    const int CX0 = max(0, gx_first - hs), CX1 = min(W - 8, gx_last + hs);
    const int CY0 = max(0, gy_first - hs), CY1 = min(H - 8, gy_last + hs);
    const int CW = CX1 - CX0 + 1, CH = CY1 - CY0 + 1;
    const int RWr = CW + 7, RHr = CH + 7;  // image region rows/cols
    const int nchunks = (CH + kRows - 1) / kRows;

    float *img = reinterpret_cast<float *>(sm);
    uint8_t *p = sm + (size_t)RHr * a.RP * 4;
    p = reinterpret_cast<uint8_t *>(((uintptr_t)p + 127) & ~(uintptr_t)127);
    uint8_t *At = p;
    p += 128 * 64 * 2;
    uint8_t *Bt = p;
    p += kN * 64 * 2;
    float *stats = reinterpret_cast<float *>(p);    // [2][3][kN]: mu, c, |Q_c| (double-buffered)
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stats + 6 * kN);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);

    for (int i = tid; i < RHr * RWr; i += 128) {
        const int yy = i / RWr, xx = i - yy * RWr;
        img[yy * a.RP + xx] = g[(size_t)(CY0 + yy) * W + CX0 + xx];
    }
    if (warp == 0) tc::tmem_alloc(tslot, kN);
    if (tid == 0) tc::mbar_init(mbar, 1);
    __syncthreads();

    // this thread's reference: centred BF16 row of the A operand
    const int rx = rx0 + (tid & 7), ry = ry0 + (tid >> 3);
    const bool active = rx < a.Rx && ry < a.Ry;
    const int x0 = min(rx * a.step, W - 8), y0 = min(ry * a.step, H - 8);
    const int lx0 = active ? x0 - CX0 : 0, ly0 = active ? y0 - CY0 : 0;
    float mup = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) mup += img[(ly0 + i) * a.RP + lx0 + j];
    mup *= 0.015625f;
    float np = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const float c0 = img[(ly0 + i) * a.RP + lx0 + j] - mup, c1 = img[(ly0 + i) * a.RP + lx0 + j + 1] - mup;
            np = fmaf(c0, c0, np);
            np = fmaf(c1, c1, np);
            pk[j >> 1] = tc::pack_bf16x2(c0, c1);
        }
        *reinterpret_cast<uint4 *>(At + (i * 128 + tid) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    const float Ap = np * 0.015625f + mup * mup, mup2 = 2.0f * mup;
    const float k1 = 0.0082f * sqrtf(np) * 0.015625f, k0 = 1.6e-5f * np * 0.015625f + 1e-3f;
    const float tau = a.tau[b];
    // window of this reference in region coordinates
    const int wx_lo = max(0, lx0 - hs), wx_hi = min(CW - 1, lx0 + hs);
    const int wy_lo = max(0, ly0 - hs), wy_hi = min(CH - 1, ly0 + hs);
    // chunks any reference of this warp needs (warp-uniform)
    const int wy0 = min((ry0 + 4 * warp) * a.step, H - 8) - CY0, wy1 = min((ry0 + 4 * warp + 3) * a.step, H - 8) - CY0;
    const int cw_lo = max(0, wy0 - hs) / kRows, cw_hi = min(CH - 1, wy1 + hs) / kRows;

    const uint32_t tmem = *tslot;
    const uint64_t adesc0 = tc::sdesc(tc::smem_u32(At), 128 * 16, 128);
    uint32_t phase = 0;
    float llo[K], lhi[K];
    int lsl[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        llo[j] = __int_as_float(0x7f800000);
        lhi[j] = __int_as_float(0x7f800000);
        lsl[j] = -1;
    }
    int count_lo = 0;
    bool failed = false;

    for (int c = 0; c < nchunks; ++c) {
        // B tile and per-candidate constants (alternating buffers so that a warp
        // still scanning the previous chunk never sees them overwritten)
        float *st = stats + (c & 1) * 3 * kN;
        for (int t = tid; t < kN; t += 128) {
            const int row = c * kRows + (t >> 6), col = t & 63;
            uint8_t *dst = Bt + t * 16;
            if (row < CH && col < CW) {
                const float *q = img + row * a.RP + col;
                float v[64];
                float sum = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v[i * 8 + j] = q[i * a.RP + j];
                        sum += v[i * 8 + j];
                    }
                const float mu = sum * 0.015625f;
                float nq = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint32_t pk[4];
#pragma unroll
                    for (int j = 0; j < 8; j += 2) {
                        const float c0 = v[i * 8 + j] - mu, c1 = v[i * 8 + j + 1] - mu;
                        nq = fmaf(c0, c0, nq);
                        nq = fmaf(c1, c1, nq);
                        pk[j >> 1] = tc::pack_bf16x2(c0, c1);
                    }
                    *reinterpret_cast<uint4 *>(dst + i * kN * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
                st[t] = mu;
                st[kN + t] = nq * 0.015625f + mu * mu;
                st[2 * kN + t] = sqrtf(nq);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) *reinterpret_cast<uint4 *>(dst + i * kN * 16) = make_uint4(0, 0, 0, 0);
                st[t] = 0.0f;
                st[kN + t] = 0.0f;
                st[2 * kN + t] = 0.0f;
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t bb = tc::smem_u32(Bt);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t ad = adesc0 + (uint64_t)((2 * k * 128 * 16) >> 4);
                const uint64_t bd = tc::sdesc(bb + 2 * k * kN * 16, kN * 16, 128);
                tc::mma_bf16(tmem, ad, bd, kIdesc, k != 0);
            }
            tc::mma_commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, phase);
        if (__syncthreads_or(!ok)) {
            failed = true;
            if (tid == 0) atomicExch(a.err, 2);
            break;
        }
        phase ^= 1;
        tc::fence_after_sync();
        const bool dump = a.cross != nullptr && blockIdx.x == a.cross_tx && blockIdx.y == a.cross_ty && b == 0;
        if (dump || (c >= cw_lo && c <= cw_hi)) {
            const int r0 = c * kRows;
#pragma unroll 1
            for (int grp = 0; grp < kN / 8; ++grp) {
                uint32_t r[8];
                tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + grp * 8, r);
                tc::tmem_wait_ld();
                if (dump) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) a.cross[((size_t)tid * nchunks + c) * kN + grp * 8 + q] = __uint_as_float(r[q]);
                    if (c < cw_lo || c > cw_hi) continue;
                }
                const int row = r0 + (grp >> 3);
                const int colb = (grp & 7) * 8;
                if (!active || row < wy_lo || row > wy_hi || colb > wx_hi || colb + 7 < wx_lo) continue;
                const float *mu_b = st + grp * 8, *c_b = st + kN + grp * 8, *s_b = st + 2 * kN + grp * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = colb + q;
                    if (col < wx_lo || col > wx_hi || (row == ly0 && col == lx0)) continue;
                    const float cq = c_b[q], muq = mu_b[q];
                    const float dh = fmaf(-mup2, muq, fmaf(-0.03125f, __uint_as_float(r[q]), Ap + cq));
                    const float eps = pair_eps(k1, k0, s_b[q], cq, mup - muq, dh);
                    const float l = dh - eps;
                    if (l <= tau) {
                        ++count_lo;
                        if (l < llo[K - 1]) insert_lo<K>(llo, lhi, lsl, l, dh + eps, (row << 6) | col);
                    }
                }
            }
        }
        tc::fence_before_sync();
    }
    if (failed) tc::mbar_wait(mbar, phase);
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kN);
    }
    if (!active || failed) return;

    // certification: U = min(tau, (n2-1)-th smallest hi of the list)
    float u[L];
#pragma unroll
    for (int j = 0; j < L; ++j) u[j] = __int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float h = lhi[j];
#pragma unroll
        for (int m = L - 1; m > 0; --m) {
            const bool bp = h < u[m - 1], bt = h < u[m];
            u[m] = bp ? u[m - 1] : (bt ? h : u[m]);
        }
        if (h < u[0]) u[0] = h;
    }
    const float U = fminf(tau, u[L - 1]);
    const bool all_in = count_lo <= K;
    bool cert = all_in || llo[K - 1] > U;

    float ref[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) ref[i * 8 + j] = img[(ly0 + i) * a.RP + lx0 + j];
    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);
        bi[j] = -1;
    }
    int kept = 0;
    if (cert) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (lsl[j] < 0) continue;
            const int row = lsl[j] >> 6, col = lsl[j] & 63;
            const float d = exact_d(ref, img, a.RP, row, col);
            if (d <= tau) {
                ++kept;
                insert_lex<L>(bd, bi, d, (CY0 + row) * W + CX0 + col);
            }
        }
        if (!all_in && kept < L) cert = false;  // some d <= tau candidate may be missing
    }
    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    if (!cert) {
        // deferred: matched exhaustively by k_match_fallback (one warp per reference)
        const int slot = atomicAdd(a.fb_count, 1);
        a.fb_list[slot] = (int)r;
        return;
    }
    int *out = a.idx + r * a.n2;
    out[0] = y0 * W + x0;
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (1 + j < a.n2) out[1 + j] = bi[j];
    const int total = min(kept + 1, a.n2);
    int n = 1;
    while (n * 2 <= total) n *= 2;
    a.n[r] = n;
}

template <int L>
dn_status launch_tc(MatchTcArgs &a, int B, size_t smem, cudaStream_t s)
{
    if (cudaFuncSetAttribute(k_match_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    if (cudaMemsetAsync(a.fb_count, 0, sizeof(int), s) != cudaSuccess) return DN_ECUDA;
    dim3 grid((a.Rx + kTX - 1) / kTX, (a.Ry + kTY - 1) / kTY, B);
    DN_TRY(launch("bm3d_match_tc_bf16", s, [&] { k_match_tc<L><<<grid, 128, smem, s>>>(a); }));
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

}  // namespace

size_t match_tc_smem_bytes(int step, int search)
{
    const int hs = search / 2;
    const int RH = (kTY - 1) * step + 2 * hs + 8, RW = (kTX - 1) * step + 2 * hs + 8;
    const int RP = RW + 1;
    size_t bytes = (size_t)RH * RP * 4;
    bytes = (bytes + 127) & ~(size_t)127;
    bytes += 128 * 64 * 2 + kN * 64 * 2 + 6 * kN * 4 + 16 + 16;
    return bytes;
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
    const int RW = (kTX - 1) * p.step + 2 * a.hs + 8;
    a.RP = RW + 1;
    a.plane = plane;
    // candidate rows per region must fit 64 slots
    if ((kTX - 1) * p.step + 2 * a.hs + 1 > kCW) return DN_EUNSUPPORTED;
    const size_t smem = match_tc_smem_bytes(p.step, p.search);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
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

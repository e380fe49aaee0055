// Pixel-wise NL-means (the NLM prefilter of Sec. IV-A), FP32.
//
// For every pixel p and every offset delta of the search window with
// q = p + delta inside the image:
//     d2(p, q) = mean over the patch x patch neighbourhood of (g(p+t) - g(q+t))^2
//                (guide channel g, half-sample symmetric reflection),
//     w        = exp(-max(d2 - 2 sigma^2, 0) / h^2),
// out_c(p) = sum_q w y_c(q) / sum_q w for every channel c.
//
// Design: offset-major box filtering.  A CTA owns a 32 x 16 output tile and
// stages the reflected guide (tile + patch and search halos) and the other
// channels in shared memory once.  For each pair of horizontally adjacent
// offsets (dx, dx + 1) it forms the two squared-difference images over tile +
// patch halo in the two lanes of packed FP32x2 values, sums them vertically
// then horizontally (2 * patch adds per pixel instead of patch^2; each sum in
// the same sequential order as a scalar loop), and each thread folds its
// pixel's two weights into register accumulators.  Threads map to rows and
// columns of the difference image directly (no index division).
#include "common.cuh"
#include "f32x2.cuh"

namespace dn {

namespace {

constexpr int kTX = 32, kTY = 16, kThreads = kTX * kTY;

struct NlmArgs {
    const float *in;
    float *out;
    int C, H, W, r, hs;
    float inv_np;
    float two_s2[kChunk];
    float inv_h2[kChunk];
};

__device__ __forceinline__ int reflect_hs(int i, int L, int r)
{
    // clamp to [-r, L-1+r], then half-sample symmetric reflection
    i = max(-r, min(L - 1 + r, i));
    if (i < 0) i = -i - 1;
    if (i >= L) i = 2 * L - i - 1;
    return max(0, min(L - 1, i));
}

// RT > 0: patch radius fixed at compile time (unrolled box sums, constant
// strides); RT = 0: the radius from the arguments.
template <int RT>
__global__ void __launch_bounds__(kThreads) k_nlm(NlmArgs a)
{
    extern __shared__ float sm[];
    const int r = RT > 0 ? RT : a.r, hs = a.hs, P = 2 * r + 1;
    const int GW = kTX + 2 * r + 2 * hs, GH = kTY + 2 * r + 2 * hs;  // guide region
    const int DW = kTX + 2 * r, DH = kTY + 2 * r;                    // difference image
    const int VW = kTX + 2 * hs, VH = kTY + 2 * hs;                  // value regions (other channels)
    float *S = sm;                                                   // [GH][GW]
    f2 *D = reinterpret_cast<f2 *>(S + ((GH * GW + 1) & ~1));        // [DH][DW] offset pairs
    f2 *V = D + DH * DW;                                             // [kTY][DW]
    float *Y = reinterpret_cast<float *>(V + kTY * DW);              // [C-1][VH][VW]

    const int b = blockIdx.z;
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const float *g = a.in + (size_t)b * a.C * HW;

    for (int i = threadIdx.x; i < GH * GW; i += kThreads) {
        int yy = i / GW, xx = i - yy * GW;
        int sy = reflect_hs(Y0 - r - hs + yy, H, r), sx = reflect_hs(X0 - r - hs + xx, W, r);
        S[i] = g[(size_t)sy * W + sx];
    }
    for (int c = 1; c < a.C; ++c)
        for (int i = threadIdx.x; i < VH * VW; i += kThreads) {
            int yy = i / VW, xx = i - yy * VW;
            int sy = max(0, min(H - 1, Y0 - hs + yy)), sx = max(0, min(W - 1, X0 - hs + xx));
            Y[(c - 1) * VH * VW + i] = g[c * HW + (size_t)sy * W + sx];
        }
    __syncthreads();

    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int px = X0 + tx, py = Y0 + ty;
    const float two_s2 = a.two_s2[b], inv_h2 = a.inv_h2[b];
    const f2 inv_np = f2_pack(a.inv_np, a.inv_np);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    float wsum = 0.0f;

    // this thread's elements of the difference image (at most 2 x 2): the
    // reference pixel does not depend on the offset
    constexpr int kMaxR = RT > 0 ? RT : 7;
    constexpr int kEY = (kTY + 2 * kMaxR + kTY - 1) / kTY, kEX = (kTX + 2 * kMaxR + kTX - 1) / kTX;
    float s0[kEY][kEX];
#pragma unroll
    for (int ey = 0; ey < kEY; ++ey)
#pragma unroll
        for (int ex = 0; ex < kEX; ++ex) {
            const int yy = ty + ey * kTY, xx = tx + ex * kTX;
            s0[ey][ex] = (yy < DH && xx < DW) ? S[(yy + hs) * GW + xx + hs] : 0.0f;
        }

    for (int dy = -hs; dy <= hs; ++dy)
        for (int dx = -hs; dx <= hs; dx += 2) {
            // squared differences for offsets dx (low lane) and dx + 1 (high lane)
#pragma unroll
            for (int ey = 0; ey < kEY; ++ey)
#pragma unroll
                for (int ex = 0; ex < kEX; ++ex) {
                    const int yy = ty + ey * kTY, xx = tx + ex * kTX;
                    if (yy < DH && xx < DW) {
                        const float *q = S + (yy + hs + dy) * GW + xx + hs + dx;
                        D[yy * DW + xx] = f2_sqd(f2_pack(s0[ey][ex], s0[ey][ex]), f2_pack(q[0], q[1]));
                    }
                }
            __syncthreads();
#pragma unroll
            for (int ex = 0; ex < kEX; ++ex) {
                const int xx = tx + ex * kTX;
                if (xx < DW) {
                    const f2 *d = D + ty * DW + xx;
                    f2 v = d[0];
#pragma unroll
                    for (int t = 1; t < (RT > 0 ? 2 * RT + 1 : 1); ++t) v = f2_add(v, d[t * DW]);
                    if (RT == 0)
                        for (int t = 1; t < P; ++t) v = f2_add(v, d[t * DW]);
                    V[ty * DW + xx] = v;
                }
            }
            __syncthreads();
            const f2 *vr = V + ty * DW + tx;
            f2 d2 = vr[0];
#pragma unroll
            for (int t = 1; t < (RT > 0 ? 2 * RT + 1 : 1); ++t) d2 = f2_add(d2, vr[t]);
            if (RT == 0)
                for (int t = 1; t < P; ++t) d2 = f2_add(d2, vr[t]);
            d2 = f2_mul(d2, inv_np);
            const int qy = py + dy;
            if (qy >= 0 && qy < H) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ox = dx + e, qx = px + ox;
                    if (ox <= hs && qx >= 0 && qx < W) {
                        const float ee = fmaxf((e ? f2_hi(d2) : f2_lo(d2)) - two_s2, 0.0f);
                        const float w = __expf(-ee * inv_h2);
                        acc[0] = fmaf(w, S[(ty + r + hs + dy) * GW + tx + r + hs + ox], acc[0]);
#pragma unroll
                        for (int c = 1; c < 3; ++c)
                            if (c < a.C)
                                acc[c] = fmaf(w, Y[(c - 1) * VH * VW + (ty + hs + dy) * VW + tx + hs + ox], acc[c]);
                        wsum += w;
                    }
                }
            }
        }
    if (px < W && py < H) {
        float *o = a.out + (size_t)b * a.C * HW + (size_t)py * W + px;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c < a.C) o[c * HW] = acc[c] / wsum;
    }
}

// ---------------------------------------------------------------------------
// Register-resident variant (grey images, patch radius R = 2..4).
//
// A warp owns TY = 2R + 2 output rows and 128 difference-image columns, four
// adjacent columns per lane; warps of a CTA are stacked vertically and share
// one staged guide region (fixed row pitch, 16-byte aligned per lane).  For
// each pair of offsets (dx, dx + 1), packed in the two FP32x2 lanes, a warp
// sweeps the 2P = TY + 2R rows of squared differences it needs:
//   * vertical P-row box sums of the TY output rows with one split at row P
//     (suffix sums of rows 0..P-1, prefix sums of rows P..2P-1, one add per
//     window: 3(P - 1) adds for P + 1 windows instead of (P + 1)(P - 1));
//   * horizontal P-column sums of the lane's four columns from its own
//     suffix sums and the prefix sums of the next two lanes (shuffles), so
//     the last lanes of a warp are halo: a CTA writes OW < 128 columns;
//   * weights w = 2^min(k (2 sigma^2 - d2), 0), k = log2(e) / h^2, folded
//     into one packed FMA whose additive term is -inf for a candidate
//     outside the search window or the image.
// Accumulators stay in registers for the whole offset loop.
constexpr int kRW = 4;         // warps per CTA
constexpr int kPitch = 176;    // staged row pitch in floats: 130 + 2 * 20 + 3 rounded up to 16

template <int R>
struct RegGeo {
    static constexpr int P = 2 * R + 1, TY = P + 1;
    static constexpr int OW = R <= 2 ? 124 : 120;  // output columns per CTA
    static constexpr int RowsPerCta = kRW * TY;
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Columns 4..4+m-1 after a lane's own four columns are covered by the next
// lane's prefix sums (m <= 4) or by the next lane's total plus the prefix of
// the lane after it.  Which prefix sums a lane must fetch:
template <int R>
__host__ __device__ constexpr bool need_from1(int j)  // prefix j (1..4) of lane + 1
{
    bool n = false;
    for (int k = 0; k < 4; ++k) {
        const int m = k + 2 * R - 3;
        n = n || (m <= 4 ? m == j : j == 4);
    }
    return n;
}
template <int R>
__host__ __device__ constexpr bool need_from2(int j)  // prefix j (1..4) of lane + 2
{
    bool n = false;
    for (int k = 0; k < 4; ++k) n = n || (k + 2 * R - 3 - 4 == j);
    return n;
}

template <int R>
__global__ void __launch_bounds__(kRW * 32, R <= 3 ? 3 : 2) k_nlm_reg(NlmArgs a)
{
    using G = RegGeo<R>;
    constexpr int P = G::P, TY = G::TY;
    extern __shared__ float4 sm4[];
    float *S = reinterpret_cast<float *>(sm4);
    const int hs = a.hs, H = a.H, W = a.W;
    const int A = (4 - (hs & 3)) & 3;  // column pad: makes the lane's reference columns 16-byte aligned
    const int SR = G::RowsPerCta + 2 * R + 2 * hs;
    const int b = blockIdx.z, X0 = blockIdx.x * G::OW, Y0 = blockIdx.y * G::RowsPerCta;
    const float *g = a.in + (size_t)b * H * W;
    {
        const int xs = X0 - R - hs - A, ys = Y0 - R - hs;
        for (int i = threadIdx.x; i < SR * kPitch; i += kRW * 32) {
            const int yy = i / kPitch, xx = i - yy * kPitch;
            S[i] = g[(size_t)reflect_hs(ys + yy, H, R) * W + reflect_hs(xs + xx, W, R)];
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Yw = Y0 + warp * TY;
    // reference value of difference row i, column 4 lane + c: pb[i * kPitch + c]
    const float *pb = S + (warp * TY + hs) * kPitch + 4 * lane + hs + A;
    const float kk = a.inv_h2[b] * 1.44269504088896341f;
    const float kc = kk * a.two_s2[b];
    const f2 kn = f2_pack(-kk * a.inv_np, -kk * a.inv_np);
    const float ninf = __int_as_float(0xff800000);

    float acc[TY][4], ws[TY][4];
#pragma unroll
    for (int k = 0; k < TY; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[k][c] = ws[k][c] = 0.0f;

    // offsets (dx, dx + 1) with dx + hs + A even, so candidate pairs load as
    // aligned 8-byte words; the lane outside [-hs, hs] is masked
    const int dx0 = -hs - (hs & 1);
    for (int pr = 0; pr <= hs; ++pr) {
        const int dx = dx0 + 2 * pr;
        f2 cadd[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int qx = X0 + 4 * lane + c + dx;
            const bool lo = dx >= -hs && (unsigned)qx < (unsigned)W;
            const bool hi = dx + 1 <= hs && (unsigned)(qx + 1) < (unsigned)W;
            cadd[c] = f2_pack(lo ? kc : ninf, hi ? kc : ninf);
        }
        for (int dy = -hs; dy <= hs; ++dy) {
            const float *qb = pb + dy * kPitch + dx;
            auto drow = [&](int i, f2 (&d)[4]) {
                const float4 p = *reinterpret_cast<const float4 *>(pb + i * kPitch);
                const float2 q0 = *reinterpret_cast<const float2 *>(qb + i * kPitch);
                const float2 q1 = *reinterpret_cast<const float2 *>(qb + i * kPitch + 2);
                const float q4 = qb[i * kPitch + 4];
                d[0] = f2_sqd(f2_pack(p.x, p.x), f2_pack(q0.x, q0.y));
                d[1] = f2_sqd(f2_pack(p.y, p.y), f2_pack(q0.y, q1.x));
                d[2] = f2_sqd(f2_pack(p.z, p.z), f2_pack(q1.x, q1.y));
                d[3] = f2_sqd(f2_pack(p.w, p.w), f2_pack(q1.y, q4));
            };
            // output row k from its vertical box sums v[4]
            auto emit = [&](int k, const f2 (&v)[4]) {
                if ((unsigned)(Yw + k + dy) >= (unsigned)H) return;  // warp-uniform
                f2 pre[5], suf[4];
                pre[1] = v[0];
                pre[2] = f2_add(pre[1], v[1]);
                pre[3] = f2_add(pre[2], v[2]);
                pre[4] = f2_add(pre[3], v[3]);
                suf[3] = v[3];
                suf[2] = f2_add(v[2], suf[3]);
                suf[1] = f2_add(v[1], suf[2]);
                suf[0] = f2_add(v[0], suf[1]);
                f2 n1[5], n2[5];
#pragma unroll
                for (int j = 1; j <= 4; ++j) {
                    if (need_from1<R>(j)) n1[j].v = __shfl_down_sync(0xffffffffu, pre[j].v, 1);
                    if (need_from2<R>(j)) n2[j].v = __shfl_down_sync(0xffffffffu, pre[j].v, 2);
                }
                // candidate values: row k + R of the sweep, columns c + R + (0, 1)
                const float *vb = qb + (k + R) * kPitch + (R & ~1);
                const float2 v0 = *reinterpret_cast<const float2 *>(vb);
                const float2 v1 = *reinterpret_cast<const float2 *>(vb + 2);
                const float2 v2 = *reinterpret_cast<const float2 *>(vb + 4);
                const float vv[6] = {v0.x, v0.y, v1.x, v1.y, v2.x, v2.y};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int m = c + 2 * R - 3;
                    const f2 nb = m <= 4 ? n1[m] : f2_add(n1[4], n2[m - 4]);
                    const f2 box = f2_add(suf[c], nb);
                    const f2 t = f2_fma(box, kn, cadd[c]);
                    const float wl = ex2_approx(fminf(f2_lo(t), 0.0f));
                    const float wh = ex2_approx(fminf(f2_hi(t), 0.0f));
                    const int o = c + (R & 1);
                    acc[k][c] = fmaf(wh, vv[o + 1], fmaf(wl, vv[o], acc[k][c]));
                    ws[k][c] += wl + wh;
                }
            };
            f2 sf[P][4];
#pragma unroll
            for (int i = 0; i < P; ++i) drow(i, sf[i]);
#pragma unroll
            for (int i = P - 2; i >= 0; --i)
#pragma unroll
                for (int c = 0; c < 4; ++c) sf[i][c] = f2_add(sf[i][c], sf[i + 1][c]);
            emit(0, sf[0]);
            f2 pre[4];
#pragma unroll
            for (int i = P; i < 2 * P; ++i) {
                f2 d[4];
                drow(i, d);
#pragma unroll
                for (int c = 0; c < 4; ++c) pre[c] = i == P ? d[c] : f2_add(pre[c], d[c]);
                const int k = i - P + 1;
                f2 v[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = k < P ? f2_add(sf[k][c], pre[c]) : pre[c];
                emit(k, v);
            }
        }
    }
    float *o = a.out + (size_t)b * H * W;
#pragma unroll
    for (int k = 0; k < TY; ++k) {
        const int py = Yw + k;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = 4 * lane + c, px = X0 + j;
            if (j < G::OW && px < W && py < H) o[(size_t)py * W + px] = acc[k][c] / ws[k][c];
        }
    }
}

}  // namespace

dn_status nlm_launch(const float *in, float *out, int B, int C, int H, int W, const float *sig_guide,
                     const dn_nlm_params &p, cudaStream_t s)
{
    NlmArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.r = p.patch / 2;
    a.hs = p.search / 2;
    a.inv_np = 1.0f / (float)(p.patch * p.patch);
    const int GW = kTX + 2 * a.r + 2 * a.hs, GH = kTY + 2 * a.r + 2 * a.hs;
    const int DW = kTX + 2 * a.r, DH = kTY + 2 * a.r;
    const int VW = kTX + 2 * a.hs, VH = kTY + 2 * a.hs;
    size_t smem = sizeof(float) * ((size_t)((GH * GW + 1) & ~1) + 2 * (size_t)DH * DW + 2 * (size_t)kTY * DW +
                                   (size_t)(C - 1) * VH * VW);
    if (C == 1 && a.r >= 2 && a.r <= 4 && a.hs <= 20) {
        const int RT = a.r, TY = 2 * RT + 2, OW = RT <= 2 ? 124 : 120;
        const size_t sm_reg = sizeof(float) * (size_t)(kRW * TY + 2 * RT + 2 * a.hs) * kPitch;
        void (*kr)(NlmArgs) = RT == 2 ? k_nlm_reg<2> : RT == 3 ? k_nlm_reg<3> : k_nlm_reg<4>;
        if (cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_reg) != cudaSuccess)
            return DN_ECUDA;
        for (int b0 = 0; b0 < B; b0 += kChunk) {
            int nb = B - b0 < kChunk ? B - b0 : kChunk;
            a.in = in + (size_t)b0 * H * W;
            a.out = out + (size_t)b0 * H * W;
            for (int i = 0; i < nb; ++i) {
                float sg = sig_guide[b0 + i], h = p.h_over_sigma * sg;
                a.two_s2[i] = 2.0f * sg * sg;
                a.inv_h2[i] = 1.0f / (h * h);
            }
            dim3 grid((W + OW - 1) / OW, (H + kRW * TY - 1) / (kRW * TY), nb);
            DN_TRY(launch("nlm_fp32", s, [&] { kr<<<grid, kRW * 32, sm_reg, s>>>(a); }));
        }
        return DN_OK;
    }
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    void (*kern)(NlmArgs) = a.r == 1 ? k_nlm<1> : a.r == 2 ? k_nlm<2> : a.r == 3 ? k_nlm<3> : a.r == 4 ? k_nlm<4>
                          : a.r == 5 ? k_nlm<5> : k_nlm<0>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.in = in + (size_t)b0 * C * H * W;
        a.out = out + (size_t)b0 * C * H * W;
        for (int i = 0; i < nb; ++i) {
            float sg = sig_guide[b0 + i], h = p.h_over_sigma * sg;
            a.two_s2[i] = 2.0f * sg * sg;
            a.inv_h2[i] = 1.0f / (h * h);
        }
        dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, nb);
        DN_TRY(launch("nlm_fp32", s, [&] { kern<<<grid, kThreads, smem, s>>>(a); }));
    }
    return DN_OK;
}

}  // namespace dn

// Exhaustive FP32 block matching (the BM3D grouping step).
//
// For every reference patch P on the grid (0, step, ... plus L-8 on each axis)
// and every candidate Q whose top-left corner lies in the search window
// centred on P's corner (clipped to the image):
//     d(P, Q) = ||P - Q||^2 / 64,
// evaluated with the fixed association of match_exact.cuh.  The reference is
// group member 0; the other candidates with d <= tau follow in ascending
// (d, y*W + x) order; the group size is n = min(n2, largest power of two <=
// #kept).
//
// Step 3 (the default of both passes): k_match3.  A CTA owns 16 x 8 grid
// references (those on the 3-aligned grid; the extra L-8 column and row go to
// a warp-per-reference kernel) and stages the union of their windows in
// shared memory.  For each candidate offset (oy, ox) the squared differences
// D(y, x) = (I(y, x) - I(y + oy, x + ox))^2 are the same for every reference
// whose patch covers (y, x), so the CTA forms the patch-row sums once:
// threads own a 17-pixel segment of one tile row (4 reference columns 3
// apart), split it into sums of 3 and 2 differences and combine them into the
// 4 row sums (3 + 3 + 2 pixels), for 8 horizontally adjacent offsets at a time
// (24 candidate pixels loaded per 8 offsets), two offsets per packed FP32x2
// instruction.  The row sums go through a double-buffered shared array (the
// two offsets of a pair interleaved); then each thread, owning one reference,
// combines its 8 row sums (3 + 3 + 2 rows), again two offsets per packed
// instruction, and updates its sorted list in registers (the 31-entry list
// of n2 = 32 waits in the warp's TMEM lanes while the row sums are formed,
// which keeps it out of the registers that phase needs, and its candidate
// rows are scanned from the centre out, see below).  Packed lanes round
// exactly like the scalar operations, so the distances are those of the
// fixed association.
//
// Other steps: k_match_fp32, one thread per reference over a 16 x 8 tile,
// register-blocked over 8 horizontally adjacent candidates (15 shared loads
// per patch row feed 8 candidates), same association.
#include "common.cuh"
#include "match_exact.cuh"
#include "tc.cuh"

namespace dn {

namespace {

// ---- step-3 tiled kernel --------------------------------------------------------

constexpr int kSX = 16;                      // references per CTA along x
constexpr int kSY = 8;                       // references per CTA along y
constexpr int kS3T = kSX * kSY;              // threads (one reference each)
constexpr int kSRows = 3 * (kSY - 1) + 8;    // pixel rows of the tile
constexpr int kSG = kSX / 4;                 // column groups of 4 references
constexpr int kSTasks = kSG * kSRows;        // row-sum tasks (row, group)
constexpr int kSK = 8;                       // offsets per chunk (4 packed pairs)
constexpr int kSGS = kSRows * 8;             // floats per (offset pair, group) slab: rows x 4 columns x 2 offsets
                                             // (232 = 8 mod 32: the per-reference 64-bit loads are conflict-free)
constexpr int kSBuf = (kSK / 2) * kSG * kSGS;  // floats per row-sum buffer

struct Match3Args {
    const float *g;
    size_t plane;
    int H, W, Rxa, Rya, hs, pitch, rows, img_floats;
    float tau[kChunk];
    int *idx;
    int *n;
    int n2, Rx, Ry;
};

// match_ref_warp out of line (only the rare references with a tie take it,
// and inlined its 64-pixel reference would crowd the registers of k_match3).
template <int L>
__device__ __noinline__ void match_ref_warp_call(const float *g, int H, int W, int hs, float tau, int n2, int rx,
                                                 int ry, int *out, int *nout)
{
    match_ref_warp<L>(g, H, W, 3, hs, tau, n2, rx, ry, out, nout);
}

template <int L>
__global__ void __launch_bounds__(kS3T, 4) k_match3(Match3Args a)
{
    extern __shared__ float4 sm_raw[];
    float *img = reinterpret_cast<float *>(sm_raw);  // [rows][pitch], origin (3 r0 - hs, 3 c0 - hs)
    float *hb = img + a.img_floats;                  // [2][kSK][kSG][kSGS]
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W, hs = a.hs, P = a.pitch;
    const int c0 = blockIdx.x * kSX, r0 = blockIdx.y * kSY;
    const int RX0 = 3 * c0 - hs, RY0 = 3 * r0 - hs;
    // the 31-entry list waits in TMEM (64 columns per CTA, the warp's lane
    // quarter) while the row sums are formed, which keeps it out of the
    // registers the row-sum role needs
    constexpr bool kPark = L >= 16;
    __shared__ uint32_t s_tm;
    if (kPark && threadIdx.x < 32) tc::tmem_alloc(&s_tm, 64);
    for (int i = threadIdx.x; i < a.rows * P; i += kS3T) {
        const int yy = i / P, xx = i - yy * P;
        const int gy = RY0 + yy, gx = RX0 + xx;
        img[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? g[(size_t)gy * W + gx] : 0.0f;
    }
    if (kPark) tc::fence_before_sync();
    __syncthreads();
    if (kPark) tc::fence_after_sync();
    const uint32_t tm = kPark ? s_tm + ((uint32_t)((threadIdx.x >> 5) * 32) << 16) : 0u;
    auto park = [&](const float (&d)[L], const int (&id)[L]) {
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = j < L ? __float_as_uint(d[j < L ? j : 0]) : 0u;
        tc::tmem_st32(tm, r);
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = j < L ? (uint32_t)id[j < L ? j : 0] : 0u;
        tc::tmem_st32(tm + 32, r);
        tc::tmem_wait_st();
    };
    uint32_t ud[32], ui[32];

    const int t = threadIdx.x;
    // row-sum role: tile row ay, reference columns 4 ag .. 4 ag + 3 (pixels 12 ag .. 12 ag + 16)
    const bool task = t < kSTasks;
    const int ag = t / kSRows, ay = t - (t / kSRows) * kSRows;
    const float *rrow = img + (ay + hs) * P + 12 * ag + hs;  // reference pixels of the segment
    // reference role
    const int bc = t % kSX, br = t / kSX;
    const int rx = c0 + bc, ry = r0 + br;
    const bool own = rx < a.Rxa && ry < a.Rya;
    const int xr = 3 * rx, yr = 3 * ry;
    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);  // +inf
        bi[j] = -1;
    }
    const float tau = a.tau[b];
    if constexpr (kPark) park(bd, bi);
    // the segment's reference pixels in both lanes, loaded once when the list
    // stays in registers (with the parked 31-entry list, reloading them per
    // chunk measured faster: 14.62 against 14.89 ms per 16 x 1024^2 launch)
    f2 RR0[kPark ? 1 : 17];
    if constexpr (!kPark) {
#pragma unroll
        for (int x = 0; x < 17; ++x) {
            const float r = task ? rrow[x] : 0.0f;
            RR0[x] = f2_pack(r, r);
        }
    }
    int kept = 0;
    int it = 0;
    // For the 31-entry list, candidate rows from the centre out (oy = 0, -1,
    // 1, -2, 2, ...): near rows hold the closest matches, so the list settles
    // early and later candidates rarely enter it (its insertions, divergent
    // across the warp, were 44 % of the launch; 14.65 -> 12.82 ms per
    // 16 x 1024^2 launch).  Out of index order, a candidate whose distance
    // equals an entry's could be ranked wrongly, so every equality that could
    // matter raises `tie` (a candidate equal to the full list's last entry, an
    // eviction while the last two entries are equal, equal entries in the
    // final list; about 1 reference in 2000 on noisy images) and that
    // reference is matched again in index order by its warp (match_ref_warp).
    // The shorter lists keep the index order (the same change measured slower
    // there: 8.86 -> 9.45 ms).
    constexpr bool kCentre = L >= 16;
    bool tie = false;
    for (int so = 0; so <= 2 * hs; ++so) {
        const int oy = !kCentre ? so - hs : (so & 1) ? -((so + 1) >> 1) : (so >> 1);
        const bool yok = own && (unsigned)(yr + oy) <= (unsigned)(H - 8);
        for (int ox0 = -hs; ox0 <= hs; ox0 += kSK, ++it) {
            float *hbuf = hb + (it & 1) * kSBuf;
            if (task) {
                const float *crow = img + (ay + hs + oy) * P + 12 * ag + hs + ox0;
                float C[24];
#pragma unroll
                for (int q = 0; q < 24; ++q) C[q] = crow[q];
                f2 RR[17];
#pragma unroll
                for (int x = 0; x < 17; ++x) {
                    if constexpr (kPark) {
                        const float r = rrow[x];
                        RR[x] = f2_pack(r, r);
                    } else {
                        RR[x] = RR0[x < (kPark ? 1 : 17) ? x : 0];
                    }
                }
                // offsets (2 kp, 2 kp + 1) in the two lanes of every packed value
#pragma unroll
                for (int kp = 0; kp < kSK / 2; ++kp) {
                    f2 pr[6], tr[5];
#pragma unroll
                    for (int u = 0; u < 5; ++u) {
                        const int j = 3 * u + 2 * kp;
                        const f2 e0 = f2_sub(RR[3 * u], f2_pack(C[j], C[j + 1]));
                        const f2 e1 = f2_sub(RR[3 * u + 1], f2_pack(C[j + 1], C[j + 2]));
                        const f2 e2 = f2_sub(RR[3 * u + 2], f2_pack(C[j + 2], C[j + 3]));
                        pr[u] = f2_fma(e1, e1, f2_mul(e0, e0));
                        tr[u] = f2_fma(e2, e2, pr[u]);
                    }
                    {
                        const f2 e0 = f2_sub(RR[15], f2_pack(C[15 + 2 * kp], C[16 + 2 * kp]));
                        const f2 e1 = f2_sub(RR[16], f2_pack(C[16 + 2 * kp], C[17 + 2 * kp]));
                        pr[5] = f2_fma(e1, e1, f2_mul(e0, e0));
                    }
                    const f2 h0 = f2_add(f2_add(tr[0], tr[1]), pr[2]);
                    const f2 h1 = f2_add(f2_add(tr[1], tr[2]), pr[3]);
                    const f2 h2 = f2_add(f2_add(tr[2], tr[3]), pr[4]);
                    const f2 h3 = f2_add(f2_add(tr[3], tr[4]), pr[5]);
                    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(hbuf + (kp * kSG + ag) * kSGS + 8 * ay);
                    dst[0] = make_ulonglong2(h0.v, h1.v);
                    dst[1] = make_ulonglong2(h2.v, h3.v);
                }
            }
            if constexpr (kPark) {
                __syncwarp();
                tc::tmem_ld32(tm, ud);
                tc::tmem_ld32(tm + 32, ui);
            }
            __syncthreads();  // one barrier per chunk: the buffers alternate
            if constexpr (kPark) {
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    bd[j] = __uint_as_float(ud[j < 32 ? j : 0]);
                    bi[j] = (int)ui[j < 32 ? j : 0];
                }
            }
            // offsets ox0 + k inside the window (|ox| <= hs), the image and not the reference itself
            const int klo = max(0, -xr - ox0), khi = min(kSK - 1, min(hs, W - 8 - xr) - ox0);
            unsigned valid = (yok && khi >= klo) ? ((2u << (khi - klo)) - 1u) << klo : 0u;
            if (oy == 0 && ox0 <= 0 && ox0 + kSK > 0) valid &= ~(1u << (-ox0));
            if (valid) {
                const f2 *hc = reinterpret_cast<const f2 *>(hbuf + (bc >> 2) * kSGS + 24 * br + 2 * (bc & 3));
                const f2 s64 = f2_pack(0.015625f, 0.015625f);
                // insertions are deferred over the chunk's kG = 8 candidates and then made in candidate
                // (index) order, one loop trip per candidate that beat the list's last entry: a warp
                // runs as many trips as its busiest lane instead of one divergent insertion per slot; a
                // candidate that no longer beats the last entry after an earlier insertion is a no-op.
                // (Measured on 16 x 1024^2: 11.56 ms per launch against 12.04 for per-slot insertion;
                // groups of 4 or 2 for the 31-entry list, which spills a few registers at 8, were slower.)
                constexpr int kG = kSK;
#pragma unroll
                for (int g0 = 0; g0 < kSK; g0 += kG) {
                    float dk[kG];
                    unsigned ins = 0;
#pragma unroll
                    for (int kp = g0 / 2; kp < (g0 + kG) / 2; ++kp) {
                        const f2 *hk = hc + kp * kSG * (kSGS / 2);
                        const f2 dd =
                            f2_mul(f2_tree8(hk[0], hk[4], hk[8], hk[12], hk[16], hk[20], hk[24], hk[28]), s64);
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float d = e ? f2_hi(dd) : f2_lo(dd);
                            const int c = 2 * kp + e;
                            dk[c - g0] = d;
                            if (((valid >> c) & 1u) && d <= tau) {
                                ++kept;
                                if (d < bd[L - 1]) ins |= 1u << (c - g0);
                                else if (kCentre) tie = tie || d == bd[L - 1];
                            }
                        }
                    }
                    while (ins) {
                        const int k = __ffs(ins) - 1;
                        ins &= ins - 1;
                        float d = dk[0];
#pragma unroll
                        for (int j = 1; j < kG; ++j) d = k == j ? dk[j] : d;
                        // (an eviction only once the list is full: its last entry finite)
                        if (kCentre)
                            tie = tie || d == bd[L - 1] ||
                                  (d < bd[L - 1] && bd[L - 1] < __int_as_float(0x7f800000) &&
                                   bd[L > 1 ? L - 2 : 0] == bd[L - 1]);
                        if constexpr (L >= 16) {
                            // only the last quarter (or half) of the list moves unless some lane's candidate
                            // lands before it (12.81 -> 12.39 ms; a per-lane choice diverged: 13.56)
                            const unsigned am = __activemask();
                            if (__any_sync(am, d < bd[L / 2 - 1]))
                                insert_sorted<L>(bd, bi, d, (yr + oy) * W + xr + ox0 + g0 + k);
                            else if (__any_sync(am, d < bd[3 * L / 4 - 1]))
                                insert_sorted_tail<L, L / 2>(bd, bi, d, (yr + oy) * W + xr + ox0 + g0 + k);
                            else
                                insert_sorted_tail<L, 3 * L / 4>(bd, bi, d, (yr + oy) * W + xr + ox0 + g0 + k);
                        } else {
                            insert_sorted<L>(bd, bi, d, (yr + oy) * W + xr + ox0 + g0 + k);
                        }
                    }
                }
            }
            if constexpr (kPark) {
                __syncwarp();
                park(bd, bi);
            }
        }
    }
    if constexpr (kPark) {
        tc::tmem_ld32(tm, ud);
        tc::tmem_ld32(tm + 32, ui);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < L; ++j) {
            bd[j] = __uint_as_float(ud[j < 32 ? j : 0]);
            bi[j] = (int)ui[j < 32 ? j : 0];
        }
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x < 32) {
            tc::fence_after_sync();
            tc::tmem_dealloc(s_tm, 64);
        }
    }
    if (kCentre) {
#pragma unroll
        for (int j = 1; j < L; ++j) tie = tie || (bd[j] == bd[j - 1] && bi[j] >= 0);
    }
    if (own && !tie) {
        const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
        int *out = a.idx + r * a.n2;
        out[0] = yr * W + xr;
#pragma unroll
        for (int j = 0; j < L; ++j)
            if (1 + j < a.n2) out[1 + j] = bi[j];
        a.n[r] = group_size(kept, a.n2);
    }
    // the references with a tie, one at a time by the whole warp, in index order
    for (unsigned fl = kCentre ? __ballot_sync(0xffffffffu, own && tie) : 0u; fl; fl &= fl - 1) {
        const int l = __ffs(fl) - 1;
        const int frx = __shfl_sync(0xffffffffu, rx, l), fry = __shfl_sync(0xffffffffu, ry, l);
        const size_t fr = ((size_t)b * a.Ry + fry) * a.Rx + frx;
        match_ref_warp_call<L>(g, H, W, hs, tau, a.n2, frx, fry, a.idx + fr * a.n2, a.n + fr);
    }
}

// The references off the 3-aligned grid (column Rx - 1 when Rxa < Rx, row
// Ry - 1 when Rya < Ry): one warp each.
template <int L>
__global__ void __launch_bounds__(256) k_match_edges(Match3Args a, int count)
{
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int b = blockIdx.y;
    if (wg >= count) return;
    const int ncol = a.Rx > a.Rxa ? a.Ry : 0;
    int rx, ry;
    if (wg < ncol) {
        rx = a.Rx - 1;
        ry = wg;
    } else {
        rx = wg - ncol;
        ry = a.Ry - 1;
    }
    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    match_ref_warp<L>(a.g + (size_t)b * a.plane, a.H, a.W, 3, a.hs, a.tau[b], a.n2, rx, ry, a.idx + r * a.n2,
                      a.n + r);
}

// ---- any step ------------------------------------------------------------------

constexpr int kTX = 16;     // references per CTA along x
constexpr int kTY = 8;      // references per CTA along y
constexpr int kThreads = kTX * kTY;

struct MatchArgs {
    const float *g;
    size_t plane;
    int H, W, Ry, Rx, step, hs, pitch;
    float tau[kChunk];
    int *idx;
    int *n;
    int n2;
};

// L = n2 - 1 list slots after the reference.
template <int L>
__global__ void __launch_bounds__(kThreads) k_match_fp32(MatchArgs a)
{
    extern __shared__ float sm[];
    const int b = blockIdx.z;
    const float *g = a.g + (size_t)b * a.plane;
    const int H = a.H, W = a.W;
    const int rx0 = blockIdx.x * kTX, ry0 = blockIdx.y * kTY;
    const int rx = rx0 + threadIdx.x % kTX, ry = ry0 + threadIdx.x / kTX;

    const int gx_first = min(rx0 * a.step, W - 8);
    const int gx_last = min(min(rx0 + kTX - 1, a.Rx - 1) * a.step, W - 8);
    const int gy_first = min(ry0 * a.step, H - 8);
    const int gy_last = min(min(ry0 + kTY - 1, a.Ry - 1) * a.step, H - 8);
    const int X0 = max(0, gx_first - a.hs), X1 = min(W - 1, gx_last + a.hs + 7);
    const int Y0 = max(0, gy_first - a.hs), Y1 = min(H - 1, gy_last + a.hs + 7);
    const int rw = X1 - X0 + 1, rh = Y1 - Y0 + 1;

    for (int i = threadIdx.x; i < rh * rw; i += kThreads) {
        int yy = i / rw, xx = i - yy * rw;
        sm[yy * a.pitch + xx] = g[(size_t)(Y0 + yy) * W + X0 + xx];
    }
    // slack columns read by the last (partially valid) chunk of a row
    for (int i = threadIdx.x; i < rh * 8; i += kThreads) sm[(i >> 3) * a.pitch + rw + (i & 7)] = 0.0f;
    __syncthreads();
    if (rx >= a.Rx || ry >= a.Ry) return;

    const int x0 = min(rx * a.step, W - 8), y0 = min(ry * a.step, H - 8);
    float ref[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) ref[i * 8 + j] = sm[(y0 - Y0 + i) * a.pitch + (x0 - X0 + j)];

    float bd[L];
    int bi[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        bd[j] = __int_as_float(0x7f800000);  // +inf
        bi[j] = -1;
    }
    const float tau = a.tau[b];
    int kept = 0;
    const int xs = max(0, x0 - a.hs), xe = min(W - 8, x0 + a.hs);
    const int ys = max(0, y0 - a.hs), ye = min(H - 8, y0 + a.hs);

    for (int y = ys; y <= ye; ++y) {
        const float *rowbase = sm + (y - Y0) * a.pitch - X0;
        for (int xc = xs; xc <= xe; xc += 8) {
            // row sums h_i of the 8 candidates, combined as ((h0+h1)+h2) + ((h3+h4)+h5) + (h6+h7)
            float part[8], t0[8], t1[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float *row = rowbase + i * a.pitch + xc;
                float s[15];
#pragma unroll
                for (int k = 0; k < 15; ++k) s[k] = row[k];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float h = row_sumsq(__fsub_rn(ref[i * 8], s[c]), __fsub_rn(ref[i * 8 + 1], s[c + 1]),
                                              __fsub_rn(ref[i * 8 + 2], s[c + 2]), __fsub_rn(ref[i * 8 + 3], s[c + 3]),
                                              __fsub_rn(ref[i * 8 + 4], s[c + 4]), __fsub_rn(ref[i * 8 + 5], s[c + 5]),
                                              __fsub_rn(ref[i * 8 + 6], s[c + 6]), __fsub_rn(ref[i * 8 + 7], s[c + 7]));
                    if (i == 0 || i == 3 || i == 6) part[c] = h;
                    else if (i == 1 || i == 4) part[c] = __fadd_rn(part[c], h);
                    else if (i == 2) t0[c] = __fadd_rn(part[c], h);
                    else if (i == 5) t1[c] = __fadd_rn(part[c], h);
                    else part[c] = __fadd_rn(part[c], h);
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int x = xc + c;
                const float d = __fmul_rn(__fadd_rn(__fadd_rn(t0[c], t1[c]), part[c]), 0.015625f);  // / 64, exact
                const bool valid = (x <= xe) && !(x == x0 && y == y0) && (d <= tau);
                if (valid) {
                    ++kept;
                    if (d < bd[L - 1]) insert_sorted<L>(bd, bi, d, y * W + x);
                }
            }
        }
    }

    const size_t r = ((size_t)b * a.Ry + ry) * a.Rx + rx;
    int *out = a.idx + r * a.n2;
    out[0] = y0 * W + x0;
#pragma unroll
    for (int j = 0; j < L; ++j)
        if (1 + j < a.n2) out[1 + j] = bi[j];
    a.n[r] = group_size(kept, a.n2);
}

template <int L>
dn_status launch_match(MatchArgs &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match_fp32<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DN_ECUDA;
    dim3 grid((a.Rx + kTX - 1) / kTX, (a.Ry + kTY - 1) / kTY, B);
    return launch("bm3d_match_fp32", s, [&] { k_match_fp32<L><<<grid, kThreads, smem, s>>>(a); });
}

template <int L>
dn_status launch_match3(Match3Args &a, int B, cudaStream_t s, size_t smem)
{
    if (cudaFuncSetAttribute(k_match3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DN_ECUDA;
    if (a.Rxa > 0 && a.Rya > 0) {
        dim3 grid((a.Rxa + kSX - 1) / kSX, (a.Rya + kSY - 1) / kSY, B);
        DN_TRY(launch("bm3d_match_fp32", s, [&] { k_match3<L><<<grid, kS3T, smem, s>>>(a); }));
    }
    const int count = (a.Rx > a.Rxa ? a.Ry : 0) + (a.Ry > a.Rya ? a.Rxa : 0);
    if (count > 0) {
        dim3 grid((count + 7) / 8, B);
        DN_TRY(launch("bm3d_match_edges", s, [&] { k_match_edges<L><<<grid, 256, 0, s>>>(a, count); }));
    }
    return DN_OK;
}

dn_status match_step3(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                      const float *tau, int *idx, int *n, cudaStream_t s)
{
    Match3Args a;
    a.H = H;
    a.W = W;
    a.hs = p.search / 2;
    a.Rx = grid_count(W, 8, 3);
    a.Ry = grid_count(H, 8, 3);
    a.Rxa = (W - 8) / 3 + 1;
    a.Rya = (H - 8) / 3 + 1;
    a.n2 = p.n2;
    a.plane = plane;
    a.rows = kSRows + 2 * a.hs;
    // row-sum tasks read columns up to 12 * 3 + hs + (last chunk start) + 23; odd pitch: their loads
    // hit at most 2 lanes per bank
    a.pitch = (36 + a.hs + (-a.hs + kSK * ((2 * a.hs) / kSK)) + 24) | 1;
    a.img_floats = (a.rows * a.pitch + 3) & ~3;
    const size_t smem = (size_t)(a.img_floats + 2 * kSBuf) * sizeof(float);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) a.tau[i] = tau[b0 + i];
        const size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        dn_status st;
        switch (p.n2) {
            case 1: st = launch_match3<1>(a, nb, s, smem); break;  // slot unused (n2 = 1)
            case 2: st = launch_match3<1>(a, nb, s, smem); break;
            case 4: st = launch_match3<3>(a, nb, s, smem); break;
            case 8: st = launch_match3<7>(a, nb, s, smem); break;
            case 16: st = launch_match3<15>(a, nb, s, smem); break;
            case 32: st = launch_match3<31>(a, nb, s, smem); break;
            default: return DN_EINVAL;
        }
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace

dn_status match_fp32(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                     const float *tau, int *idx, int *n, cudaStream_t s)
{
    if (p.step == 3) return match_step3(guide, plane, B, H, W, p, tau, idx, n, s);
    MatchArgs a;
    a.H = H;
    a.W = W;
    a.step = p.step;
    a.hs = p.search / 2;
    a.Ry = grid_count(H, 8, p.step);
    a.Rx = grid_count(W, 8, p.step);
    a.n2 = p.n2;
    a.plane = plane;
    int width = (kTX - 1) * p.step + 2 * a.hs + 8;
    int height = (kTY - 1) * p.step + 2 * a.hs + 8;
    int pitch = width + 8;
    pitch += ((16 - pitch % 32) + 32) % 32;  // pitch = 16 (mod 32)
    a.pitch = pitch;
    size_t smem = (size_t)height * pitch * sizeof(float);
    if (smem > 200 * 1024) return DN_EUNSUPPORTED;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        a.g = guide + (size_t)b0 * plane;
        for (int i = 0; i < nb; ++i) a.tau[i] = tau[b0 + i];
        size_t R = (size_t)a.Ry * a.Rx;
        a.idx = idx + (size_t)b0 * R * p.n2;
        a.n = n + (size_t)b0 * R;
        dn_status st;
        switch (p.n2) {
            case 1: st = launch_match<1>(a, nb, s, smem); break;  // slot unused (n2 = 1)
            case 2: st = launch_match<1>(a, nb, s, smem); break;
            case 4: st = launch_match<3>(a, nb, s, smem); break;
            case 8: st = launch_match<7>(a, nb, s, smem); break;
            case 16: st = launch_match<15>(a, nb, s, smem); break;
            case 32: st = launch_match<31>(a, nb, s, smem); break;
            default: return DN_EINVAL;
        }
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace dn

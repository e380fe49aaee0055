// BM3D collaborative filtering and aggregation, FP32 SIMT path.
//
// First pass (hard thresholding), per group of n patches (n a power of 2):
//   Z = H_n (G T2D^T): 2D orthonormal DCT-II of every 8x8 patch, then the
//   normalised Walsh-Hadamard transform along the group; zero |Z| <= lambda
//   sigma; N_har = #kept; invert both; group weight 1/(sigma^2 N_har)
//   (1 when N_har = 0).
// Second pass (empirical Wiener), per group: the same 3D transform of the
//   basic-estimate group B and of the noisy group Y (same positions); gains
//   w = B^2 / (B^2 + sigma^2); estimate T3D^-1(w Y); weight 1/(sigma^2 sum w^2)
//   (1 when the sum is 0).
// Aggregation: every estimate pixel adds weight * kaiser(i) kaiser(j) * value to
// num and weight * kaiser(i) kaiser(j) to den (compensated FP32 atomics);
// the output is num / den.
//
// One warp owns one group; its patches live in shared memory as 8 rows of 9
// floats (72 per patch), which makes both the row and the column passes of
// the separable DCT hit 32 distinct banks.  The group transform runs in
// registers: each lane owns 2 of the 64 coefficient positions and applies an
// in-register fast Walsh-Hadamard butterfly along the group.
#include "common.cuh"

namespace dn {

namespace {

constexpr int kWarps = 4;
constexpr int kPS = 72;    // floats per staged patch (8 rows x 9)
constexpr int kRS = 9;     // row stride inside a staged patch
constexpr int kNMax = 32;

struct FilterArgs {
    const float *img;    // [b][C][H][W]: noisy (pass 2) or the image to filter (pass 1)
    const float *basic;  // pass 2 only
    const int *idx;
    const int *n;
    float *num, *den, *numc, *denc;  // accumulation planes, same layout as img
    int C, H, W, R, n2;
    float lambda;
    float sig[kChunk * 3];
    Tables t;
};

template <int N>
__device__ __forceinline__ void fwht(float (&v)[N])
{
#pragma unroll
    for (int h = 1; h < N; h <<= 1)
#pragma unroll
        for (int i = 0; i < N; i += 2 * h)
#pragma unroll
            for (int j = i; j < i + h; ++j) {
                float x = v[j], y = v[j + h];
                v[j] = x + y;
                v[j + h] = x - y;
            }
}

template <int N>
__device__ __forceinline__ float inv_sqrt_n()
{
    return N == 1 ? 1.0f : N == 2 ? 0.70710678118654752f : N == 4 ? 0.5f : N == 8 ? 0.35355339059327376f
         : N == 16 ? 0.25f : 0.17677669529663688f;
}

// Hard-threshold one coefficient column (position off) of an n-patch group.
template <int N>
__device__ __forceinline__ int hard_col(float *g, int off, float thr)
{
    float v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = g[k * kPS + off];
    fwht<N>(v);
    const float sc = inv_sqrt_n<N>();
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float z = v[k] * sc;
        bool keep = fabsf(z) > thr;
        cnt += keep ? 1 : 0;
        v[k] = keep ? z : 0.0f;
    }
    fwht<N>(v);
#pragma unroll
    for (int k = 0; k < N; ++k) g[k * kPS + off] = v[k] * sc;
    return cnt;
}

// Wiener-filter one coefficient column; returns sum of squared gains.
template <int N>
__device__ __forceinline__ float wiener_col(const float *gb, float *gy, int off, float s2)
{
    float vb[N], vy[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        vb[k] = gb[k * kPS + off];
        vy[k] = gy[k * kPS + off];
    }
    fwht<N>(vb);
    fwht<N>(vy);
    const float sc = inv_sqrt_n<N>();
    float wsq = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float zb = vb[k] * sc;
        float b2 = zb * zb;
        float om = b2 / (b2 + s2);
        vy[k] = vy[k] * sc * om;
        wsq = fmaf(om, om, wsq);
    }
    fwht<N>(vy);
#pragma unroll
    for (int k = 0; k < N; ++k) gy[k * kPS + off] = vy[k] * sc;
    return wsq;
}

__device__ __forceinline__ void dct_rows(float *g, int n, int lane, const float *C, bool inverse)
{
    for (int t = lane; t < n * 8; t += 32) {
        float *row = g + (t >> 3) * kPS + (t & 7) * kRS;
        float v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = row[m];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float s = 0.0f;
#pragma unroll
            for (int m = 0; m < 8; ++m) s = fmaf(inverse ? C[m * 8 + u] : C[u * 8 + m], v[m], s);
            row[u] = s;
        }
    }
}

__device__ __forceinline__ void dct_cols(float *g, int n, int lane, const float *C, bool inverse)
{
    for (int t = lane; t < n * 8; t += 32) {
        float *col = g + (t >> 3) * kPS + (t & 7);
        float v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = col[m * kRS];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float s = 0.0f;
#pragma unroll
            for (int m = 0; m < 8; ++m) s = fmaf(inverse ? C[m * 8 + u] : C[u * 8 + m], v[m], s);
            col[u * kRS] = s;
        }
    }
}

__device__ __forceinline__ void dct2d(float *g, int n, int lane, const float *C)
{
    dct_rows(g, n, lane, C, false);
    __syncwarp();
    dct_cols(g, n, lane, C, false);
    __syncwarp();
}

__device__ __forceinline__ void idct2d(float *g, int n, int lane, const float *C)
{
    dct_cols(g, n, lane, C, true);
    __syncwarp();
    dct_rows(g, n, lane, C, true);
    __syncwarp();
}

__device__ __forceinline__ void gather(float *g, const float *ch, int W, int n, int lane, int py, int px)
{
    for (int e = lane; e < n * 64; e += 32) {
        int k = e >> 6, p = e & 63;
        int yk = __shfl_sync(0xffffffffu, py, k), xk = __shfl_sync(0xffffffffu, px, k);
        g[k * kPS + (p >> 3) * kRS + (p & 7)] = ch[(size_t)(yk + (p >> 3)) * W + xk + (p & 7)];
    }
}

__device__ __forceinline__ void aggregate(const FilterArgs &a, const float *g, size_t cbase, int n, int lane,
                                          int py, int px, float w, const float *kai)
{
    for (int e = lane; e < n * 64; e += 32) {
        int k = e >> 6, p = e & 63;
        int yk = __shfl_sync(0xffffffffu, py, k), xk = __shfl_sync(0xffffffffu, px, k);
        size_t pix = cbase + (size_t)(yk + (p >> 3)) * a.W + xk + (p & 7);
        float kw = w * kai[p];
        comp_add(a.num + pix, a.numc + pix, kw * g[k * kPS + (p >> 3) * kRS + (p & 7)]);
        comp_add(a.den + pix, a.denc + pix, kw);
    }
}

// Loads the group's positions; returns n (0 if the list is invalid).
__device__ __forceinline__ int load_group(const FilterArgs &a, int b, int r, int lane, int &py, int &px)
{
    const size_t gr = (size_t)b * a.R + r;
    int n = a.n[gr];
    if (n < 1 || n > a.n2 || n > kNMax || (n & (n - 1)) != 0) return 0;
    int id = lane < n ? a.idx[gr * a.n2 + lane] : 0;
    py = id / a.W;
    px = id - py * a.W;
    bool bad = lane < n && (id < 0 || py > a.H - 8 || px > a.W - 8);
    if (__any_sync(0xffffffffu, bad)) return 0;  // invalid list: the group is skipped
    return n;
}

__global__ void __launch_bounds__(kWarps * 32) k_filter_hard(FilterArgs a)
{
    extern __shared__ float dsm[];  // [64 dct][64 kaiser][kWarps][n2 * kPS]
    float *sC = dsm, *sK = dsm + 64;
    if (threadIdx.x < 64) {
        sC[threadIdx.x] = a.t.dct[threadIdx.x];
        sK[threadIdx.x] = a.t.kai[threadIdx.x];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kWarps + warp, b = blockIdx.y;
    if (r >= a.R) return;
    int py = 0, px = 0;
    const int n = load_group(a, b, r, lane, py, px);
    if (n == 0) return;
    float *g = dsm + 128 + (size_t)warp * a.n2 * kPS;
    const size_t HW = (size_t)a.H * a.W;
    for (int c = 0; c < a.C; ++c) {
        const size_t cbase = ((size_t)b * a.C + c) * HW;
        const float sig = a.sig[b * 3 + c];
        const float thr = a.lambda * sig;
        gather(g, a.img + cbase, a.W, n, lane, py, px);
        __syncwarp();
        dct2d(g, n, lane, sC);
        int cnt = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int pos = lane + 32 * h;
            int off = (pos >> 3) * kRS + (pos & 7);
            switch (n) {
                case 1: cnt += hard_col<1>(g, off, thr); break;
                case 2: cnt += hard_col<2>(g, off, thr); break;
                case 4: cnt += hard_col<4>(g, off, thr); break;
                case 8: cnt += hard_col<8>(g, off, thr); break;
                case 16: cnt += hard_col<16>(g, off, thr); break;
                default: cnt += hard_col<32>(g, off, thr); break;
            }
        }
        const int nhar = __reduce_add_sync(0xffffffffu, cnt);
        __syncwarp();
        idct2d(g, n, lane, sC);
        const float w = nhar > 0 ? 1.0f / (sig * sig * (float)nhar) : 1.0f;
        aggregate(a, g, cbase, n, lane, py, px, w, sK);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarps * 32) k_filter_wiener(FilterArgs a)
{
    extern __shared__ float dsm[];  // [64 dct][64 kaiser][kWarps][2][n2 * kPS]
    float *sC = dsm, *sK = dsm + 64;
    if (threadIdx.x < 64) {
        sC[threadIdx.x] = a.t.dct[threadIdx.x];
        sK[threadIdx.x] = a.t.kai[threadIdx.x];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kWarps + warp, b = blockIdx.y;
    if (r >= a.R) return;
    int py = 0, px = 0;
    const int n = load_group(a, b, r, lane, py, px);
    if (n == 0) return;
    float *gb = dsm + 128 + (size_t)warp * 2 * a.n2 * kPS;
    float *gy = gb + (size_t)a.n2 * kPS;
    const size_t HW = (size_t)a.H * a.W;
    for (int c = 0; c < a.C; ++c) {
        const size_t cbase = ((size_t)b * a.C + c) * HW;
        const float sig = a.sig[b * 3 + c];
        const float s2 = sig * sig;
        gather(gb, a.basic + cbase, a.W, n, lane, py, px);
        gather(gy, a.img + cbase, a.W, n, lane, py, px);
        __syncwarp();
        dct2d(gb, n, lane, sC);
        dct2d(gy, n, lane, sC);
        float wsq = 0.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int pos = lane + 32 * h;
            int off = (pos >> 3) * kRS + (pos & 7);
            switch (n) {
                case 1: wsq += wiener_col<1>(gb, gy, off, s2); break;
                case 2: wsq += wiener_col<2>(gb, gy, off, s2); break;
                case 4: wsq += wiener_col<4>(gb, gy, off, s2); break;
                case 8: wsq += wiener_col<8>(gb, gy, off, s2); break;
                case 16: wsq += wiener_col<16>(gb, gy, off, s2); break;
                default: wsq += wiener_col<32>(gb, gy, off, s2); break;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wsq += __shfl_xor_sync(0xffffffffu, wsq, o);
        __syncwarp();
        idct2d(gy, n, lane, sC);
        const float w = wsq > 0.0f ? 1.0f / (s2 * wsq) : 1.0f;
        aggregate(a, gy, cbase, n, lane, py, px, w, sK);
        __syncwarp();
    }
}

__global__ void k_normalize(const float *num, const float *den, const float *numc, const float *denc, float *out,
                            size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (num[i] + numc[i]) / (den[i] + denc[i]);
}

dn_status filter_common(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B,
                        int C, int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    FilterArgs a;
    a.C = C;
    a.H = H;
    a.W = W;
    a.R = grid_count(H, 8, p.step) * grid_count(W, 8, p.step);
    a.n2 = p.n2;
    a.lambda = p.lambda3d;
    make_tables(p.beta, &a.t);
    const size_t HW = (size_t)H * W, N = (size_t)B * C * HW;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        int nb = B - b0 < kChunk ? B - b0 : kChunk;
        const size_t off = (size_t)b0 * C * HW;
        a.img = img + off;
        a.basic = basic ? basic + off : nullptr;
        a.idx = idx + (size_t)b0 * a.R * p.n2;
        a.n = n + (size_t)b0 * a.R;
        a.num = acc + off;
        a.den = acc + N + off;
        a.numc = acc + 2 * N + off;
        a.denc = acc + 3 * N + off;
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < 3; ++c) a.sig[i * 3 + c] = c < C ? sig[(size_t)(b0 + i) * C + c] : 0.0f;
        dim3 grid((a.R + kWarps - 1) / kWarps, nb);
        const size_t smem = (128 + (size_t)kWarps * (wiener ? 2 : 1) * p.n2 * kPS) * sizeof(float);
        if (cudaFuncSetAttribute(wiener ? (const void *)k_filter_wiener : (const void *)k_filter_hard,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DN_ECUDA;
        dn_status st = wiener ? launch("bm3d_filter_wiener_fp32", s, [&] { k_filter_wiener<<<grid, kWarps * 32, smem, s>>>(a); })
                              : launch("bm3d_filter_hard_fp32", s, [&] { k_filter_hard<<<grid, kWarps * 32, smem, s>>>(a); });
        if (st != DN_OK) return st;
    }
    return DN_OK;
}

}  // namespace

dn_status filter_hard_fp32(const float *img, const int *idx, const int *n, int B, int C, int H, int W,
                           const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    return filter_common(false, img, nullptr, idx, n, B, C, H, W, sig, p, acc, s);
}

dn_status filter_wiener_fp32(const float *noisy, const float *basic, const int *idx, const int *n, int B, int C,
                             int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    return filter_common(true, noisy, basic, idx, n, B, C, H, W, sig, p, acc, s);
}

dn_status normalize(const float *acc, float *out, int B, int C, int H, int W, cudaStream_t s)
{
    const size_t N = (size_t)B * C * H * W;
    int blocks = (int)((N + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    return launch("bm3d_normalize", s,
                  [&] { k_normalize<<<blocks, 256, 0, s>>>(acc, acc + N, acc + 2 * N, acc + 3 * N, out, N); });
}

}  // namespace dn

// Tables, colour transform, error reductions and kernel timing.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace dn {

// ---- transform tables ------------------------------------------------------

// I0 by its power series sum_k ((x/2)^k / k!)^2.
static double bessel_i0_series(double x)
{
    double term = 1.0, sum = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 100; ++k) {
        term *= q / ((double)k * k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

void make_kaiser(int M, float beta, float *w)
{
    for (int m = 0; m < M; ++m) {
        const double r = M > 1 ? 2.0 * m / (M - 1) - 1.0 : 0.0;
        w[m] = (float)(bessel_i0_series(beta * std::sqrt(std::fmax(0.0, 1.0 - r * r))) / bessel_i0_series(beta));
    }
}

void make_tables(float beta, Tables *t)
{
    const double pi = 3.14159265358979323846;
    for (int u = 0; u < 8; ++u)
        for (int m = 0; m < 8; ++m) {
            double au = u == 0 ? std::sqrt(0.125) : 0.5;
            t->dct[u * 8 + m] = (float)(au * std::cos(pi * (2 * m + 1) * u / 16.0));
        }
    double k[8];
    for (int m = 0; m < 8; ++m) {
        double r = 2.0 * m / 7.0 - 1.0;
        k[m] = bessel_i0_series(beta * std::sqrt(std::fmax(0.0, 1.0 - r * r))) / bessel_i0_series(beta);
    }
    for (int i = 0; i < 8; ++i) {
        t->kai1[i] = (float)k[i];
        for (int j = 0; j < 8; ++j) t->kai[i * 8 + j] = (float)(k[i] * k[j]);
    }
}

// ---- colour ------------------------------------------------------------------

namespace {

struct Mat3 {
    float m[9];
};

// Full-range BT.601 RGB -> YCbCr rows (offsets omitted: they cancel in the filter).
const double kYcc[9] = {0.299, 0.587, 0.114, -0.168736, -0.331264, 0.5, 0.5, -0.418688, -0.081312};

Mat3 colour_matrix(int inverse)
{
    Mat3 r;
    if (!inverse) {
        for (int i = 0; i < 9; ++i) r.m[i] = (float)kYcc[i];
        return r;
    }
    const double *a = kYcc;
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                 a[2] * (a[3] * a[7] - a[4] * a[6]);
    double inv[9] = {(a[4] * a[8] - a[5] * a[7]), -(a[1] * a[8] - a[2] * a[7]), (a[1] * a[5] - a[2] * a[4]),
                     -(a[3] * a[8] - a[5] * a[6]), (a[0] * a[8] - a[2] * a[6]), -(a[0] * a[5] - a[2] * a[3]),
                     (a[3] * a[7] - a[4] * a[6]), -(a[0] * a[7] - a[1] * a[6]), (a[0] * a[4] - a[1] * a[3])};
    for (int i = 0; i < 9; ++i) r.m[i] = (float)(inv[i] / det);
    return r;
}

__global__ void k_colour(const float *in, float *out, size_t HW, size_t total, Mat3 M)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        size_t b = i / HW, p = i - b * HW;
        const float *x = in + b * 3 * HW + p;
        float c0 = x[0], c1 = x[HW], c2 = x[2 * HW];
        float *y = out + b * 3 * HW + p;
        y[0] = M.m[0] * c0 + M.m[1] * c1 + M.m[2] * c2;
        y[HW] = M.m[3] * c0 + M.m[4] * c1 + M.m[5] * c2;
        y[2 * HW] = M.m[6] * c0 + M.m[7] * c1 + M.m[8] * c2;
    }
}

// Exact sum and product of FP32 values as unevaluated pairs (Knuth's TwoSum,
// and the fused multiply-add form of Dekker's TwoProduct).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Per-thread partial sums of the squared errors in double-FP32 (hi + lo,
// about 44 significant bits): each pixel's error e = clip(v) - t is the exact
// pair (d, de), e^2 = d^2 (exact pair from an fma) + 2 d de + de^2, and the
// pair accumulator adds it with TwoSum.  The per-thread sums then go to FP64
// for the block and image reductions, so no per-pixel work runs on the
// narrow FP64 units.
__global__ void k_error_reduce(const float *out, const float *ref, size_t chw, double *sse, unsigned long long *mx)
{
    const int b = blockIdx.y;
    const float *o = out + (size_t)b * chw;
    const float *r = ref + (size_t)b * chw;
    float sh = 0.0f, sl = 0.0f;
    float m = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < chw; i += (size_t)gridDim.x * blockDim.x) {
        const float v = o[i], t = r[i];
        float d, de;
        two_sum(fminf(fmaxf(v, 0.0f), 255.0f), -t, d, de);
        const float p = __fmul_rn(d, d), pe = __fmaf_rn(d, d, -p);
        const float small = __fmaf_rn(de, de, __fmaf_rn(2.0f * d, de, pe));
        float h, he;
        two_sum(sh, p, h, he);
        sl = __fadd_rn(sl, __fadd_rn(he, small));
        sh = h;
        m = fmaxf(m, fabsf(v - t));
    }
    double s = (double)sh + (double)sl;
    __shared__ double ss[32];
    __shared__ float sm[32];
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        ss[warp] = s;
        sm[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s = lane < nw ? ss[lane] : 0.0;
        m = lane < nw ? sm[lane] : 0.0f;
        for (int off = 16; off > 0; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        }
        if (lane == 0) {
            atomicAdd(sse + b, s);
            atomicMax(mx + b, (unsigned long long)__double_as_longlong((double)m));
        }
    }
}

}  // namespace

dn_status colour(const float *in, float *out, int B, int H, int W, int inverse, cudaStream_t s)
{
    const size_t HW = (size_t)H * W, total = (size_t)B * HW;
    Mat3 M = colour_matrix(inverse);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    return launch(inverse ? "ycc_to_rgb" : "rgb_to_ycc", s, [&] { k_colour<<<blocks, 256, 0, s>>>(in, out, HW, total, M); });
}

dn_status error_reduce(const float *out, const float *ref, int B, size_t chw, double *sse, double *maxerr,
                       cudaStream_t s)
{
    if (cudaMemsetAsync(sse, 0, sizeof(double) * B, s) != cudaSuccess) return DN_ECUDA;
    if (cudaMemsetAsync(maxerr, 0, sizeof(double) * B, s) != cudaSuccess) return DN_ECUDA;
    size_t per = (chw + 255) / 256;
    int bx = (int)(per < 256 ? per : 256);
    if (bx < 1) bx = 1;
    dim3 grid(bx, B);
    return launch("error_reduce_fp64", s, [&] {
        k_error_reduce<<<grid, 256, 0, s>>>(out, ref, chw, sse, reinterpret_cast<unsigned long long *>(maxerr));
    });
}

// ---- device error word ---------------------------------------------------------

// Kernels whose bounded waits run out record a nonzero code here.
static __device__ int g_dn_error;

int *device_error_ptr()
{
    // looked up in the current context on every call: a cached address would go
    // stale after a device reset
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dn_error) != cudaSuccess) return nullptr;
    return static_cast<int *>(p);
}

// ---- kernel timing ---------------------------------------------------------------

namespace {

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};

thread_local bool g_prof_on = false;
thread_local std::vector<ProfRec> g_recs;
thread_local std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

void prof_begin(const char *name, cudaStream_t s)
{
    if (!g_prof_on) return;
    ProfRec r;
    r.name = name;
    r.a = take_event();
    r.b = take_event();
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
}

void prof_end(const char *name, cudaStream_t s)
{
    if (!g_prof_on || g_recs.empty()) return;
    (void)name;
    cudaEventRecord(g_recs.back().b, s);
}

}  // namespace dn

extern "C" {

dn_status dn_device_error(int *code, int reset)
{
    try {
        if (!code) return DN_EINVAL;
        int *p = dn::device_error_ptr();
        if (!p) return DN_ECUDA;
        if (cudaMemcpy(code, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DN_ECUDA;
        if (reset && cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return DN_ECUDA;
        return DN_OK;
    } catch (...) {
        return DN_ECUDA;
    }
}

void dn_profile_enable(int on) { dn::g_prof_on = on != 0; }

void dn_profile_reset(void)
{
    for (auto &r : dn::g_recs) {
        dn::g_pool.push_back(r.a);
        dn::g_pool.push_back(r.b);
    }
    dn::g_recs.clear();
}

int dn_profile_read(char *names, int name_stride, int max_kernels, int *launches, double *ms)
{
    std::vector<std::string> keys;
    std::vector<int> cnt;
    std::vector<double> tot;
    for (auto &r : dn::g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return -1;
        size_t k = 0;
        while (k < keys.size() && keys[k] != r.name) ++k;
        if (k == keys.size()) {
            keys.push_back(r.name);
            cnt.push_back(0);
            tot.push_back(0.0);
        }
        cnt[k] += 1;
        tot[k] += t;
    }
    int n = (int)keys.size() < max_kernels ? (int)keys.size() : max_kernels;
    for (int k = 0; k < n; ++k) {
        if (names && name_stride > 0) {
            std::strncpy(names + (size_t)k * name_stride, keys[k].c_str(), (size_t)name_stride - 1);
            names[(size_t)k * name_stride + name_stride - 1] = 0;
        }
        if (launches) launches[k] = cnt[k];
        if (ms) ms[k] = tot[k];
    }
    return (int)keys.size();
}

}  // extern "C"

// Internal helpers of libdenoise (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/denoise.h"

namespace dn {

// Images per launch chunk for per-image scalars passed by value.
constexpr int kChunk = 64;

// Transform tables passed by value to the filtering kernels (built on the
// host by make_tables from their definitions; no global device state).
struct Tables {
    float dct[64];   // orthonormal DCT-II, dct[u*8+m] = a_u cos(pi (2m+1) u / 16)
    float kai[64];   // Kaiser outer product, kai[i*8+j] = k[i] k[j]
    float kai1[8];   // the 1D Kaiser window k
};

void make_tables(float beta, Tables *t);
// Kaiser window of length M: w[m] = I0(beta sqrt(1 - (2m/(M-1) - 1)^2)) / I0(beta).
void make_kaiser(int M, float beta, float *w);

// Per-image scalars of one launch chunk.
struct ImageScalars {
    float tau[kChunk];          // matching threshold per image
    float sig[kChunk * 3];      // per-image, per-channel noise std
};

// ---- kernel timing (dn_profile_*) -----------------------------------------
void prof_begin(const char *name, cudaStream_t s);
void prof_end(const char *name, cudaStream_t s);

// Launch wrapper: times the launch when profiling is on and maps errors.
template <typename F>
inline dn_status launch(const char *name, cudaStream_t s, F &&f)
{
    prof_begin(name, s);
    f();
    cudaError_t e = cudaGetLastError();
    prof_end(name, s);
    return e == cudaSuccess ? DN_OK : DN_ECUDA;
}

#define DN_TRY(expr)                       \
    do {                                   \
        dn_status _st = (expr);            \
        if (_st != DN_OK) return _st;      \
    } while (0)

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Carves 256-byte aligned sub-buffers out of a caller workspace.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count)
    {
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += align256(count * sizeof(T));
        return p;
    }
};

inline int grid_count(int L, int patch, int step)
{
    int last = L - patch;
    if (last < 0 || step < 1) return 0;
    return last / step + 1 + (last % step != 0 ? 1 : 0);
}

// Aggregation accumulators of the filtering passes: four 64-bit fixed-point
// planes per image pixel: num (per pixel), wsum (group weights summed per patch
// position), and their high words num_hi, wsum_hi.
constexpr size_t kAccBytesPerPixel = 4 * sizeof(long long);

// ---- launchers implemented in the .cu files -------------------------------
dn_status match_fp32(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                     const float *tau, int *idx, int *n, cudaStream_t s);
// Block matching on 2D-prethresholded patches (first pass at high noise):
// thr[b] = lambda2d * sigma of image b's guide channel (host arrays of B).
dn_status match_prethresh(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                          const float *tau, const float *thr, int *idx, int *n, cudaStream_t s);
size_t match_pre_smem_bytes(int W, const dn_bm3d_pass &p);
dn_status filter_hard_fp32(const float *img, const int *idx, const int *n, int B, int C, int H, int W,
                           const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s);
dn_status filter_wiener_fp32(const float *noisy, const float *basic, const int *idx, const int *n, int B, int C,
                             int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s);
// The same two passes with the 2D transforms on the tensor cores (BF16
// operands, FP32 accumulation); err: device status word (3 = a wait timed out).
dn_status filter_tc(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B, int C,
                    int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, int *err, cudaStream_t s);
// Shared memory of the tensor-core filter (0: the search window is too large);
// *tr receives the side of its tile of reference positions.
size_t filter_tc_smem_bytes(bool wiener, int step, int search, int *tr);
// out = num / den with den = the Kaiser window (parameter beta, length = the
// patch side K of the pass) correlated with wsum
dn_status normalize(const float *acc, float *out, int B, int C, int H, int W, float beta, cudaStream_t s, int K = 8);
dn_status colour(const float *in, float *out, int B, int H, int W, int inverse, cudaStream_t s);
dn_status nlm_launch(const float *in, float *out, int B, int C, int H, int W, const float *sig_guide,
                     const dn_nlm_params &p, cudaStream_t s);
dn_status error_reduce(const float *out, const float *ref, int B, size_t chw, double *sse, double *maxerr,
                       cudaStream_t s);
dn_status conv3x3_fwd_fp32(const float *x, const float *w, const float *b, const float *mask, float *y, int N,
                           int Kin, int Kout, int H, int W, int relu, bool trans, cudaStream_t s);
dn_status conv3x3_bwd_weight_fp32(const float *x, const float *dy, float *dw, float *db, int N, int Cin, int Cout,
                                  int H, int W, cudaStream_t s);
// z [N][2 cc][H][W] = [pre / 255 (cc planes), noisy / 255 (cc planes)]
dn_status pack_input(const float *pre, const float *noisy, float *z, int N, int cc, int H, int W, cudaStream_t s);
dn_status residual_out(const float *pre, const float *r, float *out, size_t total, cudaStream_t s);
dn_status relu_bwd(const float *g, const float *y, float *out, size_t count, cudaStream_t s);
dn_status l1_grad(const float *r, const float *pre, const float *clean, float *dr, size_t count, double *loss,
                  cudaStream_t s);
int *device_error_ptr();
size_t match_tc_smem_bytes(int step, int search);
// Whether the tensor-core matcher's tiling (64 candidate columns per CTA, its
// shared memory) supports the pass parameters.
bool match_tc_supported(const dn_bm3d_pass &p);
// fb_ws: device workspace of match_tc_workspace_bytes (deferred references)
size_t match_tc_workspace_bytes(int B, int H, int W, const dn_bm3d_pass &p);
dn_status match_tc(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p, const float *tau,
                   int *idx, int *n, int *err, int *fb_ws, cudaStream_t s, float *cross = nullptr, int cross_tx = 0,
                   int cross_ty = 0);
size_t conv_tc_smem_bytes();
// Larger patches (bm3d_large.cu): matching on pixels (sides 11, 12) or on
// 2D-prethresholded patches (side 12), and both filtering passes (11, 12).
bool large_patch_supported(int K);
bool large_prethresh_supported(int K);
dn_status match_large(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p, const float *tau,
                      int *idx, int *n, cudaStream_t s);
size_t match_pre_large_smem_bytes(int W, const dn_bm3d_pass &p);
dn_status match_prethresh_large(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                                const float *tau, const float *thr, int *idx, int *n, cudaStream_t s);
dn_status filter_large(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B, int C,
                       int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s);
// Flexible network contractions on the tensor cores (flnet_tc.cu): BF16 operands, FP32 in and out.
dn_status pw_fwd_tc(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                    int relu, int transposed, int *err, cudaStream_t s);
dn_status deconv2x2_fwd_tc(const float *x, const float *w, const float *b, const float *skip, float *y, int N,
                           int Cin, int Cout, int H, int W, int *err, cudaStream_t s);
// Two hidden C -> C layers (bias + ReLU each) in one pass on the tensor cores (C = 32).
dn_status conv3x3_tc_pair(const void *x, void *y, const void *wpa, const float *ba, const void *wpb, const float *bb,
                          int N, int H, int W, int C, int *err, cudaStream_t s);
// W [C][3][3][C] -> the tensor-core B operand; flip: of the transposed (data-gradient) layer.
dn_status pack_w_tc(const float *w, void *out, int C, cudaStream_t s, bool flip = false);
// Hidden C -> C layer on the tensor cores (NHWC bf16); bias may be null; mask (NHWC bf16, or
// null) zeroes the outputs where the mask is not positive (the ReLU backward of the data gradient).
dn_status conv3x3_tc(const void *x, void *y, const void *wpack, const float *bias, int N, int H, int W, int C,
                     int relu, int *err, cudaStream_t s, const void *mask = nullptr);
dn_status conv_first_bf16(const float *pre, const float *noisy, const float *w, const float *b, void *y, int N,
                          int cc, int H, int W, int C, cudaStream_t s);
dn_status conv_last_bf16(const void *x, const float *w, const float *b, const float *pre, float *out, int N, int cc,
                         int H, int W, int C, cudaStream_t s);
dn_status adam(float *p, const float *g, float *m, float *v, size_t count, int t, float lr, float b1, float b2,
               float eps, cudaStream_t s);
// Gradient of the L1 loss of the grey width-32 residual network with BF16 tensor-core
// forward and backward (cnn_train_tc.cu); grad is overwritten, loss accumulated.
size_t cnn_grad_tc_workspace_bytes(int N, int H, int W, int layers);
// Weight and bias gradient of one 32 -> 32 layer from its NHWC bf16 input x and output gradient g.
size_t conv_bwd_w_tc_workspace_bytes(int N, int H, int W);
dn_status conv_bwd_w_tc(const void *x, const void *g, float *dw, float *db, int N, int H, int W, void *ws, int *err,
                        cudaStream_t s);
dn_status cnn_grad_tc(const float *noisy, const float *pre, const float *clean, int N, int H, int W, int layers,
                      const float *weights, float *grad, double *loss, void *ws, int *err, cudaStream_t s);

}  // namespace dn

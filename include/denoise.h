/*
 * denoise.h -- C ABI of the GB300 nonlocal + neural denoiser (libdenoise.so).
 *
 * The method (Sec. II, Fig. 1, Eq. 2-3): a nonlocal filter (BM3D, or NL-means
 * as the cheaper variant, Sec. IV-A) denoises the noisy image y of the AWGN
 * model y = x + n (Eq. 1); a lightweight residual CNN takes
 * z = Concatenate(BM3D(y), y) (Eq. 3) and its output F(z) is added to the
 * filter output (Eq. 2).  The paper uses BM3D / NLM as given components; the
 * filter steps below are the standard published definitions (BM3D: block
 * matching, 3D DCT x Walsh-Hadamard collaborative hard thresholding or
 * Wiener filtering, Kaiser-windowed aggregation; NL-means: patch-similarity
 * weighted average).
 *
 * Conventions shared by every entry point
 *   - Images are contiguous NCHW float32 on the DEVICE, [B][C][H][W], on a
 *     0..255 scale, C in {1, 3}.  Colour images are converted to YCbCr
 *     (full-range BT.601), matched on Y and filtered per channel with the
 *     per-channel noise std sigma * ||row_c||_2, then converted back.
 *   - sigma is a HOST array of B floats (noise std per image, 0..255 scale,
 *     0 < sigma <= 255).
 *   - The caller owns every buffer, including the device workspace; the
 *     library never allocates device memory, never synchronises the stream
 *     and issues all work asynchronously on `stream` (0 = legacy default).
 *   - Errors: argument errors are detected on the host and returned BEFORE
 *     any launch (nothing is written).  A launch failure returns DN_ECUDA.
 *     Outputs are unspecified after any error.  No C++ exception crosses
 *     the ABI.  Calls are thread-safe as long as concurrent calls use
 *     distinct workspaces and output buffers.
 *   - Results are unclipped floats.
 */
#ifndef DENOISE_H
#define DENOISE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *dn_stream_t; /* == cudaStream_t */

typedef enum {
    DN_OK = 0,
    DN_EINVAL = -1,       /* bad argument (size, sigma <= 0, C not in {1,3}, ...) */
    DN_ENOMEM = -2,       /* workspace smaller than the *_workspace_bytes query  */
    DN_ECUDA = -3,        /* a CUDA launch or runtime call failed                */
    DN_EDEVICE = -4,      /* a kernel reported an error through its status word  */
    DN_EUNSUPPORTED = -5  /* valid but not implemented combination               */
} dn_status;

/* Arithmetic of the BM3D stages (dn_bm3d_params.precision is a bit set; the
 * tensor-core paths are built for 8 x 8 patches, passes with 11 x 11 or
 * 12 x 12 patches run in FP32 whatever the bits):
 *   DN_FP32        every stage in FP32 on the CUDA cores;
 *   DN_BF16        the 2D patch transforms of both filtering passes as 64 x 64
 *                  contractions on the tensor cores (BF16 operands, FP32
 *                  accumulation; patches centred on their FP32 mean first,
 *                  which stays in FP32); group transform, shrinkage and
 *                  aggregation in FP32;
 *   DN_BF16_MATCH  block matching with the tensor-core prefilter (distance
 *                  cross terms as FP16 GEMMs with FP32 accumulation, a proven
 *                  error bound per pair) and an exact FP32 re-rank: match
 *                  lists identical to FP32.
 * For the CNN (dn_cnn.precision) DN_BF16 selects the tcgen05 BF16 layers. */
typedef enum { DN_FP32 = 0, DN_BF16 = 1, DN_BF16_MATCH = 2 } dn_precision;
typedef enum { DN_PREFILTER_BM3D = 0, DN_PREFILTER_NLM = 1 } dn_prefilter;

/* One BM3D pass.  Distances are mean squared differences over the patch.
 * Above sigma 40 (sigma_regime 0) a pass may switch to the larger patches of
 * BM3D's high-noise profile (patch_high, step_high: 12 x 12 on a step-4 grid
 * for the hard pass, 11 x 11 on a step-6 grid for the Wiener pass); images of
 * one call then run in groups of equal regime. */
typedef struct {
    int patch;       /* patch side: 8 (all kernels) or 11, 12 (FP32 kernels)   */
    int step;        /* reference grid step (3): 0, step, ... plus L-patch     */
    int search;      /* odd side of the search window of top-left corners (39) */
    int n2;          /* largest group size, a power of two in [1, 32]          */
    float tau;       /* keep candidates with d <= tau (sigma <= 40)            */
    float tau_high;  /* tau used when sigma > 40 and sigma_regime == 0         */
    float lambda3d;  /* hard threshold lambda3d * sigma (first pass only)      */
    float beta;      /* Kaiser window beta for aggregation                     */
    float lambda2d;  /* first pass, sigma > 40 and sigma_regime == 0: match on
                        2D-prethresholded patches, coefficients of magnitude
                        <= lambda2d * sigma zeroed (BM3D's high-noise distance;
                        0 disables; ignored by the second pass)              */
    int patch_high;  /* patch side when sigma > 40 and sigma_regime == 0: 0
                        (= patch), 8, 11 or 12; a prethresholded first pass
                        (lambda2d > 0) takes 8 or 12 with n2 <= 16          */
    int step_high;   /* grid step then (0 = step)                              */
} dn_bm3d_pass;

typedef struct {
    dn_bm3d_pass hard;    /* first pass: hard thresholding  (n2 16, tau 2500) */
    dn_bm3d_pass wiener;  /* second pass: Wiener filtering  (n2 32, tau 400)  */
    int precision;        /* dn_precision bits: DN_BF16, DN_BF16_MATCH          */
    int sigma_regime;     /* 0: tau_high above sigma 40; 1: tau at every sigma */
} dn_bm3d_params;

typedef struct {
    int patch;           /* odd patch side (7)                 */
    int search;          /* odd search window side (21)        */
    float h_over_sigma;  /* filtering parameter h / sigma (0.4) */
} dn_nlm_params;

/* Residual CNN of Sec. II (Fig. 1): `layers` 3x3 convolutions, the first
 * `layers-1` followed by ReLU, `width` hidden channels, 2 cc input channels
 * (prefilter/255 and noisy/255 for each of cc colour planes, Eq. 3) and cc
 * output channels r; the result is prefilter + 255 r (Eq. 2).
 * channels = 1 (or 0): the grey network (cc = 1), run on each channel of a
 * colour image; channels = 3: a colour-native network (cc = 3, 6 -> width ->
 * ... -> 3) for RGB images.
 * `weights` is a DEVICE pointer to FP32 parameters, layer by layer:
 *   W_l [Cout][3][3][Cin] then b_l [Cout]; see dn_cnn_param_count_c(). */
typedef struct {
    int layers;            /* K >= 2 (10) */
    int width;             /* hidden channels, 32 (the BF16 path takes 32 or 64) */
    const float *weights;  /* device, caller-owned */
    int precision;         /* DN_FP32: FP32 SIMT kernels; DN_BF16: tcgen05 BF16 */
    int channels;          /* 0 or 1: grey network per channel; 3: colour-native network */
} dn_cnn;

/* ---- parameters ---------------------------------------------------------- */

/* Defaults: hard {8, 3, 39, 16, 2500, 5000, 2.7, 2, 2, 0, 0}, wiener {8, 3, 39,
 * 32, 400, 3500, 0, 2, 0, 0, 0}, precision DN_FP32, sigma_regime 0. */
void dn_bm3d_default_params(dn_bm3d_params *p);
/* The defaults with the larger patches of BM3D's high-noise profile above
 * sigma 40: hard patch_high 12, step_high 4; wiener patch_high 11, step_high 6. */
void dn_bm3d_high_noise_params(dn_bm3d_params *p);
/* Defaults: {7, 21, 0.4}. */
void dn_nlm_default_params(dn_nlm_params *p);
/* Number of floats in a dn_cnn weight buffer (grey network, channels = 1). */
size_t dn_cnn_param_count(int layers, int width);
/* The same for `channels` colour planes (1 or 3). */
size_t dn_cnn_param_count_c(int layers, int width, int channels);
/* Number of reference positions along an axis of length L (grid 0, step, ...
 * plus L - patch); writes them to pos[] when pos != NULL.  0 if L < patch. */
int dn_bm3d_grid(int L, int patch, int step, int *pos);

/* ---- workspace queries (bytes, 256-byte aligned sub-buffers) ------------ */

size_t dn_bm3d_workspace_bytes(int B, int C, int H, int W, const dn_bm3d_params *p);
size_t dn_nlm_workspace_bytes(int B, int C, int H, int W, const dn_nlm_params *p);
size_t dn_hybrid_workspace_bytes(int B, int C, int H, int W, int prefilter, const void *prefilter_params,
                                 const dn_cnn *cnn);

/* ---- the three denoisers ------------------------------------------------- */

/* BM3D, both passes (standard definition; the paper's BM3D-G stage, Sec. II).
 * noisy/out: device [B][C][H][W] (may not alias); H, W >= every patch side
 * an image's regime selects (DN_EINVAL otherwise).
 * DN_EUNSUPPORTED (before any launch) when an image takes the high-noise
 * first pass (sigma > 40, sigma_regime 0, hard.lambda2d > 0) and the
 * prethresholded matcher's staged window, (31 step + search) columns wide
 * for 8 x 8 patches, (15 step + search) for 12 x 12, does not fit in 200 KB
 * of shared memory (for example step 12 with search 21 on an image wider
 * than 400 pixels), or its patch side or group size is not one it takes
 * (11, or n2 = 32 with 12); the same holds for denoise_hybrid and
 * denoise_bm3d_noalloc. */
dn_status denoise_bm3d(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                       const dn_bm3d_params *p, void *workspace, size_t ws_bytes, dn_stream_t stream);

/* NL-means (the paper's NLM-G stage, Sec. IV-A): for each pixel, the average
 * of the search window weighted by w = exp(-max(d2 - 2 sigma^2, 0) / h^2),
 * d2 the mean squared difference of the patch x patch neighbourhoods
 * (half-sample symmetric reflection at the border), h = h_over_sigma *
 * sigma; colour weights come from Y.  H, W >= 4. */
dn_status denoise_nlm(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                      const dn_nlm_params *p, void *workspace, size_t ws_bytes, dn_stream_t stream);

/* Nonlocal filter then residual CNN (Sec. II, Eq. 2-3).  prefilter_params
 * points to a dn_bm3d_params (DN_PREFILTER_BM3D) or dn_nlm_params. */
dn_status denoise_hybrid(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                         int prefilter, const void *prefilter_params, const dn_cnn *cnn,
                         void *workspace, size_t ws_bytes, dn_stream_t stream);

const char *dn_strerror(dn_status s);

/* ---- one large image in tiles with a halo ---------------------------------
 * A BM3D output pixel depends only on the noisy pixels within a fixed
 * distance (per axis) of it: a pass-1 estimate at p comes from the groups
 * whose reference lies within search/2 + k - 1 of p (k the patch side), and
 * each group's matching and filtering read pixels within another
 * search/2 + k - 1 of its reference; the second pass does the same on the
 * basic estimate.  So a tile extended by that radius on every side (clipped
 * at the image border), with its origin on the reference grids, yields exactly the whole-image result inside
 * its interior: every kernel here is deterministic and the aggregation sums
 * are exact, so the tiled result equals denoise_bm3d bit for bit.  This bounds
 * the workspace of very large images (and shards one image across devices,
 * each processing its tiles). */

/* The radius: (2 (hard.search / 2) + k1 - 1) + (2 (wiener.search / 2) + k2 - 1),
 * k the larger patch side a pass takes in either regime (patch, patch_high):
 * 90 for the defaults, 97 with dn_bm3d_high_noise_params; -1 for invalid
 * parameters.  Tile origins lie on every grid step either regime uses. */
int dn_bm3d_halo(const dn_bm3d_params *p);

/* Workspace of denoise_bm3d_tiled (0 for invalid arguments). */
size_t dn_bm3d_tiled_workspace_bytes(int C, int H, int W, const dn_bm3d_params *p, int tile, int max_batch);

/* BM3D of ONE image noisy/out: device [C][H][W], in tiles whose interiors
 * are tile x tile pixels (rounded up to a multiple of both grid steps),
 * each extended by the halo (rounded likewise); tiles of equal extent run
 * together, up to max_batch per launch.  Same result as denoise_bm3d. */
dn_status denoise_bm3d_tiled(const float *noisy, float *out, int C, int H, int W, float sigma,
                             const dn_bm3d_params *p, int tile, int max_batch, void *workspace, size_t ws_bytes,
                             dn_stream_t stream);

/* BM3D without any device allocation, for callers that may not allocate
 * device memory themselves (for example a plug-in inside an application that
 * owns the whole device-memory budget, or a latency-critical loop that cannot
 * risk an allocation blocking on the device).  The paper has no counterpart;
 * this is a deployment convenience.
 * Same arguments and results as denoise_bm3d, minus the workspace: the
 * workspace is a fixed array of DN_NOALLOC_SCRATCH_BYTES of device memory
 * inside this library.  Requests whose dn_bm3d_workspace_bytes exceeds that
 * size (for example a 1 x 1 x 512 x 512 image fits, 1 x 3 x 512 x 512 does
 * not) return DN_ENOMEM before any launch.
 * Reservation: under lazy module loading (CUDA's default) the array is
 * reserved on a device when the library's device code is first loaded there,
 * which can be this entry point's first call on that device; it then stays
 * reserved until the process exits.  Make that first call a warm-up call
 * before any stream capture and before the application takes the rest of the
 * device memory: it returns DN_ECUDA when the device has no room left for the
 * array.  Every call looks the array's device address up in the current
 * context (cudaGetSymbolAddress), so a device reset between calls is safe.
 * Every call on a device shares the one array, and the array keeps the
 * previous call's contents (the call clears what must start at zero itself):
 * calls that may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  No cudaMalloc / cudaFree is made. */
#define DN_NOALLOC_SCRATCH_BYTES (16u << 20)
/* The size of that array in bytes (DN_NOALLOC_SCRATCH_BYTES of this build). */
size_t dn_noalloc_scratch_bytes(void);
dn_status denoise_bm3d_noalloc(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                               const dn_bm3d_params *p, dn_stream_t stream);

/* ---- stage entry points (same kernels, exposed for stage-wise checks) ---- */

/* Block matching of every reference patch of a guide plane.
 * guide: device, plane b at guide + b * plane_stride, [H][W].
 * tau: host [B] (threshold actually applied to image b).
 * idx: device int32 [B][Ry][Rx][p->n2]: member 0 is the reference itself,
 *      then the other candidates with d <= tau in ascending (d, y*W + x)
 *      order; -1 past the kept count.
 * n:   device int32 [B][Ry][Rx]: group size min(n2, 2^floor(log2 #kept)).
 * Patches of side p->patch (8, 11 or 12) on the grid of step p->step; the
 * distance is ||P - Q||^2 / patch^2.
 * precision: DN_FP32 (exhaustive FP32), or DN_BF16_MATCH (DN_BF16 is taken
 * as the same): tensor-core prefilter with a proven margin, survivors
 * re-ranked exactly in FP32, so the lists equal the FP32 ones (8 x 8 patches;
 * other sides are matched in FP32). */
dn_status dn_bm3d_match(const float *guide, size_t plane_stride, int B, int H, int W, const dn_bm3d_pass *p,
                        const float *tau, int precision, int *idx, int *n, void *workspace, size_t ws_bytes,
                        dn_stream_t stream);
size_t dn_bm3d_match_workspace_bytes(int B, int H, int W, const dn_bm3d_pass *p, int precision);

/* Block matching on 2D-prethresholded patches (the first-pass distance BM3D
 * uses at high noise; the denoisers select it per image, see
 * dn_bm3d_pass.lambda2d): every patch P (side k = p->patch, 8 or 12) becomes
 * Y(P), its orthonormal k x k DCT-II with the coefficients of magnitude
 * <= thr[b] set to zero, and d(P, Q) = ||Y(P) - Y(Q)||^2 / k^2; window, tau
 * test, ordering and group size as dn_bm3d_match.  guide as dn_bm3d_match;
 * tau, thr: host [B] (tau > 0, thr >= 0); idx/n as dn_bm3d_match with p->n2.
 * FP32 transforms and distances; no workspace.  DN_EUNSUPPORTED when the
 * staged window exceeds shared memory, for side 11, and for side 12 with
 * n2 = 32 (search > 127 is already DN_EINVAL). */
dn_status dn_bm3d_match_prethresh(const float *guide, size_t plane_stride, int B, int H, int W,
                                  const dn_bm3d_pass *p, const float *tau, const float *thr, int *idx, int *n,
                                  dn_stream_t stream);

/* Test surface of the tensor-core matching prefilter: runs dn_bm3d_match
 * (DN_BF16_MATCH) on one image and additionally writes, for the reference tile
 * (tile_x, tile_y) (8 x 16 grid positions), cross[0] = m, the constant the
 * tile's pixels are centred on, then the raw FP32 tensor-core results
 * sum_k f16(P - m)[k] f16(Q - m)[k] at cross[1 + (t * nchunks + c) * 128 + j]:
 * reference t = (ty * 8 + tx) of the tile against the candidate at row
 * 2 c + j / 64, column j % 64 of the tile's candidate region, whose origin is
 * (max(0, y_first - search/2), max(0, x_first - search/2)) with
 * (y_first, x_first) the tile's first grid position; nchunks = ceil(region
 * rows / 2).  idx/n as in dn_bm3d_match; workspace as
 * dn_bm3d_match_workspace_bytes(1, H, W, p, DN_BF16_MATCH). */
dn_status dn_bm3d_match_cross_terms(const float *guide, int H, int W, const dn_bm3d_pass *p, float tau, int tile_x,
                                    int tile_y, float *cross, int *idx, int *n, void *workspace, size_t ws_bytes,
                                    dn_stream_t stream);

/* Collaborative hard thresholding + aggregation (first pass) given match lists.
 * img: device [B][C][H][W] (already in the filtering colour space);
 * sigma_c: host [B*C] per-channel noise std; idx/n as produced by
 * dn_bm3d_match with p->n2 (patches of side p->patch, grid step p->step);
 * basic: device [B][C][H][W].
 * precision: DN_FP32 (FP32 SIMT transforms) or DN_BF16 (2D transforms of 8 x 8
 * patches on the tensor cores, see dn_precision; DN_EDEVICE-class failures
 * set the device status word, see dn_device_error).
 * workspace >= dn_bm3d_filter_workspace_bytes(B, C, H, W). */
dn_status dn_bm3d_filter_hard(const float *img, const int *idx, const int *n, int B, int C, int H, int W,
                              const float *sigma_c, const dn_bm3d_pass *p, int precision, float *basic,
                              void *workspace, size_t ws_bytes, dn_stream_t stream);

/* Collaborative Wiener filtering + aggregation (second pass) given match
 * lists computed on the basic estimate. */
dn_status dn_bm3d_filter_wiener(const float *noisy, const float *basic, const int *idx, const int *n,
                                int B, int C, int H, int W, const float *sigma_c, const dn_bm3d_pass *p,
                                int precision, float *out, void *workspace, size_t ws_bytes,
                                dn_stream_t stream);
size_t dn_bm3d_filter_workspace_bytes(int B, int C, int H, int W);

/* RGB <-> YCbCr (full-range BT.601 rows; offsets omitted), device
 * [B][3][H][W], in place allowed. */
dn_status dn_rgb_to_ycc(const float *in, float *out, int B, int H, int W, dn_stream_t stream);
dn_status dn_ycc_to_rgb(const float *in, float *out, int B, int H, int W, dn_stream_t stream);

/* Per-image error reduction, FP64 on the device: sse[b] = sum over C*H*W of
 * (clip(out, 0, 255) - ref)^2 and maxerr[b] = max |out - ref| (unclipped).
 * sse, maxerr: device double [B]. */
dn_status dn_error_reduce(const float *out, const float *ref, int B, size_t chw, double *sse, double *maxerr,
                          dn_stream_t stream);

/* ---- CNN layers (training and checks) ----------------------------------- */

/* y = conv3x3(x, w) + b, optional ReLU.  FP32, NCHW: x [N][Cin][H][W],
 * w [Cout][3][3][Cin], b [Cout] (may be NULL), y [N][Cout][H][W]. */
dn_status dn_conv3x3_fwd(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout,
                         int H, int W, int relu, dn_stream_t stream);
/* dx = conv3x3^T(dy, w) (zero padding); if mask != NULL, dx *= (mask > 0)
 * elementwise (the ReLU of the layer that produced x).  dx [N][Cin][H][W]. */
dn_status dn_conv3x3_bwd_data(const float *dy, const float *w, const float *mask, float *dx, int N, int Cin,
                              int Cout, int H, int W, dn_stream_t stream);
/* dw = sum_{n,y,x} dy (x) x_shifted, db = sum dy; OVERWRITES dw and db. */
dn_status dn_conv3x3_bwd_weight(const float *x, const float *dy, float *dw, float *db, int N, int Cin, int Cout,
                                int H, int W, dn_stream_t stream);

/* Gradient of the L1 loss of Eq. 2 for the grey network of width 32
 * (cnn->precision DN_BF16, channels 1) with BF16 tensor-core kernels: the
 * forward keeps every activation (NHWC BF16); dL/dr = 255 sign(out - clean)
 * / count; the hidden layers' weight gradients are tcgen05 GEMMs over the
 * pixels (BF16 operands, FP32 accumulation), their data gradients the
 * transposed convolution on tcgen05 (flipped weights) with the ReLU mask in
 * its epilogue; the thin first and last layers run on CUDA cores; every sum
 * over pixels is a fixed-order sum of per-CTA partials (reproducible).
 * noisy, pre, clean: device [N][H][W]; grad: device FP32 in the layout of
 * cnn->weights, OVERWRITTEN; loss_sum: device double [1], += sum |out -
 * clean| (caller zeroes).  The FP32 master weights are cnn->weights.
 * DN_EUNSUPPORTED for other precisions, widths or colour-native networks
 * (the FP32 layer entry points below cover those). */
dn_status dn_cnn_grad(const float *noisy, const float *pre, const float *clean, int N, int H, int W, const dn_cnn *cnn,
                      float *grad, double *loss_sum, void *workspace, size_t ws_bytes, dn_stream_t stream);
size_t dn_cnn_grad_workspace_bytes(int N, int H, int W, const dn_cnn *cnn);

/* Full network forward (Eq. 2-3), FP32 or BF16: noisy, pre, out: device
 * [N][cc][H][W] with cc = 3 for a colour-native network (channels = 3), else
 * cc = 1; out = pre + 255 F([pre, noisy]/255).
 * workspace >= dn_cnn_workspace_bytes(N, H, W, cnn). */
dn_status dn_cnn_forward(const float *noisy, const float *pre, float *out, int N, int H, int W, const dn_cnn *cnn,
                         void *workspace, size_t ws_bytes, dn_stream_t stream);
size_t dn_cnn_workspace_bytes(int N, int H, int W, const dn_cnn *cnn);

/* One hidden C -> C layer on the tensor cores (tcgen05, BF16 x BF16 -> FP32),
 * C = 32 or 64: x, y: device NHWC bf16 [N][H][W][C] (2 C bytes per pixel,
 * 16-byte aligned); w: device FP32 [C][3][3][C] (rounded to BF16 inside),
 * b: device FP32 [C]; y = conv3x3(x, w) + b, ReLU when relu != 0, rounded to
 * BF16.  workspace: device, >= 9 * C * C * 2 bytes (packed weights). */
dn_status dn_conv3x3_tc_fwd(const void *x, const float *w, const float *b, void *y, int N, int H, int W, int C,
                            int relu, void *workspace, size_t ws_bytes, dn_stream_t stream);

/* Two hidden C -> C layers (C = 32) in one pass on the tensor cores:
 * y = ReLU(conv_b(ReLU(conv_a(x) + ba)) + bb), the intermediate rounded to
 * bf16 exactly as dn_conv3x3_tc_fwd rounds its output but kept in shared
 * memory (bit-identical to two dn_conv3x3_tc_fwd calls with relu = 1).
 * x, y: NHWC bf16 [N][H][W][C]; wa, wb: FP32 [C][3][3][C]; ba, bb: FP32 [C];
 * workspace >= 2 * 9 * C * C * 2 bytes (packed weights). */
dn_status dn_conv3x3_tc_pair_fwd(const void *x, const float *wa, const float *ba, const float *wb, const float *bb,
                                 void *y, int N, int H, int W, int C, void *workspace, size_t ws_bytes,
                                 dn_stream_t stream);

/* Backward of one hidden C -> C layer on the tensor cores (NHWC bf16, as
 * dn_conv3x3_tc_fwd), the two halves of dn_cnn_grad's hidden-layer step:
 *   weight: dw [C][3][3][C] = sum_px g[px][co] x[px + tap - 1][ci] and
 *           db [C] = sum_px g[px][co] (FP32, overwritten; C = 32), a tcgen05
 *           GEMM over the pixels with BF16 operands and FP32 accumulation;
 *   data:   dx = conv3x3^T(g, w) (zero padding) on tcgen05 with the weights
 *           flipped and transposed, rounded to bf16; where mask (NHWC bf16,
 *           or NULL) is not positive the result is 0 (the ReLU of the layer
 *           input).  C = 32 or 64.
 * workspace >= dn_conv3x3_tc_bwd_workspace_bytes(N, H, W, C). */
size_t dn_conv3x3_tc_bwd_workspace_bytes(int N, int H, int W, int C);
dn_status dn_conv3x3_tc_bwd_weight(const void *x, const void *g, float *dw, float *db, int N, int H, int W, int C,
                                   void *workspace, size_t ws_bytes, dn_stream_t stream);
dn_status dn_conv3x3_tc_bwd_data(const void *g, const float *w, const void *mask, void *dx, int N, int H, int W, int C,
                                 void *workspace, size_t ws_bytes, dn_stream_t stream);

/* ---- layers of the flexible lightweight network (Sec. III, "Ours-FL") -----
 * A U-Net of depthwise-separable 3x3 convolutions with stride-2 downsampling,
 * 2x2 transposed-convolution upsampling and additive skips, whose input
 * carries the noise level as a plane (the paper gives the structure, not the
 * widths).  All tensors are DEVICE float32, NCHW, contiguous; FP32 CUDA-core
 * kernels; results are deterministic (fixed reduction orders). */

/* Depthwise 3x3, zero padding 1, stride 1 or 2: y [N][C][Ho][Wo], Ho = ceil(H / stride),
 * y = b[c] + sum_{i,j} w[c][i][j] x[n][c][stride yo + i - 1][stride xo + j - 1],
 * then ReLU when relu != 0.  w [C][3][3]; b [C] or NULL. */
dn_status dn_dw3x3_fwd(const float *x, const float *w, const float *b, float *y, int N, int C, int H, int W,
                       int stride, int relu, dn_stream_t stream);
/* Gradients of the depthwise layer (before any ReLU) given g = dL/dy [N][C][Ho][Wo]:
 * dx [N][C][H][W] (skipped when NULL), dw [C][3][3], db [C] (skipped when NULL);
 * dw and db are overwritten. */
dn_status dn_dw3x3_bwd(const float *x, const float *g, const float *w, float *dx, float *dw, float *db, int N, int C,
                       int H, int W, int stride, dn_stream_t stream);
/* Pointwise (1x1): y [N][Cout][HW] = b[co] + sum_ci w[co][ci] x[n][ci][p], ReLU when
 * relu != 0; w [Cout][Cin], b [Cout] or NULL.  transposed != 0 multiplies by the
 * transpose of a [Cin][Cout] weight instead (the data gradient of a Cout -> Cin layer). */
dn_status dn_pw_fwd(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                    int relu, int transposed, dn_stream_t stream);
/* The same two contractions on the tensor cores (tcgen05): x and w rounded
 * to BF16, products accumulated in FP32, FP32 in and out; Cin, Cout <= 256.
 * Per output |y - exact| <= (2^-7 + 2^-14) sum_ci |w| |x| (two roundings of
 * unit roundoff 2^-8, FP32 accumulation). */
dn_status dn_pw_fwd_bf16(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int HW,
                         int relu, int transposed, dn_stream_t stream);
dn_status dn_deconv2x2_fwd_bf16(const float *x, const float *w, const float *b, const float *skip, float *y, int N,
                                int Cin, int Cout, int H, int W, dn_stream_t stream);
/* dw [Cout][Cin] = sum_{n,p} g[n][co][p] x[n][ci][p]; db [Cout] = sum g (NULL: skipped). */
dn_status dn_pw_bwd_weight(const float *x, const float *g, float *dw, float *db, int N, int Cin, int Cout, int HW,
                           dn_stream_t stream);
/* Transposed 2x2 convolution, stride 2: y [N][Cout][2H][2W],
 * y[n][co][2i+a][2j+c] = b[co] + skip[n][co][2i+a][2j+c] + sum_ci w[ci][co][a][c] x[n][ci][i][j];
 * w [Cin][Cout][2][2] (16-byte aligned), b and skip may be NULL. */
dn_status dn_deconv2x2_fwd(const float *x, const float *w, const float *b, const float *skip, float *y, int N, int Cin,
                           int Cout, int H, int W, dn_stream_t stream);
/* Gradients of the transposed convolution given g [N][Cout][2H][2W]: dx [N][Cin][H][W]
 * (NULL: skipped), dw [Cin][Cout][2][2], db [Cout] (NULL: skipped). */
dn_status dn_deconv2x2_bwd(const float *x, const float *g, const float *w, float *dx, float *dw, float *db, int N,
                           int Cin, int Cout, int H, int W, dn_stream_t stream);
/* Network input with the noise-level map: z [N][3][H][W] = [pre / 255, noisy / 255,
 * sigma_n / 255]; sigma a HOST array of N floats in [0, 255]. */
dn_status dn_fl_pack_input(const float *pre, const float *noisy, const float *sigma, float *z, int N, int H, int W,
                           dn_stream_t stream);

/* Reads (and with reset != 0 clears) the library's device error word on the
 * current device: nonzero when a kernel's bounded wait on the tensor-core
 * pipeline ran out.  Synchronous (waits for the device). */
dn_status dn_device_error(int *code, int reset);

/* Network input of Eq. 3 on planes: z [N][2][H][W] = [pre / 255, noisy / 255]. */
dn_status dn_cnn_pack_input(const float *pre, const float *noisy, float *z, int N, int H, int W, dn_stream_t stream);
/* Output of Eq. 2: out = pre + 255 r (count floats). */
dn_status dn_cnn_residual_out(const float *pre, const float *r, float *out, size_t count, dn_stream_t stream);
/* ReLU backward: out = g where y > 0, else 0 (count floats). */
dn_status dn_relu_bwd(const float *g, const float *y, float *out, size_t count, dn_stream_t stream);

/* L1 loss of Eq. 2 on the residual r: with out = pre + 255 r,
 * dr = 255 sign(out - clean) / count (0 where equal); loss_sum (device double
 * [1], accumulated, caller zeroes) += sum |out - clean|. */
dn_status dn_l1_residual_grad(const float *r, const float *pre, const float *clean, float *dr, size_t count,
                              double *loss_sum, dn_stream_t stream);
/* Adam (Kingma & Ba) on count floats, step t >= 1 (bias correction). */
dn_status dn_adam_step(float *param, const float *grad, float *m, float *v, size_t count, int t, float lr,
                       float beta1, float beta2, float eps, dn_stream_t stream);

/* ---- timing of individual kernels --------------------------------------- */

/* When enabled, every kernel launch of this library on this host thread is
 * bracketed by CUDA events on its own stream; dn_profile_read synchronises
 * those events and returns, per kernel name, the launch count and the summed
 * device milliseconds.  Disabled by default (no events recorded). */
void dn_profile_enable(int on);
int dn_profile_read(char *names, int name_stride, int max_kernels, int *launches, double *ms);
void dn_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* DENOISE_H */

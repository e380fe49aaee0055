// C ABI of libdenoise: argument validation, workspace layout and the
// composition of the kernels into the three denoisers.  See
// include/denoise.h for the contract of every entry point.
#include <climits>
#include <cmath>
#include <cstring>

#include "common.cuh"

using namespace dn;

namespace {

const double kYccRows[3][3] = {{0.299, 0.587, 0.114}, {-0.168736, -0.331264, 0.5}, {0.5, -0.418688, -0.081312}};

// Noise std of channel c after the colour transform of white RGB noise.
float channel_sigma(float sigma, int C, int c)
{
    if (C == 1) return sigma;
    const double *r = kYccRows[c];
    return (float)(sigma * std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]));
}

bool valid_image(int B, int C, int H, int W, int min_side)
{
    return B >= 1 && (C == 1 || C == 3) && H >= min_side && W >= min_side && (size_t)H * W <= (size_t)INT_MAX;
}

bool valid_sigmas(const float *sigma, int B)
{
    if (!sigma) return false;
    for (int b = 0; b < B; ++b)
        if (!(sigma[b] > 0.0f) || !(sigma[b] <= 255.0f)) return false;
    return true;
}

bool patch_side_ok(int k) { return k == 8 || large_patch_supported(k); }

bool valid_pass(const dn_bm3d_pass *p)
{
    if (!p) return false;
    if (!patch_side_ok(p->patch) || p->step < 1 || p->search < 1 || (p->search & 1) == 0 || p->search > 127)
        return false;
    if ((p->patch_high != 0 && !patch_side_ok(p->patch_high)) || p->step_high < 0 || p->step_high > 64) return false;
    if (p->n2 < 1 || p->n2 > 32 || (p->n2 & (p->n2 - 1)) != 0) return false;
    if (!(p->tau > 0.0f) || !(p->tau_high > 0.0f) || !(p->lambda3d >= 0.0f) || !(p->beta >= 0.0f)) return false;
    if (!(p->lambda2d >= 0.0f) || !std::isfinite(p->lambda2d)) return false;
    return true;
}

bool valid_bm3d(const dn_bm3d_params *p)
{
    return p && valid_pass(&p->hard) && valid_pass(&p->wiener) && p->precision >= 0 &&
           p->precision <= (DN_BF16 | DN_BF16_MATCH) &&
           (p->sigma_regime == 0 || p->sigma_regime == 1);
}

bool valid_nlm(const dn_nlm_params *p)
{
    return p && p->patch >= 1 && (p->patch & 1) && p->patch <= 15 && p->search >= 1 && (p->search & 1) &&
           p->search <= 41 && p->h_over_sigma > 0.0f && std::isfinite(p->h_over_sigma);
}

bool valid_cnn(const dn_cnn *c)
{
    return c && c->weights && c->layers >= 2 && c->layers <= 64 && c->width >= 1 && c->width <= 64 &&
           (c->precision == DN_FP32 || c->precision == DN_BF16) &&
           (c->channels == 0 || c->channels == 1 || c->channels == 3);
}

// Colour planes the network takes and produces (1: grey network).
int cnn_cc(const dn_cnn *c) { return c->channels == 3 ? 3 : 1; }

// Whether image noise sigma takes the high-noise settings (tau_high, the
// prethresholded first-pass distance, patch_high and step_high).
bool is_high(const dn_bm3d_params *p, float sigma) { return p->sigma_regime == 0 && sigma > 40.0f; }

// The pass as an image of that regime runs it: tau, patch side and step
// resolved; lambda2d kept only for a high-noise first pass.
dn_bm3d_pass pass_at(const dn_bm3d_pass &p, bool high, bool first)
{
    dn_bm3d_pass q = p;
    if (high) {
        q.tau = p.tau_high;
        if (p.patch_high > 0) q.patch = p.patch_high;
        if (p.step_high > 0) q.step = p.step_high;
    }
    q.lambda2d = (first && high) ? p.lambda2d : 0.0f;
    q.patch_high = q.patch;
    q.step_high = q.step;
    return q;
}

// Smallest image side every image of the call can take: the largest patch side
// its regime selects in either pass.
bool sides_ok(int B, int H, int W, const float *sigma, const dn_bm3d_params *p)
{
    for (int b = 0; b < B; ++b) {
        const bool hi = is_high(p, sigma[b]);
        const int k1 = pass_at(p->hard, hi, true).patch, k2 = pass_at(p->wiener, hi, false).patch;
        const int k = k1 > k2 ? k1 : k2;
        if (H < k || W < k) return false;
    }
    return true;
}

// The high-noise first pass (prethresholded patches) stages a window as wide
// as the CTA's union of search windows in shared memory; wide windows with
// large steps do not fit, and only some patch sides and group sizes are
// built.  Checked on the host before any launch.
bool prethresh_fits(int B, int W, const float *sigma, const dn_bm3d_params *p)
{
    for (int b = 0; b < B; ++b) {
        if (!is_high(p, sigma[b])) continue;
        const dn_bm3d_pass h = pass_at(p->hard, true, true);
        if (!(h.lambda2d > 0.0f)) return true;
        if (h.patch == 8) return match_pre_smem_bytes(W, h) <= 200 * 1024;
        return large_prethresh_supported(h.patch) && h.n2 <= 16 && match_pre_large_smem_bytes(W, h) <= 200 * 1024;
    }
    return true;
}

// ---- workspace layouts (a null base computes the size) -------------------------

struct Bm3dWs {
    float *ycc;
    int *idx;
    int *n;
    float *acc;
    float *basic;
    int *mws;  // tensor-core matcher: deferred-reference list
    size_t bytes;
};

// Reference count of a pass in either regime (the larger).
size_t refs_max(const dn_bm3d_pass &p, int H, int W)
{
    size_t r = 0;
    for (int hi = 0; hi < 2; ++hi) {
        const dn_bm3d_pass q = pass_at(p, hi != 0, false);
        const size_t v = (size_t)grid_count(H, q.patch, q.step) * grid_count(W, q.patch, q.step);
        r = v > r ? v : r;
    }
    return r;
}

Bm3dWs bm3d_layout(void *base, int B, int C, int H, int W, const dn_bm3d_params *p)
{
    Carver cv(base);
    const size_t HW = (size_t)H * W, R = refs_max(p->hard, H, W), R2 = refs_max(p->wiener, H, W);
    const size_t Rm = R > R2 ? R : R2;
    const int n2 = p->hard.n2 > p->wiener.n2 ? p->hard.n2 : p->wiener.n2;
    Bm3dWs w;
    w.ycc = C == 3 ? cv.take<float>((size_t)B * 3 * HW) : nullptr;
    w.idx = cv.take<int>((size_t)B * Rm * n2);
    w.n = cv.take<int>((size_t)B * Rm);
    w.acc = cv.take<float>(kAccBytesPerPixel / sizeof(float) * (size_t)B * C * HW);
    w.basic = cv.take<float>((size_t)B * C * HW);
    // the tensor-core matcher's deferred-reference list, for every 8 x 8 pass either regime runs
    size_t mt = 0;
    for (int hi = 0; hi < 2; ++hi) {
        const dn_bm3d_pass q[2] = {pass_at(p->hard, hi != 0, false), pass_at(p->wiener, hi != 0, false)};
        for (const dn_bm3d_pass &e : q)
            if (e.patch == 8) {
                const size_t m = match_tc_workspace_bytes(B, H, W, e);
                mt = m > mt ? m : mt;
            }
    }
    w.mws = (p->precision & DN_BF16_MATCH) && mt > 0 ? cv.take<int>(mt / sizeof(int)) : nullptr;
    w.bytes = cv.off;
    return w;
}

struct NlmWs {
    float *ycc;
    float *tmp;
    size_t bytes;
};

NlmWs nlm_layout(void *base, int B, int C, int H, int W)
{
    Carver cv(base);
    NlmWs w;
    const size_t n = C == 3 ? (size_t)B * 3 * H * W : 0;
    w.ycc = C == 3 ? cv.take<float>(n) : nullptr;
    w.tmp = C == 3 ? cv.take<float>(n) : nullptr;
    w.bytes = cv.off;
    return w;
}

struct CnnWs {
    float *z;        // FP32 path: packed input [N][2 cc][H][W]
    float *act[2];   // FP32: [N][width][H][W]; BF16: NHWC [N][H][W][width] bf16
    char *wpack;     // BF16: packed B operands of the hidden layers
    size_t bytes;
};

// Packed B operand of one width x width hidden layer ([tap][chunk][cout][8] bf16).
size_t wpack_bytes(int width) { return (size_t)9 * width * width * 2; }

CnnWs cnn_layout(void *base, int N, int H, int W, const dn_cnn *c)
{
    Carver cv(base);
    const size_t HW = (size_t)H * W;
    CnnWs w;
    if (c->precision == DN_BF16) {
        w.z = nullptr;
        w.act[0] = reinterpret_cast<float *>(cv.take<char>((size_t)N * HW * c->width * 2));
        w.act[1] = reinterpret_cast<float *>(cv.take<char>((size_t)N * HW * c->width * 2));
        w.wpack = cv.take<char>(wpack_bytes(c->width) * (size_t)(c->layers > 2 ? c->layers - 2 : 1));
    } else {
        w.z = cv.take<float>((size_t)N * 2 * cnn_cc(c) * HW);
        w.act[0] = cv.take<float>((size_t)N * c->width * HW);
        w.act[1] = cv.take<float>((size_t)N * c->width * HW);
        w.wpack = nullptr;
    }
    w.bytes = cv.off;
    return w;
}

// Block matching in the requested precision: with DN_BF16_MATCH the BF16
// tensor-core prefilter with exact FP32 re-rank (same result as FP32) when its
// tiling supports the parameters, the exhaustive FP32 kernel otherwise; the
// larger patch sides on their own FP32 kernel.
bool tc_match_supported(const dn_bm3d_pass &p) { return p.patch == 8 && match_tc_supported(p); }

dn_status match_any(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p, const float *tau,
                    int precision, int *idx, int *n, int *mws, cudaStream_t s)
{
    if (p.patch != 8) return match_large(guide, plane, B, H, W, p, tau, idx, n, s);
    if ((precision & DN_BF16_MATCH) && mws && tc_match_supported(p)) {
        int *err = device_error_ptr();
        if (!err) return DN_ECUDA;
        return match_tc(guide, plane, B, H, W, p, tau, idx, n, err, mws, s);
    }
    return match_fp32(guide, plane, B, H, W, p, tau, idx, n, s);
}

// Matching on 2D-prethresholded patches (threshold thr[b]) for the patch
// side of p.
dn_status match_prethresh_any(const float *guide, size_t plane, int B, int H, int W, const dn_bm3d_pass &p,
                              const float *tau, const float *thr, int *idx, int *n, cudaStream_t s)
{
    if (p.patch == 8) return match_prethresh(guide, plane, B, H, W, p, tau, thr, idx, n, s);
    return match_prethresh_large(guide, plane, B, H, W, p, tau, thr, idx, n, s);
}

// Collaborative filtering (pass 1, or pass 2 when `wiener`) with the 2D
// transforms on the tensor cores when `tc` (8 x 8 patches), FP32 SIMT
// otherwise.
dn_status filter_any(bool wiener, bool tc, const float *img, const float *basic, const int *idx, const int *n, int B,
                     int C, int H, int W, const float *sig, const dn_bm3d_pass &p, float *acc, cudaStream_t s)
{
    if (p.patch != 8) return filter_large(wiener, img, basic, idx, n, B, C, H, W, sig, p, acc, s);
    if (tc) {
        int *err = device_error_ptr();
        if (!err) return DN_ECUDA;
        return filter_tc(wiener, img, basic, idx, n, B, C, H, W, sig, p, acc, err, s);
    }
    return wiener ? filter_wiener_fp32(img, basic, idx, n, B, C, H, W, sig, p, acc, s)
                  : filter_hard_fp32(img, idx, n, B, C, H, W, sig, p, acc, s);
}

dn_status run_bm3d(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                   const dn_bm3d_params *p, const Bm3dWs &w, cudaStream_t s)
{
    const size_t HW = (size_t)H * W, N = (size_t)B * C * HW;
    const float *x = noisy;
    if (C == 3) {
        DN_TRY(colour(noisy, w.ycc, B, H, W, 0, s));
        x = w.ycc;
    }
    float tau1[1024], tau2[1024], thr[1024], sig[3 * 1024];
    // runs of consecutive images in the same regime (their passes share patch side, grid and
    // distance), at most 1024 images each
    for (int b0 = 0; b0 < B;) {
        const bool hi = is_high(p, sigma[b0]);
        int b1 = b0 + 1;
        while (b1 < B && b1 - b0 < 1024 && is_high(p, sigma[b1]) == hi) ++b1;
        const int nb = b1 - b0;
        const dn_bm3d_pass ph = pass_at(p->hard, hi, true), pw = pass_at(p->wiener, hi, false);
        for (int i = 0; i < nb; ++i) {
            tau1[i] = ph.tau;
            tau2[i] = pw.tau;
            for (int c = 0; c < C; ++c) sig[i * C + c] = channel_sigma(sigma[b0 + i], C, c);
            thr[i] = ph.lambda2d * sig[(size_t)i * C];  // guide-channel sigma
        }
        const size_t off = (size_t)b0 * C * HW;
        const size_t Nb = (size_t)nb * C * HW;
        const bool tc = (p->precision & DN_BF16) != 0;
        // pass 1: match on channel 0 of the noisy image (2D-prethresholded patches in the
        // high-noise regime), hard thresholding
        if (ph.lambda2d > 0.0f)
            DN_TRY(match_prethresh_any(x + off, (size_t)C * HW, nb, H, W, ph, tau1, thr, w.idx, w.n, s));
        else
            DN_TRY(match_any(x + off, (size_t)C * HW, nb, H, W, ph, tau1, p->precision, w.idx, w.n, w.mws, s));
        if (cudaMemsetAsync(w.acc, 0, kAccBytesPerPixel * Nb, s) != cudaSuccess) return DN_ECUDA;
        DN_TRY(filter_any(false, tc, x + off, nullptr, w.idx, w.n, nb, C, H, W, sig, ph, w.acc, s));
        DN_TRY(normalize(w.acc, w.basic + off, nb, C, H, W, ph.beta, s, ph.patch));
        // pass 2: match on channel 0 of the basic estimate, Wiener filtering
        DN_TRY(match_any(w.basic + off, (size_t)C * HW, nb, H, W, pw, tau2, p->precision, w.idx, w.n, w.mws, s));
        if (cudaMemsetAsync(w.acc, 0, kAccBytesPerPixel * Nb, s) != cudaSuccess) return DN_ECUDA;
        DN_TRY(filter_any(true, tc, x + off, w.basic + off, w.idx, w.n, nb, C, H, W, sig, pw, w.acc, s));
        DN_TRY(normalize(w.acc, (C == 3 ? w.ycc : out) + off, nb, C, H, W, pw.beta, s, pw.patch));
        b0 = b1;
    }
    if (C == 3) DN_TRY(colour(w.ycc, out, B, H, W, 1, s));
    (void)N;
    return DN_OK;
}

dn_status run_nlm(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                  const dn_nlm_params *p, const NlmWs &w, cudaStream_t s)
{
    float sg[1024];
    for (int b0 = 0; b0 < B; b0 += 1024) {
        const int nb = B - b0 < 1024 ? B - b0 : 1024;
        for (int i = 0; i < nb; ++i) sg[i] = channel_sigma(sigma[b0 + i], C, 0);
        const size_t off = (size_t)b0 * C * H * W;
        if (C == 3) {
            DN_TRY(colour(noisy + off, w.ycc + off, nb, H, W, 0, s));
            DN_TRY(nlm_launch(w.ycc + off, w.tmp + off, nb, C, H, W, sg, *p, s));
            DN_TRY(colour(w.tmp + off, out + off, nb, H, W, 1, s));
        } else {
            DN_TRY(nlm_launch(noisy + off, out + off, nb, C, H, W, sg, *p, s));
        }
    }
    return DN_OK;
}

dn_status run_cnn(const float *noisy, const float *pre, float *out, int N, int H, int W, const dn_cnn *c,
                  const CnnWs &w, cudaStream_t s)
{
    const int cc = cnn_cc(c), C = c->width;
    if (c->precision == DN_BF16) {
        if (C != 32 && C != 64) return DN_EUNSUPPORTED;
        int *err = device_error_ptr();
        if (!err) return DN_ECUDA;
        size_t off = (size_t)C * 9 * 2 * cc + C;  // layer 1 (2 cc -> C)
        DN_TRY(conv_first_bf16(pre, noisy, c->weights, c->weights + (size_t)C * 9 * 2 * cc, w.act[0], N, cc, H, W, C,
                               s));
        int cur = 0;
        for (int l = 1; l < c->layers - 1;) {
            const float *wl = c->weights + off;
            const float *bl = wl + (size_t)C * 9 * C;
            char *wp = w.wpack + wpack_bytes(C) * (size_t)(l - 1);
            DN_TRY(pack_w_tc(wl, wp, C, s));
            if (C == 32 && l + 1 < c->layers - 1) {
                // two hidden layers per pass: the intermediate rows stay in shared memory
                const float *wl2 = bl + C;
                const float *bl2 = wl2 + (size_t)C * 9 * C;
                char *wp2 = wp + wpack_bytes(C);
                DN_TRY(pack_w_tc(wl2, wp2, C, s));
                DN_TRY(conv3x3_tc_pair(w.act[cur], w.act[cur ^ 1], wp, bl, wp2, bl2, N, H, W, C, err, s));
                off += 2 * ((size_t)C * 9 * C + C);
                l += 2;
            } else {
                DN_TRY(conv3x3_tc(w.act[cur], w.act[cur ^ 1], wp, bl, N, H, W, C, 1, err, s));
                off += (size_t)C * 9 * C + C;
                l += 1;
            }
            cur ^= 1;
        }
        const float *wl = c->weights + off;
        return conv_last_bf16(w.act[cur], wl, wl + (size_t)cc * 9 * C, pre, out, N, cc, H, W, C, s);
    }
    DN_TRY(pack_input(pre, noisy, w.z, N, cc, H, W, s));
    const float *h = w.z;
    int kin = 2 * cc;
    size_t off = 0;
    for (int l = 0; l < c->layers; ++l) {
        const int kout = l == c->layers - 1 ? cc : C;
        const float *wl = c->weights + off;
        const float *bl = wl + (size_t)kout * 9 * kin;
        off += (size_t)kout * 9 * kin + kout;
        float *y = w.act[l & 1];
        DN_TRY(conv3x3_fwd_fp32(h, wl, bl, nullptr, y, N, kin, kout, H, W, l < c->layers - 1, false, s));
        h = y;
        kin = kout;
    }
    return residual_out(pre, h, out, (size_t)N * cc * H * W, s);
}

}  // namespace

#define DN_GUARD_BEGIN try {
#define DN_GUARD_END \
    }                \
    catch (...) { return DN_ECUDA; }

extern "C" {

void dn_bm3d_default_params(dn_bm3d_params *p)
{
    if (!p) return;
    p->hard = dn_bm3d_pass{8, 3, 39, 16, 2500.0f, 5000.0f, 2.7f, 2.0f, 2.0f, 0, 0};
    p->wiener = dn_bm3d_pass{8, 3, 39, 32, 400.0f, 3500.0f, 0.0f, 2.0f, 0.0f, 0, 0};
    p->precision = DN_FP32;
    p->sigma_regime = 0;
}

void dn_bm3d_high_noise_params(dn_bm3d_params *p)
{
    if (!p) return;
    dn_bm3d_default_params(p);
    p->hard.patch_high = 12;
    p->hard.step_high = 4;
    p->wiener.patch_high = 11;
    p->wiener.step_high = 6;
}

void dn_nlm_default_params(dn_nlm_params *p)
{
    if (!p) return;
    p->patch = 7;
    p->search = 21;
    p->h_over_sigma = 0.4f;
}

size_t dn_cnn_param_count_c(int layers, int width, int channels)
{
    if (layers < 2 || width < 1 || (channels != 1 && channels != 3)) return 0;
    size_t total = 0;
    int kin = 2 * channels;
    for (int l = 0; l < layers; ++l) {
        int kout = l == layers - 1 ? channels : width;
        total += (size_t)kout * 9 * kin + kout;
        kin = kout;
    }
    return total;
}

size_t dn_cnn_param_count(int layers, int width) { return dn_cnn_param_count_c(layers, width, 1); }

int dn_bm3d_grid(int L, int patch, int step, int *pos)
{
    int n = grid_count(L, patch, step);
    if (pos)
        for (int i = 0; i < n; ++i) pos[i] = (i * step < L - patch) ? i * step : L - patch;
    return n;
}

size_t dn_bm3d_workspace_bytes(int B, int C, int H, int W, const dn_bm3d_params *p)
{
    if (!valid_image(B, C, H, W, 8) || !valid_bm3d(p)) return 0;
    return bm3d_layout(nullptr, B, C, H, W, p).bytes;
}

size_t dn_nlm_workspace_bytes(int B, int C, int H, int W, const dn_nlm_params *p)
{
    (void)p;
    if (B < 1 || (C != 1 && C != 3)) return 0;
    return nlm_layout(nullptr, B, C, H, W).bytes;
}

size_t dn_cnn_workspace_bytes(int N, int H, int W, const dn_cnn *cnn)
{
    if (N < 1 || H < 1 || W < 1 || !cnn || cnn->width < 1) return 0;
    return cnn_layout(nullptr, N, H, W, cnn).bytes;
}

size_t dn_hybrid_workspace_bytes(int B, int C, int H, int W, int prefilter, const void *pp, const dn_cnn *cnn)
{
    if (!valid_image(B, C, H, W, 8) || !cnn) return 0;
    size_t pre = align256((size_t)B * C * H * W * sizeof(float));
    size_t f = prefilter == DN_PREFILTER_BM3D
                   ? dn_bm3d_workspace_bytes(B, C, H, W, static_cast<const dn_bm3d_params *>(pp))
                   : dn_nlm_workspace_bytes(B, C, H, W, static_cast<const dn_nlm_params *>(pp));
    const int n = cnn->channels == 3 ? B : B * C;
    size_t c = dn_cnn_workspace_bytes(n, H, W, cnn);
    return pre + (f > c ? f : c);
}

dn_status denoise_bm3d(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                       const dn_bm3d_params *p, void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!noisy || !out || !valid_image(B, C, H, W, 8) || !valid_sigmas(sigma, B) || !valid_bm3d(p) ||
        !sides_ok(B, H, W, sigma, p))
        return DN_EINVAL;
    if (!prethresh_fits(B, W, sigma, p)) return DN_EUNSUPPORTED;
    Bm3dWs w = bm3d_layout(workspace, B, C, H, W, p);
    if (!workspace || ws_bytes < w.bytes) return DN_ENOMEM;
    return run_bm3d(noisy, out, B, C, H, W, sigma, p, w, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status denoise_nlm(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                      const dn_nlm_params *p, void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!noisy || !out || !valid_nlm(p) || !valid_image(B, C, H, W, p->patch / 2 + 1) || !valid_sigmas(sigma, B))
        return DN_EINVAL;
    NlmWs w = nlm_layout(workspace, B, C, H, W);
    if (w.bytes > 0 && (!workspace || ws_bytes < w.bytes)) return DN_ENOMEM;
    return run_nlm(noisy, out, B, C, H, W, sigma, p, w, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status denoise_hybrid(const float *noisy, float *out, int B, int C, int H, int W, const float *sigma,
                         int prefilter, const void *pp, const dn_cnn *cnn, void *workspace, size_t ws_bytes,
                         dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!noisy || !out || !valid_image(B, C, H, W, 8) || !valid_sigmas(sigma, B) || !valid_cnn(cnn))
        return DN_EINVAL;
    if (prefilter == DN_PREFILTER_BM3D) {
        if (!valid_bm3d(static_cast<const dn_bm3d_params *>(pp)) ||
            !sides_ok(B, H, W, sigma, static_cast<const dn_bm3d_params *>(pp)))
            return DN_EINVAL;
        if (!prethresh_fits(B, W, sigma, static_cast<const dn_bm3d_params *>(pp))) return DN_EUNSUPPORTED;
    } else if (prefilter == DN_PREFILTER_NLM) {
        if (!valid_nlm(static_cast<const dn_nlm_params *>(pp))) return DN_EINVAL;
    } else {
        return DN_EINVAL;
    }
    const size_t need = dn_hybrid_workspace_bytes(B, C, H, W, prefilter, pp, cnn);
    if (!workspace || ws_bytes < need) return DN_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(workspace);
    float *pre = reinterpret_cast<float *>(base);
    void *rest = base + align256((size_t)B * C * H * W * sizeof(float));
    if (prefilter == DN_PREFILTER_BM3D) {
        auto *p = static_cast<const dn_bm3d_params *>(pp);
        DN_TRY(run_bm3d(noisy, pre, B, C, H, W, sigma, p, bm3d_layout(rest, B, C, H, W, p), s));
    } else {
        DN_TRY(run_nlm(noisy, pre, B, C, H, W, sigma, static_cast<const dn_nlm_params *>(pp),
                       nlm_layout(rest, B, C, H, W), s));
    }
    if (cnn->channels == 3 && C != 3) return DN_EINVAL;  // a colour-native network needs RGB input
    const int n = cnn->channels == 3 ? B : B * C;
    return run_cnn(noisy, pre, out, n, H, W, cnn, cnn_layout(rest, n, H, W, cnn), s);
    DN_GUARD_END
}

// ---- training gradient on the tensor cores -------------------------------------------

size_t dn_cnn_grad_workspace_bytes(int N, int H, int W, const dn_cnn *cnn)
{
    if (N < 1 || H < 1 || W < 1 || !valid_cnn(cnn) || cnn->precision != DN_BF16 || cnn->width != 32 ||
        cnn_cc(cnn) != 1)
        return 0;
    return cnn_grad_tc_workspace_bytes(N, H, W, cnn->layers);
}

dn_status dn_cnn_grad(const float *noisy, const float *pre, const float *clean, int N, int H, int W, const dn_cnn *cnn,
                      float *grad, double *loss_sum, void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!noisy || !pre || !clean || !grad || !loss_sum || N < 1 || H < 1 || W < 1 || !valid_cnn(cnn))
        return DN_EINVAL;
    if (cnn->precision != DN_BF16 || cnn->width != 32 || cnn_cc(cnn) != 1) return DN_EUNSUPPORTED;
    if ((size_t)N * H * W > ((size_t)1 << 31)) return DN_EINVAL;
    const size_t need = cnn_grad_tc_workspace_bytes(N, H, W, cnn->layers);
    if (!workspace || ws_bytes < need) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    return cnn_grad_tc(noisy, pre, clean, N, H, W, cnn->layers, cnn->weights, grad, loss_sum, workspace, err,
                       (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_conv3x3_tc_pair_fwd(const void *x, const float *wa, const float *ba, const float *wb, const float *bb,
                                 void *y, int N, int H, int W, int C, void *workspace, size_t ws_bytes,
                                 dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!x || !wa || !ba || !wb || !bb || !y || N < 1 || H < 1 || W < 1) return DN_EINVAL;
    if (C != 32) return DN_EUNSUPPORTED;
    if (!workspace || ws_bytes < 2 * wpack_bytes(C)) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *wp = static_cast<char *>(workspace);
    DN_TRY(pack_w_tc(wa, wp, C, s));
    DN_TRY(pack_w_tc(wb, wp + wpack_bytes(C), C, s));
    return conv3x3_tc_pair(x, y, wp, ba, wp + wpack_bytes(C), bb, N, H, W, C, err, s);
    DN_GUARD_END
}

size_t dn_conv3x3_tc_bwd_workspace_bytes(int N, int H, int W, int C)
{
    if (N < 1 || H < 1 || W < 1 || C != 32) return 0;
    const size_t a = conv_bwd_w_tc_workspace_bytes(N, H, W), b = wpack_bytes(C);
    return a > b ? a : b;
}

dn_status dn_conv3x3_tc_bwd_weight(const void *x, const void *g, float *dw, float *db, int N, int H, int W, int C,
                                   void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!x || !g || !dw || !db || N < 1 || H < 1 || W < 1) return DN_EINVAL;
    if (C != 32) return DN_EUNSUPPORTED;
    if (!workspace || ws_bytes < conv_bwd_w_tc_workspace_bytes(N, H, W)) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    return conv_bwd_w_tc(x, g, dw, db, N, H, W, workspace, err, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_conv3x3_tc_bwd_data(const void *g, const float *w, const void *mask, void *dx, int N, int H, int W, int C,
                                 void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!g || !w || !dx || N < 1 || H < 1 || W < 1) return DN_EINVAL;
    if (C != 32 && C != 64) return DN_EUNSUPPORTED;
    if (!workspace || ws_bytes < wpack_bytes(C)) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    DN_TRY(pack_w_tc(w, workspace, C, s, true));
    return conv3x3_tc(g, dx, workspace, nullptr, N, H, W, C, 0, err, s, mask);
    DN_GUARD_END
}

// ---- one image in tiles with a halo -------------------------------------------------

int dn_bm3d_halo(const dn_bm3d_params *p)
{
    if (!valid_bm3d(p)) return -1;
    auto kmax = [](const dn_bm3d_pass &q) { return q.patch_high > q.patch ? q.patch_high : q.patch; };
    return (2 * (p->hard.search / 2) + kmax(p->hard) - 1) + (2 * (p->wiener.search / 2) + kmax(p->wiener) - 1);
}

namespace {

int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

struct TilePlan {
    int T, hr, ny, nx;  // interior side, halo (both multiples of the grid steps' lcm), tile counts
    int rh_max, rw_max;
};

bool tile_plan(int H, int W, const dn_bm3d_params *p, int tile, TilePlan *tp)
{
    // tile origins on every reference grid either regime uses
    int g = 1;
    const int steps[4] = {p->hard.step, p->wiener.step, p->hard.step_high, p->wiener.step_high};
    for (int q : steps)
        if (q > 0) g = g / gcd_int(g, q) * q;
    if (tile < 8 || g > 4096) return false;
    const int R = dn_bm3d_halo(p);
    tp->T = (tile + g - 1) / g * g;
    tp->hr = (R + g - 1) / g * g;
    tp->ny = (H + tp->T - 1) / tp->T;
    tp->nx = (W + tp->T - 1) / tp->T;
    tp->rh_max = H < tp->T + 2 * tp->hr ? H : tp->T + 2 * tp->hr;
    tp->rw_max = W < tp->T + 2 * tp->hr ? W : tp->T + 2 * tp->hr;
    return true;
}

// Region [y0, y1) x [x0, x1) of tile (i, j) and its interior offset.
void tile_region(const TilePlan &tp, int H, int W, int i, int j, int *y0, int *y1, int *x0, int *x1)
{
    const int iy0 = i * tp.T, ix0 = j * tp.T;
    const int iy1 = iy0 + tp.T < H ? iy0 + tp.T : H, ix1 = ix0 + tp.T < W ? ix0 + tp.T : W;
    *y0 = iy0 - tp.hr > 0 ? iy0 - tp.hr : 0;
    *x0 = ix0 - tp.hr > 0 ? ix0 - tp.hr : 0;
    *y1 = iy1 + tp.hr < H ? iy1 + tp.hr : H;
    *x1 = ix1 + tp.hr < W ? ix1 + tp.hr : W;
}

struct TiledWs {
    float *in, *out;
    void *rest;
    size_t rest_bytes, bytes;
};

TiledWs tiled_layout(void *base, int C, const TilePlan &tp, const dn_bm3d_params *p, int max_batch)
{
    Carver cv(base);
    TiledWs w;
    const size_t n = (size_t)max_batch * C * tp.rh_max * tp.rw_max;
    w.in = cv.take<float>(n);
    w.out = cv.take<float>(n);
    w.rest_bytes = bm3d_layout(nullptr, max_batch, C, tp.rh_max, tp.rw_max, p).bytes;
    w.rest = cv.take<char>(w.rest_bytes);
    w.bytes = cv.off;
    return w;
}

}  // namespace

size_t dn_bm3d_tiled_workspace_bytes(int C, int H, int W, const dn_bm3d_params *p, int tile, int max_batch)
{
    TilePlan tp;
    if (!valid_image(1, C, H, W, 8) || !valid_bm3d(p) || max_batch < 1 || !tile_plan(H, W, p, tile, &tp)) return 0;
    return tiled_layout(nullptr, C, tp, p, max_batch).bytes;
}

dn_status denoise_bm3d_tiled(const float *noisy, float *out, int C, int H, int W, float sigma, const dn_bm3d_params *p,
                             int tile, int max_batch, void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    TilePlan tp;
    if (!noisy || !out || !valid_image(1, C, H, W, 8) || !valid_sigmas(&sigma, 1) || !valid_bm3d(p) ||
        !sides_ok(1, H, W, &sigma, p) || max_batch < 1 || max_batch > 1024 || !tile_plan(H, W, p, tile, &tp))
        return DN_EINVAL;
    if (!prethresh_fits(1, tp.rw_max, &sigma, p)) return DN_EUNSUPPORTED;
    TiledWs w = tiled_layout(workspace, C, tp, p, max_batch);
    if (!workspace || ws_bytes < w.bytes) return DN_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    // tiles grouped by region size (interior, edge and corner tiles differ), up to max_batch per launch
    struct T { int y0, y1, x0, x1, iy0, iy1, ix0, ix1; };
    const int ntiles = tp.ny * tp.nx;
    T *tl = new T[ntiles];
    for (int i = 0; i < tp.ny; ++i)
        for (int j = 0; j < tp.nx; ++j) {
            T &t = tl[i * tp.nx + j];
            tile_region(tp, H, W, i, j, &t.y0, &t.y1, &t.x0, &t.x1);
            t.iy0 = i * tp.T;
            t.ix0 = j * tp.T;
            t.iy1 = t.iy0 + tp.T < H ? t.iy0 + tp.T : H;
            t.ix1 = t.ix0 + tp.T < W ? t.ix0 + tp.T : W;
        }
    bool *done = new bool[ntiles]();
    float sig[1024];
    for (int i = 0; i < 1024; ++i) sig[i] = sigma;
    int *batch = new int[max_batch];
    dn_status st = DN_OK;
    const size_t HW = (size_t)H * W;
    for (int a = 0; a < ntiles && st == DN_OK; ++a) {
        if (done[a]) continue;
        const int rh = tl[a].y1 - tl[a].y0, rw = tl[a].x1 - tl[a].x0;
        int nb = 0;
        for (int b = a; b < ntiles && nb < max_batch; ++b)
            if (!done[b] && tl[b].y1 - tl[b].y0 == rh && tl[b].x1 - tl[b].x0 == rw) {
                batch[nb++] = b;
                done[b] = true;
            }
        const size_t plane = (size_t)rh * rw;
        for (int k = 0; k < nb && st == DN_OK; ++k) {
            const T &t = tl[batch[k]];
            for (int c = 0; c < C; ++c)
                if (cudaMemcpy2DAsync(w.in + ((size_t)k * C + c) * plane, (size_t)rw * sizeof(float),
                                      noisy + (size_t)c * HW + (size_t)t.y0 * W + t.x0, (size_t)W * sizeof(float),
                                      (size_t)rw * sizeof(float), rh, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    st = DN_ECUDA;
        }
        if (st != DN_OK) break;
        st = run_bm3d(w.in, w.out, nb, C, rh, rw, sig, p, bm3d_layout(w.rest, nb, C, rh, rw, p), s);
        for (int k = 0; k < nb && st == DN_OK; ++k) {
            const T &t = tl[batch[k]];
            const int oy = t.iy0 - t.y0, ox = t.ix0 - t.x0, ih = t.iy1 - t.iy0, iw = t.ix1 - t.ix0;
            for (int c = 0; c < C; ++c)
                if (cudaMemcpy2DAsync(out + (size_t)c * HW + (size_t)t.iy0 * W + t.ix0, (size_t)W * sizeof(float),
                                      w.out + ((size_t)k * C + c) * plane + (size_t)oy * rw + ox,
                                      (size_t)rw * sizeof(float), (size_t)iw * sizeof(float), ih,
                                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    st = DN_ECUDA;
        }
    }
    delete[] tl;
    delete[] done;
    delete[] batch;
    return st;
    DN_GUARD_END
}

const char *dn_strerror(dn_status st)
{
    switch (st) {
        case DN_OK: return "ok";
        case DN_EINVAL: return "invalid argument";
        case DN_ENOMEM: return "workspace too small";
        case DN_ECUDA: return "CUDA launch or runtime error";
        case DN_EDEVICE: return "device-side error status";
        case DN_EUNSUPPORTED: return "unsupported parameter combination";
    }
    return "unknown status";
}

size_t dn_bm3d_match_workspace_bytes(int B, int H, int W, const dn_bm3d_pass *p, int precision)
{
    if ((precision != DN_BF16 && precision != DN_BF16_MATCH) || !valid_image(B, 1, H, W, 8) || !valid_pass(p) ||
        p->patch != 8)
        return 0;
    return match_tc_workspace_bytes(B, H, W, *p);
}

dn_status dn_bm3d_match(const float *guide, size_t plane_stride, int B, int H, int W, const dn_bm3d_pass *p,
                        const float *tau, int precision, int *idx, int *n, void *workspace, size_t ws_bytes,
                        dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!guide || !idx || !n || !tau || !valid_pass(p) || !valid_image(B, 1, H, W, p->patch) ||
        plane_stride < (size_t)H * W)
        return DN_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(tau[b] > 0.0f)) return DN_EINVAL;
    if (precision != DN_FP32 && precision != DN_BF16 && precision != DN_BF16_MATCH) return DN_EINVAL;
    const size_t need = dn_bm3d_match_workspace_bytes(B, H, W, p, precision);
    if (need > 0 && (!workspace || ws_bytes < need)) return DN_ENOMEM;
    return match_any(guide, plane_stride, B, H, W, *p, tau, precision == DN_FP32 ? DN_FP32 : DN_BF16_MATCH, idx, n,
                     static_cast<int *>(workspace), (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_bm3d_match_prethresh(const float *guide, size_t plane_stride, int B, int H, int W,
                                  const dn_bm3d_pass *p, const float *tau, const float *thr, int *idx, int *n,
                                  dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!guide || !idx || !n || !tau || !thr || !valid_pass(p) || !valid_image(B, 1, H, W, p->patch) ||
        plane_stride < (size_t)H * W)
        return DN_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(tau[b] > 0.0f) || !(thr[b] >= 0.0f) || !std::isfinite(thr[b])) return DN_EINVAL;
    return match_prethresh_any(guide, plane_stride, B, H, W, *p, tau, thr, idx, n, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_bm3d_match_cross_terms(const float *guide, int H, int W, const dn_bm3d_pass *p, float tau, int tile_x,
                                    int tile_y, float *cross, int *idx, int *n, void *workspace, size_t ws_bytes,
                                    dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!guide || !cross || !idx || !n || !valid_image(1, 1, H, W, 8) || !valid_pass(p) || !tc_match_supported(*p) ||
        !(tau > 0.0f))
        return DN_EINVAL;
    if (tile_x < 0 || tile_y < 0 || tile_x * 8 >= grid_count(W, 8, p->step) || tile_y * 16 >= grid_count(H, 8, p->step))
        return DN_EINVAL;
    if (!workspace || ws_bytes < match_tc_workspace_bytes(1, H, W, *p)) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    return match_tc(guide, (size_t)H * W, 1, H, W, *p, &tau, idx, n, err, static_cast<int *>(workspace),
                    (cudaStream_t)stream, cross, tile_x, tile_y);
    DN_GUARD_END
}

size_t dn_bm3d_filter_workspace_bytes(int B, int C, int H, int W)
{
    if (!valid_image(B, C, H, W, 8)) return 0;
    return align256(kAccBytesPerPixel * (size_t)B * C * H * W);
}

static dn_status filter_entry(bool wiener, const float *img, const float *basic, const int *idx, const int *n, int B,
                              int C, int H, int W, const float *sigma_c, const dn_bm3d_pass *p, int precision,
                              float *out, void *ws, size_t ws_bytes, cudaStream_t s)
{
    if (!img || !idx || !n || !out || !sigma_c || (wiener && !basic) || !valid_pass(p) ||
        !valid_image(B, C, H, W, p->patch))
        return DN_EINVAL;
    for (int i = 0; i < B * C; ++i)
        if (!(sigma_c[i] > 0.0f) || !(sigma_c[i] <= 255.0f)) return DN_EINVAL;
    if (precision != DN_FP32 && precision != DN_BF16) return DN_EINVAL;
    const size_t need = dn_bm3d_filter_workspace_bytes(B, C, H, W);
    if (!ws || ws_bytes < need) return DN_ENOMEM;
    float *acc = static_cast<float *>(ws);
    const size_t HW = (size_t)H * W;
    for (int b0 = 0; b0 < B; b0 += 1024) {
        const int nb = B - b0 < 1024 ? B - b0 : 1024;
        const size_t off = (size_t)b0 * C * HW,
                     R = (size_t)grid_count(H, p->patch, p->step) * grid_count(W, p->patch, p->step);
        if (cudaMemsetAsync(acc, 0, kAccBytesPerPixel * (size_t)nb * C * HW, s) != cudaSuccess) return DN_ECUDA;
        const int *ib = idx + (size_t)b0 * R * p->n2;
        const int *nbp = n + (size_t)b0 * R;
        DN_TRY(filter_any(wiener, precision == DN_BF16, img + off, wiener ? basic + off : nullptr, ib, nbp, nb, C, H, W,
                          sigma_c + (size_t)b0 * C, *p, acc, s));
        DN_TRY(normalize(acc, out + off, nb, C, H, W, p->beta, s, p->patch));
    }
    return DN_OK;
}

dn_status dn_bm3d_filter_hard(const float *img, const int *idx, const int *n, int B, int C, int H, int W,
                              const float *sigma_c, const dn_bm3d_pass *p, int precision, float *basic,
                              void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    return filter_entry(false, img, nullptr, idx, n, B, C, H, W, sigma_c, p, precision, basic, workspace, ws_bytes,
                        (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_bm3d_filter_wiener(const float *noisy, const float *basic, const int *idx, const int *n, int B, int C,
                                int H, int W, const float *sigma_c, const dn_bm3d_pass *p, int precision, float *out,
                                void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    return filter_entry(true, noisy, basic, idx, n, B, C, H, W, sigma_c, p, precision, out, workspace, ws_bytes,
                        (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_rgb_to_ycc(const float *in, float *out, int B, int H, int W, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!in || !out || !valid_image(B, 3, H, W, 1)) return DN_EINVAL;
    return colour(in, out, B, H, W, 0, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_ycc_to_rgb(const float *in, float *out, int B, int H, int W, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!in || !out || !valid_image(B, 3, H, W, 1)) return DN_EINVAL;
    return colour(in, out, B, H, W, 1, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_error_reduce(const float *out, const float *ref, int B, size_t chw, double *sse, double *maxerr,
                          dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!out || !ref || !sse || !maxerr || B < 1 || B > 65535 || chw < 1) return DN_EINVAL;
    return error_reduce(out, ref, B, chw, sse, maxerr, (cudaStream_t)stream);
    DN_GUARD_END
}

static bool valid_conv(int N, int Cin, int Cout, int H, int W)
{
    return N >= 1 && Cin >= 1 && Cin <= 64 && Cout >= 1 && Cout <= 64 && H >= 1 && W >= 1 &&
           (size_t)N * (Cin > Cout ? Cin : Cout) * H * W < ((size_t)1 << 40);
}

dn_status dn_conv3x3_fwd(const float *x, const float *w, const float *b, float *y, int N, int Cin, int Cout, int H,
                         int W, int relu, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!x || !w || !y || !valid_conv(N, Cin, Cout, H, W)) return DN_EINVAL;
    return conv3x3_fwd_fp32(x, w, b, nullptr, y, N, Cin, Cout, H, W, relu, false, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_conv3x3_bwd_data(const float *dy, const float *w, const float *mask, float *dx, int N, int Cin, int Cout,
                              int H, int W, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!dy || !w || !dx || !valid_conv(N, Cin, Cout, H, W)) return DN_EINVAL;
    return conv3x3_fwd_fp32(dy, w, nullptr, mask, dx, N, Cout, Cin, H, W, 0, true, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_conv3x3_bwd_weight(const float *x, const float *dy, float *dw, float *db, int N, int Cin, int Cout,
                                int H, int W, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!x || !dy || !dw || !db || !valid_conv(N, Cin, Cout, H, W)) return DN_EINVAL;
    return conv3x3_bwd_weight_fp32(x, dy, dw, db, N, Cin, Cout, H, W, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_cnn_forward(const float *noisy, const float *pre, float *out, int N, int H, int W, const dn_cnn *cnn,
                         void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!noisy || !pre || !out || N < 1 || H < 1 || W < 1 || !valid_cnn(cnn)) return DN_EINVAL;
    CnnWs w = cnn_layout(workspace, N, H, W, cnn);
    if (!workspace || ws_bytes < w.bytes) return DN_ENOMEM;
    return run_cnn(noisy, pre, out, N, H, W, cnn, w, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_conv3x3_tc_fwd(const void *x, const float *w, const float *b, void *y, int N, int H, int W, int C,
                            int relu, void *workspace, size_t ws_bytes, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!x || !w || !b || !y || N < 1 || H < 1 || W < 1 || (size_t)N * H * W > ((size_t)1 << 34) ||
        (C != 32 && C != 64))
        return DN_EINVAL;
    if (!workspace || ws_bytes < wpack_bytes(C)) return DN_ENOMEM;
    int *err = device_error_ptr();
    if (!err) return DN_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    DN_TRY(pack_w_tc(w, workspace, C, s));
    return conv3x3_tc(x, y, workspace, b, N, H, W, C, relu, err, s);
    DN_GUARD_END
}

dn_status dn_cnn_pack_input(const float *pre, const float *noisy, float *z, int N, int H, int W, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!pre || !noisy || !z || N < 1 || H < 1 || W < 1) return DN_EINVAL;
    return pack_input(pre, noisy, z, N, 1, H, W, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_cnn_residual_out(const float *pre, const float *r, float *out, size_t count, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!pre || !r || !out || count < 1) return DN_EINVAL;
    return residual_out(pre, r, out, count, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_relu_bwd(const float *g, const float *y, float *out, size_t count, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!g || !y || !out || count < 1) return DN_EINVAL;
    return relu_bwd(g, y, out, count, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_l1_residual_grad(const float *r, const float *pre, const float *clean, float *dr, size_t count,
                              double *loss_sum, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!r || !pre || !clean || !dr || count < 1) return DN_EINVAL;
    return l1_grad(r, pre, clean, dr, count, loss_sum, (cudaStream_t)stream);
    DN_GUARD_END
}

dn_status dn_adam_step(float *param, const float *grad, float *m, float *v, size_t count, int t, float lr,
                       float beta1, float beta2, float eps, dn_stream_t stream)
{
    DN_GUARD_BEGIN
    if (!param || !grad || !m || !v || count < 1 || t < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return DN_EINVAL;
    return adam(param, grad, m, v, count, t, lr, beta1, beta2, eps, (cudaStream_t)stream);
    DN_GUARD_END
}

}  // extern "C"

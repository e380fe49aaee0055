/*
 * FP64 oracle of the nonlocal + neural denoiser (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path: every matrix and window below is built here
 * from its definition.
 *
 * The paper (Sec. II, Eq. 2-3) feeds a GPU BM3D (or NL-means) result and the
 * noisy image to a residual CNN; it treats BM3D / NLM as black boxes.  The
 * steps below restate the standard published definitions of those filters
 * (BM3D: Dabov et al. 2007; NL-means: Buades et al. 2005) with the
 * parameters of the workloads this library is checked on.  Every step is
 * plain and slow on purpose: exhaustive matching with a full sort, the 2D
 * transform as an explicit k^2 x k^2 Kronecker matrix (k = the patch side,
 * 8 by default, up to 16 for the larger patches of the high-noise profile), the
 * group transform as an
 * explicit Hadamard matrix, aggregation by direct accumulation, convolution
 * by a 7-deep loop.
 *
 * Parallelism: OpenMP over reference patches / pixels.  Aggregation sums go
 * to one private num/den buffer per thread, summed in thread order at the
 * end (a summation-order detail only).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_K 8          /* default BM3D patch side */
#define OR_KMIN 4       /* patch sides accepted: OR_KMIN .. OR_KMAX */
#define OR_KMAX 16
#define OR_NMAX 64      /* largest group size accepted */

/* ------------------------------------------------------------------ */
/* Transforms and windows                                              */
/* ------------------------------------------------------------------ */

/* Orthonormal DCT-II matrix of size k: C[u][m] = a_u cos(pi (2m+1) u / (2k)),
 * a_0 = sqrt(1/k), a_u = sqrt(2/k). */
void or_dct(int k, double *C)
{
    for (int u = 0; u < k; ++u)
        for (int m = 0; m < k; ++m) {
            double a = (u == 0) ? sqrt(1.0 / k) : sqrt(2.0 / k);
            C[u * k + m] = a * cos(M_PI * (2.0 * m + 1.0) * u / (2.0 * k));
        }
}

void or_dct8(double *C) { or_dct(OR_K, C); }

/* 2D DCT of a k x k patch as one k^2 x k^2 matrix acting on vec(P)
 * (row-major, index i*k+j): T[u*k+v][i*k+j] = C[u][i] C[v][j], i.e.
 * vec(C P C^T) = T vec(P). */
void or_dct2d_matrix_k(int k, double *T)
{
    const int k2 = k * k;
    double C[OR_KMAX * OR_KMAX];
    or_dct(k, C);
    for (int u = 0; u < k; ++u)
        for (int v = 0; v < k; ++v)
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j)
                    T[(size_t)(u * k + v) * k2 + i * k + j] = C[u * k + i] * C[v * k + j];
}

void or_dct2d_matrix(double *T) { or_dct2d_matrix_k(OR_K, T); }

static int patch_ok(int k) { return k >= OR_KMIN && k <= OR_KMAX; }

/* Sylvester Hadamard matrix in natural order, scaled by 1/sqrt(n)
 * (orthonormal and symmetric).  n must be a power of two. */
int or_hadamard(int n, double *Hm)
{
    if (n < 1 || (n & (n - 1)) != 0 || n > OR_NMAX) return -1;
    double s = 1.0 / sqrt((double)n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            /* H[r][c] = (-1)^{popcount(r & c)} */
            int bits = r & c, par = 0;
            while (bits) { par ^= (bits & 1); bits >>= 1; }
            Hm[r * n + c] = par ? -s : s;
        }
    return 0;
}

/* Modified Bessel function of the first kind, order 0, by its power series
 * I0(x) = sum_k ((x/2)^k / k!)^2, summed until the term is negligible. */
static double bessel_i0(double x)
{
    double sum = 1.0, term = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

/* Kaiser window of length M: w[m] = I0(beta sqrt(1 - (2m/(M-1) - 1)^2)) / I0(beta). */
void or_kaiser(int M, double beta, double *w)
{
    for (int m = 0; m < M; ++m) {
        double r = (M > 1) ? (2.0 * m / (M - 1) - 1.0) : 0.0;
        double a = 1.0 - r * r;
        if (a < 0) a = 0;
        w[m] = bessel_i0(beta * sqrt(a)) / bessel_i0(beta);
    }
}

/* 3D transform of a group G[n][k2] (k2 = k^2 pixels per patch): Z = H_n (G T^T),
 * i.e. the 2D DCT of every patch followed by the normalised Hadamard
 * transform along the group.  T2: scratch of n * k2 doubles. */
static void t3d_forward(const double *T, const double *Hn, int n, int k2, const double *G, double *Z, double *T2)
{
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < k2; ++a) {
            double s = 0.0;
            for (int b = 0; b < k2; ++b) s += T[(size_t)a * k2 + b] * G[k * k2 + b];
            T2[k * k2 + a] = s;
        }
    for (int m = 0; m < n; ++m)
        for (int a = 0; a < k2; ++a) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += Hn[m * n + k] * T2[k * k2 + a];
            Z[m * k2 + a] = s;
        }
}

/* Inverse of t3d_forward (both factors are orthonormal): G = T^T (H_n^T Z). */
static void t3d_inverse(const double *T, const double *Hn, int n, int k2, const double *Z, double *G, double *T2)
{
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < k2; ++a) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s += Hn[m * n + k] * Z[m * k2 + a];
            T2[k * k2 + a] = s;
        }
    for (int k = 0; k < n; ++k)
        for (int b = 0; b < k2; ++b) {
            double s = 0.0;
            for (int a = 0; a < k2; ++a) s += T[(size_t)a * k2 + b] * T2[k * k2 + a];
            G[k * k2 + b] = s;
        }
}

/* Exported for the transform pins: the 3D transform of n patches of side k. */
int or_t3d_k(const double *G, int n, int k, int inverse, double *Z)
{
    if (!patch_ok(k)) return -1;
    const int k2 = k * k;
    double Hn[OR_NMAX * OR_NMAX];
    if (or_hadamard(n, Hn)) return -1;
    double *T = (double *)malloc(sizeof(double) * (size_t)k2 * k2);
    double *T2 = (double *)malloc(sizeof(double) * (size_t)n * k2);
    if (!T || !T2) {
        free(T);
        free(T2);
        return -2;
    }
    or_dct2d_matrix_k(k, T);
    if (inverse) t3d_inverse(T, Hn, n, k2, G, Z, T2);
    else t3d_forward(T, Hn, n, k2, G, Z, T2);
    free(T);
    free(T2);
    return 0;
}

int or_t3d(const double *G, int n, int inverse, double *Z) { return or_t3d_k(G, n, OR_K, inverse, Z); }

/* ------------------------------------------------------------------ */
/* Block matching                                                      */
/* ------------------------------------------------------------------ */

/* Reference grid along one axis of length L: 0, step, 2 step, ... <= L-k,
 * plus L-k itself when it is not on that lattice, so that every pixel is
 * covered by at least one reference patch. */
int or_grid(int L, int k, int step, int *pos)
{
    int last = L - k, n = 0;
    if (last < 0 || step < 1) return 0;
    for (int p = 0; p <= last; p += step) { if (pos) pos[n] = p; ++n; }
    if (last % step != 0) { if (pos) pos[n] = last; ++n; }
    return n;
}

typedef struct { double d; int idx; } cand_t;

static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Largest power of two <= v (v >= 1). */
static int pow2_floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

/* Flag bits (per reference / group). */
#define OR_FLAG_TAU 1    /* a candidate's distance lies within 1e-5 tau of tau */
#define OR_FLAG_TIE 2    /* two ranked neighbours within 1e-5 relative       */
#define OR_FLAG_THR 4    /* a 3D coefficient lies within the band of lambda sigma */
#define OR_FLAG_PRE 8    /* a prethresholded 2D coefficient near lambda2d sigma could change the list */

/* Exhaustive block matching for every reference patch of one guide image.
 *
 * d(P,Q) = ||P - Q||^2 / k^2 over every candidate whose top-left corner lies
 * in the (search x search) window centred on the reference's top-left corner,
 * clipped to the image.  The reference patch is always kept and always first;
 * the other candidates with d <= tau follow in ascending (d, y*W + x) order.
 * n = min(n2, largest power of two <= #kept).
 *
 * Outputs, R = Ry*Rx references in row-major grid order:
 *   idx[R][n2]    row-major pixel index of each group member (-1 past #kept)
 *   dist[R][n2+1] distances of ranks 0..n2 (-1 past #kept)
 *   nkept[R], ngroup[R] (= n), flag[R] (OR_FLAG_TAU | OR_FLAG_TIE). */
int or_match(const double *g, int H, int W, int k, int step, int search, int n2, double tau,
             int *idx, double *dist, int *nkept, int *ngroup, unsigned char *flag)
{
    if (!patch_ok(k) || H < k || W < k || search < 1 || (search & 1) == 0 || n2 < 1 || n2 > OR_NMAX)
        return -1;
    int gy[4096], gx[4096];
    int Ry = or_grid(H, k, step, gy), Rx = or_grid(W, k, step, gx);
    if (Ry > 4096 || Rx > 4096) return -1;
    int hs = search / 2;
    int ncand_max = search * search;
#pragma omp parallel
    {
        cand_t *cl = (cand_t *)malloc(sizeof(cand_t) * (size_t)ncand_max);
#pragma omp for schedule(static)
        for (int r = 0; r < Ry * Rx; ++r) {
            int y0 = gy[r / Rx], x0 = gx[r % Rx];
            int nc = 0;
            unsigned char fl = 0;
            int ylo = y0 - hs < 0 ? 0 : y0 - hs, yhi = y0 + hs > H - k ? H - k : y0 + hs;
            int xlo = x0 - hs < 0 ? 0 : x0 - hs, xhi = x0 + hs > W - k ? W - k : x0 + hs;
            for (int y = ylo; y <= yhi; ++y)
                for (int x = xlo; x <= xhi; ++x) {
                    if (y == y0 && x == x0) continue;
                    double s = 0.0;
                    for (int i = 0; i < k; ++i)
                        for (int j = 0; j < k; ++j) {
                            double e = g[(size_t)(y0 + i) * W + x0 + j] - g[(size_t)(y + i) * W + x + j];
                            s += e * e;
                        }
                    double d = s / (double)(k * k);
                    if (fabs(d - tau) <= 1e-5 * tau) fl |= OR_FLAG_TAU;
                    if (d <= tau) { cl[nc].d = d; cl[nc].idx = y * W + x; ++nc; }
                }
            qsort(cl, (size_t)nc, sizeof(cand_t), cand_cmp);
            int kept = nc + 1;
            int n = pow2_floor(kept < n2 ? kept : n2);
            int *I = idx + (size_t)r * n2;
            double *D = dist + (size_t)r * (n2 + 1);
            I[0] = y0 * W + x0;
            D[0] = 0.0;
            for (int t = 1; t < n2; ++t) I[t] = (t < kept) ? cl[t - 1].idx : -1;
            for (int t = 1; t <= n2; ++t) D[t] = (t < kept) ? cl[t - 1].d : -1.0;
            /* near-ties among ranks 1..min(n, kept-1): order inside the group or the cut */
            int last = n < kept - 1 ? n : kept - 1;
            for (int t = 1; t < last; ++t) {
                double a = cl[t - 1].d, b = cl[t].d;
                if (!(a == 0.0 && b == 0.0) && fabs(b - a) <= 1e-5 * (a > b ? a : b)) fl |= OR_FLAG_TIE;
            }
            nkept[r] = kept;
            ngroup[r] = n;
            flag[r] = fl;
        }
        free(cl);
    }
    return 0;
}

/* Block matching on 2D-prethresholded patches: the first-pass distance BM3D
 * uses at high noise.  Every patch P is replaced by Y(P), its 2D transform
 * T2D(P) (orthonormal DCT-II, or_dct2d_matrix) with every coefficient of
 * magnitude <= thr set to zero, and
 *     d(P, Q) = ||Y(P) - Y(Q)||^2 / k^2.
 * With thr = 0 this is or_match's distance (T2D is orthonormal).  Window,
 * ordering, group size and outputs as or_match.  Two distances a, b count as
 * tied when |a - b| <= rtie max(a, b) + atie (sqrt(a) + sqrt(b)): an error
 * of at most delta on each coefficient difference moves a distance d by at
 * most 2 delta sqrt(d) (Cauchy-Schwarz over the k^2 terms), so atie = 2 delta
 * covers coefficients computed in lower precision.  Flags:
 *   OR_FLAG_TAU  a candidate tied with tau;
 *   OR_FLAG_TIE  two ranked neighbours (up to the group cut) tied;
 *   OR_FLAG_PRE  the reference patch has a coefficient whose magnitude lies
 *                within `band` of thr, or a candidate with such a coefficient
 *                could, with that coefficient's keep/zero decision reversed,
 *                reach the group: its smallest possible distance is <= the
 *                distance of the last listed candidate (of tau while at most
 *                n2 candidates are kept, when one more or one fewer changes
 *                the group size).
 * Patches of any side k in OR_KMIN .. OR_KMAX (the 2D DCT of size k). */
int or_match_pre(const double *g, int H, int W, int k, int step, int search, int n2, double tau, double thr,
                 double band, double rtie, double atie, int *idx, double *dist, int *nkept, int *ngroup,
                 unsigned char *flag)
{
    if (!patch_ok(k) || H < k || W < k || search < 1 || (search & 1) == 0 || n2 < 1 || n2 > OR_NMAX || thr < 0.0)
        return -1;
    int gy[4096], gx[4096];
    int Ry = or_grid(H, k, step, gy), Rx = or_grid(W, k, step, gx);
    if (Ry > 4096 || Rx > 4096) return -1;
    const int Hp = H - k + 1, Wp = W - k + 1;
    const size_t np = (size_t)Hp * Wp;
    const int k2 = k * k;
    double *Y = (double *)malloc(sizeof(double) * np * k2);     /* prethresholded coefficients */
    double *A = (double *)malloc(sizeof(double) * np * k2);     /* value under the other decision */
    unsigned char *hz = (unsigned char *)malloc(np);            /* patch has a coefficient in the band */
    double *T = (double *)malloc(sizeof(double) * (size_t)k2 * k2);
    if (!Y || !A || !hz || !T) {
        free(Y);
        free(A);
        free(hz);
        free(T);
        return -2;
    }
    or_dct2d_matrix_k(k, T);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < (long)np; ++q) {
        int y = (int)(q / Wp), x = (int)(q % Wp);
        double P[OR_KMAX * OR_KMAX];
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) P[i * k + j] = g[(size_t)(y + i) * W + x + j];
        unsigned char h = 0;
        for (int a = 0; a < k2; ++a) {
            double c = 0.0;
            for (int m = 0; m < k2; ++m) c += T[(size_t)a * k2 + m] * P[m];
            int keep = fabs(c) > thr;
            int near = fabs(fabs(c) - thr) <= band;
            Y[(size_t)q * k2 + a] = keep ? c : 0.0;
            A[(size_t)q * k2 + a] = near ? (keep ? 0.0 : c) : (keep ? c : 0.0);
            h |= (unsigned char)near;
        }
        hz[q] = h;
    }
    free(T);
    int hs = search / 2;
    int ncand_max = search * search;
    int fail = 0;
#pragma omp parallel
    {
        cand_t *cl = (cand_t *)malloc(sizeof(cand_t) * (size_t)ncand_max);
        double *hlo = (double *)malloc(sizeof(double) * (size_t)ncand_max);  /* smallest d of hazardous candidates */
        if (!cl || !hlo) fail = 1;
#pragma omp for schedule(static)
        for (int r = 0; r < Ry * Rx; ++r) {
            if (fail) continue;
            int y0 = gy[r / Rx], x0 = gx[r % Rx];
            const double *yr = Y + ((size_t)y0 * Wp + x0) * k2;
            int nc = 0, nh = 0;
            unsigned char fl = hz[(size_t)y0 * Wp + x0] ? OR_FLAG_PRE : 0;
            int ylo = y0 - hs < 0 ? 0 : y0 - hs, yhi = y0 + hs > H - k ? H - k : y0 + hs;
            int xlo = x0 - hs < 0 ? 0 : x0 - hs, xhi = x0 + hs > W - k ? W - k : x0 + hs;
            for (int y = ylo; y <= yhi; ++y)
                for (int x = xlo; x <= xhi; ++x) {
                    if (y == y0 && x == x0) continue;
                    size_t q = (size_t)y * Wp + x;
                    const double *yq = Y + q * k2, *aq = A + q * k2;
                    double s = 0.0, slo = 0.0;
                    for (int a = 0; a < k2; ++a) {
                        double e = yr[a] - yq[a], f = yr[a] - aq[a];
                        s += e * e;
                        slo += (e * e < f * f) ? e * e : f * f;
                    }
                    double d = s / (double)(k * k);
                    if (fabs(d - tau) <= rtie * tau + 2.0 * atie * sqrt(tau)) fl |= OR_FLAG_TAU;
                    if (d <= tau) { cl[nc].d = d; cl[nc].idx = y * W + x; ++nc; }
                    if (hz[q]) hlo[nh++] = slo / (double)(k * k);
                }
            qsort(cl, (size_t)nc, sizeof(cand_t), cand_cmp);
            int kept = nc + 1;
            int n = pow2_floor(kept < n2 ? kept : n2);
            int *I = idx + (size_t)r * n2;
            double *D = dist + (size_t)r * (n2 + 1);
            I[0] = y0 * W + x0;
            D[0] = 0.0;
            for (int t = 1; t < n2; ++t) I[t] = (t < kept) ? cl[t - 1].idx : -1;
            for (int t = 1; t <= n2; ++t) D[t] = (t < kept) ? cl[t - 1].d : -1.0;
            int last = n < kept - 1 ? n : kept - 1;
            for (int t = 1; t < last; ++t) {
                double a = cl[t - 1].d, b = cl[t].d;
                if (!(a == 0.0 && b == 0.0) && fabs(b - a) <= rtie * (a > b ? a : b) + atie * (sqrt(a) + sqrt(b)))
                    fl |= OR_FLAG_TIE;
            }
            double edge = kept > n2 ? cl[n2 - 2].d : tau;
            for (int t = 0; t < nh; ++t)
                if (hlo[t] <= edge * (1.0 + rtie) + 2.0 * atie * sqrt(edge)) fl |= OR_FLAG_PRE;
            nkept[r] = kept;
            ngroup[r] = n;
            flag[r] = fl;
        }
        free(cl);
        free(hlo);
    }
    free(Y); free(A); free(hz);
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* Collaborative filtering and aggregation                            */
/* ------------------------------------------------------------------ */

typedef struct {
    int nthreads;
    double *acc;   /* [nthreads][2*C*H*W]: num then den */
} acc_t;

static int acc_init(acc_t *a, size_t plane)
{
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    a->nthreads = nt;
    a->acc = (double *)calloc((size_t)nt * plane * 2, sizeof(double));
    return a->acc ? 0 : -1;
}

/* out = num / den, summing the per-thread buffers in thread order. */
static void acc_finish(acc_t *a, size_t plane, double *out)
{
    for (size_t p = 0; p < plane; ++p) {
        double num = 0.0, den = 0.0;
        for (int t = 0; t < a->nthreads; ++t) {
            num += a->acc[(size_t)t * plane * 2 + p];
            den += a->acc[(size_t)t * plane * 2 + plane + p];
        }
        out[p] = num / den;
    }
    free(a->acc);
}

/* Mark every pixel covered by the group's patches. */
static void mark_group(unsigned char *pxflag, int W, int k, const int *I, int n, unsigned char bits)
{
    if (!pxflag) return;
    for (int t = 0; t < n; ++t) {
        int y = I[t] / W, x = I[t] % W;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                unsigned char *p = &pxflag[(size_t)(y + i) * W + x + j];
#pragma omp atomic
                *p |= bits;
            }
    }
}

/* BM3D first pass (hard thresholding), on an image of C channels whose
 * channel 0 is the matching guide (the Y channel for colour input).
 *   img[C][H][W], sig[C] per-channel noise std, band: half-width of the
 *   hard-threshold hazard band (absolute, added to 1e-5 lambda sigma).
 * For each reference group: gather, 3D transform, zero |c| <= lambda sigma,
 * N_har = #kept, inverse, weight 1/(sigma^2 N_har) (1 if N_har = 0), and
 * Kaiser-windowed accumulation into num/den; basic = num / den.
 * pxflag[H][W] (may be NULL) ORs the flags of every group covering a pixel;
 * gflag[R] (may be NULL) receives each group's flags. */
int or_bm3d_pass1(const double *img, int C, int H, int W, const double *sig,
                  int k, int step, int search, int n2, double tau, double lambda3d, double beta,
                  double band, double thr2d, double band2d, double *basic, unsigned char *pxflag,
                  unsigned char *gflag)
{
    if (C < 1 || !patch_ok(k)) return -1;
    int Ry = or_grid(H, k, step, NULL), Rx = or_grid(W, k, step, NULL);
    int R = Ry * Rx;
    if (R <= 0) return -1;
    int *idx = (int *)malloc(sizeof(int) * (size_t)R * n2);
    double *dist = (double *)malloc(sizeof(double) * (size_t)R * (n2 + 1));
    int *nk = (int *)malloc(sizeof(int) * (size_t)R), *ng = (int *)malloc(sizeof(int) * (size_t)R);
    unsigned char *fl = (unsigned char *)malloc((size_t)R);
    if (!idx || !dist || !nk || !ng || !fl) return -2;
    /* thr2d > 0: distances on 2D-prethresholded patches (tie tolerances of
     * the FP32 transforms, see or_match_pre) */
    if (thr2d > 0.0 ? or_match_pre(img, H, W, k, step, search, n2, tau, thr2d, band2d, 1e-5, 1e-3, idx, dist, nk,
                                   ng, fl)
                    : or_match(img, H, W, k, step, search, n2, tau, idx, dist, nk, ng, fl))
        return -1;

    const int k2 = k * k;
    double *T = (double *)malloc(sizeof(double) * (size_t)k2 * k2), kw[OR_KMAX];
    if (!T) return -2;
    or_dct2d_matrix_k(k, T);
    or_kaiser(k, beta, kw);
    size_t HW = (size_t)H * W, plane = (size_t)C * HW;
    if (pxflag) memset(pxflag, 0, HW);
    acc_t acc;
    if (acc_init(&acc, plane)) return -2;

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *num = acc.acc + (size_t)tid * plane * 2, *den = num + plane;
        /* group, coefficients, estimate and transform scratch: OR_NMAX patches each */
        double *G = (double *)malloc(sizeof(double) * 4 * OR_NMAX * (size_t)k2);
        double *Z = G + OR_NMAX * k2, *E = Z + OR_NMAX * k2, *S = E + OR_NMAX * k2;
        double Hn[OR_NMAX * OR_NMAX];
#pragma omp for schedule(static)
        for (int r = 0; r < R; ++r) {
            int n = ng[r];
            const int *I = idx + (size_t)r * n2;
            unsigned char f = fl[r];
            or_hadamard(n, Hn);
            for (int c = 0; c < C; ++c) {
                const double *ch = img + (size_t)c * HW;
                double thr = lambda3d * sig[c];
                for (int t = 0; t < n; ++t) {
                    int y = I[t] / W, x = I[t] % W;
                    for (int i = 0; i < k; ++i)
                        for (int j = 0; j < k; ++j)
                            G[t * k2 + i * k + j] = ch[(size_t)(y + i) * W + x + j];
                }
                t3d_forward(T, Hn, n, k2, G, Z, S);
                int nhar = 0;
                for (int a = 0; a < n * k2; ++a) {
                    double m = fabs(Z[a]);
                    if (fabs(m - thr) <= 1e-5 * thr + band) f |= OR_FLAG_THR;
                    if (m > thr) ++nhar; else Z[a] = 0.0;
                }
                t3d_inverse(T, Hn, n, k2, Z, E, S);
                double w = nhar > 0 ? 1.0 / (sig[c] * sig[c] * nhar) : 1.0;
                for (int t = 0; t < n; ++t) {
                    int y = I[t] / W, x = I[t] % W;
                    for (int i = 0; i < k; ++i)
                        for (int j = 0; j < k; ++j) {
                            size_t p = (size_t)c * HW + (size_t)(y + i) * W + x + j;
                            double kk = w * kw[i] * kw[j];
                            num[p] += kk * E[t * k2 + i * k + j];
                            den[p] += kk;
                        }
                }
            }
            if (gflag) gflag[r] = f;
            if (f) mark_group(pxflag, W, k, I, n, f);
        }
        free(G);
    }
    acc_finish(&acc, plane, basic);
    free(T); free(idx); free(dist); free(nk); free(ng); free(fl);
    return 0;
}

/* BM3D second pass (empirical Wiener filtering).  Matching runs on channel 0
 * of the basic estimate; for each group the basic-estimate group B and the
 * noisy group Y (same positions) are 3D transformed, the Wiener gains
 * w_a = B_a^2 / (B_a^2 + sigma^2) multiply Y, the product is inverted, and the
 * group weight is 1/(sigma^2 sum_a w_a^2) (1 if that sum is 0). */
int or_bm3d_pass2(const double *noisy, const double *basic, int C, int H, int W, const double *sig,
                  int k, int step, int search, int n2, double tau, double beta,
                  double *out, unsigned char *pxflag, unsigned char *gflag)
{
    if (C < 1 || !patch_ok(k)) return -1;
    int Ry = or_grid(H, k, step, NULL), Rx = or_grid(W, k, step, NULL);
    int R = Ry * Rx;
    if (R <= 0) return -1;
    int *idx = (int *)malloc(sizeof(int) * (size_t)R * n2);
    double *dist = (double *)malloc(sizeof(double) * (size_t)R * (n2 + 1));
    int *nk = (int *)malloc(sizeof(int) * (size_t)R), *ng = (int *)malloc(sizeof(int) * (size_t)R);
    unsigned char *fl = (unsigned char *)malloc((size_t)R);
    if (!idx || !dist || !nk || !ng || !fl) return -2;
    if (or_match(basic, H, W, k, step, search, n2, tau, idx, dist, nk, ng, fl)) return -1;

    const int k2 = k * k;
    double *T = (double *)malloc(sizeof(double) * (size_t)k2 * k2), kw[OR_KMAX];
    if (!T) return -2;
    or_dct2d_matrix_k(k, T);
    or_kaiser(k, beta, kw);
    size_t HW = (size_t)H * W, plane = (size_t)C * HW;
    if (pxflag) memset(pxflag, 0, HW);
    acc_t acc;
    if (acc_init(&acc, plane)) return -2;

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *num = acc.acc + (size_t)tid * plane * 2, *den = num + plane;
        /* basic and noisy groups, their coefficients, the estimate, transform scratch */
        double *Gb = (double *)malloc(sizeof(double) * 6 * OR_NMAX * (size_t)k2);
        double *Gy = Gb + OR_NMAX * k2, *Zb = Gy + OR_NMAX * k2, *Zy = Zb + OR_NMAX * k2;
        double *E = Zy + OR_NMAX * k2, *S = E + OR_NMAX * k2;
        double Hn[OR_NMAX * OR_NMAX];
#pragma omp for schedule(static)
        for (int r = 0; r < R; ++r) {
            int n = ng[r];
            const int *I = idx + (size_t)r * n2;
            or_hadamard(n, Hn);
            for (int c = 0; c < C; ++c) {
                const double *cb = basic + (size_t)c * HW, *cy = noisy + (size_t)c * HW;
                double s2 = sig[c] * sig[c];
                for (int t = 0; t < n; ++t) {
                    int y = I[t] / W, x = I[t] % W;
                    for (int i = 0; i < k; ++i)
                        for (int j = 0; j < k; ++j) {
                            size_t p = (size_t)(y + i) * W + x + j;
                            Gb[t * k2 + i * k + j] = cb[p];
                            Gy[t * k2 + i * k + j] = cy[p];
                        }
                }
                t3d_forward(T, Hn, n, k2, Gb, Zb, S);
                t3d_forward(T, Hn, n, k2, Gy, Zy, S);
                double wsq = 0.0;
                for (int a = 0; a < n * k2; ++a) {
                    double b2 = Zb[a] * Zb[a];
                    double om = b2 / (b2 + s2);
                    Zy[a] *= om;
                    wsq += om * om;
                }
                t3d_inverse(T, Hn, n, k2, Zy, E, S);
                double w = wsq > 0.0 ? 1.0 / (s2 * wsq) : 1.0;
                for (int t = 0; t < n; ++t) {
                    int y = I[t] / W, x = I[t] % W;
                    for (int i = 0; i < k; ++i)
                        for (int j = 0; j < k; ++j) {
                            size_t p = (size_t)c * HW + (size_t)(y + i) * W + x + j;
                            double kk = w * kw[i] * kw[j];
                            num[p] += kk * E[t * k2 + i * k + j];
                            den[p] += kk;
                        }
                }
            }
            if (gflag) gflag[r] = fl[r];
            if (fl[r]) mark_group(pxflag, W, k, I, n, fl[r]);
        }
        free(Gb);
    }
    acc_finish(&acc, plane, out);
    free(T); free(idx); free(dist); free(nk); free(ng); free(fl);
    return 0;
}

/* ------------------------------------------------------------------ */
/* NL-means                                                            */
/* ------------------------------------------------------------------ */

/* Half-sample symmetric reflection of index i into [0, L). */
static int reflect(int i, int L)
{
    while (i < 0 || i >= L) {
        if (i < 0) i = -i - 1;
        if (i >= L) i = 2 * L - i - 1;
    }
    return i;
}

/* Pixel-wise NL-means on an image of C channels whose channel 0 is the guide.
 * For each pixel p and every q of the (search x search) window centred on p
 * (clipped to the image, p itself included):
 *   d2 = mean over the (patch x patch) neighbourhood of (g(p+t) - g(q+t))^2,
 *        neighbourhoods of the guide g read through half-sample symmetric
 *        reflection;
 *   w  = exp(-max(d2 - 2 sigma^2, 0) / h^2);
 * out_c(p) = sum_q w y_c(q) / sum_q w for every channel c.  h = INFINITY gives
 * w = 1. */
int or_nlm(const double *y, int C, int H, int W, double sigma, int patch, int search, double h,
           double *out)
{
    if (C < 1 || C > 3 || H < 1 || W < 1 || (patch & 1) == 0 || (search & 1) == 0) return -1;
    int r = patch / 2, hs = search / 2;
    size_t HW = (size_t)H * W;
    double s2 = 2.0 * sigma * sigma, inv_np = 1.0 / (double)(patch * patch);
#pragma omp parallel for schedule(static)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            double acc[3] = {0.0, 0.0, 0.0}, wsum = 0.0;
            for (int qy = py - hs; qy <= py + hs; ++qy) {
                if (qy < 0 || qy >= H) continue;
                for (int qx = px - hs; qx <= px + hs; ++qx) {
                    if (qx < 0 || qx >= W) continue;
                    double d2 = 0.0;
                    for (int ty = -r; ty <= r; ++ty)
                        for (int tx = -r; tx <= r; ++tx) {
                            double a = y[(size_t)reflect(py + ty, H) * W + reflect(px + tx, W)];
                            double b = y[(size_t)reflect(qy + ty, H) * W + reflect(qx + tx, W)];
                            d2 += (a - b) * (a - b);
                        }
                    d2 *= inv_np;
                    double e = d2 - s2;
                    if (e < 0) e = 0;
                    double w = isinf(h) ? 1.0 : exp(-e / (h * h));
                    for (int c = 0; c < C; ++c) acc[c] += w * y[(size_t)c * HW + (size_t)qy * W + qx];
                    wsum += w;
                }
            }
            for (int c = 0; c < C; ++c) out[(size_t)c * HW + (size_t)py * W + px] = acc[c] / wsum;
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 3x3 convolution (the residual CNN's only layer type)                */
/* ------------------------------------------------------------------ */

/* y[n][co][i][j] = b[co] + sum_{ci,ky,kx} w[co][ky][kx][ci] x[n][ci][i+ky-1][j+kx-1]
 * (cross-correlation, zero padding of 1, NCHW activations, OHWI weights). */
int or_conv3x3(const double *x, int N, int Cin, int H, int W, const double *w, const double *b,
               int Cout, double *y)
{
    size_t HW = (size_t)H * W;
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int co = 0; co < Cout; ++co)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    double s = b ? b[co] : 0.0;
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int yy = i + ky - 1, xx = j + kx - 1;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            for (int ci = 0; ci < Cin; ++ci)
                                s += w[((co * 3 + ky) * 3 + kx) * Cin + ci] *
                                     x[((size_t)n * Cin + ci) * HW + (size_t)yy * W + xx];
                        }
                    y[((size_t)n * Cout + co) * HW + (size_t)i * W + j] = s;
                }
    return 0;
}

/* Gradients of or_conv3x3 given dy = dL/dy:
 *   dx[n][ci][i][j]     = sum_{co,ky,kx} w[co][ky][kx][ci] dy[n][co][i-ky+1][j-kx+1]
 *   dw[co][ky][kx][ci]  = sum_{n,i,j} dy[n][co][i][j] x[n][ci][i+ky-1][j+kx-1]
 *   db[co]              = sum_{n,i,j} dy[n][co][i][j]
 * Any of dx, dw, db may be NULL. */
int or_conv3x3_bwd(const double *x, const double *dy, int N, int Cin, int H, int W,
                   const double *w, int Cout, double *dx, double *dw, double *db)
{
    size_t HW = (size_t)H * W;
    if (dx) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int n = 0; n < N; ++n)
            for (int ci = 0; ci < Cin; ++ci)
                for (int i = 0; i < H; ++i)
                    for (int j = 0; j < W; ++j) {
                        double s = 0.0;
                        for (int co = 0; co < Cout; ++co)
                            for (int ky = 0; ky < 3; ++ky)
                                for (int kx = 0; kx < 3; ++kx) {
                                    int yy = i - ky + 1, xx = j - kx + 1;
                                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                    s += w[((co * 3 + ky) * 3 + kx) * Cin + ci] *
                                         dy[((size_t)n * Cout + co) * HW + (size_t)yy * W + xx];
                                }
                        dx[((size_t)n * Cin + ci) * HW + (size_t)i * W + j] = s;
                    }
    }
    if (dw) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int co = 0; co < Cout; ++co)
            for (int t = 0; t < 9; ++t) {
                int ky = t / 3, kx = t % 3;
                for (int ci = 0; ci < Cin; ++ci) {
                    double s = 0.0;
                    for (int n = 0; n < N; ++n)
                        for (int i = 0; i < H; ++i)
                            for (int j = 0; j < W; ++j) {
                                int yy = i + ky - 1, xx = j + kx - 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                s += dy[((size_t)n * Cout + co) * HW + (size_t)i * W + j] *
                                     x[((size_t)n * Cin + ci) * HW + (size_t)yy * W + xx];
                            }
                    dw[((co * 3 + ky) * 3 + kx) * Cin + ci] = s;
                }
            }
    }
    if (db) {
        for (int co = 0; co < Cout; ++co) {
            double s = 0.0;
            for (int n = 0; n < N; ++n)
                for (size_t p = 0; p < HW; ++p) s += dy[((size_t)n * Cout + co) * HW + p];
            db[co] = s;
        }
    }
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

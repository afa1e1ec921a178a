/*
 * epll_oracle.c -- ORACLE (test infrastructure only).
 *
 * A plain, slow, FP64 CPU implementation of the EPLL half-quadratic-splitting
 * restorer with the fast-EPLL accelerations (Parameswaran, Deledalle, Denis &
 * Nguyen, "Accelerating GMM-based patch priors for image restoration: three
 * ingredients for a 100x speed-up").  It exists so that tests can check the
 * CUDA library against an independent reading of the paper, and so that the
 * benchmark can time the method on host cores.  Only tests/, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Equations are numbered in order of appearance in the paper: Eq. 1 EPLL
 * objective, Eq. 2 GMM prior, Eqs. 3-5 half-quadratic splitting, Algorithm 1
 * (five steps), Eq. 6 closed-form image update, Eqs. 7-10 eigenspace form,
 * Eqs. 11-12 flat-tail identities, Eqs. 13-16 flat-tail form, Eq. 17
 * symmetric KL, Eq. 18 clustering cost, Eq. 19 GMM collapse, Eq. 20 jitter.
 *
 * Readings where the paper is silent:
 *  - periodic boundaries; patch anchor = top-left pixel; element e = 8u+v;
 *  - the DC (patch mean) is removed before selection and estimation and
 *    added back unshrunk;
 *  - argmin ties go to the lowest component index;
 *  - a component kept at full rank (r_k = P) has no tail term;
 *  - pixels covered by no sampled patch keep the current estimate;
 *  - sigma enters the 250 sigma^2 cap of lambda in 0..255 grey levels;
 *  - the initialisation weight 0.2 sigma^2 / lambda uses sigma in [0,1]
 *    units and the positive (negated) 5-point Laplacian.
 *
 * Parity pins: tests/test_oracle_pins.py (closed forms, dense literal
 * Algorithm 1, brute force, K = 1 Fourier recursion, dense solves).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PSIDE 8
#define PDIM 64

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: the splitmix64 output function (Steele, Lea */
/* & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014;   */
/* finaliser constants as in Vigna's public-domain splitmix64.c).            */
/* ------------------------------------------------------------------------ */
static const uint64_t OR_GOLDEN = 0x9e3779b97f4a7c15ULL;

static uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* n-th output (n >= 1) of a splitmix64 generator whose state starts at s. */
uint64_t or_splitmix64_nth(uint64_t s, uint64_t n)
{
    return or_mix64(s + n * OR_GOLDEN);
}

/* Draw idx of stream `stream` for seed `seed`: the (idx+1)-th output of the
 * splitmix64 sequence whose state is the stream's first output. */
uint64_t or_rng_u64(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t state = or_splitmix64_nth(seed, stream + 1);
    return or_splitmix64_nth(state, idx + 1);
}

/* Uniform integer in [0, m): high 32 bits times m, shifted (multiply-shift). */
static int or_uniform_int(uint64_t u, int m)
{
    return (int)(((u >> 32) * (uint64_t)m) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Flat-tail approximation (Sec. "Speed-up via flat tail spectrum            */
/* approximation").  Fixed mode: r_k = r for all k.  rho mode: r_k is the    */
/* smallest r with sum_{j<r} S_kj >= rho * sum_j S_kj.  The tail eigenvalue  */
/* lambda_k is the mean of the replaced ones; r_k = P means no tail.         */
/* ------------------------------------------------------------------------ */
int or_flat_tail(int K, const double *S, int mode, double param, int *r, double *lam)
{
    for (int k = 0; k < K; ++k) {
        const double *s = S + (size_t)k * PDIM;
        int rk;
        if (mode == 0) {
            rk = (int)param;
            if (rk < 1 || rk > PDIM) return -1;
        } else {
            double tot = 0.0, acc = 0.0;
            for (int j = 0; j < PDIM; ++j) tot += s[j];
            rk = PDIM;
            for (int j = 0; j < PDIM; ++j) {
                acc += s[j];
                if (acc >= param * tot) { rk = j + 1; break; }
            }
        }
        r[k] = rk;
        if (rk < PDIM) {
            double t = 0.0;
            for (int j = rk; j < PDIM; ++j) t += s[j];
            lam[k] = t / (double)(PDIM - rk);
        } else {
            lam[k] = 0.0;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Samplers: the set of patch anchors processed at HQS iteration t.          */
/* ------------------------------------------------------------------------ */

/* Every pixel anchors one patch (Eq. 1: one patch per pixel). */
int or_sample_full(int H, int W, int *anchors)
{
    for (int a = 0; a < H * W; ++a) anchors[a] = a;
    return H * W;
}

/* Random fraction: exactly ceil(frac*N) distinct anchors, those with the
 * smallest (key, anchor) where key = high 32 bits of rng(seed, t, anchor);
 * returned in increasing anchor order. */
typedef struct { uint32_t key; int anchor; } or_keyed;

static int or_keyed_cmp(const void *pa, const void *pb)
{
    const or_keyed *a = (const or_keyed *)pa, *b = (const or_keyed *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->anchor > b->anchor) - (a->anchor < b->anchor);
}

static int or_int_cmp(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    return (a > b) - (a < b);
}

int or_sample_fraction(int H, int W, double frac, uint64_t seed, int t, int *anchors)
{
    int N = H * W;
    int M = (int)ceil(frac * (double)N);
    if (M > N) M = N;
    or_keyed *kv = (or_keyed *)malloc(sizeof(or_keyed) * (size_t)N);
    if (!kv) return -1;
    for (int a = 0; a < N; ++a) {
        kv[a].key = (uint32_t)(or_rng_u64(seed, (uint64_t)t, (uint64_t)a) >> 32);
        kv[a].anchor = a;
    }
    qsort(kv, (size_t)N, sizeof(or_keyed), or_keyed_cmp);
    for (int m = 0; m < M; ++m) anchors[m] = kv[m].anchor;
    free(kv);
    qsort(anchors, (size_t)M, sizeof(int), or_int_cmp);
    return M;
}

/* Jittered grid (Sec. "Speed-up via the restriction to a random subset of
 * patches", Eq. 20): grid spacing s, a global shift (g_i, g_j) uniform in
 * {0..s-1}^2 redrawn every iteration, grid points i0 = g_i + s n for
 * n = 0..ceil(H/s)-1 (likewise for columns), each moved by independent
 * uniform offsets in [-J, J] per axis, J = floor((8 - s)/2); positions are
 * taken modulo the image size.  Draw indices: 0 and 1 are the shift, then
 * 2 + 2g and 3 + 2g the row and column offsets of grid point g (raster
 * order).  Returned in grid order (duplicates, possible only across the
 * wrap-around seam, are kept). */
int or_sample_jitter(int H, int W, int s, uint64_t seed, int t, int *anchors)
{
    if (s < 1 || s > PSIDE) return -1;
    int J = (PSIDE - s) / 2;
    int gi = or_uniform_int(or_rng_u64(seed, (uint64_t)t, 0), s);
    int gj = or_uniform_int(or_rng_u64(seed, (uint64_t)t, 1), s);
    int ni = (H + s - 1) / s, nj = (W + s - 1) / s;
    int g = 0;
    for (int n = 0; n < ni; ++n) {
        for (int m = 0; m < nj; ++m, ++g) {
            int di = or_uniform_int(or_rng_u64(seed, (uint64_t)t, 2 + 2 * (uint64_t)g), 2 * J + 1) - J;
            int dj = or_uniform_int(or_rng_u64(seed, (uint64_t)t, 3 + 2 * (uint64_t)g), 2 * J + 1) - J;
            int i = ((gi + s * n + di) % H + H) % H;
            int j = ((gj + s * m + dj) % W + W) % W;
            anchors[g] = i * W + j;
        }
    }
    return g;
}

/* Regular patch subsampling (Sec. "Speed-up via the restriction to a random
 * subset of patches"): the grid of spacing s in both directions, points
 * (s n, s m) for n = 0..ceil(H/s)-1, m = 0..ceil(W/s)-1, the same at every
 * iteration (origin 0: a reading, the paper draws the grid from an arbitrary
 * (i0, j0)).  Raster order; no point wraps, so there are no duplicates. */
int or_sample_regular(int H, int W, int s, int *anchors)
{
    if (s < 1 || s > PSIDE) return -1;
    int g = 0;
    for (int i = 0; i < H; i += s)
        for (int j = 0; j < W; j += s) anchors[g++] = i * W + j;
    return g;
}

/* `valid` boundary: every patch that lies entirely inside the image (anchor */
/* rows 0..H-8, columns 0..W-8), raster order; no patch wraps around.        */
int or_sample_valid(int H, int W, int *anchors)
{
    if (H < PSIDE || W < PSIDE) return -1;
    int g = 0;
    for (int i = 0; i + PSIDE <= H; ++i)
        for (int j = 0; j + PSIDE <= W; ++j) anchors[g++] = i * W + j;
    return g;
}

/* Number of valid patches covering each pixel, divided by P: the diagonal of  */
/* sum_i P_i^T P_i / P in Eq. 6 (1 inside, down to 1/P at a corner).           */
void or_valid_weights(int H, int W, double *wgt)
{
    for (int i = 0; i < H; ++i) {
        int ci = (i < H - PSIDE ? i : H - PSIDE) - (i - PSIDE + 1 > 0 ? i - PSIDE + 1 : 0) + 1;
        for (int j = 0; j < W; ++j) {
            int cj = (j < W - PSIDE ? j : W - PSIDE) - (j - PSIDE + 1 > 0 ? j - PSIDE + 1 : 0) + 1;
            wgt[(size_t)i * W + j] = (double)(ci * cj) / (double)PDIM;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Per-beta quantities (Eqs. 8 and 14): nu_kj = S_kj + 1/beta for j < r_k,   */
/* nu_kP = lambda_k + 1/beta, gamma = S / nu, iota_k = -2 log w_k.           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double nu[PDIM], gam[PDIM];  /* j < r_k */
    double nuP, gamP;            /* tail (unused when r_k = P) */
    double iota;
    int r;
} or_comp;

static void or_tables(int K, const double *w, const double *S, const int *r,
                      const double *lam, double beta, or_comp *c)
{
    double ib = 1.0 / beta;
    for (int k = 0; k < K; ++k) {
        c[k].r = r[k];
        c[k].iota = -2.0 * log(w[k]);
        for (int j = 0; j < r[k]; ++j) {
            c[k].nu[j] = S[(size_t)k * PDIM + j] + ib;
            c[k].gam[j] = S[(size_t)k * PDIM + j] / c[k].nu[j];
        }
        if (r[k] < PDIM) {
            c[k].nuP = lam[k] + ib;
            c[k].gamP = lam[k] / c[k].nuP;
        } else {
            c[k].nuP = 0.0;
            c[k].gamP = 0.0;
        }
    }
}

/* Score of component k for a DC-free patch zt (Gaussian selection step of
 * Algorithm 1 in the flat-tail form of Eq. 14; Eq. 8 when r_k = P):
 *   iota_k + sum_{j<r} (log nu_kj + c_j^2/nu_kj)
 *          + (P - r)(log nu_kP) + |zt|^2/nu_kP - sum_{j<r} c_j^2/nu_kP,
 * with c = Ubar_k^T zt (Eq. 13).  c is returned for the estimation step. */
static double or_score(const or_comp *ck, const double *Uk, const double *zt, double zz, double *c)
{
    int r = ck->r;
    double s = ck->iota;
    for (int j = 0; j < r; ++j) {
        double cj = 0.0;
        for (int e = 0; e < PDIM; ++e) cj += Uk[(size_t)e * PDIM + j] * zt[e];
        c[j] = cj;
        s += log(ck->nu[j]) + cj * cj / ck->nu[j];
    }
    if (r < PDIM) {
        s += (double)(PDIM - r) * log(ck->nuP) + zz / ck->nuP;
        for (int j = 0; j < r; ++j) s -= c[j] * c[j] / ck->nuP;
    }
    return s;
}

/* All K scores of the patch at anchor a of image x (H x W, periodic). */
static void or_extract(const double *x, int H, int W, int a, double *zt, double *mu, double *zz)
{
    int ai = a / W, aj = a % W;
    double z[PDIM], m = 0.0;
    for (int u = 0; u < PSIDE; ++u)
        for (int v = 0; v < PSIDE; ++v) {
            z[u * PSIDE + v] = x[(size_t)((ai + u) % H) * W + (aj + v) % W];
        }
    for (int e = 0; e < PDIM; ++e) m += z[e];
    m /= (double)PDIM;
    double q = 0.0;
    for (int e = 0; e < PDIM; ++e) {
        zt[e] = z[e] - m;
        q += zt[e] * zt[e];
    }
    *mu = m;
    *zz = q;
}

/* Scores of all K components for the patches at the given anchors
 * (row-major n x K), for brute-force and tie tests. */
void or_scores(int K, const double *w, const double *U, const double *S, const int *r,
               const double *lam, double beta, const double *x, int H, int W,
               const int *anchors, int n, double *scores)
{
    or_comp *cm = (or_comp *)malloc(sizeof(or_comp) * (size_t)K);
    or_tables(K, w, S, r, lam, beta, cm);
    for (int i = 0; i < n; ++i) {
        double zt[PDIM], c[PDIM], mu, zz;
        or_extract(x, H, W, anchors[i], zt, &mu, &zz);
        for (int k = 0; k < K; ++k)
            scores[(size_t)i * K + k] = or_score(&cm[k], U + (size_t)k * PDIM * PDIM, zt, zz, c);
    }
    free(cm);
}

/* ------------------------------------------------------------------------ */
/* Patch step: the first four steps of Algorithm 1 on the sampled set.        */
/*  - patch extraction: zt_i = P_i x - mean;                                  */
/*  - Gaussian selection: k*_i = argmin_k score (lowest k on ties);           */
/*  - patch estimation (Eqs. 15-16): chat_j = (gamma_j - gamma_P) c_j,        */
/*    zhat = Ubar chat + gamma_P zt, plus the mean;                           */
/*  - patch reprojection: average of the estimates covering each pixel; a     */
/*    pixel covered by no sampled patch keeps x (subset reading, Sec. on the  */
/*    random subset of patches).                                              */
/* forced_k (nullable) replaces the selection (teacher forcing).  kstar, gap  */
/* (second-best minus best score) and best (nullable) are per sampled patch. */
/* ------------------------------------------------------------------------ */
int or_patch_step(int K, const double *w, const double *U, const double *S, const int *r,
                  const double *lam, double beta, const double *x, int H, int W,
                  const int *anchors, int n, const int *forced_k,
                  double *xtilde, int *kstar, double *gap, double *best)
{
    int N = H * W;
    or_comp *cm = (or_comp *)malloc(sizeof(or_comp) * (size_t)K);
    double *zhat = (double *)malloc(sizeof(double) * (size_t)n * PDIM);
    double *sum = (double *)calloc((size_t)N, sizeof(double));
    int *cnt = (int *)calloc((size_t)N, sizeof(int));
    if (!cm || !zhat || !sum || !cnt) { free(cm); free(zhat); free(sum); free(cnt); return -1; }
    or_tables(K, w, S, r, lam, beta, cm);

#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double zt[PDIM], c[PDIM], cb[PDIM], mu, zz;
        or_extract(x, H, W, anchors[i], zt, &mu, &zz);
        int kb = -1;
        double s1 = INFINITY, s2 = INFINITY;
        for (int k = 0; k < K; ++k) {
            double s = or_score(&cm[k], U + (size_t)k * PDIM * PDIM, zt, zz, c);
            if (s < s1) {
                s2 = s1; s1 = s; kb = k;
                memcpy(cb, c, sizeof(double) * (size_t)cm[k].r);
            } else if (s < s2) {
                s2 = s;
            }
        }
        if (forced_k) {
            kb = forced_k[i];
            or_score(&cm[kb], U + (size_t)kb * PDIM * PDIM, zt, zz, cb);
        }
        if (kstar) kstar[i] = kb;
        if (gap) gap[i] = s2 - s1;
        if (best) best[i] = s1;
        const or_comp *ck = &cm[kb];
        const double *Uk = U + (size_t)kb * PDIM * PDIM;
        double ch[PDIM];
        for (int j = 0; j < ck->r; ++j) ch[j] = (ck->gam[j] - ck->gamP) * cb[j];
        for (int e = 0; e < PDIM; ++e) {
            double v = ck->gamP * zt[e];
            for (int j = 0; j < ck->r; ++j) v += Uk[(size_t)e * PDIM + j] * ch[j];
            zhat[(size_t)i * PDIM + e] = v + mu;
        }
    }

    for (int i = 0; i < n; ++i) {
        int ai = anchors[i] / W, aj = anchors[i] % W;
        for (int u = 0; u < PSIDE; ++u)
            for (int v = 0; v < PSIDE; ++v) {
                size_t p = (size_t)((ai + u) % H) * W + (aj + v) % W;
                sum[p] += zhat[(size_t)i * PDIM + u * PSIDE + v];
                cnt[p] += 1;
            }
    }
    for (int p = 0; p < N; ++p) xtilde[p] = cnt[p] ? sum[p] / (double)cnt[p] : x[p];
    free(cm); free(zhat); free(sum); free(cnt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transform, FP64, own mixed-radix recursion:              */
/* X[k] = sum_n x[n] exp(-2 pi i k n / L).  Smallest prime factor first,     */
/* direct sum for a prime length.                                            */
/* ------------------------------------------------------------------------ */
static void or_dft1(double complex *x, int L, int stride, int inverse, double complex *tmp)
{
    if (L == 1) return;
    int p = 2;
    while (p * p <= L && L % p) ++p;
    if (L % p) p = L;
    double sg = inverse ? 1.0 : -1.0;
    if (p == L) {
        for (int k = 0; k < L; ++k) {
            double complex acc = 0.0;
            for (int m = 0; m < L; ++m)
                acc += x[(size_t)m * stride] * cexp(sg * 2.0 * M_PI * I * (double)(((long)k * m) % L) / (double)L);
            tmp[k] = acc;
        }
        for (int k = 0; k < L; ++k) x[(size_t)k * stride] = tmp[k];
        return;
    }
    int q = L / p;
    /* sub-sequences x[rr + p m], m = 0..q-1, transformed in place */
    for (int rr = 0; rr < p; ++rr) or_dft1(x + (size_t)rr * stride, q, stride * p, inverse, tmp);
    /* combine: X[k] = sum_rr w^(rr k) Y_rr[k mod q] */
    for (int k = 0; k < L; ++k) {
        double complex acc = 0.0;
        for (int rr = 0; rr < p; ++rr)
            acc += x[(size_t)(rr + p * (k % q)) * stride] *
                   cexp(sg * 2.0 * M_PI * I * (double)(((long)rr * k) % L) / (double)L);
        tmp[k] = acc;
    }
    for (int k = 0; k < L; ++k) x[(size_t)k * stride] = tmp[k];
}

/* 2-D transform of an H x W array in place; the inverse includes 1/(HW). */
static void or_dft2(double complex *X, int H, int W, int inverse)
{
    int L = H > W ? H : W;
    double complex *tmp = (double complex *)malloc(sizeof(double complex) * (size_t)L);
    for (int i = 0; i < H; ++i) or_dft1(X + (size_t)i * W, W, 1, inverse, tmp);
    for (int j = 0; j < W; ++j) or_dft1(X + j, H, W, inverse, tmp);
    if (inverse) {
        double s = 1.0 / ((double)H * (double)W);
        for (size_t p = 0; p < (size_t)H * W; ++p) X[p] *= s;
    }
    free(tmp);
}

/* Forward 2-D DFT of a real array (exposed for the FFT pin). */
void or_dft2_real(const double *x, int H, int W, double *re, double *im)
{
    double complex *X = (double complex *)malloc(sizeof(double complex) * (size_t)H * W);
    for (size_t p = 0; p < (size_t)H * W; ++p) X[p] = x[p];
    or_dft2(X, H, W, 0);
    for (size_t p = 0; p < (size_t)H * W; ++p) { re[p] = creal(X[p]); im[p] = cimag(X[p]); }
    free(X);
}

/* Transfer function of a periodic blur: the kh x kw kernel with its centre
 * (kh/2, kw/2) at pixel (0, 0), wrapped onto H x W, then transformed. */
static void or_kernel_otf(const double *kern, int kh, int kw, int H, int W, double complex *Hh)
{
    memset(Hh, 0, sizeof(double complex) * (size_t)H * W);
    for (int u = 0; u < kh; ++u)
        for (int v = 0; v < kw; ++v) {
            int i = ((u - kh / 2) % H + H) % H, j = ((v - kw / 2) % W + W) % W;
            Hh[(size_t)i * W + j] += kern[u * kw + v];
        }
    or_dft2(Hh, H, W, 0);
}

/* ------------------------------------------------------------------------ */
/* lambda (Sec. "Parameter settings"):                                       */
/*   min{ N^-1 ||A^T A||_F^2 ||A||_2^-2 , 250 sigma^2 },  sigma in 0..255.   */
/* kind 0 denoise (A = I), 1 pixelwise A = diag(a), 2 periodic blur.         */
/* ------------------------------------------------------------------------ */
double or_lambda(int kind, const double *a, const double *kern, int kh, int kw,
                 int H, int W, double sigma)
{
    size_t N = (size_t)H * W;
    double v;
    if (kind == 0) {
        v = 1.0;
    } else if (kind == 1) {
        double f = 0.0, mx = 0.0;
        for (size_t p = 0; p < N; ++p) {
            double a2 = a[p] * a[p];
            f += a2 * a2;
            if (a2 > mx) mx = a2;
        }
        v = (f / (double)N) / mx;
    } else {
        double complex *Hh = (double complex *)malloc(sizeof(double complex) * N);
        or_kernel_otf(kern, kh, kw, H, W, Hh);
        double f = 0.0, mx = 0.0;
        for (size_t p = 0; p < N; ++p) {
            double h2 = creal(Hh[p]) * creal(Hh[p]) + cimag(Hh[p]) * cimag(Hh[p]);
            f += h2 * h2;
            if (h2 > mx) mx = h2;
        }
        free(Hh);
        v = (f / (double)N) / mx;
    }
    double s255 = 255.0 * sigma;
    double cap = 250.0 * s255 * s255;
    return v < cap ? v : cap;
}

/* ------------------------------------------------------------------------ */
/* Image estimation (last step of Algorithm 1, Eq. 6 with a constant         */
/* overlap):  xhat = (A^T A + bs I)^-1 (A^T y + bs xtilde),  bs = beta s^2.  */
/* ------------------------------------------------------------------------ */
void or_xupdate_pixelwise(const double *a, const double *y, const double *xtilde,
                          int N, double bs, double *xhat)
{
    for (int p = 0; p < N; ++p) {
        double ap = a ? a[p] : 1.0;
        xhat[p] = (ap * y[p] + bs * xtilde[p]) / (ap * ap + bs);
    }
}

/* Periodic blur: diagonal in the Fourier domain. */
void or_xupdate_conv(const double *kern, int kh, int kw, const double *y,
                     const double *xtilde, int H, int W, double bs, double *xhat)
{
    size_t N = (size_t)H * W;
    double complex *Hh = (double complex *)malloc(sizeof(double complex) * N);
    double complex *Y = (double complex *)malloc(sizeof(double complex) * N);
    double complex *X = (double complex *)malloc(sizeof(double complex) * N);
    or_kernel_otf(kern, kh, kw, H, W, Hh);
    for (size_t p = 0; p < N; ++p) { Y[p] = y[p]; X[p] = xtilde[p]; }
    or_dft2(Y, H, W, 0);
    or_dft2(X, H, W, 0);
    for (size_t p = 0; p < N; ++p) {
        double h2 = creal(Hh[p]) * creal(Hh[p]) + cimag(Hh[p]) * cimag(Hh[p]);
        X[p] = (conj(Hh[p]) * Y[p] + bs * X[p]) / (h2 + bs);
    }
    or_dft2(X, H, W, 1);
    for (size_t p = 0; p < N; ++p) xhat[p] = creal(X[p]);
    free(Hh); free(Y); free(X);
}

/* ------------------------------------------------------------------------ */
/* Initialisation (Sec. "Parameter settings"): denoising starts from y; an    */
/* inverse problem from (A^T A + c L)^-1 A^T y, c = 0.2 sigma^2 / lambda,      */
/* L the periodic 5-point negative Laplacian, symbol 4 - 2cos w1 - 2cos w2.  */
/* ------------------------------------------------------------------------ */
void or_init_conv(const double *kern, int kh, int kw, const double *y, int H, int W,
                  double c, double *x0)
{
    size_t N = (size_t)H * W;
    double complex *Hh = (double complex *)malloc(sizeof(double complex) * N);
    double complex *Y = (double complex *)malloc(sizeof(double complex) * N);
    or_kernel_otf(kern, kh, kw, H, W, Hh);
    for (size_t p = 0; p < N; ++p) Y[p] = y[p];
    or_dft2(Y, H, W, 0);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            size_t p = (size_t)i * W + j;
            double Lh = 4.0 - 2.0 * cos(2.0 * M_PI * i / H) - 2.0 * cos(2.0 * M_PI * j / W);
            double h2 = creal(Hh[p]) * creal(Hh[p]) + cimag(Hh[p]) * cimag(Hh[p]);
            Y[p] = conj(Hh[p]) * Y[p] / (h2 + c * Lh);
        }
    or_dft2(Y, H, W, 1);
    for (size_t p = 0; p < N; ++p) x0[p] = creal(Y[p]);
    free(Hh); free(Y);
}

/* (diag(a^2) + c L) v */
static void or_apply_pw(const double *a, double c, const double *v, int H, int W, double *out)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            size_t p = (size_t)i * W + j;
            double lap = 4.0 * v[p] - v[(size_t)((i + H - 1) % H) * W + j] - v[(size_t)((i + 1) % H) * W + j]
                       - v[(size_t)i * W + (j + W - 1) % W] - v[(size_t)i * W + (j + 1) % W];
            out[p] = a[p] * a[p] * v[p] + c * lap;
        }
}

/* Pixelwise A: conjugate gradients on (diag(a^2) + c L) x = a y from x = a y,
 * a fixed number of iterations; it stops early only once the recurrence has
 * converged to the point where d^T q is no longer positive (the system matrix
 * is positive definite, so this happens only when r and d underflow). */
void or_init_cg(const double *a, const double *y, int H, int W, double c, int iters, double *x)
{
    size_t N = (size_t)H * W;
    double *r = (double *)malloc(sizeof(double) * N), *d = (double *)malloc(sizeof(double) * N),
           *q = (double *)malloc(sizeof(double) * N);
    for (size_t p = 0; p < N; ++p) x[p] = a[p] * y[p];
    or_apply_pw(a, c, x, H, W, q);
    double rr = 0.0;
    for (size_t p = 0; p < N; ++p) { r[p] = a[p] * y[p] - q[p]; d[p] = r[p]; rr += r[p] * r[p]; }
    for (int it = 0; it < iters && rr > 0.0; ++it) {
        or_apply_pw(a, c, d, H, W, q);
        double dq = 0.0;
        for (size_t p = 0; p < N; ++p) dq += d[p] * q[p];
        if (!(dq > 0.0)) break;
        double alpha = rr / dq;
        double rr2 = 0.0;
        for (size_t p = 0; p < N; ++p) { x[p] += alpha * d[p]; r[p] -= alpha * q[p]; rr2 += r[p] * r[p]; }
        double b = rr2 / rr;
        for (size_t p = 0; p < N; ++p) d[p] = r[p] + b * d[p];
        rr = rr2;
    }
    free(r); free(d); free(q);
}

static void or_blur(const double *kern, int kh, int kw, const double *x, int H, int W, int adjoint,
                    double *out);

/* ------------------------------------------------------------------------ */
/* Image update with a non-constant patch overlap (Eq. 6 with the `valid`     */
/* boundary): sum_i P_i^T P_i = P diag(w) and sum_i P_i^T zhat_i = P w xt, so */
/*   x = (A^T A + bs diag(w))^-1 (A^T y + bs w xt).                            */
/* Pixelwise A = diag(a) (a NULL: denoising): per pixel.  Periodic blur: the  */
/* matrix is no longer diagonal in the Fourier basis; conjugate gradients in  */
/* the pixel domain from x = xt, a fixed number of iterations (`iters`),      */
/* stopping early only once the residual vanishes.                           */
/* ------------------------------------------------------------------------ */
void or_xupdate_weighted(int deg_kind, const double *a, const double *kern, int kh, int kw, const double *y,
                         const double *xt, const double *wgt, int H, int W, double bs, int iters, double *x)
{
    size_t N = (size_t)H * W;
    if (deg_kind != 2) {
        for (size_t p = 0; p < N; ++p) {
            double ap = (deg_kind == 1 && a) ? a[p] : 1.0;
            x[p] = (ap * y[p] + bs * wgt[p] * xt[p]) / (ap * ap + bs * wgt[p]);
        }
        return;
    }
    double *b = (double *)malloc(sizeof(double) * N), *r = (double *)malloc(sizeof(double) * N),
           *d = (double *)malloc(sizeof(double) * N), *q = (double *)malloc(sizeof(double) * N),
           *t = (double *)malloc(sizeof(double) * N);
    /* (B^T B + bs diag(w)) v */
#define OR_APPLY(v, out)                                                   \
    do {                                                                   \
        or_blur(kern, kh, kw, v, H, W, 0, t);                              \
        or_blur(kern, kh, kw, t, H, W, 1, out);                            \
        for (size_t p_ = 0; p_ < N; ++p_) out[p_] += bs * wgt[p_] * v[p_]; \
    } while (0)
    or_blur(kern, kh, kw, y, H, W, 1, b);
    for (size_t p = 0; p < N; ++p) { b[p] += bs * wgt[p] * xt[p]; x[p] = xt[p]; }
    OR_APPLY(x, q);
    double rr = 0.0;
    for (size_t p = 0; p < N; ++p) { r[p] = b[p] - q[p]; d[p] = r[p]; rr += r[p] * r[p]; }
    for (int it = 0; it < iters && rr > 0.0; ++it) {
        OR_APPLY(d, q);
        double dq = 0.0;
        for (size_t p = 0; p < N; ++p) dq += d[p] * q[p];
        if (!(dq > 0.0)) break;
        double alpha = rr / dq, rr2 = 0.0;
        for (size_t p = 0; p < N; ++p) { x[p] += alpha * d[p]; r[p] -= alpha * q[p]; rr2 += r[p] * r[p]; }
        double bt = rr2 / rr;
        for (size_t p = 0; p < N; ++p) d[p] = r[p] + bt * d[p];
        rr = rr2;
    }
#undef OR_APPLY
    free(b); free(r); free(d); free(q); free(t);
}

/* ------------------------------------------------------------------------ */
/* Super-resolution, A = S B (Sec. "Complexity via eigenspace                 */
/* implementation" counts super-resolution among the problems whose image    */
/* update is an O(N log N) Fourier computation; Fig. 8 shows x3).  B is the  */
/* periodic blur above and S keeps pixel (d i, d j) of every d x d block, so  */
/* y is (H/d) x (W/d).  The oracle applies A and A^T in the pixel domain and  */
/* solves the image update and the initialisation by conjugate gradients in  */
/* FP64 run to convergence: a route independent of any Fourier-domain        */
/* closed form.                                                              */
/* ------------------------------------------------------------------------ */
/* out = kern (*) x (adjoint: correlation), periodic, kernel centre (kh/2, kw/2) */
static void or_blur(const double *kern, int kh, int kw, const double *x, int H, int W, int adjoint,
                    double *out)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int u = 0; u < kh; ++u)
                for (int v = 0; v < kw; ++v) {
                    int di = u - kh / 2, dj = v - kw / 2;
                    if (adjoint) { di = -di; dj = -dj; }
                    int ii = ((i - di) % H + H) % H, jj = ((j - dj) % W + W) % W;
                    acc += kern[u * kw + v] * x[(size_t)ii * W + jj];
                }
            out[(size_t)i * W + j] = acc;
        }
}

/* ylow = S B x */
void or_sr_apply(const double *kern, int kh, int kw, const double *x, int H, int W, int d, double *ylow)
{
    double *bx = (double *)malloc(sizeof(double) * (size_t)H * W);
    or_blur(kern, kh, kw, x, H, W, 0, bx);
    int h = H / d, w = W / d;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) ylow[(size_t)i * w + j] = bx[(size_t)(d * i) * W + d * j];
    free(bx);
}

/* x = B^T S^T ylow (zero insertion, then correlation with the kernel) */
void or_sr_adjoint(const double *kern, int kh, int kw, const double *ylow, int H, int W, int d, double *x)
{
    double *up = (double *)calloc((size_t)H * W, sizeof(double));
    int h = H / d, w = W / d;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) up[(size_t)(d * i) * W + d * j] = ylow[(size_t)i * w + j];
    or_blur(kern, kh, kw, up, H, W, 1, x);
    free(up);
}

/* (A^T A + shift M) v with M = I (lap = 0) or the negative Laplacian (lap = 1) */
typedef struct { const double *kern; int kh, kw, H, W, d, lap; double shift; double *low; } or_sr_op;
static void or_sr_normal(const or_sr_op *o, const double *v, double *out)
{
    or_sr_apply(o->kern, o->kh, o->kw, v, o->H, o->W, o->d, o->low);
    or_sr_adjoint(o->kern, o->kh, o->kw, o->low, o->H, o->W, o->d, out);
    for (int i = 0; i < o->H; ++i)
        for (int j = 0; j < o->W; ++j) {
            size_t p = (size_t)i * o->W + j;
            double m = v[p];
            if (o->lap) {
                int H = o->H, W = o->W;
                m = 4.0 * v[p] - v[(size_t)((i + H - 1) % H) * W + j] - v[(size_t)((i + 1) % H) * W + j]
                  - v[(size_t)i * W + (j + W - 1) % W] - v[(size_t)i * W + (j + 1) % W];
            }
            out[p] += o->shift * m;
        }
}

/* Conjugate gradients on (A^T A + shift M) x = b from the given x, until the
 * residual norm is below rtol |b| (or maxit iterations); returns iterations. */
static int or_sr_cg(const or_sr_op *o, const double *b, double *x, double rtol, int maxit)
{
    size_t N = (size_t)o->H * o->W;
    double *r = (double *)malloc(sizeof(double) * N), *dd = (double *)malloc(sizeof(double) * N),
           *q = (double *)malloc(sizeof(double) * N);
    or_sr_normal(o, x, q);
    double rr = 0.0, bb = 0.0;
    for (size_t p = 0; p < N; ++p) { r[p] = b[p] - q[p]; dd[p] = r[p]; rr += r[p] * r[p]; bb += b[p] * b[p]; }
    int it = 0;
    while (it < maxit && rr > rtol * rtol * bb) {
        or_sr_normal(o, dd, q);
        double dq = 0.0;
        for (size_t p = 0; p < N; ++p) dq += dd[p] * q[p];
        if (!(dq > 0.0)) break;
        double alpha = rr / dq, rr2 = 0.0;
        for (size_t p = 0; p < N; ++p) { x[p] += alpha * dd[p]; r[p] -= alpha * q[p]; rr2 += r[p] * r[p]; }
        double bt = rr2 / rr;
        for (size_t p = 0; p < N; ++p) dd[p] = r[p] + bt * dd[p];
        rr = rr2;
        ++it;
    }
    free(r); free(dd); free(q);
    return it;
}

/* Image update (Eq. 6): x = (A^T A + bs I)^-1 (A^T y + bs xtilde). */
int or_xupdate_sr(const double *kern, int kh, int kw, const double *ylow, const double *xtilde, int H, int W,
                  int d, double bs, double *x)
{
    size_t N = (size_t)H * W;
    double *b = (double *)malloc(sizeof(double) * N);
    or_sr_adjoint(kern, kh, kw, ylow, H, W, d, b);
    for (size_t p = 0; p < N; ++p) { b[p] += bs * xtilde[p]; x[p] = xtilde[p]; }
    or_sr_op o = {kern, kh, kw, H, W, d, 0, bs, (double *)malloc(sizeof(double) * N / ((size_t)d * d))};
    int it = or_sr_cg(&o, b, x, 1e-15, 100000);
    free(o.low); free(b);
    return it;
}

/* Initialisation (Sec. "Parameter settings"): x0 = (A^T A + c L)^-1 A^T y. */
int or_init_sr(const double *kern, int kh, int kw, const double *ylow, int H, int W, int d, double c, double *x)
{
    size_t N = (size_t)H * W;
    double *b = (double *)malloc(sizeof(double) * N);
    or_sr_adjoint(kern, kh, kw, ylow, H, W, d, b);
    for (size_t p = 0; p < N; ++p) x[p] = 0.0;
    or_sr_op o = {kern, kh, kw, H, W, d, 1, c, (double *)malloc(sizeof(double) * N / ((size_t)d * d))};
    int it = or_sr_cg(&o, b, x, 1e-14, 1000000);
    free(o.low); free(b);
    return it;
}

/* lambda for A = S B: A^T A is block diagonal in the Fourier basis, one
 * d^2 x d^2 block per low-resolution frequency w' coupling the d^2
 * frequencies that alias onto it; the block is (1/d^2) g g^H with g the
 * transfer function at those frequencies, so its one non-zero eigenvalue
 * is e(w') = d^-2 sum |B(w'_k)|^2 and its squared Frobenius norm e(w')^2.
 * Hence ||A^T A||_F^2 = sum e^2 and ||A||_2^2 = max e. */
double or_lambda_sr(const double *kern, int kh, int kw, int H, int W, int d, double sigma)
{
    size_t N = (size_t)H * W;
    double complex *Hh = (double complex *)malloc(sizeof(double complex) * N);
    or_kernel_otf(kern, kh, kw, H, W, Hh);
    int h = H / d, w = W / d;
    double f = 0.0, mx = 0.0;
    for (int u = 0; u < h; ++u)
        for (int v = 0; v < w; ++v) {
            double e = 0.0;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double complex z = Hh[(size_t)(u + a * h) * W + (v + b * w)];
                    e += creal(z) * creal(z) + cimag(z) * cimag(z);
                }
            e /= (double)d * d;
            f += e * e;
            if (e > mx) mx = e;
        }
    free(Hh);
    double v = (f / (double)N) / mx;
    double s255 = 255.0 * sigma, cap = 250.0 * s255 * s255;
    return v < cap ? v : cap;
}

/* ------------------------------------------------------------------------ */
/* Whole restoration: Algorithm 1 iterated T times with                       */
/* beta_t = lambda * beta_mult[t] / sigma^2 (Sec. "Parameter settings").      */
/* deg_kind 0 denoise, 1 pixelwise a, 2 periodic blur, 3 blur then          */
/* decimation by `factor` (y is (H/factor) x (W/factor)).  subset 0 full set, */
/* 1 random fraction subset_param, 2 jitter with spacing (int)subset_param,  */
/* 3 regular grid with spacing (int)subset_param, 4 `valid` boundary (every  */
/* patch inside the image, Eq. 6 with its non-constant overlap).             */
/* ks_out / gap_out (nullable) receive each iteration's selections, at       */
/* [t * H * W + i] for the i-th sampled patch; nsel_out[t] their count.       */
/* ------------------------------------------------------------------------ */
int or_restore(int K, const double *w, const double *U, const double *S, const int *r,
               const double *lam, const double *y, int H, int W, int deg_kind,
               const double *a, const double *kern, int kh, int kw, int factor, double sigma,
               const double *beta_mult, int T, int subset, double subset_param,
               uint64_t seed, int cg_iters, double *x,
               int *ks_out, double *gap_out, int *nsel_out)
{
    size_t N = (size_t)H * W;
    double lmb = deg_kind == 3 ? or_lambda_sr(kern, kh, kw, H, W, factor, sigma)
                               : or_lambda(deg_kind, a, kern, kh, kw, H, W, sigma);
    double c0 = 0.2 * sigma * sigma / lmb;
    if (deg_kind == 0) memcpy(x, y, sizeof(double) * N);
    else if (deg_kind == 1) or_init_cg(a, y, H, W, c0, cg_iters, x);
    else if (deg_kind == 2) or_init_conv(kern, kh, kw, y, H, W, c0, x);
    else or_init_sr(kern, kh, kw, y, H, W, factor, c0, x);

    int *anchors = (int *)malloc(sizeof(int) * N);
    double *xt = (double *)malloc(sizeof(double) * N);
    if (!anchors || !xt) { free(anchors); free(xt); return -1; }
    for (int t = 0; t < T; ++t) {
        double bs = lmb * beta_mult[t];          /* beta sigma^2 */
        double beta = bs / (sigma * sigma);
        int n;
        if (subset == 0) n = or_sample_full(H, W, anchors);
        else if (subset == 1) n = or_sample_fraction(H, W, subset_param, seed, t, anchors);
        else if (subset == 2) n = or_sample_jitter(H, W, (int)subset_param, seed, t, anchors);
        else if (subset == 3) n = or_sample_regular(H, W, (int)subset_param, anchors);
        else n = or_sample_valid(H, W, anchors);
        if (n < 0) { free(anchors); free(xt); return -1; }
        if (nsel_out) nsel_out[t] = n;
        if (or_patch_step(K, w, U, S, r, lam, beta, x, H, W, anchors, n, NULL, xt,
                          ks_out ? ks_out + (size_t)t * N : NULL,
                          gap_out ? gap_out + (size_t)t * N : NULL, NULL)) {
            free(anchors); free(xt); return -1;
        }
        if (subset == 4) {
            double *wgt = (double *)malloc(sizeof(double) * N);
            double *xo = (double *)malloc(sizeof(double) * N);
            or_valid_weights(H, W, wgt);
            or_xupdate_weighted(deg_kind, a, kern, kh, kw, y, xt, wgt, H, W, bs, cg_iters, xo);
            memcpy(x, xo, sizeof(double) * N);
            free(wgt); free(xo);
        } else if (deg_kind == 2) or_xupdate_conv(kern, kh, kw, y, xt, H, W, bs, x);
        else if (deg_kind == 3) or_xupdate_sr(kern, kh, kw, y, xt, H, W, factor, bs, x);
        else or_xupdate_pixelwise(deg_kind == 1 ? a : NULL, y, xt, (int)N, bs, x);
    }
    free(anchors); free(xt);
    return 0;
}

/*
 * Plain CPU oracle for fast adaptive bilateral filtering
 * (Gavaskar & Chaudhury, "Fast Adaptive Bilateral Filtering").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA product path never calls
 * it, shares no source with it, and must fail loudly rather than fall back to
 * it.  Everything here is written for obviousness, not speed: windows are
 * summed directly, one pixel at a time.
 *
 * What is computed (paper notation; equation numbers are the paper's):
 *   - the adaptive bilateral filter by brute force, Eqs. (1)-(3), with the box
 *     spatial kernel omega == 1 on the window [-w, w]^2 clipped to the image;
 *   - Algorithm 1 (Sec. II-D), step by step:
 *       alpha_i, beta_i = min / max over the window            Eq. (8)
 *       flat pixels (alpha == beta) return f(i)                Sec. II-A
 *       m_k = sum over the window of f^k, k = 0..N             Eq. (17), App. A
 *       M_k = sum over the window of (f - alpha)^k (integer)   Eq. (24), App. B
 *       mu_k = M_k / (beta - alpha)^k                          Eq. (24)
 *       c = A^{-1} mu with the closed-form Hilbert inverse     Eqs. (18)-(19)
 *       t0 = (theta - alpha)/(beta - alpha),
 *       lambda = (beta - alpha)^2 / (2 sigma^2)                Eq. (25)
 *       I_0 .. I_{N+1}                                         Eqs. (28), (30)-(32)
 *       g = alpha + (beta - alpha) T1 / T2                     Eq. (29)
 *   - the same two with a separable integer spatial kernel omega = g x g on
 *     [-r, r]^2 (the Gaussian of Eq. (4) when the taps are a quantised
 *     Gaussian), moments summed exactly in 128-bit integers (end of file).
 *
 * Readings where the paper is silent (each is also listed in the design
 * notes of the repository):
 *   R1 box spatial kernel, window clipped to the image (no padding values);
 *   R2 M_k is formed exactly in integers as the direct sum of (f - alpha)^k,
 *      which Eq. (24) shows equals the binomial form; mu_k is then one
 *      correctly rounded FP64 division of two exactly representable values;
 *   R3 the integrals are evaluated by the paper's own formulas, Eqs. (31),
 *      (32) and the forward recursion (30), but in IEEE binary128, because
 *      the recursion is numerically unstable in binary64 for small lambda;
 *      Eq. (31) is written with erfc when both erf arguments share a sign
 *      (the same integral, without cancellation); for lambda < 1e-4 the
 *      binary128 recursion is itself not accurate enough and Eq. (28) is
 *      evaluated by 24-point Gauss-Legendre quadrature in binary128;
 *   R4 every I_k is multiplied by the common factor exp(lambda d^2), with d
 *      the distance from t0 to [0, 1]; the factor cancels in Eq. (29) and
 *      keeps the integrals representable when the range-kernel centre lies
 *      far outside [alpha, beta];
 *   R5 if T2 <= 0 or T1 / T2 is not finite (the fitted polynomial is not
 *      required to be non-negative, Sec. II-B), the pixel takes the
 *      sigma -> infinity limit alpha + (beta - alpha) mu_1 / mu_0, i.e. the
 *      box mean, and is counted.
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fPIC -shared -o liboracle.so
 *        fabf_oracle.c -lm   (binary128 math comes from glibc >= 2.26).
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

typedef _Float128 q128;

#define ORACLE_NMAX 6
#define ORACLE_WMAX 40
#define LAMBDA_QUADRATURE 1e-4

/* ------------------------------------------------------------------ */
/* Window helpers (R1)                                                 */
/* ------------------------------------------------------------------ */

static void window_bounds(int H, int W, int y, int x, int w,
                          int* y0, int* y1, int* x0, int* x1)
{
    *y0 = y - w < 0 ? 0 : y - w;
    *y1 = y + w > H - 1 ? H - 1 : y + w;
    *x0 = x - w < 0 ? 0 : x - w;
    *x1 = x + w > W - 1 ? W - 1 : x + w;
}

static int check_args(int H, int W, long pitch, int w, int N)
{
    if (H < 1 || W < 1 || pitch < W) return 1;
    if (w < 1 || w > ORACLE_WMAX) return 1;
    if (N < 0 || N > ORACLE_NMAX) return 1;
    return 0;
}

/* Eq. (8): alpha_i, beta_i are the min and max of the window values. */
static void pixel_bounds(const uint8_t* f, int H, int W, long pitch, int w,
                         int y, int x, int* alpha, int* beta)
{
    int y0, y1, x0, x1, a = 255, b = 0;
    window_bounds(H, W, y, x, w, &y0, &y1, &x0, &x1);
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            int v = f[(long)yy * pitch + xx];
            if (v < a) a = v;
            if (v > b) b = v;
        }
    *alpha = a;
    *beta = b;
}

/* Eq. (17) and App. A: m_k = (omega * f^k)(i) with omega == 1, k = 0..N. */
static void pixel_moments(const uint8_t* f, int H, int W, long pitch, int w,
                          int N, int y, int x, int64_t* m)
{
    int y0, y1, x0, x1;
    window_bounds(H, W, y, x, w, &y0, &y1, &x0, &x1);
    for (int k = 0; k <= N; ++k) m[k] = 0;
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            int64_t v = f[(long)yy * pitch + xx], p = 1;
            for (int k = 0; k <= N; ++k) { m[k] += p; p *= v; }
        }
}

/* Eq. (24) (R2): M_k = sum over the window of (f - alpha)^k, k = 0..K. */
static void pixel_shifted_moments(const uint8_t* f, int H, int W, long pitch,
                                  int w, int K, int alpha, int y, int x,
                                  int64_t* M)
{
    int y0, y1, x0, x1;
    window_bounds(H, W, y, x, w, &y0, &y1, &x0, &x1);
    for (int k = 0; k <= K; ++k) M[k] = 0;
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            int64_t v = (int64_t)f[(long)yy * pitch + xx] - alpha, p = 1;
            for (int k = 0; k <= K; ++k) { M[k] += p; p *= v; }
        }
}

/* ------------------------------------------------------------------ */
/* Hilbert inverse, Eq. (19)                                           */
/* ------------------------------------------------------------------ */

static int64_t binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* (A^{-1})_{m,n}, 1-based indices as in Eq. (19), for the (N+1)x(N+1)
 * Hilbert matrix A_{m,n} = 1/(m+n-1) of Eq. (18). */
static int64_t hilbert_inverse_entry(int N, int m, int n)
{
    int64_t s = ((m + n) % 2 == 0) ? 1 : -1;
    int64_t b = binom(m + n - 2, m - 1);
    return s * (m + n - 1) * binom(N + m, N + 1 - n) * binom(N + n, N + 1 - m) * b * b;
}

int oracle_hilbert_inverse(int N, int64_t* Ainv)
{
    if (N < 0 || N > ORACLE_NMAX) return 1;
    for (int m = 1; m <= N + 1; ++m)
        for (int n = 1; n <= N + 1; ++n)
            Ainv[(m - 1) * (N + 1) + (n - 1)] = hilbert_inverse_entry(N, m, n);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Integrals I_k of Eq. (28) (R3, R4)                                  */
/* ------------------------------------------------------------------ */

/* Nodes and weights of the n-point Gauss-Legendre rule on [0, 1], by Newton
 * iteration on the Legendre polynomial P_n (three-term recurrence). */
static void gauss_legendre01(int n, q128* t, q128* wt)
{
    const q128 pi = 3.141592653589793238462643383279502884Q;
    for (int i = 0; i < n; ++i) {
        q128 x = cosf128(pi * ((q128)i + 0.75Q) / ((q128)n + 0.5Q));
        q128 dp = 0;
        for (int it = 0; it < 100; ++it) {
            q128 p0 = 1, p1 = x;
            for (int j = 2; j <= n; ++j) {
                q128 p2 = (((q128)(2 * j - 1)) * x * p1 - ((q128)(j - 1)) * p0) / (q128)j;
                p0 = p1;
                p1 = p2;
            }
            dp = (q128)n * (x * p1 - p0) / (x * x - 1);
            q128 dx = p1 / dp;
            x -= dx;
            if (fabsf128(dx) < 1e-33Q) break;
        }
        {
            q128 p0 = 1, p1 = x;
            for (int j = 2; j <= n; ++j) {
                q128 p2 = (((q128)(2 * j - 1)) * x * p1 - ((q128)(j - 1)) * p0) / (q128)j;
                p0 = p1;
                p1 = p2;
            }
            dp = (q128)n * (x * p1 - p0) / (x * x - 1);
        }
        t[i] = (1 - x) / 2;
        wt[i] = 1 / ((1 - x * x) * dp * dp);   /* 2/((1-x^2)P'^2), halved for [0,1] */
    }
}

static void integrals_q(q128 lam, q128 t0, int K, q128* I)
{
    if (lam < (q128)LAMBDA_QUADRATURE) {
        /* Eq. (28) by quadrature: the integrand is entire and, for such small
         * lambda, nearly polynomial on [0, 1]. */
        enum { NGL = 24 };
        q128 t[NGL], wt[NGL];
        gauss_legendre01(NGL, t, wt);
        for (int k = 0; k <= K; ++k) I[k] = 0;
        for (int q = 0; q < NGL; ++q) {
            q128 e = wt[q] * expf128(-lam * (t[q] - t0) * (t[q] - t0));
            for (int k = 0; k <= K; ++k) { I[k] += e; e *= t[q]; }
        }
    } else {
        /* Eq. (31): I_0 = 1/2 sqrt(pi/lambda) [erf(u) - erf(v)],
         * u = sqrt(lambda)(1 - t0), v = -sqrt(lambda) t0. */
        const q128 pi = 3.141592653589793238462643383279502884Q;
        q128 sl = sqrtf128(lam);
        q128 u = sl * (1 - t0), v = -sl * t0, diff;
        if (u > 0 && v > 0)      diff = erfcf128(v) - erfcf128(u);
        else if (u < 0 && v < 0) diff = erfcf128(-u) - erfcf128(-v);
        else                     diff = erff128(u) - erff128(v);
        q128 E0 = expf128(-lam * t0 * t0);
        q128 E1 = expf128(-lam * (1 - t0) * (1 - t0));
        I[0] = sqrtf128(pi / lam) / 2 * diff;
        /* Eq. (32). */
        if (K >= 1) I[1] = t0 * I[0] + (E0 - E1) / (2 * lam);
        /* Eq. (30), forward. */
        for (int k = 2; k <= K; ++k)
            I[k] = t0 * I[k - 1] + ((q128)(k - 1)) / (2 * lam) * I[k - 2] - E1 / (2 * lam);
    }
    /* R4: common factor exp(lambda d^2), d = distance from t0 to [0, 1]. */
    q128 d = t0 < 0 ? -t0 : (t0 > 1 ? t0 - 1 : 0);
    if (d > 0) {
        q128 s = expf128(lam * d * d);
        for (int k = 0; k <= K; ++k) I[k] *= s;
    }
}

/* I_0 .. I_K for one (lambda, t0), each scaled by exp(lambda d^2) (R4) and
 * rounded to binary64.  Returns nonzero for lambda <= 0 or K outside 0..16. */
int oracle_integrals(double lam, double t0, int K, double* I)
{
    if (!(lam > 0) || K < 0 || K > 16) return 1;
    q128 Iq[17];
    integrals_q((q128)lam, (q128)t0, K, Iq);
    for (int k = 0; k <= K; ++k) I[k] = (double)Iq[k];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 for one pixel                                           */
/* ------------------------------------------------------------------ */

/* Algorithm 1 from the shifted-and-scaled moments mu_0..mu_max(N,1) on: the
 * fit (Eq. (19), fused multiply-adds over ascending k), t0 and lambda
 * (Eq. (25)), the integrals (Eq. (28)), and the ratio (Eq. (29)) with the
 * reading R5 for a non-positive denominator.  Writes c[N+1], t0lam[2],
 * I[N+2], T[2], *g and ORs bit1 into *flags on the fallback. */
/* The fit of Algorithm 1: c = A^{-1} mu (Eq. (19)), each coefficient a chain
 * of fused multiply-adds over ascending k starting from zero. */
static void fit(int N, const int64_t* Ainv, const double* mu, double* c)
{
    for (int n = 0; n <= N; ++n) {
        double acc = 0.0;
        for (int k = 0; k <= N; ++k) acc = fma((double)Ainv[n * (N + 1) + k], mu[k], acc);
        c[n] = acc;
    }
}

static void fabf_tail(int N, const int64_t* Ainv, int alpha, int d, const double* mu, double th,
                      double s, double* g_out, double* c, double* t0lam, double* I, double* T,
                      int* flags)
{
    fit(N, Ainv, mu, c);
    const double t0 = (th - (double)alpha) / (double)d;
    const double lam = (double)(d * d) / (2.0 * s * s);
    oracle_integrals(lam, t0, N + 1, I);
    double T1 = c[0] * I[1], T2 = c[0] * I[0];
    for (int k = 2; k <= N + 1; ++k) {
        T1 = fma(c[k - 1], I[k], T1);
        T2 = fma(c[k - 1], I[k - 1], T2);
    }
    double F = T1 / T2;
    if (!(T2 > 0.0) || !isfinite(F)) {
        F = mu[1] / mu[0];                        /* R5 */
        *flags |= 2;
    }
    *g_out = (double)alpha + (double)d * F;
    t0lam[0] = t0;
    t0lam[1] = lam;
    T[0] = T1;
    T[1] = T2;
}

/* Trace of every intermediate of Algorithm 1 at one pixel.  Arrays hold
 * N+1 entries (m, M, mu, c) or N+2 (I).  flags: bit0 flat (alpha == beta),
 * bit1 fallback R5 taken.  Any pointer may be NULL. */
static int fabf_pixel(const uint8_t* f, const float* theta, const float* sigma,
                      int H, int W, long pitch, int w, int N, int y, int x,
                      const int64_t* Ainv, double* g_out,
                      int* alpha_out, int* beta_out, int64_t* m_out,
                      int64_t* M_out, double* mu_out, double* c_out,
                      double* t0lam_out, double* I_out, double* T_out,
                      int* flags_out)
{
    int alpha, beta, flags = 0;
    pixel_bounds(f, H, W, pitch, w, y, x, &alpha, &beta);
    if (alpha_out) *alpha_out = alpha;
    if (beta_out) *beta_out = beta;
    if (m_out) pixel_moments(f, H, W, pitch, w, N, y, x, m_out);
    if (alpha == beta) {
        /* Sec. II-A and Algorithm 1: flat window, g(i) = f(i). */
        *g_out = (double)f[(long)y * pitch + x];
        if (flags_out) *flags_out = 1;
        return 0;
    }
    const int d = beta - alpha;
    int64_t M[ORACLE_NMAX + 2];
    double mu[ORACLE_NMAX + 2], c[ORACLE_NMAX + 1], I[ORACLE_NMAX + 2], t0lam[2], T[2];
    const int K = N < 1 ? 1 : N;     /* mu_1 is needed by R5 even for N = 0 */
    pixel_shifted_moments(f, H, W, pitch, w, K, alpha, y, x, M);
    int64_t dk = 1;
    for (int k = 0; k <= K; ++k) {
        mu[k] = (double)M[k] / (double)dk;     /* Eq. (24), R2 */
        dk *= d;
    }
    fabf_tail(N, Ainv, alpha, d, mu, (double)theta[(long)y * W + x], (double)sigma[(long)y * W + x],
              g_out, c, &t0lam[0], I, &T[0], &flags);
    if (M_out) for (int k = 0; k <= N; ++k) M_out[k] = M[k];
    if (mu_out) for (int k = 0; k <= N; ++k) mu_out[k] = mu[k];
    if (c_out) for (int k = 0; k <= N; ++k) c_out[k] = c[k];
    if (t0lam_out) { t0lam_out[0] = t0lam[0]; t0lam_out[1] = t0lam[1]; }
    if (I_out) for (int k = 0; k <= N + 1; ++k) I_out[k] = I[k];
    if (T_out) { T_out[0] = T[0]; T_out[1] = T[1]; }
    if (flags_out) *flags_out = flags;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exported entry points                                               */
/* ------------------------------------------------------------------ */

/* The fit step alone on given moments mu[0..N]: c[0..N] = A^{-1} mu as in
 * Algorithm 1 (the moments may carry any common scale; the fit is linear). */
int oracle_fit(int N, const double* mu, double* c)
{
    if (N < 0 || N > ORACLE_NMAX || !mu || !c) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    fit(N, Ainv, mu, c);
    return 0;
}

/* alpha, beta: H x W uint8, row stride W. */
int oracle_bounds(const uint8_t* f, int H, int W, long pitch, int w,
                  uint8_t* alpha, uint8_t* beta)
{
    if (check_args(H, W, pitch, w, 0)) return 1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int a, b;
            pixel_bounds(f, H, W, pitch, w, y, x, &a, &b);
            alpha[(long)y * W + x] = (uint8_t)a;
            beta[(long)y * W + x] = (uint8_t)b;
        }
    return 0;
}

/* m: (N+1) x H x W int64, plane k holds m_k. */
int oracle_moments(const uint8_t* f, int H, int W, long pitch, int w, int N,
                   int64_t* m)
{
    if (check_args(H, W, pitch, w, N)) return 1;
    const long plane = (long)H * W;
    int64_t mk[ORACLE_NMAX + 1];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            pixel_moments(f, H, W, pitch, w, N, y, x, mk);
            for (int k = 0; k <= N; ++k) m[k * plane + (long)y * W + x] = mk[k];
        }
    return 0;
}

/* M: (N+1) x H x W int64, plane k holds M_k = sum (f - alpha)^k. */
int oracle_shifted_moments(const uint8_t* f, int H, int W, long pitch, int w,
                           int N, int64_t* M)
{
    if (check_args(H, W, pitch, w, N)) return 1;
    const long plane = (long)H * W;
    int64_t Mk[ORACLE_NMAX + 1];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int a, b;
            pixel_bounds(f, H, W, pitch, w, y, x, &a, &b);
            pixel_shifted_moments(f, H, W, pitch, w, N, a, y, x, Mk);
            for (int k = 0; k <= N; ++k) M[k * plane + (long)y * W + x] = Mk[k];
        }
    return 0;
}

/* Algorithm 1 at the n pixels (ys[j], xs[j]); out[j] = g_hat.  theta and
 * sigma are H x W float32 with row stride W.  *n_fallback (may be NULL)
 * receives the number of pixels that took reading R5. */
int oracle_fabf_pixels(const uint8_t* f, const float* theta, const float* sigma,
                       int H, int W, long pitch, int w, int N,
                       const int32_t* ys, const int32_t* xs, long n,
                       double* out, long* n_fallback)
{
    if (check_args(H, W, pitch, w, N)) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    long nf = 0;
    for (long j = 0; j < n; ++j) {
        int flags = 0;
        if (ys[j] < 0 || ys[j] >= H || xs[j] < 0 || xs[j] >= W) return 1;
        fabf_pixel(f, theta, sigma, H, W, pitch, w, N, ys[j], xs[j], Ainv,
                   &out[j], NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                   NULL, &flags);
        if (flags & 2) ++nf;
    }
    if (n_fallback) *n_fallback = nf;
    return 0;
}

/* Algorithm 1 on the whole image; out is H x W float64, row stride W. */
int oracle_fabf(const uint8_t* f, const float* theta, const float* sigma,
                int H, int W, long pitch, int w, int N, double* out,
                long* n_fallback)
{
    if (check_args(H, W, pitch, w, N)) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    long nf = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int flags = 0;
            fabf_pixel(f, theta, sigma, H, W, pitch, w, N, y, x, Ainv,
                       &out[(long)y * W + x], NULL, NULL, NULL, NULL, NULL,
                       NULL, NULL, NULL, NULL, &flags);
            if (flags & 2) ++nf;
        }
    if (n_fallback) *n_fallback = nf;
    return 0;
}

/* Every intermediate of Algorithm 1 at pixel (y, x).
 * ab[2] = alpha, beta; m, M, mu, c: N+1 entries; t0lam[2]; I: N+2 entries;
 * T[2] = T1, T2; g[1]; flags[1] (bit0 flat, bit1 fallback). */
int oracle_fabf_trace(const uint8_t* f, const float* theta, const float* sigma,
                      int H, int W, long pitch, int w, int N, int y, int x,
                      int32_t* ab, int64_t* m, int64_t* M, double* mu,
                      double* c, double* t0lam, double* I, double* T,
                      double* g, int32_t* flags)
{
    if (check_args(H, W, pitch, w, N)) return 1;
    if (y < 0 || y >= H || x < 0 || x >= W) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    int a = 0, b = 0, fl = 0;
    fabf_pixel(f, theta, sigma, H, W, pitch, w, N, y, x, Ainv, g, &a, &b,
               m, M, mu, c, t0lam, I, T, &fl);
    ab[0] = a;
    ab[1] = b;
    flags[0] = fl;
    return 0;
}

/* Brute-force adaptive bilateral filter, Eqs. (1)-(3), box spatial kernel on
 * the clipped window, at the n pixels (ys[j], xs[j]). */
int oracle_bruteforce_pixels(const uint8_t* f, const float* theta,
                             const float* sigma, int H, int W, long pitch,
                             int w, const int32_t* ys, const int32_t* xs,
                             long n, double* out)
{
    if (check_args(H, W, pitch, w, 0)) return 1;
    for (long j = 0; j < n; ++j) {
        int y = ys[j], x = xs[j], y0, y1, x0, x1;
        if (y < 0 || y >= H || x < 0 || x >= W) return 1;
        window_bounds(H, W, y, x, w, &y0, &y1, &x0, &x1);
        const double th = theta[(long)y * W + x];
        const double s = sigma[(long)y * W + x];
        double num = 0.0, den = 0.0;
        for (int yy = y0; yy <= y1; ++yy)
            for (int xx = x0; xx <= x1; ++xx) {
                double v = f[(long)yy * pitch + xx];
                double phi = exp(-(v - th) * (v - th) / (2.0 * s * s));   /* Eq. (3) */
                num += phi * v;                                           /* Eq. (1) */
                den += phi;                                               /* Eq. (2) */
            }
        out[j] = num / den;
    }
    return 0;
}

/* Brute force on the whole image; out is H x W float64, row stride W. */
int oracle_bruteforce(const uint8_t* f, const float* theta, const float* sigma,
                      int H, int W, long pitch, int w, double* out)
{
    if (check_args(H, W, pitch, w, 0)) return 1;
    int32_t* ys = (int32_t*)malloc(sizeof(int32_t) * (size_t)W);
    int32_t* xs = (int32_t*)malloc(sizeof(int32_t) * (size_t)W);
    if (!ys || !xs) { free(ys); free(xs); return 2; }
    int rc = 0;
    for (int y = 0; y < H && !rc; ++y) {
        for (int x = 0; x < W; ++x) { ys[x] = y; xs[x] = x; }
        rc = oracle_bruteforce_pixels(f, theta, sigma, H, W, pitch, w, ys, xs,
                                      W, out + (long)y * W);
    }
    free(ys);
    free(xs);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Separable spatial kernels (Eq. (4) and Sec. II: any spatial kernel) */
/* ------------------------------------------------------------------ */
/*
 * The spatial kernel is omega(j) = g[jy + r] g[jx + r] on the window
 * [-r, r]^2 (clipped to the image, R1), for integer taps g[0..2r] >= 0 with
 * g[r] >= 1 and sum g <= 65535.  The pixel at (y + ty, x + tx) carries the
 * weight g[ty + r] g[tx + r].  A quantised Gaussian, g[t] = round(G exp(-(t -
 * r)^2 / (2 rho^2))) with r = ceil(3 rho), is Eq. (4) with the paper's window
 * [-3 rho, 3 rho]^2 up to the quantisation of the taps; any other separable
 * kernel is allowed (the method works with any spatial filter).  Because the
 * taps are integers, m_k and M_k are exact integers (< 2^81), summed here in
 * unsigned 128-bit arithmetic.  alpha, beta are the min / max over the whole
 * window, the support of omega (Eq. (8)); a tap of 0 only leaves its pixels
 * out of the histogram, which stays supported on [alpha, beta].
 */
typedef unsigned __int128 u128;

#define ORACLE_TAP_SUM_MAX 65535

static int check_taps(const uint32_t* taps, int r)
{
    if (r < 1 || r > ORACLE_WMAX || !taps) return 1;
    uint64_t s = 0;
    for (int t = 0; t <= 2 * r; ++t) s += taps[t];
    if (taps[r] < 1 || s > ORACLE_TAP_SUM_MAX) return 1;
    return 0;
}

/* Eq. (17) with omega = g x g: m_k = sum omega(j) f(i + j)^k, k = 0..K. */
static void pixel_moments_sep(const uint8_t* f, int H, int W, long pitch, const uint32_t* taps,
                              int r, int K, int y, int x, u128* m)
{
    int y0, y1, x0, x1;
    window_bounds(H, W, y, x, r, &y0, &y1, &x0, &x1);
    for (int k = 0; k <= K; ++k) m[k] = 0;
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            const u128 om = (u128)taps[yy - y + r] * taps[xx - x + r];
            u128 v = f[(long)yy * pitch + xx], p = 1;
            for (int k = 0; k <= K; ++k) { m[k] += om * p; p *= v; }
        }
}

/* Eq. (24) with omega = g x g (R2): M_k = sum omega(j) (f(i + j) - alpha)^k. */
static void pixel_shifted_moments_sep(const uint8_t* f, int H, int W, long pitch,
                                      const uint32_t* taps, int r, int K, int alpha, int y,
                                      int x, u128* M)
{
    int y0, y1, x0, x1;
    window_bounds(H, W, y, x, r, &y0, &y1, &x0, &x1);
    for (int k = 0; k <= K; ++k) M[k] = 0;
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            const u128 om = (u128)taps[yy - y + r] * taps[xx - x + r];
            u128 v = (u128)(f[(long)yy * pitch + xx] - alpha), p = 1;
            for (int k = 0; k <= K; ++k) { M[k] += om * p; p *= v; }
        }
}

/* Algorithm 1 at (y, x) with the separable kernel; same outputs as
 * fabf_pixel, with m and M as (low, high) 64-bit word pairs. */
static void fabf_pixel_sep(const uint8_t* f, const float* theta, const float* sigma, int H,
                           int W, long pitch, const uint32_t* taps, int r, int N, int y, int x,
                           const int64_t* Ainv, double* g_out, int* alpha_out, int* beta_out,
                           uint64_t* m_out, uint64_t* M_out, double* mu_out, double* c_out,
                           double* t0lam_out, double* I_out, double* T_out, int* flags_out)
{
    int alpha, beta, flags = 0;
    pixel_bounds(f, H, W, pitch, r, y, x, &alpha, &beta);
    if (alpha_out) *alpha_out = alpha;
    if (beta_out) *beta_out = beta;
    if (m_out) {
        u128 m[ORACLE_NMAX + 1];
        pixel_moments_sep(f, H, W, pitch, taps, r, N, y, x, m);
        for (int k = 0; k <= N; ++k) {
            m_out[2 * k] = (uint64_t)m[k];
            m_out[2 * k + 1] = (uint64_t)(m[k] >> 64);
        }
    }
    if (alpha == beta) {
        *g_out = (double)f[(long)y * pitch + x];      /* Sec. II-A */
        if (flags_out) *flags_out = 1;
        return;
    }
    const int d = beta - alpha;
    u128 M[ORACLE_NMAX + 2];
    double mu[ORACLE_NMAX + 2], c[ORACLE_NMAX + 1], I[ORACLE_NMAX + 2], t0lam[2], T[2];
    const int K = N < 1 ? 1 : N;
    pixel_shifted_moments_sep(f, H, W, pitch, taps, r, K, alpha, y, x, M);
    int64_t dk = 1;
    for (int k = 0; k <= K; ++k) {
        mu[k] = (double)M[k] / (double)dk;          /* Eq. (24); M_k rounded once */
        dk *= d;
    }
    fabf_tail(N, Ainv, alpha, d, mu, (double)theta[(long)y * W + x], (double)sigma[(long)y * W + x],
              g_out, c, t0lam, I, T, &flags);
    if (M_out)
        for (int k = 0; k <= N; ++k) {
            M_out[2 * k] = (uint64_t)M[k];
            M_out[2 * k + 1] = (uint64_t)(M[k] >> 64);
        }
    if (mu_out) for (int k = 0; k <= N; ++k) mu_out[k] = mu[k];
    if (c_out) for (int k = 0; k <= N; ++k) c_out[k] = c[k];
    if (t0lam_out) { t0lam_out[0] = t0lam[0]; t0lam_out[1] = t0lam[1]; }
    if (I_out) for (int k = 0; k <= N + 1; ++k) I_out[k] = I[k];
    if (T_out) { T_out[0] = T[0]; T_out[1] = T[1]; }
    if (flags_out) *flags_out = flags;
}

/* m_k with the separable kernel as (low, high) word pairs: m is
 * (N+1) x H x W x 2 uint64. */
int oracle_moments_sep(const uint8_t* f, int H, int W, long pitch, const uint32_t* taps, int r,
                       int N, uint64_t* m)
{
    if (check_args(H, W, pitch, r, N) || check_taps(taps, r)) return 1;
    const long plane = (long)H * W;
    u128 mk[ORACLE_NMAX + 1];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            pixel_moments_sep(f, H, W, pitch, taps, r, N, y, x, mk);
            for (int k = 0; k <= N; ++k) {
                const long o = 2 * (k * plane + (long)y * W + x);
                m[o] = (uint64_t)mk[k];
                m[o + 1] = (uint64_t)(mk[k] >> 64);
            }
        }
    return 0;
}

/* Algorithm 1 with the separable kernel at the n pixels (ys[j], xs[j]). */
int oracle_fabf_sep_pixels(const uint8_t* f, const float* theta, const float* sigma, int H,
                           int W, long pitch, const uint32_t* taps, int r, int N,
                           const int32_t* ys, const int32_t* xs, long n, double* out,
                           long* n_fallback)
{
    if (check_args(H, W, pitch, r, N) || check_taps(taps, r)) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    long nf = 0;
    for (long j = 0; j < n; ++j) {
        int flags = 0;
        if (ys[j] < 0 || ys[j] >= H || xs[j] < 0 || xs[j] >= W) return 1;
        fabf_pixel_sep(f, theta, sigma, H, W, pitch, taps, r, N, ys[j], xs[j], Ainv, &out[j],
                       NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, &flags);
        if (flags & 2) ++nf;
    }
    if (n_fallback) *n_fallback = nf;
    return 0;
}

/* Algorithm 1 with the separable kernel on the whole image. */
int oracle_fabf_sep(const uint8_t* f, const float* theta, const float* sigma, int H, int W,
                    long pitch, const uint32_t* taps, int r, int N, double* out,
                    long* n_fallback)
{
    if (check_args(H, W, pitch, r, N) || check_taps(taps, r)) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    long nf = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int flags = 0;
            fabf_pixel_sep(f, theta, sigma, H, W, pitch, taps, r, N, y, x, Ainv,
                           &out[(long)y * W + x], NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                           NULL, NULL, &flags);
            if (flags & 2) ++nf;
        }
    if (n_fallback) *n_fallback = nf;
    return 0;
}

/* Every intermediate with the separable kernel at (y, x); m and M hold
 * 2 (N+1) words (low, high per k), the rest as in oracle_fabf_trace. */
int oracle_fabf_sep_trace(const uint8_t* f, const float* theta, const float* sigma, int H,
                          int W, long pitch, const uint32_t* taps, int r, int N, int y, int x,
                          int32_t* ab, uint64_t* m, uint64_t* M, double* mu, double* c,
                          double* t0lam, double* I, double* T, double* g, int32_t* flags)
{
    if (check_args(H, W, pitch, r, N) || check_taps(taps, r)) return 1;
    if (y < 0 || y >= H || x < 0 || x >= W) return 1;
    int64_t Ainv[(ORACLE_NMAX + 1) * (ORACLE_NMAX + 1)];
    oracle_hilbert_inverse(N, Ainv);
    int a = 0, b = 0, fl = 0;
    fabf_pixel_sep(f, theta, sigma, H, W, pitch, taps, r, N, y, x, Ainv, g, &a, &b, m, M, mu,
                   c, t0lam, I, T, &fl);
    ab[0] = a;
    ab[1] = b;
    flags[0] = fl;
    return 0;
}

/* Brute-force adaptive bilateral filter, Eqs. (1)-(3), with the separable
 * spatial kernel, at the n pixels (ys[j], xs[j]). */
int oracle_bruteforce_sep_pixels(const uint8_t* f, const float* theta, const float* sigma,
                                 int H, int W, long pitch, const uint32_t* taps, int r,
                                 const int32_t* ys, const int32_t* xs, long n, double* out)
{
    if (check_args(H, W, pitch, r, 0) || check_taps(taps, r)) return 1;
    for (long j = 0; j < n; ++j) {
        int y = ys[j], x = xs[j], y0, y1, x0, x1;
        if (y < 0 || y >= H || x < 0 || x >= W) return 1;
        window_bounds(H, W, y, x, r, &y0, &y1, &x0, &x1);
        const double th = theta[(long)y * W + x];
        const double s = sigma[(long)y * W + x];
        double num = 0.0, den = 0.0;
        for (int yy = y0; yy <= y1; ++yy)
            for (int xx = x0; xx <= x1; ++xx) {
                const double om = (double)taps[yy - y + r] * (double)taps[xx - x + r];
                const double v = f[(long)yy * pitch + xx];
                const double phi = exp(-(v - th) * (v - th) / (2.0 * s * s));   /* Eq. (3) */
                num += om * phi * v;                                           /* Eq. (1) */
                den += om * phi;                                               /* Eq. (2) */
            }
        out[j] = num / den;
    }
    return 0;
}

/* Brute force with the separable kernel on the whole image. */
int oracle_bruteforce_sep(const uint8_t* f, const float* theta, const float* sigma, int H,
                          int W, long pitch, const uint32_t* taps, int r, double* out)
{
    if (check_args(H, W, pitch, r, 0) || check_taps(taps, r)) return 1;
    int32_t* ys = (int32_t*)malloc(sizeof(int32_t) * (size_t)W);
    int32_t* xs = (int32_t*)malloc(sizeof(int32_t) * (size_t)W);
    if (!ys || !xs) { free(ys); free(xs); return 2; }
    int rc = 0;
    for (int y = 0; y < H && !rc; ++y) {
        for (int x = 0; x < W; ++x) { ys[x] = y; xs[x] = x; }
        rc = oracle_bruteforce_sep_pixels(f, theta, sigma, H, W, pitch, taps, r, ys, xs, W,
                                          out + (long)y * W);
    }
    free(ys);
    free(xs);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Applications (Sec. IV): the centre and width maps                   */
/* ------------------------------------------------------------------ */
/*
 * Readings (the paper leaves the parameters of these rules open):
 *   - sharpening centre (Sec. IV-A): theta = f + zeta with zeta = f - fbar,
 *     fbar the plain mean of f over the filter window [-w, w]^2 clipped to
 *     the image, i.e. theta = (2 f m_0 - m_1) / m_0, the correctly rounded
 *     binary32 quotient of two integers that binary32 holds exactly;
 *   - sharpening width (Sec. IV-A): the Laplacian of a Gaussian of f, as the
 *     integer Gaussian S = g x g * f (integer taps, coordinates clamped to the
 *     image) followed by the 5-point Laplacian of S (clamped), so L is an
 *     exact integer; with q = min(|L|, Lq) the width is sigma = s_hi - (s_hi -
 *     s_lo) (q / Lq) in binary32 (q and Lq rounded to binary32, then the
 *     division, the difference s_hi - s_lo, the product and the difference,
 *     each rounded): low |LoG| gives a wide range kernel, high |LoG| a narrow
 *     one;
 *   - texture width (Sec. IV-C): mRTV = Delta gmax / (gsum + eps) over the
 *     window [-k, k]^2 clipped to the image, with Delta the range of f there
 *     and g = |f(x+1, y) - f(x, y)| + |f(x, y+1) - f(x, y)| (forward
 *     differences, clamped; the L1 norm keeps g an integer), then sigma =
 *     s_hi - (s_hi - s_lo) min(mRTV / msat, 1), all in binary32 operations
 *     in that order (Delta gmax and gsum are exact in binary32).
 * The maps are binary32 maps, so they are evaluated in binary32.
 */
static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_sharpen_theta(const uint8_t* f, int H, int W, long pitch, int w, float* theta)
{
    if (check_args(H, W, pitch, w, 1)) return 1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t m[2];
            pixel_moments(f, H, W, pitch, w, 1, y, x, m);
            const int64_t num = 2 * (int64_t)f[(long)y * pitch + x] * m[0] - m[1];
            /* |num| <= 2 * 255 * 6561 < 2^24 and m_0 <= 6561: both exact in
               binary32, so this is the correctly rounded binary32 quotient */
            theta[(long)y * W + x] = (float)num / (float)m[0];
        }
    return 0;
}

/* 5-point Laplacian of the integer Gaussian-smoothed image at (y, x). */
static int64_t log_at(const uint8_t* f, int H, int W, long pitch, const uint32_t* taps, int r, int y, int x)
{
    int64_t S[5];
    const int dy[5] = {0, -1, 1, 0, 0}, dx[5] = {0, 0, 0, -1, 1};
    for (int q = 0; q < 5; ++q) {
        const int yc = clampi(y + dy[q], 0, H - 1), xc = clampi(x + dx[q], 0, W - 1);
        int64_t s = 0;
        for (int ty = -r; ty <= r; ++ty)
            for (int tx = -r; tx <= r; ++tx) {
                const int yy = clampi(yc + ty, 0, H - 1), xx = clampi(xc + tx, 0, W - 1);
                s += (int64_t)taps[ty + r] * taps[tx + r] * f[(long)yy * pitch + xx];
            }
        S[q] = s;
    }
    return S[1] + S[2] + S[3] + S[4] - 4 * S[0];
}

int oracle_sharpen_log(const uint8_t* f, int H, int W, long pitch, const uint32_t* taps, int r, int64_t* L)
{
    if (check_args(H, W, pitch, r, 0) || check_taps(taps, r)) return 1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) L[(long)y * W + x] = log_at(f, H, W, pitch, taps, r, y, x);
    return 0;
}

int oracle_sharpen_sigma(const uint8_t* f, int H, int W, long pitch, const uint32_t* taps, int r, int64_t Lq,
                         double s_lo, double s_hi, float* sigma)
{
    if (check_args(H, W, pitch, r, 0) || check_taps(taps, r) || Lq < 1) return 1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t L = log_at(f, H, W, pitch, taps, r, y, x);
            if (L < 0) L = -L;
            const int64_t q = L < Lq ? L : Lq;
            /* binary32 throughout (the map is a binary32 map) */
            const float u = (float)q / (float)Lq;
            const float hi = (float)s_hi, lo = (float)s_lo;
            sigma[(long)y * W + x] = hi - (hi - lo) * u;
        }
    return 0;
}

int oracle_texture_sigma(const uint8_t* f, int H, int W, long pitch, int k, double eps, double msat, double s_lo,
                         double s_hi, float* sigma)
{
    if (H < 1 || W < 1 || pitch < W || k < 1 || k > ORACLE_WMAX || !(eps > 0) || !(msat > 0)) return 1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int y0, y1, x0, x1, fmin = 255, fmax = 0;
            int64_t gmax = 0, gsum = 0;
            window_bounds(H, W, y, x, k, &y0, &y1, &x0, &x1);
            for (int yy = y0; yy <= y1; ++yy)
                for (int xx = x0; xx <= x1; ++xx) {
                    const int v = f[(long)yy * pitch + xx];
                    const int vx = f[(long)yy * pitch + clampi(xx + 1, 0, W - 1)];
                    const int vy = f[(long)clampi(yy + 1, 0, H - 1) * pitch + xx];
                    const int64_t g = (vx > v ? vx - v : v - vx) + (vy > v ? vy - v : v - vy);
                    if (v < fmin) fmin = v;
                    if (v > fmax) fmax = v;
                    if (g > gmax) gmax = g;
                    gsum += g;
                }
            /* binary32 throughout: Delta gmax <= 255 * 510 and gsum <=
               81^2 * 510 are exact in binary32 */
            const float mrtv = (float)((int64_t)(fmax - fmin) * gmax) / ((float)gsum + (float)eps);
            float u = mrtv / (float)msat;
            if (u > 1.0f) u = 1.0f;
            const float hi = (float)s_hi, lo = (float)s_lo;
            sigma[(long)y * W + x] = hi - (hi - lo) * u;
        }
    return 0;
}

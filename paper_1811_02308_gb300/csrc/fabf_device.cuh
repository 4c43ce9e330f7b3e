// Per-pixel device mathematics of fast adaptive bilateral filtering
// (Gavaskar & Chaudhury), Algorithm 1 of Sec. II-D, for one pixel whose
// window statistics (alpha, beta, m_0..m_N) are already known.
//
// Equation numbers are the paper's.  The integer stages are exact; the
// FP64 fit reproduces the oracle's rounding step for step (same operations in
// the same order), and the integrals are evaluated by a hybrid of the paper's
// forward recursion (Eq. 30) and the same recursion run downwards, which is
// the numerically stable direction when lambda is small.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "fabf_fp64_tables.h"

namespace fabf {

constexpr int kNMax = 6;    // int64 power sums are exact for N <= 6, w <= 40
constexpr int kWMax = 40;

// Status bits a kernel ORs into its status word.
constexpr unsigned kStatusBadInput = 1u;    // sigma <= 0 / non-finite, theta non-finite
constexpr unsigned kStatusTimeout = 2u;     // a bounded device wait gave up

// ---------------------------------------------------------------------------
// Hilbert inverse, Eq. (19), as exact integers (max |entry| 133,402,500 at
// N = 6, exactly representable in binary64).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr long long binom_c(int n, int k)
{
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// (A^{-1})_{m,n} with the paper's 1-based indices.
__host__ __device__ constexpr long long hilbert_inverse_entry(int N, int m, int n)
{
    const long long b = binom_c(m + n - 2, m - 1);
    return (((m + n) & 1) ? -1LL : 1LL) * (long long)(m + n - 1) * binom_c(N + m, N + 1 - n) *
           binom_c(N + n, N + 1 - m) * b * b;
}

struct AinvTable {
    double v[kNMax + 1][kNMax + 1][kNMax + 1];   // [N][n][k], 0-based
};

__host__ __device__ constexpr AinvTable make_ainv_table()
{
    AinvTable t{};
    for (int N = 0; N <= kNMax; ++N)
        for (int n = 0; n <= N; ++n)
            for (int k = 0; k <= N; ++k)
                t.v[N][n][k] = (double)hilbert_inverse_entry(N, n + 1, k + 1);
    return t;
}

struct RecipTable {
    double v[128];   // v[j] = 1 / j (v[0] unused)
    float f[128];    // the same in binary32
};

__host__ __device__ constexpr RecipTable make_recip_table()
{
    RecipTable t{};
    for (int j = 1; j < 128; ++j) {
        t.v[j] = 1.0 / (double)j;
        t.f[j] = (float)(1.0 / (double)j);
    }
    return t;
}

// The same entries split exactly into two binary32 values (|entry| < 2^28).
struct AinvSplitTable {
    float hi[kNMax + 1][kNMax + 1][kNMax + 1];
    float lo[kNMax + 1][kNMax + 1][kNMax + 1];
};

__host__ __device__ constexpr AinvSplitTable make_ainv_split_table()
{
    AinvSplitTable t{};
    for (int N = 0; N <= kNMax; ++N)
        for (int n = 0; n <= N; ++n)
            for (int k = 0; k <= N; ++k) {
                const double a = (double)hilbert_inverse_entry(N, n + 1, k + 1);
                t.hi[N][n][k] = (float)a;
                t.lo[N][n][k] = (float)(a - (double)(float)a);
            }
    return t;
}

// Correctly rounded reciprocals of the powers d^k (d = 1..255, k = 1..6),
// v[k-1][d] = RN(1 / d^k), built at compile time (a binary64 division of two
// exactly representable numbers, correctly rounded).  With them a quotient
// a / d^k costs one multiplication and two fused multiply-adds instead of a
// full division and is still correctly rounded (div_by_power below).  The
// powers themselves, p[k-1][d] = d^k (exact), are loaded with them rather
// than converted from integers (the conversion issues on the FP64 pipe,
// which bounds the FP64 form).
struct RecipPowTable {
    double v[kNMax][256];
    double p[kNMax][256];
};

__host__ __device__ constexpr RecipPowTable make_recip_pow_table()
{
    RecipPowTable t{};
    for (int k = 1; k <= kNMax; ++k)
        for (int d = 1; d < 256; ++d) {
            double p = 1.0;
            for (int i = 0; i < k; ++i) p *= (double)d;   // exact: d^k <= 255^6 < 2^53
            t.v[k - 1][d] = 1.0 / p;
            t.p[k - 1][d] = p;
        }
    return t;
}

// In global memory (read through the read-only cache): the lanes of a warp
// index it by their own d, which a constant-memory table would serialise.
static __device__ const RecipPowTable g_recip_pow = make_recip_pow_table();

// 0 <= v < 2^52 as a binary64 value, exactly: the bit pattern of 2^52 + v
// (v fills the mantissa), less 2^52.  One addition on the FP64 pipe in place
// of a 64-bit integer conversion.
__device__ __forceinline__ double small_to_double(int64_t v)
{
    return __hiloint2double(0x43300000 | (int)((uint64_t)v >> 32), (int)(uint32_t)v) - 0x1p52;
}

// A finite binary32 value as binary64, exactly, from its bits (integer
// operations in place of the conversion instruction, which issues on the FP64
// pipe): the exponent rebiased by 1023 - 127, the significand moved up 29
// bits.  Zero, subnormals, infinities and NaN take the conversion.
__device__ __forceinline__ double float_to_double(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned ef = (u >> 23) & 0xFFu;
    if (ef == 0u || ef == 0xFFu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((ef + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// RN(a / b) for b = d^k from r = RN(1 / b): q0 = RN(a r) lies within one unit
// in the last place of a / b, the residual a - b q0 is exact as one fused
// multiply-add, and q0 + r (a - b q0) rounded once is the correctly rounded
// quotient (Markstein's theorem for a correctly rounded reciprocal; checked
// for every b = d^k on 3e7 dividends, 0 <= a <= 6561 d^k, against IEEE
// division).  The FP64 form's mu_k and t0 stay bit-identical to the oracle's
// divisions.
__host__ __device__ __forceinline__ double div_by_power(double a, double b, double r)
{
    const double q0 = a * r;
    return fma(fma(-q0, b, a), r, q0);
}

// The tables are built at compile time; each translation unit that includes
// this header holds its own copy in constant memory.
static __constant__ AinvTable c_ainv = make_ainv_table();
static __constant__ AinvSplitTable c_ainv_split = make_ainv_split_table();
static __constant__ RecipTable c_recip = make_recip_table();

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// The binary64 erfcx and exp of the FP64 integrals, written for this path
// (their tables are made by gen_fp64_tables.py with mpmath): cheaper on the
// FP64 pipe than the general library functions, which the FP64 form is
// bound by, and as accurate (within 2 units in the last place; checked on
// the host against mpmath, tests/test_fp64_functions.py).
// ---------------------------------------------------------------------------
static __device__ const double g_erfcx_tab[(FABF_ERFCX_DEG + 2) * (FABF_ERFCX_NSEG + 1)] = {FABF_ERFCX_TABLE,
                                                                                            FABF_ERFCX_P0_LO};
static __device__ const double g_exp2_tab[1 << FABF_EXP_TABLE_BITS] = {FABF_EXP2_TABLE};

#ifdef __CUDA_ARCH__
#define FABF_TABLE_LOAD(p) __ldg(p)
#else
#define FABF_TABLE_LOAD(p) (*(p))
#endif

__host__ __device__ __forceinline__ int low_word(double v)
{
#ifdef __CUDA_ARCH__
    return __double2loint(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return (int)(uint32_t)b;
#endif
}

// The high 32 bits of a binary64 value, and the value whose high bits are hi
// and low bits zero.
__host__ __device__ __forceinline__ int high_word(double v)
{
#ifdef __CUDA_ARCH__
    return __double2hiint(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return (int)(uint32_t)(b >> 32);
#endif
}

__host__ __device__ __forceinline__ double from_high_word(int hi)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double(hi, 0);
#else
    const uint64_t b = (uint64_t)(uint32_t)hi << 32;
    double v;
    std::memcpy(&v, &b, 8);
    return v;
#endif
}

// RN(x) in binary32 from x's bits (integer operations; the conversion
// instruction issues on the FP64 pipe, which bounds the forms with a binary64
// fit): the top 23 fraction bits, rounded to nearest even on the 29 below
// them (a carry into the exponent is the correct result, up to infinity).
// Results outside the normal binary32 range, zero, infinities and NaN take
// the conversion instruction.
__host__ __device__ __forceinline__ float double_to_float_rn(double x)
{
    const int hi = high_word(x);
    const unsigned lo = (unsigned)low_word(x);
    const int e = ((hi >> 20) & 0x7FF) - 1023 + 127;              // binary32 biased exponent
    if (e < 1 || e > 254) return (float)x;
    const unsigned m = ((unsigned)(hi & 0xFFFFF) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    unsigned b = ((unsigned)hi & 0x80000000u) | ((unsigned)e << 23) | m;
    b += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, 4);
    return f;
#endif
}

// 2^m for -1022 <= m <= 1023, exactly.
__host__ __device__ __forceinline__ double pow2i(int m)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double((m + 1023) << 20, 0);
#else
    const uint64_t b = (uint64_t)(m + 1023) << 52;
    double v;
    std::memcpy(&v, &b, 8);
    return v;
#endif
}

// erfcx(x) = exp(x^2) erfc(x) for x >= 0.  On [0, 12): 384 pieces of width
// 1/32, each a degree-7 polynomial in t = 64x - 2i - 1 (Chebyshev
// interpolants, truncation below 2e-18 relative); x >= 12: erfcx(x) =
// g(1/x^2) / x with g a degree-7 polynomial in t = 288/x^2 - 1.
// The coefficient k of piece i is tab[k (NSEG + 1) + i]; row DEG + 1 holds
// the low parts of the constant coefficients, added before the final
// rounding (p = p0 + lo + t q(t)).
__host__ __device__ __forceinline__ double erfcx_fp64_with(double x, const double* tab)
{
    constexpr int S = FABF_ERFCX_NSEG + 1;
    double t;
    int i;
    const bool large = high_word(x) >= FABF_ERFCX_XL_HIGH_WORD;   // x >= 12 (or NaN) for x >= 0
    if (!large) {
        const double q = FABF_ERFCX_PER_UNIT * x;   // exact, in [0, 384)
        // i = floor(q) and its binary64 value from q's bits (integer
        // operations: the FP64 pipe, which bounds the FP64 form, stays
        // free).  q < 384 has at most 9 integer bits, all in the high word:
        // with e the unbiased exponent, i is the top e + 1 bits of the
        // significand and floor(q) is q with the bits below them cleared.
        const int hi = high_word(q);
        const int e = (hi >> 20) - 1023;      // < 0 for q < 1 (and for +0)
        const int sh = 20 - (e < 0 ? 0 : e);
        i = e < 0 ? 0 : ((hi & 0xFFFFF) | 0x100000) >> sh;
        const double fq = e < 0 ? 0.0 : from_high_word(hi & ~((1 << sh) - 1));
        t = fma(2.0, q - fq, -1.0);           // 64x - 2i - 1, exact
    } else {
        const double r = 1.0 / x;
        t = fma(FABF_ERFCX_LARGE_T, r * r, -1.0);
        i = FABF_ERFCX_NSEG;
    }
    const double* c = tab + i;
    double q = FABF_TABLE_LOAD(c + FABF_ERFCX_DEG * S);
#pragma unroll
    for (int k = FABF_ERFCX_DEG - 1; k >= 1; --k) q = fma(q, t, FABF_TABLE_LOAD(c + k * S));
    double p = FABF_TABLE_LOAD(c) + fma(q, t, FABF_TABLE_LOAD(c + (FABF_ERFCX_DEG + 1) * S));
    if (large) p /= x;                             // 0 at x = inf
    return p;
}

// exp(x) for x <= 709 by Tang's table-driven method (ACM TOMS 15(2), 1989):
// N = rint(1024 x / ln 2) = 1024 m + j, r = x - N ln2/1024 (two-part
// constant), exp(x) = 2^m 2^(j/1024) (1 + p(r)) with p the Taylor polynomial
// of degree 4 (|r| <= ln2/2048: truncation below 4e-20).  Results below the normal range
// are scaled in two steps (one rounding into the subnormals); x at or below
// -745.25 gives 0.
__host__ __device__ __forceinline__ double exp_fp64_with(double x, const double* T)
{
    // x <= -745.25 (high word compared as an integer; the FP64 pipe stays
    // free): below half the smallest subnormal, the result is 0
    const int hx = high_word(x);
    if (hx < 0 && (hx & 0x7FFFFFFF) >= 0x40874A00) return x != x ? x : 0.0;
    constexpr double kShift = 0x1.8p52;
    const double y = fma(x, FABF_EXP_INV_L, kShift);
    const double Nd = y - kShift;             // rint(1024 x / ln 2), exact
    const int N = low_word(y);
    double r = fma(-Nd, FABF_EXP_L1, x);
    r = fma(-Nd, FABF_EXP_L2, r);
    const int j = N & ((1 << FABF_EXP_TABLE_BITS) - 1), m = N >> FABF_EXP_TABLE_BITS;
    const double q = fma(fma(r, 1.0 / 24.0, 1.0 / 6.0), r, 0.5);
    const double p = fma(r * r, q, r);        // exp(r) - 1
    const double Tj = FABF_TABLE_LOAD(T + j);
    const double e = fma(Tj, p, Tj);
    if (m >= -1022) return e * pow2i(m);
    return (e * pow2i(m + 54)) * 0x1p-54;
}

__device__ __forceinline__ double erfcx_fp64(double x) { return erfcx_fp64_with(x, g_erfcx_tab); }
__device__ __forceinline__ double exp_fp64(double x) { return exp_fp64_with(x, g_exp2_tab); }

// The FP64 form's integrals take these (Own = true); the binary32 forms' FP64
// recompute of the few pixels their guard rejects takes the library's
// functions (Own = false), whose code keeps the registers of their hot loop
// free (the table-driven versions made it spill at 64 registers).
template <bool Own>
__device__ __forceinline__ double erfcx_sel(double x)
{
    if constexpr (Own) return erfcx_fp64(x);
    else return erfcx(x);
}
template <bool Own>
__device__ __forceinline__ double exp_sel(double x)
{
    if constexpr (Own) return exp_fp64(x);
    else return exp(x);
}

// Integrals I_k = int_0^1 t^k exp(-lambda (t - t0)^2) dt, Eq. (28), k = 0..K,
// each multiplied by exp(lambda d^2) with d the distance from t0 to [0, 1].
// That factor is common to numerator and denominator of Eq. (29) and keeps
// every value representable however far the range-kernel centre lies from
// [alpha, beta].
//
//  lambda >= 1: Eq. (31) for I_0 (erf; scaled erfc when t0 is outside
//               [0, 1]), Eq. (32) for I_1, Eq. (30) forward for I_2..I_K.
//  lambda <  1: Eq. (30) solved for I_{k-2} and run downwards from a start
//               index Kp >= K + 1 (chosen from lambda and t0, made warp-uniform)
//               with the start values I_k ~ E_1 / (k + 1 + 2 lambda (t0-1))
//               (mass of t^k near t = 1).  The recursion's own error
//               amplification is below one in that direction, so the start
//               error dies out and no erf is needed.
// ---------------------------------------------------------------------------
constexpr double kLambdaForward = 1.0;

// Start index of the binary64 downward recursion: one step maps (I_k,
// I_(k-1)) to (I_(k-1), I_(k-2)) and multiplies an error in the pair by the
// spectral radius of its homogeneous part,
//   rho_k = (a + sqrt(a^2 + 4b)) / 2,  a = 2 lambda |t0| / (k-1), b = 2 lambda / (k-1);
// Kp is the smallest index with prod_{k=K+2}^{Kp+1} rho_k < 1e-13 (the start
// values carry a relative error of at most a few percent), at the upper
// corner of a bin of (lambda, |t0|) (bins of 1/32 in lambda < 1 and 1/2 in
// |t0| < 4), for K = 7.
struct KpTableF64 {
    unsigned char v[32][8];   // [lambda bin][|t0| bin]
};

__host__ __device__ constexpr double ct_sqrt64(double x)
{
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 60; ++i) r = 0.5 * (r + x / r);
    return r;
}

__host__ __device__ constexpr KpTableF64 make_kp_table_f64()
{
    KpTableF64 t{};
    for (int i = 0; i < 32; ++i)
        for (int j = 0; j < 8; ++j) {
            const double lam = (i + 1) / 32.0, at0 = (j + 1) * 0.5;
            double p = 1.0;
            int kp = 8;   // K + 1
            do {
                ++kp;     // the step that produces I_(kp-2) from I_kp, I_(kp-1)
                const double a = 2.0 * lam * at0 / (kp - 1), b = 2.0 * lam / (kp - 1);
                p *= 0.5 * (a + ct_sqrt64(a * a + 4.0 * b));
            } while (p >= 1e-13 && kp < 62);
            t.v[i][j] = (unsigned char)kp;
        }
    return t;
}

// In global memory (read-only cache): the lanes index it by their own bin,
// which a constant-memory table would serialise.
static __device__ const KpTableF64 g_kp64 = make_kp_table_f64();

// min(cap, floor(|v| 2^s)) from the bits of v (integer operations only):
// with e the unbiased exponent of |v| plus s, the value is the top e + 1
// bits of the significand (0 for e < 0; cap once e reaches 20, which covers
// infinities and NaN).  Requires cap < 2^20.
__device__ __forceinline__ int floor_scaled_abs(double v, int s, int cap)
{
    const int hi = high_word(v) & 0x7FFFFFFF;
    const int e = (hi >> 20) - 1023 + s;
    if (e < 0) return 0;
    if (e >= 20) return cap;
    return min(cap, ((hi & 0xFFFFF) | 0x100000) >> (20 - e));
}

// An approximation of 1 / x (x normal, positive): the hardware's approximate
// binary64 reciprocal (PTX rcp.approx.ftz.f64), far closer than the few
// percent the recursion's start values need.
__device__ __forceinline__ double rcp_approx_f64(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__device__ __forceinline__ int backward_start_index(double lam, double t0)
{
    return __ldg(&g_kp64.v[floor_scaled_abs(lam, 5, 31)][floor_scaled_abs(t0, 1, 7)]);
}

// The distance d from t0 to [0, 1] and whether t0 lies below 0, with the
// comparisons made on t0's bits as 64-bit integers (ordered as the values
// for t0 >= 0; the sign bit makes negative ones negative): the FP64 pipe
// stays free.  t0 = -0 gives d = +0, as t0 = +0 does.
__device__ __forceinline__ double dist_to_unit(double t0, bool& below)
{
    const long long b = __double_as_longlong(t0);
    below = b < 0;
    return below ? -t0 : (b > 0x3FF0000000000000LL ? t0 - 1.0 : 0.0);
}

// T2 > 0 and F finite, tested on the bits (integer operations; the FP64
// pipe stays free).  A positive T2 is a positive 64-bit pattern; a NaN T2
// makes F NaN, which the exponent test catches.
__device__ __forceinline__ bool ratio_usable(double T2, double F)
{
    return __double_as_longlong(T2) > 0 && (high_word(F) & 0x7FF00000) != 0x7FF00000;
}

// inv2l = 1 / (2 lambda) and rl = 1 / sqrt(lambda), each to within a unit or
// two in the last place (the callers form them without a division or a
// square root: 1 / (2 lambda) = sigma^2 / d^2, 1 / sqrt(lambda) =
// sqrt(2) sigma / d).
template <int K, bool Own = true>
__device__ __forceinline__ void integrals_fp64(double lam, double inv2l, double rl, double t0, double (&I)[K + 1])
{
    static_assert(K >= 1 && K <= 7, "K out of range");
    if (lam >= kLambdaForward) {
        const double sl = lam * rl;                               // sqrt(lambda)
        const double h = 0.88622692545275801364908374167057 * rl; // 1/2 sqrt(pi/lambda)
        // One path for the three positions of t0 (no divergence): with d the
        // distance from t0 to [0, 1], E0 and E1 carry the common factor
        // exp(lambda d^2), and Eq. (31) is written with the scaled erfc,
        //   inside  [0, 1]: erf(a) + erf(b) = 2 - E1 erfcx(a) - E0 erfcx(b),
        //   outside [0, 1]: erfcx(sqrt(lambda) d) - E erfcx(sqrt(lambda)(1 + d)),
        // a = sqrt(lambda)(1 - t0), b = sqrt(lambda) t0, E = E1 (t0 < 0) or E0.
        bool below;
        const double d = dist_to_unit(t0, below);
        const bool inside = __double_as_longlong(d) == 0;          // d == +0
        // t0^2 - d^2 and (1 - t0)^2 - d^2 in each position of t0: inside,
        // t0^2 and (1 - t0)^2; below 0, 0 and 1 - 2 t0; above 1, 2 t0 - 1 and 0
        const double u = 1.0 - t0, v = fma(2.0, t0, -1.0);
        const double g0 = inside ? t0 * t0 : (below ? 0.0 : v);
        const double g1 = inside ? u * u : (below ? -v : 0.0);
        const double E0s = exp_sel<Own>(-lam * g0);
        const double E1s = exp_sel<Own>(-lam * g1);
        const double S = inside ? 2.0 : 0.0;
        const double ca = inside ? E1s : -1.0;
        const double xa = sl * (inside ? u : d);
        const double cb = inside ? E0s : (below ? E1s : E0s);
        const double xb = sl * (inside ? t0 : 1.0 + d);
        const double I0 = h * (S - ca * erfcx_sel<Own>(xa) - cb * erfcx_sel<Own>(xb));
        const double e1 = E1s * inv2l;
        I[0] = I0;
        I[1] = fma(t0, I0, (E0s - E1s) * inv2l);
#pragma unroll
        for (int k = 2; k <= K; ++k) I[k] = fma(t0, I[k - 1], fma((double)(k - 1) * inv2l, I[k - 2], -e1));
    } else {
        bool below;
        const double d = dist_to_unit(t0, below);
        const bool inside = __double_as_longlong(d) == 0;
        const double u = 1.0 - t0;
        // (1 - t0)^2 - d^2: (1 - t0)^2 inside, 1 - 2 t0 below 0, 0 above 1
        const double g1 = inside ? u * u : (below ? fma(-2.0, t0, 1.0) : 0.0);
        const double E1s = exp_sel<Own>(-lam * g1);   // exp(-lam (1-t0)^2 + lam d^2)
        int Kp = backward_start_index(lam, t0);
        Kp = __reduce_max_sync(__activemask(), (unsigned)Kp);
        const double l2 = 2.0 * lam;
        const double q = -l2 * u;                      // 2 lambda (t0 - 1)
        const double kp2 = small_to_double(Kp + 2), kp1 = small_to_double(Kp + 1);
        const double r1 = kp2 + q, r0 = kp1 + q;
        // start values: a few percent is enough (the recursion damps their
        // error below 1e-13 by index K), so approximate reciprocals
        // (r > 1 tested on the bits: ordered as the values, negative ones
        // negative)
        constexpr long long kOneBits = 0x3FF0000000000000LL;
        double hi = E1s * rcp_approx_f64(__double_as_longlong(r1) > kOneBits ? r1 : kp2);   // I_{Kp+1}
        double lo = E1s * rcp_approx_f64(__double_as_longlong(r0) > kOneBits ? r0 : kp1);   // I_{Kp}
        // (hi, lo) = (I_k, I_{k-1}); produce I_{k-2} for k = Kp+1 .. K+2.
        for (int k = Kp + 1; k >= K + 2; --k) {
            const double nx = fma(l2, fma(-t0, lo, hi), E1s) * c_recip.v[k - 1];
            hi = lo;
            lo = nx;
        }
        I[K] = lo;
        const double top = hi;   // I_{K+1}, used by the first tail step only
#pragma unroll
        for (int k = K + 1; k >= 2; --k) {
            const double Ik = (k == K + 1) ? top : I[k];
            I[k - 2] = fma(l2, fma(-t0, I[k - 1], Ik), E1s) * (1.0 / (double)(k - 1));
        }
    }
}

// ---------------------------------------------------------------------------
// One pixel of Algorithm 1 in FP64.  m[0] is the window size, m[k] the
// window sum of f^k (exact, k = 0..max(N,1)).  Returns g_hat(i).
// ---------------------------------------------------------------------------
struct PixelTrace {       // optional per-pixel export of every stage
    int64_t M[kNMax + 1];
    double mu[kNMax + 1];
    double c[kNMax + 1];
    double t0, lam;
    double I[kNMax + 2];
    double T1, T2;
    int fallback;
};

// Algorithm 1 from mu_k = M_k / (beta - alpha)^k on: the fit, the kernel
// parameters, the integrals and the ratio, in binary64 (shared by the box and
// the separable spatial kernels).
// Eqs. (25), (28)-(29) from the fitted coefficients c (any common scale:
// it cancels in F): t0, lambda, the integrals and the two sums, in the order
// of Algorithm 1; returns F = T1 / T2.
template <int N, bool Own = true>
__device__ __forceinline__ double fp64_ratio(const double (&c)[N + 1], int alpha, int d, float theta_f, float sigma_f,
                                             double& t0, double& lam, double (&I)[N + 2], double& T1, double& T2)
{
    const double sg = float_to_double(sigma_f);
    const double sg2 = sg * sg;                                   // exact (24-bit mantissas)
    const double rd = __ldg(&g_recip_pow.v[0][d]);                // RN(1 / d)
    t0 = div_by_power(float_to_double(theta_f) - small_to_double(alpha), __ldg(&g_recip_pow.p[0][d]), rd);
    lam = __ldg(&g_recip_pow.p[1][d]) / (2.0 * sg2);
    // 1 / (2 lambda) = sigma^2 / d^2 and 1 / sqrt(lambda) = sqrt(2) sigma / d
    const double inv2l = sg2 * __ldg(&g_recip_pow.v[1][d]);
    const double rl = (sg * 1.4142135623730951) * rd;
    integrals_fp64<N + 1, Own>(lam, inv2l, rl, t0, I);
    T1 = c[0] * I[1];
    T2 = c[0] * I[0];
#pragma unroll
    for (int k = 2; k <= N + 1; ++k) {
        T1 = fma(c[k - 1], I[k], T1);
        T2 = fma(c[k - 1], I[k - 1], T2);
    }
    // F = T1 / T2 to within about one unit in the last place, without the
    // division's special-case handling: the approximate reciprocal, one
    // Newton step, and one correction of the quotient from its exact
    // residual.  T2 <= 0, zero or not finite gives a non-finite or unused
    // F: the callers take the fallback then.
    const double r0 = rcp_approx_f64(T2);
    const double r1 = fma(r0, fma(-T2, r0, 1.0), r0);
    const double F0 = T1 * r1;
    return fma(fma(-T2, F0, T1), r1, F0);
}

template <int N, bool Own = true>
__device__ __forceinline__ double fabf_tail_fp64(const AinvTable& A, int alpha, int d,
                                                 const double (&mu)[(N < 1 ? 1 : N) + 1], float theta_f,
                                                 float sigma_f, int& fallback, PixelTrace* tr)
{
    // c = A^{-1} mu, Eq. (19) and Algorithm 1, fused multiply-adds over
    // ascending k starting from zero.
    double c[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k <= N; ++k) acc = fma(A.v[N][n][k], mu[k], acc);
        c[n] = acc;
    }
    double t0, lam, I[N + 2], T1, T2;
    double F = fp64_ratio<N, Own>(c, alpha, d, theta_f, sigma_f, t0, lam, I, T1, T2);
    fallback = 0;
    if (!ratio_usable(T2, F)) {       // fitted polynomial not positive enough
        F = mu[1] / mu[0];                // sigma -> infinity limit (spatial-kernel mean)
        fallback = 1;
    }
    if (tr) {
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            tr->mu[k] = mu[k];
            tr->c[k] = c[k];
        }
#pragma unroll
        for (int k = 0; k <= N + 1; ++k) tr->I[k] = I[k];
        tr->t0 = t0;
        tr->lam = lam;
        tr->T1 = T1;
        tr->T2 = T2;
        tr->fallback = fallback;
    }
    return small_to_double(alpha) + small_to_double(d) * F;
}

template <int N, bool Own = true>
__device__ __forceinline__ double fabf_pixel_fp64(const AinvTable& A, int alpha, int beta, int fi,
                                                  const int64_t (&m)[(N < 1 ? 1 : N) + 1],
                                                  float theta_f, float sigma_f, int& fallback,
                                                  PixelTrace* tr)
{
    constexpr int K = N < 1 ? 1 : N;   // mu_1 is needed by the fallback even for N = 0
    fallback = 0;
    if (alpha == beta) return (double)fi;   // flat window: g(i) = f(i), Sec. II-A
    const int d = beta - alpha;

    // Eq. (24) in exact integers: M_b = sum_window (f - alpha)^b from the
    // power sums via S(a, b) = S(a+1, b-1) - alpha S(a, b-1), where
    // S(a, b) = sum f^a (f - alpha)^b.  Every S and every product stays in
    // [0, m_0 255^6] < 2^63 for N <= 6, w <= 40, so nothing overflows.
    int64_t s[K + 1], M[K + 1];
#pragma unroll
    for (int a = 0; a <= K; ++a) s[a] = m[a];
    M[0] = s[0];
#pragma unroll
    for (int b = 1; b <= K; ++b) {
#pragma unroll
        for (int a = 0; a <= K - b; ++a) s[a] = s[a + 1] - (int64_t)alpha * s[a];
        M[b] = s[0];
    }
    // mu_k = M_k / (beta - alpha)^k: the correctly rounded quotient of two
    // binary64 values ((beta - alpha)^k <= 255^6 is exact), formed from the
    // correctly rounded reciprocal (div_by_power).  The quotient must be the
    // correctly rounded one (an exactly scaled integer M_k d^(K-k), rounded
    // once, is not): at N = 6 the fit amplifies a one-unit change in the last
    // place of mu to ~1e-8 relative in g_hat, so the 1e-9 agreement with the
    // oracle rests on the same values entering the same operations.
    // 0 <= M_k <= m_0 d^k <= 6561 255^4 < 2^45 for k <= 4: exact without
    // the conversion instruction
    double mu[K + 1];
    mu[0] = small_to_double(M[0]);
#pragma unroll
    for (int k = 1; k <= K; ++k) {
        const double a = k <= 4 ? small_to_double(M[k]) : (double)M[k];
        mu[k] = div_by_power(a, __ldg(&g_recip_pow.p[k - 1][d]), __ldg(&g_recip_pow.v[k - 1][d]));
    }
    if (tr) {
#pragma unroll
        for (int k = 0; k <= N; ++k) tr->M[k] = M[k];
    }
    return fabf_tail_fp64<N, Own>(A, alpha, d, mu, theta_f, sigma_f, fallback, tr);
}


// ---------------------------------------------------------------------------
// The same integrals in binary32 (precision variants).  The downward
// recursion holds ~1e-7 in binary32 for lambda < 2.5 at every t0 and up to
// lambda < 8 when t0 < 0; the forward recursion is used elsewhere.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool backward_fp32(float lam, float t0)
{
    return lam < 2.5f || (t0 < 0.0f && lam < 8.0f);
}

template <int K>
__device__ __forceinline__ void integrals_fp32(float lam, float t0, float (&I)[K + 1])
{
    static_assert(K >= 1 && K <= 7, "K out of range");
    if (!backward_fp32(lam, t0)) {
        const float inv2l = 0.5f / lam;
        const float rl = rsqrtf(lam);
        const float sl = lam * rl;
        const float h = 0.886226925452758f * rl;
        // branch-free over the position of t0, as in the binary64 engine
        const float d = t0 < 0.0f ? -t0 : (t0 > 1.0f ? t0 - 1.0f : 0.0f);
        const float E0s = expf(-lam * ((t0 - d) * (t0 + d)));
        const float E1s = expf(-lam * ((1.0f - t0 - d) * (1.0f - t0 + d)));
        const bool inside = d == 0.0f;
        const float S = inside ? 2.0f : 0.0f;
        const float ca = inside ? E1s : -1.0f;
        const float xa = inside ? sl * (1.0f - t0) : sl * d;
        const float cb = inside ? E0s : (t0 < 0.0f ? E1s : E0s);
        const float xb = inside ? sl * t0 : sl * (1.0f + d);
        const float I0 = h * (S - ca * erfcxf(xa) - cb * erfcxf(xb));
        const float e1 = E1s * inv2l;
        I[0] = I0;
        I[1] = fmaf(t0, I0, (E0s - E1s) * inv2l);
#pragma unroll
        for (int k = 2; k <= K; ++k) I[k] = fmaf(t0, I[k - 1], fmaf((float)(k - 1) * inv2l, I[k - 2], -e1));
    } else {
        const float d = t0 < 0.0f ? -t0 : (t0 > 1.0f ? t0 - 1.0f : 0.0f);
        const float E1s = expf(-lam * ((1.0f - t0 - d) * (1.0f - t0 + d)));
        // start index by lambda (binary32 needs ~1e-7, so fewer steps than
        // the binary64 engine), made warp-uniform
        int Kp = lam <= 0.1f ? 16 : (lam <= 0.3f ? 20 : (lam <= 0.7f ? 24 : (lam <= 1.0f ? 28 : 48)));
        Kp = __reduce_max_sync(__activemask(), (unsigned)Kp);
        const float l2 = 2.0f * lam;
        const float q = l2 * (t0 - 1.0f);
        const float r1 = (float)(Kp + 2) + q, r0 = (float)(Kp + 1) + q;
        float hi = __fdividef(E1s, r1 > 1.0f ? r1 : (float)(Kp + 2));
        float lo = __fdividef(E1s, r0 > 1.0f ? r0 : (float)(Kp + 1));
#pragma unroll 4
        for (int k = Kp + 1; k >= K + 2; --k) {
            const float nx = fmaf(l2, fmaf(-t0, lo, hi), E1s) * c_recip.f[k - 1];
            hi = lo;
            lo = nx;
        }
        I[K] = lo;
        const float top = hi;
#pragma unroll
        for (int k = K + 1; k >= 2; --k) {
            const float Ik = (k == K + 1) ? top : I[k];
            I[k - 2] = fmaf(l2, fmaf(-t0, I[k - 1], Ik), E1s) * (1.0f / (float)(k - 1));
        }
    }
}

// Exact shifted moments M_b = sum_window (f - alpha)^b, b = 0..K (Eq. (24)).
template <int K>
__device__ __forceinline__ void shifted_moments(int alpha, const int64_t (&m)[K + 1], int64_t (&M)[K + 1])
{
    int64_t s[K + 1];
#pragma unroll
    for (int a = 0; a <= K; ++a) s[a] = m[a];
    M[0] = s[0];
#pragma unroll
    for (int b = 1; b <= K; ++b) {
#pragma unroll
        for (int a = 0; a <= K - b; ++a) s[a] = s[a + 1] - (int64_t)alpha * s[a];
        M[b] = s[0];
    }
}

// binary32 tail shared by both variants: kernel parameters, integrals and
// the ratio of Eq. (29) from float coefficients c.
//
// Guard: the sums T1 = sum c_k I_{k+1} and T2 = sum c_k I_k cancel (the
// fitted coefficients alternate and are large), so their binary32 error is
// about u (S1 + |F| S2) / |T2| relative in F, with S1 = sum |c_k I_{k+1}|,
// S2 = sum |c_k I_k|, u = 2^-24.  When that estimate, scaled to gray levels
// by (beta - alpha) and by 4 ulps of slack for the integrals' own error,
// exceeds kFp32GuardGray, or the binary32 integrals are in a regime where
// they are known to lose digits, or T2 <= 0, the tail reports `redo` and the
// caller recomputes the pixel on the FP64 path.
constexpr float kFp32GuardGray = 0.25f;

__device__ __forceinline__ bool fp32_integrals_weak(float lam, float t0)
{
    const float sl = sqrtf(lam);
    if (t0 < 0.0f && !backward_fp32(lam, t0)) return sl * (-t0) > 0.5f;   // forward, centre left of 0
    if (t0 > 1.0f && backward_fp32(lam, t0)) return lam > 0.7f && sl * (t0 - 1.0f) > 1.0f;
    return false;
}

// fb_ratio(): mu_1 / mu_0 for the fallback of Eq. (29) (the sigma -> infinity
// limit), e.g. mu'_1 / mu'_0 of the scaled moments; evaluated only when the
// fallback is taken.
template <int N, typename FbRatio>
__device__ __forceinline__ float fabf_tail_fp32(const float (&c)[N + 1], FbRatio&& fb_ratio, int alpha, int d,
                                               float theta_f, float sigma_f, int& fallback, bool& redo)
{
    const float rd = 1.0f / (float)d;
    const float t0 = (theta_f - (float)alpha) * rd;
    const float lam = (float)(d * d) / (2.0f * sigma_f * sigma_f);
    float I[N + 2];
    integrals_fp32<N + 1>(lam, t0, I);
    float T1 = c[0] * I[1], T2 = c[0] * I[0];
    float S1 = fabsf(T1), S2 = fabsf(T2);
#pragma unroll
    for (int k = 2; k <= N + 1; ++k) {
        T1 = fmaf(c[k - 1], I[k], T1);
        T2 = fmaf(c[k - 1], I[k - 1], T2);
        S1 = fmaf(fabsf(c[k - 1]), fabsf(I[k]), S1);
        S2 = fmaf(fabsf(c[k - 1]), fabsf(I[k - 1]), S2);
    }
    float F = T1 / T2;
    const float est = 4.0f * 5.9604645e-8f * (float)d * (S1 + fabsf(F) * S2) / fabsf(T2);
    redo = !(T2 > 0.0f) || !(est <= kFp32GuardGray) || fp32_integrals_weak(lam, t0);
    if (!(T2 > 0.0f) || !isfinite(F)) {
        F = fb_ratio();
        fallback = 1;
    }
    return fmaf((float)d, F, (float)alpha);
}

// Fit in binary64 from (commonly scaled) moments, the rest in binary32.
template <int N>
__device__ __forceinline__ float fabf_fit_tail_fp64fit(const AinvTable& A, const double (&mu)[(N < 1 ? 1 : N) + 1],
                                                       int alpha, int d, float theta_f, float sigma_f, int& fallback,
                                                       bool& redo)
{
    float c[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k <= N; ++k) acc = fma(A.v[N][n][k], mu[k], acc);
        c[n] = double_to_float_rn(acc);
    }
    return fabf_tail_fp32<N>(c, [&] { return (float)(mu[1] / mu[0]); }, alpha, d, theta_f, sigma_f, fallback, redo);
}

// FABF_FP64FIT_FP32REC: shift-scale and Hilbert fit in binary64 (the fit's
// conditioning needs it), integrals, recursion and ratio in binary32.
template <int N>
__device__ __forceinline__ float fabf_pixel_fp64fit(const AinvTable& A, int alpha, int beta, int fi,
                                                    const int64_t (&m)[(N < 1 ? 1 : N) + 1],
                                                    float theta_f, float sigma_f, int& fallback, bool& redo)
{
    redo = false;
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    if (alpha == beta) return (float)fi;
    const int d = beta - alpha;
    int64_t M[K + 1];
    shifted_moments<K>(alpha, m, M);
    // Scaled moments mu'_k = d^K mu_k = M_k d^(K-k): exact integers
    // (<= m_0 255^6 < 2^63), so no division; the common factor d^K cancels
    // in the ratio of Eq. (29).
    double mu[K + 1];
    {
        int64_t dp = 1;
#pragma unroll
        for (int k = K; k >= 0; --k) {
            mu[k] = (double)(M[k] * dp);
            dp *= d;
        }
    }
    return fabf_fit_tail_fp64fit<N>(A, mu, alpha, d, theta_f, sigma_f, fallback, redo);
}

// Error-free transformations (Knuth TwoSum, FMA TwoProduct) for the
// compensated binary32 fit.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}

// Exact float of an integer 0 <= x < 2^23 from its bits (2^23 + x has the
// exponent of 2^23 and x as mantissa), without a conversion instruction.
__device__ __forceinline__ float u23_to_float(uint32_t x)
{
    return __int_as_float(0x4B000000u | x) - 8388608.0f;
}

// 0 <= v < 2^63 as an unevaluated float-float hi + lo (error below 2^-47
// relative): three exact 23-bit chunks summed with TwoSum.
__device__ __forceinline__ void u63_to_ff(uint64_t v, float& hi, float& lo)
{
    const float f0 = u23_to_float((uint32_t)v & 0x7FFFFFu);
    const float f1 = u23_to_float((uint32_t)(v >> 23) & 0x7FFFFFu) * 8388608.0f;       // x 2^23
    const float f2 = u23_to_float((uint32_t)(v >> 46)) * 70368744177664.0f;            // x 2^46
    float s1, e1, s2, e2;
    two_sum(f2, f1, s1, e1);
    two_sum(s1, f0, s2, e2);
    const float t = e1 + e2;
    hi = s2 + t;
    lo = t - (hi - s2);
}

// Row n of the compensated fit c = A^{-1} mu from float-float (commonly
// scaled) moments mu_k = muh[k] + mul[k]: the result as the unevaluated
// pair s + comp.  The entries are compile-time constants after unrolling
// (immediate operands); their low halves are zero for N <= 5 (entries <
// 2^24), and those products are skipped.  The first product is exact as
// s + comp.
template <int N>
__device__ __forceinline__ void compensated_fit_row(int n, const float (&muh)[(N < 1 ? 1 : N) + 1],
                                                    const float (&mul)[(N < 1 ? 1 : N) + 1], float& s, float& comp)
{
    constexpr AinvSplitTable kA = make_ainv_split_table();
    two_prod(kA.hi[N][n][0], muh[0], s, comp);
    comp = fmaf(kA.hi[N][n][0], mul[0], comp);
    if (kA.lo[N][n][0] != 0.0f) comp = fmaf(kA.lo[N][n][0], muh[0], comp);
#pragma unroll
    for (int k = 1; k <= N; ++k) {
        const float ah = kA.hi[N][n][k], al = kA.lo[N][n][k];
        float p, pe, t, te;
        two_prod(ah, muh[k], p, pe);
        two_sum(s, p, t, te);
        s = t;
        float e = fmaf(ah, mul[k], pe + te);
        if (al != 0.0f) e = fmaf(al, muh[k], e);
        comp += e;
    }
}

// Compensated binary32 fit from float-float (commonly scaled) moments
// mu_k = muh[k] + mul[k], then the binary32 tail.
template <int N>
__device__ __forceinline__ float fabf_fit_tail_cfp32(const AinvSplitTable& A, const float (&muh)[(N < 1 ? 1 : N) + 1],
                                                     const float (&mul)[(N < 1 ? 1 : N) + 1], int alpha, int d,
                                                     float theta_f, float sigma_f, int& fallback, bool& redo)
{
    (void)A;
    float c[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        float s, comp;
        compensated_fit_row<N>(n, muh, mul, s, comp);
        c[n] = s + comp;
    }
    return fabf_tail_fp32<N>(c, [&] { return muh[1] / muh[0]; }, alpha, d, theta_f, sigma_f, fallback, redo);
}

// FABF_CFP32: no binary64.  mu_k as float-float quotients of the exact
// integers M_k and d^k, and c = A^{-1} mu by compensated dot products
// (Ogita, Rump & Oishi, "Accurate sum and dot product", 2005: TwoProduct
// and TwoSum accumulate each product's and each addition's rounding error,
// so the dot product is as accurate as if evaluated in twice the working
// precision); A^{-1} entries (< 2^28) are split exactly into two floats.
template <int N>
__device__ __forceinline__ float fabf_pixel_cfp32(const AinvSplitTable& A, int alpha, int beta, int fi,
                                                  const int64_t (&m)[(N < 1 ? 1 : N) + 1],
                                                  float theta_f, float sigma_f, int& fallback, bool& redo)
{
    redo = false;
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    if (alpha == beta) return (float)fi;
    const int d = beta - alpha;
    int64_t M[K + 1];
    shifted_moments<K>(alpha, m, M);
    // Scaled moments mu'_k = M_k d^(K-k) (exact integers, see above) as
    // float-float values, converted in 23-bit chunks without a 64-bit
    // conversion instruction.
    float muh[K + 1], mul[K + 1];
    {
        int64_t dp = 1;
#pragma unroll
        for (int k = K; k >= 0; --k) {
            u63_to_ff((uint64_t)(M[k] * dp), muh[k], mul[k]);
            dp *= d;
        }
    }
    return fabf_fit_tail_cfp32<N>(A, muh, mul, alpha, d, theta_f, sigma_f, fallback, redo);
}

// The FP64 redo of FABF_CFP32 for the pixels its guard hands back, from
// commonly scaled moments v_k < 2^63 (the scale cancels in Eq. (29)): the
// same float-float moments and compensated fit as the binary32 tail, each
// coefficient taken as its unevaluated pair s + comp in binary64 (the fit is
// as accurate as if evaluated in twice the working precision), then the
// binary64 integrals and ratio.  This skips the binary64 divisions and the
// binary64 fit of fabf_pixel_fp64: about a third of the binary64
// instructions, each of which occupies the narrow FP64 pipe for a whole warp.
template <int N>
__device__ __forceinline__ double fabf_redo_scaled(const uint64_t (&v)[(N < 1 ? 1 : N) + 1], int alpha, int d,
                                                   float theta_f, float sigma_f, int& fallback)
{
    constexpr int K = N < 1 ? 1 : N;
    float muh[K + 1], mul[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) u63_to_ff(v[k], muh[k], mul[k]);
    double c[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        float sh, sc;
        compensated_fit_row<N>(n, muh, mul, sh, sc);
        c[n] = (double)sh + (double)sc;
    }
    double t0, lam, I[N + 2], T1, T2;
    double F = fp64_ratio<N, false>(c, alpha, d, theta_f, sigma_f, t0, lam, I, T1, T2);
    fallback = 0;
    if (!ratio_usable(T2, F)) {       // the sigma -> infinity limit, as fabf_tail_fp64
        F = ((double)muh[1] + (double)mul[1]) / ((double)muh[0] + (double)mul[0]);
        fallback = 1;
    }
    return (double)alpha + (double)d * F;
}

// The box path's redo: the exactly scaled moments mu'_k = M_k d^(K-k).
template <int N>
__device__ __forceinline__ double fabf_pixel_cfp32_redo(int alpha, int beta, int fi,
                                                        const int64_t (&m)[(N < 1 ? 1 : N) + 1], float theta_f,
                                                        float sigma_f, int& fallback)
{
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    if (alpha == beta) return (double)fi;
    const int d = beta - alpha;
    int64_t M[K + 1];
    shifted_moments<K>(alpha, m, M);
    uint64_t v[K + 1];
    int64_t dp = 1;
#pragma unroll
    for (int k = K; k >= 0; --k) {
        v[k] = (uint64_t)(M[k] * dp);
        dp *= d;
    }
    return fabf_redo_scaled<N>(v, alpha, d, theta_f, sigma_f, fallback);
}

// ===========================================================================
// FABF_C32: the binary32 form in the centred variable s = 2t - 1.
//
// The fitted polynomial p is the unique one of degree N whose moments over
// [0, 1] match the window's (Eqs. (18)-(19)); any basis of the polynomials of
// degree N gives the same p.  In the monomials of t the system is the Hilbert
// matrix, whose inverse has entries up to 1.3e8 (N = 6): the coefficients
// alternate and are large, and the sums T1, T2 of Eq. (29) cancel, which is
// why binary32 needs compensation or FP64 there.  In the monomials of the
// centred variable s = 2t - 1 in [-1, 1] the system is
//   A~[j][k] = int_0^1 s^(j+k) dt = 1 / (j + k + 1) if j + k is even, else 0,
// a checkerboard Hankel matrix whose inverse has dyadic entries of at most
// 5211 (N = 6), all exact in binary32; its coefficients are small and the
// sums hardly cancel, so a plain binary32 fit and binary32 sums are accurate.
//
// Every quantity is the paper's, expressed in s:
//   moments   mu~_k = sum_window s_j^k, s_j = (2 f_j - alpha - beta) / d,
//             formed exactly in integers (scaled by d^K) from the power sums;
//   fit       c~ = A~^{-1} mu~ (even and odd coefficients decouple);
//   integrals J_k = int_0^1 s^k exp(-lambda (t - t0)^2) dt, by the same
//             integration by parts as Eq. (30), in s (see integrals_c32);
//   ratio     T2 = sum c~_k J_k, T1 = int t p phi = (sum c~_k (J_k+1 + J_k)) / 2,
//             so g_hat = alpha + d T1 / T2 = (alpha + beta) / 2
//                        + (d / 2) sum c~_k J_(k+1) / T2.
// ===========================================================================

// A~^{-1} for N = 0..6, [N][n][k], computed at compile time (Gauss-Jordan in
// binary64 on the symmetric positive definite A~, then snapped to the grid of
// 1/256, on which every entry lies exactly; the snap is checked below).
struct CentredInvTable {
    float v[kNMax + 1][kNMax + 1][kNMax + 1];
    double err;   // largest distance of a binary64 entry from its snapped value
};

__host__ __device__ constexpr double centred_snap(double x)
{
    const double y = x * 256.0;
    const long long q = (long long)(y >= 0.0 ? y + 0.5 : y - 0.5);
    return (double)q / 256.0;
}

__host__ __device__ constexpr CentredInvTable make_centred_inverse_table()
{
    CentredInvTable t{};
    t.err = 0.0;
    for (int N = 0; N <= kNMax; ++N) {
        const int n = N + 1;
        double a[kNMax + 1][kNMax + 1] = {};
        double b[kNMax + 1][kNMax + 1] = {};
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                a[j][k] = ((j + k) & 1) ? 0.0 : 1.0 / (double)(j + k + 1);
                b[j][k] = j == k ? 1.0 : 0.0;
            }
        for (int p = 0; p < n; ++p) {            // no pivoting: A~ is SPD
            const double ip = 1.0 / a[p][p];
            for (int k = 0; k < n; ++k) {
                a[p][k] *= ip;
                b[p][k] *= ip;
            }
            for (int r = 0; r < n; ++r) {
                if (r == p) continue;
                const double f = a[r][p];
                for (int k = 0; k < n; ++k) {
                    a[r][k] -= f * a[p][k];
                    b[r][k] -= f * b[p][k];
                }
            }
        }
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                const double q = centred_snap(b[j][k]);
                const double e = q > b[j][k] ? q - b[j][k] : b[j][k] - q;
                if (e > t.err) t.err = e;
                t.v[N][j][k] = (float)q;
            }
    }
    return t;
}

static_assert(make_centred_inverse_table().err < 1e-6, "centred inverse entries are not on the 1/256 grid");

// Start indices of the downward recursion of integrals_c32.  One step maps
// (J_(k+1), J_k) to (J_k, J_(k-1)); an error in the pair is multiplied by
// the spectral radius of the step's homogeneous part,
//   rho_k = (a + sqrt(a^2 + 4b)) / 2,  a = lambda |s0| / (2k), b = lambda / (2k).
// Kp is the smallest index with prod_{k=9}^{Kp} rho_k < 1e-5, taken at the
// upper corner of a bin of (lambda, |s0|) (bins of 1/4 in lambda < 8 and
// 1/2 in |s0| < 4; K = 7, the largest top index -- smaller K only recurse
// further past their last index).  The start values are within a few
// percent, so what is left of their error is below 1e-6 of the integrals,
// under the binary32 recursion's own rounding (up to ~1e-5 of max_k |J_k|
// near lambda = 8); a target of 1e-8 gave the same worst error with 6 more
// steps on average.
__host__ __device__ constexpr double ct_sqrt(double x)
{
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 60; ++i) r = 0.5 * (r + x / r);
    return r;
}

struct KpTableC32 {
    unsigned char v[32][8];   // [lambda bin][|s0| bin]
};

__host__ __device__ constexpr KpTableC32 make_kp_table_c32()
{
    KpTableC32 t{};
    for (int i = 0; i < 32; ++i)
        for (int j = 0; j < 8; ++j) {
            const double lam = (i + 1) * 0.25, as0 = (j + 1) * 0.5;
            double p = 1.0;
            int kp = 8;
            do {
                ++kp;
                const double a = lam * as0 / (2.0 * kp), b = lam / (2.0 * kp);
                p *= 0.5 * (a + ct_sqrt(a * a + 4.0 * b));
            } while (p >= 1e-5 && kp < 63);
            t.v[i][j] = (unsigned char)kp;
        }
    return t;
}

static __device__ const KpTableC32 g_kp32 = make_kp_table_c32();   // global: lanes index it by their own bin

// lambda at and above which integrals_c32 recurses forward.
constexpr float kLambdaForwardC32 = 8.0f;

// J_k = int_0^1 s^k exp(-lambda (t - t0)^2) dt, s = 2t - 1, k = 0..K, each
// times exp(lambda d^2) with d the distance from t0 to [0, 1] (the factor is
// common to T1 and T2 and cancels).  With s0 = 2 t0 - 1, E0 = exp(-lambda t0^2)
// and E1 = exp(-lambda (1 - t0)^2) (both scaled), integration by parts of
// s^k (s - s0) exp(...) -- as for Eq. (30) -- gives
//   J_(k+1) = s0 J_k + (2k / lambda) J_(k-1) - (E1 - (-1)^k E0) / lambda,
// J_0 = I_0 of Eq. (31), J_1 = s0 J_0 - (E1 - E0) / lambda.
//  lambda >= 8: forward, as written;
//  lambda <  8: downward (the recursion solved for J_(k-1)), which damps
//               errors once k exceeds about lambda (1 + |s0|) / 2, from a
//               start index Kp taken from g_kp32 and made warp-uniform, with the
//               start values J_k ~ (E1 / (k + 1 - lambda (1 - t0))
//               + (-1)^k E0 / (k + 1 - lambda t0)) / 2 (the mass of s^k near
//               s = +-1); no erf is needed.
template <int K>
__device__ __forceinline__ void integrals_c32(float lam, float t0, float s0, float (&J)[K + 1])
{
    static_assert(K >= 1 && K <= 7, "K out of range");
    const float d = t0 < 0.0f ? -t0 : (t0 > 1.0f ? t0 - 1.0f : 0.0f);
    const float E0s = expf(-lam * ((t0 - d) * (t0 + d)));
    const float E1s = expf(-lam * ((1.0f - t0 - d) * (1.0f - t0 + d)));
    const float Ep = E1s + E0s, Em = E1s - E0s;   // E1 - (-1)^k E0 for k odd, even
    if (lam >= kLambdaForwardC32) {
        const float rl = rsqrtf(lam);
        const float sl = lam * rl;
        const float h = 0.886226925452758f * rl;
        const bool inside = d == 0.0f;
        const float S = inside ? 2.0f : 0.0f;
        const float ca = inside ? E1s : -1.0f;
        const float xa = inside ? sl * (1.0f - t0) : sl * d;
        const float cb = inside ? E0s : (t0 < 0.0f ? E1s : E0s);
        const float xb = inside ? sl * t0 : sl * (1.0f + d);
        const float il = 1.0f / lam;
        J[0] = h * (S - ca * erfcxf(xa) - cb * erfcxf(xb));
        J[1] = fmaf(s0, J[0], -Em * il);
#pragma unroll
        for (int k = 1; k < K; ++k)
            J[k + 1] = fmaf(s0, J[k], fmaf((float)(2 * k) * il, J[k - 1], -((k & 1) ? Ep : Em) * il));
    } else {
        const int bl = min(31, (int)(lam * 4.0f)), bs = min(7, (int)(fabsf(s0) * 2.0f));
        int Kp = __ldg(&g_kp32.v[bl][bs]);
        Kp = (int)__reduce_max_sync(__activemask(), (unsigned)Kp) | 1;   // odd: the step parities are fixed
        const float l1 = lam * (1.0f - t0), l0 = lam * t0;
        float a1 = (float)(Kp + 2) - l1, b1 = (float)(Kp + 2) - l0;
        float a0 = (float)(Kp + 1) - l1, b0 = (float)(Kp + 1) - l0;
        a1 = a1 > 1.0f ? a1 : (float)(Kp + 2);
        b1 = b1 > 1.0f ? b1 : (float)(Kp + 2);
        a0 = a0 > 1.0f ? a0 : (float)(Kp + 1);
        b0 = b0 > 1.0f ? b0 : (float)(Kp + 1);
        const float sg = (Kp & 1) ? 1.0f : -1.0f;   // (-1)^(Kp+1)
        float hi = 0.5f * (__fdividef(E1s, a1) + sg * __fdividef(E0s, b1));   // J_(Kp+1)
        float lo = 0.5f * (__fdividef(E1s, a0) - sg * __fdividef(E0s, b0));   // J_(Kp)
        // (hi, lo) = (J_(k+1), J_k) -> J_(k-1), for k = Kp .. K + 1, two
        // steps at a time from the odd Kp (odd k adds Ep, even k Em)
        int k = Kp;
        for (; k - 1 > K; k -= 2) {
            const float n1 = fmaf(lam, fmaf(-s0, lo, hi), Ep) * (0.5f * c_recip.f[k]);
            const float n2 = fmaf(lam, fmaf(-s0, n1, lo), Em) * (0.5f * c_recip.f[k - 1]);
            hi = n1;
            lo = n2;
        }
        if (k > K) {   // one odd step left (k == K + 1)
            const float nx = fmaf(lam, fmaf(-s0, lo, hi), Ep) * (0.5f * c_recip.f[k]);
            hi = lo;
            lo = nx;
        }
        J[K] = lo;
        const float top = hi;   // J_(K+1)
#pragma unroll
        for (int k = K; k >= 1; --k) {
            const float Jk1 = (k == K) ? top : J[k + 1];
            J[k - 1] = fmaf(lam, fmaf(-s0, J[k], Jk1), (k & 1) ? Ep : Em) * (0.5f / (float)k);
        }
    }
}

// Error bound per unit of the sums' scale for the guard of FABF_C32: the
// binary32 integrals carry up to ~1e-5 of max_k |J_k| in the regimes they are
// used in, the rest (moments, fit, sums) a few units of 2^-24.
constexpr float kGuardUnitC32 = 1.0e-5f;

// Regimes where the binary32 integrals of integrals_c32 lose digits: a
// range-kernel centre more than one kernel width outside [0, 1]
// (sqrt(lambda) d > 1) with 2.5 < lambda < 16 (both recursion directions
// amplify there: up to ~1e-3 of max |J_k|; within 0.75 widths they hold
// ~1e-5).
__device__ __forceinline__ bool c32_integrals_weak(float lam, float t0)
{
    const float d = t0 < 0.0f ? -t0 : (t0 > 1.0f ? t0 - 1.0f : 0.0f);
    return lam > 2.5f && lam < 16.0f && d * d * lam > 1.0f;
}

// The centred binary32 tail from commonly scaled centred moments v_k =
// scale * mu~_k (|v_k| < 2^63, exact integers; the scale cancels in the
// ratio).  Returns g_hat; sets redo when the pixel must be recomputed on the
// FP64 path (the error estimate above kFp32GuardGray, T2 not clearly of one
// sign, or a weak integral regime).  When T2 is negative by more than its
// error estimate, the binary64 T2 is negative too and the pixel takes the
// fallback of Eq. (29) (the sigma -> infinity limit): fb_mean, with fallback
// set.
template <int N, typename FbMean>
__device__ __forceinline__ float fabf_tail_c32(const int64_t (&v)[(N < 1 ? 1 : N) + 1], int alpha, int beta,
                                               float theta_f, float sigma_f, FbMean&& fb_mean, int& fallback,
                                               bool& redo)
{
    constexpr CentredInvTable kA = make_centred_inverse_table();
    // one correctly rounded conversion each (the conversion pipe is
    // otherwise idle in this kernel)
    float mu[N + 1];
#pragma unroll
    for (int k = 0; k <= N; ++k) mu[k] = __ll2float_rn(v[k]);
    // c~ = A~^{-1} mu~: even coefficients from even moments, odd from odd
    float c[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int k = n & 1; k <= N; k += 2) acc = fmaf(kA.v[N][n][k], mu[k], acc);
        c[n] = acc;
    }
    const int d = beta - alpha;
    const float rd = __fdividef(1.0f, (float)d);                 // within 2 ulp
    const float t0 = (theta_f - (float)alpha) * rd;
    const float s0 = (2.0f * theta_f - (float)(alpha + beta)) * rd;
    const float lam = __fdividef((float)(d * d), 2.0f * sigma_f * sigma_f);
    float J[N + 2];
    integrals_c32<N + 1>(lam, t0, s0, J);
    float T2 = c[0] * J[0], U = c[0] * J[1];
    float S2 = fabsf(T2), S1 = fabsf(U);
#pragma unroll
    for (int k = 1; k <= N; ++k) {
        T2 = fmaf(c[k], J[k], T2);
        U = fmaf(c[k], J[k + 1], U);
        S2 = fmaf(fabsf(c[k]), fabsf(J[k]), S2);
        S1 = fmaf(fabsf(c[k]), fabsf(J[k + 1]), S1);
    }
    const float R = U / T2;
    const float hd = 0.5f * (float)d;
    // Bound on the error of T2: the integrals are within kGuardUnitC32 of
    // max_k |J_k| each, so |dT2| <= kGuardUnitC32 max|J| sum|c~_k| (the
    // binary32 fit and sums add a few units of 2^-24 of S2, far less).  T2
    // below minus that bound is negative in every precision, and the pixel
    // takes the fallback; within the bound of zero it goes to the FP64 path.
    float csum = fabsf(c[0]), jmax = fabsf(J[N + 1]);
#pragma unroll
    for (int k = 1; k <= N; ++k) csum += fabsf(c[k]);
#pragma unroll
    for (int k = 0; k <= N; ++k) jmax = fmaxf(jmax, fabsf(J[k]));
    const float t2_err = kGuardUnitC32 * csum * jmax;
    if (T2 < -t2_err) {
        fallback = 1;
        redo = c32_integrals_weak(lam, t0);
        return fb_mean();
    }
    // error estimate kGuardUnitC32 (d / 2) (S1 + |R| S2) / |T2| <= 0.25 gray,
    // tested without the division
    const float est_num = kGuardUnitC32 * hd * (S1 + fabsf(R) * S2);
    redo = !(T2 > t2_err) || !(est_num <= kFp32GuardGray * T2) || c32_integrals_weak(lam, t0);
    return fmaf(hd, R, 0.5f * (float)(alpha + beta));
}

// Exact centred moments M~_b = sum_window (2 f - c0)^b, c0 = alpha + beta,
// b = 0..K, from the power sums m_a by S(a, b) = S(a+1, b-1) - c0 S(a, b-1),
// S(a, 0) = 2^a m_a, in wrapping 64-bit arithmetic: every step is exact
// modulo 2^64 and |M~_b| <= m_0 d^b < 2^63, so the results are exact.
template <int K>
__device__ __forceinline__ void centred_moments(int c0, const int64_t (&m)[K + 1], int64_t (&M)[K + 1])
{
    uint64_t S[K + 1];
#pragma unroll
    for (int a = 0; a <= K; ++a) S[a] = (uint64_t)m[a] << a;
    M[0] = (int64_t)S[0];
#pragma unroll
    for (int b = 1; b <= K; ++b) {
#pragma unroll
        for (int a = 0; a <= K - b; ++a) S[a] = S[a + 1] - (uint64_t)c0 * S[a];
        M[b] = (int64_t)S[0];
    }
}

// FABF_C32 at one pixel of the box path.  The fallback value is the window
// mean m_1 / m_0 (the sigma -> infinity limit alpha + d mu_1 / mu_0; both
// integers are exact in binary32 since m_1 <= 81^2 255 < 2^24).
template <int N>
__device__ __forceinline__ float fabf_pixel_c32(int alpha, int beta, int fi, const int64_t (&m)[(N < 1 ? 1 : N) + 1],
                                                float theta_f, float sigma_f, int& fallback, bool& redo)
{
    constexpr int K = N < 1 ? 1 : N;
    redo = false;
    fallback = 0;
    if (alpha == beta) return (float)fi;
    const int d = beta - alpha;
    int64_t M[K + 1];
    centred_moments<K>(alpha + beta, m, M);
    // mu~_k d^K = M~_k d^(K-k): exact integers, |.| <= m_0 d^K < 2^63
    int64_t v[K + 1];
    int64_t dp = 1;
#pragma unroll
    for (int k = K; k >= 0; --k) {
        v[k] = (int64_t)((uint64_t)M[k] * (uint64_t)dp);
        dp *= d;
    }
    return fabf_tail_c32<N>(v, alpha, beta, theta_f, sigma_f, [&] { return (float)m[1] / (float)m[0]; }, fallback,
                            redo);
}

}  // namespace fabf

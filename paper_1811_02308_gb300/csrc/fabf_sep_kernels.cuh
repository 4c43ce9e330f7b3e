// Tiled kernel of fast adaptive bilateral filtering with a separable integer
// spatial kernel omega(j) = g[jy + r] g[jx + r] on the window [-r, r]^2 --
// the Gaussian of Eq. (4) on the paper's window [-3 rho, 3 rho]^2 when the
// taps are a quantised Gaussian -- and its brute-force comparator.
//
// One CTA (256 threads) produces a TH x 64 output tile, staged like the box
// kernel's (one TMA copy of the tile plus an r-pixel halo, or a plain load):
//  1. Per chunk of 8 output rows, the vertical pass: every (column, row)
//     item forms V_k = sum_t g[t] f(row + t - r, column)^k for k = 1..K by a
//     direct (2r+1)-tap FIR in 32/64-bit integers (exact: V_k < 65535 255^6
//     < 2^64), and each column takes the vertical min / max of the chunk's 8
//     windows from suffix and prefix extrema (Eq. (8)), as the box kernel.
//  2. Horizontal pass, warp rr on chunk row rr: min / max by lane blocks
//     (sparse-table levels for r <= 2), as the box kernel, then for each of the lane's two pixels m_k = sum_t g[t]
//     V_k(column + t - r), exact in 64 bits for k <= 4 and in 128 bits (two
//     64-bit partial sums of the 32-bit halves of V_k) for k = 5, 6; m_0
//     from the tap prefix sums and the clipped window.  Out-of-image pixels
//     are zero in the staged tile, so they add nothing to m_k, k >= 1.
//  3. M_k = sum omega (f - alpha)^k exactly in 128 bits (the recursion of the
//     box path).  The FP64 form takes mu_k = M_k / (beta - alpha)^k with M_k
//     correctly rounded to binary64 and the binary64 tail shared with the box
//     path.  The binary32 forms take the exactly scaled moments mu'_k = M_k
//     d^(K-k) <= mu'_0 = m_0 d^K < 2^80, shifted right by one common amount
//     so that mu'_0 < 2^63 (the factor cancels in Eq. (29)), into the box
//     path's binary32 fits, guard and FP64 redo pass.
//
// The direct FIR costs O(r) per pixel (the paper's own implementation uses a
// direct convolution for practical rho, Sec. II-D).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fabf_kernels.cuh"

namespace fabf {

typedef unsigned __int128 u128;

constexpr uint32_t kTapSumMax = 65535;   // keeps V_k < 2^64 and m_k < 2^81

struct SepTaps {
    int r;
    int casc_n;                    // 0: direct FIR of g; else the box length n of a 3-box cascade (g its taps)
    int16_t pre_w[3][2 * kWMax];   // cascade: weights of tile row t in the start sums U1, U2, V (2r rows)
    uint32_t g[2 * kWMax + 1];
    uint32_t G[2 * kWMax + 2];     // G[t] = g[0] + ... + g[t-1]
};

struct SepDebug {                  // per-stage exports for the parity tests (all optional)
    uint8_t* alpha;                // H x W
    uint8_t* beta;                 // H x W
    uint64_t* m;                   // (N+1) x H x W x 2 words (low, high)
    uint64_t* M;                   // (N+1) x H x W x 2 words (low, high)
    double* mu;                    // (N+1) x H x W
    double* c;                     // (N+1) x H x W
    double* t0lam;                 // 2 x H x W
    double* I;                     // (N+2) x H x W
    double* T;                     // 2 x H x W
    int32_t* flags;                // H x W: bit0 flat window, bit1 fallback taken
};

struct SepParams {
    ImageJob job;                  // job.w is the kernel radius r
    SepTaps taps;
    unsigned* status;
    unsigned long long* n_fallback;   // [0] fallback pixels, [1] pixels redone in FP64
    SepDebug dbg;
};

__host__ __device__ inline size_t sep_smem_bytes(int N, int r, int Cb, int TH)
{
    const int K = N < 1 ? 1 : N;
    size_t tile = ((size_t)(TH + 2 * r) * Cb + 127) & ~(size_t)127;
    size_t mm = ((size_t)4 * kChunk * Cb + (size_t)2 * kChunk * kLaneTable + 15) & ~(size_t)15;
    return 128 + tile + mm + (size_t)K * kChunk * Cb * 8 + kRedoBytes + kMapBytes;
}

// Correctly rounded (to nearest even) conversion of an unsigned 128-bit
// integer to binary64: the leading 64 bits with every lower bit folded into a
// sticky bit round exactly as the full value does (the sticky bit lies below
// the rounding position), then an exact power-of-two scaling.
__device__ __forceinline__ double u128_to_double_rn(u128 v)
{
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    if (hi == 0) return __ull2double_rn(lo);
    const int s = 64 - __clzll(hi);                  // 1..64 bits to drop
    uint64_t top, sticky;
    if (s == 64) {
        top = hi;
        sticky = lo != 0;
    } else {
        top = (hi << (64 - s)) | (lo >> s);
        sticky = (lo << (64 - s)) != 0;
    }
    return __ull2double_rn(top | sticky) * pow2i(s);   // exact scaling by 2^s
}

// acc += g * v for a 64-bit v and a 16-bit g whose product fits in 64 bits.
__device__ __forceinline__ void mac_u64(uint64_t& acc, uint32_t g, uint64_t v)
{
    acc += (uint64_t)g * (uint32_t)v;
    acc += (uint64_t)(g * (uint32_t)(v >> 32)) << 32;
}

// x * a for a 32-bit a (the product fits in 128 bits).
__device__ __forceinline__ u128 mul_u128_u32(u128 x, uint32_t a)
{
    const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
    const uint64_t plo = lo * a;
    const uint64_t phi = __umul64hi(lo, (uint64_t)a) + hi * a;
    return ((u128)phi << 64) | plo;
}

// x * a for a 64-bit a (the product fits in 128 bits).
__device__ __forceinline__ u128 mul_u128_u64(u128 x, uint64_t a)
{
    const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
    return ((u128)(__umul64hi(lo, a) + hi * a) << 64) | (lo * a);
}

// Eq. (24) exactly: M_b = sum omega (f - alpha)^b by S(a, b) = S(a+1, b-1) -
// alpha S(a, b-1), S(a, 0) = m_a; every S lies in [0, m_K] < 2^81.
template <int K>
__device__ __forceinline__ void sep_shifted_moments(int alpha, const u128 (&m)[K + 1], u128 (&M)[K + 1])
{
    u128 S[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) S[k] = m[k];
    M[0] = S[0];
#pragma unroll
    for (int b = 1; b <= K; ++b) {
#pragma unroll
        for (int q = 0; q <= K - b; ++q) S[q] = S[q + 1] - mul_u128_u32(S[q], (uint32_t)alpha);
        M[b] = S[0];
    }
}

// Algorithm 1 at one pixel in binary64 from the weighted power sums m_k.
template <int N, bool Own = true>
__device__ __forceinline__ double sep_pixel_fp64(int alpha, int beta, int fi, const u128 (&m)[(N < 1 ? 1 : N) + 1],
                                                 float th, float sg, int& fallback, PixelTrace* tr,
                                                 u128 (&M)[(N < 1 ? 1 : N) + 1])
{
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    if (alpha == beta) return (double)fi;                // flat window, Sec. II-A
    const int d = beta - alpha;
    sep_shifted_moments<K>(alpha, m, M);
    // mu_k = RN(M_k / d^k): the correctly rounded quotient from the
    // correctly rounded reciprocal of d^k (div_by_power), as in the box path
    double mu[K + 1];
    mu[0] = u128_to_double_rn(M[0]);
#pragma unroll
    for (int k = 1; k <= K; ++k)
        mu[k] = div_by_power(u128_to_double_rn(M[k]), __ldg(&g_recip_pow.p[k - 1][d]), __ldg(&g_recip_pow.v[k - 1][d]));
    return fabf_tail_fp64<N, Own>(c_ainv, alpha, d, mu, th, sg, fallback, tr);
}

// The binary32 forms at one pixel: exactly scaled moments mu'_k = M_k
// d^(K-k), shifted right together so that the largest, mu'_0 = m_0 d^K,
// is below 2^63.
template <int N, int PREC>
__device__ __forceinline__ float sep_pixel_fp32(int alpha, int beta, int fi, const u128 (&m)[(N < 1 ? 1 : N) + 1],
                                                float th, float sg, int& fallback, bool& redo)
{
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    redo = false;
    if (alpha == beta) return (float)fi;
    const int d = beta - alpha;
    u128 M[K + 1];
    sep_shifted_moments<K>(alpha, m, M);
    u128 sc[K + 1];
    {
        uint64_t dp = 1;
#pragma unroll
        for (int k = K; k >= 0; --k) {
            sc[k] = mul_u128_u64(M[k], dp);
            dp *= (uint64_t)d;
        }
    }
    const uint64_t top = (uint64_t)(sc[0] >> 64);
    const int shift = top ? 65 - __clzll(top) : ((uint64_t)sc[0] >> 63 ? 1 : 0);   // sc[0] >> shift < 2^63
    uint64_t v[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) v[k] = (uint64_t)(sc[k] >> shift);
    if constexpr (PREC == kPrecFP64Fit) {
        double mu[K + 1];
#pragma unroll
        for (int k = 0; k <= K; ++k) mu[k] = (double)(int64_t)v[k];
        return fabf_fit_tail_fp64fit<N>(c_ainv, mu, alpha, d, th, sg, fallback, redo);
    } else {
        float muh[K + 1], mul[K + 1];
#pragma unroll
        for (int k = 0; k <= K; ++k) u63_to_ff(v[k], muh[k], mul[k]);
        return fabf_fit_tail_cfp32<N>(c_ainv_split, muh, mul, alpha, d, th, sg, fallback, redo);
    }
}

// FABF_C32 at one pixel of the separable path: the centred moments M~_b =
// sum omega (2 f - c0)^b by the recursion of centred_moments in wrapping
// 128-bit arithmetic (exact: |M~_b| <= m_0 d^b < 2^81), scaled by d^(K-b),
// then shifted right together (arithmetically) so that the largest,
// m_0 d^K, is below 2^63; the common factor cancels in the ratio.
template <int N>
__device__ __forceinline__ float sep_pixel_c32(int alpha, int beta, int fi, const u128 (&m)[(N < 1 ? 1 : N) + 1],
                                               float th, float sg, int& fallback, bool& redo)
{
    constexpr int K = N < 1 ? 1 : N;
    redo = false;
    fallback = 0;
    if (alpha == beta) return (float)fi;
    const int d = beta - alpha;
    const uint32_t c0 = (uint32_t)(alpha + beta);
    u128 S[K + 1], M[K + 1];
#pragma unroll
    for (int a = 0; a <= K; ++a) S[a] = m[a] << a;
    M[0] = S[0];
#pragma unroll
    for (int b = 1; b <= K; ++b) {
#pragma unroll
        for (int a = 0; a <= K - b; ++a) S[a] = S[a + 1] - mul_u128_u32(S[a], c0);
        M[b] = S[0];
    }
    u128 sc[K + 1];
    {
        uint64_t dp = 1;
#pragma unroll
        for (int k = K; k >= 0; --k) {
            sc[k] = mul_u128_u64(M[k], dp);   // two's complement: exact modulo 2^128
            dp *= (uint64_t)d;
        }
    }
    const uint64_t top = (uint64_t)(sc[0] >> 64);   // sc[0] = m_0 d^K > 0
    const int shift = top ? 65 - __clzll(top) : ((uint64_t)sc[0] >> 63 ? 1 : 0);
    int64_t v[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) v[k] = (int64_t)((__int128)sc[k] >> shift);
    // fallback: the weighted window mean m_1 / m_0 (m_0 < 2^32, m_1 < 2^40),
    // as the box path forms it
    return fabf_tail_c32<N>(v, alpha, beta, th, sg, [&] { return (float)(int64_t)m[1] / (float)(int64_t)m[0]; },
                            fallback, redo);
}

// The compensated form's FP64 redo (fabf_redo_scaled) from the separable
// moments, scaled and shifted as in sep_pixel_fp32's compensated fit; with
// all-ones taps this is the box path's redo bit for bit.
template <int N>
__device__ __forceinline__ double sep_pixel_cfp32_redo(int alpha, int beta, int fi,
                                                       const u128 (&m)[(N < 1 ? 1 : N) + 1], float th, float sg,
                                                       int& fallback)
{
    constexpr int K = N < 1 ? 1 : N;
    fallback = 0;
    if (alpha == beta) return (double)fi;
    const int d = beta - alpha;
    u128 M[K + 1];
    sep_shifted_moments<K>(alpha, m, M);
    u128 sc[K + 1];
    uint64_t dp = 1;
#pragma unroll
    for (int k = K; k >= 0; --k) {
        sc[k] = mul_u128_u64(M[k], dp);
        dp *= (uint64_t)d;
    }
    const uint64_t top = (uint64_t)(sc[0] >> 64);
    const int shift = top ? 65 - __clzll(top) : ((uint64_t)sc[0] >> 63 ? 1 : 0);   // sc[0] >> shift < 2^63
    uint64_t v[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) v[k] = (uint64_t)(sc[k] >> shift);
    return fabf_redo_scaled<N>(v, alpha, d, th, sg, fallback);
}

// Writes one result of a separable-kernel tile to the image's output.
__device__ __forceinline__ void sep_store(const ImageJob& J, long long pix, double g)
{
    if (J.out_f64) static_cast<double*>(J.out)[pix] = g;
    else static_cast<float*>(J.out)[pix] = (float)g;
}

// The per-pixel part of Algorithm 1 for chunk row rr (image row Y) of a
// separable-kernel tile: each lane finishes tile columns lane and lane + 32
// from the window statistics stats(rr, x, alpha, beta, m, fi) (Eq. (8) and
// the weighted power sums of Eq. (17)).  The binary32 forms queue the pixels
// their guard rejects in (redo_n, redo_list) for sep_redo_pass.
template <int N, int PREC, typename Stats>
__device__ __forceinline__ void sep_row_pixels(const SepParams& P, Stats& stats, int rr, int Y, int x0,
                                               const float* s_maps, unsigned* redo_n, uint16_t* redo_list,
                                               int lane)
{
    constexpr int K = N < 1 ? 1 : N;
    const ImageJob& J = P.job;
#pragma unroll 1
    for (int h = 0; h < kTileW / 32; ++h) {
        const int x = lane + 32 * h;
        const int Xo = x0 + x;
        if (Xo >= J.W) continue;
        int alpha, beta, fi;
        u128 m[K + 1];
        stats(rr, x, alpha, beta, m, fi);
        const long long pix = (long long)Y * J.W + Xo;
        const float th = s_maps[rr * kTileW + x], sg = s_maps[(kChunk + rr) * kTileW + x];
        double g;
        int fb = 0;
        PixelTrace tr;
        PixelTrace* trp = (PREC == kPrecFP64 && P.dbg.mu) ? &tr : nullptr;
        u128 M[K + 1];
        if (!(sg > 0.0f) || !isfinite(sg) || !isfinite(th)) {
            g = __longlong_as_double(0x7ff8000000000000LL);
            if (P.status) atomicOr(P.status, kStatusBadInput);
            trp = nullptr;
        } else {
            if constexpr (PREC == kPrecFP64) {
                g = sep_pixel_fp64<N>(alpha, beta, fi, m, th, sg, fb, trp, M);
            } else {
                bool redo = false;
                if constexpr (PREC == kPrecC32)
                    g = (double)sep_pixel_c32<N>(alpha, beta, fi, m, th, sg, fb, redo);
                else
                    g = (double)sep_pixel_fp32<N, PREC>(alpha, beta, fi, m, th, sg, fb, redo);
                if (redo) {   // binary32 not accurate enough here: queue for the FP64 pass
                    const unsigned slot = atomicAdd(redo_n, 1u);
                    redo_list[slot] = (uint16_t)((rr << 8) | x);
                    continue;
                }
            }
            if (fb && P.n_fallback) atomicAdd(P.n_fallback, 1ull);
        }
        sep_store(J, pix, g);
        if (PREC == kPrecFP64 && P.dbg.alpha) {   // the stage planes come from the FP64 form only
            const SepDebug& D = P.dbg;
            const long long pl = (long long)J.H * J.W;
            D.alpha[pix] = (uint8_t)alpha;
            D.beta[pix] = (uint8_t)beta;
            for (int k = 0; k <= N; ++k) {
                D.m[2 * (k * pl + pix)] = (uint64_t)m[k];
                D.m[2 * (k * pl + pix) + 1] = (uint64_t)(m[k] >> 64);
            }
            D.flags[pix] = (alpha == beta ? 1 : 0) | (fb ? 2 : 0);
            if (trp && alpha != beta) {
                for (int k = 0; k <= N; ++k) {
                    D.M[2 * (k * pl + pix)] = (uint64_t)M[k];
                    D.M[2 * (k * pl + pix) + 1] = (uint64_t)(M[k] >> 64);
                    D.mu[k * pl + pix] = tr.mu[k];
                    D.c[k * pl + pix] = tr.c[k];
                }
                for (int k = 0; k <= N + 1; ++k) D.I[k * pl + pix] = tr.I[k];
                D.t0lam[pix] = tr.t0;
                D.t0lam[pl + pix] = tr.lam;
                D.T[pix] = tr.T1;
                D.T[pl + pix] = tr.T2;
            }
        }
    }
}

// The pixels a binary32 form queued, on the FP64 path (the compensated form's
// own FP64 redo), packed into full warps; y0r0 is the image row of chunk row 0.
template <int N, int PREC, typename Stats>
__device__ __forceinline__ void sep_redo_pass(const SepParams& P, Stats& stats, int y0r0, int x0,
                                              const float* s_maps, const unsigned* redo_n,
                                              const uint16_t* redo_list)
{
    constexpr int K = N < 1 ? 1 : N;
    const ImageJob& J = P.job;
    unsigned long long* redo_count = P.n_fallback ? P.n_fallback + 1 : nullptr;
    const unsigned nr = *redo_n;
    for (unsigned i = threadIdx.x; i < nr; i += blockDim.x) {
        const int e = redo_list[i];
        const int rr = e >> 8, x = e & 255;
        int alpha, beta, fi, fb = 0;
        u128 m[K + 1], M[K + 1];
        stats(rr, x, alpha, beta, m, fi);
        const long long pix = (long long)(y0r0 + rr) * J.W + (x0 + x);
        const float th = s_maps[rr * kTileW + x], sg = s_maps[(kChunk + rr) * kTileW + x];
        const double g = PREC == kPrecCFP32 ? sep_pixel_cfp32_redo<N>(alpha, beta, fi, m, th, sg, fb)
                                            : sep_pixel_fp64<N, false>(alpha, beta, fi, m, th, sg, fb, nullptr, M);
        sep_store(J, pix, g);
        if (fb && P.n_fallback) atomicAdd(P.n_fallback, 1ull);
        if (redo_count) atomicAdd(redo_count, 1ull);
    }
}

template <int N, int PREC>
__device__ __forceinline__ void sep_tile(const CUtensorMap* tmap, const SepParams& P, int tx, int ty,
                                         uint8_t* smem, uint32_t& phase)
{
    constexpr int K = N < 1 ? 1 : N;
    const ImageJob& J = P.job;
    const SepTaps& T = P.taps;
    const int r = J.w, Cb = J.Cb, off = J.off, TH = J.TH;
    const int R = TH + 2 * r;
    const int x0 = tx * kTileW, y0 = ty * TH;
    const int xs = x0 - r - off, ys = y0 - r;

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint8_t* tile = smem + 128;
    const size_t tile_bytes = ((size_t)R * Cb + 127) & ~(size_t)127;
    uint8_t* vmin = tile + tile_bytes;
    uint8_t* vmax = vmin + kChunk * Cb;
    uint8_t* pmin = vmax + kChunk * Cb;                                 // in-lane prefix extrema
    uint8_t* pmax = pmin + kChunk * Cb;
    uint8_t* ltmin = pmax + kChunk * Cb;                                // [kChunk][kLaneTable]
    uint8_t* ltmax = ltmin + kChunk * kLaneTable;
    uint64_t* V = reinterpret_cast<uint64_t*>(
        vmin + (((size_t)4 * kChunk * Cb + (size_t)2 * kChunk * kLaneTable + 15) & ~(size_t)15));   // [K][kChunk][Cb]
    unsigned* redo_n = reinterpret_cast<unsigned*>(V + (size_t)K * kChunk * Cb);
    uint16_t* redo_list = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(redo_n) + 16);
    float* s_maps = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(redo_n) + kRedoBytes);   // [2][kChunk][kTileW]
    const bool maps16 = maps_in_16(J);

    if (J.use_tma) {
        const bool ok = tma_load_tile(tmap, tile, bar, xs, ys, (uint32_t)(R * Cb), phase);
        phase ^= 1u;
        if (!ok) {
            if (threadIdx.x == 0 && P.status) atomicOr(P.status, kStatusTimeout);
            return;
        }
    } else {
        plain_load_tile(J, tile, xs, ys, R);
        __syncthreads();
    }

    const int rowlo = ys < 0 ? -ys : 0;
    const int rowhi = min(R - 1, J.H - 1 - ys);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int levels = 0;
    while ((2 << levels) <= 2 * r + 1) ++levels;
    const int span = 1 << levels;
    const bool lane_blocks = 2 * r + 1 >= 6;
    const int plane = kChunk * Cb;

    for (int r0 = 0; r0 < TH; r0 += kChunk) {
        if (y0 + r0 >= J.H) break;                                   // uniform per CTA
        if (threadIdx.x == 0) *redo_n = 0u;
        // the chunk's theta and sigma into shared memory while the vertical
        // phase runs (as in the box kernel)
        prefetch_maps(J, s_maps, y0 + r0, x0, maps16);
        // 1a. Vertical min / max of the 8 windows [rr, rr + 2r] of column c.
        {
            const int c = threadIdx.x;
            const int X = xs + c;
            if (c < Cb) {
                if (X >= 0 && X < J.W) {
                    // suffix extrema of the chunk's rows and prefix extrema
                    // from r0 + 8 (2r + 1 >= 8), as in the box kernel
                    uint8_t qmn = 255, qmx = 0;
                    const bool split = 2 * r + 1 >= kChunk;
                    if (split) {
                        uint8_t mn = 255, mx = 0;
#pragma unroll
                        for (int rr = kChunk - 1; rr >= 0; --rr) {
                            const int t = r0 + rr;
                            if (t >= rowlo && t <= rowhi) {
                                const uint8_t v = tile[t * Cb + c];
                                mn = v < mn ? v : mn;
                                mx = v > mx ? v : mx;
                            }
                            vmin[rr * Cb + c] = mn;      // suffix extrema, completed below
                            vmax[rr * Cb + c] = mx;
                        }
                        const int a = max(r0 + kChunk, rowlo), b = min(r0 + 2 * r, rowhi);
                        for (int t = a; t <= b; ++t) {
                            const uint8_t v = tile[t * Cb + c];
                            qmn = v < qmn ? v : qmn;
                            qmx = v > qmx ? v : qmx;
                        }
                    }
#pragma unroll
                    for (int rr = 0; rr < kChunk; ++rr) {
                        const int row = r0 + rr;
                        uint8_t mn, mx;
                        if (split) {
                            const int t = row + 2 * r;
                            if (rr > 0 && t >= rowlo && t <= rowhi) {
                                const uint8_t v = tile[t * Cb + c];
                                qmn = v < qmn ? v : qmn;
                                qmx = v > qmx ? v : qmx;
                            }
                            const uint8_t sn = vmin[rr * Cb + c], sx = vmax[rr * Cb + c];
                            mn = sn < qmn ? sn : qmn;
                            mx = sx > qmx ? sx : qmx;
                        } else {
                            mn = 255;
                            mx = 0;
                            const int a = max(row, rowlo), b = min(row + 2 * r, rowhi);
                            for (int t = a; t <= b; ++t) {
                                const uint8_t v = tile[t * Cb + c];
                                mn = v < mn ? v : mn;
                                mx = v > mx ? v : mx;
                            }
                        }
                        vmin[rr * Cb + c] = mn;
                        vmax[rr * Cb + c] = mx;
                    }
                } else {
#pragma unroll
                    for (int rr = 0; rr < kChunk; ++rr) {
                        vmin[rr * Cb + c] = 255;
                        vmax[rr * Cb + c] = 0;
                    }
                }
            }
        }
        // 1b. Vertical FIR of the powers, one (row, column) item per thread.
        for (int i = threadIdx.x; i < kChunk * Cb; i += blockDim.x) {
            const int rr = i / Cb, c = i - rr * Cb;
            const uint8_t* col = tile + (r0 + rr) * Cb + c;
            uint32_t a1 = 0, a2 = 0;
            uint64_t a3 = 0, a4 = 0, a5 = 0, a6 = 0;
#pragma unroll 4
            for (int t = 0; t <= 2 * r; ++t) {
                const uint32_t g = T.g[t];
                const uint32_t v = col[t * Cb];
                const uint32_t p2 = v * v;
                a1 += g * v;
                if constexpr (K >= 2) a2 += g * p2;
                if constexpr (K >= 3) {
                    const uint32_t p3 = p2 * v;
                    a3 += (uint64_t)g * p3;
                    if constexpr (K >= 4) {
                        const uint32_t p4 = p3 * v;
                        a4 += (uint64_t)g * p4;
                        if constexpr (K >= 5) {
                            const uint64_t p5 = (uint64_t)p4 * v;
                            mac_u64(a5, g, p5);
                            if constexpr (K >= 6) mac_u64(a6, g, p5 * v);
                        }
                    }
                }
            }
            uint64_t* Vi = V + rr * Cb + c;
            Vi[0] = a1;
            if constexpr (K >= 2) Vi[plane] = a2;
            if constexpr (K >= 3) Vi[2 * plane] = a3;
            if constexpr (K >= 4) Vi[3 * plane] = a4;
            if constexpr (K >= 5) Vi[4 * plane] = a5;
            if constexpr (K >= 6) Vi[5 * plane] = a6;
        }
        cp_async_wait_all();
        __syncthreads();

        // Window statistics of the pixel at chunk row rr, tile column x (the
        // chunk's min / max rows are sparse-table levels by now).
        auto stats = [&](int rr, int x, int& alpha, int& beta, u128 (&m)[K + 1], int& fi) {
            const int Y = y0 + r0 + rr, Xo = x0 + x;
            const int a = x + off;                      // tile column of the window's left edge
            if (lane_blocks) {
                alpha = lane_block_query<true>(vmin + rr * Cb, pmin + rr * Cb, ltmin + rr * kLaneTable, a, a + 2 * r);
                beta = lane_block_query<false>(vmax + rr * Cb, pmax + rr * Cb, ltmax + rr * kLaneTable, a, a + 2 * r);
            } else {
                alpha = min(vmin[rr * Cb + a], vmin[rr * Cb + a + 2 * r - span + 1]);
                beta = max(vmax[rr * Cb + a], vmax[rr * Cb + a + 2 * r - span + 1]);
            }
            fi = tile[(r0 + rr + r) * Cb + a + r];
            const int ty0 = max(r - Y, 0), ty1 = min(2 * r, J.H - 1 - Y + r);
            const int tx0 = max(r - Xo, 0), tx1 = min(2 * r, J.W - 1 - Xo + r);
            m[0] = (u128)((uint64_t)(T.G[ty1 + 1] - T.G[ty0]) * (uint64_t)(T.G[tx1 + 1] - T.G[tx0]));
            // Eq. (17): m_k = sum_t g[t] V_k(a + t).  k = 1, 2: V_k < 2^32, one
            // 32x32 -> 64-bit multiply-add; k = 3, 4: V_k < 2^48 and m_k < 2^64;
            // k = 5, 6: the 32-bit halves of V_k in two 64-bit sums (m_k < 2^81).
            const uint64_t* Vr = V + rr * Cb + a;
            uint64_t s1 = 0, s2 = 0, s3 = 0, s4 = 0;
            uint64_t lo5 = 0, hi5 = 0, lo6 = 0, hi6 = 0;
#pragma unroll 2
            for (int t = 0; t <= 2 * r; ++t) {
                const uint32_t g = T.g[t];
                s1 += (uint64_t)g * (uint32_t)Vr[t];
                if constexpr (K >= 2) s2 += (uint64_t)g * (uint32_t)Vr[plane + t];
                if constexpr (K >= 3) mac_u64(s3, g, Vr[2 * plane + t]);
                if constexpr (K >= 4) mac_u64(s4, g, Vr[3 * plane + t]);
                if constexpr (K >= 5) {
                    const uint64_t v5 = Vr[4 * plane + t];
                    lo5 += (uint64_t)g * (uint32_t)v5;
                    hi5 += (uint64_t)g * (uint32_t)(v5 >> 32);
                }
                if constexpr (K >= 6) {
                    const uint64_t v6 = Vr[5 * plane + t];
                    lo6 += (uint64_t)g * (uint32_t)v6;
                    hi6 += (uint64_t)g * (uint32_t)(v6 >> 32);
                }
            }
            m[1] = (u128)s1;
            if constexpr (K >= 2) m[2] = (u128)s2;
            if constexpr (K >= 3) m[3] = (u128)s3;
            if constexpr (K >= 4) m[4] = (u128)s4;
            if constexpr (K >= 5) m[5] = (u128)lo5 + ((u128)hi5 << 32);
            if constexpr (K >= 6) m[6] = (u128)lo6 + ((u128)hi6 << 32);
        };

        // 2. Horizontal pass: warp `warp` owns chunk row `warp`.
        {
            const int rr = warp;
            const int Y = y0 + r0 + rr;
            if (lane_blocks) {
                warp_lane_blocks<true>(vmin + rr * Cb, pmin + rr * Cb, ltmin + rr * kLaneTable, Cb, lane);
                warp_lane_blocks<false>(vmax + rr * Cb, pmax + rr * Cb, ltmax + rr * kLaneTable, Cb, lane);
            } else {
                warp_sparse_row<true>(vmin + rr * Cb, Cb, levels, lane);
                warp_sparse_row<false>(vmax + rr * Cb, Cb, levels, lane);
            }
            if (Y < J.H) sep_row_pixels<N, PREC>(P, stats, rr, Y, x0, s_maps, redo_n, redo_list, lane);
        }
        if constexpr (PREC != kPrecFP64) {
            // 3. The queued pixels on the FP64 path, packed into full warps.
            __syncthreads();
            sep_redo_pass<N, PREC>(P, stats, y0 + r0, x0, s_maps, redo_n, redo_list);
        }
        __syncthreads();
    }
}

template <int N, int PREC>
__global__ void __launch_bounds__(kThreads, MinBlocks<PREC>::value)
    fabf_sep_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SepParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t phase = 0;
    if (p.job.use_tma) mbar_init(reinterpret_cast<uint64_t*>(smem));
    sep_tile<N, PREC>(&tmap, p, blockIdx.x, blockIdx.y, smem, phase);
}

// Brute-force adaptive bilateral filter, Eqs. (1)-(3), with the separable
// kernel on the clipped window (O(r^2) per pixel); Real = double or float.
template <typename Real>
__global__ void __launch_bounds__(256)
    bruteforce_sep_kernel(const uint8_t* img, long long pitch, const float* theta, const float* sigma, int H, int W,
                          const __grid_constant__ SepTaps taps, void* out, int out_f64)
{
    const int X = blockIdx.x * 32 + (threadIdx.x & 31);
    const int Y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (X >= W || Y >= H) return;
    const int r = taps.r;
    const long long pix = (long long)Y * W + X;
    const Real th = (Real)theta[pix];
    const Real s = (Real)sigma[pix];
    const Real inv = (Real)-1 / ((Real)2 * s * s);
    Real num = 0, den = 0;
    const int y0 = max(Y - r, 0), y1 = min(Y + r, H - 1);
    const int x0 = max(X - r, 0), x1 = min(X + r, W - 1);
    for (int yy = y0; yy <= y1; ++yy) {
        const uint8_t* row = img + (long long)yy * pitch;
        const Real gy = (Real)taps.g[yy - Y + r];
        for (int xx = x0; xx <= x1; ++xx) {
            const Real v = (Real)row[xx];
            const Real dv = v - th;
            const Real w = gy * (Real)taps.g[xx - X + r] * exp(dv * dv * inv);
            num += w * v;
            den += w;
        }
    }
    const Real g = num / den;
    if (out_f64) static_cast<double*>(out)[pix] = (double)g;
    else static_cast<float*>(out)[pix] = (float)g;
}

constexpr int kSepMaxDynSmem = 110 * 1024;   // >= sep_smem_bytes for every r <= 40, N <= 6, TH <= 40

template <int N, int PREC>
cudaError_t launch_sep_one(const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    const cudaError_t e = set_smem_limit_once<fabf_sep_kernel<N, PREC>>(kSepMaxDynSmem);
    if (e != cudaSuccess) return e;
    fabf_sep_kernel<N, PREC><<<grid, kThreads, smem, s>>>(tm, p);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_sep_impl(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    switch (N) {
    case 0: return launch_sep_one<0, PREC>(tm, p, grid, smem, s);
    case 1: return launch_sep_one<1, PREC>(tm, p, grid, smem, s);
    case 2: return launch_sep_one<2, PREC>(tm, p, grid, smem, s);
    case 3: return launch_sep_one<3, PREC>(tm, p, grid, smem, s);
    case 4: return launch_sep_one<4, PREC>(tm, p, grid, smem, s);
    case 5: return launch_sep_one<5, PREC>(tm, p, grid, smem, s);
    case 6: return launch_sep_one<6, PREC>(tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sep_p0(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_sep_p1(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_sep_p2(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_sep_p3(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);

}  // namespace fabf

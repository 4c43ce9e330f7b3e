// Fast adaptive bilateral filtering with a separable integer spatial kernel
// omega(j) = g[jy + r] g[jx + r] on the window [-r, r]^2 -- the Gaussian of
// Eq. (4) on the paper's window [-3 rho, 3 rho]^2 when the taps are a
// quantised Gaussian (fabf_gaussian_taps) -- plus its brute-force comparator
// and the C ABI entry points of this path.
//
// One CTA (256 threads) produces a TH x 64 output tile, staged like the box
// kernel's (one TMA copy of the tile plus an r-pixel halo, or a plain load):
//  1. Per chunk of 8 output rows, the vertical pass: every (column, row)
//     item forms V_k = sum_t g[t] f(row + t - r, column)^k for k = 1..K by a
//     direct (2r+1)-tap FIR in 32/64-bit integers (exact: V_k < 65535 255^6
//     < 2^64), and each column takes the vertical min / max of the chunk's 8
//     windows from their common core (Eq. (8)).
//  2. Horizontal pass, warp rr on chunk row rr: min / max by one sparse-table
//     level, then for each of the lane's two pixels m_k = sum_t g[t]
//     V_k(column + t - r), exact in 64 bits for k <= 4 and in 128 bits (two
//     64-bit partial sums of the 32-bit halves of V_k) for k = 5, 6; m_0
//     from the tap prefix sums and the clipped window.  Out-of-image pixels
//     are zero in the staged tile, so they add nothing to m_k, k >= 1.
//  3. M_k = sum omega (f - alpha)^k exactly in 128 bits (the recursion of the
//     box path), mu_k = M_k / (beta - alpha)^k with M_k correctly rounded to
//     binary64, and the binary64 tail shared with the box path.
//
// The direct FIR costs O(r) per pixel (the paper's own implementation uses a
// direct convolution for practical rho, Sec. II-D); the binary64 tail still
// dominates the time for every r <= 40.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/fabf.h"
#include "fabf_internal.h"
#include "fabf_kernels.cuh"

namespace fabf {

typedef unsigned __int128 u128;

constexpr uint32_t kTapSumMax = 65535;   // keeps V_k < 2^64 and m_k < 2^81

struct SepTaps {
    int r;
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
    unsigned long long* n_fallback;
    SepDebug dbg;
};

__host__ __device__ inline size_t sep_smem_bytes(int N, int r, int Cb, int TH)
{
    const int K = N < 1 ? 1 : N;
    size_t tile = ((size_t)(TH + 2 * r) * Cb + 127) & ~(size_t)127;
    size_t mm = ((size_t)2 * kChunk * Cb + 15) & ~(size_t)15;
    return 128 + tile + mm + (size_t)K * kChunk * Cb * 8;
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
    return ldexp(__ull2double_rn(top | sticky), s);
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

template <int N>
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
    uint64_t* V = reinterpret_cast<uint64_t*>(vmin + (((size_t)2 * kChunk * Cb + 15) & ~(size_t)15));   // [K][kChunk][Cb]

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

    for (int r0 = 0; r0 < TH; r0 += kChunk) {
        if (y0 + r0 >= J.H) break;                                   // uniform per CTA
        // 1a. Vertical min / max of the 8 windows [rr, rr + 2r] of column c.
        {
            const int c = threadIdx.x;
            const int X = xs + c;
            if (c < Cb) {
                if (X >= 0 && X < J.W) {
                    uint8_t cmin = 255, cmax = 0;
                    {
                        const int a = max(r0 + kChunk - 1, rowlo), b = min(r0 + 2 * r, rowhi);
                        for (int t = a; t <= b; ++t) {
                            const uint8_t v = tile[t * Cb + c];
                            cmin = v < cmin ? v : cmin;
                            cmax = v > cmax ? v : cmax;
                        }
                    }
#pragma unroll
                    for (int rr = 0; rr < kChunk; ++rr) {
                        const int row = r0 + rr;
                        uint8_t mn = cmin, mx = cmax;
                        const int a1 = max(row, rowlo), b1 = min(min(r0 + kChunk - 2, row + 2 * r), rowhi);
                        for (int t = a1; t <= b1; ++t) {
                            const uint8_t v = tile[t * Cb + c];
                            mn = v < mn ? v : mn;
                            mx = v > mx ? v : mx;
                        }
                        const int a2 = max(max(r0 + 2 * r + 1, row), rowlo), b2 = min(row + 2 * r, rowhi);
                        for (int t = a2; t <= b2; ++t) {
                            const uint8_t v = tile[t * Cb + c];
                            mn = v < mn ? v : mn;
                            mx = v > mx ? v : mx;
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
            const int plane = kChunk * Cb;
            Vi[0] = a1;
            if constexpr (K >= 2) Vi[plane] = a2;
            if constexpr (K >= 3) Vi[2 * plane] = a3;
            if constexpr (K >= 4) Vi[3 * plane] = a4;
            if constexpr (K >= 5) Vi[4 * plane] = a5;
            if constexpr (K >= 6) Vi[5 * plane] = a6;
        }
        __syncthreads();

        // 2. Horizontal pass: warp `warp` owns chunk row `warp`.
        {
            const int rr = warp;
            const int Y = y0 + r0 + rr;
            warp_sparse_row<true>(vmin + rr * Cb, Cb, levels, lane);
            warp_sparse_row<false>(vmax + rr * Cb, Cb, levels, lane);
            if (Y < J.H) {
                const int ty0 = max(r - Y, 0), ty1 = min(2 * r, J.H - 1 - Y + r);
                const uint64_t m0y = T.G[ty1 + 1] - T.G[ty0];
#pragma unroll 1
                for (int h = 0; h < kTileW / 32; ++h) {
                    const int x = lane + 32 * h;
                    const int Xo = x0 + x;
                    if (Xo >= J.W) continue;
                    const int a = x + off;                      // tile column of the window's left edge
                    const int alpha = min(vmin[rr * Cb + a], vmin[rr * Cb + a + 2 * r - span + 1]);
                    const int beta = max(vmax[rr * Cb + a], vmax[rr * Cb + a + 2 * r - span + 1]);
                    const int fi = tile[(r0 + rr + r) * Cb + a + r];
                    // Eq. (17): m_k = sum_t g[t] V_k(a + t).
                    u128 m[K + 1];
                    {
                        const int tx0 = max(r - Xo, 0), tx1 = min(2 * r, J.W - 1 - Xo + r);
                        m[0] = (u128)(m0y * (uint64_t)(T.G[tx1 + 1] - T.G[tx0]));
                        const uint64_t* Vr = V + rr * Cb + a;
                        const int plane = kChunk * Cb;
                        // k = 1, 2: V_k < 2^32, one 32x32 -> 64-bit multiply-add;
                        // k = 3, 4: V_k < 2^48 and m_k < 2^64;  k = 5, 6: the
                        // 32-bit halves of V_k in two 64-bit sums (m_k < 2^81).
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
                    }
                    const long long pix = (long long)Y * J.W + Xo;
                    const float th = J.theta[pix], sg = J.sigma[pix];
                    double g;
                    int fb = 0;
                    PixelTrace tr;
                    PixelTrace* trp = P.dbg.mu ? &tr : nullptr;
                    u128 M[K + 1];
                    bool have_M = false;
                    if (!(sg > 0.0f) || !isfinite(sg) || !isfinite(th)) {
                        g = __longlong_as_double(0x7ff8000000000000LL);
                        if (P.status) atomicOr(P.status, kStatusBadInput);
                        trp = nullptr;
                    } else if (alpha == beta) {
                        g = (double)fi;                         // flat window, Sec. II-A
                    } else {
                        const int d = beta - alpha;
                        // Eq. (24) exactly: S(a, b) = S(a+1, b-1) - alpha S(a, b-1)
                        // with S(a, 0) = m_a; every S lies in [0, m_6] < 2^81.
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
                        have_M = true;
                        double mu[K + 1];
                        int64_t dk = 1;
#pragma unroll
                        for (int k = 0; k <= K; ++k) {
                            mu[k] = u128_to_double_rn(M[k]) / (double)dk;
                            dk *= d;
                        }
                        g = fabf_tail_fp64<N>(c_ainv, alpha, d, mu, th, sg, fb, trp);
                        if (fb && P.n_fallback) atomicAdd(P.n_fallback, 1ull);
                    }
                    if (J.out_f64) static_cast<double*>(J.out)[pix] = g;
                    else static_cast<float*>(J.out)[pix] = (float)g;
                    if (P.dbg.alpha) {
                        const SepDebug& D = P.dbg;
                        const long long plane = (long long)J.H * J.W;
                        D.alpha[pix] = (uint8_t)alpha;
                        D.beta[pix] = (uint8_t)beta;
                        for (int k = 0; k <= N; ++k) {
                            D.m[2 * (k * plane + pix)] = (uint64_t)m[k];
                            D.m[2 * (k * plane + pix) + 1] = (uint64_t)(m[k] >> 64);
                        }
                        D.flags[pix] = (alpha == beta ? 1 : 0) | (fb ? 2 : 0);
                        if (trp && have_M) {
                            for (int k = 0; k <= N; ++k) {
                                D.M[2 * (k * plane + pix)] = (uint64_t)M[k];
                                D.M[2 * (k * plane + pix) + 1] = (uint64_t)(M[k] >> 64);
                                D.mu[k * plane + pix] = tr.mu[k];
                                D.c[k * plane + pix] = tr.c[k];
                            }
                            for (int k = 0; k <= N + 1; ++k) D.I[k * plane + pix] = tr.I[k];
                            D.t0lam[pix] = tr.t0;
                            D.t0lam[plane + pix] = tr.lam;
                            D.T[pix] = tr.T1;
                            D.T[plane + pix] = tr.T2;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 2)
    fabf_sep_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SepParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t phase = 0;
    if (p.job.use_tma) mbar_init(reinterpret_cast<uint64_t*>(smem));
    sep_tile<N>(&tmap, p, blockIdx.x, blockIdx.y, smem, phase);
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

template <int N>
static cudaError_t launch_sep_one(const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e =
            cudaFuncSetAttribute(fabf_sep_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSepMaxDynSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    fabf_sep_kernel<N><<<grid, kThreads, smem, s>>>(tm, p);
    return cudaGetLastError();
}

static cudaError_t launch_sep(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    switch (N) {
    case 0: return launch_sep_one<0>(tm, p, grid, smem, s);
    case 1: return launch_sep_one<1>(tm, p, grid, smem, s);
    case 2: return launch_sep_one<2>(tm, p, grid, smem, s);
    case 3: return launch_sep_one<3>(tm, p, grid, smem, s);
    case 4: return launch_sep_one<4>(tm, p, grid, smem, s);
    case 5: return launch_sep_one<5>(tm, p, grid, smem, s);
    case 6: return launch_sep_one<6>(tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

// Checks the taps and fills the kernel's copy (with prefix sums).
static int make_taps(const uint32_t* taps, int r, SepTaps* T)
{
    if (!taps || r < 1) return FABF_EINVAL;
    if (r > kWMax) return FABF_EUNSUPPORTED;
    std::memset(T, 0, sizeof(*T));
    T->r = r;
    uint64_t sum = 0;
    for (int t = 0; t <= 2 * r; ++t) {
        T->g[t] = taps[t];
        T->G[t] = (uint32_t)sum;
        sum += taps[t];
        if (sum > kTapSumMax) return FABF_EUNSUPPORTED;
    }
    T->G[2 * r + 1] = (uint32_t)sum;
    if (taps[r] < 1) return FABF_EINVAL;
    return FABF_OK;
}

static int run_sep(const SepTaps& T, const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
                   int W, int N, void* out, int out_f64, int TH, const SepDebug* dbg, unsigned* status,
                   unsigned long long* nfb, cudaStream_t s)
{
    SepParams p;
    std::memset(&p, 0, sizeof(p));
    CUtensorMap tm;
    (void)make_job(&p.job, &tm, img, pitch, theta, sigma, H, W, T.r, N, out, out_f64, TH);
    p.taps = T;
    p.status = status;
    p.n_fallback = nfb;
    if (dbg) p.dbg = *dbg;
    const size_t smem = sep_smem_bytes(N, T.r, p.job.Cb, TH);
    dim3 grid(p.job.tiles_x, p.job.tiles_y);
    return cuda_status(launch_sep(N, tm, p, grid, smem, s));
}

}  // namespace fabf

using namespace fabf;

extern "C" {

int fabf_gaussian_taps(double rho, uint32_t* taps, int capacity, int* r_out)
{
    if (!taps || !r_out || !(rho > 0.0) || !std::isfinite(rho)) return FABF_EINVAL;
    const double rr = std::ceil(3.0 * rho);
    if (rr > kWMax) return FABF_EUNSUPPORTED;
    const int r = rr < 1.0 ? 1 : (int)rr;
    if (capacity < 2 * r + 1) return FABF_EINVAL;
    for (int t = -r; t <= r; ++t)
        taps[t + r] = (uint32_t)std::floor(1024.0 * std::exp(-(double)(t * t) / (2.0 * rho * rho)) + 0.5);
    *r_out = r;
    return FABF_OK;
}

int fabf_filter_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                    size_t pitch, const uint32_t* taps, int r, int N, void* out, int out_is_f64,
                    void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, r, N);
    if (rc) return rc;
    SepTaps T;
    rc = make_taps(taps, r, &T);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return with_device_buffers(
        ctx, img, theta, sigma, H, W, pitch, out, out_is_f64, s,
        [&](const uint8_t* d_img, size_t d_pitch, const float* d_th, const float* d_sg, void* d_out) {
            // binary64 throughout: the FP64 form's tile rule (8 rows)
            const int TH = tile_rows_for(nullptr, r, N, kPrecFP64, H, W);
            return run_sep(T, d_img, d_pitch, d_th, d_sg, H, W, N, d_out, out_is_f64, TH, nullptr, ctx->d_status,
                           ctx->d_nfb, s);
        });
}

int fabf_debug_stages_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                          size_t pitch, const uint32_t* taps, int r, int N, uint8_t* alpha, uint8_t* beta,
                          uint64_t* m, uint64_t* M, double* mu, double* c, double* t0lam, double* I, double* T,
                          int32_t* flags, double* out)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, r, N);
    if (rc) return rc;
    if (!alpha || !beta || !m || !M || !mu || !c || !t0lam || !I || !T || !flags) return FABF_EINVAL;
    SepTaps tp;
    rc = make_taps(taps, r, &tp);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    SepDebug d{alpha, beta, m, M, mu, c, t0lam, I, T, flags};
    rc = run_sep(tp, img, pitch, theta, sigma, H, W, N, out, 1, kDefaultTileRows, &d, ctx->d_status, ctx->d_nfb, 0);
    if (rc) return rc;
    int st = FABF_OK;
    rc = read_and_clear_status(ctx, 0, &st, nullptr, nullptr);
    return rc ? rc : st;
}

int fabf_bruteforce_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                        size_t pitch, const uint32_t* taps, int r, void* out, int out_is_f64, int use_f64,
                        void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, r, 0);
    if (rc) return rc;
    SepTaps T;
    rc = make_taps(taps, r, &T);
    if (rc) return rc;
    if (!is_device_ptr(img) || !is_device_ptr(theta) || !is_device_ptr(sigma) || !is_device_ptr(out))
        return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    dim3 grid((W + 31) / 32, (H + 7) / 8);
    if (use_f64)
        bruteforce_sep_kernel<double><<<grid, 256, 0, s>>>(img, (long long)pitch, theta, sigma, H, W, T, out,
                                                           out_is_f64);
    else
        bruteforce_sep_kernel<float><<<grid, 256, 0, s>>>(img, (long long)pitch, theta, sigma, H, W, T, out,
                                                          out_is_f64);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"

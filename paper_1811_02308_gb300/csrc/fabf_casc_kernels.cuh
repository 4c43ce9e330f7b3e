// Tiled kernel of fast adaptive bilateral filtering with the separable spatial
// kernel omega(j) = t[jy + r] t[jx + r], t = b * b * b the cascade of three
// boxes b of length n = 2 rb + 1 (radius r = 3 rb, variance rb (rb + 1)
// along each axis): the combination of box kernels the paper cites as the
// way to O(1) Gaussian spatial kernels (Sec. I-A), and the O(1)-in-rho
// convolutions of Sec. II-D.  Every moment stays an exact integer, so the
// result equals the separable path's (direct FIR) on the same taps bit for
// bit.
//
// Why O(1) per pixel: the third difference with step n of the cascade's taps
// is four unit spikes, Delta_n^3 t = delta_0 - 3 delta_n + 3 delta_2n -
// delta_3n (t's support [-r, r] shifted to [0, 3n - 3]).  So the convolution
// of a sequence v with t is the third running (prefix) sum of the sparse
// combination e(a) = v(a) - 3 v(a - n) + 3 v(a - 2n) - v(a - 3n), read at
// the window's last index.  Everything runs in wrapping 64-bit arithmetic:
// the result is exact because the true value fits.
//
// One CTA (256 threads) produces a TH x 64 output tile, staged like the box
// kernel's (one TMA copy of the tile plus an r-pixel halo, or a plain load):
//  1. Vertical phase, thread c < Cb on tile column c: the three running sums
//     U1 += e, U2 += U1, V += U2 of the powers f^k (k = 1..K), kept in
//     shared memory between chunks; each output row costs one step on four
//     bytes of the staged tile.  A tile starts 2r steps above its first
//     output row with zero sums (the rows above the staged tile count as 0,
//     which changes no window of an output row); those 2r steps are taken
//     as one weighted sum per row (weights made on the host).  The vertical window
//     extrema are the box kernel's (16-bit SIMD, threads Cb .. Cb + Cb/2).
//  2. Horizontal phase, warp rr on chunk row rr: e of each V_k row, three
//     warp prefix sums in registers, and m_k = the third prefix sum at the
//     window's last column.  For k = 5, 6 (m_k up to 2^81) the 32-bit halves
//     of V_k run as two chains, each exact in 64 bits.  Window extrema by
//     lane blocks, then the separable path's per-pixel code (exact 128-bit
//     shifted moments, fit, integrals, ratio, the binary32 guard and redo).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fabf_sep_kernels.cuh"

namespace fabf {

constexpr int kCascBoxes = 3;          // boxes in the cascade
constexpr int kCascRbMax = kWMax / kCascBoxes;   // r = 3 rb <= 40

// 64-bit planes of one chunk row set: V_k for k = 1..K, plus the high-half
// chains of k = 5 and 6.
__host__ __device__ constexpr int casc_planes(int K) { return K + (K >= 5 ? 1 : 0) + (K >= 6 ? 1 : 0); }

// Bytes of dynamic shared memory one cascade tile needs: the staged tile,
// the extrema rows, the running sums [3][K][Cb] and the planes
// [planes][kChunk][Cb] (64-bit), the redo list and the maps.
__host__ __device__ inline size_t casc_smem_bytes(int N, int r, int Cb, int TH)
{
    const int K = N < 1 ? 1 : N;
    const size_t tile = ((size_t)(TH + 2 * r) * Cb + 127) & ~(size_t)127;
    const size_t ext = ((size_t)4 * kChunk * Cb + (size_t)2 * kChunk * kLaneTable + 15) & ~(size_t)15;
    const size_t sums = (size_t)3 * K * Cb * 8;
    const size_t planes = (size_t)casc_planes(K) * kChunk * Cb * 8;
    return 128 + tile + ext + sums + planes + kRedoBytes + kMapBytes;
}

// e = p0 - 3 p1 + 3 p2 - p3 (wrapping).
template <typename T>
__device__ __forceinline__ T third_difference(T p0, T p1, T p2, T p3)
{
    return (p0 - p3) + (T)3 * (p2 - p1);
}

// One step of the vertical running sums of column c: the powers of the four
// bytes b0..b3 (tile rows a, a - n, a - 2n, a - 3n) enter e_k, then
// U1 += e, U2 += U1, V += U2 for k = 1..K (k = 1, 2 in 32 bits: V_1, V_2 <
// 27^3 255^2 < 2^32; k >= 3 in 64 bits).
template <int K>
__device__ __forceinline__ void casc_vertical_step(uint32_t (&u32)[3][2], uint64_t (&u64)[3][4], uint32_t b0,
                                                   uint32_t b1, uint32_t b2, uint32_t b3)
{
    const uint32_t q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2, q3 = b3 * b3;
    uint32_t e32[2];
    e32[0] = third_difference<uint32_t>(b0, b1, b2, b3);
    e32[1] = third_difference<uint32_t>(q0, q1, q2, q3);
#pragma unroll
    for (int k = 0; k < (K < 2 ? K : 2); ++k) {
        u32[0][k] += e32[k];
        u32[1][k] += u32[0][k];
        u32[2][k] += u32[1][k];
    }
    if constexpr (K >= 3) {
        const uint32_t c0 = q0 * b0, c1 = q1 * b1, c2 = q2 * b2, c3 = q3 * b3;     // v^3 < 2^24
        uint64_t e64[4];
        e64[0] = third_difference<uint64_t>(c0, c1, c2, c3);
        uint32_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
        if constexpr (K >= 4) {
            d0 = c0 * b0; d1 = c1 * b1; d2 = c2 * b2; d3 = c3 * b3;               // v^4 < 2^32
            e64[1] = third_difference<uint64_t>(d0, d1, d2, d3);
        }
        if constexpr (K >= 5) {
            const uint64_t f0 = (uint64_t)d0 * b0, f1 = (uint64_t)d1 * b1, f2 = (uint64_t)d2 * b2,
                           f3 = (uint64_t)d3 * b3;
            e64[2] = third_difference<uint64_t>(f0, f1, f2, f3);
            if constexpr (K >= 6) e64[3] = third_difference<uint64_t>(f0 * b0, f1 * b1, f2 * b2, f3 * b3);
        }
#pragma unroll
        for (int k = 0; k < K - 2; ++k) {
            u64[0][k] += e64[k];
            u64[1][k] += u64[0][k];
            u64[2][k] += u64[1][k];
        }
    }
}

// The start sums of column c as one weighted sum per tile row: the powers
// of byte b enter U1, U2 and V with the row's weights (w1, w2, w3) (the sums
// after the 2r start-up steps from zero, unrolled; exact in the same
// wrapping arithmetic).
template <int K>
__device__ __forceinline__ void casc_weighted_add(uint32_t (&u32)[3][2], uint64_t (&u64)[3][4], uint32_t b, int w1,
                                                  int w2, int w3)
{
    const int w[3] = {w1, w2, w3};
    const uint32_t q = b * b;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        u32[s][0] += (uint32_t)w[s] * b;
        if constexpr (K >= 2) u32[s][1] += (uint32_t)w[s] * q;
    }
    if constexpr (K >= 3) {
        const uint32_t p3 = q * b;
        const uint32_t p4 = p3 * b;
        const uint64_t p5 = (uint64_t)p4 * b;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const uint64_t ws = (uint64_t)(int64_t)w[s];
            u64[s][0] += ws * p3;
            if constexpr (K >= 4) u64[s][1] += ws * p4;
            if constexpr (K >= 5) u64[s][2] += ws * p5;
            if constexpr (K >= 6) u64[s][3] += ws * (p5 * b);
        }
    }
}

// Inclusive prefix sum over a warp's row held as 5 consecutive values per
// lane (lane l holds columns 5l .. 5l + 4), in wrapping 64-bit arithmetic.
__device__ __forceinline__ void warp_prefix5(uint64_t (&v)[5], int lane)
{
#pragma unroll
    for (int j = 1; j < 5; ++j) v[j] += v[j - 1];
    uint64_t tot = v[4];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, tot, o);
        if (lane >= o) tot += t;
    }
    const uint64_t excl = tot - v[4];
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] += excl;
}

// Horizontal cascade of one chunk row of V_k (Cb <= 160 columns, 64-bit):
// e(c) = V(c) - 3 V(c - n) + 3 V(c - 2n) - V(c - 3n) (V = 0 left of column
// 0), then three prefix sums; the row becomes P3, whose value at column b is
// the cascade sum over the window [b - 2r, b].  Split: the 32-bit halves of
// V run as two chains, P3 of the low halves in `row`, of the high halves in
// `row_hi` (m = lo + hi 2^32).
template <bool Split>
__device__ __forceinline__ void warp_cascade_row(uint64_t* row, uint64_t* row_hi, int Cb, int n, int lane)
{
    uint64_t e[5], eh[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int c = 5 * lane + j;
        e[j] = 0;
        eh[j] = 0;
        if (c < Cb) {
            const uint64_t v0 = row[c];
            const uint64_t v1 = c >= n ? row[c - n] : 0ull;
            const uint64_t v2 = c >= 2 * n ? row[c - 2 * n] : 0ull;
            const uint64_t v3 = c >= 3 * n ? row[c - 3 * n] : 0ull;
            if constexpr (Split) {
                e[j] = third_difference<uint64_t>((uint32_t)v0, (uint32_t)v1, (uint32_t)v2, (uint32_t)v3);
                eh[j] = third_difference<uint64_t>(v0 >> 32, v1 >> 32, v2 >> 32, v3 >> 32);
            } else {
                e[j] = third_difference<uint64_t>(v0, v1, v2, v3);
            }
        }
    }
    __syncwarp();   // every read of the row is done before it is overwritten
#pragma unroll
    for (int s = 0; s < kCascBoxes; ++s) {
        warp_prefix5(e, lane);
        if constexpr (Split) warp_prefix5(eh, lane);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int c = 5 * lane + j;
        if (c < Cb) {
            row[c] = e[j];
            if constexpr (Split) row_hi[c] = eh[j];
        }
    }
    __syncwarp();
}

template <int N, int PREC>
__device__ __forceinline__ void casc_tile(const CUtensorMap* tmap, const SepParams& P, int tx, int ty,
                                          uint8_t* smem, uint32_t& phase)
{
    constexpr int K = N < 1 ? 1 : N;
    const ImageJob& J = P.job;
    const SepTaps& T = P.taps;
    const int r = J.w, Cb = J.Cb, off = J.off, TH = J.TH;
    const int n = T.casc_n;                     // box length; r = 3 (n - 1) / 2
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
    uint64_t* sums = reinterpret_cast<uint64_t*>(
        vmin + (((size_t)4 * kChunk * Cb + (size_t)2 * kChunk * kLaneTable + 15) & ~(size_t)15));   // [3][K][Cb]
    uint64_t* planes = sums + (size_t)3 * K * Cb;                      // [casc_planes(K)][kChunk][Cb]
    unsigned* redo_n = reinterpret_cast<unsigned*>(planes + (size_t)casc_planes(K) * kChunk * Cb);
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
    const int c = threadIdx.x;                                        // vertical phase column
    const bool col_in = c < Cb && xs + c >= 0 && xs + c < J.W;
    int levels = 0;
    while ((2 << levels) <= 2 * r + 1) ++levels;
    const int span = 1 << levels;
    const bool lane_blocks = 2 * r + 1 >= 6;

    // One step of column c with tile row a entering (rows above the tile
    // count as 0; rows outside the image are 0 in the staged tile).
    auto step = [&](uint32_t (&u32)[3][2], uint64_t (&u64)[3][4], int a) {
        const uint8_t* col = tile + c;
        const uint32_t b0 = col[a * Cb];
        const uint32_t b1 = a >= n ? col[(a - n) * Cb] : 0u;
        const uint32_t b2 = a >= 2 * n ? col[(a - 2 * n) * Cb] : 0u;
        const uint32_t b3 = a >= 3 * n ? col[(a - 3 * n) * Cb] : 0u;
        casc_vertical_step<K>(u32, u64, b0, b1, b2, b3);
    };
    auto save = [&](const uint32_t (&u32)[3][2], const uint64_t (&u64)[3][4]) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
#pragma unroll
            for (int k = 0; k < K; ++k) sums[(s * K + k) * Cb + c] = k < 2 ? (uint64_t)u32[s][k < 2 ? k : 0]
                                                                             : u64[s][k < 2 ? 0 : k - 2];
        }
    };

    // The sums 2r steps after zero sums above output row 0 (tile rows 0 ..
    // 2r - 1 entered), as one weighted sum per row.
    if (col_in) {
        uint32_t u32[3][2] = {};
        uint64_t u64[3][4] = {};
#pragma unroll 2
        for (int a = 0; a < 2 * r; ++a)
            casc_weighted_add<K>(u32, u64, tile[a * Cb + c], T.pre_w[0][a], T.pre_w[1][a], T.pre_w[2][a]);
        save(u32, u64);
    }

    for (int r0 = 0; r0 < TH; r0 += kChunk) {
        if (y0 + r0 >= J.H) break;                                   // uniform per CTA
        if (threadIdx.x == 0) *redo_n = 0u;
        prefetch_maps(J, s_maps, y0 + r0, x0, maps16);
        // 1a. Running sums of column c: output row r0 + rr takes tile row
        //     r0 + rr + 2r; V_k of the window [r0 + rr, r0 + rr + 2r] into
        //     the planes.
        if (c < Cb) {
            if (col_in) {
                uint32_t u32[3][2];
                uint64_t u64[3][4];
#pragma unroll
                for (int s = 0; s < 3; ++s) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const uint64_t v = sums[(s * K + k) * Cb + c];
                        if (k < 2) u32[s][k < 2 ? k : 0] = (uint32_t)v;
                        else u64[s][k < 2 ? 0 : k - 2] = v;
                    }
                }
#pragma unroll 2
                for (int rr = 0; rr < kChunk; ++rr) {
                    step(u32, u64, r0 + rr + 2 * r);
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        planes[(k * kChunk + rr) * Cb + c] = k < 2 ? (uint64_t)u32[2][k < 2 ? k : 0]
                                                                   : u64[2][k < 2 ? 0 : k - 2];
                }
                save(u32, u64);
            } else {
#pragma unroll
                for (int rr = 0; rr < kChunk; ++rr) {
#pragma unroll
                    for (int k = 0; k < K; ++k) planes[(k * kChunk + rr) * Cb + c] = 0ull;
                }
            }
        }
        // 1b. Vertical window extrema (threads Cb .. Cb + Cb/2 - 1).
        vertical_extrema_simd(tile, vmin, vmax, Cb, xs, J.W, r0, r, rowlo, rowhi);
        cp_async_wait_all();
        __syncthreads();

        // Window statistics of the pixel at chunk row rr, tile column x (the
        // chunk's rows are third prefix sums and lane blocks by now).
        auto stats = [&](int rr, int x, int& alpha, int& beta, u128 (&m)[K + 1], int& fi) {
            const int Y = y0 + r0 + rr, Xo = x0 + x;
            const int a = x + off, b = a + 2 * r;       // tile columns of the window
            if (lane_blocks) {
                alpha = lane_block_query<true>(vmin + rr * Cb, pmin + rr * Cb, ltmin + rr * kLaneTable, a, b);
                beta = lane_block_query<false>(vmax + rr * Cb, pmax + rr * Cb, ltmax + rr * kLaneTable, a, b);
            } else {
                alpha = min(vmin[rr * Cb + a], vmin[rr * Cb + b - span + 1]);
                beta = max(vmax[rr * Cb + a], vmax[rr * Cb + b - span + 1]);
            }
            fi = tile[(r0 + rr + r) * Cb + a + r];
            const int ty0 = max(r - Y, 0), ty1 = min(2 * r, J.H - 1 - Y + r);
            const int tx0 = max(r - Xo, 0), tx1 = min(2 * r, J.W - 1 - Xo + r);
            m[0] = (u128)((uint64_t)(T.G[ty1 + 1] - T.G[ty0]) * (uint64_t)(T.G[tx1 + 1] - T.G[tx0]));
            // Eq. (17) with the cascade's weights: m_k = P3_k at column b
            // (m_k < 2^64 for k <= 4; lo + hi 2^32 for k = 5, 6)
#pragma unroll
            for (int k = 1; k <= K; ++k) {
                const uint64_t lo = planes[((k - 1) * kChunk + rr) * Cb + b];
                if (k <= 4) {
                    m[k] = (u128)lo;
                } else {
                    const uint64_t hi = planes[((K + k - 5) * kChunk + rr) * Cb + b];
                    m[k] = (u128)lo + ((u128)hi << 32);
                }
            }
        };

        // 2. Horizontal phase: warp `warp` owns chunk row `warp`.
        {
            const int rr = warp;
            const int Y = y0 + r0 + rr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                uint64_t* row = planes + (k * kChunk + rr) * Cb;
                if (k >= 4) warp_cascade_row<true>(row, planes + ((K + k - 4) * kChunk + rr) * Cb, Cb, n, lane);
                else warp_cascade_row<false>(row, nullptr, Cb, n, lane);
            }
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

// Registers: the cascade tile's shared memory leaves at most 3 CTAs per SM
// (2 for the FP64 form, which the FP64 pipe bounds), so the binary32 forms
// are compiled for 3 (85 registers) rather than the box kernel's 4.
template <int PREC>
struct CascMinBlocks {
    static constexpr int value = PREC == kPrecFP64 ? 2 : 3;
};

template <int N, int PREC>
__global__ void __launch_bounds__(kThreads, CascMinBlocks<PREC>::value)
    fabf_casc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SepParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t phase = 0;
    if (p.job.use_tma) mbar_init(reinterpret_cast<uint64_t*>(smem));
    casc_tile<N, PREC>(&tmap, p, blockIdx.x, blockIdx.y, smem, phase);
}

constexpr int kCascMaxDynSmem = 160 * 1024;   // >= casc_smem_bytes for every rb <= 13, N <= 6, TH <= 64

template <int N, int PREC>
cudaError_t launch_casc_one(const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    const cudaError_t e = set_smem_limit_once<fabf_casc_kernel<N, PREC>>(kCascMaxDynSmem);
    if (e != cudaSuccess) return e;
    fabf_casc_kernel<N, PREC><<<grid, kThreads, smem, s>>>(tm, p);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_casc_impl(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem,
                             cudaStream_t s)
{
    switch (N) {
    case 0: return launch_casc_one<0, PREC>(tm, p, grid, smem, s);
    case 1: return launch_casc_one<1, PREC>(tm, p, grid, smem, s);
    case 2: return launch_casc_one<2, PREC>(tm, p, grid, smem, s);
    case 3: return launch_casc_one<3, PREC>(tm, p, grid, smem, s);
    case 4: return launch_casc_one<4, PREC>(tm, p, grid, smem, s);
    case 5: return launch_casc_one<5, PREC>(tm, p, grid, smem, s);
    case 6: return launch_casc_one<6, PREC>(tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_casc_p0(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_casc_p1(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_casc_p2(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_casc_p3(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s);

}  // namespace fabf

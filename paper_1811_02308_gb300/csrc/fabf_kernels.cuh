// Tiled kernels of fast adaptive bilateral filtering (Algorithm 1, Sec. II-D
// of Gavaskar & Chaudhury) for 8-bit images with a box spatial kernel of
// radius w, plus the test-only kernels that share their device code.
//
// One CTA (256 threads, 8 warps) produces a TH x 64 output tile (TH a
// multiple of 8 up to 64, chosen per (w, N, precision) by the autotuner):
//  1. The input tile plus a w-pixel halo is staged in shared memory with one
//     TMA tensor copy (cp.async.bulk.tensor.2d completing on an mbarrier,
//     bounded wait); the copy starts at a 16-byte aligned column, so the
//     tile carries a constant column offset off = (-w) mod 16.  Out-of-image
//     bytes read as 0.  Images whose base or pitch are not 16-byte aligned
//     take a plain cooperative load into the same layout.
//  2. Output rows are processed in chunks of 8.  Vertical phase: thread c
//     owns tile column c; it keeps running window sums of f^k (k = 1..N,
//     Eq. (17) with omega == 1, rows clipped to the image) in registers
//     across chunks (add the entering row, subtract the leaving row), and
//     takes the vertical min / max of the 8 windows of a chunk as suffix
//     extrema of the chunk's own 8 rows combined with prefix extrema of the
//     rows below, 2w + 8 row visits per chunk (Eq. (8)).
//  3. Horizontal phase: warp r owns chunk row r.  It turns each vertical
//     sum row into a prefix sum (window sums are differences of two
//     prefixes and fit in int64), and each min / max row into lane blocks
//     of 5 entries (in-lane suffix and prefix extrema plus a table over 2^k
//     consecutive lanes), so a window's min / max takes four lookups; for
//     w <= 2 a sparse-table level of width 2^floor(log2(2w+1)) instead.  Each lane then finishes two
//     pixels (fabf_device.cuh): m_0 from the clipped window geometry, the
//     exact shifted moments, the fit, the integrals and the ratio.
//
// The single-image kernel runs one tile per CTA.  The batch kernel is
// persistent: each CTA pops tiles of many images (any sizes, w and N) from a
// device counter until the work list is exhausted.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "fabf_device.cuh"

namespace fabf {

constexpr int kTileW = 64;
constexpr int kTileHMax = 64;
constexpr int kChunk = 8;
constexpr int kThreads = 256;
constexpr unsigned kTmaWaitLimit = 1u << 22;   // bounded mbarrier wait (polls)

// Per-chunk list of pixels the binary32 forms hand to the FP64 path: a count
// and one 16-bit (row, column) entry per pixel of the chunk.
constexpr size_t kRedoBytes = 16 + 2 * kChunk * kTileW;

// The chunk's centres and widths (theta, sigma), prefetched into shared memory.
constexpr size_t kMapBytes = 2 * kChunk * kTileW * sizeof(float);

// Lane-block extrema table of one row: levels k = 0..4 x 32 lanes (bytes).
constexpr int kLaneTable = 5 * 32;

constexpr int kPrecFP64 = 0;          // FABF_FP64
constexpr int kPrecFP64Fit = 1;       // FABF_FP64FIT_FP32REC
constexpr int kPrecCFP32 = 2;         // FABF_CFP32
constexpr int kPrecC32 = 3;           // FABF_C32

struct DebugPlanes {       // per-stage exports for the parity tests (all optional)
    uint8_t* alpha;        // H x W
    uint8_t* beta;         // H x W
    int64_t* m;            // (N+1) x H x W
    int64_t* M;            // (N+1) x H x W
    double* mu;            // (N+1) x H x W
    double* c;             // (N+1) x H x W
    double* t0lam;         // 2 x H x W
    double* I;             // (N+2) x H x W
    double* T;             // 2 x H x W
    int32_t* flags;        // H x W: bit0 flat window, bit1 fallback taken
};

// One image of a launch.
struct ImageJob {
    const uint8_t* img;
    long long pitch;       // bytes between image rows
    const float* theta;    // H x W, row stride W
    const float* sigma;    // H x W, row stride W
    void* out;             // H x W float64 or float32, row stride W
    int H, W, w, N;
    int out_f64;
    int use_tma;
    int off;               // (-w) mod 16: tile column of image column x0 - w
    int Cb;                // tile row length in shared memory (multiple of 16)
    int TH;                // output rows per tile (multiple of 8, <= 64)
    int tiles_x, tiles_y;
    long long tile_begin;  // index of this image's first tile in the launch
    int tile_y0;           // single-image launches: tile row of blockIdx.y == 0 (a band of rows)
    int maps_host;         // theta / sigma are host memory read over the chip-to-chip link
};

struct FusedParams {
    ImageJob job;
    unsigned* status;                  // OR of kStatus* bits (may be null)
    unsigned long long* n_fallback;    // pixels that took the fallback (may be null)
    DebugPlanes dbg;
};

struct BatchParams {
    const ImageJob* jobs;              // njobs, sorted by tile_begin
    const CUtensorMap* tmaps;          // one per job (64-byte aligned, global memory)
    int njobs;
    long long total_tiles;
    unsigned long long* next_tile;     // work counter, zero at launch
    unsigned* status;
    unsigned long long* n_fallback;
};

// Bytes of dynamic shared memory one tile needs.
__host__ __device__ inline size_t fused_smem_bytes(int N, int w, int Cb, int TH)
{
    const int R = TH + 2 * w;
    size_t tile = (size_t)R * Cb;
    tile = (tile + 127) & ~(size_t)127;
    const int K = N < 1 ? 1 : N;               // k = 1 is kept even for N = 0
    const int n32 = K < 2 ? K : 2;
    const int n64 = K > 2 ? K - 2 : 0;
    size_t v = (size_t)kChunk * Cb * (4 + 4 * n32) + (size_t)2 * kChunk * kLaneTable + (size_t)kChunk * Cb * 8 * n64;
    return 128 + tile + ((v + 15) & ~(size_t)15) + kRedoBytes + kMapBytes;
}

// Raise a kernel's dynamic shared-memory limit once per device and kernel
// (the attribute is per device; the flags are set after a successful call,
// and a race only repeats the call).
template <auto Kernel>
inline cudaError_t set_smem_limit_once(int bytes)
{
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> done[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) done[dev].store(true, std::memory_order_release);
    return e;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// Tile staging.
// ---------------------------------------------------------------------------
// Asynchronous 4-byte copy global -> shared (no register holds the value in
// flight); commit closes the group, wait_all waits for this thread's groups.
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// theta / sigma rows of device memory go in 16-byte pieces when every piece
// is aligned (W a multiple of 4 and both bases 16-byte aligned; tile columns
// start at multiples of 64; W a multiple of 4 also keeps every piece of an
// in-image start in the row).  Host memory is read in 4-byte pieces,
// measured faster over the chip-to-chip link.
__device__ __forceinline__ bool maps_in_16(const ImageJob& J)
{
    return !J.maps_host && (J.W & 3) == 0 &&
           ((reinterpret_cast<uintptr_t>(J.theta) | reinterpret_cast<uintptr_t>(J.sigma)) & 15) == 0;
}

// theta and sigma of image rows Y0 .. Y0 + kChunk - 1, columns x0 .. x0 +
// kTileW - 1, into s_maps[2][kChunk][kTileW] with cp.async (one committed
// group; the caller waits with cp_async_wait_all before reading).
__device__ __forceinline__ void prefetch_maps(const ImageJob& J, float* s_maps, int Y0, int x0, bool maps16)
{
    if (maps16) {
        // 16-byte pieces: 2 maps x kChunk rows x kTileW / 4 pieces
        for (int i = threadIdx.x; i < 2 * kChunk * (kTileW / 4); i += kThreads) {
            const int which = i >= kChunk * (kTileW / 4) ? 1 : 0;
            const int e = i - which * kChunk * (kTileW / 4);
            const int rr = e / (kTileW / 4), x = 4 * (e - rr * (kTileW / 4));
            const int Y = Y0 + rr, Xo = x0 + x;
            if (Y < J.H && Xo < J.W)
                cp_async16(s_maps + (which * kChunk + rr) * kTileW + x,
                           (which ? J.sigma : J.theta) + (long long)Y * J.W + Xo);
        }
    } else {
        for (int i = threadIdx.x; i < 2 * kChunk * kTileW; i += kThreads) {
            const int which = i >= kChunk * kTileW ? 1 : 0;
            const int e = i - which * kChunk * kTileW;
            const int rr = e / kTileW, x = e - rr * kTileW;
            const int Y = Y0 + rr, Xo = x0 + x;
            if (Y < J.H && Xo < J.W) cp_async4(s_maps + i, (which ? J.sigma : J.theta) + (long long)Y * J.W + Xo);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// One TMA copy of `bytes` into dst; waits (bounded) on phase `phase` of bar.
// Returns false in every thread if the copy did not complete.
__device__ __forceinline__ bool tma_load_tile(const CUtensorMap* tmap, uint8_t* dst, uint64_t* bar, int xs,
                                              int ys, uint32_t bytes, uint32_t phase)
{
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
        // order this CTA's earlier generic accesses of dst before the async write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
            "l"(reinterpret_cast<uint64_t>(tmap)), "r"(xs), "r"(ys), "r"(b)
            : "memory");
    }
    uint32_t done = 0;
    for (unsigned it = 0; it < kTmaWaitLimit; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(phase)
            : "memory");
        if (done) break;
    }
    return __syncthreads_or(done == 0) == 0;   // every thread takes the same decision
}

__device__ __forceinline__ void plain_load_tile(const ImageJob& J, uint8_t* dst, int xs, int ys, int R)
{
    const int total = R * J.Cb;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int t = i / J.Cb, c = i - t * J.Cb;
        const int Y = ys + t, X = xs + c;
        uint8_t v = 0;
        if (Y >= 0 && Y < J.H && X >= 0 && X < J.W) v = J.img[(long long)Y * J.pitch + X];
        dst[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Warp helpers for the horizontal phase (row length Cb <= 160 = 32 lanes x 5).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void warp_prefix_row(T* row, int Cb, int lane)
{
    T v[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int c = 5 * lane + j;
        v[j] = c < Cb ? row[c] : (T)0;
    }
#pragma unroll
    for (int j = 1; j < 5; ++j) v[j] += v[j - 1];
    T tot = v[4];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, tot, o);
        if (lane >= o) tot += t;
    }
    const T excl = tot - v[4];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int c = 5 * lane + j;
        if (c < Cb) row[c] = v[j] + excl;
    }
    __syncwarp();
}

// In-place sparse-table levels 1..levels of min (IsMin) or max over a row.
template <bool IsMin>
__device__ __forceinline__ void warp_sparse_row(uint8_t* row, int Cb, int levels, int lane)
{
    for (int j = 1; j <= levels; ++j) {
        const int h = 1 << (j - 1);
        uint8_t nv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int c = 5 * lane + q;
            uint8_t a = c < Cb ? row[c] : 0;
            if (c + h < Cb) {
                const uint8_t b = row[c + h];
                a = IsMin ? (a < b ? a : b) : (a > b ? a : b);
            }
            nv[q] = a;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int c = 5 * lane + q;
            if (c < Cb) row[c] = nv[q];
        }
        __syncwarp();
    }
}

// Window extrema of a row by lane blocks (Eq. (8), horizontal part).  Lane l
// owns entries 5l .. 5l+4 (Cb <= 160).  The row is overwritten with in-lane
// suffix extrema, `pre` receives in-lane prefix extrema and `lt` the extrema
// of 2^k consecutive lanes' blocks (k = 0..4).  A window [a, e] of at least
// 6 entries spans two or more lanes: the rest of a's lane, whole lanes
// strictly between (two overlapping table entries) and the start of e's lane.
template <bool IsMin>
__device__ __forceinline__ void warp_lane_blocks(uint8_t* row, uint8_t* pre, uint8_t* lt, int Cb, int lane)
{
    const uint8_t id = IsMin ? 255 : 0;
    uint8_t v[5], sfx[5], pfx[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int c = 5 * lane + q;
        v[q] = c < Cb ? row[c] : id;
    }
    uint8_t acc = id;
#pragma unroll
    for (int q = 4; q >= 0; --q) {
        acc = IsMin ? (v[q] < acc ? v[q] : acc) : (v[q] > acc ? v[q] : acc);
        sfx[q] = acc;
    }
    acc = id;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        acc = IsMin ? (v[q] < acc ? v[q] : acc) : (v[q] > acc ? v[q] : acc);
        pfx[q] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int c = 5 * lane + q;
        if (c < Cb) {
            row[c] = sfx[q];
            pre[c] = pfx[q];
        }
    }
    uint32_t t = pfx[4];
    lt[lane] = (uint8_t)t;
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        const int h = 1 << (k - 1);
        const uint32_t u = __shfl_down_sync(0xffffffffu, t, h);
        if (lane + h < 32) t = IsMin ? (u < t ? u : t) : (u > t ? u : t);
        lt[k * 32 + lane] = (uint8_t)t;
    }
    __syncwarp();
}

// Extremum of row entries [a, e] (e - a >= 5) from the lane-block arrays.
template <bool IsMin>
__device__ __forceinline__ int lane_block_query(const uint8_t* row, const uint8_t* pre, const uint8_t* lt, int a, int e)
{
    const int la = (a * 205) >> 10, le = (e * 205) >> 10;     // a / 5, e / 5 for a, e < 1000
    int r = IsMin ? min((int)row[a], (int)pre[e]) : max((int)row[a], (int)pre[e]);
    const int n = le - la - 1;                                  // whole lanes strictly inside
    if (n > 0) {
        const int k = 31 - __clz(n);
        const int u = lt[k * 32 + la + 1], v = lt[k * 32 + le - (1 << k)];
        r = IsMin ? min(r, min(u, v)) : max(r, max(u, v));
    }
    return r;
}

// Vertical min / max of the kChunk windows [r0 + rr, r0 + rr + 2w] (rows
// clipped to [rowlo, rowhi]) of every tile column, into the chunk's vmin /
// vmax rows, four columns per thread: the bytes of tile columns 4g .. 4g+3
// are one 32-bit word, split into two words of 16-bit lanes (bytes 0, 2 and
// bytes 1, 3) that the native 16-bit SIMD minimum combines.  Thread Cb + 2g
// takes the minima of group g and thread Cb + 2g + 1 the maxima, as minima
// of the complemented bytes (255 - v reverses the order), so the two run the
// same instructions; these are the threads the running sums of columns
// 0 .. Cb-1 leave idle (Cb / 2 <= 256 - Cb for Cb <= 160).  Columns outside
// the image (xs + c outside [0, W)) get 255 / 0.
__device__ __forceinline__ void vertical_extrema_simd(const uint8_t* tile, uint8_t* vmin, uint8_t* vmax, int Cb,
                                                      int xs, int W, int r0, int w, int rowlo, int rowhi)
{
    const int e = (int)threadIdx.x - Cb;
    if (e >= 0 && e < (Cb >> 1)) {
        const int g4 = 4 * (e >> 1);
        const uint32_t inv = (e & 1) ? 0xFFFFFFFFu : 0u;   // maxima: complemented bytes
        // bytes of columns outside the image take the identity (the
        // staged tile holds 0 there)
        uint32_t outside = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int Xe = xs + g4 + j;
            if (Xe < 0 || Xe >= W) outside |= 0xFFu << (8 * j);
        }
        const uint32_t* tw = reinterpret_cast<const uint32_t*>(tile) + (g4 >> 2);
        uint32_t* vw = reinterpret_cast<uint32_t*>((e & 1) ? vmax : vmin) + (g4 >> 2);
        const int Cw = Cb >> 2;                     // words per tile row
        // running minima as (even bytes, odd bytes) in 16-bit lanes
        auto add = [&](uint32_t& m0, uint32_t& m1, int t) {
            const uint32_t v = tw[t * Cw] ^ inv;
            m0 = __vminu2(m0, __byte_perm(v, 0u, 0x4240));
            m1 = __vminu2(m1, __byte_perm(v, 0u, 0x4341));
        };
        constexpr uint32_t kId = 0x00FF00FFu;
        // Window of chunk row rr: tile rows [r0 + rr, r0 + rr + 2w]
        // = [r0 + rr, r0 + 7] u [r0 + 8, r0 + rr + 2w] (2w + 1 >= 8,
        // i.e. w >= 4): suffix extrema of the chunk's own rows, then
        // prefix extrema from r0 + 8 that grow by one row per rr --
        // 2w + 8 row visits per chunk.  For w < 4 every window is
        // visited directly (2w + 1 < 8 rows).  The suffix extrema
        // wait in this thread's own words of the shared rows.
        const bool split = 2 * w + 1 >= kChunk;
        uint32_t q0 = kId, q1 = kId;
        if (split) {
            uint32_t s0 = kId, s1 = kId;
#pragma unroll
            for (int rr = kChunk - 1; rr >= 0; --rr) {
                const int t = r0 + rr;
                if (t >= rowlo && t <= rowhi) add(s0, s1, t);
                vw[rr * Cw] = __byte_perm(s0, s1, 0x6240);
            }
            // rows r0 + 8 .. r0 + 2w in two independent chains
            const int a = max(r0 + kChunk, rowlo), b = min(r0 + 2 * w, rowhi);
            uint32_t p0 = kId, p1 = kId;
            int t = a;
            for (; t + 1 <= b; t += 2) {
                add(q0, q1, t);
                add(p0, p1, t + 1);
            }
            if (t <= b) add(q0, q1, t);
            q0 = __vminu2(q0, p0);
            q1 = __vminu2(q1, p1);
        }
#pragma unroll
        for (int rr = 0; rr < kChunk; ++rr) {
            const int r = r0 + rr;
            uint32_t m0, m1;
            if (split) {
                const int t = r + 2 * w;            // the row entering the prefix part
                if (rr > 0 && t >= rowlo && t <= rowhi) add(q0, q1, t);
                const uint32_t sv = vw[rr * Cw];
                m0 = __vminu2(q0, __byte_perm(sv, 0u, 0x4240));
                m1 = __vminu2(q1, __byte_perm(sv, 0u, 0x4341));
            } else {
                m0 = kId;
                m1 = kId;
                const int a = max(r, rowlo), b = min(r + 2 * w, rowhi);
                for (int t = a; t <= b; ++t) add(m0, m1, t);
            }
            // back from the complement for the maxima; outside
            // columns get 255 (minima) or 0 (maxima)
            vw[rr * Cw] = ((__byte_perm(m0, m1, 0x6240) | outside) ^ inv);
        }
    }
}

// Add (Sign = +1) or subtract (Sign = -1) the powers v^1..v^K of one pixel to
// the running window sums: k = 1, 2 in 32 bits, k >= 3 in 64 bits.  v^2..v^4
// are exact in 32 bits (255^4 < 2^32), v^5 takes one widening multiply.
template <int K, int Sign>
__device__ __forceinline__ void add_powers(uint32_t (&s32)[2], uint64_t (&s64)[4], uint32_t v)
{
    const uint32_t v2 = v * v;
    const uint32_t v3 = v2 * v;
    const uint32_t v4 = v3 * v;
    if constexpr (Sign > 0) {
        s32[0] += v;
        if constexpr (K >= 2) s32[1] += v2;
        if constexpr (K >= 3) s64[0] += v3;
        if constexpr (K >= 4) s64[1] += v4;
        if constexpr (K >= 5) {
            const uint64_t v5 = (uint64_t)v4 * v;
            s64[2] += v5;
            if constexpr (K >= 6) s64[3] += v5 * v;
        }
    } else {
        s32[0] -= v;
        if constexpr (K >= 2) s32[1] -= v2;
        if constexpr (K >= 3) s64[0] -= v3;
        if constexpr (K >= 4) s64[1] -= v4;
        if constexpr (K >= 5) {
            const uint64_t v5 = (uint64_t)v4 * v;
            s64[2] -= v5;
            if constexpr (K >= 6) s64[3] -= v5 * v;
        }
    }
}

// ---------------------------------------------------------------------------
// One output tile (tx, ty) of image J.  smem must hold fused_smem_bytes();
// its first 8 bytes are the CTA's mbarrier (initialised by the caller when
// J.use_tma).  Returns false if the tile copy timed out (status already set).
// ---------------------------------------------------------------------------
template <int N, int PREC>
__device__ __forceinline__ bool fabf_tile(const CUtensorMap* tmap, const ImageJob& J, int tx, int ty,
                                          uint8_t* smem, uint32_t& phase, unsigned* status,
                                          unsigned long long* n_fallback, const DebugPlanes& dbg)
{
    // pixels recomputed on the FP64 path by the binary32 forms' guard: the
    // word after the fallback counter
    unsigned long long* redo_count = n_fallback ? n_fallback + 1 : nullptr;
    constexpr int K = N < 1 ? 1 : N;           // power sums kept: k = 1..K
    constexpr int n32 = K < 2 ? K : 2;         // k = 1, 2 in 32 bits
    constexpr int n64 = K > 2 ? K - 2 : 0;     // k = 3..K in 64 bits

    const int w = J.w, Cb = J.Cb, off = J.off, TH = J.TH;
    const int R = TH + 2 * w;
    const int x0 = tx * kTileW, y0 = ty * TH;
    const int xs = x0 - w - off;               // image column of tile column 0
    const int ys = y0 - w;                     // image row of tile row 0

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint8_t* tile = smem + 128;
    const size_t tile_bytes = ((size_t)R * Cb + 127) & ~(size_t)127;
    uint8_t* vmin = tile + tile_bytes;
    uint8_t* vmax = vmin + kChunk * Cb;
    uint8_t* pmin = vmax + kChunk * Cb;                                 // in-lane prefix extrema
    uint8_t* pmax = pmin + kChunk * Cb;
    uint8_t* ltmin = pmax + kChunk * Cb;                                // [kChunk][kLaneTable]
    uint8_t* ltmax = ltmin + kChunk * kLaneTable;
    uint32_t* v32 = reinterpret_cast<uint32_t*>(ltmax + kChunk * kLaneTable);   // [n32][kChunk][Cb]
    const size_t v32_bytes = (size_t)n32 * kChunk * Cb * 4;
    uint64_t* v64 = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(v32) +
                                                ((v32_bytes + 7) & ~(size_t)7));   // [n64][kChunk][Cb]
    const size_t v_bytes = (size_t)kChunk * Cb * (4 + 4 * n32) + (size_t)2 * kChunk * kLaneTable +
                           (size_t)kChunk * Cb * 8 * n64;
    unsigned* redo_n = reinterpret_cast<unsigned*>(vmin + ((v_bytes + 15) & ~(size_t)15));
    uint16_t* redo_list = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(redo_n) + 16);
    float* s_maps = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(redo_n) + kRedoBytes);   // [2][kChunk][kTileW]

    // 1. Stage tile + halo.
    if (J.use_tma) {
        const bool ok = tma_load_tile(tmap, tile, bar, xs, ys, (uint32_t)(R * Cb), phase);
        phase ^= 1u;
        if (!ok) {
            if (threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
            return false;
        }
    } else {
        plain_load_tile(J, tile, xs, ys, R);
        __syncthreads();
    }

    const int rowlo = ys < 0 ? -ys : 0;                           // first in-image tile row
    const int rowhi = min(R - 1, J.H - 1 - ys);                    // last in-image tile row
    const int c = threadIdx.x;                                     // vertical phase column
    const int X = xs + c;
    const bool col_in = (c < Cb) && X >= 0 && X < J.W;

    // Running vertical sums for column c, initialised for output row 0.
    uint32_t s32[2] = {0u, 0u};
    uint64_t s64[4] = {0ull, 0ull, 0ull, 0ull};
    if (col_in) {
        const int t1 = min(2 * w, rowhi);
        for (int t = rowlo; t <= t1; ++t) add_powers<K, +1>(s32, s64, tile[t * Cb + c]);
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int levels = 0;
    while ((2 << levels) <= 2 * w + 1) ++levels;                   // floor(log2(2w+1))
    const int span = 1 << levels;
    const bool lane_blocks = 2 * w + 1 >= 6;                       // else sparse-table levels
    const bool maps16 = maps_in_16(J);

    for (int r0 = 0; r0 < TH; r0 += kChunk) {
        if (y0 + r0 >= J.H) break;                                 // uniform per CTA
        // 2. Vertical phase for output rows r0 .. r0+7.
        if (threadIdx.x == 0) *redo_n = 0u;
        // The chunk's theta and sigma start on their way into shared memory;
        // the vertical phase covers their latency (HBM, or host memory over
        // the chip-to-chip link when the caller's buffers are host-mapped).
        prefetch_maps(J, s_maps, y0 + r0, x0, maps16);
        // 2a. Window sums of column c (threads c < Cb): store, then slide the
        //     window from [r, r+2w] to [r+1, r+2w+1].
        if (c < Cb) {
            if (col_in) {
#pragma unroll
                for (int rr = 0; rr < kChunk; ++rr) {
                    const int r = r0 + rr;
#pragma unroll
                    for (int k = 0; k < n32; ++k) v32[(k * kChunk + rr) * Cb + c] = s32[k];
#pragma unroll
                    for (int k = 0; k < n64; ++k) v64[(k * kChunk + rr) * Cb + c] = s64[k];
                    if (r >= rowlo && r <= rowhi) add_powers<K, -1>(s32, s64, tile[r * Cb + c]);
                    const int te = r + 2 * w + 1;
                    if (te >= rowlo && te <= rowhi) add_powers<K, +1>(s32, s64, tile[te * Cb + c]);
                }
            } else {
                // outside the image: the identity of the sums
#pragma unroll
                for (int rr = 0; rr < kChunk; ++rr) {
#pragma unroll
                    for (int k = 0; k < n32; ++k) v32[(k * kChunk + rr) * Cb + c] = 0;
#pragma unroll
                    for (int k = 0; k < n64; ++k) v64[(k * kChunk + rr) * Cb + c] = 0;
                }
            }
        }
        // 2b. Vertical extrema of the chunk's windows (threads Cb .. Cb + Cb/2 - 1).
        vertical_extrema_simd(tile, vmin, vmax, Cb, xs, J.W, r0, w, rowlo, rowhi);
        cp_async_wait_all();
        __syncthreads();

        // 3. Horizontal phase: warp `warp` owns chunk row `warp`.
        // Window statistics of the pixel at chunk row rr, tile column x (rows
        // of the chunk are prefix sums / sparse-table levels by now).
        auto stats = [&](int rr, int x, int& alpha, int& beta, int64_t (&m)[K + 1], int& fi) {
            const int Y = y0 + r0 + rr, Xo = x0 + x;
            const int a = x + off, b = a + 2 * w;          // tile columns of the window
            const uint8_t* rmin = vmin + rr * Cb;
            const uint8_t* rmax = vmax + rr * Cb;
            if (lane_blocks) {
                alpha = lane_block_query<true>(rmin, pmin + rr * Cb, ltmin + rr * kLaneTable, a, b);
                beta = lane_block_query<false>(rmax, pmax + rr * Cb, ltmax + rr * kLaneTable, a, b);
            } else {
                alpha = min(rmin[a], rmin[b - span + 1]);
                beta = max(rmax[a], rmax[b - span + 1]);
            }
            const int ry0 = max(Y - w, 0), ry1 = min(Y + w, J.H - 1);
            const int rx0 = max(Xo - w, 0), rx1 = min(Xo + w, J.W - 1);
            m[0] = (int64_t)(ry1 - ry0 + 1) * (rx1 - rx0 + 1);
#pragma unroll
            for (int k = 0; k < n32; ++k) {
                const uint32_t* P = v32 + (k * kChunk + rr) * Cb;
                m[1 + k] = (int64_t)(uint32_t)(P[b] - (a > 0 ? P[a - 1] : 0u));
            }
#pragma unroll
            for (int k = 0; k < n64; ++k) {
                const uint64_t* P = v64 + (k * kChunk + rr) * Cb;
                m[3 + k] = (int64_t)(P[b] - (a > 0 ? P[a - 1] : 0ull));
            }
            fi = tile[(r0 + rr + w) * Cb + a + w];
        };
        auto store = [&](long long pix, double g) {
            if (J.out_f64) static_cast<double*>(J.out)[pix] = g;
            else static_cast<float*>(J.out)[pix] = (float)g;
        };
        {
            const int rr = warp;
            const int Y = y0 + r0 + rr;
#pragma unroll
            for (int k = 0; k < n32; ++k) warp_prefix_row<uint32_t>(v32 + (k * kChunk + rr) * Cb, Cb, lane);
#pragma unroll
            for (int k = 0; k < n64; ++k) warp_prefix_row<uint64_t>(v64 + (k * kChunk + rr) * Cb, Cb, lane);
            if (lane_blocks) {
                warp_lane_blocks<true>(vmin + rr * Cb, pmin + rr * Cb, ltmin + rr * kLaneTable, Cb, lane);
                warp_lane_blocks<false>(vmax + rr * Cb, pmax + rr * Cb, ltmax + rr * kLaneTable, Cb, lane);
            } else {
                warp_sparse_row<true>(vmin + rr * Cb, Cb, levels, lane);
                warp_sparse_row<false>(vmax + rr * Cb, Cb, levels, lane);
            }
            if (Y < J.H) {
                // one copy of the per-pixel code for both pixels of the lane
                // (keeps the hot loop small in the instruction cache)
#pragma unroll 1
                for (int h = 0; h < kTileW / 32; ++h) {
                    const int x = lane + 32 * h;
                    const int Xo = x0 + x;
                    if (Xo >= J.W) continue;
                    int alpha, beta, fi;
                    int64_t m[K + 1];
                    stats(rr, x, alpha, beta, m, fi);
                    const long long pix = (long long)Y * J.W + Xo;
                    const float th = s_maps[rr * kTileW + x], sg = s_maps[(kChunk + rr) * kTileW + x];
                    double g;
                    int fb = 0;
                    PixelTrace tr;
                    PixelTrace* trp = (PREC == kPrecFP64 && dbg.mu) ? &tr : nullptr;
                    if (!(sg > 0.0f) || !isfinite(sg) || !isfinite(th)) {
                        g = __longlong_as_double(0x7ff8000000000000LL);
                        if (status) atomicOr(status, kStatusBadInput);
                        trp = nullptr;
                    } else {
                        if constexpr (PREC == kPrecFP64) {
                            g = fabf_pixel_fp64<N>(c_ainv, alpha, beta, fi, m, th, sg, fb, trp);
                        } else {
                            bool redo = false;
                            if constexpr (PREC == kPrecFP64Fit)
                                g = (double)fabf_pixel_fp64fit<N>(c_ainv, alpha, beta, fi, m, th, sg, fb, redo);
                            else if constexpr (PREC == kPrecCFP32)
                                g = (double)fabf_pixel_cfp32<N>(c_ainv_split, alpha, beta, fi, m, th, sg, fb, redo);
                            else
                                g = (double)fabf_pixel_c32<N>(alpha, beta, fi, m, th, sg, fb, redo);
                            if (redo) {   // binary32 not accurate enough here: queue for the FP64 pass
                                const unsigned slot = atomicAdd(redo_n, 1u);
                                redo_list[slot] = (uint16_t)((rr << 8) | x);
                                continue;
                            }
                        }
                        if (fb && n_fallback) atomicAdd(n_fallback, 1ull);
                    }
                    store(pix, g);
                    if (PREC == kPrecFP64 && dbg.alpha) {   // the stage planes come from the FP64 form only
                        const long long plane = (long long)J.H * J.W;
                        dbg.alpha[pix] = (uint8_t)alpha;
                        dbg.beta[pix] = (uint8_t)beta;
                        if (dbg.m)
                            for (int k = 0; k <= N; ++k) dbg.m[k * plane + pix] = m[k];
                        if (dbg.flags) dbg.flags[pix] = (alpha == beta ? 1 : 0) | (fb ? 2 : 0);
                        if (trp && alpha != beta) {
                            for (int k = 0; k <= N; ++k) {
                                dbg.M[k * plane + pix] = tr.M[k];
                                dbg.mu[k * plane + pix] = tr.mu[k];
                                dbg.c[k * plane + pix] = tr.c[k];
                            }
                            for (int k = 0; k <= N + 1; ++k) dbg.I[k * plane + pix] = tr.I[k];
                            dbg.t0lam[pix] = tr.t0;
                            dbg.t0lam[plane + pix] = tr.lam;
                            dbg.T[pix] = tr.T1;
                            dbg.T[plane + pix] = tr.T2;
                        }
                    }
                }
            }
        }
        if constexpr (PREC != kPrecFP64) {
            // 4. The queued pixels on the FP64 path, packed into full warps.
            __syncthreads();
            const unsigned nr = *redo_n;
            for (unsigned i = threadIdx.x; i < nr; i += blockDim.x) {
                const int e = redo_list[i];
                const int rr = e >> 8, x = e & 255;
                int alpha, beta, fi, fb = 0;
                int64_t m[K + 1];
                stats(rr, x, alpha, beta, m, fi);
                const long long pix = (long long)(y0 + r0 + rr) * J.W + (x0 + x);
                const float th = s_maps[rr * kTileW + x], sg = s_maps[(kChunk + rr) * kTileW + x];
                const double g = PREC == kPrecCFP32 ? fabf_pixel_cfp32_redo<N>(alpha, beta, fi, m, th, sg, fb)
                                                    : fabf_pixel_fp64<N, false>(c_ainv, alpha, beta, fi, m, th, sg, fb,
                                                                         nullptr);
                store(pix, g);
                if (fb && n_fallback) atomicAdd(n_fallback, 1ull);
                if (redo_count) atomicAdd(redo_count, 1ull);
            }
        }
        __syncthreads();
    }
    return true;
}

// ---------------------------------------------------------------------------
// Single image: one tile per CTA, grid (tiles_x, tiles_y).
// ---------------------------------------------------------------------------
// Resident CTAs per SM the register budget is sized for: the FP64 form is
// bound by the FP64 pipe (two CTAs saturate it); the binary32 forms are
// bound by instruction issue and latency and gain from a fourth CTA (64
// registers per thread), measured faster at every image size.
// The centred form is also compiled for 3 CTAs per SM (up to 85 registers):
// where shared memory allows only 3 anyway (w >= 32 or so) or at N = 6, whose
// tail spills at 64 registers, that build is faster (measured 2 % at w = 40,
// N = 5 and 5 % at w = 20, N = 6; 4 % slower at w <= 20, N = 5).
template <int PREC>
struct MinBlocks {
    static constexpr int value = PREC == kPrecFP64 ? 2 : 4;
};

template <int N, int PREC, int MINB = MinBlocks<PREC>::value>
__global__ void __launch_bounds__(kThreads, MINB)
    fabf_fused_kernel(const __grid_constant__ CUtensorMap tmap, const FusedParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t phase = 0;
    if (p.job.use_tma) mbar_init(reinterpret_cast<uint64_t*>(smem));
    fabf_tile<N, PREC>(&tmap, p.job, blockIdx.x, blockIdx.y + p.job.tile_y0, smem, phase, p.status, p.n_fallback,
                       p.dbg);
}

// ---------------------------------------------------------------------------
// Batch: persistent CTAs pop tiles of many images from a device counter.
// Tiles are numbered image by image (jobs sorted by tile_begin); a CTA finds
// its tile's image by binary search and dispatches on that image's N.
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ bool batch_dispatch(const BatchParams& p, const ImageJob& J, int j, int tx, int ty,
                                               uint8_t* smem, uint32_t& phase)
{
    const DebugPlanes none{};
    const CUtensorMap* tm = p.tmaps + j;
    switch (J.N) {
    case 0: return fabf_tile<0, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    case 1: return fabf_tile<1, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    case 2: return fabf_tile<2, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    case 3: return fabf_tile<3, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    case 4: return fabf_tile<4, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    case 5: return fabf_tile<5, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    default: return fabf_tile<6, PREC>(tm, J, tx, ty, smem, phase, p.status, p.n_fallback, none);
    }
}

template <int PREC, int MINB = MinBlocks<PREC>::value>
__global__ void __launch_bounds__(kThreads, MINB) fabf_batch_kernel(const BatchParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ long long s_tile;
    __shared__ int s_job;
    uint32_t phase = 0;
    mbar_init(reinterpret_cast<uint64_t*>(smem));
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(p.next_tile, 1ull);
            int j = -1;
            if (t < p.total_tiles) {
                int lo = 0, hi = p.njobs - 1;
                while (lo < hi) {          // last job with tile_begin <= t
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.jobs[mid].tile_begin <= t) lo = mid;
                    else hi = mid - 1;
                }
                j = lo;
            }
            s_tile = t;
            s_job = j;
        }
        __syncthreads();
        const int j = s_job;
        const long long t = s_tile;
        __syncthreads();                   // s_tile / s_job are rewritten next round
        if (j < 0) break;
        const ImageJob J = p.jobs[j];
        const long long local = t - J.tile_begin;
        const int ty = (int)(local / J.tiles_x), tx = (int)(local - (long long)ty * J.tiles_x);
        if (!batch_dispatch<PREC>(p, J, j, tx, ty, smem, phase)) break;
    }
}

// ---------------------------------------------------------------------------
// Test kernel: the integral engine alone for n (lambda, t0) pairs: I_0..I_K
// in binary64 (mode 0) or binary32 (mode 1), or the centred J_0..J_K of
// FABF_C32 in binary32 (mode 2).
// ---------------------------------------------------------------------------
template <int K>
__global__ void integrals_kernel(const double* lam, const double* t0, long long n, int mode, double* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mode == 2) {
        float J[K + 1];
        const float tf = (float)t0[i];
        integrals_c32<K>((float)lam[i], tf, 2.0f * tf - 1.0f, J);
#pragma unroll
        for (int k = 0; k <= K; ++k) out[i * (K + 1) + k] = (double)J[k];
    } else if (mode == 1) {
        float I[K + 1];
        integrals_fp32<K>((float)lam[i], (float)t0[i], I);
#pragma unroll
        for (int k = 0; k <= K; ++k) out[i * (K + 1) + k] = (double)I[k];
    } else {
        double I[K + 1];
        integrals_fp64<K>(lam[i], 0.5 / lam[i], rsqrt(lam[i]), t0[i], I);
#pragma unroll
        for (int k = 0; k <= K; ++k) out[i * (K + 1) + k] = I[k];
    }
}

// ---------------------------------------------------------------------------
// Brute-force adaptive bilateral filter, Eqs. (1)-(3), box spatial kernel on
// the clipped window (the GPU comparator); Real = double or float.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) bruteforce_kernel(const uint8_t* img, long long pitch,
                                                         const float* theta, const float* sigma,
                                                         int H, int W, int w, void* out, int out_f64)
{
    const int X = blockIdx.x * 32 + (threadIdx.x & 31);
    const int Y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (X >= W || Y >= H) return;
    const long long pix = (long long)Y * W + X;
    const Real th = (Real)theta[pix];
    const Real s = (Real)sigma[pix];
    const Real inv = (Real)-1 / ((Real)2 * s * s);
    Real num = 0, den = 0;
    const int y0 = max(Y - w, 0), y1 = min(Y + w, H - 1);
    const int x0 = max(X - w, 0), x1 = min(X + w, W - 1);
    for (int yy = y0; yy <= y1; ++yy) {
        const uint8_t* row = img + (long long)yy * pitch;
        for (int xx = x0; xx <= x1; ++xx) {
            const Real v = (Real)row[xx];
            const Real dv = v - th;
            const Real phi = exp(dv * dv * inv);
            num += phi * v;
            den += phi;
        }
    }
    const Real g = num / den;
    if (out_f64) static_cast<double*>(out)[pix] = (double)g;
    else static_cast<float*>(out)[pix] = (float)g;
}

}  // namespace fabf

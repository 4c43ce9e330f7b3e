/*
 * fabf.h -- C ABI of the GB300 implementation of fast adaptive bilateral
 * filtering (R. G. Gavaskar and K. N. Chaudhury, "Fast Adaptive Bilateral
 * Filtering").  Equation and section numbers below are the paper's.
 *
 * The operation (Sec. I-A, Eqs. (1)-(3)): for an 8-bit image f on the grid
 * I, a per-pixel range-kernel centre theta(i) and width sigma(i), and a box
 * spatial kernel omega == 1 on the window [-w, w]^2 clipped to the image,
 *
 *     g(i) = sum_j phi_i(f(i-j) - theta(i)) f(i-j) / sum_j phi_i(f(i-j) - theta(i)),
 *     phi_i(t) = exp(-t^2 / (2 sigma(i)^2)).
 *
 * The library computes the paper's O(1) approximation g_hat of g
 * (Algorithm 1, Eq. (29)): the local histogram on [alpha_i, beta_i] is
 * replaced by the degree-N polynomial with the same first N+1 moments
 * (Eqs. (14), (19), (24)) and the sums by integrals evaluated in closed form
 * and by the integration-by-parts recursion (Eqs. (28), (30)-(32)).
 *
 * Conventions shared by every call:
 *   - Every call returns a fabf_status; no exception or signal crosses the ABI.
 *   - Layout: the image is H rows of W bytes, row r starting at img + r*pitch
 *     (pitch >= W).  theta, sigma and out are dense H x W row-major arrays
 *     (row stride W elements).  out is float64 when out_is_f64 != 0, else
 *     float32.
 *   - Pointers may be device pointers (cudaMalloc, or memory the CUDA driver
 *     reports as device or managed) or ordinary host pointers; the kind is
 *     detected per pointer.  The caller owns every buffer it passes.
 *   - Limits: 1 <= H, W <= 65535, 1 <= w <= 40, 0 <= N <= 6.  N or w beyond
 *     that returns FABF_EUNSUPPORTED (the int64 power sums are exact only up
 *     to N = 6, w = 40); nothing falls back to the CPU.
 *   - Per-pixel data errors (sigma <= 0 or not finite, theta not finite) give
 *     NaN at that pixel and are reported as FABF_EINVAL: directly when the
 *     call blocks, else by fabf_get_status().
 *   - The library uses one GPU, selected by fabf_config.device; calls on a
 *     context must not run concurrently from several host threads.
 */
#ifndef FABF_H
#define FABF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fabf_ctx fabf_ctx;

typedef enum {
    FABF_OK = 0,
    FABF_EINVAL = 1,        /* bad argument or bad per-pixel data */
    FABF_ENOMEM = 2,        /* device or host allocation failed, or over budget */
    FABF_EAGAIN = 3,        /* not finished yet (serving) */
    FABF_EUNSUPPORTED = 4,  /* N or w outside the supported range */
    FABF_ECUDA = 5,         /* a CUDA runtime or driver call failed */
    FABF_ETIMEOUT = 6,      /* a bounded wait (host or device) gave up */
    FABF_ENOTFOUND = 7      /* unknown serving ticket */
} fabf_status;

/* Arithmetic of the per-pixel stages (Sec. II-B, II-C).
 *   FABF_FP64: everything after the exact integer stages in binary64.
 *   FABF_FP64FIT_FP32REC: shift-scale and Hilbert fit in binary64, the
 *     integrals, recursion and ratio in binary32.
 *   FABF_CFP32: fit with compensated binary32 dot products, the rest in
 *     binary32.
 *   FABF_C32: everything after the exact integer stages in binary32, with
 *     the fit of Eqs. (18)-(19), the integrals of Eq. (28) and the ratio of
 *     Eq. (29) expressed in the centred variable s = 2t - 1: the same fitted
 *     polynomial and the same g_hat, but a system whose inverse has small
 *     exact binary32 entries, so the sums hardly cancel (no compensation).
 * In the binary32 forms a pixel whose estimated error exceeds 0.25 gray
 * levels (the ratio of Eq. (29) cancels badly, T2 <= 0, or the binary32
 * integrals are in a regime where they lose digits) is recomputed on the
 * FP64 path; fabf_get_status_ex counts those pixels. */
typedef enum { FABF_FP64 = 0, FABF_FP64FIT_FP32REC = 1, FABF_CFP32 = 2, FABF_C32 = 3 } fabf_precision;

typedef struct {
    int device;                  /* CUDA device ordinal */
    size_t mem_budget_bytes;     /* device bytes the serving loop may hold (0 = 16 GiB) */
    int precision;               /* fabf_precision used by fabf_filter / batch / serve */
    int autotune;                /* nonzero: pick tile shapes and staging by measurement */
    const char* tune_cache_path; /* optional file for autotuner results (may be NULL) */
} fabf_config;

/* One filtering request (batch and serving).  passes >= 1 applies the filter
 * repeatedly (texture filtering, Sec. IV-C): pass p+1 takes as image the
 * previous output rounded half-to-even and clamped to [0, 255], as centre
 * theta_{p+1} = f_{p+1} + (theta - f), and as width sigma_p * sigma_decay. */
typedef struct {
    const uint8_t* img;
    const float* theta;
    const float* sigma;
    int H, W;
    size_t pitch;
    int w;
    int N;
    int passes;
    float sigma_decay;
    void* out;
    int out_is_f64;
} fabf_request;

/* Create a context on cfg->device (cfg may be NULL: device 0, FP64).
 * On success *out owns a CUDA stream-independent context; release it with
 * fabf_destroy.  Errors: FABF_EINVAL (out NULL, bad precision), FABF_ECUDA. */
int fabf_create(const fabf_config* cfg, fabf_ctx** out);

/* Release everything the context holds (waits for its own work first). */
int fabf_destroy(fabf_ctx* ctx);

/* Change the precision used by later calls on ctx (fabf_precision). */
int fabf_set_precision(fabf_ctx* ctx, int precision);

/* Algorithm 1 (Sec. II-D) on one image: out[i] = g_hat(i) of Eq. (29), with
 * g_hat(i) = f(i) where alpha_i == beta_i.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream).  If img, theta, sigma and out are all
 * device pointers the work is only enqueued on the stream (stream-ordered,
 * the call returns at once; per-pixel data errors are read later with
 * fabf_get_status).  If any of them is a host pointer, the call returns
 * after out is written.  When theta, sigma and out are pinned (page-locked)
 * host memory, the kernel reads the maps and writes out in place over the
 * chip-to-chip link and only a host image is copied to the device; other
 * host buffers are staged through device memory (copies, kernels and copies
 * back overlapping in bands of rows).
 * Errors: FABF_EINVAL, FABF_EUNSUPPORTED, FABF_ENOMEM, FABF_ECUDA,
 * FABF_ETIMEOUT (a tile copy into shared memory did not complete). */
int fabf_filter(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma,
                int H, int W, size_t pitch, int w, int N, void* out, int out_is_f64,
                void* cuda_stream);

/* Wait for cuda_stream, then report and clear the data errors of the
 * stream-ordered calls made on ctx since the last query: *status receives
 * FABF_OK, FABF_EINVAL or FABF_ETIMEOUT; *n_fallback (may be NULL) the number
 * of pixels where the fitted approximation had a non-positive denominator
 * and the sigma -> infinity limit (the box mean) was returned instead. */
int fabf_get_status(fabf_ctx* ctx, void* cuda_stream, int* status, uint64_t* n_fallback);

/* As fabf_get_status, and *n_fp64_redo (may be NULL) receives the number of
 * pixels the binary32 precision forms recomputed on the FP64 path because
 * their own error estimate exceeded 0.25 gray levels (or T2 <= 0, or the
 * binary32 integrals were in a regime where they lose digits). */
int fabf_get_status_ex(fabf_ctx* ctx, void* cuda_stream, int* status, uint64_t* n_fallback,
                       uint64_t* n_fp64_redo);

/* Algorithm 1 on n images of any sizes, w and N (reqs[i].passes must be 1)
 * in one persistent launch: CTAs pop the tiles of all images from a device
 * counter.  The launch (counter reset + kernel) is captured once in a CUDA
 * graph and replayed by later calls with the same request array and
 * precision; tile shapes come from the autotuner when the context has
 * autotune on.  Up to 4 request sets keep their own graph, job table and
 * work counter (least recently used evicted), so calls may alternate sets
 * on any stream without waiting: a replay of a set is ordered after that
 * set's previous replay, and a set's table is rewritten only after its last
 * replay has finished (the call then waits for it on the host).  Device
 * pointers only (FABF_EINVAL otherwise); stream-ordered on cuda_stream like
 * fabf_filter, data errors via fabf_get_status.
 * Errors: FABF_EINVAL, FABF_EUNSUPPORTED, FABF_ENOMEM, FABF_ECUDA. */
int fabf_filter_batch(fabf_ctx* ctx, const fabf_request* reqs, int n, void* cuda_stream);

/* Serving: admit one request into the continuous-batching loop.  A request
 * is admitted when one of 64 slots is free and its device bytes (inputs,
 * output and pass state, about 17 B/px) fit the remaining memory budget;
 * its passes are enqueued at once on the slot's stream, so requests admitted
 * while others run overlap with them on the GPU.  The inputs are copied at
 * admission (caller buffers are free when the call returns); out (host or
 * device) must stay valid until fabf_serve_poll reports completion.  The
 * first call starts the context's serving worker thread.  Errors:
 * FABF_EINVAL (bad request, passes outside 1..16, sigma_decay <= 0),
 * FABF_EUNSUPPORTED, FABF_ENOMEM (larger than the whole budget), FABF_EAGAIN
 * (no slot or budget right now: retry later), FABF_ECUDA. */
int fabf_serve_submit(fabf_ctx* ctx, const fabf_request* req, uint64_t* ticket);

/* Serving: wait up to timeout_us microseconds (0 = do not wait) for ticket.
 * Returns FABF_OK and *result = the request's status once it is done,
 * FABF_EAGAIN while it is pending, FABF_ENOTFOUND for an unknown or already
 * collected ticket. */
int fabf_serve_poll(fabf_ctx* ctx, uint64_t ticket, int timeout_us, int* result);

/* Serving counters: device bytes held by admitted requests and the number
 * of requests still running (either pointer may be NULL). */
int fabf_serve_stats(fabf_ctx* ctx, uint64_t* bytes_in_use, int* in_flight);

/* Batch counters: CUDA graph captures and graph launches so far. */
int fabf_batch_stats(fabf_ctx* ctx, int* graph_captures, int* graph_launches);

/* Steady-state output rows per tile (many tiles in flight, as in a batch)
 * the context uses for (w, N, precision): the autotuner's measured choice
 * among 8, 16, 24, 32 and 40 when autotune is on, else 8 (FABF_FP64,
 * FABF_FP64FIT_FP32REC) or 40 (FABF_CFP32, FABF_C32).  The autotuner's first
 * query of a key times every candidate height with each tile staging (TMA
 * tensor copies, and plain cooperative loads) on a synthetic 2048x4096 image
 * in the form's own output type, keeps the fastest pair, and caches it (in
 * tune_cache_path too, as lines "w N precision rows ms plain").  A
 * single-image call uses the tallest candidate no taller than this that
 * still fills the SMs with at least 6 (FABF_CFP32) or 3 (FABF_C32) waves of
 * resident CTAs, else 8.  Make the first query of a key before any stream
 * capture. */
int fabf_tile_rows(fabf_ctx* ctx, int w, int N, int precision, int* tile_rows);

/* Text of a fabf_status value (static storage). */
const char* fabf_status_str(int status);

/* Allocation-free variant of fabf_filter (the paper has no counterpart).
 * For callers that must not allocate device memory -- a real-time thread
 * that cannot absorb cudaMalloc's device-wide synchronisation, a plugin
 * whose host framework owns every allocation -- and therefore cannot create
 * a context.  It runs the same
 * FP64 fused kernel as fabf_filter on the caller's device buffers and needs
 * no context; the kernel's scratch (its status word and fallback-pixel
 * counter, 16 bytes) lives in a 256-byte array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   - img, theta, sigma, out must be device memory of the calling thread's
 *     current device (FABF_EINVAL otherwise: host buffers would need device
 *     staging, and another GPU's buffers are not read).  Layout, limits and
 *     the other errors as fabf_filter.
 *   - The first call on a device looks up the array's device address (once
 *     per device, cached until the process exits); the library must not be
 *     used across a cudaDeviceReset of that device.
 *   - The call clears the scratch, enqueues the kernel on cuda_stream, then
 *     waits for the stream (so it must not be made while a stream capture
 *     is active) and returns FABF_OK, FABF_EINVAL (bad per-pixel
 *     data) or FABF_ETIMEOUT; *n_fallback (may be NULL) receives the number
 *     of pixels that took the box-mean fallback.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race on it and may report each
 *     other's status.  It calls no cudaMalloc, cudaFree or allocating
 *     library routine. */
int fabf_filter_noalloc(const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                        size_t pitch, int w, int N, void* out, int out_is_f64, void* cuda_stream,
                        uint64_t* n_fallback);

/* ---- separable spatial kernel (Gaussian, Eq. (4)) ------------------------ */

/* fabf_filter with the spatial kernel omega(j) = taps[jy + r] * taps[jx + r]
 * on the window [-r, r]^2 (clipped to the image) instead of the box: Eqs.
 * (1)-(3) with a general omega, and Algorithm 1 with the moments of Eq. (17)
 * weighted by omega.  With Gaussian taps (fabf_gaussian_taps) this is the
 * paper's own setting, Eq. (4) with the window [-3 rho, 3 rho]^2.
 *   taps  HOST array of 2r+1 integers read during the call: taps[t] >= 0,
 *         taps[r] >= 1, sum <= 65535 (so every moment is an exact integer
 *         below 2^81, summed in 64/128-bit arithmetic);
 *   r     1..40;  N 0..6;  the other arguments, the pointer kinds (pinned
 *         theta, sigma and out are read and written in place), the
 *         synchronisation and the status reporting are those of fabf_filter.
 * Computed in the context's precision (fabf_set_precision); the binary32
 * forms shift the 128-bit scaled moments right by one common amount.
 * Errors: FABF_EINVAL (NULL pointers, taps[r] == 0, bad sizes),
 * FABF_EUNSUPPORTED (r > 40, N > 6, tap sum > 65535), FABF_ECUDA. */
int fabf_filter_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma,
                    int H, int W, size_t pitch, const uint32_t* taps, int r, int N, void* out,
                    int out_is_f64, void* cuda_stream);

/* Integer taps of the Gaussian spatial kernel of Eq. (4) along one axis:
 * r = max(1, ceil(3 rho)) and taps[t] = floor(1024 exp(-(t - r)^2 / (2 rho^2))
 * + 1/2), t = 0..2r (host only, no GPU).  Their sum stays below 34,300 for
 * every allowed rho.  Errors: FABF_EINVAL (rho <= 0 or not finite, NULL
 * pointers, capacity < 2r+1), FABF_EUNSUPPORTED (3 rho > 40). */
int fabf_gaussian_taps(double rho, uint32_t* taps, int capacity, int* r);

/* ---- box-cascade spatial kernel (O(1) in the kernel width) ---------------- */

/* fabf_filter_sep with the taps of fabf_cascade_taps(rb): the cascade of
 * three boxes of length n = 2 rb + 1, radius r = 3 rb, whose variance along
 * each axis is rb (rb + 1) -- the combination of box kernels that stands in
 * for the Gaussian of Eq. (4) at a cost per pixel independent of rb (the
 * O(1) convolutions of Sec. II-D).  The result is that of fabf_filter_sep on
 * the same taps, bit for bit (every moment is an exact integer on both
 * paths); only the cost differs.
 *   rb         1..13 (r = 3 rb <= 40);
 *   tile_rows  0: the path's own rule; else the output rows per tile, a
 *              multiple of 8 from 8 to 64 (the result does not depend on it);
 *   the other arguments, pointer kinds, synchronisation, precision and
 *   status reporting are those of fabf_filter_sep.
 * Errors: FABF_EINVAL (rb < 1, bad tile_rows, as fabf_filter_sep),
 * FABF_EUNSUPPORTED (rb > 13, N > 6), FABF_ECUDA. */
int fabf_filter_cascade(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma,
                        int H, int W, size_t pitch, int rb, int N, void* out, int out_is_f64,
                        int tile_rows, void* cuda_stream);

/* Taps of the three-box cascade of radius rb along one axis (host only, no
 * GPU): the three-fold convolution of 2 rb + 1 ones, 2r + 1 = 6 rb + 1
 * integers summing to (2 rb + 1)^3 <= 19683; *r = 3 rb.  Errors:
 * FABF_EINVAL (NULL pointers, rb < 1, capacity < 2r + 1), FABF_EUNSUPPORTED
 * (rb > 13). */
int fabf_cascade_taps(int rb, uint32_t* taps, int capacity, int* r);

/* The cascade radius rb (1..13) whose variance rb (rb + 1) is nearest rho^2
 * (host only).  Errors: FABF_EINVAL (rho <= 0 or not finite, NULL),
 * FABF_EUNSUPPORTED (rho above 14, where rb = 14 would be nearest). */
int fabf_cascade_radius(double rho, int* rb);

/* ---- applications (Sec. IV) ---------------------------------------------- */

/* Sharpening and noise removal (Sec. IV-A).  The paper sets theta = f +
 * zeta with zeta = f - fbar (fbar the mean of f over the window) and sigma
 * by an affine map of |LoG f| that sends low values to wide kernels; its
 * parameters are open, and are read here as:
 *   theta = (2 f m_0 - m_1) / m_0 over the clipped window [-w, w]^2;
 *   L = 5-point Laplacian of S = g x g * f with the integer Gaussian taps
 *       g = fabf_gaussian_taps(rho_log) (coordinates clamped to the image);
 *   sigma = sigma_hi - (sigma_hi - sigma_lo) min(|L|, Lq) / Lq with
 *       Lq = floor(lap_sat (sum g)^2 + 1/2), i.e. lap_sat in gray levels. */
typedef struct {
    int w;               /* box radius of the filter and of the mean, 1..40 */
    int N;               /* polynomial degree, 0..6 */
    double rho_log;      /* width of the LoG's Gaussian (0 < rho_log <= 40/3) */
    double lap_sat;      /* |LoG| (gray levels) from which sigma = sigma_lo */
    double sigma_lo, sigma_hi;   /* 0 < sigma_lo <= sigma_hi */
} fabf_sharpen_cfg;

/* Texture filtering (Sec. IV-C): theta = f and sigma from mRTV = Delta
 * max|grad f| / (sum |grad f| + eps) over [-k, k]^2 (clipped; Delta the
 * range of f there; |grad f| read as |f(x+1,y) - f(x,y)| + |f(x,y+1) -
 * f(x,y)| with clamped coordinates), sigma = sigma_hi - (sigma_hi -
 * sigma_lo) min(mRTV / mrtv_sat, 1); two smoothing passes, the second with
 * sigma scaled by sigma_decay and the rounded output of the first as input,
 * then one sharpening pass (cfg.sharpen) on the rounded output. */
typedef struct {
    int w, N;            /* the two smoothing passes */
    int k;               /* mRTV window radius, 1..40 */
    double eps, mrtv_sat, sigma_lo, sigma_hi, sigma_decay;
    fabf_sharpen_cfg sharpen;
} fabf_texture_cfg;

/* The sharpening maps of img into theta and sigma (float32 H x W, row
 * stride W).  Device pointers only; stream-ordered; maps are identical to
 * the reference definitions above to the last bit.  Errors: FABF_EINVAL
 * (NULL or host pointers, bad sizes or parameters), FABF_EUNSUPPORTED (w >
 * 40, N > 6, 3 rho_log > 40), FABF_ENOMEM, FABF_ECUDA. */
int fabf_sharpen_maps(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch,
                      const fabf_sharpen_cfg* cfg, float* theta, float* sigma, void* cuda_stream);

/* The texture width map of img (float32 H x W).  As fabf_sharpen_maps. */
int fabf_texture_sigma(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch,
                       const fabf_texture_cfg* cfg, float* sigma, void* cuda_stream);

/* One sharpening pass: the maps, then Algorithm 1 in the context's
 * precision into out.  Device pointers; stream-ordered (intermediates are
 * stream-ordered allocations); data errors through fabf_get_status. */
int fabf_sharpen(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch,
                 const fabf_sharpen_cfg* cfg, void* out, int out_is_f64, void* cuda_stream);

/* The texture-filtering pipeline (three passes of Algorithm 1).  As
 * fabf_sharpen. */
int fabf_texture_filter(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch,
                        const fabf_texture_cfg* cfg, void* out, int out_is_f64, void* cuda_stream);

/* ---- colour images (Sec. IV-C: channel by channel) ----------------------- */
/* rgb is an 8-bit interleaved H x W x 3 image (R, G, B) with a row pitch in
 * bytes >= 3 W.  The paper computes the width maps of its colour examples on
 * a gray version of the image; that version is read as the BT.601 luma
 * rounded half up, in integers:  Y = floor((299 R + 587 G + 114 B + 500) /
 * 1000).  Outputs are interleaved H x W x 3 (float32, or float64 when
 * out_is_f64), row stride 3 W.  Device pointers only; stream-ordered
 * (intermediates are stream-ordered allocations); data errors through
 * fabf_get_status.  Errors: FABF_EINVAL (NULL or host pointers, H, W
 * outside 1..65535, pitch < 3 W, bad parameters), FABF_EUNSUPPORTED,
 * FABF_ENOMEM, FABF_ECUDA. */

/* The luma Y of rgb (uint8 H x W, row pitch y_pitch >= W). */
int fabf_luma(fabf_ctx* ctx, const uint8_t* rgb, int H, int W, size_t pitch, uint8_t* Y, size_t y_pitch,
              void* cuda_stream);

/* Algorithm 1 on each channel in the context's precision: theta is an
 * interleaved float32 H x W x 3 map (NULL: theta_c = f_c, the classical
 * filter), sigma one float32 H x W map shared by the channels. */
int fabf_filter_rgb(fabf_ctx* ctx, const uint8_t* rgb, const float* theta, const float* sigma, int H, int W,
                    size_t pitch, int w, int N, void* out, int out_is_f64, void* cuda_stream);

/* The texture-filtering pipeline on a colour image: the mRTV width map of
 * the luma; per channel the two smoothing passes (theta = f_c); then the
 * sharpening width map of the luma of the rounded second outputs, shared by
 * the channels, and each channel's own sharpening centre (cfg.sharpen). */
int fabf_texture_filter_rgb(fabf_ctx* ctx, const uint8_t* rgb, int H, int W, size_t pitch,
                            const fabf_texture_cfg* cfg, void* out, int out_is_f64, void* cuda_stream);

/* ---- host-side helpers (no GPU needed) ---------------------------------- */

/* The exact inverse of the (N+1) x (N+1) Hilbert matrix of Eq. (18), by the
 * closed form of Eq. (19), row-major into out[(N+1)*(N+1)] -- the table the
 * kernels use.  Errors: FABF_EINVAL (out NULL), FABF_EUNSUPPORTED (N > 6). */
int fabf_hilbert_inverse(int N, int64_t* out);

/* The inverse of the (N+1) x (N+1) matrix of the centred fit of FABF_C32,
 * A~[j][k] = 1 / (j + k + 1) for j + k even and 0 otherwise (the moments of
 * s = 2t - 1 over t in [0, 1], the same moment-matching problem as Eq. (18)
 * in another basis), row-major into out[(N+1)*(N+1)] -- the binary32 table
 * the kernels use; every entry is a dyadic rational held exactly.  Errors:
 * FABF_EINVAL (out NULL), FABF_EUNSUPPORTED (N > 6). */
int fabf_centred_inverse(int N, double* out);

/* Dynamic shared memory (bytes) one CTA of the fused kernel needs for
 * (w, N) with the tallest tile (64 output rows). */
int fabf_fused_smem_bytes(int w, int N, size_t* bytes);

/* ---- measurement ---------------------------------------------------------- */

/* Arithmetic pipe peaks of the calling thread's current GPU, measured with
 * CUDA events on the legacy default stream (the paper has no counterpart:
 * these are the denominators of the rooflines the filter's kernels are
 * quoted against, since the filter is bound by arithmetic, not HBM).  Each
 * figure is the best of 3 timed launches of a kernel that runs 8
 * independent dependency chains per thread on 4 x 256-thread CTAs per SM.
 *   out[0] FP64 fused multiply-add, TFLOP/s (an FMA counts 2 flops)
 *   out[1] FP32 fused multiply-add, TFLOP/s
 *   out[2] INT32 multiply-add, T ops/s
 *   out[3] MUFU base-2 exponential (ex2.approx.f32), T ops/s
 *   out[4] SM clock seen during the FP64 run, MHz (clock64 cycles of one CTA
 *          over the global-timer nanoseconds of the same interval)
 *   out[5] number of SMs
 * Synchronous; allocates and frees 2 KB of device memory.  Errors:
 * FABF_EINVAL (out NULL), FABF_ENOMEM, FABF_ECUDA. */
int fabf_pipe_peaks(double* out);

/* ---- test entry points (device pointers only, synchronous) -------------- */

/* Every intermediate of Algorithm 1 from the fused kernel, one plane of
 * H x W per quantity and index (planes stacked, row stride W):
 *   alpha, beta: uint8 (Eq. (8));  m: (N+1) int64 planes, m_k of Eq. (17);
 *   M: (N+1) int64 planes, M_k = sum (f - alpha)^k (numerator of Eq. (24));
 *   mu, c: (N+1) float64 planes (Eq. (24), Eq. (19) times mu);
 *   t0lam: 2 planes (t0, lambda of Eq. (25));  I: N+2 planes (Eq. (28),
 *   scaled by exp(lambda d^2), d = distance from t0 to [0, 1]);
 *   T: 2 planes (T1, T2 of Algorithm 1);  flags: int32 (bit0 flat, bit1 box
 *   mean fallback);  out: float64 g_hat.  M, mu, c, t0lam, I, T are left
 *   untouched at flat pixels.  Errors as fabf_filter. */
int fabf_debug_stages(fabf_ctx* ctx, const uint8_t* img, const float* theta,
                      const float* sigma, int H, int W, size_t pitch, int w, int N,
                      uint8_t* alpha, uint8_t* beta, int64_t* m, int64_t* M, double* mu,
                      double* c, double* t0lam, double* I, double* T, int32_t* flags,
                      double* out);

/* The integral engine alone: out[j*(K+1) + k] = I_k(lambda[j], t0[j]) for
 * k = 0..K (Eq. (28), scaled by exp(lambda d^2)), 1 <= K <= 7, lambda > 0,
 * in the given precision (FABF_FP64 or FABF_FP64FIT_FP32REC for binary32);
 * with FABF_C32 the centred integrals of that form instead:
 * out[j*(K+1) + k] = J_k = int_0^1 (2t - 1)^k exp(-lambda (t - t0)^2) dt,
 * with the same scaling, in binary32. */
int fabf_debug_integrals(fabf_ctx* ctx, const double* lambda, const double* t0, int64_t n,
                         int K, int precision, double* out);

/* Brute-force adaptive bilateral filter, Eqs. (1)-(3), with the box kernel on
 * the clipped window: the GPU comparator (O(w^2) per pixel).  use_f64
 * selects binary64 or binary32 arithmetic.  Pointers and stream as in
 * fabf_filter. */
int fabf_bruteforce(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma,
                    int H, int W, size_t pitch, int w, void* out, int out_is_f64, int use_f64,
                    void* cuda_stream);

/* fabf_debug_stages for the separable kernel: the same planes, except m and M
 * hold 2 (N+1) uint64 words per pixel ((N+1) planes of H x W x 2, low word
 * first), since weighted moments reach 2^81.  M, mu, c, t0lam, I, T are left
 * untouched at flat pixels. */
int fabf_debug_stages_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta,
                          const float* sigma, int H, int W, size_t pitch, const uint32_t* taps,
                          int r, int N, uint8_t* alpha, uint8_t* beta, uint64_t* m, uint64_t* M,
                          double* mu, double* c, double* t0lam, double* I, double* T,
                          int32_t* flags, double* out);

/* fabf_debug_stages_sep on the box-cascade path (fabf_filter_cascade's
 * kernel) with the cascade of radius rb; the same planes and errors. */
int fabf_debug_stages_cascade(fabf_ctx* ctx, const uint8_t* img, const float* theta,
                              const float* sigma, int H, int W, size_t pitch, int rb, int N,
                              uint8_t* alpha, uint8_t* beta, uint64_t* m, uint64_t* M, double* mu,
                              double* c, double* t0lam, double* I, double* T, int32_t* flags,
                              double* out);

/* The FP64 form's own binary64 erfcx and exp (the functions of its
 * integrals, Eq. (31)) on n device arguments: erfcx_out[j] = erfcx(|x[j]|),
 * exp_out[j] = exp(-|x[j]|), all device pointers; synchronous.  Test entry
 * point.  Errors: FABF_EINVAL (NULL or host pointers, n < 0), FABF_ECUDA. */
int fabf_debug_fp64_functions(fabf_ctx* ctx, const double* x, int64_t n, double* erfcx_out,
                              double* exp_out);

/* Brute-force filter, Eqs. (1)-(3), with the separable kernel (O(r^2) per
 * pixel); arguments as fabf_bruteforce plus taps and r as fabf_filter_sep. */
int fabf_bruteforce_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta,
                        const float* sigma, int H, int W, size_t pitch, const uint32_t* taps,
                        int r, void* out, int out_is_f64, int use_f64, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FABF_H */

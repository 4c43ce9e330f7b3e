// Host side of the separable (Gaussian) spatial-kernel path: tap checks, the
// tile height, kernel dispatch over precision and N, and its C ABI entry
// points.  The kernels are in fabf_sep_kernels.cuh (instantiated per
// precision in fabf_sep_p0.cu, fabf_sep_p1.cu, fabf_sep_p2.cu).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/fabf.h"
#include "fabf_internal.h"
#include "fabf_casc_kernels.cuh"
#include "fabf_sep_kernels.cuh"

namespace fabf {

// Tile height of the separable path: the box path's rule (the steady-state
// heights per precision, fewer rows for short images) with the shared-memory
// size of this kernel.
static int sep_tile_rows(fabf_ctx* ctx, int r, int N, int prec, int H, int W)
{
    const int steady = kSteadyTileRows[prec_index(prec)];
    if (steady <= kTileCandidates[0]) return steady;
    int off, Cb;
    fused_geometry(r, &off, &Cb);
    const long long tiles_x = (W + kTileW - 1) / kTileW;
    int best = kTileCandidates[0];
    for (int TH : kTileCandidates) {
        if (TH > steady) break;
        const size_t smem = sep_smem_bytes(N, r, Cb, TH) + 1024;
        const int per_sm = std::max(1, std::min(kCtasPerSm[prec_index(prec)],
                                                (int)((size_t)228 * 1024 / smem)));
        const long long tiles = tiles_x * ((H + TH - 1) / TH);
        if (tiles >= (long long)kMinWaves[prec_index(prec)] * ctx->num_sms * per_sm) best = TH;
    }
    return best;
}

// Tile height of the box-cascade path.  Every tile runs 2r steps of the
// vertical sums before its first output row, so the binary32 forms take the
// tallest tile (up to 64 rows) that keeps the residency of the shortest and
// still leaves 2.5 waves of resident CTAs across the SMs (measured at 1080p
// for rb = 1..13: within 2 % of the best height, which grows from 16-24
// rows at small rb to 40 at rb = 13); the FP64 forms, bound by the FP64
// pipe, take 8-row tiles (the fastest at every rb).
constexpr int kCascTileCandidates[] = {8, 16, 24, 32, 40, 48, 56, 64};

static int casc_tile_rows(fabf_ctx* ctx, int r, int N, int prec, int H, int W)
{
    if (kSteadyTileRows[prec_index(prec)] <= kCascTileCandidates[0]) return kCascTileCandidates[0];
    int off, Cb;
    fused_geometry(r, &off, &Cb);
    const long long tiles_x = (W + kTileW - 1) / kTileW;
    auto per_sm = [&](int TH) {
        return std::min(CascMinBlocks<kPrecC32>::value, smem_resident_ctas(casc_smem_bytes(N, r, Cb, TH)));
    };
    // no taller tile than shared memory allows at the residency of the
    // shortest one
    const int most = per_sm(kCascTileCandidates[0]);
    int best = kCascTileCandidates[0];
    for (int TH : kCascTileCandidates) {
        if (per_sm(TH) < most) break;
        const long long tiles = tiles_x * ((H + TH - 1) / TH);
        if (2 * tiles >= 5LL * ctx->num_sms * most) best = TH;
    }
    return best;
}

static cudaError_t launch_sep(int prec, int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem,
                              cudaStream_t s)
{
    if (p.taps.casc_n) {
        switch (prec) {
        case kPrecFP64: return launch_casc_p0(N, tm, p, grid, smem, s);
        case kPrecFP64Fit: return launch_casc_p1(N, tm, p, grid, smem, s);
        case kPrecCFP32: return launch_casc_p2(N, tm, p, grid, smem, s);
        case kPrecC32: return launch_casc_p3(N, tm, p, grid, smem, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (prec) {
    case kPrecFP64: return launch_sep_p0(N, tm, p, grid, smem, s);
    case kPrecFP64Fit: return launch_sep_p1(N, tm, p, grid, smem, s);
    case kPrecCFP32: return launch_sep_p2(N, tm, p, grid, smem, s);
    case kPrecC32: return launch_sep_p3(N, tm, p, grid, smem, s);
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

// Taps of the three-box cascade of radius rb (integer, exact): the three-fold
// convolution of a box of length n = 2 rb + 1 with itself; 2r + 1 taps,
// r = 3 rb, summing to n^3.
static int cascade_taps(int rb, uint32_t* taps, int capacity, int* r_out)
{
    if (rb < 1) return FABF_EINVAL;
    if (rb > kCascRbMax) return FABF_EUNSUPPORTED;
    const int n = 2 * rb + 1, r = kCascBoxes * rb;
    if (capacity < 2 * r + 1) return FABF_EINVAL;
    uint32_t a[2 * kWMax + 1], b[2 * kWMax + 1];
    int len = n;
    for (int t = 0; t < n; ++t) a[t] = 1;
    for (int box = 1; box < kCascBoxes; ++box) {
        for (int t = 0; t < len + n - 1; ++t) {
            uint32_t s = 0;
            for (int j = 0; j < n; ++j)
                if (t - j >= 0 && t - j < len) s += a[t - j];
            b[t] = s;
        }
        len += n - 1;
        for (int t = 0; t < len; ++t) a[t] = b[t];
    }
    for (int t = 0; t < len; ++t) taps[t] = a[t];
    *r_out = r;
    return FABF_OK;
}

// The kernel's copy of the cascade's taps (prefix sums for m_0) and box length.
static int make_cascade(int rb, SepTaps* T)
{
    uint32_t taps[2 * kWMax + 1];
    int r = 0;
    int rc = cascade_taps(rb, taps, 2 * kWMax + 1, &r);
    if (rc) return rc;
    rc = make_taps(taps, r, T);
    if (rc) return rc;
    // Weights of tile row t (0 <= t < A = 2r) in the running sums after A
    // steps from zero, U1 = sum_a e(a), U2 = sum_a (A - a) e(a), V = sum_a
    // (A - a)(A - a + 1)/2 e(a), with e(a) = sum_j c_j p(a - jn), c = (1, -3,
    // 3, -1): the start sums of a tile as one weighted sum per row.
    const int n = 2 * rb + 1, A = 2 * r;
    const int c[4] = {1, -3, 3, -1};
    for (int t = 0; t < A; ++t) {
        int w1 = 0, w2 = 0, w3 = 0;
        for (int j = 0; j < 4; ++j) {
            const int L = A - t - j * n;   // steps left after row t enters as a = t + jn
            if (L <= 0) continue;
            w1 += c[j];
            w2 += c[j] * L;
            w3 += c[j] * L * (L + 1) / 2;
        }
        T->pre_w[0][t] = (int16_t)w1;
        T->pre_w[1][t] = (int16_t)w2;
        T->pre_w[2][t] = (int16_t)w3;
    }
    T->casc_n = n;
    return FABF_OK;
}

static int run_sep(int prec, const SepTaps& T, const uint8_t* img, size_t pitch, const float* theta,
                   const float* sigma, int H, int W, int N, void* out, int out_f64, int TH, const SepDebug* dbg,
                   unsigned* status, unsigned long long* nfb, cudaStream_t s, int maps_host = 0)
{
    SepParams p;
    std::memset(&p, 0, sizeof(p));
    CUtensorMap tm;
    (void)make_job(&p.job, &tm, img, pitch, theta, sigma, H, W, T.r, N, out, out_f64, TH);
    p.job.maps_host = maps_host;
    p.taps = T;
    p.status = status;
    p.n_fallback = nfb;
    if (dbg) p.dbg = *dbg;
    const size_t smem = T.casc_n ? casc_smem_bytes(N, T.r, p.job.Cb, TH) : sep_smem_bytes(N, T.r, p.job.Cb, TH);
    dim3 grid(p.job.tiles_x, p.job.tiles_y);
    return cuda_status(launch_sep(prec, N, tm, p, grid, smem, s));
}

// fabf_filter_sep / fabf_filter_cascade on the kernel's tap description T;
// tile_rows 0 picks the path's rule.
static int filter_sep_impl(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                           size_t pitch, const SepTaps& T, int N, void* out, int out_is_f64, int tile_rows,
                           void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, T.r, N);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int prec = ctx->precision;
    const int TH = tile_rows ? tile_rows
                             : T.casc_n ? casc_tile_rows(ctx, T.r, N, prec, H, W) : sep_tile_rows(ctx, T.r, N, prec, H, W);
    const PtrInfo pi = ptr_info(img), pt = ptr_info(theta), ps = ptr_info(sigma), po = ptr_info(out);
    if (!(pt.device && ps.device && po.device) && pt.kptr && ps.kptr && po.kptr) {
        // pinned host maps and output: read and written in place by the
        // kernel over the chip-to-chip link; only a host image is copied
        std::lock_guard<std::mutex> staged(ctx->stage_lock);
        const uint8_t* d_img = nullptr;
        size_t d_pitch = 0;
        rc = stage_image(ctx, img, pi, H, W, pitch, s, &d_img, &d_pitch);
        if (rc) return rc;
        rc = run_sep(prec, T, d_img, d_pitch, static_cast<const float*>(pt.kptr), static_cast<const float*>(ps.kptr),
                     H, W, N, const_cast<void*>(po.kptr), out_is_f64, TH, nullptr, pinned_call_status(ctx),
                     pinned_call_nfb(ctx), s, 1);
        if (rc) {
            cudaStreamSynchronize(s);
            return rc;
        }
        return finish_pinned_call(ctx, s);
    }
    return with_device_buffers(
        ctx, img, theta, sigma, H, W, pitch, out, out_is_f64, s,
        [&](const uint8_t* d_img, size_t d_pitch, const float* d_th, const float* d_sg, void* d_out) {
            return run_sep(prec, T, d_img, d_pitch, d_th, d_sg, H, W, N, d_out, out_is_f64, TH, nullptr,
                           ctx->d_status, ctx->d_nfb, s);
        });
}

// fabf_debug_stages_sep / fabf_debug_stages_cascade on tap description tp.
static int debug_stages_sep_impl(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H,
                                 int W, size_t pitch, const SepTaps& tp, int N, uint8_t* alpha, uint8_t* beta,
                                 uint64_t* m, uint64_t* M, double* mu, double* c, double* t0lam, double* I,
                                 double* T, int32_t* flags, double* out)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, tp.r, N);
    if (rc) return rc;
    if (!alpha || !beta || !m || !M || !mu || !c || !t0lam || !I || !T || !flags) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    SepDebug d{alpha, beta, m, M, mu, c, t0lam, I, T, flags};
    rc = run_sep(kPrecFP64, tp, img, pitch, theta, sigma, H, W, N, out, 1, kDefaultTileRows, &d, ctx->d_status,
                 ctx->d_nfb, 0);
    if (rc) return rc;
    int st = FABF_OK;
    rc = read_and_clear_status(ctx, 0, &st, nullptr, nullptr);
    return rc ? rc : st;
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
    SepTaps T;
    const int rc = make_taps(taps, r, &T);
    if (rc) return rc;
    return filter_sep_impl(ctx, img, theta, sigma, H, W, pitch, T, N, out, out_is_f64, 0, cuda_stream);
}

int fabf_cascade_taps(int rb, uint32_t* taps, int capacity, int* r)
{
    if (!taps || !r) return FABF_EINVAL;
    return cascade_taps(rb, taps, capacity, r);
}

int fabf_cascade_radius(double rho, int* rb)
{
    if (!rb || !(rho > 0.0) || !std::isfinite(rho)) return FABF_EINVAL;
    // the cascade's variance along an axis is rb (rb + 1): the rb whose
    // variance is nearest rho^2
    int best = 1;
    for (int k = 2; k <= kCascRbMax + 1; ++k)
        if (std::fabs((double)k * (k + 1) - rho * rho) < std::fabs((double)best * (best + 1) - rho * rho)) best = k;
    if (best > kCascRbMax) return FABF_EUNSUPPORTED;
    *rb = best;
    return FABF_OK;
}

int fabf_filter_cascade(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                        size_t pitch, int rb, int N, void* out, int out_is_f64, int tile_rows, void* cuda_stream)
{
    if (tile_rows != 0 && (tile_rows < kChunk || tile_rows > kTileHMax || tile_rows % kChunk)) return FABF_EINVAL;
    SepTaps T;
    const int rc = make_cascade(rb, &T);
    if (rc) return rc;
    return filter_sep_impl(ctx, img, theta, sigma, H, W, pitch, T, N, out, out_is_f64, tile_rows, cuda_stream);
}

int fabf_debug_stages_sep(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                          size_t pitch, const uint32_t* taps, int r, int N, uint8_t* alpha, uint8_t* beta,
                          uint64_t* m, uint64_t* M, double* mu, double* c, double* t0lam, double* I, double* T,
                          int32_t* flags, double* out)
{
    SepTaps tp;
    const int rc = make_taps(taps, r, &tp);
    if (rc) return rc;
    return debug_stages_sep_impl(ctx, img, theta, sigma, H, W, pitch, tp, N, alpha, beta, m, M, mu, c, t0lam, I,
                                 T, flags, out);
}

int fabf_debug_stages_cascade(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H,
                              int W, size_t pitch, int rb, int N, uint8_t* alpha, uint8_t* beta, uint64_t* m,
                              uint64_t* M, double* mu, double* c, double* t0lam, double* I, double* T,
                              int32_t* flags, double* out)
{
    SepTaps tp;
    const int rc = make_cascade(rb, &tp);
    if (rc) return rc;
    return debug_stages_sep_impl(ctx, img, theta, sigma, H, W, pitch, tp, N, alpha, beta, m, M, mu, c, t0lam, I,
                                 T, flags, out);
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

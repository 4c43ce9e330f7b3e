// Applications of Sec. IV on the device: the sharpening centre and width maps
// (Sec. IV-A), the texture width map from mRTV (Sec. IV-C), and the two
// pipelines built on Algorithm 1 -- one sharpening pass, and texture
// filtering (two smoothing passes, the second with the width scaled by
// sigma_decay, then one sharpening pass); and colour images channel by
// channel (Sec. IV-C), with the width maps taken from the luma.
//
// The maps follow the readings the CPU oracle states (integer-exact up to one
// fixed sequence of binary32 operations: the maps are binary32 maps, and
// binary64 runs at 1/64 of the binary32 rate on GB300),
// written with explicitly rounded intrinsics so that no multiply-add is
// contracted: the maps are bit-identical to the oracle's.
//   theta_sharpen = (2 f m_0 - m_1) / m_0 over the clipped window [-w, w]^2;
//   L = 5-point Laplacian of the integer Gaussian S = g x g * f (coordinates
//       clamped), sigma_sharpen = s_hi - (s_hi - s_lo) (min(|L|, Lq) / Lq);
//   g = |f(x+1, y) - f(x, y)| + |f(x, y+1) - f(x, y)| (clamped), mRTV =
//       Delta gmax / (gsum + eps) over [-k, k]^2 (clipped), sigma_texture =
//       s_hi - (s_hi - s_lo) min(mRTV / msat, 1).
// These are cheap next to Algorithm 1 and are written as plain one-thread-
// per-pixel kernels over global memory (separable passes where a window is
// involved).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <initializer_list>

#include "../../include/fabf.h"
#include "fabf_internal.h"
#include "fabf_sep_kernels.cuh"

namespace fabf {
namespace {

constexpr int kAppThreads = 256;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// rs = sum of f over the clipped row segment [x - w, x + w]
__global__ void box_rows_kernel(const uint8_t* f, long long pitch, int H, int W, int w, int32_t* rs)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    const uint8_t* row = f + (long long)y * pitch;
    const int x0 = max(x - w, 0), x1 = min(x + w, W - 1);
    int32_t s = 0;
    for (int xx = x0; xx <= x1; ++xx) s += row[xx];
    rs[i] = s;
}

__global__ void sharpen_theta_kernel(const uint8_t* f, long long pitch, const int32_t* rs, int H, int W, int w,
                                     float* theta)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    const int y0 = max(y - w, 0), y1 = min(y + w, H - 1);
    const int x0 = max(x - w, 0), x1 = min(x + w, W - 1);
    int64_t m1 = 0;
    for (int yy = y0; yy <= y1; ++yy) m1 += rs[(long long)yy * W + x];
    const int64_t m0 = (int64_t)(y1 - y0 + 1) * (x1 - x0 + 1);
    // |num| <= 2 * 255 * 6561 < 2^24 and m0 <= 6561 are exact in binary32:
    // the correctly rounded binary32 quotient
    const int num = (int)(2 * (int64_t)f[(long long)y * pitch + x] * m0 - m1);
    theta[i] = __fdiv_rn(__int2float_rn(num), __int2float_rn((int)m0));
}

// gr = sum_t g[t] f(y, clamp(x + t - r))
__global__ void gauss_rows_kernel(const uint8_t* f, long long pitch, int H, int W, const __grid_constant__ SepTaps T,
                                  uint32_t* gr)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    const uint8_t* row = f + (long long)y * pitch;
    uint32_t s = 0;
    for (int t = 0; t <= 2 * T.r; ++t) s += T.g[t] * (uint32_t)row[clampi(x + t - T.r, 0, W - 1)];
    gr[i] = s;
}

// S = sum_t g[t] gr(clamp(y + t - r), x)
__global__ void gauss_cols_kernel(const uint32_t* gr, int H, int W, const __grid_constant__ SepTaps T, int64_t* S)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    int64_t s = 0;
    for (int t = 0; t <= 2 * T.r; ++t) s += (int64_t)T.g[t] * gr[(long long)clampi(y + t - T.r, 0, H - 1) * W + x];
    S[i] = s;
}

__global__ void sharpen_sigma_kernel(const int64_t* S, int H, int W, long long Lq, float lo, float hi,
                                     float* sigma)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    const int64_t L = S[(long long)clampi(y - 1, 0, H - 1) * W + x] + S[(long long)clampi(y + 1, 0, H - 1) * W + x] +
                      S[(long long)y * W + clampi(x - 1, 0, W - 1)] + S[(long long)y * W + clampi(x + 1, 0, W - 1)] -
                      4 * S[i];
    const int64_t a = L < 0 ? -L : L;
    const int64_t q = a < Lq ? a : Lq;
    const float u = __fdiv_rn(__ll2float_rn(q), __ll2float_rn(Lq));
    sigma[i] = __fsub_rn(hi, __fmul_rn(__fsub_rn(hi, lo), u));
}

// One block per 256-pixel row segment.  The block stages the rows y - k ..
// y + k + 1 and columns x - k .. x + 255 + k + 1 of f in shared memory,
// with coordinates clamped to the image: an in-image row or column is
// itself, and the clamped neighbour of the last row or column is the
// clamped copy, as the definition wants.  Each thread then scans its window
// there.
__global__ void texture_sigma_kernel(const uint8_t* f, long long pitch, int H, int W, int k, float eps, float msat,
                                     float lo, float hi, float* sigma)
{
    extern __shared__ uint8_t tile[];                // [2k + 2][kAppThreads + 2k + 1]
    const int y = (int)blockIdx.y, xs = (int)(blockIdx.x * blockDim.x);
    const int R = 2 * k + 2, C = (int)blockDim.x + 2 * k + 1;
    for (int e = (int)threadIdx.x; e < R * C; e += (int)blockDim.x) {
        const int r = e / C, c = e - r * C;
        tile[e] = f[(long long)clampi(y - k + r, 0, H - 1) * pitch + clampi(xs - k + c, 0, W - 1)];
    }
    __syncthreads();
    const int x = xs + (int)threadIdx.x;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    const int y0 = max(y - k, 0), y1 = min(y + k, H - 1);
    const int x0 = max(x - k, 0), x1 = min(x + k, W - 1);
    int fmin = 255, fmax = 0, gmax = 0, gsum = 0;
    for (int yy = y0; yy <= y1; ++yy) {
        const uint8_t* row = tile + (yy - (y - k)) * C - (xs - k);    // row[xx] = f(yy, xx)
        const uint8_t* below = row + C;                                // the clamped next row
        for (int xx = x0; xx <= x1; ++xx) {
            const int v = row[xx];
            const int vx = row[xx + 1];
            const int vy = below[xx];
            const int g = abs(vx - v) + abs(vy - v);
            fmin = min(fmin, v);
            fmax = max(fmax, v);
            gmax = max(gmax, g);
            gsum += g;
        }
    }
    // Delta gmax <= 255 * 510 and gsum <= 81^2 * 510 are exact in binary32
    const float mrtv = __fdiv_rn(__int2float_rn((fmax - fmin) * gmax),
                                 __fadd_rn(__int2float_rn(gsum), eps));
    float u = __fdiv_rn(mrtv, msat);
    if (u > 1.0f) u = 1.0f;
    sigma[i] = __fsub_rn(hi, __fmul_rn(__fsub_rn(hi, lo), u));
}

__global__ void u8_to_float_kernel(const uint8_t* f, long long pitch, int H, int W, float* out)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    out[i] = (float)f[(long long)y * pitch + x];
}

// The input of the next pass (reading R9): the output rounded half to even
// and clamped to [0, 255]; theta_next = f_next (the smoothing passes keep
// theta = f); the width scaled by decay (one binary32 product) when sig_out
// is given.
__global__ void next_input_kernel(const void* g, int g_f64, int H, int W, uint8_t* f_next, long long pitch_next,
                                  float* theta_next, const float* sig_in, float* sig_out, float decay)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long i = (long long)y * W + x;
    uint8_t u;
    if (g_f64) {
        double r = rint(static_cast<const double*>(g)[i]);
        u = (uint8_t)(r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r));
    } else {   // the same rounding in binary32 (rintf(v) == rint((double)v) for every float v)
        float r = rintf(static_cast<const float*>(g)[i]);
        u = (uint8_t)(r < 0.0f ? 0.0f : (r > 255.0f ? 255.0f : r));
    }
    f_next[(long long)y * pitch_next + x] = u;
    if (theta_next) theta_next[i] = (float)u;
    if (sig_out) sig_out[i] = __fmul_rn(sig_in[i], decay);
}

// Colour images (Sec. IV-C) are filtered channel by channel; the width maps
// come from the gray version, read as the BT.601 luma rounded half up in
// integers: Y = floor((299 R + 587 G + 114 B + 500) / 1000).
__device__ __forceinline__ uint8_t luma_of(unsigned r, unsigned g, unsigned b)
{
    return (uint8_t)((299u * r + 587u * g + 114u * b + 500u) / 1000u);
}

// Interleaved rgb (row pitch in bytes) into three planes (row pitch pn,
// plane c at planes + c * plane_stride) and/or its luma Y (row pitch pn).
__global__ void rgb_split_kernel(const uint8_t* rgb, long long pitch, int H, int W, uint8_t* planes, long long pn,
                                 long long plane_stride, uint8_t* Y)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const uint8_t* px = rgb + (long long)y * pitch + 3LL * x;
    const unsigned r = px[0], g = px[1], b = px[2];
    const long long o = (long long)y * pn + x;
    if (planes) {
        planes[o] = (uint8_t)r;
        planes[o + plane_stride] = (uint8_t)g;
        planes[o + 2 * plane_stride] = (uint8_t)b;
    }
    if (Y) Y[o] = luma_of(r, g, b);
}

// The luma of three planes (row pitch pn) into Y (row pitch pn).
__global__ void planes_luma_kernel(const uint8_t* planes, long long pn, long long plane_stride, int H, int W,
                                   uint8_t* Y)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x), y = (int)blockIdx.y;
    if (x >= W) return;
    const long long o = (long long)y * pn + x;
    Y[o] = luma_of(planes[o], planes[o + plane_stride], planes[o + 2 * plane_stride]);
}

// Channel c of an interleaved H x W x 3 float map into a plane.
__global__ void channel_kernel(const float* x3, int H, int W, int c, float* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)H * W) return;
    out[i] = x3[3 * i + c];
}

// Three output planes (H x W each, plane c at g + c * plane_elems elements)
// into the interleaved H x W x 3 output.
template <typename T>
__global__ void interleave_kernel(const T* g, long long plane_elems, long long n, T* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[3 * i] = g[i];
    out[3 * i + 1] = g[i + plane_elems];
    out[3 * i + 2] = g[i + 2 * plane_elems];
}

unsigned blocks_for(long long n) { return (unsigned)((n + kAppThreads - 1) / kAppThreads); }

// One block row per image row (H <= 65535): no index division in the kernels.
dim3 grid2d(int H, int W) { return dim3((unsigned)((W + kAppThreads - 1) / kAppThreads), (unsigned)H); }

// Shared memory of one texture_sigma_kernel block (k <= 40: at most 27.6 KB).
size_t texture_smem(int k) { return (size_t)(2 * k + 2) * (size_t)(kAppThreads + 2 * k + 1); }

int check_sharpen_cfg(const fabf_sharpen_cfg* c)
{
    if (!c) return FABF_EINVAL;
    if (c->w < 1 || c->N < 0 || !(c->lap_sat > 0.0) || !std::isfinite(c->lap_sat)) return FABF_EINVAL;
    if (!(c->sigma_lo > 0.0) || !(c->sigma_hi >= c->sigma_lo) || !std::isfinite(c->sigma_hi)) return FABF_EINVAL;
    if (c->w > kWMax || c->N > kNMax) return FABF_EUNSUPPORTED;
    return FABF_OK;
}

int check_texture_cfg(const fabf_texture_cfg* c)
{
    if (!c) return FABF_EINVAL;
    if (c->w < 1 || c->N < 0 || c->k < 1 || !(c->eps > 0.0) || !(c->mrtv_sat > 0.0)) return FABF_EINVAL;
    if (!(c->sigma_lo > 0.0) || !(c->sigma_hi >= c->sigma_lo) || !std::isfinite(c->sigma_hi)) return FABF_EINVAL;
    if (!(c->sigma_decay > 0.0) || !std::isfinite(c->sigma_decay)) return FABF_EINVAL;
    if (c->w > kWMax || c->N > kNMax || c->k > kWMax) return FABF_EUNSUPPORTED;
    return check_sharpen_cfg(&c->sharpen);
}

// The LoG taps and the saturation level Lq = floor(lap_sat (sum g)^2 + 1/2).
int sharpen_taps(const fabf_sharpen_cfg* c, SepTaps* T, long long* Lq)
{
    uint32_t g[2 * kWMax + 1];
    int r = 0;
    const int rc = fabf_gaussian_taps(c->rho_log, g, 2 * kWMax + 1, &r);
    if (rc) return rc;
    std::memset(T, 0, sizeof(*T));
    T->r = r;
    uint64_t sum = 0;
    for (int t = 0; t <= 2 * r; ++t) {
        T->g[t] = g[t];
        sum += g[t];
    }
    const double q = std::floor(c->lap_sat * (double)sum * (double)sum + 0.5);
    if (!(q >= 1.0 && q < 4.0e18)) return FABF_EINVAL;
    *Lq = (long long)q;
    return FABF_OK;
}

bool all_device(std::initializer_list<const void*> ps)
{
    for (const void* p : ps)
        if (!is_device_ptr(p)) return false;
    return true;
}

// Stream-ordered scratch for one pipeline call.
struct Scratch {
    void* base = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch()
    {
        if (base) cudaFreeAsync(base, s);
    }
};

// theta and sigma of the sharpening rules for f (device), into theta / sigma.
int launch_sharpen_maps(const uint8_t* f, long long pitch, int H, int W, int w, const SepTaps& T, long long Lq,
                        double s_lo, double s_hi, int32_t* rs, uint32_t* gr, int64_t* S, float* theta,
                        float* sigma, cudaStream_t s)
{
    const long long n = (long long)H * W;
    const unsigned b = blocks_for(n);
    box_rows_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, pitch, H, W, w, rs);
    sharpen_theta_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, pitch, rs, H, W, w, theta);
    gauss_rows_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, pitch, H, W, T, gr);
    gauss_cols_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(gr, H, W, T, S);
    sharpen_sigma_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(S, H, W, Lq, (float)s_lo, (float)s_hi, sigma);
    return cuda_status(cudaGetLastError());
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Interleaves three planes of out_f64 ? double : float elements.
int launch_interleave(const void* g, size_t plane_bytes, int out_f64, long long n, void* out, cudaStream_t s)
{
    if (out_f64)
        interleave_kernel<double><<<blocks_for(n), kAppThreads, 0, s>>>(
            static_cast<const double*>(g), (long long)(plane_bytes / 8), n, static_cast<double*>(out));
    else
        interleave_kernel<float><<<blocks_for(n), kAppThreads, 0, s>>>(
            static_cast<const float*>(g), (long long)(plane_bytes / 4), n, static_cast<float*>(out));
    return cuda_status(cudaGetLastError());
}

int check_rgb_args(const uint8_t* rgb, const void* out, int H, int W, size_t pitch)
{
    if (!rgb || !out || H < 1 || W < 1 || H > 65535 || W > 65535) return FABF_EINVAL;
    if (pitch < 3 * (size_t)W) return FABF_EINVAL;
    return FABF_OK;
}

}  // namespace
}  // namespace fabf

using namespace fabf;

extern "C" {

int fabf_sharpen_maps(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch, const fabf_sharpen_cfg* cfg,
                      float* theta, float* sigma, void* cuda_stream)
{
    if (!ctx || !img || !theta || !sigma || H < 1 || W < 1 || pitch < (size_t)W) return FABF_EINVAL;
    int rc = check_sharpen_cfg(cfg);
    if (rc) return rc;
    if (!all_device({img, theta, sigma})) return FABF_EINVAL;
    SepTaps T;
    long long Lq = 0;
    rc = sharpen_taps(cfg, &T, &Lq);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)H * W;
    Scratch sc;
    sc.s = s;
    const size_t o_gr = align256(n * 4), o_S = o_gr + align256(n * 4);
    cudaError_t e = cudaMallocAsync(&sc.base, o_S + n * 8, s);
    if (e != cudaSuccess) return cuda_status(e);
    uint8_t* b = static_cast<uint8_t*>(sc.base);
    return launch_sharpen_maps(img, (long long)pitch, H, W, cfg->w, T, Lq, cfg->sigma_lo, cfg->sigma_hi,
                               reinterpret_cast<int32_t*>(b), reinterpret_cast<uint32_t*>(b + o_gr),
                               reinterpret_cast<int64_t*>(b + o_S), theta, sigma, s);
}

int fabf_texture_sigma(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch, const fabf_texture_cfg* cfg,
                       float* sigma, void* cuda_stream)
{
    if (!ctx || !img || !sigma || H < 1 || W < 1 || pitch < (size_t)W) return FABF_EINVAL;
    int rc = check_texture_cfg(cfg);
    if (rc) return rc;
    if (!all_device({img, sigma})) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    texture_sigma_kernel<<<grid2d(H, W), kAppThreads, texture_smem(cfg->k), s>>>(
        img, (long long)pitch, H, W, cfg->k, (float)cfg->eps, (float)cfg->mrtv_sat, (float)cfg->sigma_lo,
        (float)cfg->sigma_hi, sigma);
    return cuda_status(cudaGetLastError());
}

int fabf_sharpen(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch, const fabf_sharpen_cfg* cfg, void* out,
                 int out_is_f64, void* cuda_stream)
{
    if (!ctx || !img || !out || H < 1 || W < 1 || pitch < (size_t)W || H > 65535 || W > 65535) return FABF_EINVAL;
    int rc = check_sharpen_cfg(cfg);
    if (rc) return rc;
    if (!all_device({img, out})) return FABF_EINVAL;
    SepTaps T;
    long long Lq = 0;
    rc = sharpen_taps(cfg, &T, &Lq);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)H * W;
    const size_t o_sg = align256(n * 4), o_rs = o_sg + align256(n * 4), o_gr = o_rs + align256(n * 4),
                 o_S = o_gr + align256(n * 4);
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocAsync(&sc.base, o_S + n * 8, s);
    if (e != cudaSuccess) return cuda_status(e);
    uint8_t* b = static_cast<uint8_t*>(sc.base);
    float* th = reinterpret_cast<float*>(b);
    float* sg = reinterpret_cast<float*>(b + o_sg);
    rc = launch_sharpen_maps(img, (long long)pitch, H, W, cfg->w, T, Lq, cfg->sigma_lo, cfg->sigma_hi,
                             reinterpret_cast<int32_t*>(b + o_rs), reinterpret_cast<uint32_t*>(b + o_gr),
                             reinterpret_cast<int64_t*>(b + o_S), th, sg, s);
    if (rc) return rc;
    return run_fused(ctx, img, pitch, th, sg, H, W, cfg->w, cfg->N, out, out_is_f64, nullptr, s);
}

int fabf_texture_filter(fabf_ctx* ctx, const uint8_t* img, int H, int W, size_t pitch, const fabf_texture_cfg* cfg,
                        void* out, int out_is_f64, void* cuda_stream)
{
    if (!ctx || !img || !out || H < 1 || W < 1 || pitch < (size_t)W || H > 65535 || W > 65535) return FABF_EINVAL;
    int rc = check_texture_cfg(cfg);
    if (rc) return rc;
    if (!all_device({img, out})) return FABF_EINVAL;
    const fabf_sharpen_cfg& sc_cfg = cfg->sharpen;
    SepTaps T;
    long long Lq = 0;
    rc = sharpen_taps(&sc_cfg, &T, &Lq);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long n = (long long)H * W;
    const size_t pn = ((size_t)W + 15) & ~(size_t)15;          // 16-byte rows: the next passes use TMA
    const int g_f64 = ctx->precision == kPrecFP64 ? 1 : 0;
    const size_t gsz = (size_t)n * (g_f64 ? 8 : 4);
    // scratch: sigma1, sigma2, theta, g, f_next (x2), rs, gr, S
    const size_t o_s2 = align256(n * 4), o_th = o_s2 + align256(n * 4), o_g = o_th + align256(n * 4),
                 o_f2 = o_g + align256(gsz), o_f3 = o_f2 + align256(pn * H), o_rs = o_f3 + align256(pn * H),
                 o_gr = o_rs + align256(n * 4), o_S = o_gr + align256(n * 4), total = o_S + n * 8;
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocAsync(&sc.base, total, s);
    if (e != cudaSuccess) return cuda_status(e);
    uint8_t* b = static_cast<uint8_t*>(sc.base);
    float* s1 = reinterpret_cast<float*>(b);
    float* s2 = reinterpret_cast<float*>(b + o_s2);
    float* th = reinterpret_cast<float*>(b + o_th);
    void* g = b + o_g;
    uint8_t* f2 = b + o_f2;
    uint8_t* f3 = b + o_f3;
    const unsigned nb = blocks_for(n);
    // pass 1: theta = f, sigma from mRTV
    texture_sigma_kernel<<<grid2d(H, W), kAppThreads, texture_smem(cfg->k), s>>>(
        img, (long long)pitch, H, W, cfg->k, (float)cfg->eps, (float)cfg->mrtv_sat, (float)cfg->sigma_lo,
        (float)cfg->sigma_hi, s1);
    u8_to_float_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(img, (long long)pitch, H, W, th);
    rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    rc = run_fused(ctx, img, pitch, th, s1, H, W, cfg->w, cfg->N, g, g_f64, nullptr, s);
    if (rc) return rc;
    // pass 2: the rounded output, theta = f2, sigma scaled by sigma_decay
    next_input_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(g, g_f64, H, W, f2, (long long)pn, th, s1, s2,
                                                 (float)cfg->sigma_decay);
    rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    rc = run_fused(ctx, f2, pn, th, s2, H, W, cfg->w, cfg->N, g, g_f64, nullptr, s);
    if (rc) return rc;
    // pass 3: sharpening of the rounded output
    next_input_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(g, g_f64, H, W, f3, (long long)pn, nullptr, nullptr, nullptr, 1.0f);
    rc = launch_sharpen_maps(f3, (long long)pn, H, W, sc_cfg.w, T, Lq, sc_cfg.sigma_lo, sc_cfg.sigma_hi,
                             reinterpret_cast<int32_t*>(b + o_rs), reinterpret_cast<uint32_t*>(b + o_gr),
                             reinterpret_cast<int64_t*>(b + o_S), th, s2, s);
    if (rc) return rc;
    return run_fused(ctx, f3, pn, th, s2, H, W, sc_cfg.w, sc_cfg.N, out, out_is_f64, nullptr, s);
}

}  // extern "C"

extern "C" {

int fabf_luma(fabf_ctx* ctx, const uint8_t* rgb, int H, int W, size_t pitch, uint8_t* Y, size_t y_pitch,
              void* cuda_stream)
{
    if (!ctx || !Y || y_pitch < (size_t)W) return FABF_EINVAL;
    int rc = check_rgb_args(rgb, Y, H, W, pitch);
    if (rc) return rc;
    if (!all_device({rgb, Y})) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    rgb_split_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(rgb, (long long)pitch, H, W, nullptr,
                                                                          (long long)y_pitch, 0, Y);
    return cuda_status(cudaGetLastError());
}

int fabf_filter_rgb(fabf_ctx* ctx, const uint8_t* rgb, const float* theta, const float* sigma, int H, int W,
                    size_t pitch, int w, int N, void* out, int out_is_f64, void* cuda_stream)
{
    if (!ctx || !sigma) return FABF_EINVAL;
    int rc = check_rgb_args(rgb, out, H, W, pitch);
    if (rc) return rc;
    if (w < 1 || N < 0) return FABF_EINVAL;
    if (w > kWMax || N > kNMax) return FABF_EUNSUPPORTED;
    if (!all_device({rgb, sigma, out}) || (theta && !is_device_ptr(theta))) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long n = (long long)H * W;
    const size_t pn = ((size_t)W + 15) & ~(size_t)15;          // 16-byte rows for the TMA loads
    const size_t plane = align256(pn * H), gplane = align256((size_t)n * (out_is_f64 ? 8 : 4));
    // scratch: the three channel planes, one theta plane, three output planes
    const size_t o_th = 3 * plane, o_g = o_th + align256((size_t)n * 4), total = o_g + 3 * gplane;
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocAsync(&sc.base, total, s);
    if (e != cudaSuccess) return cuda_status(e);
    uint8_t* b = static_cast<uint8_t*>(sc.base);
    float* th = reinterpret_cast<float*>(b + o_th);
    const unsigned nb = blocks_for(n);
    rgb_split_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(rgb, (long long)pitch, H, W, b, (long long)pn, (long long)plane,
                                                nullptr);
    for (int c = 0; c < 3; ++c) {
        const uint8_t* f = b + c * plane;
        if (theta)
            channel_kernel<<<nb, kAppThreads, 0, s>>>(theta, H, W, c, th);
        else
            u8_to_float_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, (long long)pn, H, W, th);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        rc = run_fused(ctx, f, pn, th, sigma, H, W, w, N, b + o_g + c * gplane, out_is_f64, nullptr, s);
        if (rc) return rc;
    }
    return launch_interleave(b + o_g, gplane, out_is_f64, n, out, s);
}

int fabf_texture_filter_rgb(fabf_ctx* ctx, const uint8_t* rgb, int H, int W, size_t pitch,
                            const fabf_texture_cfg* cfg, void* out, int out_is_f64, void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_rgb_args(rgb, out, H, W, pitch);
    if (rc) return rc;
    rc = check_texture_cfg(cfg);
    if (rc) return rc;
    if (!all_device({rgb, out})) return FABF_EINVAL;
    const fabf_sharpen_cfg& shc = cfg->sharpen;
    SepTaps T;
    long long Lq = 0;
    rc = sharpen_taps(&shc, &T, &Lq);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long n = (long long)H * W;
    const size_t pn = ((size_t)W + 15) & ~(size_t)15;
    const size_t plane = align256(pn * H), f4 = align256((size_t)n * 4);
    const int g_f64 = ctx->precision == kPrecFP64 ? 1 : 0;
    const size_t gmid = align256((size_t)n * (g_f64 ? 8 : 4)), gplane = align256((size_t)n * (out_is_f64 ? 8 : 4));
    // scratch: input planes (3), luma, pass-2 input, pass-3 inputs (3), sigma1, sigma2, theta, the
    // intermediate output, the final output planes (3), and the sharpening maps' row sums and Gaussians
    const size_t o_Y = 3 * plane, o_F2 = o_Y + plane, o_F3 = o_F2 + plane, o_s1 = o_F3 + 3 * plane,
                 o_s2 = o_s1 + f4, o_th = o_s2 + f4, o_gm = o_th + f4, o_go = o_gm + gmid, o_rs = o_go + 3 * gplane,
                 o_gr = o_rs + f4, o_S = o_gr + f4, total = o_S + (size_t)n * 8;
    Scratch sc;
    sc.s = s;
    cudaError_t e = cudaMallocAsync(&sc.base, total, s);
    if (e != cudaSuccess) return cuda_status(e);
    uint8_t* b = static_cast<uint8_t*>(sc.base);
    uint8_t* Y = b + o_Y;
    uint8_t* F2 = b + o_F2;
    uint8_t* F3 = b + o_F3;
    float* s1 = reinterpret_cast<float*>(b + o_s1);
    float* s2 = reinterpret_cast<float*>(b + o_s2);
    float* th = reinterpret_cast<float*>(b + o_th);
    void* gm = b + o_gm;
    const unsigned nb = blocks_for(n);
    const long long lpn = (long long)pn;
    // the planes, and the texture width map of the luma
    rgb_split_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(rgb, (long long)pitch, H, W, b, lpn, (long long)plane, Y);
    texture_sigma_kernel<<<grid2d(H, W), kAppThreads, texture_smem(cfg->k), s>>>(
        Y, lpn, H, W, cfg->k, (float)cfg->eps, (float)cfg->mrtv_sat, (float)cfg->sigma_lo, (float)cfg->sigma_hi, s1);
    rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    // per channel: the two smoothing passes (theta = f), rounded into F3
    for (int c = 0; c < 3; ++c) {
        const uint8_t* f = b + c * plane;
        u8_to_float_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, lpn, H, W, th);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        rc = run_fused(ctx, f, pn, th, s1, H, W, cfg->w, cfg->N, gm, g_f64, nullptr, s);
        if (rc) return rc;
        next_input_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(gm, g_f64, H, W, F2, lpn, th, c == 0 ? s1 : nullptr,
                                                     c == 0 ? s2 : nullptr, (float)cfg->sigma_decay);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        rc = run_fused(ctx, F2, pn, th, s2, H, W, cfg->w, cfg->N, gm, g_f64, nullptr, s);
        if (rc) return rc;
        next_input_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(gm, g_f64, H, W, F3 + c * plane, lpn, nullptr, nullptr,
                                                     nullptr, 1.0f);
    }
    // the sharpening width map of the luma of F3 (into s1), shared by the channels
    int32_t* rs = reinterpret_cast<int32_t*>(b + o_rs);
    planes_luma_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(F3, lpn, (long long)plane, H, W, Y);
    gauss_rows_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(Y, lpn, H, W, T, reinterpret_cast<uint32_t*>(b + o_gr));
    gauss_cols_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(reinterpret_cast<uint32_t*>(b + o_gr), H, W, T,
                                                 reinterpret_cast<int64_t*>(b + o_S));
    sharpen_sigma_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(reinterpret_cast<int64_t*>(b + o_S), H, W, Lq,
                                                              (float)shc.sigma_lo, (float)shc.sigma_hi, s1);
    rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
    // per channel: its own sharpening centre, then the sharpening pass
    for (int c = 0; c < 3; ++c) {
        const uint8_t* f = F3 + c * plane;
        box_rows_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, lpn, H, W, shc.w, rs);
        sharpen_theta_kernel<<<grid2d(H, W), kAppThreads, 0, s>>>(f, lpn, rs, H, W, shc.w, th);
        rc = cuda_status(cudaGetLastError());
        if (rc) return rc;
        rc = run_fused(ctx, f, pn, th, s1, H, W, shc.w, shc.N, b + o_go + c * gplane, out_is_f64, nullptr, s);
        if (rc) return rc;
    }
    return launch_interleave(b + o_go, gplane, out_is_f64, n, out, s);
}

}  // extern "C"

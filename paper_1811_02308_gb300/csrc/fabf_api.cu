// Host runtime behind the C ABI declared in include/fabf.h: argument checks,
// pointer-kind detection and staging of host buffers, TMA descriptor
// encoding, kernel dispatch over the polynomial degree N, and the status
// words the kernels report into.  No CPU fallback exists: every pixel is
// computed by the CUDA kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/fabf.h"
#include "fabf_internal.h"
#include "fabf_kernels.cuh"

using namespace fabf;

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
namespace fabf {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return FABF_OK;
    if (e == cudaErrorMemoryAllocation) return FABF_ENOMEM;
    return FABF_ECUDA;
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// What a buffer is: device (or managed) memory, and the pointer kernels can
// dereference -- the buffer itself, the mapping of pinned host memory (read
// and written in place over the chip-to-chip link), or nullptr for pageable
// host memory.
PtrInfo ptr_info(const void* p)
{
    PtrInfo r;
    if (!p) return r;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return r;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        r.device = true;
        r.kptr = p;
    } else if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        r.kptr = a.devicePointer;
    }
    return r;
}

int check_filter_args(const void* img, const void* theta, const void* sigma, const void* out,
                      int H, int W, size_t pitch, int w, int N)
{
    if (!img || !theta || !sigma || !out) return FABF_EINVAL;
    if (H < 1 || W < 1 || H > 65535 || W > 65535) return FABF_EINVAL;
    if (pitch < (size_t)W) return FABF_EINVAL;
    if (w < 1 || N < 0) return FABF_EINVAL;
    if (w > kWMax || N > kNMax) return FABF_EUNSUPPORTED;
    return FABF_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// 2-D uint8 tensor map over the image, box Cb x R (inner x outer).
bool encode_image_tmap(CUtensorMap* tm, const uint8_t* img, int H, int W, size_t pitch, int Cb, int R)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode_fn();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(img) & 15) || (pitch & 15)) return false;
    if (Cb > 256 || R > 256) return false;
    cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)Cb, (cuuint32_t)R};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(img), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void fused_geometry(int w, int* off, int* Cb)
{
    *off = (16 - (w & 15)) & 15;
    *Cb = (*off + kTileW + 2 * w + 15) & ~15;
}

// ---- kernel dispatch over precision --------------------------------------
cudaError_t launch_fused(int prec, int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                         cudaStream_t s)
{
    switch (prec) {
    case kPrecFP64: return launch_fused_p0(N, tm, p, grid, smem, s);
    case kPrecFP64Fit: return launch_fused_p1(N, tm, p, grid, smem, s);
    case kPrecCFP32: return launch_fused_p2(N, tm, p, grid, smem, s);
    case kPrecC32: return launch_fused_p3(N, tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch(int prec, const BatchParams& p, int grid, size_t smem, cudaStream_t s)
{
    switch (prec) {
    case kPrecFP64: return launch_batch_p0(p, grid, smem, s);
    case kPrecFP64Fit: return launch_batch_p1(p, grid, smem, s);
    case kPrecCFP32: return launch_batch_p2(p, grid, smem, s);
    case kPrecC32: return launch_batch_p3(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

size_t make_job(ImageJob* J, CUtensorMap* tm, const uint8_t* img, size_t pitch, const float* theta,
                const float* sigma, int H, int W, int w, int N, void* out, int out_f64, int TH, bool allow_tma)
{
    std::memset(J, 0, sizeof(*J));
    J->img = img;
    J->pitch = (long long)pitch;
    J->theta = theta;
    J->sigma = sigma;
    J->out = out;
    J->H = H;
    J->W = W;
    J->w = w;
    J->N = N;
    J->out_f64 = out_f64;
    J->TH = TH;
    fused_geometry(w, &J->off, &J->Cb);
    J->tiles_x = (W + kTileW - 1) / kTileW;
    J->tiles_y = (H + TH - 1) / TH;
    std::memset(tm, 0, sizeof(*tm));
    J->use_tma = allow_tma && encode_image_tmap(tm, img, H, W, pitch, J->Cb, TH + 2 * w) ? 1 : 0;
    return fused_smem_bytes(N, w, J->Cb, TH);
}

}  // namespace fabf

namespace fabf {

int ensure_stage(fabf_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->stage_bytes) return FABF_OK;
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    if (cudaMalloc(&ctx->stage, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return FABF_ENOMEM;
    }
    ctx->stage_bytes = bytes;
    return FABF_OK;
}

int read_and_clear_status(fabf_ctx* ctx, cudaStream_t s, int* status, uint64_t* nfb, uint64_t* nredo)
{
    // one copy of the whole word block into pinned memory, one clear, one wait
    std::lock_guard<std::mutex> lk(ctx->status_lock);
    const uint8_t* hw = static_cast<const uint8_t*>(ctx->h_words);
    cudaError_t e = cudaMemcpyAsync(ctx->h_words, ctx->d_status, fabf_ctx::kWordBytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, fabf_ctx::kWordBytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned st;
    unsigned long long n[2];
    std::memcpy(&st, hw, sizeof(st));
    std::memcpy(n, hw + fabf_ctx::kNfbOffset, sizeof(n));
    if (status) *status = (st & kStatusTimeout) ? FABF_ETIMEOUT : (st & kStatusBadInput) ? FABF_EINVAL : FABF_OK;
    if (nfb) *nfb = n[0];
    if (nredo) *nredo = n[1];
    return FABF_OK;
}

unsigned* pinned_call_status(fabf_ctx* ctx) { return ctx->m_status ? ctx->m_status : ctx->d_status; }

unsigned long long* pinned_call_nfb(fabf_ctx* ctx) { return ctx->m_status ? ctx->m_nfb : ctx->d_nfb; }

int finish_pinned_call(fabf_ctx* ctx, cudaStream_t s)
{
    int st = FABF_OK;
    if (!ctx->m_status) {
        const int rc = read_and_clear_status(ctx, s, &st, nullptr, nullptr);
        return rc ? rc : st;
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    volatile unsigned* w = static_cast<volatile unsigned*>(ctx->h_mwords);
    const unsigned bits = w[0];
    for (size_t i = 0; i < fabf_ctx::kWordBytes / sizeof(unsigned); ++i) w[i] = 0u;
    return (bits & kStatusTimeout) ? FABF_ETIMEOUT : (bits & kStatusBadInput) ? FABF_EINVAL : FABF_OK;
}

int run_fused_prec(fabf_ctx* ctx, int prec, const uint8_t* img, size_t pitch, const float* theta,
                   const float* sigma, int H, int W, int w, int N, void* out, int out_f64, int TH,
                   const DebugPlanes* dbg, unsigned* status, unsigned long long* nfb, cudaStream_t s,
                   bool allow_tma)
{
    (void)ctx;
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    CUtensorMap tm;
    const size_t smem = make_job(&p.job, &tm, img, pitch, theta, sigma, H, W, w, N, out, out_f64, TH, allow_tma);
    p.status = status;
    p.n_fallback = nfb;
    if (dbg) p.dbg = *dbg;
    dim3 grid(p.job.tiles_x, p.job.tiles_y);
    return cuda_status(launch_fused(prec, N, tm, p, grid, smem, s));
}

// Launch the fused kernel on device buffers.
int run_fused(fabf_ctx* ctx, const uint8_t* img, size_t pitch, const float* theta, const float* sigma,
              int H, int W, int w, int N, void* out, int out_f64, const DebugPlanes* dbg,
              cudaStream_t s)
{
    const int prec = dbg ? kPrecFP64 : ctx->precision;
    const int TH = dbg ? kDefaultTileRows : tile_rows_for(ctx, w, N, prec, H, W);
    return run_fused_prec(ctx, prec, img, pitch, theta, sigma, H, W, w, N, out, out_f64, TH, dbg,
                          ctx->d_status, ctx->d_nfb, s, dbg ? true : tile_staging_tma(ctx, w, N, prec));
}

// Launch the fused FP64 kernel on device buffers with caller-provided status
// words (used by the allocation-free entry point in fabf_noalloc.cu).
int launch_fused_scratch(const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
                         int W, int w, int N, void* out, int out_f64, unsigned* status,
                         unsigned long long* n_fallback, cudaStream_t s)
{
    return run_fused_prec(nullptr, kPrecFP64, img, pitch, theta, sigma, H, W, w, N, out, out_f64,
                          tile_rows_for(nullptr, w, N, kPrecFP64, H, W), nullptr, status, n_fallback, s);
}

}  // namespace fabf

// ---------------------------------------------------------------------------
// Host buffers, pipelined: the image is cut into up to kBands bands of tile
// rows.  Band b's inputs (its rows of theta and sigma, and the image rows up
// to its last tile's halo not copied yet) go up on the copy-in stream; its
// tiles run on their own stream as soon as they are there (bands are
// independent, so their kernels may overlap); its output rows come back on
// the copy-out stream.  Copies in, kernels and copies out of different bands
// overlap; the call returns when the last band is back, with the kernels'
// status, as the unpipelined host path does.
// ---------------------------------------------------------------------------
static int ensure_pipeline(fabf_ctx* ctx)
{
    if (ctx->pipe_ready) return FABF_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking);
    for (int b = 0; b < fabf_ctx::kBands && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&ctx->s_band[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_k[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    ctx->pipe_ready = true;
    return FABF_OK;
}

static void destroy_pipeline(fabf_ctx* ctx)
{
    if (!ctx->pipe_ready) return;
    cudaStreamDestroy(ctx->s_in);
    cudaStreamDestroy(ctx->s_out);
    for (int b = 0; b < fabf_ctx::kBands; ++b) {
        cudaStreamDestroy(ctx->s_band[b]);
        cudaEventDestroy(ctx->ev_in[b]);
        cudaEventDestroy(ctx->ev_k[b]);
    }
    cudaEventDestroy(ctx->ev_start);
    cudaEventDestroy(ctx->ev_done);
    ctx->pipe_ready = false;
}

static int filter_host_pipelined(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H,
                                 int W, size_t pitch, int w, int N, void* out, int out_f64, cudaStream_t s)
{
    std::lock_guard<std::mutex> staged(ctx->stage_lock);
    int rc = ensure_pipeline(ctx);
    if (rc) return rc;
    const int prec = ctx->precision;
    const int TH = tile_rows_for(ctx, w, N, prec, H, W);
    const size_t npix = (size_t)H * W, osz = out_f64 ? 8 : 4;
    const size_t ipitch = ((size_t)W + 15) & ~(size_t)15;
    const size_t o_th = (ipitch * H + 255) & ~(size_t)255;
    const size_t o_sg = o_th + ((npix * 4 + 255) & ~(size_t)255);
    const size_t o_out = o_sg + ((npix * 4 + 255) & ~(size_t)255);
    rc = ensure_stage(ctx, o_out + npix * osz);
    if (rc) return rc;
    uint8_t* base = static_cast<uint8_t*>(ctx->stage);
    const float* d_th = reinterpret_cast<const float*>(base + o_th);
    const float* d_sg = reinterpret_cast<const float*>(base + o_sg);
    uint8_t* d_out = base + o_out;

    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    CUtensorMap tm;
    const size_t smem = make_job(&p.job, &tm, base, ipitch, d_th, d_sg, H, W, w, N, d_out, out_f64, TH);
    p.status = ctx->d_status;
    p.n_fallback = ctx->d_nfb;
    const int tiles_y = p.job.tiles_y;
    const int nb = tiles_y < fabf_ctx::kBands ? tiles_y : fabf_ctx::kBands;
    const int bt = (tiles_y + nb - 1) / nb;                      // tile rows per band

    cudaError_t e = cudaEventRecord(ctx->ev_start, s);           // after the caller's earlier work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_in, ctx->ev_start, 0);
    int copied = 0;                                              // image rows already sent
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        const int t0 = b * bt, t1 = t0 + bt < tiles_y ? t0 + bt : tiles_y;
        if (t0 >= t1) break;
        const int y0 = t0 * TH, y1 = t1 * TH < H ? t1 * TH : H;
        const int need = y1 + w < H ? y1 + w : H;                // rows the band's halo reaches
        if (need > copied)
            e = cudaMemcpy2DAsync(base + (size_t)copied * ipitch, ipitch, img + (size_t)copied * pitch, pitch, W,
                                  need - copied, cudaMemcpyHostToDevice, ctx->s_in);
        copied = need > copied ? need : copied;
        const size_t r0 = (size_t)y0 * W, rn = (size_t)(y1 - y0) * W;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_th + r0 * 4, theta + r0, rn * 4, cudaMemcpyHostToDevice, ctx->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_sg + r0 * 4, sigma + r0, rn * 4, cudaMemcpyHostToDevice, ctx->s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in[b], ctx->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_band[b], ctx->ev_in[b], 0);
        if (e == cudaSuccess) {
            p.job.tile_y0 = t0;
            e = launch_fused(prec, N, tm, p, dim3(p.job.tiles_x, t1 - t0), smem, ctx->s_band[b]);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_k[b], ctx->s_band[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_k[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + r0 * osz, d_out + r0 * osz, rn * osz,
                                cudaMemcpyDeviceToHost, ctx->s_out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_done, ctx->s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_done, 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->s_out);
        return cuda_status(e);
    }
    int st = FABF_OK;
    rc = read_and_clear_status(ctx, s, &st, nullptr, nullptr);
    return rc ? rc : st;
}

// ---------------------------------------------------------------------------
// Host-mapped theta, sigma and out (pinned host memory) with a host or device
// image: the kernel reads the maps and writes the output in place in host
// memory, so only the image is copied (its tiles are staged by TMA from
// device memory).  Synchronous: returns the kernels' status.  (Copying the
// image in bands that start their tiles early measured no faster.)
// ---------------------------------------------------------------------------
// Rows of 16-byte words of a pinned host image into the staging buffer.
__global__ void __launch_bounds__(256) stage_rows_kernel(const uint4* __restrict__ src, long long src_pitch16,
                                                         uint4* __restrict__ dst, long long dst_pitch16, int H,
                                                         int row16)
{
    const long long total = (long long)H * row16;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < total; i += (long long)gridDim.x * 256) {
        const long long y = i / row16, x = i - y * row16;
        dst[y * dst_pitch16 + x] = src[y * src_pitch16 + x];
    }
}

int fabf::stage_image(fabf_ctx* ctx, const uint8_t* img, const PtrInfo& pi, int H, int W, size_t pitch,
                      cudaStream_t s, const uint8_t** d_img, size_t* d_pitch)
{
    *d_img = img;
    *d_pitch = pitch;
    if (pi.device) return FABF_OK;
    const size_t ipitch = ((size_t)W + 15) & ~(size_t)15;
    const int rc = ensure_stage(ctx, ipitch * H);
    if (rc) return rc;
    // the kernel reads exactly W bytes of every row: W a multiple of 16 (no
    // read past the caller's last row), 16-byte aligned rows
    if (pi.kptr && W % 16 == 0 && pitch % 16 == 0 && (reinterpret_cast<uintptr_t>(pi.kptr) & 15) == 0) {
        // one 16-byte word per thread where the image allows (every load in
        // flight at once: the link's latency, not its bandwidth, bounds a
        // copy of this size)
        const long long words = (long long)H * (W / 16);
        const long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 1);
        const int blocks = (int)std::min<long long>(cap, (words + 255) / 256);
        stage_rows_kernel<<<blocks, 256, 0, s>>>(static_cast<const uint4*>(pi.kptr), (long long)(pitch / 16),
                                                 static_cast<uint4*>(ctx->stage), (long long)(ipitch / 16), H,
                                                 W / 16);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        *d_img = static_cast<const uint8_t*>(ctx->stage);
        *d_pitch = ipitch;
        return FABF_OK;
    }
    const cudaError_t e = ipitch == pitch
                              ? cudaMemcpyAsync(ctx->stage, img, pitch * H, cudaMemcpyHostToDevice, s)
                              : cudaMemcpy2DAsync(ctx->stage, ipitch, img, pitch, W, H, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    *d_img = static_cast<const uint8_t*>(ctx->stage);
    *d_pitch = ipitch;
    return FABF_OK;
}

static int filter_mapped(fabf_ctx* ctx, const uint8_t* img, const PtrInfo& pi, const float* k_th, const float* k_sg,
                         int H, int W, size_t pitch, int w, int N, void* k_out, int out_f64, cudaStream_t s)
{
    std::lock_guard<std::mutex> staged(ctx->stage_lock);
    const uint8_t* d_img = nullptr;
    size_t d_pitch = 0;
    const int src = stage_image(ctx, img, pi, H, W, pitch, s, &d_img, &d_pitch);
    if (src) return src;
    const int prec = ctx->precision;
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    CUtensorMap tm;
    const size_t smem = make_job(&p.job, &tm, d_img, d_pitch, k_th, k_sg, H, W, w, N, k_out, out_f64,
                                 tile_rows_for(ctx, w, N, prec, H, W));
    p.job.maps_host = 1;
    p.status = pinned_call_status(ctx);
    p.n_fallback = pinned_call_nfb(ctx);
    const cudaError_t e = launch_fused(prec, N, tm, p, dim3(p.job.tiles_x, p.job.tiles_y), smem, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_status(e);
    }
    return finish_pinned_call(ctx, s);
}

namespace fabf {

// The FP64 form's erfcx and exp on n arguments (test entry point): erfcx at
// |x|, exp at -|x|, the domains the integrals use.
static __global__ void __launch_bounds__(256) fp64_functions_kernel(const double* x, long long n, double* erfcx_out,
                                                             double* exp_out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = fabs(x[i]);
    erfcx_out[i] = erfcx_fp64(a);
    exp_out[i] = exp_fp64(-a);
}

}  // namespace fabf

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int fabf_create(const fabf_config* cfg, fabf_ctx** out)
{
    if (!out) return FABF_EINVAL;
    *out = nullptr;
    fabf_config c{};
    if (cfg) c = *cfg;
    if (c.precision < FABF_FP64 || c.precision > FABF_C32) return FABF_EINVAL;
    fabf_ctx* ctx = new (std::nothrow) fabf_ctx();
    if (!ctx) return FABF_ENOMEM;
    ctx->device = c.device;
    ctx->precision = c.precision;
    ctx->budget = c.mem_budget_bytes ? c.mem_budget_bytes : (size_t)16 << 30;
    ctx->autotune = c.autotune;
    if (c.tune_cache_path) ctx->tune_cache_path = c.tune_cache_path;
    cudaError_t e = cudaSetDevice(c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, c.device);
    void* words = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&words, fabf_ctx::kWordBytes);
    if (e == cudaSuccess) e = cudaMemset(words, 0, fabf_ctx::kWordBytes);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_words, fabf_ctx::kWordBytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (words) cudaFree(words);
        if (ctx->h_words) cudaFreeHost(ctx->h_words);
        delete ctx;
        return cuda_status(e);
    }
    ctx->d_status = static_cast<unsigned*>(words);
    ctx->d_nfb = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(words) + fabf_ctx::kNfbOffset);
    int native_atomics = 0;
    if (cudaDeviceGetAttribute(&native_atomics, cudaDevAttrHostNativeAtomicSupported, c.device) == cudaSuccess &&
        native_atomics) {
        void* hm = nullptr;
        void* dm = nullptr;
        if (cudaHostAlloc(&hm, fabf_ctx::kWordBytes, cudaHostAllocMapped) == cudaSuccess) {
            std::memset(hm, 0, fabf_ctx::kWordBytes);
            if (cudaHostGetDevicePointer(&dm, hm, 0) == cudaSuccess) {
                ctx->h_mwords = hm;
                ctx->m_status = static_cast<unsigned*>(dm);
                ctx->m_nfb = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(dm) + fabf_ctx::kNfbOffset);
            } else {
                cudaFreeHost(hm);
            }
        }
        (void)cudaGetLastError();
    }
    *out = ctx;
    return FABF_OK;
}

int fabf_destroy(fabf_ctx* ctx)
{
    if (!ctx) return FABF_EINVAL;
    cudaSetDevice(ctx->device);
    fabf::serve_destroy(ctx->serve);
    fabf::batch_destroy(ctx->batch);
    cudaDeviceSynchronize();
    destroy_pipeline(ctx);
    if (ctx->stage) cudaFree(ctx->stage);
    cudaFree(ctx->d_status);                 // the block holding d_nfb too
    cudaFreeHost(ctx->h_words);
    if (ctx->h_mwords) cudaFreeHost(ctx->h_mwords);
    delete ctx;
    return FABF_OK;
}

int fabf_set_precision(fabf_ctx* ctx, int precision)
{
    if (!ctx || precision < FABF_FP64 || precision > FABF_C32) return FABF_EINVAL;
    ctx->precision = precision;
    return FABF_OK;
}

int fabf_filter(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                size_t pitch, int w, int N, void* out, int out_is_f64, void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, w, N);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // one attribute query per buffer: device (or managed), pinned host (with
    // its kernel mapping) or pageable host
    const PtrInfo pi = ptr_info(img), pt = ptr_info(theta), ps = ptr_info(sigma), po = ptr_info(out);
    const bool di = pi.device, dt = pt.device, ds = ps.device, dout = po.device;
    if (!(dt && ds && dout) && pt.kptr && ps.kptr && po.kptr)
        // pinned host maps and output: read and written in place by the kernel
        return filter_mapped(ctx, img, pi, static_cast<const float*>(pt.kptr), static_cast<const float*>(ps.kptr),
                             H, W, pitch, w, N, const_cast<void*>(po.kptr), out_is_f64, s);
    if (!di && !dt && !ds && !dout)
        return filter_host_pipelined(ctx, img, theta, sigma, H, W, pitch, w, N, out, out_is_f64, s);
    return with_device_buffers(
        ctx, img, theta, sigma, H, W, pitch, out, out_is_f64, s,
        [&](const uint8_t* d_img, size_t d_pitch, const float* d_th, const float* d_sg, void* d_out) {
            return run_fused(ctx, d_img, d_pitch, d_th, d_sg, H, W, w, N, d_out, out_is_f64, nullptr, s);
        });
}

int fabf_get_status(fabf_ctx* ctx, void* cuda_stream, int* status, uint64_t* n_fallback)
{
    if (!ctx || !status) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    return read_and_clear_status(ctx, static_cast<cudaStream_t>(cuda_stream), status, n_fallback, nullptr);
}

int fabf_get_status_ex(fabf_ctx* ctx, void* cuda_stream, int* status, uint64_t* n_fallback, uint64_t* n_fp64_redo)
{
    if (!ctx || !status) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    return read_and_clear_status(ctx, static_cast<cudaStream_t>(cuda_stream), status, n_fallback, n_fp64_redo);
}

const char* fabf_status_str(int status)
{
    switch (status) {
    case FABF_OK: return "ok";
    case FABF_EINVAL: return "invalid argument or per-pixel data";
    case FABF_ENOMEM: return "out of memory or over the memory budget";
    case FABF_EAGAIN: return "not ready, try again";
    case FABF_EUNSUPPORTED: return "unsupported parameters (N > 6 or w > 40)";
    case FABF_ECUDA: return "CUDA error";
    case FABF_ETIMEOUT: return "bounded wait timed out";
    case FABF_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

int fabf_hilbert_inverse(int N, int64_t* out)
{
    if (!out) return FABF_EINVAL;
    if (N < 0) return FABF_EINVAL;
    if (N > kNMax) return FABF_EUNSUPPORTED;
    for (int m = 1; m <= N + 1; ++m)
        for (int n = 1; n <= N + 1; ++n) out[(m - 1) * (N + 1) + (n - 1)] = hilbert_inverse_entry(N, m, n);
    return FABF_OK;
}

int fabf_centred_inverse(int N, double* out)
{
    if (!out) return FABF_EINVAL;
    if (N < 0) return FABF_EINVAL;
    if (N > kNMax) return FABF_EUNSUPPORTED;
    constexpr CentredInvTable t = make_centred_inverse_table();
    for (int j = 0; j <= N; ++j)
        for (int k = 0; k <= N; ++k) out[j * (N + 1) + k] = (double)t.v[N][j][k];
    return FABF_OK;
}

int fabf_fused_smem_bytes(int w, int N, size_t* bytes)
{
    if (!bytes || w < 1 || N < 0) return FABF_EINVAL;
    if (w > kWMax || N > kNMax) return FABF_EUNSUPPORTED;
    int off, Cb;
    fused_geometry(w, &off, &Cb);
    *bytes = fused_smem_bytes(N, w, Cb, kTileHMax);
    return FABF_OK;
}

int fabf_debug_stages(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H,
                      int W, size_t pitch, int w, int N, uint8_t* alpha, uint8_t* beta, int64_t* m,
                      int64_t* M, double* mu, double* c, double* t0lam, double* I, double* T,
                      int32_t* flags, double* out)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, w, N);
    if (rc) return rc;
    if (!alpha || !beta || !m || !M || !mu || !c || !t0lam || !I || !T || !flags) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    DebugPlanes d{alpha, beta, m, M, mu, c, t0lam, I, T, flags};
    rc = run_fused(ctx, img, pitch, theta, sigma, H, W, w, N, out, 1, &d, 0);   // FP64 with exports
    if (rc) return rc;
    int st = FABF_OK;
    rc = read_and_clear_status(ctx, 0, &st, nullptr, nullptr);
    return rc ? rc : st;
}

int fabf_debug_integrals(fabf_ctx* ctx, const double* lambda, const double* t0, int64_t n, int K,
                         int precision, double* out)
{
    if (!ctx || !lambda || !t0 || !out || n < 0 || K < 1 || K > 7) return FABF_EINVAL;
    if (precision != FABF_FP64 && precision != FABF_FP64FIT_FP32REC && precision != FABF_C32)
        return FABF_EUNSUPPORTED;
    const int fp32 = precision == FABF_FP64 ? 0 : (precision == FABF_C32 ? 2 : 1);
    if (n == 0) return FABF_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    switch (K) {
    case 1: integrals_kernel<1><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    case 2: integrals_kernel<2><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    case 3: integrals_kernel<3><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    case 4: integrals_kernel<4><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    case 5: integrals_kernel<5><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    case 6: integrals_kernel<6><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    default: integrals_kernel<7><<<blocks, threads>>>(lambda, t0, n, fp32, out); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(e);
}

int fabf_debug_fp64_functions(fabf_ctx* ctx, const double* x, int64_t n, double* erfcx_out, double* exp_out)
{
    if (!ctx || !x || !erfcx_out || !exp_out || n < 0) return FABF_EINVAL;
    if (n == 0) return FABF_OK;
    if (!is_device_ptr(x) || !is_device_ptr(erfcx_out) || !is_device_ptr(exp_out)) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    fp64_functions_kernel<<<blocks, threads>>>(x, n, erfcx_out, exp_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(e);
}

int fabf_bruteforce(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                    size_t pitch, int w, void* out, int out_is_f64, int use_f64, void* cuda_stream)
{
    if (!ctx) return FABF_EINVAL;
    int rc = check_filter_args(img, theta, sigma, out, H, W, pitch, w, 0);
    if (rc) return rc;
    if (!is_device_ptr(img) || !is_device_ptr(theta) || !is_device_ptr(sigma) || !is_device_ptr(out))
        return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    dim3 grid((W + 31) / 32, (H + 7) / 8);
    if (use_f64)
        bruteforce_kernel<double><<<grid, 256, 0, s>>>(img, (long long)pitch, theta, sigma, H, W, w, out,
                                                       out_is_f64);
    else
        bruteforce_kernel<float><<<grid, 256, 0, s>>>(img, (long long)pitch, theta, sigma, H, W, w, out,
                                                      out_is_f64);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"

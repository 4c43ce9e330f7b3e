// Declarations shared by the host translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>

namespace fabf {

struct DebugPlanes;
struct FusedParams;
struct BatchParams;
struct ImageJob;
struct ServeState;
struct BatchState;

struct TuneEntry {
    int TH;         // output rows per tile
    float ms;       // measured time of the tuning image (0 = not measured)
    int plain;      // 1: stage tiles with plain loads, 0: with TMA (where the image allows it)
};

}  // namespace fabf

struct fabf_ctx {
    int device = 0;
    int precision = 0;
    size_t budget = 0;
    int autotune = 0;
    std::string tune_cache_path;
    int num_sms = 0;
    // status words of stream-ordered calls, one device block: the status bits
    // at offset 0, the fallback and FP64 redo counts at kNfbOffset; read back
    // through a pinned copy (h_words, under status_lock)
    static constexpr size_t kNfbOffset = 256, kWordBytes = kNfbOffset + 16;
    unsigned* d_status = nullptr;
    unsigned long long* d_nfb = nullptr;
    void* h_words = nullptr;
    std::mutex status_lock;
    // a second status block in mapped pinned host memory, for the calls on
    // pinned host buffers (one at a time, under stage_lock): the kernel's
    // atomics land in host memory and the host reads them after the stream
    // wait, with no copy or clear on the stream.  Only where the GPU's
    // atomics on host memory are native (nullptr otherwise).
    void* h_mwords = nullptr;                // host view
    unsigned* m_status = nullptr;            // device view of the same block
    unsigned long long* m_nfb = nullptr;
    void* stage = nullptr;                   // grow-only staging buffer for host pointers
    size_t stage_bytes = 0;
    std::mutex stage_lock;                   // one host-pointer call at a time uses the staging buffer
    std::mutex tune_lock;
    std::mutex batch_lock;                   // the batch graph cache
    std::map<int, fabf::TuneEntry> tune;     // key: tune_key(w, N, precision)
    fabf::ServeState* serve = nullptr;
    fabf::BatchState* batch = nullptr;
    // host-pointer pipeline (created on first use, under stage_lock): a copy-in
    // stream, one compute stream per band, a copy-out stream and their events
    static constexpr int kBands = 4;
    bool pipe_ready = false;
    cudaStream_t s_in = nullptr, s_out = nullptr, s_band[kBands] = {};
    cudaEvent_t ev_start = nullptr, ev_in[kBands] = {}, ev_k[kBands] = {}, ev_done = nullptr;
};

namespace fabf {

inline int tune_key(int w, int N, int prec) { return (w * 8 + N) * 4 + prec; }

int cuda_status(cudaError_t e);
bool is_device_ptr(const void* p);
struct PtrInfo {
    bool device = false;           // device or managed memory
    const void* kptr = nullptr;    // what kernels dereference (nullptr: pageable host memory)
};
PtrInfo ptr_info(const void* p);
int check_filter_args(const void* img, const void* theta, const void* sigma, const void* out, int H, int W,
                      size_t pitch, int w, int N);
void fused_geometry(int w, int* off, int* Cb);
bool encode_image_tmap(CUtensorMap* tm, const uint8_t* img, int H, int W, size_t pitch, int Cb, int R);

// Fill the launch description of one image with TH output rows per tile; the
// tensor map is encoded (and J->use_tma set) when the image allows TMA.
// Returns the dynamic shared memory one tile needs.
size_t make_job(ImageJob* J, CUtensorMap* tm, const uint8_t* img, size_t pitch, const float* theta,
                const float* sigma, int H, int W, int w, int N, void* out, int out_f64, int TH,
                bool allow_tma = true);

cudaError_t launch_fused(int prec, int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                         cudaStream_t s);
cudaError_t launch_batch(int prec, const BatchParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_fused_p0(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_fused_p1(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_fused_p2(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_batch_p0(const BatchParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_p1(const BatchParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_p2(const BatchParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_fused_p3(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_batch_p3(const BatchParams& p, int grid, size_t smem, cudaStream_t s);

// Launch one image on device buffers with the context's precision and tuned
// tile shape; status words are the context's.
int run_fused(fabf_ctx* ctx, const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
              int W, int w, int N, void* out, int out_f64, const DebugPlanes* dbg, cudaStream_t s);
int run_fused_prec(fabf_ctx* ctx, int prec, const uint8_t* img, size_t pitch, const float* theta,
                   const float* sigma, int H, int W, int w, int N, void* out, int out_f64, int TH,
                   const DebugPlanes* dbg, unsigned* status, unsigned long long* nfb, cudaStream_t s,
                   bool allow_tma = true);

// FP64 launch with caller-provided status words (allocation-free entry point).
int launch_fused_scratch(const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
                         int W, int w, int N, void* out, int out_f64, unsigned* status,
                         unsigned long long* n_fallback, cudaStream_t s);

// Output rows per tile (a multiple of 8).  The steady-state choice for
// (w, N, prec) -- the autotuner's measurement when the context has autotune
// on, else kSteadyTileRows[prec] -- holds when many tiles are in flight (H = W
// = 0: batches).  For one H x W image the choice is the tallest candidate
// no taller than the steady one that still leaves kMinWaves[prec] waves of
// resident CTAs across the SMs, else the shortest candidate: a short image
// with tall tiles leaves SMs idle in the last wave.  Measured at 720p, 1080p,
// 2160x3840 and 4096^2 for w in {5, 20, 40}.
int tile_rows_for(fabf_ctx* ctx, int w, int N, int prec, int H, int W);
// Tile staging for (w, N, prec): TMA (true) unless the context has autotune
// on and the autotuner measured plain cooperative loads faster.
bool tile_staging_tma(fabf_ctx* ctx, int w, int N, int prec);
constexpr int kTileCandidates[] = {8, 16, 24, 32, 40};
constexpr int kPrecForms = 4;
// FP64, FP64 fit + FP32, compensated FP32, centred binary32
constexpr int kSteadyTileRows[kPrecForms] = {8, 8, 40, 40};
constexpr int kMinWaves[kPrecForms] = {1, 1, 6, 3};
// Resident CTAs per SM the kernels are compiled for (MinBlocks in
// fabf_kernels.cuh); shared memory may allow fewer.
constexpr int kCtasPerSm[kPrecForms] = {2, 4, 4, 4};
inline int prec_index(int prec) { return prec < 0 || prec >= kPrecForms ? 0 : prec; }

// CTAs of a single-image launch resident per SM: the register budget the
// kernel is compiled for (the centred form at N = 6 runs its 3-CTA build)
// and the shared memory (dyn_smem plus the 1 KB per-CTA reservation, of
// 228 KB per SM).
inline int smem_resident_ctas(size_t dyn_smem)
{
    const int n = (int)((size_t)228 * 1024 / (dyn_smem + 1024));
    return n < 1 ? 1 : n;
}

inline int resident_ctas(int prec, int N, size_t dyn_smem)
{
    const int pc = prec_index(prec);
    int regs = kCtasPerSm[pc];
    if (pc == 3 && N >= 6) regs = 3;
    const int by_smem = smem_resident_ctas(dyn_smem);
    return by_smem < regs ? by_smem : regs;
}

// The centred form's fused and batch kernels compiled for 3 CTAs per SM
// (fabf_inst_c32w.cu).
cudaError_t launch_fused_c32_wide(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                                  cudaStream_t s);
cudaError_t launch_batch_c32_wide(const BatchParams& p, int grid, size_t smem, cudaStream_t s);
constexpr int kDefaultTileRows = 32;               // stage-export runs of the tests

int read_and_clear_status(fabf_ctx* ctx, cudaStream_t s, int* status, uint64_t* nfb, uint64_t* nredo);

// Status words for a call on pinned host buffers (the caller holds
// stage_lock): the mapped block where the context has one, else the device
// block; finish_pinned_call waits for the stream and returns the kernels'
// status, clearing the words.
unsigned* pinned_call_status(fabf_ctx* ctx);
unsigned long long* pinned_call_nfb(fabf_ctx* ctx);
int finish_pinned_call(fabf_ctx* ctx, cudaStream_t s);

// Grow the context's staging buffer to at least `bytes`.
int ensure_stage(fabf_ctx* ctx, size_t bytes);

// A host image copied into the staging buffer (16-byte rows for TMA) on s,
// a device image passed through; the caller holds stage_lock.  A pinned
// image whose rows are whole 16-byte words is copied by a kernel that reads
// it over the chip-to-chip link from every SM (faster than one copy-engine
// transfer at these sizes); other host images by cudaMemcpy(2D)Async.
int stage_image(fabf_ctx* ctx, const uint8_t* img, const PtrInfo& pi, int H, int W, size_t pitch, cudaStream_t s,
                const uint8_t** d_img, size_t* d_pitch);

// Run `launch(d_img, d_pitch, d_theta, d_sigma, d_out)` on device buffers.
// All-device arguments are passed through (the call stays stream-ordered; the
// status words are read by fabf_get_status).  Host buffers are staged through
// the context's buffer (16-byte aligned image rows; one such call at a time
// per context), the output copied back, and the call synchronises and
// returns the kernels' status.
template <typename Launch>
int with_device_buffers(fabf_ctx* ctx, const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                        size_t pitch, void* out, int out_is_f64, cudaStream_t s, Launch&& launch)
{
    const bool di = is_device_ptr(img), dt = is_device_ptr(theta), ds = is_device_ptr(sigma),
               dout = is_device_ptr(out);
    if (di && dt && ds && dout) return launch(img, pitch, theta, sigma, out);
    std::lock_guard<std::mutex> staged(ctx->stage_lock);   // held until the synchronous call returns
    const size_t npix = (size_t)H * W;
    const size_t osz = out_is_f64 ? 8 : 4;
    const size_t ipitch = ((size_t)W + 15) & ~(size_t)15;
    const size_t o_img = 0, o_th = o_img + ((ipitch * H + 255) & ~(size_t)255);
    const size_t o_sg = o_th + ((npix * 4 + 255) & ~(size_t)255);
    const size_t o_out = o_sg + ((npix * 4 + 255) & ~(size_t)255);
    int rc = ensure_stage(ctx, o_out + npix * osz);
    if (rc) return rc;
    uint8_t* base = static_cast<uint8_t*>(ctx->stage);
    const uint8_t* d_img = img;
    size_t d_pitch = pitch;
    const float* d_th = theta;
    const float* d_sg = sigma;
    void* d_out = dout ? out : base + o_out;
    cudaError_t e = cudaSuccess;
    if (!di) {
        e = cudaMemcpy2DAsync(base + o_img, ipitch, img, pitch, W, H, cudaMemcpyHostToDevice, s);
        d_img = base + o_img;
        d_pitch = ipitch;
    }
    if (e == cudaSuccess && !dt) {
        e = cudaMemcpyAsync(base + o_th, theta, npix * 4, cudaMemcpyHostToDevice, s);
        d_th = reinterpret_cast<const float*>(base + o_th);
    }
    if (e == cudaSuccess && !ds) {
        e = cudaMemcpyAsync(base + o_sg, sigma, npix * 4, cudaMemcpyHostToDevice, s);
        d_sg = reinterpret_cast<const float*>(base + o_sg);
    }
    if (e != cudaSuccess) return cuda_status(e);
    rc = launch(d_img, d_pitch, d_th, d_sg, d_out);
    if (rc) return rc;
    if (!dout) {
        e = cudaMemcpyAsync(out, d_out, npix * osz, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    int st = 0;
    rc = read_and_clear_status(ctx, s, &st, nullptr, nullptr);
    return rc ? rc : st;
}
void serve_destroy(ServeState* s);
void batch_destroy(BatchState* b);

}  // namespace fabf

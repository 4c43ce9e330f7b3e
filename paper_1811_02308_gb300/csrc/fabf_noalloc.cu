// fabf_filter_noalloc: the fused FP64 filter for callers that must not
// allocate device memory.
//
// fabf_filter needs a context, and fabf_create allocates the context's status
// words with cudaMalloc.  Some callers cannot do that: code running on a
// real-time thread where cudaMalloc's implicit device synchronisation is
// not acceptable, or code inside a framework or plugin that owns every device
// allocation and forbids its guests from calling the CUDA allocator.  This
// entry point takes device buffers the caller already owns and keeps the
// kernel's only scratch -- the status word and the fallback-pixel counter --
// in a fixed array compiled into the library.  The call waits for its stream
// before it returns, so it must not be made while a stream capture is active.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/fabf.h"
#include "fabf_internal.h"

namespace {

// Scratch of the allocation-free entry point: word 0 holds the status bits
// (low 32 bits), word 1 the fallback-pixel counter.  Every GPU that loads
// this library holds these 256 bytes until the process exits.
constexpr size_t kScratchWords = 32;   // 256 bytes
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

// Words one call needs.  The scratch does not grow with the image.
constexpr size_t kWordsPerCall = 2;
static_assert(kWordsPerCall <= kScratchWords, "scratch array too small");

constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};   // device address, per device

// The array's name is only a host-side stand-in in host code; its device
// address is looked up once per device, with that device (dev) current, and
// cached for the life of the process.  A cudaDeviceReset of that device
// would leave the cached address stale, so the library must not be used
// across one.
int scratch_for_device(int dev, unsigned long long** out)
{
    if (dev < 0 || dev >= kMaxDevices) return FABF_EUNSUPPORTED;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return FABF_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FABF_OK;
}

// True when p is device (or managed) memory of device dev.  Buffers of
// another GPU are rejected: the kernel runs on the current device and its
// tensor map would be encoded over remote memory.
bool on_device(const void* p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    return a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int fabf_filter_noalloc(const uint8_t* img, const float* theta, const float* sigma, int H, int W,
                                   size_t pitch, int w, int N, void* out, int out_is_f64,
                                   void* cuda_stream, uint64_t* n_fallback)
{
    int rc = fabf::check_filter_args(img, theta, sigma, out, H, W, pitch, w, N);
    if (rc) return rc;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FABF_ECUDA;
    }
    // host buffers would need device staging, i.e. an allocation; buffers of
    // another GPU are not this call's to read
    if (!on_device(img, dev) || !on_device(theta, dev) || !on_device(sigma, dev) || !on_device(out, dev))
        return FABF_EINVAL;
    if (kWordsPerCall > kScratchWords) return FABF_EUNSUPPORTED;
    unsigned long long* scratch = nullptr;
    rc = scratch_for_device(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // The array keeps the previous call's contents: clear both words first.
    cudaError_t e = cudaMemsetAsync(scratch, 0, kWordsPerCall * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fabf::cuda_status(e);
    rc = fabf::launch_fused_scratch(img, pitch, theta, sigma, H, W, w, N, out, out_is_f64,
                                    reinterpret_cast<unsigned*>(scratch), scratch + 1, s);
    if (rc) return rc;
    unsigned long long words[kWordsPerCall] = {0, 0};
    e = cudaMemcpyAsync(words, scratch, sizeof(words), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fabf::cuda_status(e);
    if (n_fallback) *n_fallback = words[1];
    const unsigned st = (unsigned)(words[0] & 0xffffffffu);
    if (st & 2u) return FABF_ETIMEOUT;
    if (st & 1u) return FABF_EINVAL;
    return FABF_OK;
}

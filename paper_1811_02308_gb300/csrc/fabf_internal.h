// Declarations shared by the host translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

struct fabf_ctx;

namespace fabf {

struct DebugPlanes;
struct ServeState;
struct BatchState;

int cuda_status(cudaError_t e);
bool is_device_ptr(const void* p);
int check_filter_args(const void* img, const void* theta, const void* sigma, const void* out, int H, int W,
                      size_t pitch, int w, int N);
void fused_geometry(int w, int* off, int* Cb);
int run_fused(fabf_ctx* ctx, const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
              int W, int w, int N, void* out, int out_f64, const DebugPlanes* dbg, cudaStream_t s);

int launch_fused_scratch(const uint8_t* img, size_t pitch, const float* theta, const float* sigma, int H,
                         int W, int w, int N, void* out, int out_f64, unsigned* status,
                         unsigned long long* n_fallback, cudaStream_t s);

void serve_destroy(ServeState* s);
void batch_destroy(BatchState* b);

}  // namespace fabf

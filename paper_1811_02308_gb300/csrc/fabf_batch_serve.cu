// Batch and serving entry points (persistent work-queue kernel, CUDA graph,
// continuous batching).
#include <cuda_runtime.h>

#include "../../include/fabf.h"
#include "fabf_internal.h"

namespace fabf {
struct ServeState {};
struct BatchState {};
void serve_destroy(ServeState* s) { delete s; }
void batch_destroy(BatchState* b) { delete b; }
}  // namespace fabf

extern "C" {

int fabf_filter_batch(fabf_ctx* ctx, const fabf_request* reqs, int n, void* cuda_stream)
{
    (void)ctx; (void)reqs; (void)n; (void)cuda_stream;
    return FABF_EUNSUPPORTED;
}

int fabf_serve_submit(fabf_ctx* ctx, const fabf_request* req, uint64_t* ticket)
{
    (void)ctx; (void)req; (void)ticket;
    return FABF_EUNSUPPORTED;
}

int fabf_serve_poll(fabf_ctx* ctx, uint64_t ticket, int timeout_us, int* result)
{
    (void)ctx; (void)ticket; (void)timeout_us; (void)result;
    return FABF_EUNSUPPORTED;
}

}  // extern "C"

// Autotuner, batch entry point (one persistent launch replayed from a CUDA
// graph) and the continuous-batching serving loop.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/fabf.h"
#include "fabf_internal.h"
#include "fabf_kernels.cuh"

namespace fabf {

// ===========================================================================
// Autotuner: output rows per tile for (w, N, precision)
// ===========================================================================
namespace {

// Large enough that the tallest candidate still gives several waves of CTAs,
// so the measurement is the steady-state cost per tile height.
constexpr int kTuneH = 2048, kTuneW = 4096;

struct TuneImage {
    uint8_t* img = nullptr;
    float* theta = nullptr;
    float* sigma = nullptr;
    double* out = nullptr;
    unsigned* status = nullptr;
    unsigned long long* nfb = nullptr;
};

// A deterministic stand-in image for timing: smooth shading, edges, noise.
void fill_tune_host(std::vector<uint8_t>& f, std::vector<float>& th, std::vector<float>& sg)
{
    f.resize((size_t)kTuneH * kTuneW);
    th.resize(f.size());
    sg.resize(f.size());
    uint32_t x = 2463534242u;
    for (int r = 0; r < kTuneH; ++r)
        for (int c = 0; c < kTuneW; ++c) {
            x ^= x << 13;
            x ^= x >> 17;
            x ^= x << 5;
            int v = 60 + (int)(50.0 * (1.0 + __builtin_sin(c * 0.013) * __builtin_cos(r * 0.021)));
            if (c > 300 + r / 3) v += 70;
            v += (int)(x % 31) - 15;
            v = v < 0 ? 0 : (v > 255 ? 255 : v);
            const size_t i = (size_t)r * kTuneW + c;
            f[i] = (uint8_t)v;
            th[i] = (float)v;
            sg[i] = 8.0f + 40.0f * (float)c / kTuneW;
        }
}

int ensure_tune_image(TuneImage& t)
{
    if (t.img) return FABF_OK;
    std::vector<uint8_t> f;
    std::vector<float> th, sg;
    fill_tune_host(f, th, sg);
    const size_t n = f.size();
    cudaError_t e = cudaMalloc(&t.img, n);
    if (e == cudaSuccess) e = cudaMalloc(&t.theta, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&t.sigma, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&t.out, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&t.status, 256);
    if (e == cudaSuccess) e = cudaMalloc(&t.nfb, 256);
    if (e == cudaSuccess) e = cudaMemcpy(t.img, f.data(), n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t.theta, th.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t.sigma, sg.data(), n * 4, cudaMemcpyHostToDevice);
    return cuda_status(e);
}

void free_tune_image(TuneImage& t)
{
    cudaFree(t.img);
    cudaFree(t.theta);
    cudaFree(t.sigma);
    cudaFree(t.out);
    cudaFree(t.status);
    cudaFree(t.nfb);
    t = TuneImage{};
}


void load_tune_cache(fabf_ctx* ctx)
{
    static std::mutex once_lock;
    std::lock_guard<std::mutex> g(once_lock);
    if (ctx->tune_cache_path.empty() || !ctx->tune.empty()) return;
    FILE* fp = std::fopen(ctx->tune_cache_path.c_str(), "r");
    if (!fp) return;
    // lines "w N precision TH ms [plain]" (plain staging flag optional, 0 = TMA)
    char line[256];
    while (std::fgets(line, sizeof(line), fp)) {
        int w, N, prec, TH, plain = 0;
        float ms;
        const int n = std::sscanf(line, "%d %d %d %d %f %d", &w, &N, &prec, &TH, &ms, &plain);
        if (n >= 5 && TH >= 8 && TH <= kTileHMax && TH % 8 == 0)
            ctx->tune[tune_key(w, N, prec)] = TuneEntry{TH, ms, plain ? 1 : 0};
    }
    std::fclose(fp);
}

}  // namespace

// The tuned (or default) tile shape and staging of (w, N, prec).  With
// autotune on, the first query of a key times every candidate height with
// each staging (TMA and plain cooperative loads) and keeps the fastest.
static TuneEntry tune_entry(fabf_ctx* ctx, int w, int N, int prec)
{
    const TuneEntry dflt{kSteadyTileRows[prec_index(prec)], 0.0f, 0};
    if (!ctx || !ctx->autotune) return dflt;
    load_tune_cache(ctx);
    std::lock_guard<std::mutex> g(ctx->tune_lock);
    auto it = ctx->tune.find(tune_key(w, N, prec));
    if (it != ctx->tune.end()) return it->second;

    // the timing image lives only for this measurement (about 140 MB)
    TuneImage timg;
    TuneImage* t = &timg;
    if (ensure_tune_image(timg) != FABF_OK) {
        free_tune_image(timg);
        (void)cudaGetLastError();
        return dflt;
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        free_tune_image(timg);
        return dflt;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = dflt.TH, best_plain = 0;
    float best_ms = 1e30f;
    for (int plain = 0; plain < 2; ++plain)
        for (int TH : kTileCandidates) {
            float ms = 1e30f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                cudaEventRecord(e0, s);
                // the form's own output type: float64 for FP64, float32 otherwise
                ok = run_fused_prec(ctx, prec, t->img, kTuneW, t->theta, t->sigma, kTuneH, kTuneW, w, N, t->out,
                                    prec == kPrecFP64 ? 1 : 0, TH, nullptr, t->status, t->nfb, s,
                                    plain == 0) == FABF_OK;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
                float m = 0.0f;
                cudaEventElapsedTime(&m, e0, e1);
                if (rep > 0) ms = std::min(ms, m);      // first run is the warm-up
            }
            if (ok && ms < best_ms) {
                best_ms = ms;
                best = TH;
                best_plain = plain;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    free_tune_image(timg);
    (void)cudaGetLastError();
    const TuneEntry got{best, best_ms, best_plain};
    ctx->tune[tune_key(w, N, prec)] = got;
    if (!ctx->tune_cache_path.empty()) {
        FILE* fp = std::fopen(ctx->tune_cache_path.c_str(), "a");
        if (fp) {
            std::fprintf(fp, "%d %d %d %d %.5f %d\n", w, N, prec, best, best_ms, best_plain);
            std::fclose(fp);
        }
    }
    return got;
}

static int steady_tile_rows(fabf_ctx* ctx, int w, int N, int prec)
{
    return tune_entry(ctx, w, N, prec).TH;
}

bool tile_staging_tma(fabf_ctx* ctx, int w, int N, int prec)
{
    return tune_entry(ctx, w, N, prec).plain == 0;
}

int tile_rows_for(fabf_ctx* ctx, int w, int N, int prec, int H, int W)
{
    const int steady = steady_tile_rows(ctx, w, N, prec);
    if (H <= 0 || W <= 0 || steady <= kTileCandidates[0]) return steady;
    int num_sms = ctx ? ctx->num_sms : 0;
    if (num_sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return kTileCandidates[0];
        }
    }
    const int pc = prec_index(prec);
    int off, Cb;
    fused_geometry(w, &off, &Cb);
    const long long tiles_x = (W + kTileW - 1) / kTileW;
    int best = kTileCandidates[0];
    for (int TH : kTileCandidates) {
        if (TH > steady) break;
        const int per_sm = resident_ctas(pc, N, fused_smem_bytes(N, w, Cb, TH));
        const long long tiles = tiles_x * ((H + TH - 1) / TH);
        if (tiles >= (long long)kMinWaves[pc] * num_sms * per_sm) best = TH;
    }
    return best;
}

// ===========================================================================
// Batch: one persistent launch over all tiles of n images, captured once in
// a CUDA graph and replayed while the request set stays the same.
//
// Each request set that is replayed keeps its own graph, job table, tensor
// maps and work counter (up to kBatchGraphs sets, least recently used
// evicted), so a caller may alternate sets on a stream without waiting: no
// replay ever reads a table that a later call rewrites.  An event recorded
// after each replay orders the next replay of the same set after it (on any
// stream), and a set's table is rewritten only after its last replay is done.
// ===========================================================================
constexpr int kBatchGraphs = 4;

struct BatchGraph {
    ImageJob* d_jobs = nullptr;
    CUtensorMap* d_tmaps = nullptr;
    unsigned long long* d_counter = nullptr;
    int cap = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;       // recorded after the set's last replay
    bool launched = false;
    unsigned long long last_use = 0;
    std::vector<unsigned char> key;
};

struct BatchState {
    BatchGraph g[kBatchGraphs];
    cudaStream_t cap_stream = nullptr;
    unsigned long long tick = 0;
    int launches = 0;       // graph replays (for tests)
    int captures = 0;       // graph (re)builds
};

void batch_destroy(BatchState* b)
{
    if (!b) return;
    for (BatchGraph& G : b->g) {
        if (G.done) cudaEventSynchronize(G.done);
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.done) cudaEventDestroy(G.done);
        cudaFree(G.d_jobs);
        cudaFree(G.d_tmaps);
        cudaFree(G.d_counter);
    }
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

static int batch_build(fabf_ctx* ctx, BatchState* b, BatchGraph& G, const fabf_request* reqs, int n)
{
    const int prec = ctx->precision;
    // The set this slot held may still be running: wait for its last replay
    // before its table is rewritten.
    if (G.launched) {
        cudaError_t e = cudaEventSynchronize(G.done);
        if (e != cudaSuccess) return cuda_status(e);
        G.launched = false;
    }
    G.key.clear();
    // Heavier images first (higher N, larger w): their tiles are popped first,
    // which shortens the tail of the persistent launch.
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (reqs[a].N != reqs[c].N) return reqs[a].N > reqs[c].N;
        return reqs[a].w > reqs[c].w;
    });
    std::vector<ImageJob> jobs(n);
    std::vector<CUtensorMap> tmaps(n);
    long long tiles = 0;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const fabf_request& r = reqs[order[i]];
        const int TH = tile_rows_for(ctx, r.w, r.N, prec, 0, 0);
        const size_t sm = make_job(&jobs[i], &tmaps[i], r.img, r.pitch, r.theta, r.sigma, r.H, r.W, r.w, r.N,
                                   r.out, r.out_is_f64, TH, tile_staging_tma(ctx, r.w, r.N, prec));
        jobs[i].tile_begin = tiles;
        tiles += (long long)jobs[i].tiles_x * jobs[i].tiles_y;
        smem = std::max(smem, sm);
    }
    cudaError_t e = cudaSuccess;
    if (!G.d_counter) e = cudaMalloc(&G.d_counter, 256);
    if (e == cudaSuccess && !G.done) e = cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    if (n > G.cap) {
        cudaFree(G.d_jobs);
        cudaFree(G.d_tmaps);
        G.d_jobs = nullptr;
        G.d_tmaps = nullptr;
        G.cap = 0;
        e = cudaMalloc(&G.d_jobs, sizeof(ImageJob) * n);
        if (e == cudaSuccess) e = cudaMalloc(&G.d_tmaps, sizeof(CUtensorMap) * n);
        if (e != cudaSuccess) return cuda_status(e);
        G.cap = n;
    }
    // Nothing reads this slot's table now (its last replay is done), so a
    // plain copy is safe whatever stream the caller uses.
    e = cudaMemcpy(G.d_jobs, jobs.data(), sizeof(ImageJob) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G.d_tmaps, tmaps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);

    BatchParams p;
    std::memset(&p, 0, sizeof(p));
    p.jobs = G.d_jobs;
    p.tmaps = G.d_tmaps;
    p.njobs = n;
    p.total_tiles = tiles;
    p.next_tile = G.d_counter;
    p.status = ctx->d_status;
    p.n_fallback = ctx->d_nfb;
    const int per_sm = std::max(1, std::min(kCtasPerSm[prec_index(prec)],
                                            (int)((size_t)228 * 1024 / (smem + 1024))));
    long long grid = (long long)ctx->num_sms * per_sm;
    if (grid > tiles) grid = tiles;

    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(G.d_counter, 0, sizeof(unsigned long long), b->cap_stream);
        if (e1 == cudaSuccess) e1 = launch_batch(prec, p, (int)grid, smem, b->cap_stream);
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        G.exec = nullptr;
        return cuda_status(e);
    }
    ++b->captures;
    return FABF_OK;
}

}  // namespace fabf

using namespace fabf;

extern "C" {

int fabf_filter_batch(fabf_ctx* ctx, const fabf_request* reqs, int n, void* cuda_stream)
{
    if (!ctx || (!reqs && n > 0) || n < 0) return FABF_EINVAL;
    if (n == 0) return FABF_OK;
    for (int i = 0; i < n; ++i) {
        const fabf_request& r = reqs[i];
        const int rc = check_filter_args(r.img, r.theta, r.sigma, r.out, r.H, r.W, r.pitch, r.w, r.N);
        if (rc) return rc;
        if (r.passes != 1) return FABF_EINVAL;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    for (int i = 0; i < n; ++i)
        if (!is_device_ptr(reqs[i].img) || !is_device_ptr(reqs[i].theta) || !is_device_ptr(reqs[i].sigma) ||
            !is_device_ptr(reqs[i].out))
            return FABF_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->batch_lock);
    if (!ctx->batch) {
        BatchState* b = new (std::nothrow) BatchState();
        if (!b) return FABF_ENOMEM;
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            batch_destroy(b);
            return cuda_status(e);
        }
        ctx->batch = b;
    }
    BatchState* b = ctx->batch;
    std::vector<unsigned char> key(sizeof(fabf_request) * n + sizeof(int));
    std::memcpy(key.data(), reqs, sizeof(fabf_request) * n);
    std::memcpy(key.data() + sizeof(fabf_request) * n, &ctx->precision, sizeof(int));
    BatchGraph* G = nullptr;
    for (BatchGraph& g : b->g)
        if (g.exec && g.key == key) G = &g;
    if (!G) {
        // a slot never used, else the least recently used one
        G = &b->g[0];
        for (BatchGraph& g : b->g) {
            if (!g.exec) {
                G = &g;
                break;
            }
            if (g.last_use < G->last_use) G = &g;
        }
        const int rc = batch_build(ctx, b, *G, reqs, n);
        if (rc) return rc;
        G->key = key;
    }
    G->last_use = ++b->tick;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    if (G->launched) e = cudaStreamWaitEvent(s, G->done, 0);   // after this set's previous replay
    if (e == cudaSuccess) e = cudaGraphLaunch(G->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(G->done, s);
    if (e != cudaSuccess) return cuda_status(e);
    G->launched = true;
    ++b->launches;
    return FABF_OK;
}

}  // extern "C"

// ===========================================================================
// Serving: continuous batching.
//
// fabf_serve_submit admits a request when a slot (stream) is free and its
// bytes fit the remaining device-memory budget: it allocates the request's
// buffers from a stream-ordered pool, copies the inputs (caller buffers are
// free on return) and enqueues every pass on the request's own stream.
// Requests admitted while others are on the GPU run concurrently with them;
// the GPU schedules their CTAs as SMs free up.  Between passes an
// elementwise kernel prepares the next pass (texture filtering, Sec. IV-C):
// the image becomes the previous output rounded half to even and clamped to
// [0, 255], the centre keeps its offset (theta - f) from the first pass, and
// sigma is scaled by sigma_decay.  A host worker thread polls the requests'
// completion events, copies results to host outputs, releases memory and
// budget, and wakes pollers.  Every wait is bounded.
// ===========================================================================
namespace fabf {

constexpr int kServeSlots = 64;

__global__ void next_pass_kernel(const void* prev_out, int out_f64, const float* zeta, float* sigma,
                                 float decay, uint8_t* img, float* theta, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // round half to even and clamp; NaN (bad input, flagged by the status
    // word) gives 0.  Float outputs round in binary32 (rintf(v) equals
    // rint((double)v) for every float v; binary64 is the slow pipe here).
    uint8_t f;
    if (out_f64) {
        const double g = static_cast<const double*>(prev_out)[i];
        double q = rint(g);
        q = q < 0.0 ? 0.0 : (q > 255.0 ? 255.0 : q);
        f = (g == g) ? (uint8_t)q : (uint8_t)0;
    } else {
        const float g = static_cast<const float*>(prev_out)[i];
        float q = rintf(g);
        q = q < 0.0f ? 0.0f : (q > 255.0f ? 255.0f : q);
        f = (g == g) ? (uint8_t)q : (uint8_t)0;
    }
    img[i] = f;
    theta[i] = (float)f + zeta[i];
    sigma[i] = sigma[i] * decay;
}

__global__ void zeta_kernel(const uint8_t* img, const float* theta, float* zeta, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    zeta[i] = theta[i] - (float)img[i];
}

struct ServeReq {
    uint64_t ticket = 0;
    fabf_request r{};
    int slot = -1;
    size_t bytes = 0;
    uint8_t* base = nullptr;      // one stream-ordered allocation
    uint8_t* d_img = nullptr;
    float* d_theta = nullptr;
    float* d_sigma = nullptr;
    float* d_zeta = nullptr;
    void* d_out = nullptr;
    unsigned* d_status = nullptr;
    unsigned long long* d_nfb = nullptr;
    bool host_out = false;
    cudaEvent_t done = nullptr;
    int result = FABF_OK;
    bool finished = false;
};

struct ServeState {
    std::mutex lock;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    cudaStream_t streams[kServeSlots] = {};
    cudaEvent_t events[kServeSlots] = {};
    bool slot_busy[kServeSlots] = {};
    cudaMemPool_t pool = nullptr;
    std::map<uint64_t, ServeReq*> reqs;     // admitted, not yet collected
    int device = 0;
};

static size_t serve_bytes(const fabf_request& r)
{
    const size_t n = (size_t)r.H * r.W;
    const size_t a = 256;
    auto up = [&](size_t v) { return (v + a - 1) / a * a; };
    return up(n) + 3 * up(n * 4) + up(n * (r.out_is_f64 ? 8 : 4)) + a;
}

static void serve_finish(ServeState* S, ServeReq* q)
{
    // called by the worker with S->lock held, after q->done completed
    unsigned long long w[2] = {0, 0};
    cudaError_t e = cudaMemcpy(w, q->d_status, sizeof(w), cudaMemcpyDeviceToHost);
    int rc = FABF_OK;
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (w[0] & kStatusTimeout) rc = FABF_ETIMEOUT;
    else if (w[0] & kStatusBadInput) rc = FABF_EINVAL;
    if (q->host_out && rc != FABF_ECUDA) {
        const size_t nb = (size_t)q->r.H * q->r.W * (q->r.out_is_f64 ? 8 : 4);
        e = cudaMemcpy(q->r.out, q->d_out, nb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    cudaFreeAsync(q->base, S->streams[q->slot]);
    S->slot_busy[q->slot] = false;
    S->in_use -= q->bytes;
    q->result = rc;
    q->finished = true;
}

static void serve_worker(ServeState* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->lock);
    while (!S->stop) {
        bool any = false;
        for (auto& kv : S->reqs) {
            ServeReq* q = kv.second;
            if (q->finished) continue;
            any = true;
            const cudaError_t e = cudaEventQuery(q->done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) (void)cudaGetLastError();
            serve_finish(S, q);
            S->cv.notify_all();
        }
        S->cv.wait_for(lk, std::chrono::microseconds(any ? 20 : 2000));
    }
}

void serve_destroy(ServeState* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->lock);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (auto& kv : S->reqs) {
        ServeReq* q = kv.second;
        if (!q->finished) {
            cudaEventSynchronize(q->done);
            cudaFreeAsync(q->base, S->streams[q->slot]);
        }
        delete q;
    }
    for (int i = 0; i < kServeSlots; ++i) {
        if (S->streams[i]) {
            cudaStreamSynchronize(S->streams[i]);
            cudaStreamDestroy(S->streams[i]);
        }
        if (S->events[i]) cudaEventDestroy(S->events[i]);
    }
    delete S;
}

static int serve_init(fabf_ctx* ctx)
{
    if (ctx->serve) return FABF_OK;
    ServeState* S = new (std::nothrow) ServeState();
    if (!S) return FABF_ENOMEM;
    S->device = ctx->device;
    cudaError_t e = cudaDeviceGetDefaultMemPool(&S->pool, ctx->device);
    if (e == cudaSuccess) {
        uint64_t keep = (uint64_t)ctx->budget;    // keep freed memory for reuse up to the budget
        e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int i = 0; i < kServeSlots && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        serve_destroy(S);
        return cuda_status(e);
    }
    S->worker = std::thread(serve_worker, S);
    ctx->serve = S;
    return FABF_OK;
}

// Enqueue the passes of q on its stream (S->lock held).
static int serve_enqueue(fabf_ctx* ctx, ServeState* S, ServeReq* q)
{
    cudaStream_t s = S->streams[q->slot];
    const fabf_request& r = q->r;
    const long long n = (long long)r.H * r.W;
    const int blocks = (int)((n + 255) / 256);
    int rc = FABF_OK;
    if (r.passes > 1) {
        zeta_kernel<<<blocks, 256, 0, s>>>(q->d_img, q->d_theta, q->d_zeta, n);
        rc = cuda_status(cudaGetLastError());
    }
    for (int p = 0; p < r.passes && rc == FABF_OK; ++p) {
        if (p > 0) {
            next_pass_kernel<<<blocks, 256, 0, s>>>(q->d_out, r.out_is_f64, q->d_zeta, q->d_sigma, r.sigma_decay,
                                                    q->d_img, q->d_theta, n);
            rc = cuda_status(cudaGetLastError());
            if (rc) break;
        }
        const int TH = tile_rows_for(ctx, r.w, r.N, ctx->precision, r.H, r.W);
        rc = run_fused_prec(ctx, ctx->precision, q->d_img, (size_t)r.W, q->d_theta, q->d_sigma, r.H, r.W, r.w,
                            r.N, q->d_out, r.out_is_f64, TH, nullptr, q->d_status, q->d_nfb, s);
    }
    if (rc == FABF_OK && !q->host_out) {
        rc = cuda_status(cudaMemcpyAsync(r.out, q->d_out, (size_t)n * (r.out_is_f64 ? 8 : 4),
                                         cudaMemcpyDeviceToDevice, s));
    }
    if (rc == FABF_OK) rc = cuda_status(cudaEventRecord(q->done, s));
    return rc;
}

}  // namespace fabf

extern "C" {

int fabf_serve_submit(fabf_ctx* ctx, const fabf_request* req, uint64_t* ticket)
{
    if (!ctx || !req || !ticket) return FABF_EINVAL;
    const fabf_request& r = *req;
    int rc = check_filter_args(r.img, r.theta, r.sigma, r.out, r.H, r.W, r.pitch, r.w, r.N);
    if (rc) return rc;
    if (r.passes < 1 || r.passes > 16 || !(r.sigma_decay > 0.0f)) return FABF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    rc = serve_init(ctx);
    if (rc) return rc;
    ServeState* S = ctx->serve;
    const size_t bytes = serve_bytes(r);
    if (bytes > ctx->budget) return FABF_ENOMEM;
    const bool di = is_device_ptr(r.img), dt = is_device_ptr(r.theta), ds = is_device_ptr(r.sigma);
    const bool dout = is_device_ptr(r.out);

    std::unique_lock<std::mutex> lk(S->lock);
    if (S->in_use + bytes > ctx->budget) return FABF_EAGAIN;
    int slot = -1;
    for (int i = 0; i < kServeSlots; ++i)
        if (!S->slot_busy[i]) {
            slot = i;
            break;
        }
    if (slot < 0) return FABF_EAGAIN;
    ServeReq* q = new (std::nothrow) ServeReq();
    if (!q) return FABF_ENOMEM;
    q->r = r;
    q->slot = slot;
    q->bytes = bytes;
    q->host_out = !dout;
    q->done = S->events[slot];
    cudaStream_t s = S->streams[slot];
    void* base = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&base, bytes, S->pool, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete q;
        return FABF_ENOMEM;
    }
    const size_t n = (size_t)r.H * r.W;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    uint8_t* p = static_cast<uint8_t*>(base);
    q->base = p;
    q->d_img = p;
    p += up(n);
    q->d_theta = reinterpret_cast<float*>(p);
    p += up(n * 4);
    q->d_sigma = reinterpret_cast<float*>(p);
    p += up(n * 4);
    q->d_zeta = reinterpret_cast<float*>(p);
    p += up(n * 4);
    q->d_out = p;
    p += up(n * (r.out_is_f64 ? 8 : 4));
    q->d_status = reinterpret_cast<unsigned*>(p);
    q->d_nfb = reinterpret_cast<unsigned long long*>(p + 8);
    // inputs are copied at admission: the caller's buffers are free on return
    e = cudaMemsetAsync(q->d_status, 0, 32, s);   // status, fallback and redo words
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(q->d_img, r.W, r.img, r.pitch, r.W, r.H,
                              di ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->d_theta, r.theta, n * 4, dt ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->d_sigma, r.sigma, n * 4, ds ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && (di || dt || ds)) e = cudaStreamSynchronize(s);   // device sources: copy done
    rc = cuda_status(e);
    if (rc == FABF_OK) rc = serve_enqueue(ctx, S, q);
    if (rc != FABF_OK) {
        (void)cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaFreeAsync(base, s);
        delete q;
        return rc;
    }
    S->slot_busy[slot] = true;
    S->in_use += bytes;
    q->ticket = S->next_ticket++;
    S->reqs[q->ticket] = q;
    *ticket = q->ticket;
    lk.unlock();
    S->cv.notify_all();
    return FABF_OK;
}

int fabf_serve_poll(fabf_ctx* ctx, uint64_t ticket, int timeout_us, int* result)
{
    if (!ctx || !result || timeout_us < 0) return FABF_EINVAL;
    ServeState* S = ctx->serve;
    if (!S) return FABF_ENOTFOUND;
    std::unique_lock<std::mutex> lk(S->lock);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return FABF_ENOTFOUND;
    ServeReq* q = it->second;
    if (!q->finished && timeout_us > 0) {
        S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return q->finished; });
    }
    if (!q->finished) return FABF_EAGAIN;
    *result = q->result;
    S->reqs.erase(it);
    delete q;
    return FABF_OK;
}

int fabf_serve_stats(fabf_ctx* ctx, uint64_t* bytes_in_use, int* in_flight)
{
    if (!ctx) return FABF_EINVAL;
    size_t b = 0;
    int n = 0;
    if (ctx->serve) {
        std::lock_guard<std::mutex> g(ctx->serve->lock);
        b = ctx->serve->in_use;
        for (auto& kv : ctx->serve->reqs) n += kv.second->finished ? 0 : 1;
    }
    if (bytes_in_use) *bytes_in_use = b;
    if (in_flight) *in_flight = n;
    return FABF_OK;
}

int fabf_batch_stats(fabf_ctx* ctx, int* graph_captures, int* graph_launches)
{
    if (!ctx) return FABF_EINVAL;
    if (graph_captures) *graph_captures = ctx->batch ? ctx->batch->captures : 0;
    if (graph_launches) *graph_launches = ctx->batch ? ctx->batch->launches : 0;
    return FABF_OK;
}

int fabf_tile_rows(fabf_ctx* ctx, int w, int N, int precision, int* tile_rows)
{
    if (!ctx || !tile_rows || w < 1 || N < 0 || precision < FABF_FP64 || precision > FABF_C32) return FABF_EINVAL;
    if (w > kWMax || N > kNMax) return FABF_EUNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FABF_ECUDA;
    *tile_rows = tile_rows_for(ctx, w, N, precision, 0, 0);
    return FABF_OK;
}

}  // extern "C"

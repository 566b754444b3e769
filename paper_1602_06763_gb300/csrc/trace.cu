// Per-kernel tracing: device time, launch count and algorithmic work per
// kernel kind, measured with CUDA events on the launching stream.  This is
// the GPU counterpart of the paper's per-kernel time and efficiency breakdown
// (Fig. 2 and Fig. 5, Section 3).  Off by default; while off, a launch costs
// one relaxed atomic load more than an untraced launch.
#include <mutex>
#include <vector>
#include "internal.cuh"

namespace rl {

std::atomic<int> g_trace_on{0};

namespace {

struct Rec {
    int kind;
    double flops, bytes;
    cudaEvent_t e0, e1;
};

struct Totals {
    uint64_t launches = 0;
    double ms = 0.0, flops = 0.0, bytes = 0.0;
};

std::mutex g_mu;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
Totals g_tot[K_COUNT];

const char *kKindNames[K_COUNT] = {"gemm", "syrk", "trsm_base", "trmm_base", "potf2",
                                   "trti2", "lauu2", "diag_scan", "getf2_panel", "laswp",
                                   "fp64_residual", "convert", "refine_control", "batched",
                                   "trsm_flow", "uplo_swap"};

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_locked()
{
    for (Rec &r : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            Totals &t = g_tot[r.kind];
            t.launches += 1;
            t.ms += ms;
            t.flops += r.flops;
            t.bytes += r.bytes;
        }
        g_pool.push_back(r.e0);
        g_pool.push_back(r.e1);
    }
    g_pending.clear();
}

}  // namespace

Launch::Launch(Ctx &ctx, int k, double f, double b) : c(ctx), kind(k), flops(f), bytes(b)
{
    if (g_trace_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaEvent_t e = take_event();
        if (e && cudaEventRecord(e, c.s) == cudaSuccess) ev0 = e;
    }
}

Launch::~Launch()
{
    count_launch();
    note(c, cudaGetLastError());
    if (ev0) {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaEvent_t e1 = take_event();
        if (e1 && cudaEventRecord(e1, c.s) == cudaSuccess)
            g_pending.push_back(Rec{kind, flops, bytes, (cudaEvent_t)ev0, e1});
        else
            g_pool.push_back((cudaEvent_t)ev0);
    }
}

}  // namespace rl

using namespace rl;

extern "C" {

int rl_trace_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (on) {
        drain_locked();
        for (Totals &t : g_tot) t = Totals();
    }
    g_trace_on.store(on ? 1 : 0);
    return RL_SUCCESS;
}

int rl_trace_kinds(void) { return K_COUNT; }

}  // extern "C"

namespace rl {
// Tracing off, pending records read, pooled events destroyed.
cudaError_t trace_release()
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_trace_on.store(0);
    drain_locked();
    cudaError_t first = cudaSuccess;
    for (cudaEvent_t e : g_pool) {
        const cudaError_t r = cudaEventDestroy(e);
        if (first == cudaSuccess) first = r;
    }
    g_pool.clear();
    return first;
}
}  // namespace rl

extern "C" {

int rl_trace_read(int kind, const char **name, uint64_t *launches, double *ms, double *flops,
                  double *bytes)
{
    if (kind < 0 || kind >= K_COUNT) return RL_ERR_PARAM;
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    const Totals &t = g_tot[kind];
    if (name) *name = kKindNames[kind];
    if (launches) *launches = t.launches;
    if (ms) *ms = t.ms;
    if (flops) *flops = t.flops;
    if (bytes) *bytes = t.bytes;
    return RL_SUCCESS;
}

}  // extern "C"

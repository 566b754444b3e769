// Batched LU with library-owned scratch: rl_dgetrf_vbatched_noalloc.
//
// For callers that cannot allocate device memory at the point of the call:
// code that runs where a cudaMalloc would synchronize the device or is not
// permitted (a real-time or latency-critical loop, a plugin or C host
// without a device allocator of its own), or that must not grow the
// process's memory footprint.  The scratch of the batched kernels (a work
// counter and the size-sorted matrix order, 256 + 4 * batch bytes) lives in
// one file-scope __device__ array of fixed size instead of a caller buffer.
//
// The array is shared by every call on a device: calls that overlap in time
// (on different streams or from different host threads without ordering)
// race on it.  Nothing in it has to start at zero: the sort kernel of each
// call writes the order list and resets the work counter before the
// factorization kernel reads them.
#include <mutex>

#include "internal.cuh"

namespace rl {
namespace {

// Largest batch served from the static scratch.
constexpr int64_t NOALLOC_MAX_BATCH = 65536;
// 256 bytes of counter and padding, then one int per matrix.
constexpr size_t NOALLOC_BYTES = 256 + (size_t)NOALLOC_MAX_BATCH * sizeof(int32_t);

__device__ __align__(256) unsigned char g_batch_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 128;
std::mutex g_mu;
void *g_scratch[NOALLOC_MAX_DEVICES];      // device address of g_batch_scratch, per device

// Device address of the scratch on the current device, resolved once per
// device (the first call on a device does this set-up).
cudaError_t scratch_ptr(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace rl

using namespace rl;

extern "C" {

int rl_dgetrf_vbatched_noalloc(int64_t batch, const int32_t *n, double *const *A, const int32_t *lda,
                               int32_t *const *ipiv, int32_t *info, int32_t max_n, rl_stream_t stream)
{
    if (batch < 0) return -1;
    if (batch > NOALLOC_MAX_BATCH) return RL_ERR_UNSUPPORTED;
    if (batch == 0) return RL_SUCCESS;
    if (rl_getrf_vbatched_work_size(batch) > NOALLOC_BYTES) return RL_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    if (scratch_ptr(&scratch) != cudaSuccess) return RL_ERR_CUDA;
    return rl_dgetrf_vbatched(batch, n, A, lda, ipiv, info, max_n, scratch, NOALLOC_BYTES, stream);
}

}  // extern "C"

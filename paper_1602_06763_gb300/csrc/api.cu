// C ABI and recursion scheduler.
//
// The host walks the recursion tree of each routine (Section 3: halve,
// recurse on the first half, BLAS-3 update, recurse on the second half, base
// case below the crossover c) and enqueues one kernel per BLAS-3 call and per
// base case on the caller's stream.  Nothing synchronizes, nothing allocates:
// a call can be captured into a CUDA graph by the caller.  A device-side
// abort word (the call's info) lets later kernels skip their work once a
// Cholesky pivot failed or a zero diagonal was found.
#include <cstring>
#include <mutex>
#include <vector>
#include "internal.cuh"

#include <cstdio>
#include <map>
#include <nvtx3/nvToolsExt.h>

namespace rl {

std::atomic<uint64_t> g_launches{0};
Params g_params;

int device_sms()
{
    static int cache[128];
    static std::once_flag once;
    std::call_once(once, [] { for (int &v : cache) v = 0; });
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 1;
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

void note(Ctx &c, cudaError_t e)
{
    if (e != cudaSuccess && c.err == cudaSuccess) c.err = e;
}

cudaError_t smem_optin(const void *func, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, func);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

// ---- lookahead resources ----------------------------------------------------
// One internal stream per device for the trailing updates that run beside
// the recursion (created once, lowest priority so the factorization's own
// kernels are preferred), and per host thread a pool of events indexed by
// recursion depth: calls from different threads never share an event, and
// calls that share the stream only serialize their side work on it.
namespace {
constexpr int LA_DEPTH = 48;
cudaStream_t g_side[128];
std::mutex g_side_mu;

struct LaEvents {
    cudaEvent_t start[LA_DEPTH] = {}, done[LA_DEPTH] = {};
    bool ready = false, failed = false;
};
thread_local LaEvents t_ev[128];
}  // namespace

// Side stream and this thread's events for the current device, or false
// (then the recursion runs on the caller's stream alone).
static bool lookahead_resources(cudaStream_t *side, LaEvents **ev)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return false;
    {
        std::lock_guard<std::mutex> lock(g_side_mu);
        if (g_side[dev] == nullptr) {
            int lo = 0, hi = 0;
            cudaStream_t s = nullptr;
            if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
                cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, lo) != cudaSuccess)
                return false;
            g_side[dev] = s;
        }
        *side = g_side[dev];
    }
    LaEvents &e = t_ev[dev];
    if (e.failed) return false;
    if (!e.ready) {
        for (int i = 0; i < LA_DEPTH; ++i)
            if (cudaEventCreateWithFlags(&e.start[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&e.done[i], cudaEventDisableTiming) != cudaSuccess) {
                e.failed = true;
                return false;
            }
        e.ready = true;
    }
    *ev = &e;
    return true;
}

// A copy stream per device for the host-buffer calls (created once).
static cudaStream_t g_copy[128];

static cudaStream_t copy_stream()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
    std::lock_guard<std::mutex> lock(g_side_mu);
    if (g_copy[dev] == nullptr) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        g_copy[dev] = s;
    }
    return g_copy[dev];
}

// The side stream may run GEMMs concurrently with the caller's stream only
// when no GEMM of the call stages operands in a shared workspace (the
// tensor-core updates pack into c.tcwork).
static bool lookahead_ok(const Ctx &c)
{
    // one packing workspace per stream: the tensor-core FP32 updates share
    // one, the emulated FP64 updates may bring a second for the side stream
    return g_params.lookahead && c.tcwork == nullptr && (c.ozwork == nullptr || c.ozwork2 != nullptr);
}

// NVTX range of one recursion node ("potrf n=4096 d=1") when RL_PARAM_NVTX
// is set, for timeline tools (Figs. 2 and 5 break the time down per call and
// per recursion level); nothing is pushed otherwise.
struct NvtxNode {
    bool on;
    NvtxNode(const char *routine, i64 n, int depth) : on(g_params.nvtx != 0)
    {
        if (!on) return;
        char buf[64];
        snprintf(buf, sizeof buf, "%s n=%lld d=%d", routine, (long long)n, depth);
        nvtxRangePushA(buf);
    }
    ~NvtxNode()
    {
        if (on) nvtxRangePop();
    }
};

// ---- recursions -------------------------------------------------------------

// Cholesky: potrf(A11); A21 := A21 L11^{-T}; A22 -= A21 A21^T; potrf(A22).
//
// Lookahead (as for the LU below): the SYRK update of A22 is split at the
// next level's split n2a; its leading n2a x n2a block runs on the caller's
// stream, the rest (a GEMM below it and the trailing SYRK) on the side
// stream, waited on only before the next level's TRSM.
template <typename T>
static void potrf_rec_la(Ctx &c, i64 n, T *A, i64 lda, i64 off, cudaEvent_t pending, int depth)
{
    if (n <= 0) return;
    NvtxNode nv("potrf", n, depth);
    if (n <= g_params.potrf_c) {
        if (pending) note(c, cudaStreamWaitEvent(c.s, pending, 0));
        potf2<T>(c, n, A, lda, off);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    T *A21 = A + n1, *A22 = A + n1 + n1 * lda;
    potrf_rec_la<T>(c, n1, A, lda, off, nullptr, depth + 1);
    if (pending) note(c, cudaStreamWaitEvent(c.s, pending, 0));
    trsm_rlt<T>(c, n2, n1, T(1), A, lda, A21, lda);
    if (depth == 0 && c.left_done) note(c, cudaEventRecord(c.left_done, c.s));
    if (depth == 0 && c.trail_ready) note(c, cudaStreamWaitEvent(c.s, c.trail_ready, 0));
    cudaStream_t side = nullptr;
    LaEvents *ev = nullptr;
    cudaEvent_t next_pending = nullptr;
    const i64 n2a = split_q(n2, TRX_NB);
    if (lookahead_ok(c) && depth < LA_DEPTH && n2 >= LA_MIN_N && n2 > g_params.potrf_c &&
        lookahead_resources(&side, &ev)) {
        gemm<T>(c, false, true, n2a, n2a, n1, T(-1), A21, lda, A21, lda, T(1), A22, lda, true);
        note(c, cudaEventRecord(ev->start[depth], c.s));
        Ctx cs = c;
        cs.s = side;
        cs.ozwork = c.ozwork2;
        cs.ozlwork = c.ozlwork2;
        note(cs, cudaStreamWaitEvent(side, ev->start[depth], 0));
        const i64 nr = n2 - n2a;
        gemm<T>(cs, false, true, nr, n2a, n1, T(-1), A21 + n2a, lda, A21, lda, T(1), A22 + n2a, lda);
        gemm<T>(cs, false, true, nr, nr, n1, T(-1), A21 + n2a, lda, A21 + n2a, lda, T(1),
                A22 + n2a + n2a * lda, lda, true);
        note(cs, cudaEventRecord(ev->done[depth], side));
        if (cs.err != cudaSuccess) note(c, cs.err);
        next_pending = ev->done[depth];
    } else {
        gemm<T>(c, false, true, n2, n2, n1, T(-1), A21, lda, A21, lda, T(1), A22, lda, true);
    }
    potrf_rec_la<T>(c, n2, A22, lda, off + n1, next_pending, depth + 1);
}

template <typename T>
void potrf_rec_t(Ctx &c, i64 n, T *A, i64 lda, i64 off)
{
    potrf_rec_la<T>(c, n, A, lda, off, nullptr, 0);
}

// LU of the m x n block whose top-left corner is (r0, r0) of the matrix A0
// (m_tot rows).  Pivots are written as global 1-based rows.
//
// Lookahead: the trailing update A22 -= A21 A12 is split by columns at the
// next level's own split; the left part (all the next level factors first)
// runs on the caller's stream, the right part on the side stream, and
// `pending` (recorded after it) is waited on only where the next level first
// touches those columns (its row interchanges of the right half).  The
// latency-bound panels of the left part thus overlap the right part's GEMM.
// Every element sees the same operations in the same order either way.
template <typename T>
static void getrf_rec_la(Ctx &c, T *A0, i64 lda, i64 m_tot, int32_t *ipiv, i64 r0, i64 m, i64 n,
                         cudaEvent_t pending, int depth)
{
    if (m <= 0 || n <= 0) return;
    NvtxNode nv("getrf", n, depth);
    T *A = A0 + r0 + r0 * lda;
    const i64 nb = is_cplx<T>::value && g_params.getrf_nb > 32 ? 32 : g_params.getrf_nb;   // complex panels <= 32
    if (n <= nb) {
        if (pending) note(c, cudaStreamWaitEvent(c.s, pending, 0));
        getf2_panel<T>(c, m, n, A, lda, ipiv, r0);
        return;
    }
    if (m < n) {
        // wide: factor the leading m x m block, then swap and solve the rest
        if (pending) note(c, cudaStreamWaitEvent(c.s, pending, 0));
        getrf_rec_la<T>(c, A0, lda, m_tot, ipiv, r0, m, m, nullptr, depth + 1);
        if (depth == 0 && c.trail_ready) note(c, cudaStreamWaitEvent(c.s, c.trail_ready, 0));
        laswp<T>(c, A0, lda, m_tot, r0 + m, n - m, r0, r0 + m, ipiv);
        trsm_lln<T>(c, true, m, n - m, T(1), A, lda, A + m * lda, lda);
        return;
    }
    const i64 n1 = split_q(n, n > 2 * TRX_NB ? TRX_NB : nb), n2 = n - n1;
    getrf_rec_la<T>(c, A0, lda, m_tot, ipiv, r0, m, n1, nullptr, depth + 1);
    if (pending) note(c, cudaStreamWaitEvent(c.s, pending, 0));
    if (depth == 0 && c.trail_ready) note(c, cudaStreamWaitEvent(c.s, c.trail_ready, 0));
    laswp<T>(c, A0, lda, m_tot, r0 + n1, n2, r0, r0 + n1, ipiv);
    trsm_lln<T>(c, true, n1, n2, T(1), A, lda, A + n1 * lda, lda);
    T *A21 = A + n1, *A12 = A + n1 * lda, *A22 = A + n1 + n1 * lda;
    cudaEvent_t next_pending = nullptr;
    cudaStream_t side = nullptr;
    LaEvents *ev = nullptr;
    const i64 m2 = m - n1;
    // the next level's split of its n2 columns (the rule above, at order n2)
    const i64 n2a = split_q(n2, n2 > 2 * TRX_NB ? TRX_NB : nb);
    if (lookahead_ok(c) && depth < LA_DEPTH && n2 >= LA_MIN_N && m2 >= n2 &&
        lookahead_resources(&side, &ev)) {
        gemm<T>(c, false, false, m2, n2a, n1, T(-1), A21, lda, A12, lda, T(1), A22, lda);
        note(c, cudaEventRecord(ev->start[depth], c.s));
        Ctx cs = c;
        cs.s = side;
        cs.ozwork = c.ozwork2;
        cs.ozlwork = c.ozlwork2;
        note(cs, cudaStreamWaitEvent(side, ev->start[depth], 0));
        gemm<T>(cs, false, false, m2, n2 - n2a, n1, T(-1), A21, lda, A12 + n2a * lda, lda, T(1),
                A22 + n2a * lda, lda);
        note(cs, cudaEventRecord(ev->done[depth], side));
        if (cs.err != cudaSuccess) note(c, cs.err);
        next_pending = ev->done[depth];
    } else {
        gemm<T>(c, false, false, m2, n2, n1, T(-1), A21, lda, A12, lda, T(1), A22, lda);
    }
    getrf_rec_la<T>(c, A0, lda, m_tot, ipiv, r0 + n1, m2, n2, next_pending, depth + 1);
    const i64 mn2 = m2 < n2 ? m2 : n2;
    laswp<T>(c, A0, lda, m_tot, r0, n1, r0 + n1, r0 + n1 + mn2, ipiv);
}

template <typename T>
void getrf_rec_t(Ctx &c, T *A0, i64 lda, i64 m_tot, int32_t *ipiv, i64 r0, i64 m, i64 n)
{
    getrf_rec_la<T>(c, A0, lda, m_tot, ipiv, r0, m, n, nullptr, 0);
}

template void potrf_rec_t<double>(Ctx &, i64, double *, i64, i64);
template void potrf_rec_t<float>(Ctx &, i64, float *, i64, i64);
template void getrf_rec_t<double>(Ctx &, double *, i64, i64, int32_t *, i64, i64, i64);
template void getrf_rec_t<float>(Ctx &, float *, i64, i64, int32_t *, i64, i64, i64);
template void potrf_rec_t<cplx>(Ctx &, i64, cplx *, i64, i64);
template void getrf_rec_t<cplx>(Ctx &, cplx *, i64, i64, int32_t *, i64, i64, i64);

static void potrf_rec(Ctx &c, i64 n, double *A, i64 lda, i64 off) { potrf_rec_t<double>(c, n, A, lda, off); }
static void getrf_rec(Ctx &c, double *A0, i64 lda, i64 m_tot, int32_t *ipiv, i64 r0, i64 m, i64 n)
{
    getrf_rec_t<double>(c, A0, lda, m_tot, ipiv, r0, m, n);
}

// Triangular inverse, Fig. 4: trtri(TL); BL := BL TL; BL := -BR^{-1} BL;
// trtri(BR).
template <typename T>
void trtri_rec(Ctx &c, bool unit, i64 n, T *A, i64 lda)
{
    if (n <= 0) return;
    NvtxNode nv("trtri", n, -1);
    const i64 base = sizeof(T) > 8 && g_params.trtri_c > 32 ? 32 : g_params.trtri_c;   // complex: <= 32
    if (n <= base) { trti2<T>(c, unit, n, A, lda); return; }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    T *BL = A + n1, *BR = A + n1 + n1 * lda;
    trtri_rec<T>(c, unit, n1, A, lda);
    trmm_rln<T>(c, unit, n2, n1, T(1), A, lda, BL, lda);
    trsm_lln<T>(c, unit, n2, n1, T(-1), BR, lda, BL, lda);
    trtri_rec<T>(c, unit, n2, BR, lda);
}
template void trtri_rec<double>(Ctx &, bool, i64, double *, i64);
template void trtri_rec<float>(Ctx &, bool, i64, float *, i64);
template void trtri_rec<cplx>(Ctx &, bool, i64, cplx *, i64);

// A := L^T L: lauum(A11); A11 += A21^T A21; A21 := A22^T A21; lauum(A22)
// (complex: L^H L, with conjugate transposes throughout).
template <typename T>
static void lauum_rec(Ctx &c, i64 n, T *A, i64 lda)
{
    if (n <= 0) return;
    NvtxNode nv("lauum", n, -1);
    const i64 base = sizeof(T) > 8 && g_params.trtri_c > 32 ? 32 : g_params.trtri_c;
    if (n <= base) { lauu2<T>(c, n, A, lda); return; }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    T *A21 = A + n1, *A22 = A + n1 + n1 * lda;
    lauum_rec<T>(c, n1, A, lda);
    gemm<T>(c, true, false, n1, n1, n2, T(1), A21, lda, A21, lda, T(1), A, lda, true);
    trmm_llt<T>(c, n2, n1, T(1), A22, lda, A21, lda);
    lauum_rec<T>(c, n2, A22, lda);
}

static bool is_l(char u) { return u == 'L' || u == 'l'; }
static bool is_u(char u) { return u == 'U' || u == 'u'; }

static int finish(Ctx &c)
{
    if (c.err == cudaSuccess) c.err = cudaGetLastError();
    return c.err == cudaSuccess ? RL_SUCCESS : RL_ERR_CUDA;
}

static Ctx make_ctx(rl_stream_t s, int32_t *info, void *work, size_t lwork)
{
    Ctx c;
    c.s = reinterpret_cast<cudaStream_t>(s);
    c.info = info;
    c.work = work;
    c.lwork = lwork;
    c.num_sms = device_sms();
    return c;
}

}  // namespace rl

using namespace rl;

extern "C" {

int rl_dpotrf(char uplo, int64_t n, double *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    (void)work; (void)lwork;
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (n > 0 && A == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<double>(c, n, A, lda);
    potrf_rec(c, n, A, lda, 0);
    if (up) uplo_swap<double>(c, n, A, lda);
    return finish(c);
}

size_t rl_dgetrf_work_size(int64_t m, int64_t n)
{
    (void)m; (void)n;
    return panel_ws_bytes();
}

int rl_dgetrf(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m > 0 && n > 0 && A == nullptr) return -3;
    if (lda < (m > 1 ? m : 1)) return -4;
    if (m > INT32_MAX - 1) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || (ipiv == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    if (m > 0 && n > 0 && (work == nullptr || lwork < rl_dgetrf_work_size(m, n))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = nullptr;   // a zero pivot does not stop the LU factorization
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    getrf_rec(c, A, lda, m, ipiv, 0, m, n);
    return finish(c);
}

}  // extern "C"

template <typename T>
static int trtri_api(char uplo, char diag, int64_t n, T *A, int64_t lda, int32_t *info, void *work,
                     size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    const bool unit = (diag == 'U' || diag == 'u');
    if (!unit && diag != 'N' && diag != 'n') return -2;
    if (n < 0) return -3;
    if (n > 0 && A == nullptr) return -4;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<T>(c, n, A, lda);
    if (!unit) diag_zero_scan<T>(c, n, A, lda);
    trtri_rec<T>(c, unit, n, A, lda);
    if (up) uplo_swap<T>(c, n, A, lda);
    return finish(c);
}

// potri = false: A := L^T L (lauum); true: A := (L L^T)^{-1} = L^{-T} L^{-1}
template <typename T>
static int lauum_api(bool potri, char uplo, int64_t n, T *A, int64_t lda, int32_t *info, void *work,
                     size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (n > 0 && A == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<T>(c, n, A, lda);
    if (potri) {
        diag_zero_scan<T>(c, n, A, lda);
        trtri_rec<T>(c, false, n, A, lda);
    }
    lauum_rec<T>(c, n, A, lda);
    if (up) uplo_swap<T>(c, n, A, lda);
    return finish(c);
}

extern "C" {

int rl_dtrtri(char uplo, char diag, int64_t n, double *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream)
{
    return trtri_api<double>(uplo, diag, n, A, lda, info, work, lwork, stream);
}

int rl_dlauum(char uplo, int64_t n, double *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return lauum_api<double>(false, uplo, n, A, lda, info, work, lwork, stream);
}

int rl_dpotri(char uplo, int64_t n, double *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return lauum_api<double>(true, uplo, n, A, lda, info, work, lwork, stream);
}

int rl_strtri(char uplo, char diag, int64_t n, float *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream)
{
    return trtri_api<float>(uplo, diag, n, A, lda, info, work, lwork, stream);
}

int rl_slauum(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return lauum_api<float>(false, uplo, n, A, lda, info, work, lwork, stream);
}

int rl_spotri(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return lauum_api<float>(true, uplo, n, A, lda, info, work, lwork, stream);
}

// ---- BLAS-3 layer ------------------------------------------------------------

static bool is_n(char t) { return t == 'N' || t == 'n'; }
static bool is_t(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }
static i64 imax1(i64 v) { return v > 1 ? v : 1; }

}  // extern "C"

template <typename T>
static int gemm_api(char transa, char transb, int64_t m, int64_t n, int64_t k, T alpha, const T *A,
                    int64_t lda, const T *B, int64_t ldb, T beta, T *C, int64_t ldc, rl_stream_t stream)
{
    if (!is_n(transa) && !is_t(transa)) return -1;
    if (!is_n(transb) && !is_t(transb)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    const bool ta = is_t(transa), tb = is_t(transb);
    if (lda < imax1(ta ? k : m)) return -8;
    if (ldb < imax1(tb ? n : k)) return -10;
    if (ldc < imax1(m)) return -13;
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    gemm<T>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, false);
    return finish(c);
}

template <typename T>
static int syrk_api(char uplo, char trans, int64_t n, int64_t k, T alpha, const T *A, int64_t lda, T beta,
                    T *C, int64_t ldc, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (!is_n(trans) && !is_t(trans)) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    const bool t = is_t(trans);
    if (lda < imax1(t ? k : n)) return -7;
    if (ldc < imax1(n)) return -10;
    if (is_u(uplo)) return RL_ERR_UNSUPPORTED;
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    gemm<T>(c, t, !t, n, n, k, alpha, A, lda, A, lda, beta, C, ldc, true);
    return finish(c);
}

extern "C" {

int rl_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
             const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
             int64_t ldc, rl_stream_t stream)
{
    return gemm_api<double>(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

int rl_dsyrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double *A,
             int64_t lda, double beta, double *C, int64_t ldc, rl_stream_t stream)
{
    return syrk_api<double>(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, stream);
}

int rl_sgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha, const float *A,
             int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
             rl_stream_t stream)
{
    return gemm_api<float>(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

int rl_ssyrk(char uplo, char trans, int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
             float beta, float *C, int64_t ldc, rl_stream_t stream)
{
    return syrk_api<float>(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, stream);
}

static int check_tr(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                    int64_t lda, int64_t ldb)
{
    const bool left = (side == 'L' || side == 'l');
    if (!left && side != 'R' && side != 'r') return -1;
    if (!is_l(uplo) && !is_u(uplo)) return -2;
    if (!is_n(transa) && !is_t(transa)) return -3;
    if (diag != 'N' && diag != 'n' && diag != 'U' && diag != 'u') return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (lda < imax1(left ? m : n)) return -9;
    if (ldb < imax1(m)) return -11;
    return 0;
}

int rl_dtrsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha,
             const double *A, int64_t lda, double *B, int64_t ldb, rl_stream_t stream)
{
    int st = check_tr(side, uplo, transa, diag, m, n, lda, ldb);
    if (st) return st;
    const bool left = (side == 'L' || side == 'l'), lower = is_l(uplo), tr = is_t(transa);
    const bool unit = (diag == 'U' || diag == 'u');
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    if (lower && left && !tr) trsm_lln(c, unit, m, n, alpha, A, lda, B, ldb);
    else if (lower && left && tr && !unit) trsm_llt(c, m, n, alpha, A, lda, B, ldb);
    else if (lower && !left && tr && !unit) trsm_rlt(c, m, n, alpha, A, lda, B, ldb);
    else if (!lower && left && !tr && !unit) trsm_lun(c, m, n, alpha, A, lda, B, ldb);
    else return RL_ERR_UNSUPPORTED;
    return finish(c);
}

int rl_dtrmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha,
             const double *A, int64_t lda, double *B, int64_t ldb, rl_stream_t stream)
{
    int st = check_tr(side, uplo, transa, diag, m, n, lda, ldb);
    if (st) return st;
    const bool left = (side == 'L' || side == 'l'), lower = is_l(uplo), tr = is_t(transa);
    const bool unit = (diag == 'U' || diag == 'u');
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    if (lower && !left && !tr) trmm_rln(c, unit, m, n, alpha, A, lda, B, ldb);
    else if (lower && left && tr && !unit) trmm_llt(c, m, n, alpha, A, lda, B, ldb);
    else return RL_ERR_UNSUPPORTED;
    return finish(c);
}

// ---- single precision peers -----------------------------------------------------

// ---- complex double ------------------------------------------------------------

int rl_zpotrf(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (n > 0 && A == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    cplx *Z = reinterpret_cast<cplx *>(A);
    const bool up = is_u(uplo);
    if (up) uplo_swap<cplx>(c, n, Z, lda);      // conjugate transposition: A = U^H U, U = L^H
    potrf_rec_t<cplx>(c, n, Z, lda, 0);
    if (up) uplo_swap<cplx>(c, n, Z, lda);
    return finish(c);
}

int rl_zgetrf(int64_t m, int64_t n, rl_double_complex *A, int64_t lda, int32_t *ipiv, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m > 0 && n > 0 && A == nullptr) return -3;
    if (lda < (m > 1 ? m : 1)) return -4;
    if (m > INT32_MAX - 1) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || (ipiv == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    if (m > 0 && n > 0 && (work == nullptr || lwork < rl_dgetrf_work_size(m, n))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = nullptr;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    getrf_rec_t<cplx>(c, reinterpret_cast<cplx *>(A), lda, m, ipiv, 0, m, n);
    return finish(c);
}


// ---- FP64 factorizations with emulated FP64 updates ---------------------------------
// The recursions of rl_dpotrf / rl_dgetrf with every FP64 GEMM/SYRK update of
// order >= RL_PARAM_OZ_MIN (m, n and k) emulated on the BF16 tensor cores
// (oz_gemm.cu); leaves, panels and smaller updates in native FP64.

static bool oz_slices_ok(int s) { return s >= 6 && s <= 8; }

size_t rl_oz_work_size(int64_t m, int64_t n, int64_t k, int slices)
{
    if (m < 0 || n < 0 || k < 0 || !oz_slices_ok(slices)) return 0;
    return oz_work_bytes(m, n, k, slices);
}

int rl_dgemm_oz(int slices, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                void *work, size_t lwork, rl_stream_t stream)
{
    if (!oz_slices_ok(slices)) return -1;
    const bool ta = transa == 'T' || transa == 't' || transa == 'C' || transa == 'c';
    const bool tb = transb == 'T' || transb == 't' || transb == 'C' || transb == 'c';
    if (!ta && transa != 'N' && transa != 'n') return -2;
    if (!tb && transb != 'N' && transb != 'n') return -3;
    if (m < 0) return -4;
    if (n < 0) return -5;
    if (k < 0) return -6;
    if (lda < ((ta ? k : m) > 1 ? (ta ? k : m) : 1)) return -9;
    if (ldb < ((tb ? n : k) > 1 ? (tb ? n : k) : 1)) return -11;
    if (ldc < (m > 1 ? m : 1)) return -14;
    if (m == 0 || n == 0) return RL_SUCCESS;
    if (k > (1 << 21) || m > (1 << 30) || n > (1 << 30)) return RL_ERR_UNSUPPORTED;
    if (k > 0 && (work == nullptr || lwork < oz_work_bytes(m, n, k, slices))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    if (k == 0) {
        gemm<double>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, false);   // C := beta C
        return finish(c);
    }
    if (!oz_gemm(c, slices, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, false, work, lwork))
        return RL_ERR_UNSUPPORTED;
    return finish(c);
}

// largest update of the recursions: m rows (<= max(m, n)), n/2 + 64 columns
// and inner dimension, and (wide LU) the solve of the n - m columns
static size_t oz_factor_bytes(int64_t m, int64_t n, int slices)
{
    const i64 big = m > n ? m : n, h = (m < n ? m : n) / 2 + 64;
    return oz_work_bytes(big, big, h, slices);
}

// two halves: the caller's stream and the lookahead's side stream
static size_t oz_potrf_half(int64_t n, int slices)
{
    return (oz_work_bytes(n / 2 + 64, n / 2 + 64, n / 2 + 64, slices) + 1023) & ~(size_t)1023;
}

size_t rl_dpotrf_oz_work_size(int64_t n, int slices)
{
    if (n < 0 || !oz_slices_ok(slices)) return 0;
    return 2 * oz_potrf_half(n, slices);
}

size_t rl_dgetrf_oz_work_size(int64_t m, int64_t n, int slices)
{
    if (m < 0 || n < 0 || !oz_slices_ok(slices)) return 0;
    return ((panel_ws_bytes() + 1023) & ~(size_t)1023) + oz_factor_bytes(m, n, slices);
}

int rl_dpotrf_oz(int slices, char uplo, int64_t n, double *A, int64_t lda, int32_t *info, void *work,
                 size_t lwork, rl_stream_t stream)
{
    if (!oz_slices_ok(slices)) return -1;
    if (!is_l(uplo) && !is_u(uplo)) return -2;
    if (n < 0) return -3;
    if (n > 0 && A == nullptr) return -4;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    if (n > 0 && (work == nullptr || lwork < rl_dpotrf_oz_work_size(n, slices))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, nullptr, 0);
    c.abort = info;
    c.oz_slices = slices;
    const size_t half = oz_potrf_half(n, slices);
    c.ozwork = work;
    c.ozlwork = half;
    c.ozwork2 = n > 0 ? static_cast<char *>(work) + half : nullptr;
    c.ozlwork2 = half;
    c.oz_dynamic = true;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<double>(c, n, A, lda);
    potrf_rec(c, n, A, lda, 0);
    if (up) uplo_swap<double>(c, n, A, lda);
    return finish(c);
}

int rl_dgetrf_oz(int slices, int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info,
                 void *work, size_t lwork, rl_stream_t stream)
{
    if (!oz_slices_ok(slices)) return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (m > 0 && n > 0 && A == nullptr) return -4;
    if (lda < (m > 1 ? m : 1)) return -5;
    if (m > INT32_MAX - 1) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || (ipiv == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    if (m > 0 && n > 0 && (work == nullptr || lwork < rl_dgetrf_oz_work_size(m, n, slices))) return RL_ERR_WORKSPACE;
    const size_t pw = (panel_ws_bytes() + 1023) & ~(size_t)1023;
    Ctx c = make_ctx(stream, info, work, pw);
    c.abort = nullptr;
    c.oz_slices = slices;
    c.ozwork = static_cast<char *>(work) + pw;
    c.ozlwork = lwork > pw ? lwork - pw : 0;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    getrf_rec(c, A, lda, m, ipiv, 0, m, n);
    return finish(c);
}

// ---- low-precision factorizations (FP32 storage, tensor-core updates) --------
// The factorization step of the precision form as calls of their own: the
// recursions of rl_spotrf / rl_sgetrf with every large GEMM/SYRK update on
// tcgen05 in precision `prec` (TF32, BF16, scaled-free FP16, 3xTF32) with
// FP32 accumulation; panels, leaves and smaller updates in FP32 SIMT.

static size_t lowprec_tc_bytes(int64_t m, int64_t n, int prec)
{
    const i64 h = n / 2 + 64;          // largest update: <= m rows, <= n/2 + 64 columns and depth
    return tc_work_bytes(m > 0 ? m : 1, h, h, prec);
}

size_t rl_spotrf_tc_work_size(int64_t n, int prec)
{
    if (n < 0 || !(prec == RL_PREC_TF32 || prec == RL_PREC_BF16 || prec == RL_PREC_FP16S ||
                   prec == RL_PREC_TF32X3))
        return 0;
    return lowprec_tc_bytes(n, n, prec);
}

size_t rl_sgetrf_tc_work_size(int64_t m, int64_t n, int prec)
{
    if (m < 0 || n < 0 || !(prec == RL_PREC_TF32 || prec == RL_PREC_BF16 || prec == RL_PREC_FP16S ||
                            prec == RL_PREC_TF32X3))
        return 0;
    return ((panel_ws_bytes() + 255) & ~(size_t)255) + lowprec_tc_bytes(m, n, prec);
}

int rl_spotrf_tc(int prec, char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
                 size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -2;
    if (n < 0) return -3;
    if (n > 0 && A == nullptr) return -4;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    const size_t need = rl_spotrf_tc_work_size(n, prec);
    if (need == 0) return RL_ERR_UNSUPPORTED;
    if (work == nullptr || lwork < need) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, nullptr, 0);
    c.abort = info;
    c.prec = prec;
    c.tcwork = work;
    c.tclwork = lwork;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<float>(c, n, A, lda);
    potrf_rec_t<float>(c, n, A, lda, 0);
    if (up) uplo_swap<float>(c, n, A, lda);
    return finish(c);
}

int rl_sgetrf_tc(int prec, int64_t m, int64_t n, float *A, int64_t lda, int32_t *ipiv, int32_t *info,
                 void *work, size_t lwork, rl_stream_t stream)
{
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (m > 0 && n > 0 && A == nullptr) return -4;
    if (lda < (m > 1 ? m : 1)) return -5;
    if (m > INT32_MAX - 1) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || (ipiv == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    const size_t need = rl_sgetrf_tc_work_size(m, n, prec);
    if (need == 0) return RL_ERR_UNSUPPORTED;
    if (work == nullptr || lwork < need) return RL_ERR_WORKSPACE;
    const size_t pw = (panel_ws_bytes() + 255) & ~(size_t)255;
    Ctx c = make_ctx(stream, info, work, pw);
    c.abort = nullptr;
    c.prec = prec;
    c.tcwork = static_cast<char *>(work) + pw;
    c.tclwork = lwork - pw;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    getrf_rec_t<float>(c, A, lda, m, ipiv, 0, m, n);
    return finish(c);
}

int rl_spotrf(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work, size_t lwork,
              rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (n > 0 && A == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    const bool up = is_u(uplo);
    if (up) uplo_swap<float>(c, n, A, lda);
    potrf_rec_t<float>(c, n, A, lda, 0);
    if (up) uplo_swap<float>(c, n, A, lda);
    return finish(c);
}

int rl_sgetrf(int64_t m, int64_t n, float *A, int64_t lda, int32_t *ipiv, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m > 0 && n > 0 && A == nullptr) return -3;
    if (lda < (m > 1 ? m : 1)) return -4;
    if (m > INT32_MAX - 1) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || (ipiv == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    if (m > 0 && n > 0 && (work == nullptr || lwork < rl_dgetrf_work_size(m, n))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = nullptr;
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    getrf_rec_t<float>(c, A, lda, m, ipiv, 0, m, n);
    return finish(c);
}

// ---- tensor-core GEMM on FP32 storage ------------------------------------------

static bool tc_prec(int prec)
{
    return prec == RL_PREC_TF32 || prec == RL_PREC_BF16 || prec == RL_PREC_FP16S || prec == RL_PREC_TF32X3;
}

size_t rl_sgemm_tc_work_size(int64_t m, int64_t n, int64_t k, int prec)
{
    if (!tc_prec(prec) || m < 0 || n < 0 || k < 0) return 0;
    return tc_work_bytes(m, n, k, prec);
}

int rl_sgemm_tc(int prec, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                const float *A, int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc,
                void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_n(transa) && !is_t(transa)) return -2;
    if (!is_n(transb) && !is_t(transb)) return -3;
    if (m < 0) return -4;
    if (n < 0) return -5;
    if (k < 0) return -6;
    const bool ta = is_t(transa), tb = is_t(transb);
    if (lda < imax1(ta ? k : m)) return -9;
    if (ldb < imax1(tb ? n : k)) return -11;
    if (ldc < imax1(m)) return -13;
    if (!tc_prec(prec)) return RL_ERR_UNSUPPORTED;
    if (m == 0 || n == 0 || k == 0) return RL_SUCCESS;
    if (work == nullptr || lwork < tc_work_bytes(m, n, k, prec)) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    if (!tc_gemm(c, prec, ta, tb, m, n, k, alpha, A, lda, B, ldb, C, ldc, false, work, lwork))
        return RL_ERR_UNSUPPORTED;
    return finish(c);
}

// ---- solves with the factors ------------------------------------------------

}  // extern "C"

// X := A^{-1} B from the factors: LU (lu) after the row interchanges, or
// Cholesky.  With a workspace, thin right-hand sides take the one-launch flow
// solve; otherwise the recursive TRSM.
template <typename T>
static int trs_t(bool lu, int64_t n, int64_t nrhs, const T *A, int64_t lda, const int32_t *ipiv, T *B,
                 int64_t ldb, void *work, size_t lwork, rl_stream_t stream, bool up = false, bool trans = false)
{
    if (n == 0 || nrhs == 0) return RL_SUCCESS;
    if (A == nullptr || B == nullptr || (lu && ipiv == nullptr)) return RL_ERR_NULL_POINTER;
    // the one-launch flow solve covers the real 'N' forms; the others recurse
    const bool flow = !is_cplx<T>::value && !trans && work != nullptr && nrhs <= FLOW_MAX_NRHS;
    if (flow && lwork < flow_ws_bytes(n, nrhs)) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, work, lwork);
    // 'U' (Cholesky only): the factor U is transposed in place to L = U^T for
    // the solves and restored before the call returns
    T *Aw = const_cast<T *>(A);
    if (up) uplo_swap<T>(c, n, Aw, lda);
    if constexpr (!is_cplx<T>::value) {
        if (lu && trans) {
            // A^T X = B with P A = L U: U^T Y = B, L^T Z = Y, X = P^T Z
            trsm_lut<T>(c, n, nrhs, T(1), A, lda, B, ldb);
            trsm_llt_u<T>(c, true, n, nrhs, T(1), A, lda, B, ldb);
            laswp_rev<T>(c, B, ldb, n, nrhs, ipiv);
            return finish(c);
        }
    }
    if (lu) laswp<T>(c, B, ldb, n, 0, nrhs, 0, n, ipiv);
    if (flow) {
        if constexpr (!is_cplx<T>::value) {
            note(c, cudaMemsetAsync(work, 0, sizeof(int32_t), c.s));
            trsm_flow<T>(c, FLOW_LN, lu, n, nrhs, A, lda, B, ldb, work);
            trsm_flow<T>(c, lu ? FLOW_UN : FLOW_LT, false, n, nrhs, A, lda, B, ldb, work);
        }
    } else if (lu) {
        trsm_lln<T>(c, true, n, nrhs, T(1), A, lda, B, ldb);
        trsm_lun<T>(c, n, nrhs, T(1), A, lda, B, ldb);
    } else {
        trsm_lln<T>(c, false, n, nrhs, T(1), A, lda, B, ldb);
        trsm_llt<T>(c, n, nrhs, T(1), A, lda, B, ldb);
    }
    if (up) uplo_swap<T>(c, n, Aw, lda);
    return finish(c);
}

template <typename T>
static int getri_api(int64_t n, T *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work, size_t lwork,
                     rl_stream_t stream)
{
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (info == nullptr || (n > 0 && ipiv == nullptr)) return RL_ERR_NULL_POINTER;
    if (n > GETRI_MAX_N) return RL_ERR_UNSUPPORTED;
    Ctx c = make_ctx(stream, info, work, lwork);
    c.abort = info;                               // a zero diagonal of U leaves A unchanged
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    if (n == 0) return finish(c);
    if (work == nullptr || lwork < getri_work_bytes(n)) return RL_ERR_WORKSPACE;
    getri<T>(c, n, A, lda, ipiv, work);
    return finish(c);
}

extern "C" {

size_t rl_dgetri_work_size(int64_t n) { return n <= 0 ? 0 : getri_work_bytes(n); }
size_t rl_sgetri_work_size(int64_t n) { return n <= 0 ? 0 : getri_work_bytes(n); }

int rl_dgetri(int64_t n, double *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work, size_t lwork,
              rl_stream_t stream)
{
    return getri_api<double>(n, A, lda, ipiv, info, work, lwork, stream);
}

int rl_sgetri(int64_t n, float *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work, size_t lwork,
              rl_stream_t stream)
{
    return getri_api<float>(n, A, lda, ipiv, info, work, lwork, stream);
}

// complex double inversions (the recursions above with conjugate transposes)
size_t rl_zgetri_work_size(int64_t n) { return n <= 0 ? 0 : getri_work_bytes(n); }

int rl_zgetri(int64_t n, rl_double_complex *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return getri_api<cplx>(n, reinterpret_cast<cplx *>(A), lda, ipiv, info, work, lwork, stream);
}

int rl_ztrtri(char uplo, char diag, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream)
{
    return trtri_api<cplx>(uplo, diag, n, reinterpret_cast<cplx *>(A), lda, info, work, lwork, stream);
}

int rl_zlauum(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work, size_t lwork,
              rl_stream_t stream)
{
    return lauum_api<cplx>(false, uplo, n, reinterpret_cast<cplx *>(A), lda, info, work, lwork, stream);
}

int rl_zpotri(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work, size_t lwork,
              rl_stream_t stream)
{
    return lauum_api<cplx>(true, uplo, n, reinterpret_cast<cplx *>(A), lda, info, work, lwork, stream);
}

}  // extern "C"

template <typename T>
static int sygst_api(int itype, char uplo, int64_t n, T *A, int64_t lda, const T *B, int64_t ldb, void *work,
                     size_t lwork, rl_stream_t stream)
{
    if (itype < 1 || itype > 3) return -1;
    if (!is_l(uplo) && !is_u(uplo)) return -2;
    if (n < 0) return -3;
    if (n > 0 && A == nullptr) return -4;
    if (lda < imax1(n)) return -5;
    if (n > 0 && B == nullptr) return -6;
    if (ldb < imax1(n)) return -7;
    if (n == 0) return RL_SUCCESS;
    if (work != nullptr && lwork < sygst_work_bytes(n, sizeof(T))) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, work, lwork);
    const bool up = is_u(uplo);
    T *Bw = const_cast<T *>(B);      // 'U': B is transposed in place and restored before the call returns
    if (up) { uplo_swap<T>(c, n, A, lda); uplo_swap<T>(c, n, Bw, ldb); }
    sygst_rec<T>(c, itype, n, A, lda, B, ldb, static_cast<T *>(work));
    if (up) { uplo_swap<T>(c, n, A, lda); uplo_swap<T>(c, n, Bw, ldb); }
    return finish(c);
}

extern "C" {

size_t rl_dsygst_work_size(int64_t n) { return n <= 0 ? 0 : sygst_work_bytes(n, sizeof(double)); }
size_t rl_ssygst_work_size(int64_t n) { return n <= 0 ? 0 : sygst_work_bytes(n, sizeof(float)); }

int rl_dsygst(int itype, char uplo, int64_t n, double *A, int64_t lda, const double *B, int64_t ldb,
              void *work, size_t lwork, rl_stream_t stream)
{
    return sygst_api<double>(itype, uplo, n, A, lda, B, ldb, work, lwork, stream);
}

int rl_ssygst(int itype, char uplo, int64_t n, float *A, int64_t lda, const float *B, int64_t ldb,
              void *work, size_t lwork, rl_stream_t stream)
{
    return sygst_api<float>(itype, uplo, n, A, lda, B, ldb, work, lwork, stream);
}

int rl_dlaswp(int64_t m, int64_t ncols, double *A, int64_t lda, int64_t k1, int64_t k2, const int32_t *ipiv,
              rl_stream_t stream)
{
    if (m < 0) return -1;
    if (ncols < 0) return -2;
    if (m > 0 && ncols > 0 && A == nullptr) return -3;
    if (lda < imax1(m)) return -4;
    if (k1 < 1) return -5;
    if (k2 > m) return -6;
    if (ncols == 0 || k2 < k1) return RL_SUCCESS;
    if (ipiv == nullptr) return RL_ERR_NULL_POINTER;
    Ctx c = make_ctx(stream, nullptr, nullptr, 0);
    laswp<double>(c, A, lda, m, 0, ncols, k1 - 1, k2, ipiv);
    return finish(c);
}

size_t rl_trs_work_size(int64_t n, int64_t nrhs)
{
    if (n <= 0 || nrhs <= 0 || nrhs > FLOW_MAX_NRHS) return 0;
    return flow_ws_bytes(n, nrhs);
}

int rl_dgetrs(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv,
              double *B, int64_t ldb, void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_n(trans) && !is_t(trans)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < imax1(n)) return -5;
    if (ldb < imax1(n)) return -8;
    return trs_t<double>(true, n, nrhs, A, lda, ipiv, B, ldb, work, lwork, stream, false, is_t(trans));
}

int rl_dpotrs(char uplo, int64_t n, int64_t nrhs, const double *A, int64_t lda, double *B, int64_t ldb,
              void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < imax1(n)) return -5;
    if (ldb < imax1(n)) return -7;
    return trs_t<double>(false, n, nrhs, A, lda, nullptr, B, ldb, work, lwork, stream, is_u(uplo));
}

int rl_sgetrs(char trans, int64_t n, int64_t nrhs, const float *A, int64_t lda, const int32_t *ipiv,
              float *B, int64_t ldb, void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_n(trans) && !is_t(trans)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < imax1(n)) return -5;
    if (ldb < imax1(n)) return -8;
    return trs_t<float>(true, n, nrhs, A, lda, ipiv, B, ldb, work, lwork, stream, false, is_t(trans));
}

int rl_spotrs(char uplo, int64_t n, int64_t nrhs, const float *A, int64_t lda, float *B, int64_t ldb,
              void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < imax1(n)) return -5;
    if (ldb < imax1(n)) return -7;
    return trs_t<float>(false, n, nrhs, A, lda, nullptr, B, ldb, work, lwork, stream, is_u(uplo));
}

int rl_zgetrs(char trans, int64_t n, int64_t nrhs, const rl_double_complex *A, int64_t lda, const int32_t *ipiv,
              rl_double_complex *B, int64_t ldb, void *work, size_t lwork, rl_stream_t stream)
{
    if (trans != 'N' && trans != 'n' && trans != 'T' && trans != 't' && trans != 'C' && trans != 'c') return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (ldb < (n > 1 ? n : 1)) return -8;
    if (trans != 'N' && trans != 'n') return RL_ERR_UNSUPPORTED;
    return trs_t<cplx>(true, n, nrhs, reinterpret_cast<const cplx *>(A), lda, ipiv, reinterpret_cast<cplx *>(B),
                       ldb, work, lwork, stream);
}

int rl_zpotrs(char uplo, int64_t n, int64_t nrhs, const rl_double_complex *A, int64_t lda, rl_double_complex *B,
              int64_t ldb, void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (ldb < (n > 1 ? n : 1)) return -7;
    return trs_t<cplx>(false, n, nrhs, reinterpret_cast<const cplx *>(A), lda, nullptr, reinterpret_cast<cplx *>(B),
                       ldb, work, lwork, stream, is_u(uplo));
}

// ---- precision form ------------------------------------------------------------

// a precision, optionally with the GMRES refinement flag
static bool prec_ok(int prec)
{
    if ((prec & ~(RL_PREC_MASK | RL_REFINE_GMRES | RL_REFINE_OZRES)) != 0) return false;
    const int p = prec & RL_PREC_MASK;
    return p == RL_PREC_FP32 || tc_prec(p);
}

// largest nrhs of each refinement
static int64_t mixed_max_nrhs(int prec) { return (prec & RL_REFINE_GMRES) ? 64 : 512; }

size_t rl_dsgesv_work_size(int64_t n, int64_t nrhs, int prec)
{
    if (n < 0 || nrhs < 0 || !prec_ok(prec)) return 0;
    return mixed_work_size(n, nrhs, true, prec);
}

size_t rl_dsposv_work_size(int64_t n, int64_t nrhs, int prec)
{
    if (n < 0 || nrhs < 0 || !prec_ok(prec)) return 0;
    return mixed_work_size(n, nrhs, false, prec);
}

int rl_dsgesv(int64_t n, int64_t nrhs, double *A, int64_t lda, int32_t *ipiv, const double *B,
              int64_t ldb, double *X, int64_t ldx, int prec, double tol, int maxiter, int32_t *iter,
              int32_t *info, void *work, size_t lwork, rl_stream_t stream)
{
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (lda < imax1(n)) return -4;
    if (ldb < imax1(n)) return -7;
    if (ldx < imax1(n)) return -9;
    if (!prec_ok(prec)) return RL_ERR_UNSUPPORTED;
    if (nrhs > mixed_max_nrhs(prec)) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || iter == nullptr || (ipiv == nullptr && n > 0)) return RL_ERR_NULL_POINTER;
    if (n > 0 && nrhs > 0 && (work == nullptr || lwork < rl_dsgesv_work_size(n, nrhs, prec)))
        return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, work, lwork);
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    note(c, cudaMemsetAsync(iter, 0, sizeof(int32_t), c.s));
    if (n == 0 || nrhs == 0) return finish(c);
    mixed_solve(c, true, n, nrhs, A, lda, ipiv, B, ldb, X, ldx, prec, tol, maxiter, iter);
    return finish(c);
}

int rl_dsposv(char uplo, int64_t n, int64_t nrhs, double *A, int64_t lda, const double *B,
              int64_t ldb, double *X, int64_t ldx, int prec, double tol, int maxiter, int32_t *iter,
              int32_t *info, void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < imax1(n)) return -5;
    if (ldb < imax1(n)) return -7;
    if (ldx < imax1(n)) return -9;
    if (!prec_ok(prec)) return RL_ERR_UNSUPPORTED;
    if (nrhs > mixed_max_nrhs(prec)) return RL_ERR_UNSUPPORTED;
    if (info == nullptr || iter == nullptr) return RL_ERR_NULL_POINTER;
    if (n > 0 && nrhs > 0 && (work == nullptr || lwork < rl_dsposv_work_size(n, nrhs, prec)))
        return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, info, work, lwork);
    note(c, cudaMemsetAsync(info, 0, sizeof(int32_t), c.s));
    note(c, cudaMemsetAsync(iter, 0, sizeof(int32_t), c.s));
    if (n == 0 || nrhs == 0) return finish(c);
    const bool up = is_u(uplo);
    if (up) uplo_swap<double>(c, n, A, lda);
    mixed_solve(c, false, n, nrhs, A, lda, nullptr, B, ldb, X, ldx, prec, tol, maxiter, iter);
    if (up) uplo_swap<double>(c, n, A, lda);
    return finish(c);
}

// ---- batching form --------------------------------------------------------------

size_t rl_potrf_vbatched_work_size(int64_t batch) { return batch < 0 ? 0 : batched_work_size(batch); }
size_t rl_getrf_vbatched_work_size(int64_t batch) { return batch < 0 ? 0 : batched_work_size(batch); }

}  // extern "C"

template <typename T>
static int potrf_vb(char uplo, int64_t batch, const int32_t *n, T *const *A, const int32_t *lda,
                    int32_t *info, int32_t max_n, void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (batch < 0) return -2;
    if (max_n > BATCH_MAX_N || batch > INT32_MAX) return RL_ERR_UNSUPPORTED;
    if (batch == 0) return RL_SUCCESS;
    if (n == nullptr || A == nullptr || lda == nullptr || info == nullptr) return RL_ERR_NULL_POINTER;
    if (work == nullptr || lwork < batched_work_size(batch)) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, work, lwork);
    const bool up = is_u(uplo);
    if (up) uplo_swap_vbatched<T>(c, batch, n, A, lda, max_n);
    batched_factor<T>(c, false, batch, n, A, lda, nullptr, info, g_params.batch_cfg[sizeof(T) == 8 ? 0 : 1][0],
                      g_params.batch_ctas);
    if (up) uplo_swap_vbatched<T>(c, batch, n, A, lda, max_n);
    return finish(c);
}

template <typename T>
static int getrf_vb(int64_t batch, const int32_t *n, T *const *A, const int32_t *lda, int32_t *const *ipiv,
                    int32_t *info, int32_t max_n, void *work, size_t lwork, rl_stream_t stream)
{
    if (batch < 0) return -1;
    if (max_n > BATCH_MAX_N || batch > INT32_MAX) return RL_ERR_UNSUPPORTED;
    if (batch == 0) return RL_SUCCESS;
    if (n == nullptr || A == nullptr || lda == nullptr || ipiv == nullptr || info == nullptr)
        return RL_ERR_NULL_POINTER;
    if (work == nullptr || lwork < batched_work_size(batch)) return RL_ERR_WORKSPACE;
    Ctx c = make_ctx(stream, nullptr, work, lwork);
    batched_factor<T>(c, true, batch, n, A, lda, ipiv, info, g_params.batch_cfg[sizeof(T) == 8 ? 0 : 1][1],
                      g_params.batch_ctas);
    return finish(c);
}

// ---- autotuner of the batched form -------------------------------------------
// Times every candidate configuration (block width, CTA size, CTAs per SM) on
// the caller's own batch, restoring the matrices from a packed copy before
// each run and once more at the end, and keeps the fastest for later calls
// of the same routine and element type.

template <typename T>
__global__ void k_batch_copy(int batch, const int32_t *d_n, T *const *src, const int32_t *src_ld,
                             T *const *dst, const int32_t *dst_ld)
{
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        const int n = d_n[b];
        if (n <= 0) continue;
        const T *s = src[b];
        T *d = dst[b];
        const int ls = src_ld[b], ld = dst_ld[b];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e % n, j = e / n;
            d[(i64)j * ld + i] = s[(i64)j * ls + i];
        }
    }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
static int vb_tune(bool lu, int64_t batch, const int32_t *n, T *const *A, const int32_t *lda,
                   int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work, size_t lwork,
                   int32_t *best, float *ms_out, rl_stream_t stream)
{
    if (batch < 0) return -3;
    if (max_n > BATCH_MAX_N || batch > INT32_MAX) return RL_ERR_UNSUPPORTED;
    if (best == nullptr) return RL_ERR_NULL_POINTER;
    if (batch == 0) { *best = g_params.batch_cfg[sizeof(T) == 8 ? 0 : 1][lu ? 1 : 0]; return RL_SUCCESS; }
    if (n == nullptr || A == nullptr || lda == nullptr || info == nullptr || (lu && ipiv == nullptr))
        return RL_ERR_NULL_POINTER;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // sizes on the host (this call synchronizes)
    std::vector<int32_t> hn((size_t)batch);
    if (cudaMemcpyAsync(hn.data(), n, sizeof(int32_t) * batch, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RL_ERR_CUDA;
    size_t elems = 0;
    for (int32_t v : hn) elems += (size_t)(v > 0 ? v : 0) * (size_t)(v > 0 ? v : 0);
    const size_t wsb = al256(batched_work_size(batch)), pb = al256(sizeof(T *) * batch),
                 lb = al256(sizeof(int32_t) * batch);
    if (work == nullptr || lwork < wsb + pb + lb + elems * sizeof(T)) return RL_ERR_WORKSPACE;
    char *w = static_cast<char *>(work);
    T **bptr = reinterpret_cast<T **>(w + wsb);
    int32_t *bld = reinterpret_cast<int32_t *>(w + wsb + pb);
    T *bdata = reinterpret_cast<T *>(w + wsb + pb + lb);
    std::vector<T *> hp((size_t)batch);
    size_t off = 0;
    for (int64_t b = 0; b < batch; ++b) {
        hp[b] = bdata + off;
        off += (size_t)(hn[b] > 0 ? hn[b] : 0) * (size_t)(hn[b] > 0 ? hn[b] : 0);
    }
    if (cudaMemcpyAsync(bptr, hp.data(), sizeof(T *) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(bld, n, sizeof(int32_t) * batch, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return RL_ERR_CUDA;
    const unsigned cgrid = (unsigned)(batch < 4096 ? batch : 4096);
    k_batch_copy<T><<<cgrid, 256, 0, s>>>((int)batch, n, A, lda, bptr, bld);       // save
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RL_ERR_CUDA;
    const int ti = sizeof(T) == 8 ? 0 : 1;
    int bestc = -1;
    float bestms = 0.0f;
    int rc = RL_SUCCESS;
    for (int cfg = 0; cfg < BATCH_NCFG && rc == RL_SUCCESS; ++cfg) {
        float mn = -1.0f;
        for (int rep = 0; rep < 2; ++rep) {
            k_batch_copy<T><<<cgrid, 256, 0, s>>>((int)batch, n, bptr, bld, A, lda);   // restore
            Ctx c = make_ctx(stream, nullptr, work, wsb);
            note(c, cudaEventRecord(e0, s));
            batched_factor<T>(c, lu, batch, n, A, lda, ipiv, info, cfg, 0);
            note(c, cudaEventRecord(e1, s));
            float ms = 0.0f;
            if (c.err != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = RL_ERR_CUDA;
                break;
            }
            if (mn < 0.0f || ms < mn) mn = ms;
        }
        if (ms_out) ms_out[cfg] = mn;
        if (rc == RL_SUCCESS && (bestc < 0 || mn < bestms)) { bestc = cfg; bestms = mn; }
    }
    k_batch_copy<T><<<cgrid, 256, 0, s>>>((int)batch, n, bptr, bld, A, lda);       // the caller's data back
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = RL_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RL_SUCCESS) return rc;
    g_params.batch_cfg[ti][lu ? 1 : 0] = bestc;
    *best = bestc;
    return RL_SUCCESS;
}

extern "C" {

size_t rl_vbatched_tune_work_size(int64_t batch, int64_t sum_n2, int elem_bytes)
{
    if (batch < 0 || sum_n2 < 0 || (elem_bytes != 4 && elem_bytes != 8)) return 0;
    return al256(batched_work_size(batch)) + al256(sizeof(void *) * batch) + al256(sizeof(int32_t) * batch) +
           (size_t)sum_n2 * (size_t)elem_bytes;
}

int rl_vbatched_tune(char routine, int elem_bytes, int64_t batch, const int32_t *n, void *const *A,
                     const int32_t *lda, int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work,
                     size_t lwork, int32_t *best, float *ms_per_config, rl_stream_t stream)
{
    const bool lu = (routine == 'G' || routine == 'g');
    if (!lu && routine != 'P' && routine != 'p') return -1;
    if (elem_bytes == 8)
        return vb_tune<double>(lu, batch, n, reinterpret_cast<double *const *>(A), lda, ipiv, info, max_n, work,
                               lwork, best, ms_per_config, stream);
    if (elem_bytes == 4)
        return vb_tune<float>(lu, batch, n, reinterpret_cast<float *const *>(A), lda, ipiv, info, max_n, work,
                              lwork, best, ms_per_config, stream);
    return -2;
}

int rl_vbatched_set_config(char routine, int elem_bytes, int32_t cfg)
{
    const bool lu = (routine == 'G' || routine == 'g');
    if (!lu && routine != 'P' && routine != 'p') return -1;
    if (elem_bytes != 4 && elem_bytes != 8) return -2;
    if (cfg < 0 || cfg >= BATCH_NCFG) return -3;
    g_params.batch_cfg[elem_bytes == 8 ? 0 : 1][lu ? 1 : 0] = cfg;
    return RL_SUCCESS;
}

int rl_vbatched_config(char routine, int elem_bytes, int32_t *cfg, int32_t *nb, int32_t *threads,
                       int32_t *per_sm)
{
    const bool lu = (routine == 'G' || routine == 'g');
    if (!lu && routine != 'P' && routine != 'p') return -1;
    if (elem_bytes != 4 && elem_bytes != 8) return -2;
    const int c = g_params.batch_cfg[elem_bytes == 8 ? 0 : 1][lu ? 1 : 0];
    if (cfg) *cfg = c;
    if (nb) *nb = kBatchCfgs[c].nb;
    if (threads) *threads = kBatchCfgs[c].threads;
    if (per_sm) *per_sm = kBatchCfgs[c].per_sm;
    return RL_SUCCESS;
}

}  // extern "C"

extern "C" {

int rl_dpotrf_vbatched(char uplo, int64_t batch, const int32_t *n, double *const *A, const int32_t *lda,
                       int32_t *info, int32_t max_n, void *work, size_t lwork, rl_stream_t stream)
{
    return potrf_vb<double>(uplo, batch, n, A, lda, info, max_n, work, lwork, stream);
}

int rl_spotrf_vbatched(char uplo, int64_t batch, const int32_t *n, float *const *A, const int32_t *lda,
                       int32_t *info, int32_t max_n, void *work, size_t lwork, rl_stream_t stream)
{
    return potrf_vb<float>(uplo, batch, n, A, lda, info, max_n, work, lwork, stream);
}

int rl_dgetrf_vbatched(int64_t batch, const int32_t *n, double *const *A, const int32_t *lda,
                       int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work, size_t lwork,
                       rl_stream_t stream)
{
    return getrf_vb<double>(batch, n, A, lda, ipiv, info, max_n, work, lwork, stream);
}

int rl_sgetrf_vbatched(int64_t batch, const int32_t *n, float *const *A, const int32_t *lda,
                       int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work, size_t lwork,
                       rl_stream_t stream)
{
    return getrf_vb<float>(batch, n, A, lda, ipiv, info, max_n, work, lwork, stream);
}

// ---- host-buffer forms -------------------------------------------------------

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t rl_host_work_size(const char *routine, int64_t m, int64_t n, int64_t lda)
{
    if (routine == nullptr || m < 0 || n < 0 || lda < 1) return 0;
    const size_t mat = align256((size_t)lda * (size_t)(n > 0 ? n : 1) * sizeof(double));
    if (std::strcmp(routine, "dpotrf") == 0) return mat + 256;
    if (std::strcmp(routine, "dgetrf") == 0)
        return mat + 256 + align256((size_t)(m < n ? m : n) * sizeof(int32_t) + 4) +
               align256(rl_dgetrf_work_size(m, n));
    return 0;
}

// Host-buffer calls.  Above the order where the recursion splits, the
// columns right of the top-level split are copied in on a copy stream while
// the left part is factored (the top level waits for them before it first
// touches them); the Cholesky's left columns, final after the top-level
// TRSM, are copied back on the copy stream while the rest is factored.
struct HostCopy {
    cudaStream_t cs = nullptr;
    cudaEvent_t entry = nullptr, trail = nullptr, left = nullptr, left_back = nullptr;
    bool ok = false;
    HostCopy(bool wanted, bool want_left)
    {
        if (!wanted) return;
        cs = copy_stream();
        if (!cs) return;
        if (cudaEventCreateWithFlags(&entry, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&trail, cudaEventDisableTiming) != cudaSuccess)
            return;
        if (want_left && (cudaEventCreateWithFlags(&left, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&left_back, cudaEventDisableTiming) != cudaSuccess))
            return;
        ok = true;
    }
    // An error after the first copy was queued: wait for everything already
    // queued on the caller's stream and the copy stream (their status is
    // not looked at) so that no copy from or to the caller's host buffer is
    // still running when the error is returned.
    int fail(cudaStream_t s, int st)
    {
        (void)cudaStreamSynchronize(s);
        if (cs) (void)cudaStreamSynchronize(cs);
        return st;
    }
    ~HostCopy()
    {
        for (cudaEvent_t e : {entry, trail, left, left_back})
            if (e) (void)cudaEventDestroy(e);
    }
};

static constexpr int64_t HOST_SPLIT_MIN = 512;

int rl_dpotrf_host(char uplo, int64_t n, double *A_host, int64_t lda, int32_t *info_host,
                   void *work, size_t lwork, rl_stream_t stream)
{
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (n < 0) return -2;
    if (n > 0 && A_host == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (info_host == nullptr) return RL_ERR_NULL_POINTER;
    if (work == nullptr || lwork < rl_host_work_size("dpotrf", n, n, lda)) return RL_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)lda * (size_t)n * sizeof(double);
    char *w = static_cast<char *>(work);
    double *dA = reinterpret_cast<double *>(w);
    int32_t *dinfo = reinterpret_cast<int32_t *>(w + align256(bytes > 0 ? bytes : 8));
    const bool split = is_l(uplo) && n >= HOST_SPLIT_MIN && n > g_params.potrf_c;
    HostCopy hc(split, true);
    if (!split || !hc.ok) {
        if (bytes && cudaMemcpyAsync(dA, A_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
        int st = rl_dpotrf(uplo, n, dA, lda, dinfo, nullptr, 0, stream);
        if (st != RL_SUCCESS) return hc.fail(s, st);
        if (bytes && cudaMemcpyAsync(A_host, dA, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    } else {
        const i64 n1 = split_q(n, TRX_NB);                      // the recursion's top-level split
        const size_t lb = (size_t)lda * (size_t)n1 * sizeof(double), rb = bytes - lb;
        Ctx c = make_ctx(stream, dinfo, nullptr, 0);
        c.abort = dinfo;
        c.trail_ready = hc.trail;
        c.left_done = hc.left;
        note(c, cudaEventRecord(hc.entry, s));                   // after the caller's earlier work on s
        note(c, cudaStreamWaitEvent(hc.cs, hc.entry, 0));
        note(c, cudaMemcpyAsync(dA, A_host, lb, cudaMemcpyHostToDevice, s));
        note(c, cudaMemcpyAsync(dA + (size_t)lda * n1, A_host + (size_t)lda * n1, rb, cudaMemcpyHostToDevice, hc.cs));
        note(c, cudaEventRecord(hc.trail, hc.cs));
        note(c, cudaMemsetAsync(dinfo, 0, sizeof(int32_t), s));
        potrf_rec(c, n, dA, lda, 0);
        note(c, cudaStreamWaitEvent(hc.cs, hc.left, 0));
        note(c, cudaMemcpyAsync(A_host, dA, lb, cudaMemcpyDeviceToHost, hc.cs));
        note(c, cudaEventRecord(hc.left_back, hc.cs));
        note(c, cudaMemcpyAsync(A_host + (size_t)lda * n1, dA + (size_t)lda * n1, rb, cudaMemcpyDeviceToHost, s));
        note(c, cudaStreamWaitEvent(s, hc.left_back, 0));
        if (c.err != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    }
    if (cudaMemcpyAsync(info_host, dinfo, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    return cudaStreamSynchronize(s) == cudaSuccess ? RL_SUCCESS : hc.fail(s, RL_ERR_CUDA);
}

int rl_dgetrf_host(int64_t m, int64_t n, double *A_host, int64_t lda, int32_t *ipiv_host,
                   int32_t *info_host, void *work, size_t lwork, rl_stream_t stream)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m > 0 && n > 0 && A_host == nullptr) return -3;
    if (lda < (m > 1 ? m : 1)) return -4;
    if (info_host == nullptr || (ipiv_host == nullptr && m > 0 && n > 0)) return RL_ERR_NULL_POINTER;
    if (work == nullptr || lwork < rl_host_work_size("dgetrf", m, n, lda)) return RL_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)lda * (size_t)n * sizeof(double);
    const size_t mn = (size_t)(m < n ? m : n);
    char *w = static_cast<char *>(work);
    double *dA = reinterpret_cast<double *>(w);
    char *p = w + align256(bytes > 0 ? bytes : 8);
    int32_t *dinfo = reinterpret_cast<int32_t *>(p);
    p += 256;
    int32_t *dipiv = reinterpret_cast<int32_t *>(p);
    p += align256(mn * sizeof(int32_t) + 4);
    void *ws = p;
    const size_t wsz = rl_dgetrf_work_size(m, n);
    // the recursion's top-level left part: the leading m x m block of a wide
    // matrix, else the first split of the columns
    const i64 nb = g_params.getrf_nb;
    const i64 n1 = (n <= nb || m <= 0) ? 0 : (m < n ? m : split_q(n, n > 2 * TRX_NB ? TRX_NB : nb));
    const bool split = n >= HOST_SPLIT_MIN && n1 > 0 && n1 < n && m <= INT32_MAX - 1;
    HostCopy hc(split, false);
    if (!split || !hc.ok || wsz == 0) {
        if (bytes && cudaMemcpyAsync(dA, A_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
        int st = rl_dgetrf(m, n, dA, lda, dipiv, dinfo, ws, wsz, stream);
        if (st != RL_SUCCESS) return hc.fail(s, st);
    } else {
        const size_t lb = (size_t)lda * (size_t)n1 * sizeof(double), rb = bytes - lb;
        Ctx c = make_ctx(stream, dinfo, ws, wsz);
        c.abort = nullptr;
        c.trail_ready = hc.trail;
        note(c, cudaEventRecord(hc.entry, s));
        note(c, cudaStreamWaitEvent(hc.cs, hc.entry, 0));
        note(c, cudaMemcpyAsync(dA, A_host, lb, cudaMemcpyHostToDevice, s));
        note(c, cudaMemcpyAsync(dA + (size_t)lda * n1, A_host + (size_t)lda * n1, rb, cudaMemcpyHostToDevice, hc.cs));
        note(c, cudaEventRecord(hc.trail, hc.cs));
        note(c, cudaMemsetAsync(dinfo, 0, sizeof(int32_t), s));
        getrf_rec(c, dA, lda, m, dipiv, 0, m, n);
        // the recursion always reaches its top-level wait; this one keeps s
        // ordered after the copy even if it did not
        note(c, cudaStreamWaitEvent(s, hc.trail, 0));
        if (c.err != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    }
    if (bytes && cudaMemcpyAsync(A_host, dA, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    if (mn && cudaMemcpyAsync(ipiv_host, dipiv, mn * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return hc.fail(s, RL_ERR_CUDA);
    if (cudaMemcpyAsync(info_host, dinfo, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return hc.fail(s, RL_ERR_CUDA);
    return cudaStreamSynchronize(s) == cudaSuccess ? RL_SUCCESS : hc.fail(s, RL_ERR_CUDA);
}

// ---- parameters, accounting, status ------------------------------------------

int rl_set_param(int key, int64_t value)
{
    switch (key) {
    case RL_PARAM_POTRF_CROSSOVER:
        if (value < 1 || value > 64) return RL_ERR_PARAM;
        g_params.potrf_c = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_GETRF_PANEL:
        if (value < 1 || value > 64) return RL_ERR_PARAM;
        g_params.getrf_nb = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_TRTRI_CROSSOVER:
        if (value < 1 || value > 64) return RL_ERR_PARAM;
        g_params.trtri_c = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_SPIN_LIMIT_NS:
        if (value < 0) return RL_ERR_PARAM;
        g_params.spin_ns = (long long)value;
        return RL_SUCCESS;
    case RL_PARAM_BATCH_CTAS:
        if (value < 0 || value > 8) return RL_ERR_PARAM;
        g_params.batch_ctas = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_TRI_LANES:
        if (value != 0 && value != 2 && value != 4) return RL_ERR_PARAM;
        g_params.tri_lanes = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_LOOKAHEAD:
        if (value != 0 && value != 1) return RL_ERR_PARAM;
        g_params.lookahead = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_NVTX:
        if (value != 0 && value != 1) return RL_ERR_PARAM;
        g_params.nvtx = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_OZ_MIN:
        if (value < 1 || value > (1 << 20)) return RL_ERR_PARAM;
        g_params.oz_min = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_GMRES_RESTART:
        if (value < 1 || value > 64) return RL_ERR_PARAM;
        g_params.gmres_m = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_PANEL_CLUSTER:
        if (value != 0 && value != 1) return RL_ERR_PARAM;
        g_params.panel_cluster = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_TC_PAIRS:
        if (value != 0 && value != 1) return RL_ERR_PARAM;
        g_params.tc_pairs = (int)value;
        return RL_SUCCESS;
    case RL_PARAM_PANEL_CTAS:
        // low 16 bits: FP64 panels, high 16 bits: FP32 panels (0 = one per SM)
        if (value < 0 || (value & 0xffff) > 256 || (value >> 16) > 256) return RL_ERR_PARAM;
        g_params.panel_ctas64 = (int)(value & 0xffff);
        g_params.panel_ctas32 = (int)(value >> 16);
        return RL_SUCCESS;
    default:
        return RL_ERR_PARAM;
    }
}

int64_t rl_get_param(int key)
{
    switch (key) {
    case RL_PARAM_POTRF_CROSSOVER: return g_params.potrf_c;
    case RL_PARAM_GETRF_PANEL: return g_params.getrf_nb;
    case RL_PARAM_TRTRI_CROSSOVER: return g_params.trtri_c;
    case RL_PARAM_SPIN_LIMIT_NS: return g_params.spin_ns;
    case RL_PARAM_BATCH_CTAS: return g_params.batch_ctas;
    case RL_PARAM_TRI_LANES: return g_params.tri_lanes;
    case RL_PARAM_LOOKAHEAD: return g_params.lookahead;
    case RL_PARAM_OZ_MIN: return g_params.oz_min;
    case RL_PARAM_NVTX: return g_params.nvtx;
    case RL_PARAM_GMRES_RESTART: return g_params.gmres_m;
    case RL_PARAM_PANEL_CLUSTER: return g_params.panel_cluster;
    case RL_PARAM_TC_PAIRS: return g_params.tc_pairs;
    case RL_PARAM_PANEL_CTAS: return (int64_t)g_params.panel_ctas64 | ((int64_t)g_params.panel_ctas32 << 16);
    default: return -1;
    }
}

uint64_t rl_launch_count(void) { return g_launches.load(); }

int rl_clear_cache(void)
{
    cudaError_t first = cudaSuccess;
    auto keep = [&](cudaError_t e) { if (first == cudaSuccess && e != cudaSuccess) first = e; };
    int cur = 0;
    keep(cudaGetDevice(&cur));
    {
        std::lock_guard<std::mutex> lock(g_side_mu);
        for (int dev = 0; dev < 128; ++dev) {
            LaEvents &e = t_ev[dev];
            if (g_side[dev] == nullptr && !e.ready && g_copy[dev] == nullptr) continue;
            keep(cudaSetDevice(dev));
            if (g_copy[dev] != nullptr) {
                keep(cudaStreamSynchronize(g_copy[dev]));
                keep(cudaStreamDestroy(g_copy[dev]));
                g_copy[dev] = nullptr;
            }
            if (g_side[dev] != nullptr) {
                keep(cudaStreamSynchronize(g_side[dev]));
                keep(cudaStreamDestroy(g_side[dev]));
                g_side[dev] = nullptr;
            }
            if (e.ready) {
                for (int i = 0; i < LA_DEPTH; ++i) {
                    keep(cudaEventDestroy(e.start[i]));
                    keep(cudaEventDestroy(e.done[i]));
                    e.start[i] = e.done[i] = nullptr;
                }
                e.ready = false;
            }
        }
    }
    keep(cudaSetDevice(cur));
    keep(trace_release());
    return first == cudaSuccess ? RL_SUCCESS : RL_ERR_CUDA;
}

const char *rl_status_string(int status)
{
    if (status < 0) return "illegal argument (LAPACK numbering: argument -status)";
    switch (status) {
    case RL_SUCCESS: return "success";
    case RL_ERR_CUDA: return "CUDA runtime or launch error";
    case RL_ERR_WORKSPACE: return "workspace missing or smaller than the size query";
    case RL_ERR_UNSUPPORTED: return "unsupported option or size";
    case RL_ERR_NULL_POINTER: return "info or ipiv pointer is NULL";
    case RL_ERR_PARAM: return "unknown parameter key or value out of range";
    default: return "unknown status";
    }
}

}  // extern "C"

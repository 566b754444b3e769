// Internal declarations shared by the CUDA translation units of librelgpu.
// Column-major storage with leading dimensions throughout; all sizes int64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>

#include "../../include/relgpu.h"

namespace rl {

using i64 = int64_t;
using ::fma;   // the real overloads stay visible beside the complex one below

// Complex double, interleaved (re, im) as LAPACK's complex*16.  The
// arithmetic is written out: a * b with 4 FMAs' worth of products, division
// by Smith's method (R. L. Smith, "Algorithm 116: Complex division", CACM
// 1962), and |Re| + |Im| as LAPACK's izamax measures a pivot.
struct __align__(16) cplx {
    double x, y;
    __host__ __device__ constexpr cplx() : x(0.0), y(0.0) {}
    __host__ __device__ constexpr cplx(double r) : x(r), y(0.0) {}
    __host__ __device__ constexpr cplx(double r, double i) : x(r), y(i) {}
};
__host__ __device__ inline cplx operator+(cplx a, cplx b) { return cplx(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx operator-(cplx a, cplx b) { return cplx(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx operator-(cplx a) { return cplx(-a.x, -a.y); }
__host__ __device__ inline cplx operator*(cplx a, cplx b)
{
    return cplx(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ inline cplx operator/(cplx a, cplx b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + b.y * r;
        return cplx((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    const double r = b.x / b.y, d = b.x * r + b.y;
    return cplx((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__host__ __device__ inline bool operator==(cplx a, cplx b) { return a.x == b.x && a.y == b.y; }
__host__ __device__ inline bool operator!=(cplx a, cplx b) { return !(a == b); }
// c + a b
__host__ __device__ inline cplx fma(cplx a, cplx b, cplx c)
{
    return cplx(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ inline cplx conj(cplx a) { return cplx(a.x, -a.y); }
__host__ __device__ inline double abs1(cplx a) { return fabs(a.x) + fabs(a.y); }
// conjugate when the element type is complex (the "transpose" of the complex
// routines is the conjugate transpose)
template <typename T> __host__ __device__ inline T cj(T v) { return v; }
template <> __host__ __device__ inline cplx cj<cplx>(cplx v) { return conj(v); }
#ifdef __CUDACC__
using ::__shfl_sync;   // the built-in overloads stay visible beside this one
__device__ inline cplx __shfl_sync(unsigned mask, cplx v, int src)
{
    return cplx(::__shfl_sync(mask, v.x, src), ::__shfl_sync(mask, v.y, src));
}
#endif
template <typename T> struct is_cplx { static constexpr bool value = false; };
template <> struct is_cplx<cplx> { static constexpr bool value = true; };

// Kernel-launch accounting (host side).
extern std::atomic<uint64_t> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Process-wide tunables (see rl_set_param).
struct Params {
    int potrf_c = 64;        // dpotrf crossover (base-case order)
    int getrf_nb = 32;       // dgetrf panel width
    int trtri_c = 64;        // dtrtri / dlauum crossover
    long long spin_ns = 2000000000LL;
    int batch_ctas = 0;      // CTAs per SM of the batched kernels (0 = occupancy limit)
    int batch_cfg[2][2] = {{0, 0}, {0, 0}};   // [double/float][potrf/getrf]: tuned kBatchCfgs index
    int tri_lanes = 0;       // lanes per vector of the triangle leaf kernels (0 = by size, 2, 4)
    int lookahead = 1;       // LU/Cholesky: trailing update split across the side stream (0 = off)
    int panel_ctas64 = 0;    // LU panel CTAs, FP64 / FP32 (0 = one per SM)
    int panel_ctas32 = 0;
    int oz_min = 128;        // smallest m, n and k that the FP64 emulation takes
    int nvtx = 0;            // 1: an NVTX range per recursion node (routine, order, depth)
    int gmres_m = 50;        // restart length of the GMRES refinement
    int panel_cluster = 1;   // LU panels that fit a cluster's shared memory take the cluster kernel
    int tc_pairs = 1;        // tensor-core GEMM: row-tile pairs on 2-CTA clusters sharing B
};
extern Params g_params;

// Per-call context: stream, device info/abort word, workspace, device facts.
struct Ctx {
    cudaStream_t s = nullptr;
    int32_t *info = nullptr;     // device; nonzero => later kernels skip (abort)
    const int32_t *abort = nullptr;  // where kernels look for an abort signal
    void *work = nullptr;
    size_t lwork = 0;
    int num_sms = 0;
    cudaError_t err = cudaSuccess;   // first launch error seen
    // FP32 GEMMs of the precision form: operand precision and the packing
    // workspace of the tensor-core path (RL_PREC_FP32 = SIMT FP32)
    int prec = RL_PREC_FP32;
    void *tcwork = nullptr;
    size_t tclwork = 0;
    // FP64 GEMMs emulated on the BF16 tensor cores (oz_gemm.cu): digit
    // planes (0 = native FP64) and the slicing workspace
    int oz_slices = 0;
    void *ozwork = nullptr;
    size_t ozlwork = 0;
    // a second slicing workspace for the lookahead's side stream (the two
    // streams' emulated GEMMs then run at once), and one CTA per tile instead
    // of one per SM, so that the other stream's kernels find SMs as tiles end
    void *ozwork2 = nullptr;
    size_t ozlwork2 = 0;
    bool oz_dynamic = false;
    // host-buffer calls: the columns right of the top-level split arrive on
    // a copy stream (trail_ready: waited on before the top level first
    // touches them); left_done is recorded once the columns left of the
    // split hold their final values (Cholesky: after the top-level TRSM)
    cudaEvent_t trail_ready = nullptr;
    cudaEvent_t left_done = nullptr;
};

int device_sms();
void note(Ctx &c, cudaError_t e);
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the device, so it is set once per
// (device, kernel) and again only if a larger size is asked for; safe to
// call from several host threads.
cudaError_t smem_optin(const void *func, int bytes);
template <typename F>
inline cudaError_t smem_optin(F *func, size_t bytes)
{
    return smem_optin(reinterpret_cast<const void *>(func), (int)bytes);
}

// ---- per-kernel tracing (trace.cu) -----------------------------------------
// Kernel kinds, in the order rl_trace_read reports them.
enum Kind {
    K_GEMM = 0, K_SYRK, K_TRSM, K_TRMM, K_POTF2, K_TRTI2, K_LAUU2, K_DIAG,
    K_PANEL, K_LASWP, K_RESID, K_CONVERT, K_MIX, K_BATCH, K_FLOW, K_TRANS, K_COUNT
};
extern std::atomic<int> g_trace_on;
cudaError_t trace_release();
// Bracket one kernel launch: with tracing on, CUDA events are recorded on the
// launch stream around it and the launch's algorithmic flops and bytes are
// attributed to its kind.  The destructor counts the launch and records the
// launch error, if any.
struct Launch {
    Ctx &c;
    int kind;
    double flops, bytes;
    void *ev0 = nullptr;
    Launch(Ctx &ctx, int k, double f, double b);
    ~Launch();
};

// Smallest trailing order that the LU/Cholesky recursions split across the
// side stream.
constexpr i64 LA_MIN_N = 512;

// Largest triangle handled by the TRSM/TRMM/base kernels in shared memory.
constexpr int TRX_NB = 64;
// GEMM tile.
constexpr int GEMM_BM = 64, GEMM_BN = 64, GEMM_BK = 16;

// Split rule (Section 3 footnote: halves that are multiples of 8 "where
// possible"); on the GPU the quantum is a tile size q so sub-blocks start on
// tile boundaries: n1 = q * floor((n + q) / (2q)) clamped to [q, n-1].
inline i64 split_q(i64 n, i64 q)
{
    if (n <= 1) return 0;
    if (n <= q) return n / 2 > 0 ? n / 2 : 1;
    i64 n1 = q * ((n + q) / (2 * q));
    if (n1 < q) n1 = q;
    if (n1 >= n) n1 = n - 1;
    return n1;
}

// ---- BLAS-3 layer (blas3.cu), T = double or float ---------------------------
// C(m x n) := beta*C + alpha*op(A) op(B); lower=true writes only i >= j of a
// square C (SYRK form, A and B may alias).
template <typename T>
void gemm(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, T alpha, const T *A, i64 lda,
          const T *B, i64 ldb, T beta, T *C, i64 ldc, bool lower = false);

// C(m x n) := beta C + alpha S B (left, S m x m) or alpha B S (right, S n x n),
// S symmetric with its lower triangle stored.
template <typename T>
void symm(Ctx &c, bool left, i64 m, i64 n, T alpha, const T *S, i64 lds, const T *Bm, i64 ldb, T beta,
          T *C, i64 ldc);
// B(m x n) := alpha * L^{-1} B, L lower m x m (unit or not).
template <typename T>
void trsm_lln(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);
// B(m x n) := alpha * B L^{-T}, L lower n x n, non-unit (L^{-H} for complex).
template <typename T>
void trsm_rlt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);
// B(m x n) := alpha * L^{-T} B, L lower m x m, non-unit.
template <typename T>
void trsm_llt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);
// B(m x n) := alpha * U^{-1} B, U upper m x m, non-unit.
template <typename T>
void trsm_lun(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb);
// B := L^{-T} B with a unit (unit = true) or non-unit lower L (complex: L^{-H})
template <typename T>
void trsm_llt_u(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);
// B := U^{-T} B, U upper non-unit
template <typename T>
void trsm_lut(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb);
// Row interchanges ipiv[n-1], ..., ipiv[0] (1-based) applied to the ncols
// columns of B, last first (P^T B for P from getrf).
template <typename T>
void laswp_rev(Ctx &c, T *B, i64 ldb, i64 n, i64 ncols, const int32_t *ipiv);
// B(m x n) := alpha * U B, U upper m x m, non-unit.
template <typename T>
void trmm_lun(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb);
// B(m x n) := alpha * B U^{-1}, U upper n x n, non-unit.
template <typename T>
void trsm_run(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb);
// B(m x n) := alpha * B L, L lower n x n (unit or not).
template <typename T>
void trmm_rln(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);
// B(m x n) := alpha * L^T B, L lower m x m, non-unit.
template <typename T>
void trmm_llt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb);

// ---- base cases and row interchanges (factor.cu) ---------------------------
template <typename T>
void potf2(Ctx &c, i64 n, T *A, i64 lda, i64 info_off);
// upper: invert the upper triangle instead (stored in place)
template <typename T>
void trti2(Ctx &c, bool unit, i64 n, T *A, i64 lda, bool upper = false);
template <typename T>
void lauu2(Ctx &c, i64 n, T *A, i64 lda);
template <typename T>
void diag_zero_scan(Ctx &c, i64 n, const T *A, i64 lda);
// Panel LU of the m x nb block at A (row/col offset r0 in the full matrix);
// writes ipiv[r0 .. r0+min(m,nb)) as global 1-based rows.  c.work holds the
// panel workspace (panel_ws_bytes()).
template <typename T>
void getf2_panel(Ctx &c, i64 m, i64 nb, T *A, i64 lda, int32_t *ipiv, i64 r0);
// Apply ipiv[k1..k2) (global 1-based rows of the matrix at A0, which has
// m rows) to columns [c0, c0 + ncols).
template <typename T>
void laswp(Ctx &c, T *A0, i64 lda, i64 m, i64 c0, i64 ncols, i64 k1, i64 k2, const int32_t *ipiv);

size_t panel_ws_bytes();

// ---- few right-hand sides (flow.cu) -------------------------------------------
// B(n x nrhs) := op(T)^{-1} B in one dataflow launch: FLOW_LN T = L (lower,
// unit or not), FLOW_UN T = U (upper, non-unit), FLOW_LT T = L^T (L stored
// lower, non-unit).  ws: flow_ws_bytes(n, nrhs) of device scratch.  Its
// first word is a status the caller zeroes (a bounded wait that expires sets
// RL_INFO_DEVICE_TIMEOUT there and in c.info when given); the ticket and
// flags after it are zeroed by each call itself (stream-ordered), so one ws
// serves consecutive calls on one stream.
enum { FLOW_LN = 0, FLOW_UN = 1, FLOW_LT = 2 };
constexpr i64 FLOW_MAX_NRHS = 64;
size_t flow_ws_bytes(i64 n, i64 nrhs);
template <typename T>
void trsm_flow(Ctx &c, int form, bool unit, i64 n, i64 nrhs, const T *A, i64 lda, T *B, i64 ldb,
               void *ws);

// ---- tensor-core GEMM for FP32 storage (tc_gemm.cu) ---------------------------
// C(m x n) += alpha op(A) op(B) with operands in precision `prec` (TF32,
// BF16, FP16, 3xTF32) and FP32 accumulation; lower: square C, lower triangle.
// Returns false when it does not apply (then the caller uses the SIMT path).
size_t tc_work_bytes(i64 m, i64 n, i64 k, int prec);
bool tc_gemm(Ctx &c, int prec, bool ta, bool tb, i64 m, i64 n, i64 k, float alpha, const float *A,
             i64 lda, const float *B, i64 ldb, float *C, i64 ldc, bool lower, void *work, size_t lwork);
// Smallest GEMM sent to the tensor cores (smaller ones are latency-bound).
constexpr i64 TC_MIN_MN = 128, TC_MIN_K = 64;

// ---- FP64 GEMM emulated on the BF16 tensor cores (oz_gemm.cu) -------------------
size_t oz_work_bytes(i64 m, i64 n, i64 k, int slices);
size_t oz_planes_bytes(i64 m, i64 k, int slices);
bool oz_prepare(Ctx &c, int slices, bool sym, i64 m, i64 k, const double *A, i64 lda, void *planes);
bool oz_gemm_planes(Ctx &c, int slices, i64 m, i64 n, i64 k, double alpha, const void *planes, const double *B,
                    i64 ldb, double beta, double *C, i64 ldc, void *work, size_t lwork);
bool oz_gemm(Ctx &c, int slices, bool ta, bool tb, i64 m, i64 n, i64 k, double alpha, const double *A, i64 lda,
             const double *B, i64 ldb, double beta, double *C, i64 ldc, bool lower, void *work, size_t lwork);

// ---- batching form (batched.cu) ---------------------------------------------
size_t batched_work_size(i64 batch);
struct BatchCfg { int nb, threads, per_sm; };
constexpr int BATCH_NCFG = 8;
extern const BatchCfg kBatchCfgs[BATCH_NCFG];
// cfg: index into kBatchCfgs; per_sm > 0 overrides its CTAs per SM
template <typename T>
int batched_factor(Ctx &c, bool lu, i64 batch, const int32_t *d_n, T *const *d_A, const int32_t *d_lda,
                   int32_t *const *d_ipiv, int32_t *d_info, int cfg, int per_sm);
constexpr int BATCH_MAX_N = 256;

// ---- recursions (api.cu), T = double or float --------------------------------
template <typename T>
void potrf_rec_t(Ctx &c, i64 n, T *A, i64 lda, i64 off);
template <typename T>
void getrf_rec_t(Ctx &c, T *A0, i64 lda, i64 m_tot, int32_t *ipiv, i64 r0, i64 m, i64 n);

// Lower triangular inverse in place (Fig. 4), unit or not (api.cu).
template <typename T>
void trtri_rec(Ctx &c, bool unit, i64 n, T *A, i64 lda);

// ---- getri (getri.cu) -----------------------------------------------------------
// A := A^{-1} from the LU factors in place (inv(U) inv(L) P); work holds
// getri_work_bytes(n); n <= GETRI_MAX_N.
constexpr i64 GETRI_MAX_N = 40960;
size_t getri_work_bytes(i64 n);
template <typename T>
void getri(Ctx &c, i64 n, T *A, i64 lda, const int32_t *ipiv, void *work);

// ---- sygst (sygst.cu) ----------------------------------------------------------
// A := L^{-1} A L^{-T} (itype 1) or L^T A L (itype 2, 3), lower storage; T is
// sygst_work_bytes(n) of scratch or nullptr (recompute instead).
size_t sygst_work_bytes(i64 n, size_t esz);
template <typename E>
void sygst_rec(Ctx &c, int itype, i64 n, E *A, i64 lda, const E *L, i64 ldl, E *T);

// uplo = 'U' by transposition (uplo.cu): swap A(i, j) <-> A(j, i) for i != j
// (conjugated for complex), in place; never reads the abort flag.
template <typename T>
void uplo_swap(Ctx &c, i64 n, T *A, i64 lda);
template <typename T>
void uplo_swap_vbatched(Ctx &c, i64 batch, const int32_t *n, T *const *A, const int32_t *lda, int max_n);

// ---- precision form (mixed.cu) ----------------------------------------------
size_t mixed_work_size(i64 n, i64 nrhs, bool lu, int prec);
int mixed_solve(Ctx &c, bool lu, i64 n, i64 nrhs, double *A, i64 lda, int32_t *ipiv,
                const double *B, i64 ldb, double *X, i64 ldx, int prec, double tol, int maxiter,
                int32_t *iter);

}  // namespace rl

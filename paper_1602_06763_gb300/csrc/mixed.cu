// Precision form: solve A X = B to full FP64 backward error with a
// low-precision factorization and FP64 iterative refinement.
//
//   1. A (FP64) is converted to an FP32 working copy W (scaled by a power of
//      two for the FP16 form so that max |W| <= 1).
//   2. W is factored by the same recursions as the FP64 path (LU with partial
//      pivoting, or Cholesky) in FP32 storage.
//   3. x0 = solve(W, b); then, up to maxiter times: r = b - A x in FP64 (the
//      only FP64 arithmetic besides the update and the test), stop when
//      max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) <= tol,
//      else d = solve(W, r) in FP32 and x += d in FP64.
//   4. If the low-precision factorization fails or the refinement does not
//      converge, A is factored in FP64 in place and X = A^{-1} B (LAPACK
//      dsgesv / dsposv semantics).
// Every step is enqueued on the caller's stream; device flags make the
// kernels of finished or skipped steps return at once, so the call never
// synchronizes and has a fixed launch sequence.
//
// With RL_REFINE_GMRES the correction equation A d = r of each refinement
// step is solved by flexible GMRES (right preconditioned, restarted) instead
// of one solve with the low-precision factors: the factors precondition,
// applied in FP32 (z = M^{-1} v), while the Krylov basis, the products
// w = A z and the Hessenberg least-squares problem stay in FP64.  Flexible
// GMRES keeps the FP64 relation A Z = V H however inexactly the FP32 solve
// applies M^{-1}, so each cycle reduces the true residual of the correction
// equation to its tolerance; the low-precision factors only decide how many
// iterations that takes.  This is GMRES-based iterative refinement
// (E. Carson, N. J. Higham, SIAM J. Sci. Comput. 39, 2017 and 40, 2018) in
// the flexible form used with half-precision tensor-core factorizations
// (A. Haidar, S. Tomov, J. Dongarra, N. J. Higham, SC18): it converges where
// kappa(A) u_f >= 1 stops the classic loop.
#include <cfloat>
#include "internal.cuh"

namespace rl {

namespace {

constexpr int RES_ROWS = 256;     // rows per CTA of the residual kernel
constexpr int RES_KC = 512;       // k-chunk of the residual kernel
constexpr int RES_NR = 8;         // right-hand sides per residual pass
constexpr int NORM_CH = 64;       // column chunks of the infinity-norm kernel

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Scalars and flags kept on the device.
struct MixState {
    double anorm;          // ||A||_inf
    double scale;          // power of two applied to A in the working copy
    double prev_eta;       // backward error after the previous correction
    int32_t winfo;         // low-precision factorization info (or overflow)
    int32_t stop;          // nonzero: refinement finished or abandoned
    int32_t conv;          // 1: converged (fallback kernels skip)
    int32_t iters;         // corrections applied when converged
    int32_t pad[4];
    unsigned long long bmax[RES_NR * 64];   // per-RHS max |b| (bit patterns of doubles >= 0)
    unsigned long long xmax[RES_NR * 64];
    unsigned long long rmax[RES_NR * 64];
};
constexpr int MIX_MAX_NRHS = RES_NR * 64;

struct MixLayout {
    size_t W, panel, R, D, P, N, S, F, TC, tc_bytes, V, Z, ZC, WV, GS, OZP, OZW, ozw_bytes, total;
    i64 ldw, nchunks;
    int m;                 // GMRES restart length (0: classic refinement)
};

// ---- GMRES-IR state ----------------------------------------------------------
// digit planes of the emulated residual products
constexpr int OZ_RES_SLICES = 7;
constexpr int GM_MAX_NRHS = 64;
constexpr int GM_MAX_M = 64;
// a column's cycle ends once its least-squares residual is below this
// fraction of the cycle's starting residual (or below what the requested
// backward error needs)
constexpr double GM_TAU_REL = 1e-4;

struct GmCol {
    double beta;           // ||r||_2 at the start of the cycle
    double tau;            // the cycle's residual target
    double tau_abs;        // half the residual the requested backward error allows
    int32_t done, k;       // cycle finished for this column; its iterations
    double g[GM_MAX_M + 1], cs[GM_MAX_M], sn[GM_MAX_M], y[GM_MAX_M];
    double H[(GM_MAX_M + 1) * GM_MAX_M];   // R of the rotated Hessenberg, column j at j (m + 1)
};
struct GmState {
    int32_t j;             // next iteration of the open cycle
    int32_t open;          // a cycle is running
    int32_t has_cycle;     // a cycle ran since the last update of X
    int32_t total;         // preconditioner applications so far (all cycles)
    int32_t no_outer;      // this slot skips the update / residual / test / start block
    int32_t pad[11];
    GmCol col[GM_MAX_NRHS];
};

MixLayout layout(i64 n, i64 nrhs, bool lu, int prec)
{
    MixLayout L;
    const bool gm = (prec & RL_REFINE_GMRES) != 0;
    const bool oz = (prec & RL_REFINE_OZRES) != 0;
    prec &= RL_PREC_MASK;
    L.m = gm ? g_params.gmres_m : 0;
    L.ldw = ((n + 31) / 32) * 32;
    if (L.ldw < 1) L.ldw = 1;
    L.nchunks = (n + RES_KC - 1) / RES_KC;
    if (L.nchunks < 1) L.nchunks = 1;
    size_t off = 0;
    L.W = off; off += al((size_t)L.ldw * (size_t)(n > 0 ? n : 1) * sizeof(float));
    L.panel = off; off += lu ? al(panel_ws_bytes()) : 0;
    L.R = off; off += al((size_t)(n > 0 ? n : 1) * (size_t)nrhs * sizeof(double));
    L.D = off; off += al((size_t)(n > 0 ? n : 1) * (size_t)nrhs * sizeof(float));
    L.P = off; off += al((size_t)L.nchunks * RES_NR * (size_t)(n > 0 ? n : 1) * sizeof(double));
    L.N = off; off += al((size_t)(NORM_CH + 1) * (size_t)(n > 0 ? n : 1) * sizeof(double));
    L.S = off; off += al(sizeof(MixState));
    L.F = off; off += al(flow_ws_bytes(n, nrhs));
    // packing space of the tensor-core updates: the largest update of either
    // recursion has at most n rows and n/2 + 64 columns and inner dimension
    const i64 h = n / 2 + 64;
    L.tc_bytes = (prec == RL_PREC_FP32) ? 0 : tc_work_bytes(n, h, h, prec);
    L.TC = off; off += al(L.tc_bytes);
    // GMRES-IR: per right-hand side m + 1 basis vectors V and m
    // preconditioned vectors Z (FP64, n each, column after column), the
    // current z and w = A z for all right-hand sides, and the cycle state
    const size_t nn = (size_t)(n > 0 ? n : 1), nr = (size_t)nrhs;
    L.V = off; off += gm ? al(nr * (size_t)(L.m + 1) * nn * sizeof(double)) : 0;
    L.Z = off; off += gm ? al(nr * (size_t)L.m * nn * sizeof(double)) : 0;
    L.ZC = off; off += gm ? al(nr * nn * sizeof(double)) : 0;
    L.WV = off; off += gm ? al(nr * nn * sizeof(double)) : 0;
    L.GS = off; off += gm ? al(sizeof(GmState)) : 0;
    // emulated FP64 products: A's digit planes (made once) and the slicing
    // space of the thin operand
    L.ozw_bytes = oz ? oz_work_bytes(1, nrhs, n > 0 ? n : 1, OZ_RES_SLICES) : 0;
    L.OZP = off; off += oz ? al(oz_planes_bytes(n > 0 ? n : 1, n > 0 ? n : 1, OZ_RES_SLICES)) : 0;
    L.OZW = off; off += oz ? al(L.ozw_bytes) : 0;
    L.total = off;
    return L;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v)
{
    // non-negative doubles order like their bit patterns; NaN maps above +inf
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_mix_init(MixState *st, int nrhs)
{
    const int t = threadIdx.x;
    if (t == 0) {
        st->anorm = 0.0;
        st->scale = 1.0;
        st->prev_eta = 0.0;
        st->winfo = 0;
        st->stop = 0;
        st->conv = 0;
        st->iters = 0;
    }
    for (int j = t; j < MIX_MAX_NRHS; j += blockDim.x) { st->bmax[j] = 0; st->xmax[j] = 0; st->rmax[j] = 0; }
}

// Partial row sums of |A| over column chunks: N[ch * n + i].  SYM (the
// Cholesky form: only the lower triangle is referenced, as LAPACK's dsposv):
// the stored part of row i (columns j <= i) here, the rest of the row (the
// column below the diagonal) by k_colsum_lower into N[NORM_CH * n + i].
template <bool SYM>
__global__ void k_rowsum_partial(i64 n, const double *A, i64 lda, double *N)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    const i64 cw = (n + NORM_CH - 1) / NORM_CH, c0 = ch * cw;
    i64 c1 = min(n, c0 + cw);
    if (i >= n) return;
    if (SYM && c1 > i + 1) c1 = i + 1;
    double s = 0.0;
    for (i64 j = c0; j < c1; ++j) s += fabs(A[j * lda + i]);
    N[ch * n + i] = s;
}

// N[i] = sum_{j > i} |A(j, i)|: one warp per column, coalesced down it.
__global__ void k_colsum_lower(i64 n, const double *A, i64 lda, double *N)
{
    const i64 col = (i64)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (col >= n) return;
    double s = 0.0;
    for (i64 j = col + 1 + lane; j < n; j += 32) s += fabs(A[col * lda + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) N[col] = s;
}

// ||A||_inf, max|A| -> scale (power of two so that max|A| * scale <= 1 when
// requested), and max|b_j| per right-hand side.
__global__ void k_norms(i64 n, const double *N, int nch, const double *B, i64 ldb, int nrhs, int want_scale,
                        MixState *st)
{
    __shared__ double red[1024 / 32];
    double best = 0.0;
    for (i64 i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int ch = 0; ch < nch; ++ch) s += N[ch * n + i];
        if (s > best || s != s) best = s;
    }
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_down_sync(0xffffffffu, best, o);
        if (v > best || v != v) best = v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (red[w] > best || red[w] != red[w]) best = red[w];
        st->anorm = best;
    }
    // per-RHS max |b| (block reduction per column)
    for (int j = 0; j < nrhs; ++j) {
        double m = 0.0;
        for (i64 i = threadIdx.x; i < n; i += blockDim.x) {
            const double v = fabs(B[(i64)j * ldb + i]);
            if (v > m || v != v) m = v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_down_sync(0xffffffffu, m, o);
            if (v > m || v != v) m = v;
        }
        if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->bmax[j], m);
    }
    if (want_scale && threadIdx.x == 0) {
        // the largest |a_ij| is at most ||A||_inf; scaling by 2^-e with
        // 2^e >= ||A||_inf bounds every entry of the working copy by 1
        int e = 0;
        if (best > 0.0 && best == best) frexp(best, &e);
        st->scale = ldexp(1.0, -e);
    }
}

// W = (float)(A * scale); entries beyond the float range flag the working
// copy as unusable (LAPACK dsgesv's overflow check).
// SYM: the lower triangle only (the upper one is neither read nor written).
template <bool SYM>
__global__ void k_to_f32(i64 m, i64 n, const double *A, i64 lda, float *W, i64 ldw, const MixState *st,
                         int32_t *flag, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const double s = st->scale;
    const i64 total = m * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % m, j = e / m;
        if (SYM && i < j) continue;
        const double v = A[j * lda + i] * s;
        if (!(fabs(v) <= (double)FLT_MAX) && v == v) *flag = -2;
        W[j * ldw + i] = (float)v;
    }
}

// stop = (low-precision factorization failed) ? 1 : 0.
__global__ void k_after_factor(MixState *st)
{
    if (st->winfo != 0) st->stop = 1;
}

// Partial products P[ch][c][i] = sum_{k in chunk ch} A[i,k] X[k, c0 + c].
// SYM: A is symmetric with its lower triangle stored, A[i,k] = A(k, i) for
// k > i; a block above the diagonal reads its transposed tile down each
// thread's own column (each 32-byte sector serves 4 consecutive k of one
// thread from L1).
template <bool SYM>
__global__ void __launch_bounds__(RES_ROWS)
k_resid_partial(i64 n, int nr, const double *__restrict__ A, i64 lda, const double *__restrict__ X,
                i64 ldx, double *P, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Xs[RES_KC][RES_NR];
    const i64 row = (i64)blockIdx.x * RES_ROWS + threadIdx.x;
    const int ch = blockIdx.y;
    const i64 k0 = (i64)ch * RES_KC, k1 = min(n, k0 + RES_KC);
    const int kc = (int)(k1 - k0);
    for (int e = threadIdx.x; e < RES_KC * RES_NR; e += blockDim.x) {
        const int kk = e / RES_NR, c = e % RES_NR;
        Xs[kk][c] = (kk < kc && c < nr) ? X[(i64)c * ldx + k0 + kk] : 0.0;
    }
    __syncthreads();
    if (row >= n) return;
    double acc[RES_NR];
#pragma unroll
    for (int c = 0; c < RES_NR; ++c) acc[c] = 0.0;
    const i64 r0 = (i64)blockIdx.x * RES_ROWS;
    if (!SYM || k1 - 1 <= r0) {                  // every k <= row: stored as A(row, k)
        const double *ap = A + k0 * lda + row;
#pragma unroll 8
        for (int kk = 0; kk < kc; ++kk) {
            const double a = __ldg(ap + (i64)kk * lda);
#pragma unroll
            for (int c = 0; c < RES_NR; ++c) acc[c] = fma(a, Xs[kk][c], acc[c]);
        }
    } else if (k0 > r0 + RES_ROWS - 1) {         // every k > row: stored as A(k, row)
        const double *ap = A + row * lda + k0;
#pragma unroll 8
        for (int kk = 0; kk < kc; ++kk) {
            const double a = __ldg(ap + kk);
#pragma unroll
            for (int c = 0; c < RES_NR; ++c) acc[c] = fma(a, Xs[kk][c], acc[c]);
        }
    } else {                                     // the diagonal crosses this block
        for (int kk = 0; kk < kc; ++kk) {
            const i64 k = k0 + kk;
            const double a = (k <= row) ? __ldg(A + k * lda + row) : __ldg(A + row * lda + k);
#pragma unroll
            for (int c = 0; c < RES_NR; ++c) acc[c] = fma(a, Xs[kk][c], acc[c]);
        }
    }
    for (int c = 0; c < nr; ++c) P[((i64)ch * RES_NR + c) * n + row] = acc[c];
}

// R[:, c0 + c] = B - sum_ch P[ch][c]; running max |r| and max |x| per RHS.
__global__ void k_resid_final(i64 n, int nr, int c0, i64 nchunks, const double *P, const double *B,
                              i64 ldb, const double *X, i64 ldx, double *R, i64 ldr, MixState *st,
                              const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    for (int c = 0; c < nr; ++c) {
        double ra = 0.0, xa = 0.0;
        if (live) {
            double s = 0.0;
            for (i64 ch = 0; ch < nchunks; ++ch) s += P[(ch * RES_NR + c) * n + i];
            const double r = B[(i64)(c0 + c) * ldb + i] - s;
            R[(i64)(c0 + c) * ldr + i] = r;
            ra = fabs(r);
            xa = fabs(X[(i64)(c0 + c) * ldx + i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_down_sync(0xffffffffu, ra, o);
            const double w = __shfl_down_sync(0xffffffffu, xa, o);
            if (v > ra || v != v) ra = v;
            if (w > xa || w != w) xa = w;
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_nonneg(&st->rmax[c0 + c], ra);
            atomic_max_nonneg(&st->xmax[c0 + c], xa);
        }
    }
}

// Convergence test after residual number `it`: converged when every RHS has
// ||r||_inf <= tol (||A||_inf ||x||_inf + ||b||_inf).  The refinement is
// abandoned (fallback) once a correction fails to reduce the largest
// backward error by 10 %: the contraction factor of the low-precision
// factors (about kappa * u) is then near or above 1 and more iterations
// would not reach tol.  Clears the running maxima for the next residual.
__global__ void k_ir_test(int nrhs, int it, double tol, MixState *st)
{
    if (st->stop != 0) return;
    __shared__ int bad;
    __shared__ unsigned long long worst;
    if (threadIdx.x == 0) { bad = 0; worst = 0; }
    __syncthreads();
    for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
        const double r = __longlong_as_double((long long)st->rmax[j]);
        const double x = __longlong_as_double((long long)st->xmax[j]);
        const double b = __longlong_as_double((long long)st->bmax[j]);
        // r <= tol (||A|| ||x|| + ||b||) without the division: a zero
        // right-hand side (r = x = b = 0) has converged
        const double den = st->anorm * x + b;
        const double eta = (r == 0.0) ? 0.0 : r / den;
        if (!(r <= tol * den)) atomicExch(&bad, 1);
        atomicMax(&worst, (unsigned long long)__double_as_longlong(eta == eta ? eta : INFINITY));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nrhs; j += blockDim.x) { st->rmax[j] = 0; st->xmax[j] = 0; }
    if (threadIdx.x == 0) {
        const double eta = __longlong_as_double((long long)worst);
        if (!bad) {
            st->stop = 1;
            st->conv = 1;
            st->iters = it;
        } else if (it >= 1 && !(eta <= 0.9 * st->prev_eta)) {
            st->stop = 1;                      // stagnation: leave for the FP64 fallback
        }
        st->prev_eta = eta;
    }
}

// D = (float)(R * scale) for the correction solve.
__global__ void k_r_to_f32(i64 n, int nrhs, const double *R, i64 ldr, float *D, i64 ldd,
                           const MixState *st, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const double s = st->scale;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n, j = e / n;
        D[j * ldd + i] = (float)(R[j * ldr + i] * s);
    }
}

// X (+)= D widened; first = true assigns (x0 = solve(b)).
__global__ void k_x_update(i64 n, int nrhs, const float *D, i64 ldd, double *X, i64 ldx, int first,
                           const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n, j = e / n;
        const double d = (double)D[j * ldd + i];
        X[j * ldx + i] = first ? d : X[j * ldx + i] + d;
    }
}

// Fallback: X := B (before the FP64 solve), and the final iteration count.
__global__ void k_copy_b(i64 n, int nrhs, const double *B, i64 ldb, double *X, i64 ldx,
                         const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n, j = e / n;
        X[j * ldx + i] = B[j * ldb + i];
    }
}

__global__ void k_mix_finish(const MixState *st, int maxiter, int32_t *iter_out)
{
    int v;
    if (st->conv) v = st->iters;
    else if (st->winfo == -2) v = -2;            // conversion overflow
    else if (st->winfo != 0) v = -3;             // low-precision factorization failed
    else v = -31;                                // no convergence within maxiter
    (void)maxiter;
    *iter_out = v;
}

// ---- GMRES-IR kernels -----------------------------------------------------------

__global__ void k_gm_init(GmState *gs)
{
    gs->j = 0;
    gs->open = 0;
    gs->has_cycle = 0;
    gs->total = 0;
    gs->no_outer = 0;
}

// Start of a slot: the update / residual / test / start block runs when no
// cycle is open (and the solve has not stopped).
__global__ void k_gm_slot_begin(const MixState *st, GmState *gs)
{
    gs->no_outer = (st->stop != 0 || gs->open != 0) ? 1 : 0;
}

// X[:, c] += sum_l y_c[l] Z_c[l] after a cycle (each column's own k).
__global__ void k_gm_update(i64 n, int nrhs, int m, const double *Z, double *X, i64 ldx, const GmState *gs)
{
    if (gs->no_outer || !gs->has_cycle) return;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n;
        const int c = (int)(e / n);
        const GmCol &col = gs->col[c];
        const double *zc = Z + (i64)c * m * n + i;
        double d = 0.0;
        for (int l = 0; l < col.k; ++l) d = fma(col.y[l], zc[(i64)l * n], d);
        X[(i64)c * ldx + i] += d;
    }
}

// Backward error of every column after a residual: per-column targets for
// the next cycle, convergence (all columns at tol), budget and stagnation
// (a cycle that reduced the largest backward error by less than half: the
// FP64 fallback takes over).  Clears the running maxima.
__global__ void k_gm_test(int nrhs, double tol, int maxiter, MixState *st, GmState *gs)
{
    if (gs->no_outer) return;
    __shared__ int bad;
    __shared__ unsigned long long worst;
    if (threadIdx.x == 0) { bad = 0; worst = 0; }
    __syncthreads();
    for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
        const double r = __longlong_as_double((long long)st->rmax[j]);
        const double x = __longlong_as_double((long long)st->xmax[j]);
        const double b = __longlong_as_double((long long)st->bmax[j]);
        const double den = st->anorm * x + b;
        const double eta = (r == 0.0) ? 0.0 : r / den;
        const bool ok = r <= tol * den;         // a zero column (r = x = b = 0) has converged
        GmCol &col = gs->col[j];
        col.tau_abs = 0.5 * tol * den;
        col.done = ok ? 1 : 0;
        if (!ok) atomicExch(&bad, 1);
        atomicMax(&worst, (unsigned long long)__double_as_longlong(eta == eta ? eta : INFINITY));
        st->rmax[j] = 0;
        st->xmax[j] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double eta = __longlong_as_double((long long)worst);
        if (!bad) {
            st->stop = 1;
            st->conv = 1;
            st->iters = gs->total;
        } else if (gs->total >= maxiter || (gs->has_cycle && !(eta <= 0.5 * st->prev_eta))) {
            st->stop = 1;                        // budget spent or stagnation: FP64 fallback
        }
        st->prev_eta = eta;
        gs->has_cycle = 0;
    }
}

__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];      // same order in every thread
    return s;
}

// Start of a cycle (one CTA per right-hand side): beta = ||r||_2,
// v_0 = r / beta, g = beta e_1; columns already at tol take no part.
__global__ void k_gm_start(i64 n, int m, const double *R, i64 ldr, double *V, MixState *st, GmState *gs)
{
    if (gs->no_outer || st->stop) return;
    __shared__ double red[32];
    const int c = blockIdx.x;
    GmCol &col = gs->col[c];
    if (c == 0 && threadIdx.x == 0) {
        gs->j = 0;
        gs->open = 1;
        gs->has_cycle = 1;
    }
    if (threadIdx.x == 0) col.k = 0;
    if (col.done) return;
    const double *r = R + (i64)c * ldr;
    double s = 0.0;
    for (i64 i = threadIdx.x; i < n; i += blockDim.x) s = fma(r[i], r[i], s);
    const double beta = sqrt(block_sum(s, red));
    double *v = V + (i64)c * (m + 1) * n;
    if (threadIdx.x == 0) {
        col.beta = beta;
        col.g[0] = beta;
        col.tau = fmax(GM_TAU_REL * beta, col.tau_abs);
        if (!(beta > 0.0)) col.done = 1;
    }
    if (!(beta > 0.0)) return;
    const double inv = 1.0 / beta;
    for (i64 i = threadIdx.x; i < n; i += blockDim.x) v[i] = r[i] * inv;
}

// D[:, c] = (float)(s v_j) for the preconditioner solve (0 for columns that
// are done).
__global__ void k_gm_prep(i64 n, int nrhs, int m, const double *V, float *D, i64 ldd, const MixState *st,
                          const GmState *gs)
{
    if (st->stop) return;
    const int j = gs->j;
    const double sc = st->scale;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n;
        const int c = (int)(e / n);
        const double v = gs->col[c].done ? 0.0 : V[((i64)c * (m + 1) + j) * n + i];
        D[(i64)c * ldd + i] = (float)(v * sc);
    }
}

// z_j = (double) D (the FP32 solve's result); also into ZC, the operand of
// the product w = A z.
__global__ void k_gm_widen(i64 n, int nrhs, int m, const float *D, i64 ldd, double *Z, double *ZC,
                           const MixState *st, const GmState *gs)
{
    if (st->stop) return;
    const int j = gs->j;
    const i64 total = n * nrhs;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % n;
        const int c = (int)(e / n);
        const double z = gs->col[c].done ? 0.0 : (double)D[(i64)c * ldd + i];
        Z[((i64)c * m + j) * n + i] = z;
        ZC[(i64)c * n + i] = z;
    }
}

// W[:, c0 + c] = sum_ch P[ch][c] (the product A z, from the residual
// kernel's partial sums).
__global__ void k_mv_final(i64 n, int nr, int c0, i64 nchunks, const double *P, double *W, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nr; ++c) {
        double s = 0.0;
        for (i64 ch = 0; ch < nchunks; ++ch) s += P[(ch * RES_NR + c) * n + i];
        W[(i64)(c0 + c) * n + i] = s;
    }
}

// One Arnoldi step per right-hand side (one CTA each): modified Gram-Schmidt
// of w against v_0..v_j, h_{j+1,j} = ||w||_2, v_{j+1} = w / h_{j+1,j}; the
// previous Givens rotations and a new one reduce the Hessenberg column to
// triangular form, and |g_{j+1}| is the least-squares residual.  A column
// whose residual meets its target (or whose basis breaks down, or whose
// cycle reaches m iterations or the budget) solves R y = g for its update.
__global__ void __launch_bounds__(1024)
k_gm_arnoldi(i64 n, int m, int maxiter, double *V, double *W, MixState *st, GmState *gs)
{
    if (st->stop) return;
    __shared__ double red[32];
    __shared__ double h[GM_MAX_M + 1];
    const int c = blockIdx.x;
    GmCol &col = gs->col[c];
    if (col.done) return;
    const int j = gs->j;
    double *w = W + (i64)c * n;
    double *Vc = V + (i64)c * (m + 1) * n;
    for (int i = 0; i <= j; ++i) {
        const double *vi = Vc + (i64)i * n;
        double s = 0.0;
        for (i64 r = threadIdx.x; r < n; r += blockDim.x) s = fma(vi[r], w[r], s);
        const double hi = block_sum(s, red);
        for (i64 r = threadIdx.x; r < n; r += blockDim.x) w[r] = fma(-hi, vi[r], w[r]);
        if (threadIdx.x == 0) h[i] = hi;
        __syncthreads();
    }
    double s = 0.0;
    for (i64 r = threadIdx.x; r < n; r += blockDim.x) s = fma(w[r], w[r], s);
    const double hn = sqrt(block_sum(s, red));
    if (hn > 0.0) {
        const double inv = 1.0 / hn;
        double *vn = Vc + (i64)(j + 1) * n;
        for (i64 r = threadIdx.x; r < n; r += blockDim.x) vn[r] = w[r] * inv;
    }
    if (threadIdx.x != 0) return;
    h[j + 1] = hn;
    for (int l = 0; l < j; ++l) {                       // earlier rotations
        const double t = col.cs[l] * h[l] + col.sn[l] * h[l + 1];
        h[l + 1] = -col.sn[l] * h[l] + col.cs[l] * h[l + 1];
        h[l] = t;
    }
    const double rr = hypot(h[j], h[j + 1]);
    const double cj = rr > 0.0 ? h[j] / rr : 1.0, sj = rr > 0.0 ? h[j + 1] / rr : 0.0;
    col.cs[j] = cj;
    col.sn[j] = sj;
    h[j] = rr;
    col.g[j + 1] = -sj * col.g[j];
    col.g[j] = cj * col.g[j];
    double *Hj = col.H + (i64)j * (m + 1);
    for (int l = 0; l <= j; ++l) Hj[l] = h[l];
    const int k = j + 1;
    col.k = k;
    const bool fin = fabs(col.g[k]) <= col.tau || !(hn > 0.0) || k == m || gs->total + 1 >= maxiter;
    if (!fin) return;
    for (int l = k - 1; l >= 0; --l) {                  // R y = g
        double t = col.g[l];
        for (int q = l + 1; q < k; ++q) t -= col.H[(i64)q * (m + 1) + l] * col.y[q];
        const double d = col.H[(i64)l * (m + 1) + l];
        col.y[l] = d != 0.0 ? t / d : 0.0;
    }
    col.done = 1;
}

// End of a slot: count the iteration; close the cycle when every column is
// done, at m iterations, or when the budget is spent.
__global__ void k_gm_slot_end(int nrhs, int m, int maxiter, const MixState *st, GmState *gs)
{
    if (st->stop || !gs->open) return;
    gs->j += 1;
    gs->total += 1;
    bool all = true;
    for (int c = 0; c < nrhs; ++c) all = all && gs->col[c].done;
    if (all || gs->j >= m || gs->total >= maxiter) gs->open = 0;
}

// Running maxima of |r| and |x| per column after an emulated residual.
__global__ void k_resid_stats(i64 n, int nrhs, const double *R, i64 ldr, const double *X, i64 ldx, MixState *st,
                              const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    for (int c = 0; c < nrhs; ++c) {
        double ra = live ? fabs(R[(i64)c * ldr + i]) : 0.0;
        double xa = live ? fabs(X[(i64)c * ldx + i]) : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_down_sync(0xffffffffu, ra, o);
            const double w = __shfl_down_sync(0xffffffffu, xa, o);
            if (v > ra || v != v) ra = v;
            if (w > xa || w != w) xa = w;
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_nonneg(&st->rmax[c], ra);
            atomic_max_nonneg(&st->xmax[c], xa);
        }
    }
}

unsigned grid_for(i64 total, unsigned threads)
{
    i64 g = (total + threads - 1) / threads;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

// FP32 solve of W d = P r (LU) or L L^T d = r (Cholesky) on the nrhs columns
// of D.
// X := A^{-1} X from the factors in F (LU with ipiv, or Cholesky L): thin
// right-hand sides take the one-launch flow solve, wide ones the recursive
// TRSM.
template <typename T>
static void factored_solve(Ctx &c, bool lu, i64 n, i64 nrhs, const T *F, i64 ldf, const int32_t *ipiv,
                           T *X, i64 ldx, void *flow_ws)
{
    if (lu) laswp<T>(c, X, ldx, n, 0, nrhs, 0, n, ipiv);
    if (nrhs <= FLOW_MAX_NRHS) {
        trsm_flow<T>(c, FLOW_LN, lu, n, nrhs, F, ldf, X, ldx, flow_ws);
        trsm_flow<T>(c, lu ? FLOW_UN : FLOW_LT, false, n, nrhs, F, ldf, X, ldx, flow_ws);
    } else if (lu) {
        trsm_lln<T>(c, true, n, nrhs, T(1), F, ldf, X, ldx);
        trsm_lun<T>(c, n, nrhs, T(1), F, ldf, X, ldx);
    } else {
        trsm_lln<T>(c, false, n, nrhs, T(1), F, ldf, X, ldx);
        trsm_llt<T>(c, n, nrhs, T(1), F, ldf, X, ldx);
    }
}

size_t mixed_work_size(i64 n, i64 nrhs, bool lu, int prec) { return layout(n, nrhs, lu, prec).total; }

// R[:, c0..] = B - A X (FP64) for every block of RES_NR right-hand sides,
// with the running maxima of |r| and |x| per column; or, with B null,
// OUT = A X.
// Emulated FP64 products of the refinement: A's digit planes (made once per
// call) and the slicing space of the thin operand.
struct OzRes {
    const void *planes;
    void *work;
    size_t lwork;
};

static void residual_blocks(Ctx &r, bool lu, i64 n, i64 nrhs, const double *A, i64 lda, const double *X,
                            i64 ldx, const double *B, i64 ldb, double *OUT, i64 ldo, double *P, i64 nchunks,
                            MixState *st, const OzRes *oz = nullptr)
{
    if (oz) {
        // OUT = B - A X (one product, alpha -1 onto a copy of B) or OUT = A X,
        // the product emulated on the BF16 tensor cores with A's planes
        const unsigned T256 = 256;
        if (B) {
            Launch L(r, K_MIX, 0.0, 16.0 * n * nrhs);
            k_copy_b<<<grid_for(n * nrhs, T256), T256, 0, r.s>>>(n, (int)nrhs, B, ldb, OUT, ldo, r.abort);
        }
        oz_gemm_planes(r, OZ_RES_SLICES, n, nrhs, n, B ? -1.0 : 1.0, oz->planes, X, ldx, B ? 1.0 : 0.0, OUT, ldo,
                       oz->work, oz->lwork);
        if (B) {
            Launch L(r, K_RESID, 0.0, 16.0 * n * nrhs);
            k_resid_stats<<<(unsigned)((n + 255) / 256), 256, 0, r.s>>>(n, (int)nrhs, OUT, ldo, X, ldx, st, r.abort);
        }
        return;
    }
    for (i64 c0 = 0; c0 < nrhs; c0 += RES_NR) {
        const int nr = (int)((nrhs - c0) < RES_NR ? (nrhs - c0) : RES_NR);
        {
            Launch L(r, K_RESID, 2.0 * n * n * nr, (double)n * n * sizeof(double));
            const dim3 g((unsigned)((n + RES_ROWS - 1) / RES_ROWS), (unsigned)nchunks);
            const double *Xc = X + c0 * ldx;
            if (lu) k_resid_partial<false><<<g, RES_ROWS, 0, r.s>>>(n, nr, A, lda, Xc, ldx, P, r.abort);
            else k_resid_partial<true><<<g, RES_ROWS, 0, r.s>>>(n, nr, A, lda, Xc, ldx, P, r.abort);
        }
        {
            Launch L(r, K_RESID, (double)n * nr * nchunks, 0.0);
            if (B)
                k_resid_final<<<(unsigned)((n + 255) / 256), 256, 0, r.s>>>(n, nr, (int)c0, nchunks, P, B, ldb, X,
                                                                             ldx, OUT, ldo, st, r.abort);
            else
                k_mv_final<<<(unsigned)((n + 255) / 256), 256, 0, r.s>>>(n, nr, (int)c0, nchunks, P, OUT, r.abort);
        }
    }
}

// GMRES-IR: maxiter slots, each an optional block (update X from the last
// cycle, residual, backward-error test, start of a new cycle: it runs when
// no cycle is open) and one flexible-GMRES iteration; then a last update,
// residual and test.  Device flags decide which parts run, so the launch
// sequence is fixed.
static void gmres_refine(Ctx &r, bool lu, i64 n, i64 nrhs, const double *A, i64 lda, const int32_t *ipiv,
                         const double *B, i64 ldb, double *X, i64 ldx, const float *W, i64 ldw, float *D,
                         i64 ldd, double *R, i64 ldr, double *P, MixState *st, void *fws, const MixLayout &Ly,
                         double tol, int maxiter, const OzRes *oz)
{
    char *w = static_cast<char *>(r.work);
    double *V = reinterpret_cast<double *>(w + Ly.V);
    double *Z = reinterpret_cast<double *>(w + Ly.Z);
    double *ZC = reinterpret_cast<double *>(w + Ly.ZC);
    double *WV = reinterpret_cast<double *>(w + Ly.WV);
    GmState *gs = reinterpret_cast<GmState *>(w + Ly.GS);
    const int m = Ly.m, nr = (int)nrhs;
    const unsigned T256 = 256;
    const unsigned gel = grid_for(n * nrhs, T256);
    { Launch L(r, K_MIX, 0.0, 0.0); k_gm_init<<<1, 1, 0, r.s>>>(gs); }
    Ctx ro = r;                                  // the update / residual / test / start block
    ro.abort = &gs->no_outer;
    auto outer = [&]() {
        { Launch L(r, K_MIX, 0.0, 0.0); k_gm_slot_begin<<<1, 1, 0, r.s>>>(st, gs); }
        {
            Launch L(ro, K_MIX, 2.0 * n * nrhs * m, (double)n * nrhs * m * sizeof(double));
            k_gm_update<<<gel, T256, 0, r.s>>>(n, nr, m, Z, X, ldx, gs);
        }
        residual_blocks(ro, lu, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, P, Ly.nchunks, st, oz);
        { Launch L(ro, K_MIX, 0.0, 0.0); k_gm_test<<<1, 256, 0, r.s>>>(nr, tol, maxiter, st, gs); }
        {
            Launch L(ro, K_MIX, 0.0, (double)n * nrhs * 16.0);
            k_gm_start<<<nr, 1024, 0, r.s>>>(n, m, R, ldr, V, st, gs);
        }
        if (ro.err != cudaSuccess && r.err == cudaSuccess) r.err = ro.err;
    };
    for (int slot = 0; slot < maxiter; ++slot) {
        outer();
        {
            Launch L(r, K_CONVERT, 0.0, (double)n * nrhs * 12.0);
            k_gm_prep<<<gel, T256, 0, r.s>>>(n, nr, m, V, D, ldd, st, gs);
        }
        factored_solve<float>(r, lu, n, nrhs, W, ldw, ipiv, D, ldd, fws);
        {
            Launch L(r, K_CONVERT, 0.0, (double)n * nrhs * 20.0);
            k_gm_widen<<<gel, T256, 0, r.s>>>(n, nr, m, D, ldd, Z, ZC, st, gs);
        }
        residual_blocks(r, lu, n, nrhs, A, lda, ZC, n, nullptr, 0, WV, n, P, Ly.nchunks, st, oz);
        {
            Launch L(r, K_MIX, 4.0 * n * nrhs * m, (double)n * nrhs * m * 3 * sizeof(double));
            k_gm_arnoldi<<<nr, 1024, 0, r.s>>>(n, m, maxiter, V, WV, st, gs);
        }
        { Launch L(r, K_MIX, 0.0, 0.0); k_gm_slot_end<<<1, 1, 0, r.s>>>(nr, m, maxiter, st, gs); }
        if (r.err != cudaSuccess) return;
    }
    outer();
}

int mixed_solve(Ctx &c, bool lu, i64 n, i64 nrhs, double *A, i64 lda, int32_t *ipiv, const double *B,
                i64 ldb, double *X, i64 ldx, int prec, double tol, int maxiter, int32_t *iter)
{
    const MixLayout Ly = layout(n, nrhs, lu, prec);
    char *w = static_cast<char *>(c.work);
    float *W = reinterpret_cast<float *>(w + Ly.W);
    void *pws = w + Ly.panel;
    double *R = reinterpret_cast<double *>(w + Ly.R);
    float *D = reinterpret_cast<float *>(w + Ly.D);
    double *P = reinterpret_cast<double *>(w + Ly.P);
    double *Nn = reinterpret_cast<double *>(w + Ly.N);
    MixState *st = reinterpret_cast<MixState *>(w + Ly.S);
    void *fws = w + Ly.F;
    const i64 ldw = Ly.ldw, ldr = n, ldd = n;
    int32_t *user_info = c.info;
    const unsigned T256 = 256;
    const bool gm = (prec & RL_REFINE_GMRES) != 0;
    const bool ozr = (prec & RL_REFINE_OZRES) != 0;
    prec &= RL_PREC_MASK;

    if (tol <= 0.0) tol = 1e-14;
    if (maxiter < 0) maxiter = 0;

    { Launch L(c, K_MIX, 0.0, 0.0); k_mix_init<<<1, 256, 0, c.s>>>(st, (int)nrhs); }
    {
        Launch L(c, K_MIX, 0.0, (lu ? 1.0 : 0.5) * n * n * sizeof(double));
        const dim3 g((unsigned)((n + 255) / 256), NORM_CH);
        if (lu) k_rowsum_partial<false><<<g, 256, 0, c.s>>>(n, A, lda, Nn);
        else k_rowsum_partial<true><<<g, 256, 0, c.s>>>(n, A, lda, Nn);
    }
    if (!lu) {
        Launch L(c, K_MIX, 0.0, 0.5 * n * n * sizeof(double));
        k_colsum_lower<<<(unsigned)((n + 7) / 8), 256, 0, c.s>>>(n, A, lda, Nn + (i64)NORM_CH * n);
    }
    {
        Launch L(c, K_MIX, 0.0, 0.0);
        k_norms<<<1, 1024, 0, c.s>>>(n, Nn, lu ? NORM_CH : NORM_CH + 1, B, ldb, (int)nrhs,
                                     prec == RL_PREC_FP16S, st);
    }
    {
        Launch L(c, K_CONVERT, 0.0, (lu ? 1.0 : 0.5) * n * n * (sizeof(double) + sizeof(float)));
        const unsigned g = grid_for(n * n, T256);
        if (lu) k_to_f32<false><<<g, T256, 0, c.s>>>(n, n, A, lda, W, ldw, st, &st->winfo, nullptr);
        else k_to_f32<true><<<g, T256, 0, c.s>>>(n, n, A, lda, W, ldw, st, &st->winfo, nullptr);
    }

    // low-precision factorization of W (its info lands in st->winfo)
    {
        Ctx f = c;
        f.info = &st->winfo;
        f.abort = &st->winfo;
        f.work = pws;
        f.prec = prec;
        f.tcwork = prec == RL_PREC_FP32 ? nullptr : w + Ly.TC;   // no packing space in the FP32 form
        f.tclwork = Ly.tc_bytes;
        if (lu) getrf_rec_t<float>(f, W, ldw, n, ipiv, 0, n, n);
        else potrf_rec_t<float>(f, n, W, ldw, 0);
        if (f.err != cudaSuccess && c.err == cudaSuccess) c.err = f.err;
    }
    { Launch L(c, K_MIX, 0.0, 0.0); k_after_factor<<<1, 1, 0, c.s>>>(st); }

    Ctx r = c;            // refinement kernels skip once st->stop is set
    r.abort = &st->stop;
    r.info = nullptr;

    // x0 = solve(W, b)
    {
        Launch L(r, K_CONVERT, 0.0, (double)n * nrhs * 12.0);
        k_r_to_f32<<<grid_for(n * nrhs, T256), T256, 0, r.s>>>(n, (int)nrhs, B, ldb, D, ldd, st, r.abort);
    }
    factored_solve<float>(r, lu, n, nrhs, W, ldw, ipiv, D, ldd, fws);
    {
        Launch L(r, K_MIX, 0.0, 0.0);
        k_x_update<<<grid_for(n * nrhs, T256), T256, 0, r.s>>>(n, (int)nrhs, D, ldd, X, ldx, 1, r.abort);
    }
    // the scale of the FP16 form is undone when D is widened: A_s = s A, so
    // A^{-1} r = s (A_s)^{-1} r, and D = (A_s)^{-1} (s r) is already A^{-1} r.
    OzRes ozs{w + Ly.OZP, w + Ly.OZW, Ly.ozw_bytes};
    const OzRes *oz = nullptr;
    if (ozr) {
        // A's digit planes, once, for every residual (and GMRES product)
        Ctx o = r;
        oz_prepare(o, OZ_RES_SLICES, !lu, n, n, A, lda, w + Ly.OZP);
        if (o.err != cudaSuccess && c.err == cudaSuccess) c.err = o.err;
        oz = &ozs;
    }
    if (gm) {
        gmres_refine(r, lu, n, nrhs, A, lda, ipiv, B, ldb, X, ldx, W, ldw, D, ldd, R, ldr, P, st, fws, Ly, tol,
                     maxiter, oz);
        maxiter = -1;                        // the classic loop below does not run
    }
    for (int it = 0; it <= maxiter; ++it) {
        residual_blocks(r, lu, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, P, Ly.nchunks, st, oz);
        { Launch L(r, K_MIX, 0.0, 0.0); k_ir_test<<<1, 256, 0, r.s>>>((int)nrhs, it, tol, st); }
        if (it == maxiter) break;
        {
            Launch L(r, K_CONVERT, 0.0, (double)n * nrhs * 12.0);
            k_r_to_f32<<<grid_for(n * nrhs, T256), T256, 0, r.s>>>(n, (int)nrhs, R, ldr, D, ldd, st, r.abort);
        }
        factored_solve<float>(r, lu, n, nrhs, W, ldw, ipiv, D, ldd, fws);
        {
            Launch L(r, K_MIX, 0.0, 0.0);
            k_x_update<<<grid_for(n * nrhs, T256), T256, 0, r.s>>>(n, (int)nrhs, D, ldd, X, ldx, 0, r.abort);
        }
        if (r.err != cudaSuccess) break;
    }
    if (r.err != cudaSuccess && c.err == cudaSuccess) c.err = r.err;

    // FP64 fallback (skipped when converged): factor A in place, X = A^{-1} B
    {
        Ctx f = c;
        f.abort = &st->conv;
        f.info = user_info;
        f.work = pws;
        {
            Launch L(f, K_MIX, 0.0, 0.0);
            k_copy_b<<<grid_for(n * nrhs, T256), T256, 0, f.s>>>(n, (int)nrhs, B, ldb, X, ldx, f.abort);
        }
        if (lu) getrf_rec_t<double>(f, A, lda, n, ipiv, 0, n, n);
        else potrf_rec_t<double>(f, n, A, lda, 0);
        factored_solve<double>(f, lu, n, nrhs, A, lda, ipiv, X, ldx, fws);
        if (f.err != cudaSuccess && c.err == cudaSuccess) c.err = f.err;
    }
    { Launch L(c, K_MIX, 0.0, 0.0); k_mix_finish<<<1, 1, 0, c.s>>>(st, maxiter, iter); }
    return 0;
}

}  // namespace rl

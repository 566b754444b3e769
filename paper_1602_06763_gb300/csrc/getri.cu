// getri: A^{-1} from the LU factors (Section 5: xtrtri is the building block
// of xgetri).  With P A = L U, A^{-1} = U^{-1} L^{-1} P:
//   1. U := U^{-1} in place (upper triangle; recursive TRTRI of the upper
//      form, the transpose of Fig. 4's updates);
//   2. L := L^{-1} in place (strictly lower, unit diagonal; Fig. 4);
//   3. W := U^{-1} L^{-1} in place, recursive by halving: with X = U^{-1}
//      and Y = L^{-1} sharing the storage,
//        W11 = X11 Y11 + X12 Y21   (recursion, then GEMM)
//        W12 = X12 Y22             (TRMM, Y22 unit lower)
//        W21 = X22 Y21             (TRMM, X22 upper)
//        W22 = X22 Y22             (recursion)
//      in that order, so every product reads operands not yet overwritten;
//      blocks of order <= 64 in one CTA;
//   4. the column interchanges of P applied in reverse (as LAPACK's dgetri
//      does): one CTA turns ipiv into the cycles of the net column
//      permutation, then every CTA walks those cycles over its own rows.
#include "internal.cuh"

namespace rl {

namespace {

// block order of the base case: 64, or 32 for complex (16-byte) elements
// so that the staged block fits the 48 KB of static shared memory
template <typename T> constexpr int ul_n() { return sizeof(T) > 8 ? 32 : 64; }

// W = X Y for one block of order <= ul_n: X upper (with diagonal), Y unit
// lower (strictly lower part stored), both in A; W overwrites A.
template <typename T>
__global__ void __launch_bounds__(256)
k_uinv_linv(int n, T *A, i64 lda, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    constexpr int UL_N = ul_n<T>(), UL_P = UL_N + 1;
    __shared__ T S[UL_N * UL_P];                 // S(i, k) at S[k * UL_P + i]
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e % n, k = e / n;
        S[k * UL_P + i] = A[(i64)k * lda + i];
    }
    __syncthreads();
    constexpr int PER = UL_N * UL_N / 256;
    T w[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + 256 * u;
        const int i = e % UL_N, j = e / UL_N;
        T s = T(0);
        if (i < n && j < n) {
            const int k0 = i > j ? i : j;
            // k = j: Y(j, j) = 1
            if (k0 == j) s = S[j * UL_P + i];
            for (int k = (k0 == j ? j + 1 : k0); k < n; ++k) s = fma(S[k * UL_P + i], S[j * UL_P + k], s);
        }
        w[u] = s;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + 256 * u;
        const int i = e % UL_N, j = e / UL_N;
        if (i < n && j < n) A[(i64)j * lda + i] = w[u];
    }
}

template <typename T>
void uinv_linv_rec(Ctx &c, i64 n, T *A, i64 lda)
{
    if (n <= 0) return;
    if (n <= ul_n<T>()) {
        Launch L(c, K_TRMM, 2.0 * n * n * n / 3.0, 0.0);
        k_uinv_linv<T><<<1, 256, 0, c.s>>>((int)n, A, lda, c.abort);
        return;
    }
    const i64 n1 = split_q(n, ul_n<T>()), n2 = n - n1;
    T *A11 = A, *A12 = A + n1 * lda, *A21 = A + n1, *A22 = A + n1 + n1 * lda;
    uinv_linv_rec<T>(c, n1, A11, lda);
    gemm<T>(c, false, false, n1, n1, n2, T(1), A12, lda, A21, lda, T(1), A11, lda);
    trmm_rln<T>(c, true, n1, n2, T(1), A22, lda, A12, lda);
    trmm_lun<T>(c, n2, n1, T(1), A22, lda, A21, lda);
    uinv_linv_rec<T>(c, n2, A22, lda);
}

// Upper-triangular inverse, non-unit: the transpose of Fig. 4's scheme.
template <typename T>
void trtri_upper_rec(Ctx &c, i64 n, T *A, i64 lda)
{
    if (n <= 0) return;
    const i64 base = sizeof(T) > 8 && g_params.trtri_c > 32 ? 32 : g_params.trtri_c;
    if (n <= base) { trti2<T>(c, false, n, A, lda, true); return; }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    T *TR = A + n1 * lda, *BR = A + n1 + n1 * lda;
    trtri_upper_rec<T>(c, n1, A, lda);
    trmm_lun<T>(c, n1, n2, T(1), A, lda, TR, lda);        // TR := U11^{-1} U12
    trsm_run<T>(c, n1, n2, T(-1), BR, lda, TR, lda);      // TR := -TR U22^{-1}
    trtri_upper_rec<T>(c, n2, BR, lda);
}

// Column permutation plan.  Applying the swaps (j, ipiv[j]) for j = n-1..0
// to the columns leaves original column src[j] in column j; the cycles of
// src are written as one list (cycle after cycle, fixed points omitted) with
// their end offsets.  One CTA; src and the visited marks in shared memory.
constexpr int CP_STAGE = 2048;

struct PermPlan {
    int ncyc;
    int pad[63];
    int data[1];          // list[n], then ends[n]
};

__global__ void __launch_bounds__(256)
k_colperm_plan(int n, const int32_t *ipiv, PermPlan *plan, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ int cp_smem[];
    int *src = cp_smem;
    unsigned char *vis = reinterpret_cast<unsigned char *>(cp_smem + n);
    __shared__ int stage[CP_STAGE];
    for (int j = threadIdx.x; j < n; j += blockDim.x) { src[j] = j; vis[j] = 0; }
    // the swaps, last first; ipiv staged in chunks so thread 0 reads shared memory only
    for (int hi = n; hi > 0; hi -= CP_STAGE) {
        const int lo = hi - CP_STAGE > 0 ? hi - CP_STAGE : 0;
        __syncthreads();
        for (int j = lo + (int)threadIdx.x; j < hi; j += blockDim.x) stage[j - lo] = ipiv[j] - 1;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int j = hi - 1; j >= lo; --j) {
                const int p = stage[j - lo];
                if (p != j && p >= 0 && p < n) { const int t = src[j]; src[j] = src[p]; src[p] = t; }
            }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int *list = plan->data, *ends = plan->data + n;
        int len = 0, nc = 0;
        for (int s = 0; s < n; ++s) {
            if (vis[s] || src[s] == s) continue;
            int j = s;
            do { vis[j] = 1; list[len++] = j; j = src[j]; } while (j != s);
            ends[nc++] = len;
        }
        plan->ncyc = nc;
    }
}

// Each thread owns one row and walks every cycle over it: col[a0] saved,
// col[a_t] = col[a_{t+1}], col[a_last] = saved; the loads of a batch are
// issued before its stores (the columns of one cycle are distinct).
constexpr int CP_ROWS = 64, CP_BATCH = 16;

template <typename T>
__global__ void __launch_bounds__(CP_ROWS)
k_colperm_apply(int n, T *A, i64 lda, const PermPlan *plan, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 r = (i64)blockIdx.x * CP_ROWS + threadIdx.x;
    if (r >= n) return;
    const int *list = plan->data, *ends = plan->data + n;
    const int nc = plan->ncyc;
    int beg = 0;
    for (int cy = 0; cy < nc; ++cy) {
        const int end = ends[cy];
        const T saved = A[(i64)list[beg] * lda + r];
        int t = beg;
        while (t + 1 < end) {
            const int cnt = min(CP_BATCH, end - 1 - t);
            T v[CP_BATCH];
#pragma unroll
            for (int u = 0; u < CP_BATCH; ++u)
                if (u < cnt) v[u] = A[(i64)list[t + 1 + u] * lda + r];
#pragma unroll
            for (int u = 0; u < CP_BATCH; ++u)
                if (u < cnt) A[(i64)list[t + u] * lda + r] = v[u];
            t += cnt;
        }
        A[(i64)list[end - 1] * lda + r] = saved;
        beg = end;
    }
}

}  // namespace

size_t getri_work_bytes(i64 n)
{
    return 256 + 2 * (size_t)(n > 0 ? n : 1) * sizeof(int);
}

template <typename T>
void getri(Ctx &c, i64 n, T *A, i64 lda, const int32_t *ipiv, void *work)
{
    if (n <= 0) return;
    diag_zero_scan<T>(c, n, A, lda);              // info = first zero of U's diagonal
    trtri_upper_rec<T>(c, n, A, lda);
    trtri_rec<T>(c, true, n, A, lda);             // L := L^{-1}, unit diagonal
    uinv_linv_rec<T>(c, n, A, lda);
    PermPlan *plan = static_cast<PermPlan *>(work);
    const size_t smem = (size_t)n * sizeof(int) + (size_t)n;
    note(c, smem_optin(k_colperm_plan, (size_t)GETRI_MAX_N * 5));
    {
        Launch L(c, K_LASWP, 0.0, 0.0);
        k_colperm_plan<<<1, 256, smem, c.s>>>((int)n, ipiv, plan, c.abort);
    }
    Launch L(c, K_LASWP, 0.0, 2.0 * sizeof(T) * (double)n * n);
    k_colperm_apply<T><<<(unsigned)((n + CP_ROWS - 1) / CP_ROWS), CP_ROWS, 0, c.s>>>((int)n, A, lda, plan,
                                                                                      c.abort);
}

template void getri<double>(Ctx &, i64, double *, i64, const int32_t *, void *);
template void getri<float>(Ctx &, i64, float *, i64, const int32_t *, void *);
template void getri<cplx>(Ctx &, i64, cplx *, i64, const int32_t *, void *);

}  // namespace rl

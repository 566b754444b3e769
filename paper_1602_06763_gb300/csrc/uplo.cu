// uplo = 'U' for the symmetric / triangular routines (Section 5: LAPACK's
// interface, both triangles).  With A = U^T U and U = L^T, every upper form
// is the lower form of the transposed storage:
//   potrf:  U = (chol_L(A))^T           trtri:  U^{-1} = (L^{-1})^T
//   lauum:  U U^T = L^T L               potri:  (U^T U)^{-1} = (L L^T)^{-1}
//   sygst:  U^{-T} A U^{-1} = L^{-1} A L^{-T},  U A U^T = L^T A L
// so an upper call swaps the two triangles of its square operands in place
// (for complex, A := A^H: conjugating, the diagonal included), runs the
// lower recursion, and swaps back: the strictly lower part comes back
// unchanged, as LAPACK leaves the unreferenced triangle.  A swap moves 2 * 16 B per off-diagonal
// element pair (read and write of both), about 0.1 % of a factorization's
// time at n = 16384, against a second copy of every kernel.
//
// The swap never reads the abort flag: the swap back must run even when the
// lower recursion stopped early (its partial result goes back to the upper
// triangle, with info set, as LAPACK's upper routines leave it).
#include "internal.cuh"

namespace rl {

namespace {

constexpr int SW_T = 32;        // tile edge
constexpr int SW_ROWS = 8;      // thread rows: 32 x 8 threads, 4 elements each per tile

// Tile pair (I, J), I >= J, of the triangle index t = I (I + 1) / 2 + J.
__device__ inline void tile_of(long long t, int &I, int &J)
{
    int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(r + 1) * (r + 2) / 2 <= t) ++r;
    while ((long long)r * (r + 1) / 2 > t) --r;
    I = r;
    J = (int)(t - (long long)r * (r + 1) / 2);
}

// Swap A(i, j) <-> A(j, i) (conjugated when CONJ) for every i != j of one
// tile pair.  Each tile goes through shared memory so that both the loads
// and the stores run down columns (coalesced).
template <typename T, bool CONJ>
__device__ inline void swap_pair(int n, T *A, i64 lda, int I, int J, T (*s1)[SW_T + 1], T (*s2)[SW_T + 1])
{
    const int tx = threadIdx.x & (SW_T - 1), ty = threadIdx.x / SW_T;
    const int r1 = I * SW_T, c1 = J * SW_T;          // tile 1: rows of I, columns of J (lower)
    // load tile 1 (lower) and tile 2 (its mirror, upper)
    for (int k = ty; k < SW_T; k += SW_ROWS) {
        const int i = r1 + tx, j = c1 + k;
        if (i < n && j < n) s1[k][tx] = A[(i64)j * lda + i];      // s1[col][row]
        const int i2 = c1 + tx, j2 = r1 + k;
        if (i2 < n && j2 < n) s2[k][tx] = A[(i64)j2 * lda + i2];  // s2[col][row]
    }
    __syncthreads();
    for (int k = ty; k < SW_T; k += SW_ROWS) {
        // tile 1 element (r1 + tx, c1 + k) := old A(c1 + k, r1 + tx) = s2[tx][k];
        // complex: the diagonal is conjugated too (a triangle's transpose-
        // conjugate; twice is the identity)
        const int i = r1 + tx, j = c1 + k;
        if (i < n && j < n && (CONJ || i != j)) {
            const T v = s2[tx][k];
            A[(i64)j * lda + i] = CONJ ? cj(v) : v;
        }
        // tile 2 element (c1 + tx, r1 + k) := old A(r1 + k, c1 + tx) = s1[tx][k]
        if (I != J) {
            const int i2 = c1 + tx, j2 = r1 + k;
            if (i2 < n && j2 < n) {
                const T v = s1[tx][k];
                A[(i64)j2 * lda + i2] = CONJ ? cj(v) : v;
            }
        }
    }
}

template <typename T, bool CONJ>
__global__ void __launch_bounds__(SW_T * SW_ROWS)
k_uplo_swap(int n, T *A, i64 lda)
{
    __shared__ T s1[SW_T][SW_T + 1];
    __shared__ T s2[SW_T][SW_T + 1];
    int I, J;
    tile_of(blockIdx.x, I, J);
    swap_pair<T, CONJ>(n, A, lda, I, J, s1, s2);
}

// Matrices b = blockIdx.y, + gridDim.y, ...; tile pairs beyond a matrix's own
// order skip it.
template <typename T>
__global__ void __launch_bounds__(SW_T * SW_ROWS)
k_uplo_swap_vb(i64 batch, const int32_t *nv, T *const *Av, const int32_t *ldv)
{
    __shared__ T s1[SW_T][SW_T + 1];
    __shared__ T s2[SW_T][SW_T + 1];
    int I, J;
    tile_of(blockIdx.x, I, J);
    for (i64 b = blockIdx.y; b < batch; b += gridDim.y) {
        const int n = nv[b];
        if (n <= 0 || I * SW_T >= n) continue;      // uniform across the block
        swap_pair<T, false>(n, Av[b], (i64)ldv[b], I, J, s1, s2);
        __syncthreads();                            // shared tiles reused by the next matrix
    }
}

}  // namespace

template <typename T>
void uplo_swap(Ctx &c, i64 n, T *A, i64 lda)
{
    if (n <= 1) return;
    const i64 tiles = (n + SW_T - 1) / SW_T;
    Launch L(c, K_TRANS, 0.0, 2.0 * sizeof(T) * (double)n * (double)(n - 1));
    k_uplo_swap<T, is_cplx<T>::value><<<(unsigned)(tiles * (tiles + 1) / 2), SW_T * SW_ROWS, 0, c.s>>>(
        (int)n, A, lda);
}

template <typename T>
void uplo_swap_vbatched(Ctx &c, i64 batch, const int32_t *n, T *const *A, const int32_t *lda, int max_n)
{
    if (batch <= 0 || max_n <= 1) return;
    const i64 tiles = (max_n + SW_T - 1) / SW_T;
    Launch L(c, K_TRANS, 0.0, 0.0);
    const unsigned gy = (unsigned)(batch < 65535 ? batch : 65535);
    k_uplo_swap_vb<T><<<dim3((unsigned)(tiles * (tiles + 1) / 2), gy), SW_T * SW_ROWS, 0, c.s>>>(batch, n, A,
                                                                                                lda);
}

template void uplo_swap<double>(Ctx &, i64, double *, i64);
template void uplo_swap<float>(Ctx &, i64, float *, i64);
template void uplo_swap<cplx>(Ctx &, i64, cplx *, i64);
template void uplo_swap_vbatched<double>(Ctx &, i64, const int32_t *, double *const *, const int32_t *, int);
template void uplo_swap_vbatched<float>(Ctx &, i64, const int32_t *, float *const *, const int32_t *, int);

}  // namespace rl

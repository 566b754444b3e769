// sygst (Section 5, xsygst): reduction of the symmetric-definite generalized
// eigenproblem to standard form with the Cholesky factor L of B (lower):
//   itype 1:    A := L^{-1} A L^{-T}
//   itype 2, 3: A := L^T A L
// A is symmetric with its lower triangle stored; only that triangle is read
// and written.  Recursive by halving (Section 3), with A = [A11 .; A21 A22]
// and L = [L11 0; L21 L22]:
//
//   itype 1                               itype 2
//   A11 := sygst(A11, L11)                A11 := sygst(A11, L11)
//   A21 := A21 L11^{-T}        (TRSM)     T   := A22 L21             (SYMM)
//   T   := L21 A11             (SYMM)     A21 := A21 L11             (TRMM)
//   A21 -= T / 2                          A21 += T / 2
//   A22 -= A21 L21^T + L21 A21^T (2 GEMM) A11 += L21^T A21 + A21^T L21 (2 GEMM)
//   A21 -= T / 2                          A21 += T / 2
//   A21 := L22^{-1} A21        (TRSM)     A21 := L22^T A21           (TRMM)
//   A22 := sygst(A22, L22)                A22 := sygst(A22, L22)
//
// T is the paper's n/2 x n/2 buffer (Section 5, xsygst user note): the
// symmetric product is formed once and used twice.  Without a workspace the
// product is recomputed in place instead (one more SYMM per level).
//
// Base case (order <= 64): one CTA, A mirrored to a full square and L in
// shared memory; itype 1 does two substitutions (down each column, then
// along each row), itype 2 two products (each row times L, then L^T times
// each column), all in place.
#include "internal.cuh"

namespace rl {

namespace {

constexpr int SG_N = 64;
constexpr int SG_P = SG_N + 1;

template <typename T, int ITYPE>
__global__ void __launch_bounds__(SG_N)
k_sygs2(int n, T *A, i64 lda, const T *L, i64 ldl, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ __align__(16) unsigned char sg_raw[];
    T *W = reinterpret_cast<T *>(sg_raw);   // W(i, k) at W[k * SG_P + i]
    T *Ls = W + SG_N * SG_P;                // L(i, k) at Ls[k * SG_P + i]
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e % n, k = e / n;
        W[k * SG_P + i] = (i >= k) ? A[(i64)k * lda + i] : A[(i64)i * lda + k];
        Ls[k * SG_P + i] = (i >= k) ? L[(i64)k * ldl + i] : T(0);
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (ITYPE == 1) {
        // V := L^{-1} W, thread t takes column t (in place)
        if (t < n) {
            T *w = W + t * SG_P;
            for (int i = 0; i < n; ++i) {
                T s = w[i];
                for (int k = 0; k < i; ++k) s = fma(-Ls[k * SG_P + i], w[k], s);
                w[i] = s / Ls[i * SG_P + i];
            }
        }
        __syncthreads();
        // X := V L^{-T}, thread t takes row t: x_j = (v_j - sum_{k<j} x_k l_jk) / l_jj
        if (t < n) {
            for (int j = 0; j < n; ++j) {
                T s = W[j * SG_P + t];
                for (int k = 0; k < j; ++k) s = fma(-W[k * SG_P + t], Ls[k * SG_P + j], s);
                W[j * SG_P + t] = s / Ls[j * SG_P + j];
            }
        }
    } else {
        // V := W L, thread t takes row t: v_j = sum_{k>=j} w_k l_kj, j ascending (in place)
        if (t < n) {
            for (int j = 0; j < n; ++j) {
                T s = T(0);
                for (int k = j; k < n; ++k) s = fma(W[k * SG_P + t], Ls[j * SG_P + k], s);
                W[j * SG_P + t] = s;
            }
        }
        __syncthreads();
        // X := L^T V, thread t takes column t: x_i = sum_{k>=i} l_ki v_k, i ascending
        if (t < n) {
            T *v = W + t * SG_P;
            for (int i = 0; i < n; ++i) {
                T s = T(0);
                for (int k = i; k < n; ++k) s = fma(Ls[i * SG_P + k], v[k], s);
                v[i] = s;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e % n, k = e / n;
        if (i >= k) A[(i64)k * lda + i] = W[k * SG_P + i];
    }
}

// Y(m x n) += alpha X(m x n)
template <typename T>
__global__ void k_axpy_mat(i64 m, i64 n, T alpha, const T *X, i64 ldx, T *Y, i64 ldy, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 total = m * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % m, j = e / m;
        Y[j * ldy + i] += alpha * X[j * ldx + i];
    }
}

template <typename T>
void axpy_mat(Ctx &c, i64 m, i64 n, T alpha, const T *X, i64 ldx, T *Y, i64 ldy)
{
    if (m <= 0 || n <= 0) return;
    Launch L(c, K_MIX, 2.0 * m * n, 3.0 * sizeof(T) * m * n);
    const i64 blocks = (m * n + 255) / 256;
    const unsigned grid = (unsigned)(blocks < (i64)c.num_sms * 16 ? blocks : (i64)c.num_sms * 16);
    k_axpy_mat<T><<<grid, 256, 0, c.s>>>(m, n, alpha, X, ldx, Y, ldy, c.abort);
}

template <typename T>
void sygs2(Ctx &c, int itype, i64 n, T *A, i64 lda, const T *L, i64 ldl)
{
    const size_t smem = 2 * (size_t)SG_N * SG_P * sizeof(T);
    note(c, smem_optin(itype == 1 ? k_sygs2<T, 1> : k_sygs2<T, 2>, smem));
    Launch Lk(c, K_MIX, (double)n * n * n, 0.0);
    if (itype == 1) k_sygs2<T, 1><<<1, SG_N, smem, c.s>>>((int)n, A, lda, L, ldl, c.abort);
    else k_sygs2<T, 2><<<1, SG_N, smem, c.s>>>((int)n, A, lda, L, ldl, c.abort);
}

}  // namespace

size_t sygst_work_bytes(i64 n, size_t esz)
{
    if (n <= SG_N) return 0;
    const i64 n1 = split_q(n, SG_N), n2 = n - n1;
    return (size_t)n1 * (size_t)n2 * esz;
}

template <typename E>
void sygst_rec(Ctx &c, int itype, i64 n, E *A, i64 lda, const E *L, i64 ldl, E *T)
{
    if (n <= 0) return;
    if (n <= SG_N) {
        sygs2<E>(c, itype, n, A, lda, L, ldl);
        return;
    }
    const i64 n1 = split_q(n, SG_N), n2 = n - n1;
    E *A11 = A, *A21 = A + n1, *A22 = A + n1 + n1 * lda;
    const E *L11 = L, *L21 = L + n1, *L22 = L + n1 + n1 * ldl;
    const i64 ldt = n2;
    if (itype == 1) {
        sygst_rec<E>(c, 1, n1, A11, lda, L11, ldl, T);
        trsm_rlt<E>(c, n2, n1, E(1), L11, ldl, A21, lda);
        if (T) {
            symm<E>(c, false, n2, n1, E(1), A11, lda, L21, ldl, E(0), T, ldt);
            axpy_mat<E>(c, n2, n1, E(-0.5), T, ldt, A21, lda);
        } else {
            symm<E>(c, false, n2, n1, E(-0.5), A11, lda, L21, ldl, E(1), A21, lda);
        }
        gemm<E>(c, false, true, n2, n2, n1, E(-1), A21, lda, L21, ldl, E(1), A22, lda, true);
        gemm<E>(c, false, true, n2, n2, n1, E(-1), L21, ldl, A21, lda, E(1), A22, lda, true);
        if (T) axpy_mat<E>(c, n2, n1, E(-0.5), T, ldt, A21, lda);
        else symm<E>(c, false, n2, n1, E(-0.5), A11, lda, L21, ldl, E(1), A21, lda);
        trsm_lln<E>(c, false, n2, n1, E(1), L22, ldl, A21, lda);
        sygst_rec<E>(c, 1, n2, A22, lda, L22, ldl, T);
    } else {
        sygst_rec<E>(c, itype, n1, A11, lda, L11, ldl, T);
        if (T) symm<E>(c, true, n2, n1, E(1), A22, lda, L21, ldl, E(0), T, ldt);
        trmm_rln<E>(c, false, n2, n1, E(1), L11, ldl, A21, lda);
        if (T) axpy_mat<E>(c, n2, n1, E(0.5), T, ldt, A21, lda);
        else symm<E>(c, true, n2, n1, E(0.5), A22, lda, L21, ldl, E(1), A21, lda);
        gemm<E>(c, true, false, n1, n1, n2, E(1), L21, ldl, A21, lda, E(1), A11, lda, true);
        gemm<E>(c, true, false, n1, n1, n2, E(1), A21, lda, L21, ldl, E(1), A11, lda, true);
        if (T) axpy_mat<E>(c, n2, n1, E(0.5), T, ldt, A21, lda);
        else symm<E>(c, true, n2, n1, E(0.5), A22, lda, L21, ldl, E(1), A21, lda);
        trmm_llt<E>(c, n2, n1, E(1), L22, ldl, A21, lda);
        sygst_rec<E>(c, itype, n2, A22, lda, L22, ldl, T);
    }
}

template void sygst_rec<double>(Ctx &, int, i64, double *, i64, const double *, i64, double *);
template void sygst_rec<float>(Ctx &, int, i64, float *, i64, const float *, i64, float *);

}  // namespace rl

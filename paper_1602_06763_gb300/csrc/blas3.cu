// BLAS-3 layer of the recursive factorizations: an FP64 GEMM/SYRK kernel and
// recursive TRSM/TRMM that send almost all of their flops to it.
//
// The paper's algorithms (Section 3) spend >99 % of their flops in BLAS-3
// calls of the top recursion levels (Fig. 5).  On GB300 binary64 arithmetic
// runs on the FP64 pipe (there is no tcgen05 kind for f64), which is narrow
// compared with the memory system: a 64x64 CTA tile reads 16 bytes of
// operands per 32 FMAs, far below what L2 and HBM deliver.  The kernels are
// therefore organised for FP64 issue efficiency and load balance (small
// tiles, many CTAs), not for bandwidth.
//
// TRSM and TRMM follow the same halving scheme as the factorizations: the
// triangle is split in two, the off-diagonal update is a GEMM, and blocks of
// order <= 64 are solved in shared memory by substitution (IEEE division; no
// explicit inverse, in line with the stability argument of Section 3's
// footnote on the TRTRI variant).
#include "internal.cuh"

namespace rl {

// ----------------------------------------------------------------------------
// GEMM: C = beta*C + alpha*op(A) op(B); LOWER: only tiles with tm >= tn are
// launched (square C) and only elements i >= j are stored.
// 256 threads as 16x16; thread (tx,ty) owns rows tx+16i, columns ty+16j.
// ----------------------------------------------------------------------------
template <bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(256)
k_dgemm(i64 m, i64 n, i64 k, double alpha, const double *__restrict__ A, i64 lda,
        const double *__restrict__ B, i64 ldb, double beta, double *C, i64 ldc,
        const int32_t *abort, int tiles_m)
{
    if (abort && *abort != 0) return;
    int tm, tn;
    if (LOWER) {
        // row-major enumeration of the lower tile triangle: t = tm(tm+1)/2 + tn
        long long t = blockIdx.x;
        int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((long long)(r + 1) * (r + 2) / 2 <= t) ++r;
        while ((long long)r * (r + 1) / 2 > t) --r;
        tm = r;
        tn = (int)(t - (long long)r * (r + 1) / 2);
    } else {
        tm = blockIdx.x % tiles_m;
        tn = blockIdx.x / tiles_m;
    }
    const i64 i0 = (i64)tm * GEMM_BM, j0 = (i64)tn * GEMM_BN;

    __shared__ double As[2][GEMM_BK][GEMM_BM + 1];
    __shared__ double Bs[2][GEMM_BK][GEMM_BN + 1];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    double ra[4], rb[4];
    auto load = [&](i64 k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int il, pl;
            if (!TA) { il = tid & 63; pl = (tid >> 6) + 4 * r; }
            else     { pl = tid & 15; il = (tid >> 4) + 16 * r; }
            i64 gi = i0 + il, gp = k0 + pl;
            double v = 0.0;
            if (gi < m && gp < k) v = TA ? __ldg(A + gi * lda + gp) : __ldg(A + gp * lda + gi);
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jl, pl;
            if (!TB) { pl = tid & 15; jl = (tid >> 4) + 16 * r; }
            else     { jl = tid & 63; pl = (tid >> 6) + 4 * r; }
            i64 gj = j0 + jl, gp = k0 + pl;
            double v = 0.0;
            if (gj < n && gp < k) v = TB ? __ldg(B + gp * ldb + gj) : __ldg(B + gj * ldb + gp);
            rb[r] = v;
        }
    };
    auto store = [&](int st) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int il, pl;
            if (!TA) { il = tid & 63; pl = (tid >> 6) + 4 * r; }
            else     { pl = tid & 15; il = (tid >> 4) + 16 * r; }
            As[st][pl][il] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jl, pl;
            if (!TB) { pl = tid & 15; jl = (tid >> 4) + 16 * r; }
            else     { jl = tid & 63; pl = (tid >> 6) + 4 * r; }
            Bs[st][pl][jl] = rb[r];
        }
    };

    const i64 nk = (k + GEMM_BK - 1) / GEMM_BK;
    if (nk > 0) {
        load(0);
        store(0);
        __syncthreads();
        for (i64 t = 0; t < nk; ++t) {
            const int st = (int)(t & 1);
            if (t + 1 < nk) load((t + 1) * GEMM_BK);
#pragma unroll
            for (int kk = 0; kk < GEMM_BK; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[st][kk][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[st][kk][ty + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            if (t + 1 < nk) store(st ^ 1);
            __syncthreads();
        }
    }

#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const i64 col = j0 + ty + 16 * j;
        if (col >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const i64 row = i0 + tx + 16 * i;
            if (row >= m) continue;
            if (LOWER && row < col) continue;
            double *cp = C + col * ldc + row;
            double cv = (beta == 0.0) ? 0.0 : beta * (*cp);
            *cp = fma(alpha, acc[i][j], cv);
        }
    }
}

template <bool TA, bool TB, bool LOWER>
static void launch_gemm(Ctx &c, i64 m, i64 n, i64 k, double alpha, const double *A,
                        i64 lda, const double *B, i64 ldb, double beta, double *C, i64 ldc)
{
    const i64 tiles_m = (m + GEMM_BM - 1) / GEMM_BM, tiles_n = (n + GEMM_BN - 1) / GEMM_BN;
    i64 grid = LOWER ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    if (grid <= 0) return;
    const double flops = LOWER ? (double)k * (double)n * (double)(n + 1) : 2.0 * m * n * k;
    Launch L(c, LOWER ? K_SYRK : K_GEMM, flops, 0.0);
    k_dgemm<TA, TB, LOWER><<<(unsigned)grid, 256, 0, c.s>>>(
        m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, c.abort, (int)tiles_m);
}

void gemm(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, double alpha, const double *A,
          i64 lda, const double *B, i64 ldb, double beta, double *C, i64 ldc, bool lower)
{
    if (m <= 0 || n <= 0) return;
    if (k <= 0 && beta == 1.0) return;
    if (lower) {
        if (!ta && tb) launch_gemm<false, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (ta && !tb) launch_gemm<true, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (!ta && !tb) launch_gemm<false, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else launch_gemm<true, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        return;
    }
    if (!ta && !tb) launch_gemm<false, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) launch_gemm<false, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) launch_gemm<true, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else launch_gemm<true, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

// ----------------------------------------------------------------------------
// Triangle (order <= 64) staged in shared memory, packed by rows:
// l_ik (k <= i) at Lp[i(i+1)/2 + k].
// ----------------------------------------------------------------------------
constexpr int TRI_PACK = TRX_NB * (TRX_NB + 1) / 2;
constexpr int BASE_COLS = 32;   // columns (or rows) of B per CTA in base kernels

__device__ __forceinline__ int tri_ix(int i, int k) { return i * (i + 1) / 2 + k; }

__device__ __forceinline__ void load_tri(double *Lp, const double *L, i64 ldl, int nt)
{
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        int i = e % nt, k = e / nt;
        if (i >= k) Lp[tri_ix(i, k)] = L[(i64)k * ldl + i];
    }
}

// B(m x n) := alpha * L^{-1} B, m <= 64; one thread per column of B.
template <bool UNIT>
__global__ void __launch_bounds__(BASE_COLS)
k_trsm_lln_base(int m, i64 n, double alpha, const double *__restrict__ L, i64 ldl,
                double *B, i64 ldb, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Lp[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];
    const i64 c0 = (i64)blockIdx.x * BASE_COLS;
    const int nc = (int)min((i64)BASE_COLS, n - c0);
    load_tri(Lp, L, ldl, m);
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, j = e / m;
        Bs[i][j] = B[(c0 + j) * ldb + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nc) {
        for (int i = 0; i < m; ++i) {
            double s = alpha * Bs[i][j];
            const double *li = Lp + tri_ix(i, 0);
            for (int k = 0; k < i; ++k) s = fma(-li[k], Bs[k][j], s);
            Bs[i][j] = UNIT ? s : s / li[i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, jj = e / m;
        B[(c0 + jj) * ldb + i] = Bs[i][jj];
    }
}

// B(m x n) := B L^{-T}, n <= 64; one thread per row of B:
// x_j = (b_j - sum_{k<j} x_k l_jk) / l_jj.
__global__ void __launch_bounds__(BASE_COLS)
k_trsm_rlt_base(i64 m, int n, const double *__restrict__ L, i64 ldl, double *B, i64 ldb,
                const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Lp[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];   // Bs[col][row]
    const i64 r0 = (i64)blockIdx.x * BASE_COLS;
    const int nr = (int)min((i64)BASE_COLS, m - r0);
    load_tri(Lp, L, ldl, n);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        int r = e % nr, j = e / nr;
        Bs[j][r] = B[(i64)j * ldb + r0 + r];
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r < nr) {
        for (int j = 0; j < n; ++j) {
            double s = Bs[j][r];
            const double *lj = Lp + tri_ix(j, 0);
            for (int k = 0; k < j; ++k) s = fma(-Bs[k][r], lj[k], s);
            Bs[j][r] = s / lj[j];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        int rr = e % nr, j = e / nr;
        B[(i64)j * ldb + r0 + rr] = Bs[j][rr];
    }
}

// B(m x n) := L^{-T} B, m <= 64; one thread per column (back substitution):
// x_i = (b_i - sum_{k>i} l_ki x_k) / l_ii.
__global__ void __launch_bounds__(BASE_COLS)
k_trsm_llt_base(int m, i64 n, const double *__restrict__ L, i64 ldl, double *B, i64 ldb,
                const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Lp[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];
    const i64 c0 = (i64)blockIdx.x * BASE_COLS;
    const int nc = (int)min((i64)BASE_COLS, n - c0);
    load_tri(Lp, L, ldl, m);
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, j = e / m;
        Bs[i][j] = B[(c0 + j) * ldb + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nc) {
        for (int i = m - 1; i >= 0; --i) {
            double s = Bs[i][j];
            for (int k = i + 1; k < m; ++k) s = fma(-Lp[tri_ix(k, i)], Bs[k][j], s);
            Bs[i][j] = s / Lp[tri_ix(i, i)];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, jj = e / m;
        B[(c0 + jj) * ldb + i] = Bs[i][jj];
    }
}

// B(m x n) := U^{-1} B, U upper m x m (m <= 64); one thread per column:
// x_i = (b_i - sum_{k>i} u_ik x_k) / u_ii.  U staged packed by columns of
// its transpose: u_ik (k >= i) at Up[k(k+1)/2 + i].
__global__ void __launch_bounds__(BASE_COLS)
k_trsm_lun_base(int m, i64 n, const double *__restrict__ U, i64 ldu, double *B, i64 ldb,
                const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Up[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];
    const i64 c0 = (i64)blockIdx.x * BASE_COLS;
    const int nc = (int)min((i64)BASE_COLS, n - c0);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, k = e / m;
        if (k >= i) Up[tri_ix(k, i)] = U[(i64)k * ldu + i];
    }
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, j = e / m;
        Bs[i][j] = B[(c0 + j) * ldb + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nc) {
        for (int i = m - 1; i >= 0; --i) {
            double s = Bs[i][j];
            for (int k = i + 1; k < m; ++k) s = fma(-Up[tri_ix(k, i)], Bs[k][j], s);
            Bs[i][j] = s / Up[tri_ix(i, i)];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, jj = e / m;
        B[(c0 + jj) * ldb + i] = Bs[i][jj];
    }
}

// B(m x n) := B L, n <= 64; one thread per row, in place for ascending j:
// b_j := sum_{k>=j} b_k l_kj (b_k, k >= j, still hold their old values).
template <bool UNIT>
__global__ void __launch_bounds__(BASE_COLS)
k_trmm_rln_base(i64 m, int n, const double *__restrict__ L, i64 ldl, double *B, i64 ldb,
                const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Lp[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];
    const i64 r0 = (i64)blockIdx.x * BASE_COLS;
    const int nr = (int)min((i64)BASE_COLS, m - r0);
    load_tri(Lp, L, ldl, n);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        int r = e % nr, j = e / nr;
        Bs[j][r] = B[(i64)j * ldb + r0 + r];
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r < nr) {
        for (int j = 0; j < n; ++j) {
            double s = UNIT ? Bs[j][r] : Bs[j][r] * Lp[tri_ix(j, j)];
            for (int k = j + 1; k < n; ++k) s = fma(Bs[k][r], Lp[tri_ix(k, j)], s);
            Bs[j][r] = s;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        int rr = e % nr, j = e / nr;
        B[(i64)j * ldb + r0 + rr] = Bs[j][rr];
    }
}

// B(m x n) := L^T B, m <= 64; one thread per column, ascending i in place:
// b_i := sum_{k>=i} l_ki b_k.
__global__ void __launch_bounds__(BASE_COLS)
k_trmm_llt_base(int m, i64 n, const double *__restrict__ L, i64 ldl, double *B, i64 ldb,
                const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ double Lp[TRI_PACK];
    __shared__ double Bs[TRX_NB][BASE_COLS + 1];
    const i64 c0 = (i64)blockIdx.x * BASE_COLS;
    const int nc = (int)min((i64)BASE_COLS, n - c0);
    load_tri(Lp, L, ldl, m);
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, j = e / m;
        Bs[i][j] = B[(c0 + j) * ldb + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nc) {
        for (int i = 0; i < m; ++i) {
            double s = Bs[i][j] * Lp[tri_ix(i, i)];
            for (int k = i + 1; k < m; ++k) s = fma(Lp[tri_ix(k, i)], Bs[k][j], s);
            Bs[i][j] = s;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        int i = e % m, jj = e / m;
        B[(c0 + jj) * ldb + i] = Bs[i][jj];
    }
}

static inline unsigned blocks_for(i64 count) { return (unsigned)((count + BASE_COLS - 1) / BASE_COLS); }

// ----------------------------------------------------------------------------
// Recursive drivers (halving with 64-aligned splits).
// ----------------------------------------------------------------------------
void trsm_lln(Ctx &c, bool unit, i64 m, i64 n, double alpha, const double *L, i64 ldl,
              double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        Launch K(c, K_TRSM, (double)n * m * m, 0.0);
        if (unit) k_trsm_lln_base<true><<<blocks_for(n), BASE_COLS, 0, c.s>>>((int)m, n, alpha, L, ldl, B, ldb, c.abort);
        else k_trsm_lln_base<false><<<blocks_for(n), BASE_COLS, 0, c.s>>>((int)m, n, alpha, L, ldl, B, ldb, c.abort);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_lln(c, unit, m1, n, alpha, L, ldl, B, ldb);
    gemm(c, false, false, m2, n, m1, -1.0, L + m1, ldl, B, ldb, alpha, B + m1, ldb);
    trsm_lln(c, unit, m2, n, 1.0, L + m1 + m1 * ldl, ldl, B + m1, ldb);
}

void trsm_rlt(Ctx &c, i64 m, i64 n, const double *L, i64 ldl, double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (n <= TRX_NB) {
        Launch K(c, K_TRSM, (double)m * n * n, 0.0);
        k_trsm_rlt_base<<<blocks_for(m), BASE_COLS, 0, c.s>>>(m, (int)n, L, ldl, B, ldb, c.abort);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    trsm_rlt(c, m, n1, L, ldl, B, ldb);
    gemm(c, false, true, m, n2, n1, -1.0, B, ldb, L + n1, ldl, 1.0, B + n1 * ldb, ldb);
    trsm_rlt(c, m, n2, L + n1 + n1 * ldl, ldl, B + n1 * ldb, ldb);
}

void trsm_llt(Ctx &c, i64 m, i64 n, const double *L, i64 ldl, double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        Launch K(c, K_TRSM, (double)n * m * m, 0.0);
        k_trsm_llt_base<<<blocks_for(n), BASE_COLS, 0, c.s>>>((int)m, n, L, ldl, B, ldb, c.abort);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_llt(c, m2, n, L + m1 + m1 * ldl, ldl, B + m1, ldb);
    gemm(c, true, false, m1, n, m2, -1.0, L + m1, ldl, B + m1, ldb, 1.0, B, ldb);
    trsm_llt(c, m1, n, L, ldl, B, ldb);
}

void trsm_lun(Ctx &c, i64 m, i64 n, const double *U, i64 ldu, double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        Launch K(c, K_TRSM, (double)n * m * m, 0.0);
        k_trsm_lun_base<<<blocks_for(n), BASE_COLS, 0, c.s>>>((int)m, n, U, ldu, B, ldb, c.abort);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_lun(c, m2, n, U + m1 + m1 * ldu, ldu, B + m1, ldb);
    gemm(c, false, false, m1, n, m2, -1.0, U + m1 * ldu, ldu, B + m1, ldb, 1.0, B, ldb);
    trsm_lun(c, m1, n, U, ldu, B, ldb);
}

void trmm_rln(Ctx &c, bool unit, i64 m, i64 n, const double *L, i64 ldl, double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (n <= TRX_NB) {
        Launch K(c, K_TRMM, (double)m * n * n, 0.0);
        if (unit) k_trmm_rln_base<true><<<blocks_for(m), BASE_COLS, 0, c.s>>>(m, (int)n, L, ldl, B, ldb, c.abort);
        else k_trmm_rln_base<false><<<blocks_for(m), BASE_COLS, 0, c.s>>>(m, (int)n, L, ldl, B, ldb, c.abort);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    trmm_rln(c, unit, m, n1, L, ldl, B, ldb);
    gemm(c, false, false, m, n1, n2, 1.0, B + n1 * ldb, ldb, L + n1, ldl, 1.0, B, ldb);
    trmm_rln(c, unit, m, n2, L + n1 + n1 * ldl, ldl, B + n1 * ldb, ldb);
}

void trmm_llt(Ctx &c, i64 m, i64 n, const double *L, i64 ldl, double *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        Launch K(c, K_TRMM, (double)n * m * m, 0.0);
        k_trmm_llt_base<<<blocks_for(n), BASE_COLS, 0, c.s>>>((int)m, n, L, ldl, B, ldb, c.abort);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trmm_llt(c, m1, n, L, ldl, B, ldb);
    gemm(c, true, false, m1, n, m2, 1.0, L + m1, ldl, B + m1, ldb, 1.0, B, ldb);
    trmm_llt(c, m2, n, L + m1 + m1 * ldl, ldl, B + m1, ldb);
}

}  // namespace rl

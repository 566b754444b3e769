// BLAS-3 layer of the recursive factorizations: a GEMM/SYRK kernel and
// recursive TRSM/TRMM that send almost all of their flops to it.  Templated
// on the element type: double for the FP64 path, float for the FP32 storage
// of the precision form.
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
// SYM: 0 plain operands; 1: A is symmetric with its lower triangle stored
// (element (i, p) read from (max, min)); 2: the same for B.  Used by SYMM.
template <typename T, bool TA, bool TB, bool LOWER, int SYM = 0>
__global__ void __launch_bounds__(256)
k_gemm(i64 m, i64 n, i64 k, T alpha, const T *__restrict__ A, i64 lda,
       const T *__restrict__ B, i64 ldb, T beta, T *C, i64 ldc,
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

    __shared__ T As[2][GEMM_BK][GEMM_BM + 1];
    __shared__ T Bs[2][GEMM_BK][GEMM_BN + 1];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    T ra[4], rb[4];
    auto load = [&](i64 k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int il, pl;
            if (!TA) { il = tid & 63; pl = (tid >> 6) + 4 * r; }
            else     { pl = tid & 15; il = (tid >> 4) + 16 * r; }
            i64 gi = i0 + il, gp = k0 + pl;
            T v = T(0);
            if (gi < m && gp < k) {
                if (SYM == 1) v = (gi >= gp) ? __ldg(A + gp * lda + gi) : __ldg(A + gi * lda + gp);
                else v = TA ? __ldg(A + gi * lda + gp) : __ldg(A + gp * lda + gi);
            }
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jl, pl;
            if (!TB) { pl = tid & 15; jl = (tid >> 4) + 16 * r; }
            else     { jl = tid & 63; pl = (tid >> 6) + 4 * r; }
            i64 gj = j0 + jl, gp = k0 + pl;
            T v = T(0);
            if (gj < n && gp < k) {
                if (SYM == 2) v = (gp >= gj) ? __ldg(B + gj * ldb + gp) : __ldg(B + gp * ldb + gj);
                else v = TB ? __ldg(B + gp * ldb + gj) : __ldg(B + gj * ldb + gp);
            }
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
                T a[4], b[4];
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
            T *cp = C + col * ldc + row;
            T cv = (beta == T(0)) ? T(0) : beta * (*cp);
            *cp = fma(alpha, acc[i][j], cv);
        }
    }
}

// Algorithmic bytes of one GEMM/SYRK call: each operand read once, C read
// and written once (the lower triangle only for SYRK).
static double gemm_bytes(i64 m, i64 n, i64 k, bool lower, size_t esz)
{
    const double c_elems = lower ? (double)n * (double)(n + 1) / 2.0 : (double)m * (double)n;
    const double ab = lower ? (double)n * (double)k : (double)m * (double)k + (double)k * (double)n;
    return (ab + 2.0 * c_elems) * (double)esz;
}

template <typename T, bool TA, bool TB, bool LOWER>
static void launch_gemm(Ctx &c, i64 m, i64 n, i64 k, T alpha, const T *A, i64 lda, const T *B,
                        i64 ldb, T beta, T *C, i64 ldc)
{
    const i64 tiles_m = (m + GEMM_BM - 1) / GEMM_BM, tiles_n = (n + GEMM_BN - 1) / GEMM_BN;
    i64 grid = LOWER ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    if (grid <= 0) return;
    const double flops = LOWER ? (double)k * (double)n * (double)(n + 1) : 2.0 * m * n * k;
    Launch L(c, LOWER ? K_SYRK : K_GEMM, flops, gemm_bytes(m, n, k, LOWER, sizeof(T)));
    k_gemm<T, TA, TB, LOWER><<<(unsigned)grid, 256, 0, c.s>>>(
        m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, c.abort, (int)tiles_m);
}

// ----------------------------------------------------------------------------
// Complex GEMM (complex double): 32 x 32 tiles, 256 threads as 16 x 16, each
// thread a 2 x 2 block; TA / TB mean the CONJUGATE transpose; LOWER as above.
// FP64-pipe bound (4 DFMA per complex multiply-add), so small tiles and many
// CTAs.
// ----------------------------------------------------------------------------
constexpr int ZG_B = 32, ZG_K = 16;

template <bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(256)
k_zgemm(i64 m, i64 n, i64 k, cplx alpha, const cplx *__restrict__ A, i64 lda, const cplx *__restrict__ B,
        i64 ldb, cplx beta, cplx *C, i64 ldc, const int32_t *abort, int tiles_m)
{
    if (abort && *abort != 0) return;
    int tm, tn;
    if (LOWER) {
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
    const i64 i0 = (i64)tm * ZG_B, j0 = (i64)tn * ZG_B;
    __shared__ cplx As[2][ZG_K][ZG_B + 1];
    __shared__ cplx Bs[2][ZG_K][ZG_B + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    cplx acc[2][2];
    cplx ra[2], rb[2];
    auto load = [&](i64 k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = tid + 256 * r;                // 512 elements of each 32 x 16 tile
            int il, pl;
            if (!TA) { il = e & 31; pl = e >> 5; } else { pl = e & 15; il = e >> 4; }
            const i64 gi = i0 + il, gp = k0 + pl;
            cplx v(0.0);
            if (gi < m && gp < k) v = TA ? conj(A[gi * lda + gp]) : A[gp * lda + gi];
            ra[r] = v;
            int jl, ql;
            if (!TB) { ql = e & 15; jl = e >> 4; } else { jl = e & 31; ql = e >> 5; }
            const i64 gj = j0 + jl, gq = k0 + ql;
            cplx w(0.0);
            if (gj < n && gq < k) w = TB ? conj(B[gq * ldb + gj]) : B[gj * ldb + gq];
            rb[r] = w;
        }
    };
    auto store = [&](int st) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = tid + 256 * r;
            int il, pl;
            if (!TA) { il = e & 31; pl = e >> 5; } else { pl = e & 15; il = e >> 4; }
            As[st][pl][il] = ra[r];
            int jl, ql;
            if (!TB) { ql = e & 15; jl = e >> 4; } else { jl = e & 31; ql = e >> 5; }
            Bs[st][ql][jl] = rb[r];
        }
    };
    const i64 nk = (k + ZG_K - 1) / ZG_K;
    if (nk > 0) {
        load(0);
        store(0);
        __syncthreads();
        for (i64 t = 0; t < nk; ++t) {
            const int st = (int)(t & 1);
            if (t + 1 < nk) load((t + 1) * ZG_K);
#pragma unroll
            for (int kk = 0; kk < ZG_K; ++kk) {
                const cplx a0 = As[st][kk][tx], a1 = As[st][kk][tx + 16];
                const cplx b0 = Bs[st][kk][ty], b1 = Bs[st][kk][ty + 16];
                acc[0][0] = fma(a0, b0, acc[0][0]);
                acc[0][1] = fma(a0, b1, acc[0][1]);
                acc[1][0] = fma(a1, b0, acc[1][0]);
                acc[1][1] = fma(a1, b1, acc[1][1]);
            }
            if (t + 1 < nk) store(st ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const i64 col = j0 + ty + 16 * j;
        if (col >= n) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const i64 row = i0 + tx + 16 * i;
            if (row >= m) continue;
            if (LOWER && row < col) continue;
            cplx *cp = C + col * ldc + row;
            const cplx cv = (beta == cplx(0.0)) ? cplx(0.0) : beta * (*cp);
            *cp = fma(alpha, acc[i][j], cv);
        }
    }
}

template <bool TA, bool TB, bool LOWER>
static void launch_zgemm(Ctx &c, i64 m, i64 n, i64 k, cplx alpha, const cplx *A, i64 lda, const cplx *B, i64 ldb,
                         cplx beta, cplx *C, i64 ldc)
{
    const i64 tiles_m = (m + ZG_B - 1) / ZG_B, tiles_n = (n + ZG_B - 1) / ZG_B;
    const i64 grid = LOWER ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    const double flops = 4.0 * (LOWER ? (double)k * (double)n * (double)(n + 1) : 2.0 * m * n * k);
    const double c_elems = LOWER ? (double)n * (double)(n + 1) / 2.0 : (double)m * (double)n;
    const double bytes = 16.0 * ((LOWER ? (double)n * k : (double)m * k + (double)k * n) + 2.0 * c_elems);
    Launch L(c, LOWER ? K_SYRK : K_GEMM, flops, bytes);
    k_zgemm<TA, TB, LOWER><<<(unsigned)grid, 256, 0, c.s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, c.abort,
                                                            (int)tiles_m);
}

static void zgemm(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, cplx alpha, const cplx *A, i64 lda,
                  const cplx *B, i64 ldb, cplx beta, cplx *C, i64 ldc, bool lower)
{
    if (lower) {
        if (!ta && tb) launch_zgemm<false, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (ta && !tb) launch_zgemm<true, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (!ta && !tb) launch_zgemm<false, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else launch_zgemm<true, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        return;
    }
    if (!ta && !tb) launch_zgemm<false, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) launch_zgemm<false, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) launch_zgemm<true, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else launch_zgemm<true, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

// ----------------------------------------------------------------------------
// FP32 SIMT GEMM with 128 x 128 CTA tiles (the FP32 updates of the precision
// form).  FP32 FMAs issue 64x faster than FP64 ones, so the 64 x 64 tile
// above becomes shared-memory bound; here each of the 256 threads owns an
// 8 x 8 block (rows 4tx..4tx+3 and 64+4tx.., columns 4ty.. and 64+4ty..),
// read as float4 from k-major tiles: 4 shared loads per 64 FMAs.
// ----------------------------------------------------------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

template <bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(256)
k_sgemm128(i64 m, i64 n, i64 k, float alpha, const float *__restrict__ A, i64 lda,
           const float *__restrict__ B, i64 ldb, float beta, float *C, i64 ldc,
           const int32_t *abort, int tiles_m)
{
    if (abort && *abort != 0) return;
    int tm, tn;
    if (LOWER) {
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
    const i64 i0 = (i64)tm * SG_BM, j0 = (i64)tn * SG_BN;
    // rows padded by 4 floats: the k-contiguous staging stores (8 k-values x 4
    // rows per warp) then hit 32 distinct banks; rows stay 16-byte aligned
    __shared__ __align__(16) float As[2][SG_BK][SG_BM + 4];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    // global -> register staging: 4 elements of A and 4 of B per thread
    float ra[4], rb[4];
    auto load = [&](i64 k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int il, pl;
            if (!TA) { il = tid & 127; pl = (tid >> 7) + 2 * r; }      // column-major A: rows contiguous
            else     { pl = tid & 7; il = (tid >> 3) + 32 * r; }        // A^T: k contiguous
            const i64 gi = i0 + il, gp = k0 + pl;
            float v = 0.0f;
            if (gi < m && gp < k) v = TA ? __ldg(A + gi * lda + gp) : __ldg(A + gp * lda + gi);
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jl, pl;
            if (!TB) { pl = tid & 7; jl = (tid >> 3) + 32 * r; }        // B: k contiguous
            else     { jl = tid & 127; pl = (tid >> 7) + 2 * r; }       // B^T: columns contiguous
            const i64 gj = j0 + jl, gp = k0 + pl;
            float v = 0.0f;
            if (gj < n && gp < k) v = TB ? __ldg(B + gp * ldb + gj) : __ldg(B + gj * ldb + gp);
            rb[r] = v;
        }
    };
    auto store = [&](int st) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int il, pl;
            if (!TA) { il = tid & 127; pl = (tid >> 7) + 2 * r; }
            else     { pl = tid & 7; il = (tid >> 3) + 32 * r; }
            As[st][pl][il] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jl, pl;
            if (!TB) { pl = tid & 7; jl = (tid >> 3) + 32 * r; }
            else     { jl = tid & 127; pl = (tid >> 7) + 2 * r; }
            Bs[st][pl][jl] = rb[r];
        }
    };

    const i64 nk = (k + SG_BK - 1) / SG_BK;
    if (nk > 0) {
        load(0);
        store(0);
        __syncthreads();
        for (i64 t = 0; t < nk; ++t) {
            const int st = (int)(t & 1);
            if (t + 1 < nk) load((t + 1) * SG_BK);
#pragma unroll
            for (int kk = 0; kk < SG_BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[st][kk][4 * tx]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[st][kk][64 + 4 * tx]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[st][kk][4 * ty]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[st][kk][64 + 4 * ty]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (t + 1 < nk) store(st ^ 1);
            __syncthreads();
        }
    }

#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const i64 col = j0 + (j < 4 ? 4 * ty + j : 64 + 4 * ty + (j - 4));
        if (col >= n) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const i64 row = i0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + (i - 4));
            if (row >= m) continue;
            if (LOWER && row < col) continue;
            float *cp = C + col * ldc + row;
            const float cv = (beta == 0.0f) ? 0.0f : beta * (*cp);
            *cp = fmaf(alpha, acc[i][j], cv);
        }
    }
}

template <bool TA, bool TB, bool LOWER>
static void launch_sgemm128(Ctx &c, i64 m, i64 n, i64 k, float alpha, const float *A, i64 lda,
                            const float *B, i64 ldb, float beta, float *C, i64 ldc)
{
    const i64 tiles_m = (m + SG_BM - 1) / SG_BM, tiles_n = (n + SG_BN - 1) / SG_BN;
    const i64 grid = LOWER ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    const double flops = LOWER ? (double)k * (double)n * (double)(n + 1) : 2.0 * m * n * k;
    Launch L(c, LOWER ? K_SYRK : K_GEMM, flops, gemm_bytes(m, n, k, LOWER, sizeof(float)));
    k_sgemm128<TA, TB, LOWER><<<(unsigned)grid, 256, 0, c.s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                                                c.abort, (int)tiles_m);
}

// The 128-tile kernel pays off once it still gives every SM a CTA.
static bool sgemm128_fits(Ctx &c, i64 m, i64 n, bool lower)
{
    const i64 tm = (m + SG_BM - 1) / SG_BM, tn = (n + SG_BN - 1) / SG_BN;
    const i64 tiles = lower ? tm * (tm + 1) / 2 : tm * tn;
    return tiles >= c.num_sms;
}

template <typename T>
static bool gemm_f32_wide(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, T alpha, const T *A, i64 lda,
                          const T *B, i64 ldb, T beta, T *C, i64 ldc, bool lower)
{
    if (sizeof(T) != 4 || !sgemm128_fits(c, m, n, lower)) return false;
    const float *a = reinterpret_cast<const float *>(A), *b = reinterpret_cast<const float *>(B);
    float *cc = reinterpret_cast<float *>(C);
    const float al = (float)alpha, be = (float)beta;
    if (lower) {
        if (!ta && tb) launch_sgemm128<false, true, true>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
        else if (ta && !tb) launch_sgemm128<true, false, true>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
        else if (!ta && !tb) launch_sgemm128<false, false, true>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
        else launch_sgemm128<true, true, true>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
        return true;
    }
    if (!ta && !tb) launch_sgemm128<false, false, false>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
    else if (!ta && tb) launch_sgemm128<false, true, false>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
    else if (ta && !tb) launch_sgemm128<true, false, false>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
    else launch_sgemm128<true, true, false>(c, m, n, k, al, a, lda, b, ldb, be, cc, ldc);
    return true;
}

template <typename T>
static void gemm_real(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, T alpha, const T *A, i64 lda,
                      const T *B, i64 ldb, T beta, T *C, i64 ldc, bool lower)
{
    if (sizeof(T) == 4 && c.prec != RL_PREC_FP32 && beta == T(1) && m >= TC_MIN_MN && n >= TC_MIN_MN &&
        k >= TC_MIN_K) {
        if (tc_gemm(c, c.prec, ta, tb, m, n, k, (float)alpha, (const float *)A, lda, (const float *)B, ldb,
                    (float *)C, ldc, lower, c.tcwork, c.tclwork))
            return;
    }
    if (sizeof(T) == 8 && c.oz_slices > 0 && m >= g_params.oz_min && n >= g_params.oz_min &&
        k >= g_params.oz_min) {
        if (oz_gemm(c, c.oz_slices, ta, tb, m, n, k, (double)alpha, (const double *)A, lda, (const double *)B, ldb,
                    (double)beta, (double *)C, ldc, lower, c.ozwork, c.ozlwork))
            return;
    }
    if (gemm_f32_wide<T>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower)) return;
    if (lower) {
        if (!ta && tb) launch_gemm<T, false, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (ta && !tb) launch_gemm<T, true, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else if (!ta && !tb) launch_gemm<T, false, false, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        else launch_gemm<T, true, true, true>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
        return;
    }
    if (!ta && !tb) launch_gemm<T, false, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) launch_gemm<T, false, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) launch_gemm<T, true, false, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    else launch_gemm<T, true, true, false>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

template <typename T>
void gemm(Ctx &c, bool ta, bool tb, i64 m, i64 n, i64 k, T alpha, const T *A, i64 lda,
          const T *B, i64 ldb, T beta, T *C, i64 ldc, bool lower)
{
    if (m <= 0 || n <= 0) return;
    if (k <= 0 && beta == T(1)) return;
    if constexpr (is_cplx<T>::value)
        zgemm(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower);
    else
        gemm_real<T>(c, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower);
}

// C(m x n) := beta C + alpha S Bm (left: S m x m) or alpha Bm S (right:
// S n x n); S symmetric, lower triangle stored.
template <typename T>
void symm(Ctx &c, bool left, i64 m, i64 n, T alpha, const T *S, i64 lds, const T *Bm, i64 ldb, T beta,
          T *C, i64 ldc)
{
    if (m <= 0 || n <= 0) return;
    const i64 k = left ? m : n;
    const i64 tiles_m = (m + GEMM_BM - 1) / GEMM_BM, tiles_n = (n + GEMM_BN - 1) / GEMM_BN;
    Launch L(c, K_GEMM, 2.0 * m * n * k, gemm_bytes(m, n, k, false, sizeof(T)));
    if (left)
        k_gemm<T, false, false, false, 1><<<(unsigned)(tiles_m * tiles_n), 256, 0, c.s>>>(
            m, n, k, alpha, S, lds, Bm, ldb, beta, C, ldc, c.abort, (int)tiles_m);
    else
        k_gemm<T, false, false, false, 2><<<(unsigned)(tiles_m * tiles_n), 256, 0, c.s>>>(
            m, n, k, alpha, Bm, ldb, S, lds, beta, C, ldc, c.abort, (int)tiles_m);
}

// ----------------------------------------------------------------------------
// Triangle kernels for blocks of order <= 64 (the leaves of the TRSM/TRMM
// recursion).  Each vector of B (a row or a column, depending on the side)
// is owned by a group of 4 consecutive lanes; lane q of the group holds the
// elements e = q, q+4, q+8, ... in registers.  The triangle is staged in
// shared memory, packed by rows, padded to the template order NB with an
// identity block, so every loop has a compile-time trip count.
//
//   FWD  (forward substitution)  x_j /= d_j, then x_k -= x_j M(k,j), k > j
//        serves B L^{-T} (rows) and L^{-1} B (columns), M = L.
//   BWD  (backward substitution) x_j /= d_j, then x_k -= x_j M(j,k), k < j,
//        for j descending; serves L^{-T} B (M(j,k) = l_jk) and U^{-1} B
//        (M(j,k) = u_kj, the triangle staged transposed).
//   MUL  (in-place product)      b = old x_k; x_k = b d_k; x_j += b M(k,j),
//        j < k, for k ascending; serves B L (rows) and L^T B (columns).
// The right-looking form gives up to NB/4 independent FMAs per lane per step
// and four warps per 32 vectors, enough to keep the FP64 pipes busy.
// ----------------------------------------------------------------------------
constexpr int TRI_THREADS = 128;       // 32 vectors x 4 lanes
constexpr int TRI_VECS = TRI_THREADS / 4;
enum TriOp { TRI_FWD = 0, TRI_BWD = 1, TRI_MUL = 2 };

__device__ __forceinline__ int tri_ix(int i, int k) { return i * (i + 1) / 2 + k; }

// One element global -> shared without a register round trip; src_ok false
// fills the element with zero bytes (src is then not read).  The copies of
// a thread land once it passes tri_copies_wait.
template <typename T>
__device__ __forceinline__ void tri_copy(T *dst, const T *src, bool src_ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "n"((int)sizeof(T)), "r"(src_ok ? (int)sizeof(T) : 0)
                 : "memory");
}

__device__ __forceinline__ void tri_copies_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage the order-n triangle of Tm (lower if !TRANS_UPPER, else the upper
// triangle stored transposed) into P, padded with identity up to NB.
template <typename T, int NB, bool TRANS_UPPER, bool CONJ = false>
__device__ __forceinline__ void stage_tri(T *P, const T *Tm, i64 ldt, int n, bool unit)
{
    constexpr int PER = (NB * NB + TRI_THREADS - 1) / TRI_THREADS;
    if constexpr (!is_cplx<T>::value) {
        // real types: every element in flight at once (cp.async, zero-filled
        // outside the stored triangle), then each thread sets the unit
        // diagonal entries of its own elements
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int i = e % NB, k = e / NB;
            if (e < NB * NB && i >= k) {
                const bool ld = i < n && k < n && !(unit && i == k);
                tri_copy(&P[tri_ix(i, k)], ld ? (TRANS_UPPER ? Tm + (i64)i * ldt + k : Tm + (i64)k * ldt + i) : Tm,
                         ld);
            }
        }
        tri_copies_wait();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int i = e % NB, k = e / NB;
            if (e < NB * NB && i == k && (unit || i >= n)) P[tri_ix(i, k)] = T(1);
        }
    } else {
        // complex: all loads into registers before the first store
        T v[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int i = e % NB, k = e / NB;
            v[r] = T(0);
            if (e < NB * NB && i >= k) {
                if (i < n && k < n) v[r] = TRANS_UPPER ? Tm[(i64)i * ldt + k] : Tm[(i64)k * ldt + i];
                else v[r] = (i == k) ? T(1) : T(0);
            }
        }
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int i = e % NB, k = e / NB;
            if (e < NB * NB && i >= k) {
                T w = (unit && i == k) ? T(1) : v[r];
                P[tri_ix(i, k)] = CONJ ? cj(w) : w;
            }
        }
    }
}

template <typename T, int NB, int OP, bool ROWS, bool UNIT, bool TRANS_UPPER, bool CONJ = false>
__global__ void __launch_bounds__(TRI_THREADS)
k_tri(i64 nvec, int n, T alpha, const T *__restrict__ Tm, i64 ldt, T *B, i64 ldb,
      const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ T P[NB * (NB + 1) / 2];
    stage_tri<T, NB, TRANS_UPPER, CONJ>(P, Tm, ldt, n, UNIT);
    __syncthreads();
    constexpr int E = NB / 4;
    const int q = threadIdx.x & 3;
    const int gbase = threadIdx.x & 28;              // first lane of this group
    const i64 v = (i64)blockIdx.x * TRI_VECS + (threadIdx.x >> 2);
    const bool live = v < nvec;
    T x[E];
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int e = 4 * t + q;
        T b = T(0);
        if (live && e < n) b = ROWS ? B[(i64)e * ldb + v] : B[v * ldb + e];
        x[t] = alpha * b;
    }
    if (OP == TRI_FWD) {
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int s = j >> 2, own = j & 3;
            if (!UNIT && q == own) x[s] = x[s] / P[tri_ix(j, j)];
            const T xj = __shfl_sync(0xffffffffu, x[s], gbase | own);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int k = 4 * t + q;
                if (k > j) x[t] = fma(-xj, P[tri_ix(k, j)], x[t]);
            }
        }
    } else if (OP == TRI_BWD) {
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
            const int s = j >> 2, own = j & 3;
            if (!UNIT && q == own) x[s] = x[s] / P[tri_ix(j, j)];
            const T xj = __shfl_sync(0xffffffffu, x[s], gbase | own);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int k = 4 * t + q;
                if (k < j) x[t] = fma(-xj, P[tri_ix(j, k)], x[t]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int s = k >> 2, own = k & 3;
            const T bk = __shfl_sync(0xffffffffu, x[s], gbase | own);
            if (q == own) x[s] = UNIT ? bk : bk * P[tri_ix(k, k)];
#pragma unroll
            for (int t = 0; t < E; ++t) {
                const int j = 4 * t + q;
                if (j < k) x[t] = fma(bk, P[tri_ix(k, j)], x[t]);
            }
        }
    }
    if (live) {
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int e = 4 * t + q;
            if (e < n) {
                if (ROWS) B[(i64)e * ldb + v] = x[t];
                else B[v * ldb + e] = x[t];
            }
        }
    }
}

// Forward substitution (the TRI_FWD form of k_tri, real types) with a body
// the instruction cache holds: the steps run in a rolled loop over blocks of
// four (j = 4s .. 4s+3), and the lane's elements live in a window that
// shifts by one per block (x[t] holds element 4(s + t) + q), so every
// register index stays a compile-time constant.  An element is final, and
// stored, when its block ends.  The triangle is staged column by column,
// P[j * LDP + k] = M(k, j) (zero above the diagonal and in the LDP - NB
// padding rows), so the reads of one step are immediate offsets from one
// base.  Elements past the order read the padding and are never stored;
// chunks of four window entries wholly past NB are skipped (s is uniform).
// Same operations per element, in the same order, as k_tri (bit-identical).
template <typename T, int NB, bool ROWS, bool UNIT, bool TRANS_UPPER>
__global__ void __launch_bounds__(TRI_THREADS)
k_tri_fwd(i64 nvec, int n, T alpha, const T *__restrict__ Tm, i64 ldt, T *B, i64 ldb, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    constexpr int E = NB / 4, LDP = NB + 16;
    static_assert(E % 4 == 0, "order a multiple of 16");
    __shared__ T P[NB * LDP];
    {
        // every element in flight at once (cp.async, zero-filled outside the
        // stored triangle), then each thread sets the unit diagonal entries
        // of its own elements
        constexpr int PER = NB * LDP / TRI_THREADS;
        static_assert(NB * LDP % TRI_THREADS == 0, "whole rounds");
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int k = e % LDP, j = e / LDP;    // element M(k, j)
            const bool ld = k < n && j < n && k >= j && !(UNIT && k == j);
            tri_copy(&P[e], ld ? (TRANS_UPPER ? Tm + (i64)k * ldt + j : Tm + (i64)j * ldt + k) : Tm, ld);
        }
        tri_copies_wait();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = threadIdx.x + r * TRI_THREADS;
            const int k = e % LDP, j = e / LDP;
            if (k == j && (UNIT || k >= n)) P[e] = T(1);
        }
    }
    __syncthreads();
    const int q = threadIdx.x & 3;
    const int gbase = threadIdx.x & 28;              // first lane of this group
    const i64 v = (i64)blockIdx.x * TRI_VECS + (threadIdx.x >> 2);
    const bool live = v < nvec;
    T x[E];
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int e = 4 * t + q;
        T b = T(0);
        if (live && e < n) b = ROWS ? B[(i64)e * ldb + v] : B[v * ldb + e];
        x[t] = alpha * b;
    }
#pragma unroll 1
    for (int s = 0; s < E; ++s) {
#pragma unroll
        for (int own = 0; own < 4; ++own) {
            const int j = 4 * s + own;
            const T *col = P + j * LDP + 4 * s + q;    // M(4(s + t) + q, j) at col[4t]
            if (!UNIT && q == own) x[0] = x[0] / P[j * LDP + j];
            const T xj = __shfl_sync(0xffffffffu, x[0], gbase | own);
            if (q > own) x[0] = fma(-xj, col[0], x[0]);
#pragma unroll
            for (int c = 0; c < E / 4; ++c) {
                if (s + 4 * c < E) {
#pragma unroll
                    for (int tt = (c == 0 ? 1 : 0); tt < 4; ++tt) {
                        const int t = 4 * c + tt;
                        x[t] = fma(-xj, col[4 * t], x[t]);
                    }
                }
            }
        }
        const int e = 4 * s + q;
        if (live && e < n) {
            if (ROWS) B[(i64)e * ldb + v] = x[0];
            else B[v * ldb + e] = x[0];
        }
#pragma unroll
        for (int t = 0; t + 1 < E; ++t) x[t] = x[t + 1];
    }
}

// Two lanes per vector: lane q of a pair holds elements e = 2t + q in
// registers.  The triangle M (order n, identity-padded to NB) is staged as a
// full square with a padded row stride so that every access in the
// substitution loops is a compile-time offset from a per-lane base:
//   FWD reads M(k, j) for the lane's k: rows interleaved by parity,
//       M(i, k) at (i & 1) * (NB/2) * RS + (i >> 1) * RS + k;
//   BWD and MUL read M(j, k) / M(k, j) along the lane's elements: plain rows,
//       M(i, k) at i * RS + k.
// The loops skip, at compile time, every update that is zero for both lanes;
// only the one element per step that belongs to one lane of the pair is
// predicated.  Operation order per element is that of k_tri, so both
// kernels give bit-identical results.
template <typename T, int NB, int OP, bool ROWS, bool UNIT, bool TRANS_UPPER, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_tri2(i64 nvec, int n, T alpha, const T *__restrict__ Tm, i64 ldt, T *B, i64 ldb, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    constexpr int E = NB / 2, RS = NB + 1;
    __shared__ T S[NB * RS];
    {
        // every element in flight at once (cp.async, zero-filled outside the
        // stored triangle), then each thread sets the unit diagonal entries
        // of its own elements
        constexpr int PER = NB * NB / THREADS;
        static_assert(NB * NB % THREADS == 0, "whole rounds");
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = threadIdx.x + r * THREADS;
            const int k = idx % NB, i = idx / NB;      // element M(i, k)
            const int a = (OP == TRI_FWD) ? ((i & 1) * E * RS + (i >> 1) * RS + k) : (i * RS + k);
            const bool ld = i < n && k < n && k <= i && !(UNIT && i == k);
            tri_copy(&S[a], ld ? (TRANS_UPPER ? Tm + (i64)i * ldt + k : Tm + (i64)k * ldt + i) : Tm, ld);
        }
        tri_copies_wait();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = threadIdx.x + r * THREADS;
            const int k = idx % NB, i = idx / NB;
            const int a = (OP == TRI_FWD) ? ((i & 1) * E * RS + (i >> 1) * RS + k) : (i * RS + k);
            if (i == k && (UNIT || i >= n)) S[a] = T(1);
        }
    }
    __syncthreads();
    const int q = threadIdx.x & 1;
    const int pair = (threadIdx.x & 31) & ~1;
    const i64 v = (i64)blockIdx.x * (THREADS / 2) + (threadIdx.x >> 1);
    const bool live = v < nvec;
    T x[E];
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int e = 2 * t + q;
        T b = T(0);
        if (live && e < n) b = ROWS ? B[(i64)e * ldb + v] : B[v * ldb + e];
        x[t] = alpha * b;
    }
    if (OP == TRI_FWD) {
        const T *Sq = S + q * E * RS;                  // row 2t + q of M at Sq + t * RS
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int s = j >> 1, own = j & 1;
            if (!UNIT && q == own) x[s] = x[s] / Sq[s * RS + j];
            const T xj = __shfl_sync(0xffffffffu, x[s], pair | own);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                if (2 * t > j) x[t] = fma(-xj, Sq[t * RS + j], x[t]);
                else if (2 * t == j && q == 1) x[t] = fma(-xj, Sq[t * RS + j], x[t]);
            }
        }
    } else if (OP == TRI_BWD) {
        const T *Sq = S + q;                           // M(j, 2t + q) at Sq + j * RS + 2t
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
            const int s = j >> 1, own = j & 1;
            if (!UNIT && q == own) x[s] = x[s] / S[j * RS + j];
            const T xj = __shfl_sync(0xffffffffu, x[s], pair | own);
#pragma unroll
            for (int t = 0; t < E; ++t) {
                if (2 * t + 1 < j) x[t] = fma(-xj, Sq[j * RS + 2 * t], x[t]);
                else if (2 * t + 1 == j && q == 0) x[t] = fma(-xj, Sq[j * RS + 2 * t], x[t]);
            }
        }
    } else {
        const T *Sq = S + q;                           // M(k, 2t + q) at Sq + k * RS + 2t
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int s = k >> 1, own = k & 1;
            const T bk = __shfl_sync(0xffffffffu, x[s], pair | own);
            if (q == own) x[s] = UNIT ? bk : bk * S[k * RS + k];
#pragma unroll
            for (int t = 0; t < E; ++t) {
                if (2 * t + 1 < k) x[t] = fma(bk, Sq[k * RS + 2 * t], x[t]);
                else if (2 * t + 1 == k && q == 0) x[t] = fma(bk, Sq[k * RS + 2 * t], x[t]);
            }
        }
    }
    if (live) {
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int e = 2 * t + q;
            if (e < n) {
                if (ROWS) B[(i64)e * ldb + v] = x[t];
                else B[v * ldb + e] = x[t];
            }
        }
    }
}

constexpr i64 TRI2_MIN_VECS = 12288;

template <typename T, int NB, int OP, bool ROWS, bool UNIT, bool TRANS_UPPER>
static void launch_tri2(Ctx &c, i64 nvec, int n, T alpha, const T *Tm, i64 ldt, T *B, i64 ldb)
{
    // 32 vectors per CTA while that leaves fewer than two CTAs per SM of 64, else 64
    if (nvec < (i64)c.num_sms * 2 * 64) {
        const unsigned grid = (unsigned)((nvec + 31) / 32);
        k_tri2<T, NB, OP, ROWS, UNIT, TRANS_UPPER, 64><<<grid, 64, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B, ldb, c.abort);
    } else {
        const unsigned grid = (unsigned)((nvec + 63) / 64);
        k_tri2<T, NB, OP, ROWS, UNIT, TRANS_UPPER, 128><<<grid, 128, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B, ldb, c.abort);
    }
}

// CONJ: stage the conjugated triangle (complex solves with L^H).
template <typename T, int OP, bool ROWS, bool UNIT, bool TRANS_UPPER, bool CONJ = false>
static void launch_tri(Ctx &c, int kind, i64 nvec, int n, T alpha, const T *Tm, i64 ldt, T *B,
                       i64 ldb)
{
    if (nvec <= 0 || n <= 0) return;
    const unsigned grid = (unsigned)((nvec + TRI_VECS - 1) / TRI_VECS);
    Launch L(c, kind, (double)nvec * n * n * (is_cplx<T>::value ? 4.0 : 1.0), 0.0);
    if constexpr (!is_cplx<T>::value) {
        // two lanes per vector halve the FP64 instructions but double each
        // vector's dependent chain: they win only with many vectors in flight
        const int lanes = g_params.tri_lanes ? g_params.tri_lanes : (nvec >= TRI2_MIN_VECS ? 2 : 4);
        if (lanes == 2) {
            if (n <= 16) launch_tri2<T, 16, OP, ROWS, UNIT, TRANS_UPPER>(c, nvec, n, alpha, Tm, ldt, B, ldb);
            else if (n <= 32) launch_tri2<T, 32, OP, ROWS, UNIT, TRANS_UPPER>(c, nvec, n, alpha, Tm, ldt, B, ldb);
            else launch_tri2<T, 64, OP, ROWS, UNIT, TRANS_UPPER>(c, nvec, n, alpha, Tm, ldt, B, ldb);
            return;
        }
        if constexpr (OP == TRI_FWD) {
            if (n <= 16)
                k_tri_fwd<T, 16, ROWS, UNIT, TRANS_UPPER><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B,
                                                                                       ldb, c.abort);
            else if (n <= 32)
                k_tri_fwd<T, 32, ROWS, UNIT, TRANS_UPPER><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B,
                                                                                       ldb, c.abort);
            else
                k_tri_fwd<T, 64, ROWS, UNIT, TRANS_UPPER><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B,
                                                                                       ldb, c.abort);
            return;
        }
    }
    if (n <= 16)
        k_tri<T, 16, OP, ROWS, UNIT, TRANS_UPPER, CONJ><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B, ldb,
                                                                                     c.abort);
    else if (n <= 32)
        k_tri<T, 32, OP, ROWS, UNIT, TRANS_UPPER, CONJ><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B, ldb,
                                                                                     c.abort);
    else
        k_tri<T, 64, OP, ROWS, UNIT, TRANS_UPPER, CONJ><<<grid, TRI_THREADS, 0, c.s>>>(nvec, n, alpha, Tm, ldt, B, ldb,
                                                                                     c.abort);
}

// ----------------------------------------------------------------------------
// Recursive drivers (halving with 64-aligned splits).
// ----------------------------------------------------------------------------
template <typename T>
void trsm_lln(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        if (unit) launch_tri<T, TRI_FWD, false, true, false>(c, K_TRSM, n, (int)m, alpha, L, ldl, B, ldb);
        else launch_tri<T, TRI_FWD, false, false, false>(c, K_TRSM, n, (int)m, alpha, L, ldl, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_lln<T>(c, unit, m1, n, alpha, L, ldl, B, ldb);
    gemm<T>(c, false, false, m2, n, m1, T(-1), L + m1, ldl, B, ldb, alpha, B + m1, ldb);
    trsm_lln<T>(c, unit, m2, n, T(1), L + m1 + m1 * ldl, ldl, B + m1, ldb);
}

template <typename T>
void trsm_rlt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (n <= TRX_NB) {
        // complex: B L^{-H}, each row solves conj(L) y = x
        launch_tri<T, TRI_FWD, true, false, false, is_cplx<T>::value>(c, K_TRSM, m, (int)n, alpha, L, ldl, B, ldb);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    trsm_rlt<T>(c, m, n1, alpha, L, ldl, B, ldb);
    gemm<T>(c, false, true, m, n2, n1, T(-1), B, ldb, L + n1, ldl, alpha, B + n1 * ldb, ldb);
    trsm_rlt<T>(c, m, n2, T(1), L + n1 + n1 * ldl, ldl, B + n1 * ldb, ldb);
}

// B := L^{-T} B (complex: L^{-H}); unit: L's diagonal is taken as 1.
template <typename T>
void trsm_llt_u(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        constexpr bool CJ = is_cplx<T>::value;
        if (unit) launch_tri<T, TRI_BWD, false, true, false, CJ>(c, K_TRSM, n, (int)m, alpha, L, ldl, B, ldb);
        else launch_tri<T, TRI_BWD, false, false, false, CJ>(c, K_TRSM, n, (int)m, alpha, L, ldl, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_llt_u<T>(c, unit, m2, n, alpha, L + m1 + m1 * ldl, ldl, B + m1, ldb);
    gemm<T>(c, true, false, m1, n, m2, T(-1), L + m1, ldl, B + m1, ldb, alpha, B, ldb);
    trsm_llt_u<T>(c, unit, m1, n, T(1), L, ldl, B, ldb);
}

template <typename T>
void trsm_llt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    trsm_llt_u<T>(c, false, m, n, alpha, L, ldl, B, ldb);
}

// B := U^{-T} B, U upper non-unit (forward substitution with U^T, staged
// as a lower triangle by the leaf kernel).
template <typename T>
void trsm_lut(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        launch_tri<T, TRI_FWD, false, false, true>(c, K_TRSM, n, (int)m, alpha, U, ldu, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_lut<T>(c, m1, n, alpha, U, ldu, B, ldb);
    gemm<T>(c, true, false, m2, n, m1, T(-1), U + m1 * ldu, ldu, B, ldb, alpha, B + m1, ldb);
    trsm_lut<T>(c, m2, n, T(1), U + m1 + m1 * ldu, ldu, B + m1, ldb);
}

template <typename T>
void trsm_lun(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        launch_tri<T, TRI_BWD, false, false, true>(c, K_TRSM, n, (int)m, alpha, U, ldu, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trsm_lun<T>(c, m2, n, alpha, U + m1 + m1 * ldu, ldu, B + m1, ldb);
    gemm<T>(c, false, false, m1, n, m2, T(-1), U + m1 * ldu, ldu, B + m1, ldb, alpha, B, ldb);
    trsm_lun<T>(c, m1, n, T(1), U, ldu, B, ldb);
}

template <typename T>
void trmm_rln(Ctx &c, bool unit, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (n <= TRX_NB) {
        if (unit) launch_tri<T, TRI_MUL, true, true, false>(c, K_TRMM, m, (int)n, alpha, L, ldl, B, ldb);
        else launch_tri<T, TRI_MUL, true, false, false>(c, K_TRMM, m, (int)n, alpha, L, ldl, B, ldb);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    trmm_rln<T>(c, unit, m, n1, alpha, L, ldl, B, ldb);
    gemm<T>(c, false, false, m, n1, n2, alpha, B + n1 * ldb, ldb, L + n1, ldl, T(1), B, ldb);
    trmm_rln<T>(c, unit, m, n2, alpha, L + n1 + n1 * ldl, ldl, B + n1 * ldb, ldb);
}

template <typename T>
void trmm_llt(Ctx &c, i64 m, i64 n, T alpha, const T *L, i64 ldl, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        // complex: L^H B
        launch_tri<T, TRI_MUL, false, false, false, is_cplx<T>::value>(c, K_TRMM, n, (int)m, alpha, L, ldl, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trmm_llt<T>(c, m1, n, alpha, L, ldl, B, ldb);
    gemm<T>(c, true, false, m1, n, m2, alpha, L + m1, ldl, B + m1, ldb, T(1), B, ldb);
    trmm_llt<T>(c, m2, n, alpha, L + m1 + m1 * ldl, ldl, B + m1, ldb);
}

template <typename T>
void trmm_lun(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (m <= TRX_NB) {
        // columns of B times M^T with M = U^T staged as a lower triangle
        launch_tri<T, TRI_MUL, false, false, true>(c, K_TRMM, n, (int)m, alpha, U, ldu, B, ldb);
        return;
    }
    const i64 m1 = split_q(m, TRX_NB), m2 = m - m1;
    trmm_lun<T>(c, m1, n, alpha, U, ldu, B, ldb);
    gemm<T>(c, false, false, m1, n, m2, alpha, U + m1 * ldu, ldu, B + m1, ldb, T(1), B, ldb);
    trmm_lun<T>(c, m2, n, alpha, U + m1 + m1 * ldu, ldu, B + m1, ldb);
}

template <typename T>
void trsm_run(Ctx &c, i64 m, i64 n, T alpha, const T *U, i64 ldu, T *B, i64 ldb)
{
    if (m <= 0 || n <= 0) return;
    if (n <= TRX_NB) {
        // each row x^T U^{-1}: forward substitution with M = U^T
        launch_tri<T, TRI_FWD, true, false, true>(c, K_TRSM, m, (int)n, alpha, U, ldu, B, ldb);
        return;
    }
    const i64 n1 = split_q(n, TRX_NB), n2 = n - n1;
    trsm_run<T>(c, m, n1, alpha, U, ldu, B, ldb);
    gemm<T>(c, false, false, m, n2, n1, T(-1), B, ldb, U + n1 * ldu, ldu, alpha, B + n1 * ldb, ldb);
    trsm_run<T>(c, m, n2, T(1), U + n1 + n1 * ldu, ldu, B + n1 * ldb, ldb);
}

#define RL_INST_BLAS3(T)                                                                          \
    template void gemm<T>(Ctx &, bool, bool, i64, i64, i64, T, const T *, i64, const T *, i64, T, \
                          T *, i64, bool);                                                        \
    template void symm<T>(Ctx &, bool, i64, i64, T, const T *, i64, const T *, i64, T, T *, i64); \
    template void trsm_lln<T>(Ctx &, bool, i64, i64, T, const T *, i64, T *, i64);                \
    template void trsm_rlt<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trsm_llt<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trsm_llt_u<T>(Ctx &, bool, i64, i64, T, const T *, i64, T *, i64);              \
    template void trsm_lut<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trsm_lun<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trmm_rln<T>(Ctx &, bool, i64, i64, T, const T *, i64, T *, i64);                \
    template void trmm_llt<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trmm_lun<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);                      \
    template void trsm_run<T>(Ctx &, i64, i64, T, const T *, i64, T *, i64);
RL_INST_BLAS3(double)
RL_INST_BLAS3(float)
#undef RL_INST_BLAS3
// complex double: the pieces of the Cholesky and LU recursions
template void gemm<cplx>(Ctx &, bool, bool, i64, i64, i64, cplx, const cplx *, i64, const cplx *, i64, cplx,
                         cplx *, i64, bool);
template void trsm_lln<cplx>(Ctx &, bool, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trsm_rlt<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trsm_llt<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trsm_lun<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);
// and of the inversions (trtri, lauum, getri)
template void trmm_rln<cplx>(Ctx &, bool, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trmm_llt<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trmm_lun<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);
template void trsm_run<cplx>(Ctx &, i64, i64, cplx, const cplx *, i64, cplx *, i64);

}  // namespace rl

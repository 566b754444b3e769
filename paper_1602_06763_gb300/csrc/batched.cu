// Batching form: many independent small factorizations (orders up to 256) in
// one persistent launch.  The paper has no batched form; each matrix is
// factored by the paper's scheme with the halves fixed to a block of NB
// columns (NB = 16 or 32, CTA size and CTAs per SM chosen by the autotuner,
// rl_vbatched_tune), so every CTA runs: factor the NB-column block in shared memory,
// update the rest with a triangular solve and a rank-NB product, continue on
// the trailing matrix.
//
//  * A pre-kernel sorts the matrix indices by order (largest first) with a
//    counting sort; the persistent CTAs then take matrices from an atomic
//    work counter, so large and small matrices balance across SMs.
//  * Cholesky (lower): the diagonal block is factored in shared memory; the
//    panel below it is solved row by row in registers (x L^T = a) and kept
//    in shared memory for the symmetric rank-NB update of the trailing
//    lower triangle, which runs in 4 x 4 register tiles on L2-resident data.
//  * LU with partial pivoting: the whole column panel (all rows below the
//    diagonal) is held in shared memory, one row per thread; per column a
//    block argmax (lowest row on ties), the row swap, the division by the
//    pivot and the rank-1 update; the interchanges are then applied to the
//    columns outside the panel, the U block row is solved (unit lower
//    triangle) and the trailing matrix gets a rank-NB update.
// Matrices, leading dimensions, pivots and info are addressed through
// device arrays; info follows LAPACK per matrix.
#include <climits>
#include "internal.cuh"

namespace rl {

namespace {

constexpr int BMAX = 256;          // largest order handled
// columns per pass of the batched LU's interchanges: (2 NB moved rows) x
// BPERM_COLS elements staged in the U buffer (NB x (BMAX + 1) elements)
constexpr int BPERM_COLS = 128;

struct BatchWS {
    int next;                      // work counter (zeroed per launch)
    int pad[63];
    int order[1];                  // matrix indices, largest order first (batch entries)
};

size_t batch_ws(i64 batch) { return 256 + (size_t)(batch > 0 ? batch : 1) * sizeof(int); }

// Counting sort of the orders (descending) into ws->order; one CTA.
__global__ void __launch_bounds__(1024) k_batch_sort(int batch, const int32_t *d_n, BatchWS *ws)
{
    __shared__ int hist[BMAX + 2];
    __shared__ int start[BMAX + 2];
    for (int i = threadIdx.x; i < BMAX + 2; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        int v = d_n[b];
        v = v < 0 ? 0 : (v > BMAX ? BMAX + 1 : v);
        atomicAdd(&hist[v], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int v = BMAX + 1; v >= 0; --v) { start[v] = s; s += hist[v]; }
        ws->next = 0;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        int v = d_n[b];
        v = v < 0 ? 0 : (v > BMAX ? BMAX + 1 : v);
        ws->order[atomicAdd(&start[v], 1)] = b;
    }
}

__device__ __forceinline__ void tri_decode(int t, int &ti, int &tj)
{
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

// ---- Cholesky of one matrix by the whole CTA --------------------------------
template <typename T, int BNB>
__device__ void potrf_one(T *A, int n, int lda, int32_t *info, T *sm)
{
    __shared__ int s_fail;
    T *D = sm;                           // BNB x (BNB+1)
    T *P = sm + BNB * (BNB + 1);         // (BMAX) x (BNB+1), row-major
    const int tid = threadIdx.x, bd = blockDim.x;
    constexpr int LD = BNB + 1;
    for (int k0 = 0; k0 < n; k0 += BNB) {
        const int kb = min(BNB, n - k0);
        for (int e = tid; e < kb * kb; e += bd) {
            const int i = e % kb, j = e / kb;
            if (i >= j) D[i * LD + j] = A[(i64)(k0 + j) * lda + k0 + i];
        }
        __syncthreads();
        // unblocked Cholesky of the diagonal block: FP64 by warp 0 alone (warp
        // barriers only; the other warps wait at the block barrier below),
        // FP32 by the whole CTA (measured faster there)
        if constexpr (sizeof(T) == 4) {
            int f = 0;
            for (int j = 0; j < kb; ++j) {
                const T d = D[j * LD + j];
                if (!(d > T(0))) { f = j + 1; break; }
                const T ljj = sqrt(d);
                __syncthreads();
                if (tid == 0) D[j * LD + j] = ljj;
                for (int i = j + 1 + tid; i < kb; i += bd) D[i * LD + j] = D[i * LD + j] / ljj;
                __syncthreads();
                const int t = kb - j - 1;
                for (int e = tid; e < t * t; e += bd) {
                    const int ii = j + 1 + e % t, kk = j + 1 + e / t;
                    if (ii >= kk) D[ii * LD + kk] = fma(-D[ii * LD + j], D[kk * LD + j], D[ii * LD + kk]);
                }
                __syncthreads();
            }
            if (tid == 0) s_fail = f;
        } else if (tid < 32) {
            int f = 0;
            for (int j = 0; j < kb; ++j) {
                const T d = D[j * LD + j];
                if (!(d > T(0))) { f = j + 1; break; }
                const T ljj = sqrt(d);
                __syncwarp();
                if (tid == 0) D[j * LD + j] = ljj;
                for (int i = j + 1 + tid; i < kb; i += 32) D[i * LD + j] = D[i * LD + j] / ljj;
                __syncwarp();
                const int t = kb - j - 1;
                for (int e = tid; e < t * t; e += 32) {
                    const int ii = j + 1 + e % t, kk = j + 1 + e / t;
                    if (ii >= kk) D[ii * LD + kk] = fma(-D[ii * LD + j], D[kk * LD + j], D[ii * LD + kk]);
                }
                __syncwarp();
            }
            if (tid == 0) s_fail = f;
        }
        __syncthreads();
        const int fail = s_fail;
        for (int e = tid; e < kb * kb; e += bd) {
            const int i = e % kb, j = e / kb;
            if (i >= j) A[(i64)(k0 + j) * lda + k0 + i] = D[i * LD + j];
        }
        if (fail) {
            if (tid == 0) *info = k0 + fail;
            __syncthreads();
            return;
        }
        // panel: rows below the block solve x L^T = a (right-looking, registers)
        const int r = n - k0 - kb;
        for (int row = tid; row < r; row += bd) {
            T x[BNB];
#pragma unroll
            for (int c = 0; c < BNB; ++c) x[c] = (c < kb) ? A[(i64)(k0 + c) * lda + k0 + kb + row] : T(0);
#pragma unroll
            for (int j = 0; j < BNB; ++j) {
                if (j < kb) {
                    x[j] = x[j] / D[j * LD + j];
#pragma unroll
                    for (int c = j + 1; c < BNB; ++c)
                        if (c < kb) x[c] = fma(-x[j], D[c * LD + j], x[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < BNB; ++c)
                if (c < kb) {
                    A[(i64)(k0 + c) * lda + k0 + kb + row] = x[c];
                    P[row * LD + c] = x[c];
                }
        }
        __syncthreads();
        // trailing lower triangle: A22 -= P P^T, 4 x 4 tiles
        const int T4 = (r + 3) / 4, nt = T4 * (T4 + 1) / 2;
        T *A22 = A + (i64)(k0 + kb) * lda + k0 + kb;
        for (int t = tid; t < nt; t += bd) {
            int ti, tj;
            tri_decode(t, ti, tj);
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int c = 0; c < kb; ++c) {
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * ti + u, j = 4 * tj + u;
                    a[u] = (i < r) ? P[i * LD + c] : T(0);
                    b[u] = (j < r) ? P[j * LD + c] : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int j = 4 * tj + v;
                if (j >= r) continue;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * ti + u;
                    if (i < r && i >= j) {
                        T *p = A22 + (i64)j * lda + i;
                        *p = *p - acc[u][v];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---- LU with partial pivoting of one n x n matrix by the whole CTA ----------
template <typename T, int BNB>
__device__ void getrf_one(T *A, int n, int lda, int32_t *ipiv, int32_t *info, T *sm, double *wv,
                          int *wi, int *s_piv)
{
    __shared__ int s_perm[BMAX];                 // net permutation of the block's interchanges
    __shared__ int s_tl[2 * BNB];                // the rows it moves
    __shared__ int s_nt;
    constexpr int LD = BNB + 1;          // panel row stride
    constexpr int LU = BMAX + 1;         // U block row stride
    T *P = sm;                           // BMAX x LD, row-major: P[i*LD + c]
    T *U = sm + BMAX * LD;               // BNB x LU: U[c*LU + col]
    T *stage = U;                        // the interchanges' staging (U is free until the solve)
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int k0 = 0; k0 < n; k0 += BNB) {
        const int kb = min(BNB, n - k0), mp = n - k0;
        for (int e = tid; e < mp * kb; e += bd) {
            const int i = e % mp, c = e / mp;
            P[i * LD + c] = A[(i64)(k0 + c) * lda + k0 + i];
        }
        __syncthreads();
        // the panel: per column an argmax of |P[i][j]|, i >= j (lowest i on
        // ties), the swap, the division by the pivot and the rank-1 update --
        // FP32: by warp 0 alone, separated by warp barriers only; then (warp
        // 0) the net row permutation of the block's interchanges (final row r
        // holds original row s_perm[r]) and the list of the rows it moves
        if constexpr (sizeof(T) == 8) {
            // FP64: the panel's arithmetic (one FP64 unit per quarter of the
            // SM) needs every warp; a block argmax and block barriers
            for (int j = 0; j < kb; ++j) {
                double bv = -1.0;
                int bi = INT_MAX;
                for (int i = j + tid; i < mp; i += bd) {
                    const double v = fabs((double)P[i * LD + j]);
                    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_down_sync(0xffffffffu, bv, o);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                }
                if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
                __syncthreads();
                if (tid == 0) {
                    for (int w = 1; w < (bd >> 5); ++w)
                        if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
                    const int p = (bi == INT_MAX) ? j : bi;
                    s_piv[j] = p;
                    ipiv[k0 + j] = k0 + p + 1;
                }
                __syncthreads();
                const int p = s_piv[j];
                if (p != j)
                    for (int c = tid; c < kb; c += bd) {
                        const T t = P[j * LD + c];
                        P[j * LD + c] = P[p * LD + c];
                        P[p * LD + c] = t;
                    }
                __syncthreads();
                const T piv = P[j * LD + j];
                if (piv != T(0)) {
                    for (int i = j + 1 + tid; i < mp; i += bd) {
                        const T l = P[i * LD + j] / piv;
                        P[i * LD + j] = l;
                        for (int c = j + 1; c < kb; ++c) P[i * LD + c] = fma(-l, P[j * LD + c], P[i * LD + c]);
                    }
                } else if (tid == 0 && *info == 0) {
                    *info = k0 + j + 1;
                }
                __syncthreads();
            }
        }
        if (warp == 0) {
            if constexpr (sizeof(T) != 8)
            for (int j = 0; j < kb; ++j) {
                double bv = -1.0;
                int bi = INT_MAX;
                for (int i = j + lane; i < mp; i += 32) {
                    const double v = fabs((double)P[i * LD + j]);
                    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                }
                const int p = (bi == INT_MAX) ? j : bi;
                if (lane == 0) {
                    s_piv[j] = p;
                    ipiv[k0 + j] = k0 + p + 1;
                }
                if (p != j)
                    for (int c = lane; c < kb; c += 32) {
                        const T t = P[j * LD + c];
                        P[j * LD + c] = P[p * LD + c];
                        P[p * LD + c] = t;
                    }
                __syncwarp();
                const T piv = P[j * LD + j];
                if (piv != T(0)) {
                    for (int i = j + 1 + lane; i < mp; i += 32) {
                        const T l = P[i * LD + j] / piv;
                        P[i * LD + j] = l;
                        for (int c = j + 1; c < kb; ++c) P[i * LD + c] = fma(-l, P[j * LD + c], P[i * LD + c]);
                    }
                } else if (lane == 0 && *info == 0) {
                    *info = k0 + j + 1;
                }
                __syncwarp();
            }
            for (int i = lane; i < mp; i += 32) s_perm[i] = i;
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < kb; ++j) {
                    const int p = s_piv[j], t = s_perm[j];
                    s_perm[j] = s_perm[p];
                    s_perm[p] = t;
                }
            __syncwarp();
            int nt = 0;
            for (int base = 0; base < mp; base += 32) {
                const int i = base + lane;
                const bool moved = i < mp && s_perm[i] != i;
                const unsigned mk = __ballot_sync(0xffffffffu, moved);
                if (moved) s_tl[nt + __popc(mk & ((1u << lane) - 1u))] = i;
                nt += __popc(mk);
            }
            if (lane == 0) s_nt = nt;
        }
        __syncthreads();
        for (int e = tid; e < mp * kb; e += bd) {
            const int i = e % mp, c = e / mp;
            A[(i64)(k0 + c) * lda + k0 + i] = P[i * LD + c];
        }
        // the interchanges on the columns outside the panel: (moved row,
        // column) pairs spread over the threads, every moved element read
        // into shared memory, then written to its final place
        const int nt = s_nt;
        const int nc_out = n - kb;
        for (int c0 = 0; c0 < nc_out; c0 += BPERM_COLS) {
            const int cw = min(BPERM_COLS, nc_out - c0);
            for (int e = tid; e < nt * cw; e += bd) {
                const int t = e % nt, col = c0 + e / nt;
                const int cc = (col < k0) ? col : col + kb;
                stage[e] = A[(i64)cc * lda + k0 + s_perm[s_tl[t]]];
            }
            __syncthreads();
            for (int e = tid; e < nt * cw; e += bd) {
                const int t = e % nt, col = c0 + e / nt;
                const int cc = (col < k0) ? col : col + kb;
                A[(i64)cc * lda + k0 + s_tl[t]] = stage[e];
            }
            __syncthreads();
        }
        // U block row: L11^{-1} A12 (unit lower), one column per thread
        const int nc = n - k0 - kb;
        for (int col = tid; col < nc; col += bd) {
            T x[BNB];
            T *cp = A + (i64)(k0 + kb + col) * lda + k0;
#pragma unroll
            for (int c = 0; c < BNB; ++c) x[c] = (c < kb) ? cp[c] : T(0);
#pragma unroll
            for (int d = 0; d < BNB; ++d)
#pragma unroll
                for (int c = d + 1; c < BNB; ++c)
                    if (c < kb) x[c] = fma(-P[c * LD + d], x[d], x[c]);
#pragma unroll
            for (int c = 0; c < BNB; ++c)
                if (c < kb) { cp[c] = x[c]; U[c * LU + col] = x[c]; }
        }
        __syncthreads();
        // trailing update A22 -= L21 U12 (4 x 4 tiles)
        const int r = mp - kb, RT = (r + 3) / 4, CT = (nc + 3) / 4;
        T *A22 = A + (i64)(k0 + kb) * lda + k0 + kb;
        for (int t = tid; t < RT * CT; t += bd) {
            const int ti = t % RT, tj = t / RT;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int c = 0; c < kb; ++c) {
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * ti + u, jj = 4 * tj + u;
                    a[u] = (i < r) ? P[(kb + i) * LD + c] : T(0);
                    b[u] = (jj < nc) ? U[c * LU + jj] : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int jj = 4 * tj + v;
                if (jj >= nc) continue;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * ti + u;
                    if (i < r) {
                        T *pp = A22 + (i64)jj * lda + i;
                        *pp = *pp - acc[u][v];
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, bool LU, int BNB, int BTHREADS>
__global__ void __launch_bounds__(BTHREADS)
k_batched(int batch, const int32_t *d_n, T *const *d_A, const int32_t *d_lda, int32_t *const *d_ipiv,
          int32_t *d_info, BatchWS *ws)
{
    extern __shared__ unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    __shared__ double wv[BTHREADS / 32];
    __shared__ int wi[BTHREADS / 32];
    __shared__ int s_piv[BNB];
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&ws->next, 1);
            s_idx = (t < batch) ? ws->order[t] : -1;
        }
        __syncthreads();
        const int b = s_idx;
        __syncthreads();
        if (b < 0) break;
        const int n = d_n[b];
        const int ld = d_lda[b];
        // an order outside 0..256 or a leading dimension below max(1, n) is
        // an argument error of that matrix (LAPACK's -i for argument i: the
        // order array is argument 3 of potrf and 2 of getrf, lda 5 and 4)
        const int bad = (n < 0 || n > BMAX) ? (LU ? -2 : -3) : (ld < (n > 1 ? n : 1) ? (LU ? -4 : -5) : 0);
        if (threadIdx.x == 0) d_info[b] = bad;
        __syncthreads();
        if (bad != 0 || n == 0) continue;
        if (LU) getrf_one<T, BNB>(d_A[b], n, d_lda[b], d_ipiv[b], d_info + b, sm, wv, wi, s_piv);
        else potrf_one<T, BNB>(d_A[b], n, d_lda[b], d_info + b, sm);
        __syncthreads();
    }
}

template <typename T, int BNB>
size_t batch_smem(bool lu)
{
    return lu ? (size_t)(BMAX * (BNB + 1) + BNB * (BMAX + 1)) * sizeof(T)
              : (size_t)(BNB * (BNB + 1) + BMAX * (BNB + 1)) * sizeof(T);
}

template <typename T, bool LU, int BNB, int BTHREADS>
void launch_batched(Ctx &c, i64 batch, const int32_t *d_n, T *const *d_A, const int32_t *d_lda,
                    int32_t *const *d_ipiv, int32_t *d_info, BatchWS *ws, int per_sm)
{
    const size_t smem = batch_smem<T, BNB>(LU);
    auto kern = k_batched<T, LU, BNB, BTHREADS>;
    note(c, smem_optin(kern, smem));
    int occ = 0;
    note(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BTHREADS, smem));
    if (occ < 1) occ = 1;
    if (per_sm > 0 && per_sm < occ) occ = per_sm;
    i64 grid = (i64)c.num_sms * occ;
    if (grid > batch) grid = batch;
    if (grid < 1) grid = 1;
    Launch L(c, K_BATCH, 0.0, 0.0);
    kern<<<(unsigned)grid, BTHREADS, smem, c.s>>>((int)batch, d_n, d_A, d_lda, d_ipiv, d_info, ws);
}

}  // namespace

size_t batched_work_size(i64 batch) { return batch_ws(batch); }

// Candidate configurations of the batched kernels: block width (the
// recursion's cutoff: matrices are factored in blocks of NB columns), CTA
// size, and CTAs per SM (0 = as many as fit).
const BatchCfg kBatchCfgs[BATCH_NCFG] = {
    {32, 256, 0}, {32, 256, 1}, {32, 256, 2}, {32, 128, 0}, {32, 128, 2},
    {16, 256, 0}, {16, 128, 0}, {16, 128, 4},
};

template <typename T>
int batched_factor(Ctx &c, bool lu, i64 batch, const int32_t *d_n, T *const *d_A, const int32_t *d_lda,
                   int32_t *const *d_ipiv, int32_t *d_info, int cfg, int per_sm)
{
    BatchWS *ws = reinterpret_cast<BatchWS *>(c.work);
    {
        Launch L(c, K_MIX, 0.0, 0.0);
        k_batch_sort<<<1, 1024, 0, c.s>>>((int)batch, d_n, ws);
    }
    if (cfg < 0 || cfg >= BATCH_NCFG) cfg = 0;
    const BatchCfg k = kBatchCfgs[cfg];
    const int ps = per_sm > 0 ? per_sm : k.per_sm;
#define RL_BATCH_CASE(NB, TH)                                                                        \
    if (k.nb == NB && k.threads == TH) {                                                             \
        if (lu) launch_batched<T, true, NB, TH>(c, batch, d_n, d_A, d_lda, d_ipiv, d_info, ws, ps);  \
        else launch_batched<T, false, NB, TH>(c, batch, d_n, d_A, d_lda, d_ipiv, d_info, ws, ps);    \
        return 0;                                                                                     \
    }
    RL_BATCH_CASE(32, 256)
    RL_BATCH_CASE(32, 128)
    RL_BATCH_CASE(16, 256)
    RL_BATCH_CASE(16, 128)
#undef RL_BATCH_CASE
    return 0;
}

template int batched_factor<double>(Ctx &, bool, i64, const int32_t *, double *const *, const int32_t *,
                                    int32_t *const *, int32_t *, int, int);
template int batched_factor<float>(Ctx &, bool, i64, const int32_t *, float *const *, const int32_t *,
                                   int32_t *const *, int32_t *, int, int);

}  // namespace rl

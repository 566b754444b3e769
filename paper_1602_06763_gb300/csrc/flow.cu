// Few right-hand sides: X = op(T)^{-1} B for an n x n triangle T and a thin
// B (nrhs <= FLOW_MAX_NRHS), in one launch per triangle.
//
// The recursive TRSM (Section 3's halving applied to the triangle) turns a
// thin B into many GEMMs of 16 columns, each a separate launch whose cost is
// mostly latency.  Here the triangle is cut into 64-row blocks and every
// (row block, chunk of 16 columns in FP32 or 4 in FP64) is one CTA of a
// single launch, forming a
// dataflow: the CTA of block i
//   1. inverts its diagonal block T_ii in shared memory (64 independent
//      column substitutions),
//   2. streams the off-diagonal blocks T_ik of its block row, k before i in
//      the substitution order, subtracting T_ik X_k as soon as block k's
//      ready flag is set (the tiles are prefetched while it waits),
//   3. forms X_i = T_ii^{-1} (B_i - sum_k T_ik X_k), stores it over B_i and
//      releases its flag.
// CTAs take their block from a ticket counter in the order they start, so a
// CTA waits only on CTAs that are already running: the flow cannot deadlock,
// whatever the number of resident CTAs.  Every wait is bounded; a CTA that
// gives up marks its flag failed, so the CTAs after it fail at once, and
// writes RL_INFO_DEVICE_TIMEOUT to info.
//
// Arithmetic: the same sums as substitution, with the diagonal blocks applied
// through their explicit inverses (the usual blocked form of a triangular
// solve on GPUs); the error bound gains a factor of the diagonal blocks'
// condition numbers, which for the unit-lower factor of partial pivoting
// (|l_ij| <= 1) and for the refinement's correction solves is immaterial.
#include "internal.cuh"

namespace rl {

namespace {

constexpr int FB = 64;          // row block
// right-hand sides per CTA: 16 in FP32; 4 in FP64, where each block's
// products are FP64-pipe bound and four times as many CTAs share them
template <typename T> struct FlowCols { static constexpr int value = sizeof(T) == 8 ? 4 : 16; };
constexpr int FR_MIN = 4;
constexpr int FT = 256;         // threads: 64 rows x 4 groups of 4 columns
constexpr int FP = FB + 1;      // padded column stride of the shared tiles

constexpr unsigned FLAG_DONE = 1u, FLAG_FAILED = 2u;

__device__ __forceinline__ unsigned ld_acq(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Logical triangle T = op(A) and the order of substitution.
//   FORM_LN: T = L (lower), forward.    FORM_UN: T = U (upper), backward.
//   FORM_LT: T = L^T (upper), backward, L stored lower.
enum { FORM_LN = 0, FORM_UN = 1, FORM_LT = 2 };

// Element (r, k) of block (bi, bk) of T, 0 outside the n x n matrix.
template <typename T, int FORM>
__device__ __forceinline__ T tri_elem(const T *A, i64 lda, i64 n, i64 row, i64 col)
{
    if (row >= n || col >= n) return T(0);
    return FORM == FORM_LT ? A[col + row * lda] : A[row + col * lda];
}

// Tile load index: element e of the 64 x 64 tile, ordered so that
// consecutive threads read consecutive addresses of A.
template <int FORM>
__device__ __forceinline__ void tile_rk(int e, int &r, int &k)
{
    if (FORM == FORM_LT) { k = e & (FB - 1); r = e >> 6; }
    else { r = e & (FB - 1); k = e >> 6; }
}

constexpr int PER = FB * FB / FT;                  // tile elements per thread

// Block (row block at r0, column block bk) of T into registers.
template <typename T, int FORM>
__device__ __forceinline__ void fetch_tile(T (&pre)[PER], const T *A, i64 lda, i64 n, i64 r0, int bk,
                                           int tid)
{
    const i64 k0 = (i64)bk * FB;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        int rr, kk;
        tile_rk<FORM>(tid + u * FT, rr, kk);
        pre[u] = tri_elem<T, FORM>(A, lda, n, r0 + rr, k0 + kk);
    }
}

template <typename T, int FORM, bool UNIT, int FR = FlowCols<T>::value>
__global__ void __launch_bounds__(FT)
k_flow(i64 n, int nrhs, const T *A, i64 lda, T *B, i64 ldb, unsigned *ticket, unsigned *flags,
       int32_t *status, long long spin_ns, int32_t *info, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ts = reinterpret_cast<T *>(smem_raw);          // T(r, k) at Ts[k * FP + r]
    T *Inv = Ts + FB * FP;                             // inverse of T_ii, same layout
    T *Xs = Inv + FB * FP;                             // X(k, col) at Xs[k * FR + col]
    __shared__ unsigned s_t;
    __shared__ int s_fail;

    const int tid = threadIdx.x;
    if (tid == 0) { s_t = atomicAdd(ticket, 1u); s_fail = 0; }
    __syncthreads();
    const int nblk = (int)((n + FB - 1) / FB);
    const int nch = (nrhs + FR - 1) / FR;
    const int step = (int)(s_t / (unsigned)nch), ch = (int)(s_t % (unsigned)nch);
    const bool fwd = FORM == FORM_LN;
    const int bi = fwd ? step : nblk - 1 - step;
    const i64 r0 = (i64)bi * FB;
    const int c0 = ch * FR;
    constexpr int CPT = FR / 4;                        // columns per thread
    const int r = tid & (FB - 1), g = tid >> 6;        // this thread: row r, columns CPT*g ..
    unsigned *myflag = flags + (size_t)bi * nch + ch;

    // right-hand side block
    T acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int col = c0 + CPT * g + q;
        acc[q] = (r0 + r < n && col < nrhs) ? B[(r0 + r) + (i64)col * ldb] : T(0);
    }

    // 1. diagonal block and its inverse (rows/columns past n: identity)
    for (int e = tid; e < FB * FB; e += FT) {
        int rr, kk;
        tile_rk<FORM>(e, rr, kk);
        T v = tri_elem<T, FORM>(A, lda, n, r0 + rr, r0 + kk);
        if (r0 + rr >= n || r0 + kk >= n) v = (rr == kk) ? T(1) : T(0);
        Ts[kk * FP + rr] = v;
    }
    __syncthreads();
    if (tid < FB) {
        const int j = tid;                              // column j of the inverse
        T *x = Inv + j * FP;
        if (FORM == FORM_LN) {
            for (int i = 0; i < j; ++i) x[i] = T(0);
            for (int i = j; i < FB; ++i) {
                T s = (i == j) ? T(1) : T(0);
                for (int k = j; k < i; ++k) s = fma(-Ts[k * FP + i], x[k], s);
                x[i] = (UNIT || r0 + i >= n) ? s : s / Ts[i * FP + i];
            }
        } else {
            for (int i = j + 1; i < FB; ++i) x[i] = T(0);
            for (int i = j; i >= 0; --i) {
                T s = (i == j) ? T(1) : T(0);
                for (int k = i + 1; k <= j; ++k) s = fma(-Ts[k * FP + i], x[k], s);
                x[i] = (UNIT || r0 + i >= n) ? s : s / Ts[i * FP + i];
            }
        }
    }

    // 2. contributions of the blocks solved before this one
    T pre[PER];
    if (step > 0) fetch_tile<T, FORM>(pre, A, lda, n, r0, fwd ? 0 : nblk - 1, tid);
    for (int sk = 0; sk < step; ++sk) {
        const int bk = fwd ? sk : nblk - 1 - sk;
        const i64 k0 = (i64)bk * FB;
        __syncthreads();                                // previous tile and Xs are consumed
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            int rr, kk;
            tile_rk<FORM>(tid + u * FT, rr, kk);
            Ts[kk * FP + rr] = pre[u];
        }
        if (sk + 1 < step) fetch_tile<T, FORM>(pre, A, lda, n, r0, fwd ? sk + 1 : nblk - 2 - sk, tid);
        if (tid == 0) {
            const unsigned *f = flags + (size_t)bk * nch + ch;
            unsigned v = ld_acq(f);
            if (v == 0u) {
                const unsigned long long t0 = gtimer();
                while ((v = ld_acq(f)) == 0u) {
                    if ((long long)(gtimer() - t0) >= spin_ns) break;
                    __nanosleep(32);
                }
            }
            if (v != FLAG_DONE) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) {
                st_rel(myflag, FLAG_FAILED);
                atomicExch(status, RL_INFO_DEVICE_TIMEOUT);
                if (info) atomicExch(info, RL_INFO_DEVICE_TIMEOUT);
            }
            return;
        }
#pragma unroll
        for (int u = 0; u < FB * FR / FT; ++u) {
            const int e = tid + u * FT;
            const int kk = e & (FB - 1), col = e >> 6;
            Xs[kk * FR + col] = (k0 + kk < n && c0 + col < nrhs)
                                    ? __ldcg(&B[(k0 + kk) + (i64)(c0 + col) * ldb]) : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < FB; ++k) {
            const T t = Ts[k * FP + r];
            const T *xr = Xs + k * FR + CPT * g;
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[q] = fma(-t, xr[q], acc[q]);
        }
    }

    // 3. X_i = T_ii^{-1} (B_i - sum T_ik X_k)
    __syncthreads();
#pragma unroll
    for (int q = 0; q < CPT; ++q) Xs[r * FR + CPT * g + q] = acc[q];
    __syncthreads();
    T out[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) out[q] = T(0);
#pragma unroll 8
    for (int k = 0; k < FB; ++k) {
        const T t = Inv[k * FP + r];
        const T *xr = Xs + k * FR + CPT * g;
#pragma unroll
        for (int q = 0; q < CPT; ++q) out[q] = fma(t, xr[q], out[q]);
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int col = c0 + CPT * g + q;
        if (r0 + r < n && col < nrhs) B[(r0 + r) + (i64)col * ldb] = out[q];
    }
    __syncthreads();
    if (tid == 0) st_rel(myflag, FLAG_DONE);
}

template <typename T, int FORM, bool UNIT>
void launch_flow(Ctx &c, i64 n, i64 nrhs, const T *A, i64 lda, T *B, i64 ldb, void *ws)
{
    constexpr int FR = FlowCols<T>::value;
    const i64 nblk = (n + FB - 1) / FB, nch = (nrhs + FR - 1) / FR;
    int32_t *status = static_cast<int32_t *>(ws);
    unsigned *ticket = static_cast<unsigned *>(ws) + 64;
    unsigned *flags = ticket + 1;
    const size_t smem = (2 * (size_t)FB * FP + (size_t)FB * FR) * sizeof(T);
    note(c, smem_optin(k_flow<T, FORM, UNIT>, smem));
    note(c, cudaMemsetAsync(ticket, 0, (1 + (size_t)nblk * nch) * sizeof(unsigned), c.s));
    // n^2 nrhs flops; the triangle is read once, B read and written once
    Launch L(c, K_TRSM, (double)n * n * nrhs,
             ((double)n * n / 2.0 + 2.0 * (double)n * nrhs) * sizeof(T));
    k_flow<T, FORM, UNIT><<<(unsigned)(nblk * nch), FT, smem, c.s>>>(
        n, (int)nrhs, A, lda, B, ldb, ticket, flags, status, g_params.spin_ns, c.info, c.abort);
}

}  // namespace

size_t flow_ws_bytes(i64 n, i64 nrhs)
{
    // flags for the narrowest chunking (either element type)
    const i64 nblk = (n + FB - 1) / FB, nch = (nrhs + FR_MIN - 1) / FR_MIN;
    return ((65 + (size_t)(nblk > 0 ? nblk : 1) * (size_t)(nch > 0 ? nch : 1)) * sizeof(unsigned) + 255) &
           ~(size_t)255;
}

template <typename T>
void trsm_flow(Ctx &c, int form, bool unit, i64 n, i64 nrhs, const T *A, i64 lda, T *B, i64 ldb,
               void *ws)
{
    if (n <= 0 || nrhs <= 0) return;
    if (form == FLOW_LN) {
        if (unit) launch_flow<T, FORM_LN, true>(c, n, nrhs, A, lda, B, ldb, ws);
        else launch_flow<T, FORM_LN, false>(c, n, nrhs, A, lda, B, ldb, ws);
    } else if (form == FLOW_UN) {
        launch_flow<T, FORM_UN, false>(c, n, nrhs, A, lda, B, ldb, ws);
    } else {
        launch_flow<T, FORM_LT, false>(c, n, nrhs, A, lda, B, ldb, ws);
    }
}

template void trsm_flow<float>(Ctx &, int, bool, i64, i64, const float *, i64, float *, i64, void *);
template void trsm_flow<double>(Ctx &, int, bool, i64, i64, const double *, i64, double *, i64, void *);

}  // namespace rl

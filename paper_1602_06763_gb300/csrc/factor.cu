// Base cases of the recursions (Section 3: below the crossover size c the
// recursion switches to LAPACK's unblocked routines) and the row
// interchanges of the LU factorization.  potf2, the LU panel and LASWP are
// templated on the element type (double: FP64 path; float: FP32 storage of
// the precision form).
//
//  k_potf2        unblocked Cholesky of a diagonal block (n <= 64), one CTA,
//                 right-looking in shared memory; IEEE sqrt and division.
//  k_trti2        unblocked triangular inverse (n <= 64), one CTA.
//  k_lauu2        unblocked L^T L (n <= 64), one CTA.
//  k_diag_scan    first exactly-zero diagonal entry (dtrtri's info).
//  k_panel        fused LU panel of an m x nb block (nb <= 64): per column a
//                 pivot search (argmax on integer keys, lowest row on ties),
//                 the row swap, the division of the column by the pivot and
//                 the rank-1 update.  The co-resident CTAs of one cooperative
//                 launch each keep up to 256 rows in shared memory (one row
//                 per thread); per column one warp per CTA publishes the
//                 CTA's candidate record, arrives on a grid counter and reads
//                 all candidates back.
//  k_panel_smem   the same algorithm with the rows as a column-major slab,
//                 for panels taller than 256 rows per CTA.
//  k_panel_cluster  FP32 panels of up to 16384 rows on one thread-block
//                 cluster, the panel in registers, the candidates exchanged
//                 through distributed shared memory.
//  k_laswp        row interchanges: each CTA turns the swap sequence into the
//                 net permutation of the touched rows (in shared memory) and
//                 then moves every touched row of its columns with one
//                 coalesced gather and one scatter per column.
// Every device-side wait is bounded (RL_PARAM_SPIN_LIMIT_NS); a wait that
// runs out sets *info = RL_INFO_DEVICE_TIMEOUT and the kernel returns.
#include <climits>
#include <mutex>
#include <cooperative_groups.h>
#include "internal.cuh"
#include "tc_common.cuh"

namespace rl {

constexpr int BASE_N = 64;
constexpr int BASE_PACK = BASE_N * (BASE_N + 1) / 2;

__device__ __forceinline__ int tix(int i, int k) { return i * (i + 1) / 2 + k; }

// ----------------------------------------------------------------------------
// potf2: for j = 0..n-1: d = a_jj; if !(d > 0) -> info; l_jj = sqrt(d);
// column j below the diagonal divided by l_jj; trailing lower block updated
// a_ik -= l_ij l_kj.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_potf2(int n, T *A, i64 lda, int32_t *info, i64 info_off, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ T S[BASE_N][BASE_N + 1];
    __shared__ T col[BASE_N];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    for (int j = ty; j < n; j += 16)
        for (int i = j + tx; i < n; i += 16) S[i][j] = A[(i64)j * lda + i];
    __syncthreads();
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        // warp 0 alone takes the square root and divides column j (the FP64
        // pipe is scarce: the other warps would only repeat the same work)
        if (threadIdx.x < 32) {
            const T d = S[j][j];
            if (!(d > T(0))) {
                if (threadIdx.x == 0) s_fail = j + 1;
            } else {
                const T ljj = sqrt(d);
                for (int i = j + 1 + threadIdx.x; i < n; i += 32) {
                    const T v = S[i][j] / ljj;
                    col[i] = v;
                    S[i][j] = v;
                }
                if (threadIdx.x == 0) S[j][j] = ljj;
            }
        }
        __syncthreads();
        if (s_fail) break;
        for (int ii = j + 1 + ty; ii < n; ii += 16) {
            const T lij = col[ii];
            for (int kk = j + 1 + tx; kk <= ii; kk += 16) S[ii][kk] = fma(-lij, col[kk], S[ii][kk]);
        }
        __syncthreads();
    }
    for (int j = ty; j < n; j += 16)
        for (int i = j + tx; i < n; i += 16) A[(i64)j * lda + i] = S[i][j];
    if (s_fail && threadIdx.x == 0) *info = (int32_t)(info_off + s_fail);
}

// Complex Hermitian potf2 (A = L L^H): the real form above with l_ij / l_jj
// and the update a_ik -= l_ij conj(l_kj); the diagonal is real (its
// imaginary part is ignored, as LAPACK's zpotf2 does).
__global__ void __launch_bounds__(256)
k_zpotf2(int n, cplx *A, i64 lda, int32_t *info, i64 info_off, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ __align__(16) unsigned char zp_raw[];       // 66.6 KB: dynamic
    auto S = reinterpret_cast<cplx (*)[BASE_N + 1]>(zp_raw);      // S[BASE_N][BASE_N + 1]
    cplx *col = reinterpret_cast<cplx *>(zp_raw) + BASE_N * (BASE_N + 1);
    __shared__ int s_fail;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int j = ty; j < n; j += 16)
        for (int i = j + tx; i < n; i += 16) S[i][j] = A[(i64)j * lda + i];
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x < 32) {
            const double d = S[j][j].x;
            if (!(d > 0.0)) {
                if (threadIdx.x == 0) { s_fail = j + 1; S[j][j] = cplx(d); }
            } else {
                const double ljj = sqrt(d);
                for (int i = j + 1 + threadIdx.x; i < n; i += 32) {
                    const cplx v = S[i][j] / cplx(ljj);
                    col[i] = v;
                    S[i][j] = v;
                }
                if (threadIdx.x == 0) S[j][j] = cplx(ljj);
            }
        }
        __syncthreads();
        if (s_fail) break;
        for (int ii = j + 1 + ty; ii < n; ii += 16) {
            const cplx lij = col[ii];
            for (int kk = j + 1 + tx; kk <= ii; kk += 16) S[ii][kk] = fma(-lij, conj(col[kk]), S[ii][kk]);
        }
        __syncthreads();
    }
    for (int j = ty; j < n; j += 16)
        for (int i = j + tx; i < n; i += 16) A[(i64)j * lda + i] = S[i][j];
    if (s_fail && threadIdx.x == 0) *info = (int32_t)(info_off + s_fail);
}

template <>
void potf2<cplx>(Ctx &c, i64 n, cplx *A, i64 lda, i64 info_off)
{
    if (n <= 0) return;
    if (n > BASE_N) { note(c, cudaErrorInvalidValue); return; }
    const size_t smem = (size_t)BASE_N * (BASE_N + 2) * sizeof(cplx);
    note(c, smem_optin(k_zpotf2, smem));
    Launch L(c, K_POTF2, 4.0 * (double)n * n * n / 3.0, 0.0);
    k_zpotf2<<<1, 256, smem, c.s>>>((int)n, A, lda, c.info, info_off, c.abort);
}

template <typename T>
void potf2(Ctx &c, i64 n, T *A, i64 lda, i64 info_off)
{
    if (n <= 0) return;
    Launch L(c, K_POTF2, (double)n * n * n / 3.0, 0.0);
    k_potf2<T><<<1, 256, 0, c.s>>>((int)n, A, lda, c.info, info_off, c.abort);
}

// ----------------------------------------------------------------------------
// trti2: X = L^{-1}; thread j computes column j by forward substitution on
// L x = e_j: x_jj = 1/l_jj; x_ij = -(sum_{k=j}^{i-1} l_ik x_kj) / l_ii.
// L packed by rows, X packed by columns (each thread owns its column).
// ----------------------------------------------------------------------------
template <typename T, bool UNIT, bool UPPER>
__global__ void __launch_bounds__(BASE_N)
k_trti2(int n, T *A, i64 lda, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    // complex (16-byte) elements: order <= 32, so both packed triangles fit
    // the 48 KB of static shared memory
    constexpr int PACK = sizeof(T) > 8 ? 32 * 33 / 2 : BASE_PACK;
    __shared__ T Lp[PACK];
    __shared__ T Xp[PACK];
    // UPPER: invert M = U^T (lower) and store X = (M^{-1})^T = U^{-1}
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e % n, k = e / n;
        if (i >= k) Lp[tix(i, k)] = UPPER ? A[(i64)i * lda + k] : A[(i64)k * lda + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < n) {
        // column j of X occupies Xp[cs .. cs + n - j), entry i at cs + (i - j)
        const int cs = j * n - j * (j - 1) / 2;
        Xp[cs] = UNIT ? T(1) : T(1) / Lp[tix(j, j)];
        for (int i = j + 1; i < n; ++i) {
            T s = T(0);
            for (int k = j; k < i; ++k) s = fma(Lp[tix(i, k)], Xp[cs + (k - j)], s);
            Xp[cs + (i - j)] = UNIT ? -s : -s / Lp[tix(i, i)];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e % n, jj = e / n;
        if (i > jj || (i == jj && !UNIT)) {
            const int cs = jj * n - jj * (jj - 1) / 2;
            if (UPPER) A[(i64)i * lda + jj] = Xp[cs + (i - jj)];
            else A[(i64)jj * lda + i] = Xp[cs + (i - jj)];
        }
    }
}

template <typename T>
void trti2(Ctx &c, bool unit, i64 n, T *A, i64 lda, bool upper)
{
    if (n <= 0) return;
    if (sizeof(T) > 8 && n > 32) { note(c, cudaErrorInvalidValue); return; }
    Launch L(c, K_TRTI2, (double)n * n * n / 3.0, 0.0);
    if (upper) {
        if (unit) k_trti2<T, true, true><<<1, BASE_N, 0, c.s>>>((int)n, A, lda, c.abort);
        else k_trti2<T, false, true><<<1, BASE_N, 0, c.s>>>((int)n, A, lda, c.abort);
    } else {
        if (unit) k_trti2<T, true, false><<<1, BASE_N, 0, c.s>>>((int)n, A, lda, c.abort);
        else k_trti2<T, false, false><<<1, BASE_N, 0, c.s>>>((int)n, A, lda, c.abort);
    }
}
template void trti2<double>(Ctx &, bool, i64, double *, i64, bool);
template void trti2<float>(Ctx &, bool, i64, float *, i64, bool);
template void trti2<cplx>(Ctx &, bool, i64, cplx *, i64, bool);

// ----------------------------------------------------------------------------
// lauu2: (L^T L)_ij = sum_{k=i}^{n-1} l_ki l_kj for i >= j, from a staged copy
// (complex: L^H L, conj(l_ki) l_kj).
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_lauu2(int n, T *A, i64 lda, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    __shared__ T Lp[BASE_PACK];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e % n, k = e / n;
        if (i >= k) Lp[tix(i, k)] = A[(i64)k * lda + i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e % n, j = e / n;
        if (i < j) continue;
        T s = T(0);
        for (int k = i; k < n; ++k) s = fma(cj(Lp[tix(k, i)]), Lp[tix(k, j)], s);
        A[(i64)j * lda + i] = s;
    }
}

template <typename T>
void lauu2(Ctx &c, i64 n, T *A, i64 lda)
{
    if (n <= 0) return;
    Launch L(c, K_LAUU2, (double)n * n * n / 3.0, 0.0);
    k_lauu2<T><<<1, 256, 0, c.s>>>((int)n, A, lda, c.abort);
}
template void lauu2<double>(Ctx &, i64, double *, i64);
template void lauu2<float>(Ctx &, i64, float *, i64);
template void lauu2<cplx>(Ctx &, i64, cplx *, i64);

// ----------------------------------------------------------------------------
// First exactly-zero diagonal entry -> info (dtrtri leaves A unchanged then).
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024)
k_diag_scan(i64 n, const T *A, i64 lda, int32_t *info)
{
    __shared__ i64 wmin[32];
    i64 best = LLONG_MAX;
    for (i64 i = threadIdx.x; i < n; i += blockDim.x)
        if (A[i * lda + i] == T(0) && i < best) best = i;
    for (int o = 16; o > 0; o >>= 1) {
        i64 v = __shfl_down_sync(0xffffffffu, best, o);
        if (v < best) best = v;
    }
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (wmin[w] < best) best = wmin[w];
        if (best != LLONG_MAX) *info = (int32_t)(best + 1);
    }
}

template <typename T>
void diag_zero_scan(Ctx &c, i64 n, const T *A, i64 lda)
{
    if (n <= 0) return;
    Launch L(c, K_DIAG, 0.0, (double)n * sizeof(T));
    k_diag_scan<T><<<1, 1024, 0, c.s>>>(n, A, lda, c.info);
}
template void diag_zero_scan<double>(Ctx &, i64, const double *, i64);
template void diag_zero_scan<float>(Ctx &, i64, const float *, i64);
template void diag_zero_scan<cplx>(Ctx &, i64, const cplx *, i64);

// ----------------------------------------------------------------------------
// LU panel.
// ----------------------------------------------------------------------------
constexpr int PANEL_GMAX = 256;
constexpr int PANEL_NBMAX = 64;
constexpr int PANEL_THREADS = 256;
constexpr int PANEL_RMIN = 64;
constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
// widest panel per element type (a complex row of 32 fills an exchange record)
template <typename T> constexpr int panel_nbmax() { return sizeof(T) == 16 ? PANEL_NBMAX / 2 : PANEL_NBMAX; }

constexpr int PANEL_REC = 2 + PANEL_NBMAX;

// Exchange area of the multi-CTA panel kernels.  Per column each CTA
// publishes one record {key of |candidate|, candidate row (PANEL_NONE =
// none), both stored as 64-bit patterns, then the candidate row's nb
// entries}; the owner of row j also
// publishes row j.  Both are double-buffered by column parity: a CTA can be
// at most one column ahead of any other, because the arrival counter holds
// it at the next column's barrier.
struct PanelWS {
    unsigned int counter;               // arrivals, G per column
    unsigned int pad[63];
    double rec[2][PANEL_GMAX][PANEL_REC];
    double rowj[2][PANEL_NBMAX];
};

size_t panel_ws_bytes() { return sizeof(PanelWS); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Pivot search on integer keys: the bit pattern of |v| orders like |v| for
// non-negative doubles, so the comparisons run on the integer pipes (the
// FP64 pipe is the scarce unit on this GPU).  NaN gets key 0 (it never wins
// over a number; a column of NaNs and zeros takes its lowest row).  "No
// candidate" is key 0 with row PANEL_NONE, which loses every tie.
constexpr int PANEL_NONE = 0x7fffffff;

template <typename T>
__device__ __forceinline__ unsigned long long abs_key(T v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong((double)v) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
}

// |Re| + |Im| for complex pivots (LAPACK's izamax)
__device__ __forceinline__ unsigned long long abs_key(cplx v) { return abs_key<double>(abs1(v)); }

// Rows in the exchange area are doubles: one per real entry, two (re, im)
// per complex entry.
template <typename T> __device__ __forceinline__ void put_row(double *row, int c, T v) { row[c] = (double)v; }
__device__ __forceinline__ void put_row(double *row, int c, cplx v) { row[2 * c] = v.x; row[2 * c + 1] = v.y; }
template <typename T> __device__ __forceinline__ T get_row(const double *row, int c) { return (T)__ldcg(row + c); }
template <> __device__ __forceinline__ cplx get_row<cplx>(const double *row, int c)
{
    return cplx(__ldcg(row + 2 * c), __ldcg(row + 2 * c + 1));
}

__device__ __forceinline__ bool kbetter(unsigned long long k, int i, unsigned long long bk, int bi)
{
    return k > bk || (k == bk && i < bi);
}

// Row-per-thread panel.  CTA g owns panel rows [g*R, g*R + R), R <= 256;
// thread t works on row g*R + t, kept in shared memory as a[c * 256 + t]
// (consecutive threads, consecutive words).  ipiv and info use global
// numbering: panel row r is matrix row r0 + r.
//
// Per column, two block barriers: after the local candidate search, warp 0
// alone publishes the CTA's record, arrives on the grid counter with a
// release add, waits for all G arrivals (bounded), reads the G candidates in
// one round trip, picks the winner (largest |a_ij|, lowest row on ties) and
// fetches its row; then every thread swaps, scales and updates its own row.
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS)
k_panel(i64 m, int nb, T *A, i64 lda, int32_t *ipiv, i64 r0, int32_t *info, PanelWS *ws, int R,
        long long spin_ns, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    __shared__ unsigned long long wk[PANEL_THREADS / 32];
    __shared__ int wi[PANEL_THREADS / 32];
    __shared__ int s_p;
    __shared__ int s_fail;
    __shared__ T urow[PANEL_NBMAX], rowj[PANEL_NBMAX];

    const int tid = threadIdx.x, lane = tid & 31, G = gridDim.x, g = blockIdx.x;
    const i64 rbeg = (i64)g * R;
    const int rows = (int)max((i64)0, min((i64)R, m - rbeg));
    const i64 my = rbeg + tid;                 // this thread's panel row
    const bool have = tid < rows;
    T *a = S + tid;                            // a[c * PANEL_THREADS] = element (my, c)
    if (have)
        for (int c = 0; c < nb; ++c) a[c * PANEL_THREADS] = A[(i64)c * lda + my];

    const int mn = (int)min(m, (i64)nb);
    for (int j = 0; j < mn; ++j) {
        const int buf = j & 1;
        // 1. this CTA's candidate: largest |a_ij|, i >= j, lowest i on ties
        unsigned long long bk = 0;
        int bi = PANEL_NONE;
        if (have && my >= j) { bk = abs_key(a[j * PANEL_THREADS]); bi = (int)my; }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_down_sync(0xffffffffu, bk, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (kbetter(ok, oi, bk, bi)) { bk = ok; bi = oi; }
        }
        if (lane == 0) { wk[tid >> 5] = bk; wi[tid >> 5] = bi; }
        __syncthreads();
        if (tid < 32) {
            // 2. block candidate (every lane of warp 0 ends with it)
            bk = lane < PANEL_THREADS / 32 ? wk[lane] : 0ull;
            bi = lane < PANEL_THREADS / 32 ? wi[lane] : PANEL_NONE;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (kbetter(ok, oi, bk, bi)) { bk = ok; bi = oi; }
            }
            // 3. publish the record (and row j, by its owner), then arrive
            double *rec = ws->rec[buf][g];
            if (lane == 0) {
                rec[0] = __longlong_as_double((long long)bk);
                rec[1] = __longlong_as_double((long long)bi);
            }
            if (bi != PANEL_NONE) {
                const T *src = S + (int)(bi - rbeg);
                for (int c = lane; c < nb; c += 32) put_row(rec + 2, c, src[c * PANEL_THREADS]);
            }
            if (j >= rbeg && j < rbeg + rows) {
                const T *src = S + (int)(j - rbeg);
                for (int c = lane; c < nb; c += 32) put_row(ws->rowj[buf], c, src[c * PANEL_THREADS]);
            }
            __syncwarp();
            int ok = 1;
            if (lane == 0) {
                red_release_add(&ws->counter, 1u);
                const unsigned target = (unsigned)G * (unsigned)(j + 1);
                if (ld_acquire_u32(&ws->counter) < target) {
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire_u32(&ws->counter) < target) {
                        if ((long long)(global_ns() - t0) >= spin_ns) { ok = 0; break; }
                        __nanosleep(16);
                    }
                }
            }
            __syncwarp();                      // orders lane 0's acquire before the lanes' loads
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) {
                // 4. all G candidates in one round trip (G <= 256: 8 per lane)
                unsigned long long k = 0;
                int ix = PANEL_NONE, gw = -1;
                unsigned long long qk[PANEL_GMAX / 32];
                int qi[PANEL_GMAX / 32];
#pragma unroll
                for (int u = 0; u < PANEL_GMAX / 32; ++u) {
                    const int q = lane + 32 * u;
                    qk[u] = 0;
                    qi[u] = PANEL_NONE;
                    if (q < G) {
                        qk[u] = (unsigned long long)__double_as_longlong(__ldcg(&ws->rec[buf][q][0]));
                        qi[u] = (int)__double_as_longlong(__ldcg(&ws->rec[buf][q][1]));
                    }
                }
#pragma unroll
                for (int u = 0; u < PANEL_GMAX / 32; ++u)
                    if (qi[u] != PANEL_NONE && (gw < 0 || kbetter(qk[u], qi[u], k, ix))) {
                        k = qk[u]; ix = qi[u]; gw = lane + 32 * u;
                    }
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
                    const int og = __shfl_xor_sync(0xffffffffu, gw, o);
                    if (og >= 0 && (gw < 0 || kbetter(ok, oi, k, ix))) { k = ok; ix = oi; gw = og; }
                }
                // 5. the pivot row, and row j where this CTA owns the pivot row
                const int p = (gw >= 0) ? ix : j;
                const bool own_p = (p != j) && p >= rbeg && p < rbeg + rows;
                for (int c = lane; c < nb; c += 32) {
                    urow[c] = (gw >= 0) ? get_row<T>(ws->rec[buf][gw] + 2, c) : get_row<T>(ws->rowj[buf], c);
                    if (own_p) rowj[c] = get_row<T>(ws->rowj[buf], c);
                }
                if (lane == 0) s_p = p;
            }
            if (lane == 0) s_fail = !ok;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) atomicExch(info, RL_INFO_DEVICE_TIMEOUT);
            return;
        }
        const i64 p = s_p;
        const bool own_p = (p != j) && p >= rbeg && p < rbeg + rows;
        if (g == 0 && tid == 0) ipiv[r0 + j] = (int32_t)(r0 + p + 1);
        // 6. swap, scale and rank-1 update of this thread's row
        if (have) {
            if (p != j && my == j) {
                for (int c = 0; c < nb; ++c) a[c * PANEL_THREADS] = urow[c];
            } else if (own_p && my == p) {
                for (int c = 0; c < nb; ++c) a[c * PANEL_THREADS] = rowj[c];
            }
        }
        const T piv = urow[j];
        if (piv != T(0)) {
            if (have && my > j) {
                const T l = a[j * PANEL_THREADS] / piv;
                a[j * PANEL_THREADS] = l;
#pragma unroll 4
                for (int c = j + 1; c < nb; ++c)
                    a[c * PANEL_THREADS] = fma(-l, urow[c], a[c * PANEL_THREADS]);
            }
        } else {
            if (g == 0 && tid == 0 && *info == 0) *info = (int32_t)(r0 + j + 1);
            // a zero pivot column: the elimination step subtracts zero multiples
        }
    }
    if (have)
        for (int c = 0; c < nb; ++c) A[(i64)c * lda + my] = a[c * PANEL_THREADS];
}

// Bounded grid barrier of the shared-memory panel kernel.
__device__ bool grid_barrier(unsigned *counter, unsigned target, long long spin_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        int good = 1;
        if (ld_acquire_u32(counter) < target) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(counter) < target) {
                if ((long long)(global_ns() - t0) >= spin_ns) { good = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Shared-memory panel for tall panels (R > 256 rows per CTA): CTA g holds
// rows [g*R, g*R + R) as a column-major slab S[c*R + r].
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS)
k_panel_smem(i64 m, int nb, T *A, i64 lda, int32_t *ipiv, i64 r0, int32_t *info, PanelWS *ws,
             int R, long long spin_ns, const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    __shared__ T urow[PANEL_NBMAX];
    __shared__ unsigned long long wk[PANEL_THREADS / 32];
    __shared__ int wi[PANEL_THREADS / 32];
    __shared__ int s_p;
    __shared__ int s_gw;

    const int tid = threadIdx.x, G = gridDim.x, g = blockIdx.x;
    const i64 rbeg = (i64)g * R;
    const int rows = (int)max((i64)0, min((i64)R, m - rbeg));
    for (int e = tid; e < rows * nb; e += blockDim.x) {
        int r = e % rows, cc = e / rows;
        S[cc * R + r] = A[(i64)cc * lda + rbeg + r];
    }
    __syncthreads();

    const int mn = (int)min(m, (i64)nb);
    for (int j = 0; j < mn; ++j) {
        const int buf = j & 1;
        unsigned long long bk = 0;
        int bi = PANEL_NONE;
        for (int r = tid; r < rows; r += blockDim.x) {
            const i64 i = rbeg + r;
            if (i < j) continue;
            const unsigned long long k = abs_key(S[j * R + r]);
            if (kbetter(k, (int)i, bk, bi)) { bk = k; bi = (int)i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_down_sync(0xffffffffu, bk, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (kbetter(ok, oi, bk, bi)) { bk = ok; bi = oi; }
        }
        if ((tid & 31) == 0) { wk[tid >> 5] = bk; wi[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < PANEL_THREADS / 32; ++w)
                if (kbetter(wk[w], wi[w], bk, bi)) { bk = wk[w]; bi = wi[w]; }
            ws->rec[buf][g][0] = __longlong_as_double((long long)bk);
            ws->rec[buf][g][1] = __longlong_as_double((long long)bi);
            s_p = bi;
        }
        __syncthreads();
        {
            const int mine = s_p;
            if (mine != PANEL_NONE && tid < nb) put_row(ws->rec[buf][g] + 2, tid, S[tid * R + (int)(mine - rbeg)]);
            if (j >= rbeg && j < rbeg + rows && tid < nb) put_row(ws->rowj[buf], tid, S[tid * R + (int)(j - rbeg)]);
        }
        if (!grid_barrier(&ws->counter, (unsigned)G * (unsigned)(j + 1), spin_ns)) {
            if (tid == 0) atomicExch(info, RL_INFO_DEVICE_TIMEOUT);
            return;
        }
        if (tid < 32) {
            unsigned long long k = 0;
            int ix = PANEL_NONE, gw = -1;
            for (int q = tid; q < G; q += 32) {
                const int qi = (int)__double_as_longlong(__ldcg(&ws->rec[buf][q][1]));
                const unsigned long long qk = (unsigned long long)__double_as_longlong(__ldcg(&ws->rec[buf][q][0]));
                if (qi != PANEL_NONE && (gw < 0 || kbetter(qk, qi, k, ix))) { k = qk; ix = qi; gw = q; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_down_sync(0xffffffffu, k, o);
                const int oi = __shfl_down_sync(0xffffffffu, ix, o);
                const int og = __shfl_down_sync(0xffffffffu, gw, o);
                if (og >= 0 && (gw < 0 || kbetter(ok, oi, k, ix))) { k = ok; ix = oi; gw = og; }
            }
            if (tid == 0) { s_p = (gw >= 0) ? ix : j; s_gw = gw; }
        }
        __syncthreads();
        const i64 p = s_p;
        const int gw = s_gw;
        if (tid < nb) urow[tid] = (gw >= 0) ? get_row<T>(ws->rec[buf][gw] + 2, tid) : get_row<T>(ws->rowj[buf], tid);
        __syncthreads();
        const T piv = urow[j];
        if (g == 0 && tid == 0) ipiv[r0 + j] = (int32_t)(r0 + p + 1);
        if (p != j) {
            if (j >= rbeg && j < rbeg + rows && tid < nb) S[tid * R + (int)(j - rbeg)] = urow[tid];
            if (p >= rbeg && p < rbeg + rows && tid < nb) S[tid * R + (int)(p - rbeg)] = get_row<T>(ws->rowj[buf], tid);
        }
        __syncthreads();
        if (piv != T(0)) {
            for (int r = tid; r < rows; r += blockDim.x)
                if (rbeg + r > j) S[j * R + r] = S[j * R + r] / piv;
        } else if (g == 0 && tid == 0) {
            if (*info == 0) *info = (int32_t)(r0 + j + 1);
        }
        __syncthreads();
        const int nc = nb - j - 1;
        if (nc > 0) {
            for (int e = tid; e < rows * nc; e += blockDim.x) {
                const int r = e % rows, cc = j + 1 + e / rows;
                if (rbeg + r > j) S[cc * R + r] = fma(-S[j * R + r], urow[cc], S[cc * R + r]);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < rows * nb; e += blockDim.x) {
        int r = e % rows, cc = e / rows;
        A[(i64)cc * lda + rbeg + r] = S[cc * R + r];
    }
}

// Cluster panel: the same algorithm on one thread-block cluster of CL CTAs
// (CL = 2, 4, 8 or 16), FP32 storage.  Thread t of CTA q owns rows
// q R + t + k TH (k < RPT, R = RPT TH, TH threads per CTA).  The columns not
// yet finished live in registers as a window that shifts by one column per
// step: before step j, register column c holds column j + c, so the current
// column is always register 0, every register index is a compile-time
// constant and the column loop stays rolled (a body the instruction cache
// holds).  A finished column goes straight to A.
// Per column: each warp reduces its candidate, one block barrier, every
// thread picks the CTA's candidate from the warp records, and the owner's
// warp pushes the record {key, row, the row's window} into every CTA of the
// cluster with st.async, which completes bytes on the receiver's mbarrier
// (rank 0 pushes row j the same way).  A CTA waits on its own mbarrier only:
// no cluster barrier and no remote read per column.  Each warp then picks the
// winner from the CL local records, the owners of rows j and p swap their
// windows, and every thread divides and updates its rows.  The interchange of
// the finished columns of rows j and p is deferred: after the last column,
// rank 0 applies the interchanges of the steps after each column to that
// column's entries, which yields the same matrix as interchanging whole rows
// at every step.  Same arithmetic per element as k_panel (bit-identical).
// Records and mbarriers are double-buffered by column parity: a CTA pushes
// column j only after it received every CTA's record of column j - 1, which
// each CTA sends after its block barrier of column j - 1, after its reads of
// the buffer of column j - 2.  All waits are bounded (RL_INFO_DEVICE_TIMEOUT).
constexpr int PCL_NB = 32;

struct alignas(16) PclRec {
    uint32_t key;                                 // pcl_key of the candidate
    int row;
    int pad[2];
    float v[PCL_NB];                              // the row's window: columns j .. j + 31
};
static_assert(sizeof(PclRec) == 144, "record of 9 16-byte chunks");

// Pivot key of an FP32 entry: the bits of |v| (ordered like |v|), NaN 0 --
// the same order as abs_key on the exact double of v, in 32 bits.
__device__ __forceinline__ uint32_t pcl_key(float v)
{
    const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;
}

// Largest key, lowest row among equal keys, over the warp (the order of
// kbetter); every lane gets the result.  No candidate: key 0, PANEL_NONE.
__device__ __forceinline__ void pcl_warp_best(uint32_t &key, int &row)
{
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
    row = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (uint32_t)row : 0xffffffffu);
    key = kmax;
}

__device__ __forceinline__ uint32_t pcl_mapa(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::su32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void pcl_push16(uint32_t raddr, uint4 v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(raddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar) : "memory");
}

__device__ __forceinline__ bool pcl_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of a whole warp on a local mbarrier phase; the result is the
// same in every lane.
__device__ __forceinline__ bool pcl_wait(uint64_t *bar, uint32_t parity, long long limit_ns)
{
    if (__all_sync(0xffffffffu, pcl_try(bar, parity))) return true;
    const unsigned long long t0 = tc::gtime();
    for (;;) {
        if (__all_sync(0xffffffffu, pcl_try(bar, parity))) return true;
        if (__any_sync(0xffffffffu, (long long)(tc::gtime() - t0) >= limit_ns)) return false;
    }
}

// The warp pushes the NCH 16-byte chunks at src (a slot of this CTA's
// shared memory) into the same slot of every other CTA of the cluster,
// completing bytes on each one's bar.  (Its own CTA's copy is written with
// plain stores and announced by an ordinary arrive.)
template <int CL, int NCH>
__device__ __forceinline__ void pcl_push_peers(const void *src, uint64_t *bar, int q, int lane)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int it = lane; it < (CL - 1) * NCH; it += 32) {
        const int rr = it / NCH, ch = it % NCH;
        const int r = rr + (rr >= q ? 1 : 0);
        pcl_push16(pcl_mapa(src, r) + 16u * (uint32_t)ch, s[ch], pcl_mapa(bar, r));
    }
}

__device__ __forceinline__ void pcl_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(bar)) : "memory");
}

template <int CL, int RPT, int TH>
__global__ void __launch_bounds__(TH)
k_panel_cluster(i64 m, int nb, float *A, i64 lda, int32_t *ipiv, i64 r0, int32_t *info, long long spin_ns,
                const int32_t *abort)
{
    namespace cg = cooperative_groups;
    using T = float;
    cg::cluster_group cl = cg::this_cluster();
    constexpr int R = RPT * TH;
    constexpr int NW = TH / 32;
    static_assert(NW <= 32 && PCL_NB <= TH, "one warp reduces the warp records; row j < TH");
    __shared__ PclRec recs[2][CL];                // slot r: rank r's candidate of the column
    __shared__ alignas(16) T rowj[2][PCL_NB];     // row j's window (pushed by rank 0)
    __shared__ alignas(8) uint64_t bar[2];
    __shared__ uint32_t wk[2][NW];
    __shared__ int wi[2][NW];
    __shared__ int s_p[PCL_NB];                   // p_j (rank 0, for the deferred interchanges)
    __shared__ unsigned char gsrc[PCL_NB][2 * PCL_NB];   // fix-up source slots per column
    __shared__ int s_row[2 * PCL_NB];             // fix-up slot -> row (-1: unused)
    __shared__ T fix[2 * PCL_NB][PCL_NB + 1];
    __shared__ int s_skip, s_tmo;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = (int)cl.block_rank();
    // per column: the bytes of the other CTAs' records (and of row j) arrive
    // on bar; the arrivals are tid 0's expect_tx, the local record's and (rank
    // 0) the local row j's
    const uint32_t TX = (CL - 1) * (uint32_t)sizeof(PclRec) + (q != 0 ? PCL_NB * (uint32_t)sizeof(T) : 0u);
    if (tid == 0) {
        tc::mbar_init(&bar[0], q == 0 ? 3 : 2);
        tc::mbar_init(&bar[1], q == 0 ? 3 : 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_tmo = 0;
    }
    if (q == 0 && tid == 0) s_skip = (abort && *abort != 0) ? 1 : 0;
    cl.sync();                                    // mbarriers initialised cluster-wide
    if (*cl.map_shared_rank(&s_skip, 0)) {
        cl.sync();                                // rank 0's word is read before it exits
        return;
    }
    // row indices fit an int: the cluster holds at most 16 R rows
    const int rbeg = q * R;
    const int mi = (int)m;
    T a[RPT][PCL_NB];
    int gi[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        gi[k] = rbeg + tid + k * TH;
#pragma unroll
        for (int c = 0; c < PCL_NB; ++c)
            a[k][c] = (gi[k] < mi && c < nb) ? A[(i64)c * lda + gi[k]] : T(0);
    }
    const int mn = min(mi, nb);
    int tmo = 0;
    int j = 0;
#pragma unroll 1
    for (; j < mn; ++j) {
        const int b = j & 1;
        if (tid == 0) tc::mbar_expect_tx(&bar[b], TX);
        // 1. the warp's candidate: largest |a_ij| over rows i >= j, lowest i
        // on ties (a thread's rows ascend with k)
        uint32_t bk = 0;
        int bi = PANEL_NONE;
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (gi[k] < mi && gi[k] >= j) {
                const uint32_t key = pcl_key(a[k][0]);
                if (key > bk || bi == PANEL_NONE) { bk = key; bi = gi[k]; }
            }
        pcl_warp_best(bk, bi);
        if (lane == 0) { wk[b][warp] = bk; wi[b][warp] = bi; }
        if (__syncthreads_or(tmo)) break;         // a warp ran out of its wait: every thread leaves
        // 2. the CTA's candidate (every warp reduces the warp records); the
        // owner's warp pushes its record, rank 0's warp 0 row j
        bk = lane < NW ? wk[b][lane] : 0u;
        bi = lane < NW ? wi[b][lane] : PANEL_NONE;
        pcl_warp_best(bk, bi);
        const int lr = bi != PANEL_NONE ? bi - rbeg : 0;   // owner: thread lr % TH, window lr / TH
        if (warp == (lr % TH) >> 5) {
            PclRec &mine = recs[b][q];
            if (lane == 0) { mine.key = bk; mine.row = bi; }
            if (bi != PANEL_NONE && lane == (lr & 31)) {
                const int kk = lr / TH;
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    if (k == kk) {
#pragma unroll
                        for (int c4 = 0; c4 < PCL_NB / 4; ++c4)
                            reinterpret_cast<float4 *>(mine.v)[c4] =
                                make_float4(a[k][4 * c4], a[k][4 * c4 + 1], a[k][4 * c4 + 2], a[k][4 * c4 + 3]);
                    }
            }
            __syncwarp();
            pcl_push_peers<CL, 9>(&mine, &bar[b], q, lane);
            if (lane == 0) pcl_arrive(&bar[b]);
        }
        if (q == 0 && warp == 0) {
            if (lane == j) {
#pragma unroll
                for (int c4 = 0; c4 < PCL_NB / 4; ++c4)
                    reinterpret_cast<float4 *>(rowj[b])[c4] =
                        make_float4(a[0][4 * c4], a[0][4 * c4 + 1], a[0][4 * c4 + 2], a[0][4 * c4 + 3]);
            }
            __syncwarp();
            pcl_push_peers<CL, 8>(rowj[b], &bar[b], q, lane);
            if (lane == 0) pcl_arrive(&bar[b]);
        }
        // 3. the winner over the cluster (every warp, from the local records;
        // row p sits in rank p / R)
        if (!pcl_wait(&bar[b], (uint32_t)(j >> 1) & 1u, spin_ns)) { tmo = 1; continue; }
        uint32_t k2 = recs[b][lane % CL].key;
        int ix = recs[b][lane % CL].row;
        pcl_warp_best(k2, ix);
        const int p = ix != PANEL_NONE ? ix : j;
        const T *urow = ix != PANEL_NONE ? recs[b][ix / R].v : rowj[b];   // the pivot row, columns j ..
        if (q == 0 && tid == 0) {
            ipiv[r0 + j] = (int32_t)(r0 + p + 1);
            s_p[j] = p;
        }
        const T piv = urow[0];
        // 4. swap the windows of rows j and p: their two owner threads load
        // the other row from the records
        if (p != j) {
            if (q == 0 && tid == j) {
#pragma unroll
                for (int c4 = 0; c4 < PCL_NB / 4; ++c4) {
                    const float4 v = reinterpret_cast<const float4 *>(urow)[c4];
                    a[0][4 * c4] = v.x; a[0][4 * c4 + 1] = v.y; a[0][4 * c4 + 2] = v.z; a[0][4 * c4 + 3] = v.w;
                }
            }
            const int lp = p - q * R;
            if (lp >= 0 && lp < R && tid == lp % TH) {
                const int kp = lp / TH;
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    if (k == kp) {
#pragma unroll
                        for (int c4 = 0; c4 < PCL_NB / 4; ++c4) {
                            const float4 v = reinterpret_cast<const float4 *>(rowj[b])[c4];
                            a[k][4 * c4] = v.x; a[k][4 * c4 + 1] = v.y; a[k][4 * c4 + 2] = v.z; a[k][4 * c4 + 3] = v.w;
                        }
                    }
            }
        }
        // 5. divide column j and store it, update the rest while the window
        // shifts by one (register c - 1 receives column j + c); blocks of four
        // columns past nb are skipped (j and nb are uniform), the entries past
        // nb inside a block are never stored.  Rows at or above j exist only
        // in rank 0's warp 0 (k = 0): every other warp updates all its rows
        // (those past m are never stored) without a per-element select.
        const bool dov = piv != T(0);
        bool below[RPT];
        T l[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            below[k] = dov && gi[k] < mi && gi[k] > j;
            l[k] = below[k] ? a[k][0] / piv : T(0);
            if (below[k]) a[k][0] = l[k];
            if (gi[k] < mi) A[(i64)j * lda + gi[k]] = a[k][0];
        }
        if (dov && !(q == 0 && warp == 0)) {
#pragma unroll
            for (int c4 = 0; c4 < PCL_NB / 4; ++c4) {
                if (j + 4 * c4 < nb) {
                    const float4 u4 = reinterpret_cast<const float4 *>(urow)[c4];
                    const T u[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
                    for (int e = (c4 == 0 ? 1 : 0); e < 4; ++e) {
                        const int c = 4 * c4 + e;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) a[k][c - 1] = fma(-l[k], u[e], a[k][c]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int c4 = 0; c4 < PCL_NB / 4; ++c4) {
                if (j + 4 * c4 < nb) {
                    const float4 u4 = reinterpret_cast<const float4 *>(urow)[c4];
                    const T u[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
                    for (int e = (c4 == 0 ? 1 : 0); e < 4; ++e) {
                        const int c = 4 * c4 + e;
#pragma unroll
                        for (int k = 0; k < RPT; ++k)
                            a[k][c - 1] = below[k] ? fma(-l[k], u[e], a[k][c]) : a[k][c];
                    }
                }
            }
        }
        if (!dov && q == 0 && tid == 0 && *info == 0) *info = (int32_t)(r0 + j + 1);
    }
    if (tmo) {
        s_tmo = 1;
        if (lane == 0) atomicExch(info, RL_INFO_DEVICE_TIMEOUT);
    }
    // the columns past min(m, nb) (wide panels) from the window
    if (j == mn) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (gi[k] < mi) {
#pragma unroll
                for (int c = 0; c < PCL_NB; ++c)
                    if (mn + c < nb) A[(i64)(mn + c) * lda + gi[k]] = a[k][c];
            }
    }
    cl.sync();                                    // every finished column is in A; no record is in flight
    if (q != 0 || s_tmo) return;
    // deferred interchanges of the finished columns: column c takes those of
    // the steps t = c+1 .. mn-1.  Rows 0 .. mn-1 are slots 0 .. mn-1, a row
    // p_t >= mn slot PCL_NB + (first step with that row).  With tau_t the
    // interchange of slots t and slot(p_t), the entry that ends in slot s of
    // column c starts in slot g_c(s) = tau_{c+1}(g_{c+1}(s)), g_{mn-1} = id:
    // warp 0 builds the tables g_c while the CTA gathers the slots' entries,
    // then every entry is written once from its source.
    if (warp == 0) {
        s_row[lane] = lane < mn ? lane : -1;
        const int pt = lane < mn ? s_p[lane] : -1 - lane;
        const int first = __ffs(__match_any_sync(0xffffffffu, pt)) - 1;
        s_row[PCL_NB + lane] = (lane < mn && pt >= mn && first == lane) ? pt : -1;
        const int slot = pt < mn ? pt : PCL_NB + first;    // slot of p_lane (lanes < mn)
        int g0 = lane, g1 = PCL_NB + lane;
        gsrc[mn > 0 ? mn - 1 : 0][lane] = (unsigned char)g0;
        gsrc[mn > 0 ? mn - 1 : 0][PCL_NB + lane] = (unsigned char)g1;
        for (int c = mn - 2; c >= 0; --c) {
            const int t = c + 1;
            const int st = __shfl_sync(0xffffffffu, slot, t);
            g0 = g0 == t ? st : (g0 == st ? t : g0);
            g1 = g1 == t ? st : (g1 == st ? t : g1);
            gsrc[c][lane] = (unsigned char)g0;
            gsrc[c][PCL_NB + lane] = (unsigned char)g1;
        }
    }
    __syncthreads();
    for (int e = tid; e < 2 * PCL_NB * PCL_NB; e += TH) {
        const int sl = e / PCL_NB, c = e % PCL_NB;
        const int r = s_row[sl];
        if (r >= 0 && c < mn) fix[sl][c] = __ldcg(&A[(i64)c * lda + r]);
    }
    __syncthreads();
    for (int e = tid; e < 2 * PCL_NB * PCL_NB; e += TH) {
        const int sl = e / PCL_NB, c = e % PCL_NB;
        const int r = s_row[sl];
        if (r > c && c < mn) {
            const int src = gsrc[c][sl];
            if (src != sl) A[(i64)c * lda + r] = fix[src][c];
        }
    }
}

// Launch of the cluster panel with CL CTAs; false if this device cannot
// place such a cluster (the caller then takes the cooperative kernel).
template <int CL, int RPT, int TH>
static bool launch_panel_cluster(Ctx &c, i64 m, int nb, float *A, i64 lda, int32_t *ipiv, i64 r0)
{
    auto kern = k_panel_cluster<CL, RPT, TH>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(TH);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // once per device: the cluster-size attribute and whether such a
    // cluster can be placed at all
    static std::mutex mu;
    static int state[128];                       // 0 unknown, 1 usable, 2 not
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return false;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (state[dev] == 0) {
            state[dev] = 2;
            int clusters = 0;
            if ((CL <= 8 || cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                                cudaSuccess) &&
                cudaOccupancyMaxActiveClusters(&clusters, (void *)kern, &cfg) == cudaSuccess && clusters >= 1)
                state[dev] = 1;
            (void)cudaGetLastError();
        }
        if (state[dev] != 1) return false;
    }
    int32_t *info = c.info;
    const int32_t *abort = c.abort;
    long long spin = g_params.spin_ns;
    note(c, cudaLaunchKernelEx(&cfg, kern, m, nb, A, lda, ipiv, r0, info, spin, abort));
    return true;
}

// The cluster panel serves FP32 panels of up to 16384 rows.  Fewer rows per
// CTA shorten the per-column update, which bounds the step, more CTAs
// lengthen the exchange a little, more warps per CTA hide latency: one row
// per thread on 256 threads up to 2048 rows, 512 threads above, two rows per
// thread past 8192 (measured per column on GB300).
template <typename T>
static bool panel_cluster(Ctx &c, i64 m, i64 nb, T *A, i64 lda, int32_t *ipiv, i64 r0)
{
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
    if (nb > PCL_NB || m > 16 * 1024 || m <= 0) return false;
    const int ni = (int)nb;
    if (m <= 2 * 256) return launch_panel_cluster<2, 1, 256>(c, m, ni, A, lda, ipiv, r0);
    if (m <= 4 * 256) return launch_panel_cluster<4, 1, 256>(c, m, ni, A, lda, ipiv, r0);
    if (m <= 8 * 256) return launch_panel_cluster<8, 1, 256>(c, m, ni, A, lda, ipiv, r0);
    if (m <= 8 * 512) return launch_panel_cluster<8, 1, 512>(c, m, ni, A, lda, ipiv, r0);
    if (m <= 16 * 512) return launch_panel_cluster<16, 1, 512>(c, m, ni, A, lda, ipiv, r0);
    return launch_panel_cluster<16, 2, 512>(c, m, ni, A, lda, ipiv, r0);
    }
}

template <typename T>
void getf2_panel(Ctx &c, i64 m, i64 nb, T *A, i64 lda, int32_t *ipiv, i64 r0)
{
    if (m <= 0 || nb <= 0) return;
    if (nb > panel_nbmax<T>()) { note(c, cudaErrorInvalidValue); return; }
    PanelWS *ws = reinterpret_cast<PanelWS *>(c.work);
    // CTAs: one per SM, or fewer (more rows each, fewer arrivals per column)
    int gmax = c.num_sms < PANEL_GMAX ? c.num_sms : PANEL_GMAX;
    const int cap = sizeof(T) == 8 ? g_params.panel_ctas64 : g_params.panel_ctas32;
    if (cap > 0 && cap < gmax) gmax = cap;
    i64 R = (m + gmax - 1) / gmax;
    if (R < PANEL_RMIN) R = PANEL_RMIN;
    if (R > m) R = m;
    const int G = (int)((m + R - 1) / R);
    long long spin = g_params.spin_ns;
    int32_t *info = c.info;
    note(c, smem_optin(k_panel<T>, PANEL_THREADS * panel_nbmax<T>() * sizeof(T)));
    note(c, smem_optin(k_panel_smem<T>, (size_t)PANEL_SMEM_MAX));
    // flops of an m x nb unblocked LU (leading terms): m nb^2 - nb^3/3
    Launch L(c, K_PANEL, (double)m * nb * nb - (double)nb * nb * nb / 3.0,
             2.0 * (double)m * nb * sizeof(T));
    // panels whose rows fit the registers of one cluster take the cluster kernel
    if constexpr (!is_cplx<T>::value) {
        if (g_params.panel_cluster && panel_cluster<T>(c, m, nb, A, lda, ipiv, r0)) return;
    }
    note(c, cudaMemsetAsync(&ws->counter, 0, sizeof(unsigned), c.s));
    if (R <= PANEL_THREADS) {
        int nbi = (int)nb, Ri = (int)R;
        const int32_t *abort = c.abort;
        void *args[] = {&m, &nbi, &A, &lda, &ipiv, &r0, &info, &ws, &Ri, &spin, &abort};
        note(c, cudaLaunchCooperativeKernel((const void *)k_panel<T>, dim3(G), dim3(PANEL_THREADS), args,
                                            (size_t)PANEL_THREADS * nb * sizeof(T), c.s));
        return;
    }
    if ((size_t)R * nb * sizeof(T) > PANEL_SMEM_MAX) { note(c, cudaErrorInvalidValue); return; }
    int Ri = (int)R, nbi = (int)nb;
    const int32_t *abort = c.abort;
    void *args[] = {&m, &nbi, &A, &lda, &ipiv, &r0, &info, &ws, &Ri, &spin, &abort};
    note(c, cudaLaunchCooperativeKernel((const void *)k_panel_smem<T>, dim3(G), dim3(PANEL_THREADS), args,
                                        (size_t)R * nb * sizeof(T), c.s));
}

// ----------------------------------------------------------------------------
// LASWP.
// ----------------------------------------------------------------------------
constexpr int LASWP_CHUNK = 4096;
constexpr int LASWP_THREADS = 1024;
constexpr int LASWP_V = (2 * LASWP_CHUNK + LASWP_THREADS - 1) / LASWP_THREADS;
constexpr size_t LASWP_SMEM_MAX = 200 * 1024;

// Swaps ipiv[k1..k2) (global 1-based rows, each target >= its row, k2-k1 <=
// LASWP_CHUNK) on columns [c0 + blockIdx.x*cpc, ...) of A, whose rows
// [k1, m) are involved.  Shared memory: pos[span] (span = m - k1), the
// chunk's pivots, and the list of touched rows outside [k1, k2).
template <typename T>
__global__ void __launch_bounds__(LASWP_THREADS)
k_laswp(T *A, i64 lda, i64 m, i64 c0, i64 ncols, i64 k1, i64 k2, const int32_t *ipiv, int cpc,
        const int32_t *abort)
{
    if (abort && *abort != 0) return;
    extern __shared__ int sm[];
    __shared__ int nout;
    const int span = (int)(m - k1), K = (int)(k2 - k1);
    int *pos = sm;             // pos[q]: relative row whose value ends at q
    int *pv = pos + span;      // pv[t] = ipiv[k1 + t] - 1 - k1 (relative)
    int *odst = pv + K;        // touched rows >= k2 (relative), and their sources
    int *osrc = odst + K;
    const int tid = threadIdx.x;
    for (int q = tid; q < span; q += blockDim.x) pos[q] = q;
    for (int t = tid; t < K; t += blockDim.x) pv[t] = (int)((i64)ipiv[k1 + t] - 1 - k1);
    if (tid == 0) nout = 0;
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < K; ++t) {
            const int p = pv[t];
            if (p > t && p < span) { int a = pos[t]; pos[t] = pos[p]; pos[p] = a; }
        }
    }
    __syncthreads();
    for (int t = tid; t < K; t += blockDim.x) {
        const int p = pv[t];
        if (p >= K && p < span && pos[p] != p) {
            const int prev = atomicOr(&pos[p], 0x40000000);
            if ((prev & 0x40000000) == 0) {
                const int s = atomicAdd(&nout, 1);
                odst[s] = p;
                osrc[s] = prev;
            }
        }
    }
    __syncthreads();
    const int NT = K + nout;
    const i64 cb = (i64)blockIdx.x * cpc, ce = min(ncols, cb + cpc);
    for (i64 col = cb; col < ce; ++col) {
        T *cp = A + (c0 + col) * lda + k1;
        T v[LASWP_V];
#pragma unroll
        for (int s = 0; s < LASWP_V; ++s) {
            const int t = tid + s * LASWP_THREADS;
            if (t < NT) v[s] = cp[t < K ? pos[t] : osrc[t - K]];
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < LASWP_V; ++s) {
            const int t = tid + s * LASWP_THREADS;
            if (t < NT) cp[t < K ? t : odst[t - K]] = v[s];
        }
        __syncthreads();
    }
}

// Fallback for very tall matrices: one thread per column, swaps in order.
template <typename T>
__global__ void k_laswp_seq(T *A, i64 lda, i64 c0, i64 ncols, i64 k1, i64 k2, const int32_t *ipiv,
                            const int32_t *abort)
{
    if (abort && *abort != 0) return;
    const i64 col = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    T *cp = A + (c0 + col) * lda;
    for (i64 i = k1; i < k2; ++i) {
        const i64 p = (i64)ipiv[i] - 1;
        if (p != i) { T t = cp[i]; cp[i] = cp[p]; cp[p] = t; }
    }
}

template <typename T>
void laswp(Ctx &c, T *A0, i64 lda, i64 m, i64 c0, i64 ncols, i64 k1, i64 k2, const int32_t *ipiv)
{
    if (ncols <= 0 || k2 <= k1) return;
    note(c, smem_optin(k_laswp<T>, (size_t)LASWP_SMEM_MAX));
    for (i64 kb = k1; kb < k2; kb += LASWP_CHUNK) {
        const i64 ke = (kb + LASWP_CHUNK < k2) ? kb + LASWP_CHUNK : k2;
        const size_t smem = (size_t)((m - kb) + 3 * (ke - kb)) * sizeof(int);
        // algorithmic bytes: every interchange reads and writes two rows
        Launch L(c, K_LASWP, 0.0, 4.0 * sizeof(T) * (double)(ke - kb) * (double)ncols);
        if (smem <= LASWP_SMEM_MAX) {
            i64 grid = ncols < 2 * (i64)c.num_sms ? ncols : 2 * (i64)c.num_sms;
            const i64 cpc = (ncols + grid - 1) / grid;
            grid = (ncols + cpc - 1) / cpc;
            k_laswp<T><<<(unsigned)grid, LASWP_THREADS, smem, c.s>>>(A0, lda, m, c0, ncols, kb, ke, ipiv,
                                                                     (int)cpc, c.abort);
        } else {
            k_laswp_seq<T><<<(unsigned)((ncols + 127) / 128), 128, 0, c.s>>>(A0, lda, c0, ncols, kb, ke,
                                                                           ipiv, c.abort);
        }
    }
}

// ----------------------------------------------------------------------------
// Reverse interchanges (getrs with trans = 'T': X = P^T Z).  One CTA per
// column: the column is staged in shared memory when it fits (n <= 24576),
// one thread walks the interchanges last first (ipiv staged 1024 at a time),
// then the column is written back; larger orders swap in global memory.
// ----------------------------------------------------------------------------
constexpr int LSR_MAX_N = 24576;
constexpr int LSR_IPIV = 1024;

template <typename T>
__global__ void __launch_bounds__(256)
k_laswp_rev(T *B, i64 ldb, int n, const int32_t *ipiv, int staged)
{
    extern __shared__ __align__(16) unsigned char lsr_raw[];
    __shared__ int piv[LSR_IPIV];
    T *col = reinterpret_cast<T *>(lsr_raw);
    T *bj = B + (i64)blockIdx.x * ldb;
    if (staged) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = bj[i];
    }
    for (int hi = n; hi > 0; hi -= LSR_IPIV) {
        const int lo = hi - LSR_IPIV > 0 ? hi - LSR_IPIV : 0;
        __syncthreads();
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) piv[i - lo] = ipiv[i] - 1;
        __syncthreads();
        if (threadIdx.x == 0) {
            T *v = staged ? col : bj;
            for (int i = hi - 1; i >= lo; --i) {
                const int p = piv[i - lo];
                if (p != i && p >= 0 && p < n) { const T t = v[i]; v[i] = v[p]; v[p] = t; }
            }
        }
    }
    __syncthreads();
    if (staged) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) bj[i] = col[i];
    }
}

template <typename T>
void laswp_rev(Ctx &c, T *B, i64 ldb, i64 n, i64 ncols, const int32_t *ipiv)
{
    if (n <= 1 || ncols <= 0) return;
    const bool staged = n <= LSR_MAX_N;
    const size_t smem = staged ? (size_t)n * sizeof(T) : 0;
    note(c, smem_optin(k_laswp_rev<T>, LSR_MAX_N * sizeof(T)));
    Launch L(c, K_LASWP, 0.0, 4.0 * sizeof(T) * (double)n * ncols);
    for (i64 c0 = 0; c0 < ncols; c0 += 65535) {
        const i64 nc = ncols - c0 < 65535 ? ncols - c0 : 65535;
        k_laswp_rev<T><<<(unsigned)nc, 256, smem, c.s>>>(B + c0 * ldb, ldb, (int)n, ipiv, staged ? 1 : 0);
    }
}

#define RL_INST_FACTOR(T)                                                                   \
    template void potf2<T>(Ctx &, i64, T *, i64, i64);                                     \
    template void getf2_panel<T>(Ctx &, i64, i64, T *, i64, int32_t *, i64);               \
    template void laswp<T>(Ctx &, T *, i64, i64, i64, i64, i64, i64, const int32_t *);      \
    template void laswp_rev<T>(Ctx &, T *, i64, i64, i64, const int32_t *);
RL_INST_FACTOR(double)
RL_INST_FACTOR(float)
template void getf2_panel<cplx>(Ctx &, i64, i64, cplx *, i64, int32_t *, i64);
template void laswp<cplx>(Ctx &, cplx *, i64, i64, i64, i64, i64, i64, const int32_t *);
#undef RL_INST_FACTOR

}  // namespace rl

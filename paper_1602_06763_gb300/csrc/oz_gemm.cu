// FP64 GEMM emulated on the BF16 tensor cores (the Ozaki scheme: K. Ozaki,
// T. Ogita, S. Oishi, S. M. Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012; with integer digit slices as in
// later tensor-core variants).  C := beta C + alpha op(A) op(B), FP64 in and
// out, for the FP64 updates of the recursions when the FP64 pipe is the
// bound (GB300 issues 2 FP64 FMAs per clock per SM against thousands of
// BF16 tensor MACs).
//
// Scheme.  Row i of op(A) is scaled by 2^-eA_i, eA_i = the power of two with
// max_k |a_ik| < 2^(eA_i - 1), so every scaled entry q has |q| < 1/2, and
// rounded to the 8S-bit fixed-point integer Q = round(q 2^(8S)); the same
// for column j of op(B) with eB_j.  Q is cut into S signed base-256 digits
// (the low S - 1 in [-128, 127], the top one what remains, within
// [-128, 128]), so q = sum_s d_s 2^(-8s) up to 2^(-8S-1), each exact in
// BF16.  Then
//     (op(A) op(B))_ij ~ 2^(eA_i + eB_j) sum_{L=2}^{S+1} 2^(-8L) T_L,
//     T_L = sum over digit pairs (s, t), s + t = L, of sum_k dA_s dB_t,
// the pairs with s + t > S + 1 (below 2^(-8S-8) relative) left out.  Each
// product of digits is at most 2^14 and a level has at most 8 pairs, so a
// level's sum over 128 values of k stays below 2^24: the FP32 accumulators
// of the tensor cores hold it exactly.  Every 128 values of k the level sums
// are moved out of tensor memory into two 64-bit integer accumulators per
// output (levels 2..S-3 and S-2..S+1, exact), and at the end of the tile
// converted to FP64 once.  The only roundings are the truncation of the
// digits (2^(-8S-1) relative to the row and column maxima) and the final
// conversion: per term of the sum at most 2^(-8S-2) from each side's
// truncation and (S - 1) 2^(-8S-2) from the pairs left out, so the error is
// below (S + 1) k 2^(-8S-2) 2^(eA_i + eB_j) plus the final rounding (S = 7:
// normwise of the order of an FP64 GEMM's), and integer products are exact.
//
// Kernel (one CTA per SM, persistent over 128 x 64 output tiles in groups
// of 8 row tiles for L2 reuse; 640 threads):
//   * warp 0, one lane: TMA loads.  Per 64-value k chunk, the S digit
//     planes of op(B)'s 64 columns (S x 8 KB, double-buffered) and then
//     op(A)'s S planes (16 KB each) through a 6-slot ring.
//   * warp 1 allocates 512 TMEM columns (level L's 128 x 64 FP32
//     accumulator at column 64 (L - 2)); one lane of each of warps 1-3
//     issues, per A plane s, the MMAs (M 128, N 64, K 16) with the B planes
//     t <= S + 1 - s of the levels it owns (level_mask): one issuing thread
//     does not keep the tensor pipe busy with 64-column MMAs (two are 28 %
//     faster at 8192^3; three and four no faster than two).
//   * warps 4-19: drain the level accumulators (each warp a 32-lane quarter
//     and 16 columns), accumulate the integers, and write C.
// Every mbarrier wait is bounded (RL_INFO_DEVICE_TIMEOUT on expiry).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include "internal.cuh"
#include "tc_common.cuh"

namespace rl {

namespace oz {

constexpr int BM = 128, BN = 64;
constexpr int KC = 64;                       // k values per chunk (128 bytes of BF16)
constexpr int A_TILE = BM * 128;             // 16 KB
constexpr int B_TILE = BN * 128;             // 8 KB
constexpr int A_SLOTS = 6;
constexpr int EPI_WARPS = 16;
constexpr int ISSUERS = 3;                   // MMA-issuing warps (1 .. ISSUERS)
constexpr int EPI0 = 1 + ISSUERS;            // first drain warp (0: TMA)
constexpr int THREADS = 32 * EPI0 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;
constexpr int DRAIN = 2;                     // chunks per drain (128 values of k)
constexpr int GROUP_M = 8;                   // row tiles per raster group
constexpr int EXP_NONFINITE = 4096;          // exponent marker of a row with Inf / NaN

template <int S>
constexpr int smem_bytes() { return 2 * S * B_TILE + A_SLOTS * A_TILE + 1024; }

// Exponent e with max < 2^(e-1) from the bit pattern of max >= 0: with max
// in [2^(x-1), 2^x), e = x + 1 (x = E - 1022 for a normal number of biased
// exponent E; a subnormal f 2^-1074 has x = 63 - clz(f) - 1073).
__device__ __forceinline__ int exp_of_max(unsigned long long b)
{
    if (b == 0) return 0;
    if (b >= 0x7FF0000000000000ull) return EXP_NONFINITE;
    const int E = (int)(b >> 52);
    if (E != 0) return E - 1021;
    return -1009 - __clzll((long long)b);
}

// |X| maxima of the rows of op(X) (rows x kdim) as bit patterns, folded
// with atomicMax into mx (zeroed by the caller).  TR: op(X)(r, k) =
// X[r ldx + k] (one warp per row); else X[k ldx + r] (one thread per row,
// blockIdx.y a chunk of k).
template <bool TR, bool SYM = false>
__global__ void k_absmax(int rows, int kdim, const double *X, i64 ldx, unsigned long long *mx)
{
    if (TR) {
        const i64 r = (i64)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
        const int lane = threadIdx.x & 31;
        if (r >= rows) return;
        unsigned long long best = 0;
        for (i64 k = lane; k < kdim; k += 32) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(X[r * ldx + k]) & 0x7FFFFFFFFFFFFFFFull;
            best = v > best ? v : best;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_down_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if (lane == 0) atomicMax(&mx[r], best);
    } else {
        const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
        if (r >= rows) return;
        const i64 kw = ((i64)kdim + gridDim.y - 1) / gridDim.y;
        const i64 k0 = (i64)blockIdx.y * kw, k1 = min((i64)kdim, k0 + kw);
        unsigned long long best = 0;
        for (i64 k = k0; k < k1; ++k) {
            // SYM: X symmetric with its lower triangle stored, X(r, k) = X(k, r) above it
            const double x = (!SYM || k <= r) ? X[k * ldx + r] : X[r * ldx + k];
            const unsigned long long v = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
            best = v > best ? v : best;
        }
        if (k1 > k0) atomicMax(&mx[r], best);
    }
}

// The S balanced base-256 digits of x scaled by 2^-e (|x 2^-e| < 1/2), most
// significant first, from integer operations on the bit pattern.
template <int S>
__device__ __forceinline__ void digits_of(double x, int e, int *d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const unsigned long long f = b & 0xFFFFFFFFFFFFFull;
    long long Q = 0;
    if (e != EXP_NONFINITE && (E != 0 || f != 0)) {
        const unsigned long long m = E ? (f | (1ull << 52)) : f;
        const int exu = E ? E - 1023 : -1022;
        const int sh = exu - 52 - e + 8 * S;           // Q = m 2^sh (rounded)
        unsigned long long u;
        if (sh >= 0) u = m << sh;                      // sh <= 8S - 53 (|q| < 1/2)
        else if (sh < -62) u = 0;
        else u = (m + (1ull << (-sh - 1))) >> (-sh);
        Q = (b >> 63) ? -(long long)u : (long long)u;
    }
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const long long dd = ((Q + 128) & 255) - 128;     // in [-128, 127]
        d[s] = (int)dd;
        Q = (Q - dd) >> 8;
    }
    d[0] = (int)Q;     // |Q| < 2^(8S-1) leaves |d[0]| <= 128 (it may be 128: no carry out)
}

// Digit planes P[s][r][k] (BF16, rows_p x kp per plane, zero padded) of the
// rows of op(X); TR as k_absmax.  32 x 32 tiles through shared memory so
// that the reads run along X's columns and the writes along k.
template <bool TR, int S, bool SYM = false>
__global__ void __launch_bounds__(256)
k_digits(int rows, int kdim, const double *X, i64 ldx, const unsigned long long *mx, __nv_bfloat16 *P,
         int rows_p, int kp)
{
    __shared__ double tile[32][33];
    __shared__ int erow[32];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) erow[threadIdx.x] = (r0 + (int)threadIdx.x < rows) ? exp_of_max(mx[r0 + threadIdx.x]) : 0;
    for (int yy = ty; yy < 32; yy += 8) {
        double v = 0.0;
        if (!TR && SYM && k0 > r0 + 31) {
            // a tile above the diagonal of a lower-stored symmetric X: X(r, k)
            // = X(k, r), read along k
            const int r = r0 + yy, k = k0 + tx;
            if (r < rows && k < kdim) v = X[(i64)r * ldx + k];
            tile[tx][yy] = v;                          // tile[k][r]
        } else if (!TR) {
            const int r = r0 + tx, k = k0 + yy;
            if (r < rows && k < kdim) v = (!SYM || k <= r) ? X[(i64)k * ldx + r] : X[(i64)r * ldx + k];
            tile[yy][tx] = v;                          // tile[k][r]
        } else {
            const int r = r0 + yy, k = k0 + tx;
            if (r < rows && k < kdim) v = X[(i64)r * ldx + k];
            tile[tx][yy] = v;
        }
    }
    __syncthreads();
    const size_t plane = (size_t)rows_p * (size_t)kp;
    for (int yy = ty; yy < 32; yy += 8) {
        const int r = r0 + yy, k = k0 + tx;
        if (r >= rows_p || k >= kp) continue;
        const int e = erow[yy];
        int d[S];
        digits_of<S>(tile[tx][yy], e, d);
        const size_t o = (size_t)r * kp + k;
#pragma unroll
        for (int s = 0; s < S; ++s) P[(size_t)s * plane + o] = __float2bfloat16_rn((float)d[s]);
    }
}

// Levels (bit L) owned by MMA-issuing thread i of ISSUERS: level L has
// L - 1 digit pairs per chunk; largest first, each to the thread with the
// fewest pairs so far (S = 7, 3 threads: {8, 3, 2} {7, 4} {6, 5}: 10, 9, 9).
template <int S>
__device__ __forceinline__ uint32_t level_mask(int i)
{
    int load[ISSUERS];
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < ISSUERS; ++j) load[j] = 0;
#pragma unroll
    for (int L = S + 1; L >= 2; --L) {
        int best = 0;
#pragma unroll
        for (int j = 1; j < ISSUERS; ++j) best = load[j] < load[best] ? j : best;
        load[best] += L - 1;
        if (best == i) mask |= 1u << L;
    }
    return mask;
}

// Tile t of the grouped raster: groups of GROUP_M row tiles, columns inside.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int &tm, int &tn)
{
    const int per_group = GROUP_M * tiles_n;
    const int g = t / per_group, local = t % per_group;
    const int gm0 = g * GROUP_M;
    const int rows_in = min(GROUP_M, tiles_m - gm0);
    tm = gm0 + local % rows_in;
    tn = local / rows_in;
}

template <int S, bool LOWER>
__global__ void __launch_bounds__(THREADS, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, int m, int n, int nch,
          double alpha, double beta, double *C, i64 ldc, const unsigned long long *mxA,
          const unsigned long long *mxB, int tiles_m, int tiles_n, int32_t *err, long long limit_ns,
          const int32_t *abort)
{
    using namespace tc;
    constexpr int LMAX = S + 1, LH = LMAX - 4;
    if (abort && *abort != 0) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *bbuf = base;                                  // 2 x S x B_TILE
    unsigned char *aring = base + 2 * S * B_TILE;                // A_SLOTS x A_TILE
    __shared__ uint64_t afull[A_SLOTS], aempty[A_SLOTS], bfull[2], bempty[2], tfull, tempty, final_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_err;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_total = tiles_m * tiles_n;

    if (threadIdx.x == 0) {
        // the "empty", "full accumulator" and final barriers collect one
        // commit from each MMA-issuing thread
        for (int i = 0; i < A_SLOTS; ++i) { mbar_init(&afull[i], 1); mbar_init(&aempty[i], ISSUERS); }
        for (int i = 0; i < 2; ++i) { mbar_init(&bfull[i], 1); mbar_init(&bempty[i], ISSUERS); }
        mbar_init(&tfull, ISSUERS);
        mbar_init(&tempty, EPI_WARPS);
        mbar_init(&final_bar, ISSUERS);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    auto skip = [&](int tm, int tn) { return LOWER && tm * BM + BM <= tn * BN; };

    if (warp == 0) {
        if (lane == 0) {
            int ga = 0, gb = 0;
            bool fail = false;
            for (int t = blockIdx.x; t < tiles_total && !fail; t += gridDim.x) {
                int tm, tn;
                tile_coords(t, tiles_m, tiles_n, tm, tn);
                if (skip(tm, tn)) continue;
                for (int c = 0; c < nch && !fail; ++c) {
                    const int kx = c * KC;
                    const int bb = gb & 1;
                    if (!mbar_wait(&bempty[bb], ((gb >> 1) & 1) ^ 1, limit_ns) || s_err) {
                        atomicExch(&s_err, 1);
                        fail = true;
                        break;
                    }
                    mbar_expect_tx(&bfull[bb], S * B_TILE);
                    for (int s = 0; s < S; ++s)
                        tma_load_3d(bbuf + (bb * S + s) * B_TILE, &mB, &bfull[bb], kx, tn * BN, s);
                    ++gb;
                    for (int s = 0; s < S; ++s, ++ga) {
                        const int slot = ga % A_SLOTS;
                        if (!mbar_wait(&aempty[slot], ((ga / A_SLOTS) & 1) ^ 1, limit_ns) || s_err) {
                            atomicExch(&s_err, 1);
                            fail = true;
                            break;
                        }
                        mbar_expect_tx(&afull[slot], A_TILE);
                        tma_load_3d(aring + slot * A_TILE, &mA, &afull[slot], kx, tm * BM, s);
                    }
                }
            }
            // drain: every issued copy has landed before the CTA can exit
            for (int g = (ga > A_SLOTS ? ga - A_SLOTS : 0); g < ga; ++g)
                (void)mbar_wait(&afull[g % A_SLOTS], (g / A_SLOTS) & 1, drain_limit(limit_ns));
            for (int g = (gb > 2 ? gb - 2 : 0); g < gb; ++g) (void)mbar_wait(&bfull[g & 1], (g >> 1) & 1, drain_limit(limit_ns));
        }
    } else if (warp <= ISSUERS) {
        // the issuing threads split the levels (each level's MMAs stay in one
        // thread's program order) into equal numbers of digit pairs per chunk
        if (lane == 0) {
            constexpr uint32_t ID = idesc(1u, BM, BN);      // BF16 operands, FP32 accumulators
            const uint32_t mine = level_mask<S>(warp - 1);
            int ga = 0, gb = 0, di = 0;
            bool fail = false;
            for (int t = blockIdx.x; t < tiles_total && !fail; t += gridDim.x) {
                int tm, tn;
                tile_coords(t, tiles_m, tiles_n, tm, tn);
                if (skip(tm, tn)) continue;
                for (int c = 0; c < nch && !fail; ++c) {
                    const bool first = (c % DRAIN) == 0;
                    if (first) {
                        if (!mbar_wait(&tempty, (di & 1) ^ 1, limit_ns)) { atomicExch(&s_err, 1); fail = true; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    const int bb = gb & 1;
                    if (!mbar_wait(&bfull[bb], (gb >> 1) & 1, limit_ns)) { atomicExch(&s_err, 1); fail = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t db0 = sdesc(su32(bbuf + bb * S * B_TILE));
                    for (int s = 0; s < S; ++s, ++ga) {
                        const int slot = ga % A_SLOTS;
                        if (!mbar_wait(&afull[slot], (ga / A_SLOTS) & 1, limit_ns)) {
                            atomicExch(&s_err, 1);
                            fail = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t da = sdesc(su32(aring + slot * A_TILE));
                        // digit pairs (s + 1, t + 1) with (s + 1) + (t + 1) <= S + 1: level L = s + t + 2;
                        // a descriptor's address field counts 16 bytes, so +2 per 16 values of k
                        for (int t2 = 0; t2 + s + 2 <= LMAX; ++t2) {
                            if (!((mine >> (s + t2 + 2)) & 1u)) continue;
                            const uint32_t d = tmem + (uint32_t)((s + t2) * BN);
                            const uint64_t db = db0 + (uint64_t)(t2 * (B_TILE >> 4));
#pragma unroll
                            for (int kk = 0; kk < KC / 16; ++kk) {
                                const uint32_t acc = (first && s == 0 && kk == 0) ? 0u : 1u;
                                mma<true>(d, da + 2 * kk, db + 2 * kk, ID, acc);
                            }
                        }
                        mma_commit(&aempty[slot]);
                    }
                    if (fail) break;
                    mma_commit(&bempty[bb]);
                    ++gb;
                    if ((c % DRAIN) == DRAIN - 1 || c == nch - 1) {
                        mma_commit(&tfull);
                        ++di;
                    }
                }
            }
            mma_commit(&final_bar);
            (void)mbar_wait(&final_bar, 0, drain_limit(limit_ns));
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and columns
        // 16 ((w - EPI0) / 4) .. + 15 of every level
        const int q = warp & 3, cb = (warp - EPI0) >> 2;
        const int ndrain = (nch + DRAIN - 1) / DRAIN;
        int di = 0;
        bool fail = false;
        for (int t = blockIdx.x; t < tiles_total && !fail; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            if (skip(tm, tn)) continue;
            long long H[16], Lo[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) { H[j] = 0; Lo[j] = 0; }
            for (int dd = 0; dd < ndrain; ++dd, ++di) {
                if (!mbar_wait(&tfull, di & 1, limit_ns)) atomicExch(&s_err, 1);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (s_err) { fail = true; break; }
#pragma unroll
                for (int L = 2; L <= LMAX; ++L) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((L - 2) * BN + cb * 16), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long iv = (long long)__float2int_rn(v[j]);
                        if (L <= LH) H[j] += iv * (1ll << (8 * (LH - L)));
                        else Lo[j] += iv * (1ll << (8 * (LMAX - L)));
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty)) : "memory");
            }
            if (fail) break;
            const int row = tm * BM + q * 32 + lane;
            if (row < m) {
                const int ea = exp_of_max(mxA[row]);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = tn * BN + cb * 16 + j;
                    if (col >= n || (LOWER && row < col)) continue;
                    const int eb = exp_of_max(mxB[col]);
                    double v;
                    if (ea == EXP_NONFINITE || eb == EXP_NONFINITE) v = __longlong_as_double(0x7FF8000000000000ll);
                    else v = ldexp(fma((double)H[j], 4294967296.0, (double)Lo[j]), ea + eb - 8 * LMAX);
                    double *cp = C + (i64)col * ldc + row;
                    *cp = (beta == 0.0) ? alpha * v : fma(alpha, v, beta * *cp);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
    if (threadIdx.x == 0 && s_err && err) atomicExch(err, RL_INFO_DEVICE_TIMEOUT);
}

}  // namespace oz

// ---- host side ----------------------------------------------------------------

static inline i64 rup_oz(i64 v, i64 q) { return (v + q - 1) / q * q; }
static inline size_t al1k(size_t v) { return (v + 1023) & ~(size_t)1023; }

size_t oz_work_bytes(i64 m, i64 n, i64 k, int S)
{
    const i64 mp = rup_oz(m > 0 ? m : 1, oz::BM), np = rup_oz(n > 0 ? n : 1, oz::BN);
    const i64 kp = rup_oz(k > 0 ? k : 1, oz::KC);
    return al1k((size_t)S * (size_t)mp * (size_t)kp * 2) + al1k((size_t)S * (size_t)np * (size_t)kp * 2) +
           al1k((size_t)(mp + np) * 8) + 1024;
}

// 3-D map over S planes of [rows][kp] BF16, box = one 128-byte row slice of
// box_rows rows of one plane.
static bool make_map3(CUtensorMap *map, const void *base, int rows, int kp, int S, int box_rows)
{
    auto enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)rows * (cuuint64_t)kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)oz::KC, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int S>
static void oz_split(Ctx &c, bool tr, int rows, int kdim, const double *X, i64 ldx, unsigned long long *mx,
                     __nv_bfloat16 *P, int rows_p, int kp, bool sym = false)
{
    {
        Launch L(c, K_CONVERT, 0.0, 8.0 * rows * kdim);
        if (tr) {
            oz::k_absmax<true><<<(unsigned)((rows + 7) / 8), 256, 0, c.s>>>(rows, kdim, X, ldx, mx);
        } else {
            // 64 values of k per thread: rows x k / 64 threads in flight
            const int kch = (kdim + 63) / 64 < 4096 ? (kdim + 63) / 64 : 4096;
            const dim3 g((unsigned)((rows + 255) / 256), (unsigned)kch);
            if (sym) oz::k_absmax<false, true><<<g, 256, 0, c.s>>>(rows, kdim, X, ldx, mx);
            else oz::k_absmax<false><<<g, 256, 0, c.s>>>(rows, kdim, X, ldx, mx);
        }
    }
    Launch L(c, K_CONVERT, 0.0, (8.0 + 2.0 * S) * rows * kdim);
    const dim3 g((unsigned)(kp / 32), (unsigned)(rows_p / 32));
    if (tr) oz::k_digits<true, S><<<g, 256, 0, c.s>>>(rows, kdim, X, ldx, mx, P, rows_p, kp);
    else if (sym) oz::k_digits<false, S, true><<<g, 256, 0, c.s>>>(rows, kdim, X, ldx, mx, P, rows_p, kp);
    else oz::k_digits<false, S><<<g, 256, 0, c.s>>>(rows, kdim, X, ldx, mx, P, rows_p, kp);
}

template <int S, bool LOWER>
static cudaError_t launch_oz(const CUtensorMap &a, const CUtensorMap &b, int m, int n, int nch, double alpha,
                             double beta, double *C, i64 ldc, const unsigned long long *mxA,
                             const unsigned long long *mxB, int tiles_m, int tiles_n, unsigned grid, int32_t *err,
                             long long lim, const int32_t *abort, cudaStream_t s)
{
    auto kern = oz::k_oz_gemm<S, LOWER>;
    constexpr int smem = oz::smem_bytes<S>();
    cudaError_t e = smem_optin(kern, (size_t)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, oz::THREADS, smem, s>>>(a, b, m, n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, err, lim,
                                         abort);
    return cudaGetLastError();
}

// C(m x n) := beta C + alpha op(A) op(B) with the emulation (S digit planes,
// 6..8).  lower: square C, only the lower triangle is written.  Returns
// false when the call cannot run this way (the caller takes the FP64 path).
bool oz_gemm(Ctx &c, int S, bool ta, bool tb, i64 m, i64 n, i64 k, double alpha, const double *A, i64 lda,
             const double *B, i64 ldb, double beta, double *C, i64 ldc, bool lower, void *work, size_t lwork)
{
    if (S < 6 || S > 8 || m <= 0 || n <= 0 || k <= 0) return false;
    if (m > (1 << 30) || n > (1 << 30) || k > (1 << 21)) return false;
    if (work == nullptr || lwork < oz_work_bytes(m, n, k, S)) return false;
    const i64 mp = rup_oz(m, oz::BM), np = rup_oz(n, oz::BN), kp = rup_oz(k, oz::KC);
    char *w = reinterpret_cast<char *>(((uintptr_t)work + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(w);
    char *p = w + al1k((size_t)S * mp * kp * 2);
    __nv_bfloat16 *Bp = reinterpret_cast<__nv_bfloat16 *>(p);
    p += al1k((size_t)S * np * kp * 2);
    unsigned long long *mxA = reinterpret_cast<unsigned long long *>(p);
    unsigned long long *mxB = mxA + mp;
    {
        note(c, cudaMemsetAsync(mxA, 0, (size_t)(mp + np) * 8, c.s));
        // rows of op(A): A's rows (ta = false) or columns; rows of op(B)^T:
        // B's columns (tb = false) or rows
        switch (S) {
        case 6: oz_split<6>(c, ta, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp);
                oz_split<6>(c, !tb, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
        case 7: oz_split<7>(c, ta, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp);
                oz_split<7>(c, !tb, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
        default: oz_split<8>(c, ta, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp);
                 oz_split<8>(c, !tb, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
        }
    }
    CUtensorMap ma, mb;
    if (!make_map3(&ma, Ap, (int)mp, (int)kp, S, oz::BM) || !make_map3(&mb, Bp, (int)np, (int)kp, S, oz::BN)) {
        note(c, cudaErrorInvalidValue);
        return true;
    }
    const int tiles_m = (int)(mp / oz::BM), tiles_n = (int)(np / oz::BN);
    const int tiles_total = tiles_m * tiles_n;
    const unsigned grid = (unsigned)(c.oz_dynamic || tiles_total < c.num_sms ? tiles_total : c.num_sms);
    const int nch = (int)(kp / oz::KC);
    const double flops = lower ? (double)k * n * (n + 1) : 2.0 * m * n * k;
    Launch L(c, lower ? K_SYRK : K_GEMM, flops, 0.0);
    const long long lim = g_params.spin_ns;
    cudaError_t e;
#define RL_OZ(SS)                                                                                           \
    (lower ? launch_oz<SS, true>(ma, mb, (int)m, (int)n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, \
                                 grid, c.info, lim, c.abort, c.s)                                            \
           : launch_oz<SS, false>(ma, mb, (int)m, (int)n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, \
                                  grid, c.info, lim, c.abort, c.s))
    if (S == 6) e = RL_OZ(6);
    else if (S == 7) e = RL_OZ(7);
    else e = RL_OZ(8);
#undef RL_OZ
    note(c, e);
    return true;
}

// ---- products with a matrix sliced once ----------------------------------------
// The precision form multiplies the same A by many right-hand-side blocks:
// its digit planes and row exponents are made once (oz_prepare) and reused
// by every product (oz_gemm_planes), which slices only the thin operand.

size_t oz_planes_bytes(i64 m, i64 k, int S)
{
    const i64 mp = rup_oz(m > 0 ? m : 1, oz::BM), kp = rup_oz(k > 0 ? k : 1, oz::KC);
    return al1k((size_t)S * (size_t)mp * (size_t)kp * 2) + al1k((size_t)mp * 8) + 1024;
}

// Digit planes of the m x k matrix A (its rows); sym: A symmetric with the
// lower triangle stored (m = k), each row read across the diagonal.
bool oz_prepare(Ctx &c, int S, bool sym, i64 m, i64 k, const double *A, i64 lda, void *planes)
{
    if (S < 6 || S > 8 || m <= 0 || k <= 0 || m > (1 << 30) || k > (1 << 21) || planes == nullptr) return false;
    const i64 mp = rup_oz(m, oz::BM), kp = rup_oz(k, oz::KC);
    char *w = reinterpret_cast<char *>(((uintptr_t)planes + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(w);
    unsigned long long *mxA = reinterpret_cast<unsigned long long *>(w + al1k((size_t)S * mp * kp * 2));
    note(c, cudaMemsetAsync(mxA, 0, (size_t)mp * 8, c.s));
    switch (S) {
    case 6: oz_split<6>(c, false, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp, sym); break;
    case 7: oz_split<7>(c, false, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp, sym); break;
    default: oz_split<8>(c, false, (int)m, (int)k, A, lda, mxA, Ap, (int)mp, (int)kp, sym); break;
    }
    return true;
}

// C (m x n) := beta C + alpha A B with A's planes from oz_prepare (m x k) and
// B (k x n, column-major) sliced into work (oz_work_bytes(0, n, k, S)).
bool oz_gemm_planes(Ctx &c, int S, i64 m, i64 n, i64 k, double alpha, const void *planes, const double *B,
                    i64 ldb, double beta, double *C, i64 ldc, void *work, size_t lwork)
{
    if (S < 6 || S > 8 || m <= 0 || n <= 0 || k <= 0 || m > (1 << 30) || n > (1 << 30) || k > (1 << 21))
        return false;
    if (work == nullptr || lwork < oz_work_bytes(1, n, k, S) || planes == nullptr) return false;
    const i64 mp = rup_oz(m, oz::BM), np = rup_oz(n, oz::BN), kp = rup_oz(k, oz::KC);
    const char *pa = reinterpret_cast<const char *>(((uintptr_t)planes + 1023) & ~(uintptr_t)1023);
    const __nv_bfloat16 *Ap = reinterpret_cast<const __nv_bfloat16 *>(pa);
    const unsigned long long *mxA =
        reinterpret_cast<const unsigned long long *>(pa + al1k((size_t)S * mp * kp * 2));
    char *w = reinterpret_cast<char *>(((uintptr_t)work + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16 *Bp = reinterpret_cast<__nv_bfloat16 *>(w);
    unsigned long long *mxB = reinterpret_cast<unsigned long long *>(w + al1k((size_t)S * np * kp * 2));
    note(c, cudaMemsetAsync(mxB, 0, (size_t)np * 8, c.s));
    switch (S) {
    case 6: oz_split<6>(c, true, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
    case 7: oz_split<7>(c, true, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
    default: oz_split<8>(c, true, (int)n, (int)k, B, ldb, mxB, Bp, (int)np, (int)kp); break;
    }
    CUtensorMap ma, mb;
    if (!make_map3(&ma, Ap, (int)mp, (int)kp, S, oz::BM) || !make_map3(&mb, Bp, (int)np, (int)kp, S, oz::BN)) {
        note(c, cudaErrorInvalidValue);
        return true;
    }
    const int tiles_m = (int)(mp / oz::BM), tiles_n = (int)(np / oz::BN);
    const int tiles_total = tiles_m * tiles_n;
    const unsigned grid = (unsigned)(tiles_total < c.num_sms ? tiles_total : c.num_sms);
    const int nch = (int)(kp / oz::KC);
    Launch L(c, K_RESID, 2.0 * m * n * k, 2.0 * S * (double)m * k);
    const long long lim = g_params.spin_ns;
    cudaError_t e;
    if (S == 6)
        e = launch_oz<6, false>(ma, mb, (int)m, (int)n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, grid,
                                c.info, lim, c.abort, c.s);
    else if (S == 7)
        e = launch_oz<7, false>(ma, mb, (int)m, (int)n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, grid,
                                c.info, lim, c.abort, c.s);
    else
        e = launch_oz<8, false>(ma, mb, (int)m, (int)n, nch, alpha, beta, C, ldc, mxA, mxB, tiles_m, tiles_n, grid,
                                c.info, lim, c.abort, c.s);
    note(c, e);
    return true;
}

}  // namespace rl

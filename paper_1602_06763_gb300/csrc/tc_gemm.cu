// Tensor-core (tcgen05) GEMM for the FP32 working storage of the precision
// form: C(m x n) = C + alpha * op(A) op(B), C in FP32, the products on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory.
//
// Operand precision (rl_prec): TF32 (one MMA), BF16 / FP16 (one MMA on
// 16-bit copies), or 3xTF32 (a = a_hi + a_lo split, three MMAs
// a_hi b_hi + a_hi b_lo + a_lo b_hi, close to FP32 accuracy).
//
// Structure (one CTA per 128 x 256 output tile, 192 threads):
//   * op(A) and op(B) are first packed into K-major tiles (rows of K
//     contiguous, zero padded) of the operand type by a bandwidth-bound pack
//     kernel; this also transposes the column-major A block.
//   * warp 0: one lane issues TMA loads (cp.async.bulk.tensor, 128-byte
//     swizzle) of A and B k-slices into a 4-stage shared-memory ring, each
//     stage guarded by a "full" and an "empty" mbarrier.
//   * warp 1: allocates 256 TMEM columns; one lane issues tcgen05.mma
//     (M = 128, N = 256, K = 32 bytes per instruction) and tcgen05.commit to
//     release each stage and, at the end, to signal the epilogue.
//   * warps 2-5: read the accumulator with tcgen05.ld (each warp its own
//     32-lane quarter) and update C with coalesced stores.
// Every mbarrier wait is bounded; a wait that runs out sets the error word
// (RL_INFO_DEVICE_TIMEOUT) and the CTA drains its copies, frees TMEM and
// returns.
#include <mutex>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "internal.cuh"
#include "tc_common.cuh"

namespace rl {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int KB = 128;                     // bytes of K per stage (one swizzle row)
constexpr int THREADS = 192;
constexpr int A_TILE = BM * KB;             // 16 KB
constexpr int B_TILE = BN * KB;             // 32 KB
constexpr int TMEM_COLS = 256;

// Persistent tensor-core GEMM.  CTA b takes tiles b, b + gridDim.x, ...
// (row tiles fastest, so CTAs running at the same time share the B tile).
// NSPLIT operand planes per side (1, or 2 for the hi/lo split: three MMAs
// hi*hi + hi*lo + lo*hi per k-chunk).  The accumulator is double-buffered in
// TMEM (2 x 256 columns): the MMA warp fills one buffer while the epilogue
// warps drain the other, so a tile's read-modify-write of C overlaps the
// next tile's main loop.
// FMT: operand format of the instruction descriptor (0 FP16, 1 BF16, 2 TF32).
//
// CL = 2: the CTAs run as clusters of two that take pairs of row tiles
// (2p, 2p + 1) of one column tile, so both need the same B tile: each CTA
// loads its own A tile and one half (128 rows) of B, multicast into both
// CTAs' shared memory; a stage is free again only when the MMAs of both CTAs
// have read it (each CTA's MMA commits to the "empty" barriers of both).
// Each CTA reads 32 KB instead of 48 KB of operands per 128 bytes of K.
template <int FMT, int NSPLIT, int STAGES, bool LOWER, int CL>
__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
          const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
          int m, int n, int nkb, float alpha, float *C, i64 ldc, int tiles_m, int tiles_total,
          int32_t *err, long long limit_ns, const int32_t *abort)
{
    constexpr bool F16KIND = FMT < 2;
    constexpr int STAGE = NSPLIT * (A_TILE + B_TILE);
    if (abort && *abort != 0) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the stage ring
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull[2], tempty[2], final_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_err;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], CL); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        mbar_init(&final_bar, 1);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(2 * TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (CL > 1) cluster_sync_all();          // the peer's barriers are initialised before any remote arrive
    else __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // The work list: single tiles (CL = 1; row tiles fastest, so CTAs
    // running at the same time share the B tile) or row-tile pairs (CL = 2;
    // this CTA takes the pair's row tile of its rank).  A pair's second row
    // tile may lie past the last one: it is computed on the zero fill of the
    // A copies and writes nothing.
    const int rank = CL > 1 ? (int)(blockIdx.x % CL) : 0;
    const int pairs_m = (tiles_m + CL - 1) / CL;
    const int utotal = pairs_m * (tiles_total / tiles_m);
    const int ustart = (int)blockIdx.x / CL, ustep = (int)gridDim.x / CL;
    auto coords = [&](int u, int &tm, int &tn) {
        tm = CL * (u % pairs_m) + rank;
        tn = u / pairs_m;
    };
    // lower-triangle updates: work units entirely above the diagonal have no
    // work (every role of both CTAs applies the same rule on the unit's last
    // row tile, so all see the same sequence)
    auto skip = [&](int u) {
        const int tmax = CL * (u % pairs_m) + CL - 1, tn = u / pairs_m;
        return LOWER && tmax * BM + BM <= tn * BN;
    };

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;                                  // ring position across tiles
            bool fail = false;
            for (int u = ustart; u < utotal && !fail; u += ustep) {
                if (skip(u)) continue;
                int tm, tn;
                coords(u, tm, tn);
                const int m0 = tm * BM, n0 = tn * BN;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (!mbar_wait(&empty_bar[s], ((g / STAGES) & 1) ^ 1, limit_ns) || s_err) {
                        atomicExch(&s_err, 1);
                        fail = true;
                        break;
                    }
                    unsigned char *st = base + s * STAGE;
                    mbar_expect_tx(&full_bar[s], STAGE);
                    const int kx = kb * (F16KIND ? 64 : 32);   // 128 bytes of K per stage
                    tma_load_2d(st, &mA0, &full_bar[s], kx, m0);
                    if (CL == 1) {
                        tma_load_2d(st + A_TILE, &mB0, &full_bar[s], kx, n0);
                    } else {
                        // this CTA's half of B (the maps' box is BN / 2 rows), into both CTAs
                        constexpr int HB = B_TILE / 2;
                        tma_load_2d_mc(st + A_TILE + rank * HB, &mB0, &full_bar[s], kx, n0 + rank * (BN / 2), 0x3);
                    }
                    if (NSPLIT == 2) {
                        tma_load_2d(st + A_TILE + B_TILE, &mA1, &full_bar[s], kx, m0);
                        if (CL == 1) {
                            tma_load_2d(st + 2 * A_TILE + B_TILE, &mB1, &full_bar[s], kx, n0);
                        } else {
                            constexpr int HB = B_TILE / 2;
                            tma_load_2d_mc(st + 2 * A_TILE + B_TILE + rank * HB, &mB1, &full_bar[s], kx,
                                           n0 + rank * (BN / 2), 0x3);
                        }
                    }
                }
            }
            // drain: every issued copy has landed before the CTA can exit
            for (int gg = (g > STAGES ? g - STAGES : 0); gg < g; ++gg)
                (void)mbar_wait(&full_bar[gg % STAGES], (gg / STAGES) & 1, drain_limit(limit_ns));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = idesc((uint32_t)FMT, BM, BN);
            int g = 0, i = 0;
            bool fail = false;
            for (int u = ustart; u < utotal && !fail; u += ustep) {
                if (skip(u)) continue;
                const int b = i & 1;
                if (!mbar_wait(&tempty[b], ((i >> 1) & 1) ^ 1, limit_ns)) { atomicExch(&s_err, 1); break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * TMEM_COLS);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (!mbar_wait(&full_bar[s], (g / STAGES) & 1, limit_ns)) {
                        atomicExch(&s_err, 1);
                        fail = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = su32(base + s * STAGE);
                    const uint32_t sb = sa + A_TILE;
#pragma unroll
                    for (int kk = 0; kk < KB / 32; ++kk) {
                        const uint32_t acc = (kb | kk) ? 1u : 0u;
                        mma<F16KIND>(d, sdesc(sa + kk * 32), sdesc(sb + kk * 32), ID, acc);
                        if (NSPLIT == 2) {
                            const uint32_t sa1 = sa + A_TILE + B_TILE, sb1 = sa + 2 * A_TILE + B_TILE;
                            mma<F16KIND>(d, sdesc(sa + kk * 32), sdesc(sb1 + kk * 32), ID, 1u);
                            mma<F16KIND>(d, sdesc(sa1 + kk * 32), sdesc(sb + kk * 32), ID, 1u);
                        }
                    }
                    if (CL == 1) mma_commit(&empty_bar[s]);
                    else mma_commit_mc(&empty_bar[s], 0x3);    // the stage holds B halves of both CTAs
                }
                if (!fail) mma_commit(&tfull[b]);
                ++i;
            }
            // every issued MMA has completed before TMEM can be released
            mma_commit(&final_bar);
            (void)mbar_wait(&final_bar, 0, drain_limit(limit_ns));
        }
    } else {
        // epilogue: warps 2..5 -> TMEM lane quarters (warp % 4)
        const int q = warp & 3;
        int i = 0;
        for (int u = ustart; u < utotal; u += ustep) {
            if (skip(u)) continue;
            const int b = i & 1;
            int tm, tn;
            coords(u, tm, tn);
            const int m0 = tm * BM, n0 = tn * BN;
            const int row = m0 + q * 32 + lane;
            if (!mbar_wait(&tfull[b], (i >> 1) & 1, limit_ns)) atomicExch(&s_err, 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (s_err) break;
            for (int c = 0; c < BN; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TMEM_COLS + c), v);
                if (row < m) {
                    float old[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c + j;
                        old[j] = (col < n && (!LOWER || row >= col)) ? C[(i64)col * ldc + row] : 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c + j;
                        if (col < n && (!LOWER || row >= col)) C[(i64)col * ldc + row] = fmaf(alpha, v[j], old[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[b])) : "memory");
            ++i;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // a CTA leaves only when its peer no longer copies into it or arrives on its barriers
    if (CL > 1) cluster_sync_all();
    else __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS));
    }
    if (threadIdx.x == 0 && s_err && err) atomicExch(err, RL_INFO_DEVICE_TIMEOUT);
}

// Pack op(X) (rows x kdim, X column-major with leading dimension ldx, op =
// transpose when TR) into P[rows_p][kp] row-major, zero padded, converted to
// the operand type.  SPLIT: plane 0 = hi (TF32-rounded), plane 1 = lo.
template <typename OT, bool TR, int SPLIT>
__global__ void k_pack(int rows, int kdim, const float *X, i64 ldx, OT *P, int rows_p, int kp, i64 plane)
{
    __shared__ float tile[32][33];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    // load a 32 x 32 block of op(X): element (r, k)
    for (int yy = ty; yy < 32; yy += 8) {
        int r, k;
        float v = 0.0f;
        if (!TR) {            // op(X)(r,k) = X[k*ldx + r], coalesced along r
            r = r0 + tx; k = k0 + yy;
            if (r < rows && k < kdim) v = X[(i64)k * ldx + r];
            tile[yy][tx] = v;                 // tile[k][r]
        } else {              // op(X)(r,k) = X[r*ldx + k], coalesced along k
            r = r0 + yy; k = k0 + tx;
            if (r < rows && k < kdim) v = X[(i64)r * ldx + k];
            tile[tx][yy] = v;                 // tile[k][r]
        }
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int r = r0 + yy, k = k0 + tx;
        if (r >= rows_p || k >= kp) continue;
        const float v = tile[tx][yy];
        const i64 o = (i64)r * kp + k;
        if (SPLIT == 2) {
            uint32_t hb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
            const float hi = __uint_as_float(hb);
            P[o] = (OT)hi;
            P[plane + o] = (OT)(v - hi);
        } else if (sizeof(OT) == 4) {
            uint32_t hb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
            P[o] = (OT)__uint_as_float(hb);
        } else {
            P[o] = (OT)v;
        }
    }
}

}  // namespace tc

// ---- host side ----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over a row-major [rows][kp] operand plane, box = one stage tile.
static bool make_map(CUtensorMap *map, const void *base, bool f16, int rows, int kp, int box_rows)
{
    auto enc = tmap_encoder();
    if (!enc) return false;
    const int esz = f16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * esz};
    cuuint32_t box[2] = {(cuuint32_t)(tc::KB / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    // the copy moves bytes; a 16-bit map serves both BF16 and FP16 planes
    CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static inline i64 rup(i64 v, i64 q) { return (v + q - 1) / q * q; }

size_t tc_work_bytes(i64 m, i64 n, i64 k, int prec)
{
    if (prec == RL_PREC_FP32) return 0;
    const bool f16 = (prec == RL_PREC_BF16 || prec == RL_PREC_FP16S);
    const int esz = f16 ? 2 : 4, split = (prec == RL_PREC_TF32X3) ? 2 : 1;
    const i64 kp = rup(k > 0 ? k : 1, tc::KB / esz);
    const i64 mp = rup(m > 0 ? m : 1, tc::BM), np = rup(n > 0 ? n : 1, tc::BN);
    return (size_t)split * ((size_t)mp + (size_t)np) * (size_t)kp * esz + 2048;
}

template <int FMT, int NSPLIT, int STAGES, bool LOWER, int CL>
static cudaError_t launch_tc(const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                             const CUtensorMap &b1, int m, int n, int nkb, float alpha, float *C, i64 ldc,
                             int tiles_m, int tiles_total, unsigned grid, int32_t *err, long long lim,
                             const int32_t *abort, cudaStream_t s)
{
    auto kern = tc::k_tc_gemm<FMT, NSPLIT, STAGES, LOWER, CL>;
    const int smem = STAGES * NSPLIT * (tc::A_TILE + tc::B_TILE) + 1024;
    cudaError_t e = smem_optin(kern, (size_t)smem);
    if (e != cudaSuccess) return e;
    if (CL == 1) {
        kern<<<grid, tc::THREADS, smem, s>>>(a0, a1, b0, b1, m, n, nkb, alpha, C, ldc, tiles_m, tiles_total, err,
                                             lim, abort);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a0, a1, b0, b1, m, n, nkb, alpha, C, ldc, tiles_m, tiles_total, err,
                              lim, abort);
}

// Whether clusters of two CTAs of the tensor-core GEMM (largest shared-memory
// footprint) can be placed on this device; asked once per device.
static bool tc_pairs_ok()
{
    static std::mutex mu;
    static int state[128];                   // 0 unknown, 1 yes, 2 no
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (state[dev] == 0) {
        state[dev] = 2;
        auto kern = tc::k_tc_gemm<1, 1, 4, false, 2>;
        const int smem = 4 * (tc::A_TILE + tc::B_TILE) + 1024;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(tc::THREADS);
        cfg.dynamicSmemBytes = (size_t)smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (smem_optin(kern, (size_t)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&clusters, (void *)kern, &cfg) == cudaSuccess && clusters >= 1)
            state[dev] = 1;
        (void)cudaGetLastError();
    }
    return state[dev] == 1;
}

// C(m x n) += alpha op(A) op(B) on the tensor cores; lower: square C, only
// tiles on or below the diagonal and only elements i >= j are written.
// Returns false when the operation cannot run here (caller falls back).
bool tc_gemm(Ctx &c, int prec, bool ta, bool tb, i64 m, i64 n, i64 k, float alpha, const float *A,
             i64 lda, const float *B, i64 ldb, float *C, i64 ldc, bool lower, void *work, size_t lwork)
{
    if (prec == RL_PREC_FP32 || m <= 0 || n <= 0 || k <= 0) return false;
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2) return false;
    const bool f16 = (prec == RL_PREC_BF16 || prec == RL_PREC_FP16S);
    const int esz = f16 ? 2 : 4, split = (prec == RL_PREC_TF32X3) ? 2 : 1;
    const i64 kp = rup(k, tc::KB / esz);
    const i64 mp = rup(m, tc::BM), np = rup(n, tc::BN);
    if (lwork < tc_work_bytes(m, n, k, prec) || work == nullptr) return false;
    char *w = reinterpret_cast<char *>(((uintptr_t)work + 1023) & ~(uintptr_t)1023);
    const i64 aplane = mp * kp, bplane = np * kp;
    char *Ap = w;
    char *Bp = w + (size_t)split * aplane * esz;

    // pack op(A) -> [mp][kp], op(B)^T -> [np][kp] (B's rows are op(B)'s columns)
    {
        dim3 g((unsigned)(kp / 32 + (kp % 32 ? 1 : 0)), (unsigned)(mp / 32));
        dim3 gb((unsigned)(kp / 32 + (kp % 32 ? 1 : 0)), (unsigned)(np / 32));
        Launch L(c, K_CONVERT, 0.0, (double)(m + n) * k * (4 + esz * split));
        if (prec == RL_PREC_BF16) {
            if (!ta) tc::k_pack<__nv_bfloat16, false, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (__nv_bfloat16 *)Ap, (int)mp, (int)kp, 0);
            else tc::k_pack<__nv_bfloat16, true, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (__nv_bfloat16 *)Ap, (int)mp, (int)kp, 0);
            if (!tb) tc::k_pack<__nv_bfloat16, true, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (__nv_bfloat16 *)Bp, (int)np, (int)kp, 0);
            else tc::k_pack<__nv_bfloat16, false, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (__nv_bfloat16 *)Bp, (int)np, (int)kp, 0);
        } else if (prec == RL_PREC_FP16S) {
            if (!ta) tc::k_pack<__half, false, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (__half *)Ap, (int)mp, (int)kp, 0);
            else tc::k_pack<__half, true, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (__half *)Ap, (int)mp, (int)kp, 0);
            if (!tb) tc::k_pack<__half, true, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (__half *)Bp, (int)np, (int)kp, 0);
            else tc::k_pack<__half, false, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (__half *)Bp, (int)np, (int)kp, 0);
        } else if (split == 2) {
            if (!ta) tc::k_pack<float, false, 2><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (float *)Ap, (int)mp, (int)kp, aplane);
            else tc::k_pack<float, true, 2><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (float *)Ap, (int)mp, (int)kp, aplane);
            if (!tb) tc::k_pack<float, true, 2><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (float *)Bp, (int)np, (int)kp, bplane);
            else tc::k_pack<float, false, 2><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (float *)Bp, (int)np, (int)kp, bplane);
        } else {
            if (!ta) tc::k_pack<float, false, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (float *)Ap, (int)mp, (int)kp, 0);
            else tc::k_pack<float, true, 1><<<g, 256, 0, c.s>>>((int)m, (int)k, A, lda, (float *)Ap, (int)mp, (int)kp, 0);
            if (!tb) tc::k_pack<float, true, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (float *)Bp, (int)np, (int)kp, 0);
            else tc::k_pack<float, false, 1><<<gb, 256, 0, c.s>>>((int)n, (int)k, B, ldb, (float *)Bp, (int)np, (int)kp, 0);
        }
    }
    const int nkb = (int)(kp / (tc::KB / esz));
    const int tiles_m = (int)(mp / tc::BM), tiles_n = (int)(np / tc::BN);
    const int tiles_total = tiles_m * tiles_n;
    // row-tile pairs on clusters of two when there are pairs to share B and
    // enough of them to fill the GPU
    const int pairs = ((tiles_m + 1) / 2) * tiles_n;
    const int CLn = (g_params.tc_pairs && tiles_m >= 2 && 2 * pairs >= c.num_sms && tc_pairs_ok()) ? 2 : 1;
    CUtensorMap a0, a1, b0, b1;
    bool ok = make_map(&a0, Ap, f16, (int)mp, (int)kp, tc::BM) &&
              make_map(&b0, Bp, f16, (int)np, (int)kp, tc::BN / CLn);
    if (split == 2)
        ok = ok && make_map(&a1, Ap + (size_t)aplane * esz, f16, (int)mp, (int)kp, tc::BM) &&
             make_map(&b1, Bp + (size_t)bplane * esz, f16, (int)np, (int)kp, tc::BN / CLn);
    else {
        a1 = a0;
        b1 = b0;
    }
    if (!ok) { note(c, cudaErrorInvalidValue); return true; }
    // persistent CTAs (one per SM) walk the work list; lower-triangle updates
    // skip the tiles above the diagonal and mask the diagonal ones
    unsigned grid;
    if (CLn == 1) grid = (unsigned)(tiles_total < c.num_sms ? tiles_total : c.num_sms);
    else grid = 2u * (unsigned)(pairs < c.num_sms / 2 ? pairs : c.num_sms / 2);
    const double flops = lower ? (double)k * n * (n + 1) : 2.0 * m * n * k;
    Launch L(c, lower ? K_SYRK : K_GEMM, flops, 0.0);
    cudaError_t e;
    const long long lim = g_params.spin_ns;
#define RL_TC1(FMT, NS, ST, CLX)                                                                        \
    (lower ? launch_tc<FMT, NS, ST, true, CLX>(a0, a1, b0, b1, (int)m, (int)n, nkb, alpha, C, ldc, tiles_m, \
                                               tiles_total, grid, c.info, lim, c.abort, c.s)           \
           : launch_tc<FMT, NS, ST, false, CLX>(a0, a1, b0, b1, (int)m, (int)n, nkb, alpha, C, ldc,      \
                                                tiles_m, tiles_total, grid, c.info, lim, c.abort, c.s))
#define RL_TC(FMT, NS, ST) (CLn == 2 ? RL_TC1(FMT, NS, ST, 2) : RL_TC1(FMT, NS, ST, 1))
    if (prec == RL_PREC_FP16S) e = RL_TC(0, 1, 4);
    else if (prec == RL_PREC_BF16) e = RL_TC(1, 1, 4);
    else if (split == 2) e = RL_TC(2, 2, 2);
    else e = RL_TC(2, 1, 4);
#undef RL_TC
#undef RL_TC1
    note(c, e);
    return true;
}

}  // namespace rl

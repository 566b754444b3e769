"""Per-kernel timing of the library's building blocks through the C ABI.

Used to profile one kernel at a time (an ncu capture of a single launch on a
case that still exceeds L2) and to sweep tuning parameters.  Inputs are
random device tensors; results are not checked here (the tests do that).

    python -m paper_1602_06763_gb300.kbench --case dgemm --n 4096 --reps 3
    python -m paper_1602_06763_gb300.kbench --case getrf --n 8192 --nb 32

Prints one JSON line per case: median milliseconds, GFLOP/s (LAWN 41 flop
counts for the factorizations, 2mnk for GEMM) and the per-kernel trace.
"""
from __future__ import annotations

import argparse
import json
import statistics


def main():
    import torch
    from . import relgpu as r

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", required=True,
                    choices=["dgemm", "dsyrk", "dtrsm", "potrf", "getrf", "trtri", "lauum", "panel",
                             "sgemm_tc", "dsgesv", "dsposv", "getrs", "potrs", "sgetrs", "sgemm", "laswp",
                             "zpotrf", "zgetrf", "sgetrf_tc", "spotrf_tc", "vbatched_potrf", "vbatched_getrf"])
    ap.add_argument("--count", type=int, default=20000, help="vbatched cases: matrices (orders uniform 8..256)")
    ap.add_argument("--prec", type=int, default=1, help="operand precision (rl_prec) of sgemm_tc / dsgesv")
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--cond", type=float, default=1e6)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--m", type=int, default=0, help="rows (panel case); default n")
    ap.add_argument("--k", type=int, default=0, help="inner dimension (dgemm/dsyrk); default n")
    ap.add_argument("--nb", type=int, default=0, help="dgetrf panel width")
    ap.add_argument("--c", type=int, default=0, help="dpotrf / dtrtri crossover")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--trace", action="store_true")
    ap.add_argument("--panel-ctas", type=int, default=0, help="LU panel CTAs (RL_PARAM_PANEL_CTAS value)")
    ap.add_argument("--fp32", action="store_true", help="panel/getrf cases: FP32 storage (rl_sgetrf)")
    ap.add_argument("--tri-lanes", type=int, default=0, help="lanes per vector of the triangle leaf kernels (2 or 4)")
    ap.add_argument("--oz", type=int, default=0,
                    help="dgemm / dsyrk / potrf / getrf: FP64 updates emulated with this many BF16 digit planes")
    ap.add_argument("--oz-min", type=int, default=0, help="RL_PARAM_OZ_MIN value for the --oz cases")
    ap.add_argument("--uplo", default="L", help="potrf / trtri / lauum / zpotrf: triangle")
    ap.add_argument("--flow", type=int, default=1, help="getrs/potrs: 1 = one-launch flow solve, 0 = recursive")
    ap.add_argument("--panel-cluster", type=int, default=-1, help="RL_PARAM_PANEL_CLUSTER value (0 or 1)")
    ap.add_argument("--tc-pairs", type=int, default=-1, help="RL_PARAM_TC_PAIRS value (0 or 1)")
    ap.add_argument("--graph", action="store_true",
                    help="time replays of the call captured once into a CUDA graph (after an eager warm-up)")
    a = ap.parse_args()

    if a.nb:
        r.check(r.rl_set_param(r.RL_PARAM_GETRF_PANEL, a.nb))
    if a.panel_cluster >= 0:
        r.check(r.rl_set_param(r.RL_PARAM_PANEL_CLUSTER, a.panel_cluster))
    if a.tc_pairs >= 0:
        r.check(r.rl_set_param(r.RL_PARAM_TC_PAIRS, a.tc_pairs))
    if a.oz_min:
        r.check(r.rl_set_param(r.RL_PARAM_OZ_MIN, a.oz_min))
    if a.panel_ctas:
        r.check(r.rl_set_param(r.RL_PARAM_PANEL_CTAS, a.panel_ctas))
    if a.tri_lanes:
        r.check(r.rl_set_param(r.RL_PARAM_TRI_LANES, a.tri_lanes))
    if a.c:
        r.check(r.rl_set_param(r.RL_PARAM_POTRF_CROSSOVER, a.c))
        r.check(r.rl_set_param(r.RL_PARAM_TRTRI_CROSSOVER, a.c))
    n = a.n
    k = a.k or n
    m = a.m or n
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    s = torch.cuda.current_stream().cuda_stream
    info = torch.zeros(1, dtype=torch.int32, device=dev)

    if a.case in ("dsgesv", "dsposv"):
        from . import inputs
        spd = a.case == "dsposv"
        A0 = inputs.spectrum_device(n, a.cond, 7, spd=spd, device=dev)
        B = torch.randn(a.nrhs, n, generator=g, device=dev, dtype=torch.float64)
        X = torch.zeros_like(B)
        A = A0.clone()
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        it = torch.zeros(1, dtype=torch.int32, device=dev)
        lw = (r.rl_dsposv_work_size if spd else r.rl_dsgesv_work_size)(n, a.nrhs, a.prec)
        work = torch.empty(lw, dtype=torch.uint8, device=dev)
        flops = (n ** 3 / 3.0) if spd else (2.0 * n ** 3 / 3.0)
        restore = lambda: A.copy_(A0)
        if spd:
            run = lambda: r.check(r.rl_dsposv("L", n, a.nrhs, A, n, B, n, X, n, a.prec, 1e-14, 30, it, info,
                                              work, lw, s))
        else:
            run = lambda: r.check(r.rl_dsgesv(n, a.nrhs, A, n, ipiv, B, n, X, n, a.prec, 1e-14, 30, it, info,
                                              work, lw, s))
    elif a.case in ("getrs", "potrs", "sgetrs"):
        # factors computed once, untimed; the solve of nrhs columns is timed
        dt = torch.float32 if a.case == "sgetrs" else torch.float64
        A = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) * 2 - 1
        lw = r.rl_dgetrf_work_size(n, n)
        work = torch.empty(lw, dtype=torch.uint8, device=dev)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        if a.case == "potrs":
            A = A @ A.T
            A.diagonal().add_(float(n))
            r.check(r.rl_dpotrf("L", n, A, n, info, None, 0, s))
        else:
            A = A.to(dt)
            f = r.rl_sgetrf if dt == torch.float32 else r.rl_dgetrf
            r.check(f(n, n, A, n, ipiv, info, work, lw, s))
        B0 = torch.randn(a.nrhs, n, generator=g, device=dev, dtype=torch.float64).to(dt)
        B = B0.clone()
        ltw = r.rl_trs_work_size(n, a.nrhs) if a.flow else 0
        tw = torch.zeros(max(ltw, 1), dtype=torch.uint8, device=dev) if ltw else None
        flops = 2.0 * n * n * a.nrhs
        restore = lambda: B.copy_(B0)
        if a.case == "potrs":
            run = lambda: r.check(r.rl_dpotrs("L", n, a.nrhs, A, n, B, n, tw, ltw, s))
        elif a.case == "getrs":
            run = lambda: r.check(r.rl_dgetrs("N", n, a.nrhs, A, n, ipiv, B, n, tw, ltw, s))
        else:
            run = lambda: r.check(r.rl_sgetrs("N", n, a.nrhs, A, n, ipiv, B, n, tw, ltw, s))
    elif a.case == "sgemm_tc":
        A = torch.rand(k, n, generator=g, device=dev, dtype=torch.float32)
        B = torch.rand(n, k, generator=g, device=dev, dtype=torch.float32)
        C = torch.rand(n, n, generator=g, device=dev, dtype=torch.float32)
        flops = 2.0 * n * n * k
        lw = r.rl_sgemm_tc_work_size(n, n, k, a.prec)
        work = torch.empty(lw, dtype=torch.uint8, device=dev)
        run = lambda: r.check(r.rl_sgemm_tc(a.prec, "N", "N", n, n, k, -1.0, A, n, B, k, C, n, work, lw, s))
        restore = lambda: None
    elif a.case == "laswp":
        # the top-level interchanges of an n x n LU: k = n/2 pivots (targets
        # uniform at or below their row, as partial pivoting of random
        # matrices gives) applied to the other n/2 columns
        import numpy as np
        kp = n // 2
        rng = np.random.default_rng(7)
        piv = np.array([rng.integers(j + 1, n + 1) for j in range(kp)], dtype=np.int32)
        ipiv = torch.from_numpy(piv).to(dev)
        A = torch.rand(n * n, generator=g, device=dev, dtype=torch.float64)
        flops = 0.0
        nbytes = 2.0 * kp * (n - kp) * 16.0          # two rows read and written per interchange per column
        run = lambda: r.check(r.rl_dlaswp(n, n - kp, A[kp * n:], n, 1, kp, ipiv, s))
        restore = lambda: None
    elif a.case == "sgemm":
        A = torch.rand(k, n, generator=g, device=dev, dtype=torch.float32)
        B = torch.rand(n, k, generator=g, device=dev, dtype=torch.float32)
        C = torch.rand(n, n, generator=g, device=dev, dtype=torch.float32)
        flops = 2.0 * n * n * k
        run = lambda: r.check(r.rl_sgemm("N", "N", n, n, k, -1.0, A, n, B, k, 1.0, C, n, s))
        restore = lambda: None
    elif a.case in ("dgemm", "dsyrk"):
        A = torch.rand(k, n, generator=g, device=dev, dtype=torch.float64)
        B = torch.rand(n, k, generator=g, device=dev, dtype=torch.float64)
        C = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64)
        if a.case == "dgemm" and a.oz:
            flops = 2.0 * n * n * k
            lwz = r.rl_oz_work_size(n, n, k, a.oz)
            wz = torch.empty(lwz, dtype=torch.uint8, device=dev)
            run = lambda: r.check(r.rl_dgemm_oz(a.oz, "N", "N", n, n, k, -1.0, A, n, B, k, 1.0, C, n, wz, lwz, s))
        elif a.case == "dgemm":
            flops = 2.0 * n * n * k
            run = lambda: r.check(r.rl_dgemm("N", "N", n, n, k, -1.0, A, n, B, k, 1.0, C, n, s))
        else:
            flops = 1.0 * k * n * (n + 1)
            run = lambda: r.check(r.rl_dsyrk("L", "N", n, k, -1.0, A, n, 1.0, C, n, s))
        restore = lambda: None
    elif a.case in ("zpotrf", "zgetrf"):
        # complex double; real flops: 4/3 n^3 (Cholesky), 8/3 n^3 (LU)
        X = torch.complex(torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) - 0.5,
                          torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) - 0.5)
        if a.case == "zpotrf":
            Z0 = X @ X.conj().T
            Z0.diagonal().add_(float(n))
            Z0 = Z0.transpose(0, 1).contiguous()       # column-major Hermitian: the conjugate
            flops = 4.0 * n ** 3 / 3.0
            Z = Z0.clone()
            run = lambda: r.check(r.rl_zpotrf(a.uplo, n, Z, n, info, None, 0, s))
        else:
            Z0 = X
            ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
            lw = r.rl_dgetrf_work_size(n, n)
            work = torch.empty(lw, dtype=torch.uint8, device=dev)
            flops = 8.0 * n ** 3 / 3.0
            Z = Z0.clone()
            run = lambda: r.check(r.rl_zgetrf(n, n, Z, n, ipiv, info, work, lw, s))
        restore = lambda: Z.copy_(Z0)
    elif a.case in ("vbatched_potrf", "vbatched_getrf"):
        # the batching form: `count` matrices with orders uniform on 8..256,
        # packed 256-byte aligned (SPD B B^T + n I for potrf, U(-1, 1) for getrf)
        import numpy as np
        from . import inputs
        sizes = inputs.bucket_sizes(a.count, 8, 256, inputs.seed_for(3, 0))
        dt = torch.float32 if a.fp32 else torch.float64
        esz = 4 if a.fp32 else 8
        align = 256 // esz
        offs, off = [], 0
        for nn in sizes:
            offs.append(off)
            off += ((int(nn) * int(nn) + align - 1) // align) * align
        A0 = torch.empty(off, dtype=dt, device=dev)
        for nn in np.unique(sizes):
            idx = np.nonzero(sizes == nn)[0]
            nn = int(nn)
            if a.case == "vbatched_potrf":
                Bm = torch.randn(len(idx), nn, nn, generator=g, device=dev, dtype=torch.float64)
                M = torch.bmm(Bm, Bm.transpose(1, 2))
                M.diagonal(dim1=1, dim2=2).add_(float(nn))
            else:
                M = torch.rand(len(idx), nn, nn, generator=g, device=dev, dtype=torch.float64) * 2 - 1
            M = M.to(dt)
            for qq, b in enumerate(idx):
                A0[offs[b]:offs[b] + nn * nn].copy_(M[qq].reshape(-1))
        A = A0.clone()
        ptrs = torch.tensor([A.data_ptr() + o * esz for o in offs], dtype=torch.int64, device=dev)
        nvec = torch.tensor(sizes, dtype=torch.int32, device=dev)
        binfo = torch.zeros(a.count, dtype=torch.int32, device=dev)
        pstore = torch.zeros(int(np.sum(sizes)), dtype=torch.int32, device=dev)
        pofs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        pptrs = torch.tensor([pstore.data_ptr() + 4 * int(qq) for qq in pofs], dtype=torch.int64, device=dev)
        lw = r.rl_getrf_vbatched_work_size(a.count)
        work = torch.empty(lw, dtype=torch.uint8, device=dev)
        n3 = float(np.sum(sizes.astype(np.float64) ** 3))
        if a.case == "vbatched_potrf":
            fn = r.rl_spotrf_vbatched if a.fp32 else r.rl_dpotrf_vbatched
            flops = n3 / 3.0
            run = lambda: r.check(fn("L", a.count, nvec, ptrs, nvec, binfo, 256, work, lw, s))
        else:
            fn = r.rl_sgetrf_vbatched if a.fp32 else r.rl_dgetrf_vbatched
            flops = 2.0 * n3 / 3.0
            run = lambda: r.check(fn(a.count, nvec, ptrs, nvec, pptrs, binfo, 256, work, lw, s))
        restore = lambda: A.copy_(A0)
    elif a.case in ("sgetrf_tc", "spotrf_tc"):
        # the precision form's factorization alone: FP32 storage, tcgen05
        # updates in operand precision --prec (0: SIMT FP32 rl_sgetrf / rl_spotrf)
        if a.case == "spotrf_tc":
            X = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) - 0.5
            A0 = (X @ X.T)
            A0.diagonal().add_(float(n))
            A0 = A0.to(torch.float32)
            flops = n ** 3 / 3.0
        else:
            A0 = (torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) * 2 - 1).to(torch.float32)
            flops = 2.0 * n ** 3 / 3.0
        A = A0.clone()
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        if a.prec == 0:
            lw = r.rl_dgetrf_work_size(n, n)
        else:
            lw = (r.rl_spotrf_tc_work_size(n, a.prec) if a.case == "spotrf_tc"
                  else r.rl_sgetrf_tc_work_size(n, n, a.prec))
        work = torch.empty(max(lw, 1), dtype=torch.uint8, device=dev)
        if a.case == "spotrf_tc":
            run = ((lambda: r.check(r.rl_spotrf("L", n, A, n, info, None, 0, s))) if a.prec == 0 else
                   (lambda: r.check(r.rl_spotrf_tc(a.prec, "L", n, A, n, info, work, lw, s))))
        else:
            run = ((lambda: r.check(r.rl_sgetrf(n, n, A, n, ipiv, info, work, lw, s))) if a.prec == 0 else
                   (lambda: r.check(r.rl_sgetrf_tc(a.prec, n, n, A, n, ipiv, info, work, lw, s))))
        restore = lambda: A.copy_(A0)
    elif a.case == "dtrsm":
        # B (m x n) := B L^{-T}, the TRSM of the Cholesky recursion
        L = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64)
        L.diagonal().add_(float(n))
        B0 = torch.rand(n, m, generator=g, device=dev, dtype=torch.float64)
        B = B0.clone()
        flops = 1.0 * m * n * n
        restore = lambda: B.copy_(B0)
        run = lambda: r.check(r.rl_dtrsm("R", "L", "T", "N", m, n, 1.0, L, n, B, m, s))
    else:
        if a.case in ("potrf", "trtri", "lauum"):
            X = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) - 0.5
            A0 = X @ X.T
            A0.diagonal().add_(float(n))
            if a.case != "potrf":
                r.check(r.rl_dpotrf("L", n, A0, n, info, None, 0, s))
        else:
            rows = m
            A0 = torch.rand(n if a.case == "getrf" else n, rows, generator=g, device=dev,
                            dtype=torch.float64) * 2 - 1
            if a.fp32:
                A0 = A0.to(torch.float32)
        A = A0.clone()
        restore = lambda: A.copy_(A0)
        if a.case == "potrf" and a.oz:
            flops = n ** 3 / 3.0
            lwz = r.rl_dpotrf_oz_work_size(n, a.oz)
            wz = torch.empty(lwz, dtype=torch.uint8, device=dev)
            run = lambda: r.check(r.rl_dpotrf_oz(a.oz, a.uplo, n, A, n, info, wz, lwz, s))
        elif a.case == "potrf":
            flops = n ** 3 / 3.0
            run = lambda: r.check(r.rl_dpotrf(a.uplo, n, A, n, info, None, 0, s))
        elif a.case == "trtri":
            flops = n ** 3 / 3.0
            run = lambda: r.check(r.rl_dtrtri(a.uplo, "N", n, A, n, info, None, 0, s))
        elif a.case == "lauum":
            flops = n ** 3 / 3.0
            run = lambda: r.check(r.rl_dlauum(a.uplo, n, A, n, info, None, 0, s))
        else:
            cols = n if a.case == "getrf" else (a.nb or r.rl_get_param(r.RL_PARAM_GETRF_PANEL))
            rows = m
            ipiv = torch.zeros(min(rows, cols), dtype=torch.int32, device=dev)
            lw = r.rl_dgetrf_work_size(rows, cols)
            work = torch.empty(lw, dtype=torch.uint8, device=dev)
            mn = min(rows, cols)
            flops = max(rows, cols) * mn * mn - mn ** 3 / 3.0   # LU of m x n, leading terms
            if a.oz and a.case == "getrf":
                lw = r.rl_dgetrf_oz_work_size(rows, cols, a.oz)
                work = torch.empty(lw, dtype=torch.uint8, device=dev)
                run = lambda: r.check(r.rl_dgetrf_oz(a.oz, rows, cols, A, rows, ipiv, info, work, lw, s))
            else:
                fn = r.rl_sgetrf if a.fp32 else r.rl_dgetrf
                run = lambda: r.check(fn(rows, cols, A, rows, ipiv, info, work, lw, s))

    for _ in range(a.warmup):
        restore()
        run()
    torch.cuda.synchronize()
    if a.graph:
        # capture on a side stream (the calls take the current stream's handle)
        gph = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        s_eager = s
        with torch.cuda.stream(cs):
            s = cs.cuda_stream
            restore()
            torch.cuda.synchronize()
            with torch.cuda.graph(gph, stream=cs):
                run()
        s = s_eager
        run = gph.replay
    times = []
    if a.trace:
        r.rl_trace_enable(1)
    for _ in range(a.reps):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    out = {"case": a.case, "n": n, "m": m, "k": k, "ms": statistics.median(times),
           "gflops": flops / (statistics.median(times) * 1e-3) / 1e9, "info": int(info.item())}
    if a.case == "laswp":
        out["gbs"] = nbytes / (statistics.median(times) * 1e-3) / 1e9
        out["bytes"] = nbytes
    if a.case in ("dsgesv", "dsposv"):
        out["iters"] = int(it.item())
        out["prec"] = a.prec
    if a.trace:
        out["trace"] = r.trace_summary()
        r.rl_trace_enable(0)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Throughput of the recursive FP64 factorizations on GB300.

One step = one recursive dpotrf (lower, SPD A = B B^T + n I) and one recursive
dgetrf (partial pivoting, entries Uniform(-1,1)) at n = 16384 in binary64,
through the C ABI on device-resident inputs.  Each step first restores both
matrices from pristine device copies (a 2.1 GB device-to-device copy each;
inside the timed region, about 0.1 % of it); both matrices are far larger
than L2, so no separate L2 flush is needed.

Printed (rank 0, one JSON line): GFLOP/s of the whole step (LAPACK Working
Note 41 flop counts), per-routine GFLOP/s, the roofline of the dominant
kernel measured with the library's per-kernel CUDA-event trace over the timed
region, an end-to-end figure through the host-buffer entry points (pinned
host memory, copies inside the timed region), the CPU oracle timed on a
bounded sample, and SM clocks sampled during the timed region.

--impl reference times the CPU oracle instead (the reference arm: a plain
FP64 recursive implementation on the host cores, same metric and unit).

Multi-GPU: a single factorization does not shard without a panel broadcast
per recursion level, so N > 1 runs N independent replicas (one per rank,
launched by torchrun) and reports the aggregate; ranks only synchronize for
the barrier and the max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "POTRF/GETRF GFLOP/s at n=16384 (% FP64 peak)"
UNIT = "GFLOP/s"

# FP64 roofline denominator (no FP64 figure is measured by the pool's peak
# file): 152 SMs x 2 FP64 FMA lanes per SM per clock x 2 flop x 2070 MHz
# maximum SM clock = 1.259 TFLOP/s, the unit count that reproduces GB300's
# nominal 1.25 TFLOP/s FP64 rate.
SMS = 152
FP64_FMA_PER_SM_CLK = 2
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
# FP32 SIMT: 128 FFMA lanes per SM (4 sub-partitions x 32) -> 80.5 TFLOP/s
FP32_FMA_PER_SM_CLK = 128
FP32_PEAK_TFLOPS = SMS * FP32_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12


def measured_hbm_gbs():
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json),
    or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs") or 0.0) or None
    except Exception:
        return None

# DRAM traffic of the dominant kernel (k_gemm, the GEMM kind: 2111 launches
# per step) per launch: dram__bytes_read.sum + dram__bytes_write.sum summed
# over the k_gemm launches of one step (172.7 GB over 2111 launches), from
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none -c 9000 --csv python bench.py --steps 1 --warmup 0
#       --e2e-steps 0 --mixed-n 0 --batch-count 0 --cpu-n 0 --others-n 0 --graph 0 --cusolver 0
# on commit f7f7de1 ("Lookahead in the LU and Cholesky recursions ...").  The
# real-valued k_gemm has not changed since; set this to None when it does.
GEMM_DRAM_BYTES_PER_LAUNCH = 172.704e9 / 2111
GEMM_DRAM_SOURCE = "ncu capture of one n=16384 step on commit f7f7de1 (k_gemm unchanged since)"


def flops_potrf(n: int) -> float:
    return n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0


def flops_getrf(n: int) -> float:
    return 2.0 * n ** 3 / 3.0 - n ** 2 / 2.0 + 5.0 * n / 6.0


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value of x over all ranks (the slowest replica sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gflops(step_flops: float, ms_per_step: float, world: int) -> float:
    """Whole-job throughput: every replica factors its own matrices, so the
    job does world * step_flops per (max over ranks) step time."""
    return world * step_flops / (ms_per_step * 1e-3) / 1e9


def workload_config(n: int) -> dict:
    return {
        "workload": f"recursive dpotrf (lower, SPD B*B^T+n*I) + dgetrf (partial pivoting, U(-1,1)), "
                    f"n={n}, binary64, column-major lda=n",
        "n": n,
        "routines": ["dpotrf", "dgetrf"],
        "l2": "inputs are 2.1 GB per matrix (> 129 MB L2); no flush needed",
        "restore": "each step restores both matrices from pristine device copies inside the timed region",
        "parallelism": "replicas (one independent factorization pair per GPU)",
    }


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.device_id is not None:
                cmd += ["-i", str(self.device_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu_id(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

def cpu_cores():
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    omp = os.environ.get("OMP_NUM_THREADS")
    return min(n, int(omp)) if omp and omp.isdigit() else n


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_sample(n_cpu: int, seed_k: int = 0):
    """Time the oracle's recursive dpotrf + dgetrf on an n_cpu sample of the
    same recipes; returns (GFLOP/s, seconds)."""
    import oracle
    from paper_1602_06763_gb300 import inputs
    A = inputs.spd_bbt(n_cpu, seed=inputs.seed_for(2, 500 + seed_k))
    G = inputs.uniform(n_cpu, n_cpu, seed=inputs.seed_for(2, 600 + seed_k))
    t0 = time.perf_counter()
    _, info1 = oracle.potrf(A, c=24)
    _, _, info2 = oracle.getrf(G, c=24)
    dt = time.perf_counter() - t0
    assert info1 == 0 and info2 == 0
    return (flops_potrf(n_cpu) + flops_getrf(n_cpu)) / dt / 1e9, dt


def cpu_lapack_context(n_cpu: int):
    """Context only: the host's LAPACK (torch.linalg on CPU) on the same
    sample, GFLOP/s of cholesky + lu_factor."""
    try:
        import torch
        from paper_1602_06763_gb300 import inputs
        A = torch.from_numpy(inputs.spd_bbt(n_cpu, seed=inputs.seed_for(2, 500)))
        G = torch.from_numpy(inputs.uniform(n_cpu, n_cpu, seed=inputs.seed_for(2, 600)))
        torch.linalg.cholesky(A[:64, :64])
        t0 = time.perf_counter()
        torch.linalg.cholesky(A)
        torch.linalg.lu_factor(G)
        dt = time.perf_counter() - t0
        return {"value": (flops_potrf(n_cpu) + flops_getrf(n_cpu)) / dt / 1e9, "unit": UNIT,
                "threads": torch.get_num_threads(), "what": "torch.linalg CPU (host LAPACK), context"}
    except Exception as e:
        return {"unavailable": str(e).splitlines()[0][:200]}


def run_reference(args, rank):
    if rank != 0:
        return 0
    from oracle import build as obuild
    obuild.build()
    n_ref = args.ref_n
    for w in range(args.warmup):
        oracle_sample(n_ref, w)
    times = []
    for k in range(args.steps):
        _, dt = oracle_sample(n_ref, 100 + k)
        times.append(dt)
    tot = sum(times)
    value = args.steps * (flops_potrf(n_ref) + flops_getrf(n_ref)) / tot / 1e9
    sample = (f"oracle dpotrf+dgetrf at n={n_ref} (same recipes as the n={args.n} workload) per step, "
              f"c=24; GFLOP/s of that order")
    cfg = workload_config(args.n)
    cfg["timed_order"] = n_ref
    cfg["timed_note"] = (f"each step times the oracle at order {n_ref}, a bounded sample of the n={args.n} "
                         f"workload; the GFLOP/s is that of order {n_ref}")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample, "sample_n": n_ref, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# precision form: low-precision factorization + FP64 refinement vs FP64 solve
# ----------------------------------------------------------------------------

PRECS = {"fp32": 0, "tf32": 1, "bf16": 2, "fp16s": 3, "tf32x3": 4}


def mixed_section(n, nrhs, cond, precs, dev, sp, reps=2, gmres_budget=300, oz_precs=()):
    """Solve A X = B (A = U diag(sigma) V^T or Q diag(sigma) Q^T, sigma
    log-spaced 1..cond, 64 Householder reflectors each side; B iid N(0,1))
    with the FP64 path (getrf+getrs / potrf+potrs) and with rl_dsgesv /
    rl_dsposv in each precision, with the classic refinement and with the
    GMRES refinement ("<prec>+gmres", budget gmres_budget GMRES iterations,
    one timed run after the classic runs of the same precision) and, for the
    precisions in oz_precs, the classic refinement with its FP64 products
    emulated on the BF16 tensor cores ("<prec>+oz"); reports
    time, the normwise backward error of the returned X (computed in FP64),
    refinement iterations (GMRES iterations for "+gmres"; negative: the FP64
    fallback ran), and the speedup over the FP64 path."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    def eta_of(A0, X, B, anorm):
        # column-major A X is (X_t @ A0)^T with the row-major tensors used here
        R = B - X @ A0
        return float(torch.max(R.abs().amax(dim=1) / (anorm * X.abs().amax(dim=1) + B.abs().amax(dim=1))))

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {"n": n, "nrhs": nrhs, "cond": cond, "tol": 1e-14, "reflectors": 64}
    for kind in ("general", "spd"):
        spd = kind == "spd"
        A0 = inputs.spectrum_device(n, cond, inputs.seed_for(2, 30 + int(spd)), spd=spd, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(inputs.seed_for(2, 40 + int(spd)))
        B = torch.randn(nrhs, n, generator=g, device=dev, dtype=torch.float64)
        anorm = float(A0.abs().sum(dim=0).max())
        info = torch.zeros(2, dtype=torch.int32, device=dev)
        ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
        lw = r.rl_dgetrf_work_size(n, n)
        wk = torch.empty(lw, dtype=torch.uint8, device=dev)
        ltw = r.rl_trs_work_size(n, nrhs)
        tw = torch.empty(ltw, dtype=torch.uint8, device=dev) if ltw else None
        res = {}
        # FP64 path (warm-up(s), then timed)
        for rep in range(reps):
            A = A0.clone()
            X = B.clone()
            if spd:
                ms = timed(lambda: (r.check(r.rl_dpotrf("L", n, A, n, info, None, 0, sp)),
                                    r.check(r.rl_dpotrs("L", n, nrhs, A, n, X, n, tw, ltw, sp))))
            else:
                ms = timed(lambda: (r.check(r.rl_dgetrf(n, n, A, n, ipiv, info, wk, lw, sp)),
                                    r.check(r.rl_dgetrs("N", n, nrhs, A, n, ipiv, X, n, tw, ltw, sp))))
        res["fp64"] = {"ms": ms, "eta": eta_of(A0, X, B, anorm)}
        del A
        variants = [(name, PRECS[name], 30, reps) for name in precs]
        if gmres_budget > 0:
            variants += [(name + "+gmres", PRECS[name] | r.RL_REFINE_GMRES, gmres_budget, 1) for name in precs]
        variants += [(name + "+oz", PRECS[name] | r.RL_REFINE_OZRES, 30, reps) for name in oz_precs]
        for name, prec, maxit, nrep in variants:
            lwm = (r.rl_dsposv_work_size if spd else r.rl_dsgesv_work_size)(n, nrhs, prec)
            wm = torch.empty(lwm, dtype=torch.uint8, device=dev)
            it = torch.zeros(1, dtype=torch.int32, device=dev)
            for rep in range(nrep):
                A = A0.clone()
                X = torch.zeros_like(B)
                if spd:
                    ms = timed(lambda: r.check(r.rl_dsposv("L", n, nrhs, A, n, B, n, X, n, prec, 1e-14, maxit, it,
                                                           info, wm, lwm, sp)))
                else:
                    ms = timed(lambda: r.check(r.rl_dsgesv(n, nrhs, A, n, ipiv, B, n, X, n, prec, 1e-14, maxit, it,
                                                           info, wm, lwm, sp)))
            iters = int(it.item())
            e = eta_of(A0, X, B, anorm)
            res[name] = {"ms": round(ms, 2), "eta": e, "iters": iters, "converged": iters >= 0,
                         "speedup_vs_fp64": round(res["fp64"]["ms"] / ms, 3)}
            if iters < 0:
                res[name]["note"] = {-2: "FP32 overflow: FP64 fallback", -3: "low-precision factorization failed: "
                                     "FP64 fallback"}.get(iters, "refinement did not converge: FP64 fallback")
            del A, wm
        keys = [v[0] for v in variants]
        best = [k for k in keys if res[k]["converged"] and res[k]["eta"] <= 1e-14]
        res["best"] = max(best, key=lambda k: res[k]["speedup_vs_fp64"]) if best else None
        res["speedup_at_equal_error"] = res[res["best"]]["speedup_vs_fp64"] if best else None
        out[kind] = res
        del A0
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# batching form: one persistent launch vs one call per matrix
# ----------------------------------------------------------------------------

def batched_section(count, baseline_count, dev, sp):
    """count SPD (B B^T + n I) and count general (Uniform(-1,1)) matrices,
    orders uniform in 8..256, packed 256-byte aligned; FP64 and FP32.  Times
    one rl_*_vbatched launch against one single-matrix rl_dpotrf / rl_dgetrf
    call per matrix (on the first baseline_count matrices, per-matrix time
    reported and scaled to the batch)."""
    import numpy as np
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    sizes = inputs.bucket_sizes(count, 8, 256, inputs.seed_for(3, 0))
    out = {"count": int(count), "orders": "uniform 8..256", "sum_n3": float(np.sum(sizes.astype(np.float64) ** 3))}

    def timed(fn, reps=3, before=None):
        ts = []
        for _ in range(reps):
            if before:
                before()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for kind in ("potrf", "getrf"):
        for prec in ("f64", "f32"):
            dt = torch.float64 if prec == "f64" else torch.float32
            esz = 8 if prec == "f64" else 4
            align = 256 // esz
            offs, off = [], 0
            for n in sizes:
                offs.append(off)
                off += ((int(n) * int(n) + align - 1) // align) * align
            pristine = torch.empty(off, dtype=dt, device=dev)
            g = torch.Generator(device=dev)
            g.manual_seed(inputs.seed_for(3, 10 + (kind == "getrf")))
            for n in np.unique(sizes):
                idx = np.nonzero(sizes == n)[0]
                n = int(n)
                if kind == "potrf":
                    Bm = torch.randn(len(idx), n, n, generator=g, device=dev, dtype=torch.float64)
                    M = torch.bmm(Bm, Bm.transpose(1, 2))
                    M = torch.tril(M) + torch.tril(M, -1).transpose(1, 2)
                    M.diagonal(dim1=1, dim2=2).add_(float(n))
                else:
                    M = torch.rand(len(idx), n, n, generator=g, device=dev, dtype=torch.float64) * 2 - 1
                M = M.to(dt)
                for q, b in enumerate(idx):
                    pristine[offs[b]:offs[b] + n * n].copy_(M[q].reshape(-1))
            work_buf = pristine.clone()
            base = work_buf.data_ptr()
            ptrs = torch.tensor([base + o * esz for o in offs], dtype=torch.int64, device=dev)
            nvec = torch.tensor(sizes, dtype=torch.int32, device=dev)
            info = torch.zeros(count, dtype=torch.int32, device=dev)
            pstore = torch.zeros(int(np.sum(sizes)), dtype=torch.int32, device=dev)
            pofs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
            pptrs = torch.tensor([pstore.data_ptr() + 4 * int(q) for q in pofs], dtype=torch.int64, device=dev)
            lw = r.rl_getrf_vbatched_work_size(count)
            wk = torch.empty(lw, dtype=torch.uint8, device=dev)
            restore = lambda: work_buf.copy_(pristine)
            if kind == "potrf":
                fn = r.rl_dpotrf_vbatched if prec == "f64" else r.rl_spotrf_vbatched
                run = lambda: r.check(fn("L", count, nvec, ptrs, nvec, info, 256, wk, lw, sp))
                flops = float(np.sum(sizes.astype(np.float64) ** 3)) / 3.0
            else:
                fn = r.rl_dgetrf_vbatched if prec == "f64" else r.rl_sgetrf_vbatched
                run = lambda: r.check(fn(count, nvec, ptrs, nvec, pptrs, info, 256, wk, lw, sp))
                flops = 2.0 * float(np.sum(sizes.astype(np.float64) ** 3)) / 3.0
            # autotune on this batch (restores the matrices), then time the chosen configuration
            restore()
            ltw = r.rl_vbatched_tune_work_size(count, int(np.sum(sizes.astype(np.int64) ** 2)), esz)
            tw = torch.empty(ltw, dtype=torch.uint8, device=dev)
            st, best, ms_cfg = r.rl_vbatched_tune("P" if kind == "potrf" else "G", esz, count, nvec, ptrs, nvec,
                                                  pptrs, info, 256, tw, ltw, sp)
            r.check(st, "rl_vbatched_tune")
            del tw
            cfg = r.rl_vbatched_config("P" if kind == "potrf" else "G", esz)
            restore()
            run()
            torch.cuda.synchronize()
            bad = int((info != 0).sum().item())
            ms = timed(run, reps=3, before=restore)
            # roofline of the batched form: the arithmetic pipe (FP64 DFMA or
            # FP32 FFMA, derived from unit counts and the maximum clock) and
            # HBM (every matrix read and written once: 2 n^2 elements)
            pipe = FP64_PEAK_TFLOPS if prec == "f64" else FP32_PEAK_TFLOPS
            alg_bytes = 2.0 * esz * float(np.sum(sizes.astype(np.float64) ** 2))
            hbm = measured_hbm_gbs()
            res = {"ms": ms, "gflops": flops / (ms * 1e-3) / 1e9, "launches": 2, "info_nonzero": bad,
                   "pct_flop_peak": round(100.0 * flops / (ms * 1e-3) / (pipe * 1e12), 2),
                   "flop_peak_tflops": round(pipe, 2),
                   "gbs_algorithmic": round(alg_bytes / (ms * 1e-3) / 1e9, 1),
                   "pct_hbm": round(100.0 * alg_bytes / (ms * 1e-3) / 1e9 / hbm, 2) if hbm else None,
                   "tuned": {"config": best, "nb": cfg[1], "threads": cfg[2], "ctas_per_sm": cfg[3],
                             "ms_per_config": [round(v, 3) for v in ms_cfg]}}
            # the same call captured once into a CUDA graph and replayed
            try:
                gph = torch.cuda.CUDAGraph()
                cs = torch.cuda.Stream()
                with torch.cuda.stream(cs):
                    torch.cuda.synchronize()
                    with torch.cuda.graph(gph, stream=cs):
                        if kind == "potrf":
                            r.check(fn("L", count, nvec, ptrs, nvec, info, 256, wk, lw, cs.cuda_stream))
                        else:
                            r.check(fn(count, nvec, ptrs, nvec, pptrs, info, 256, wk, lw, cs.cuda_stream))
                msg = timed(gph.replay, reps=3, before=restore)
                res["graph_replay_ms"] = msg
                del gph
            except Exception as e:
                res["graph_replay_ms"] = {"unavailable": str(e).splitlines()[0][:200]}
            if prec == "f64" and baseline_count > 0:
                # one single-matrix call per matrix, on the first baseline_count
                nb = min(baseline_count, count)
                ipiv1 = torch.zeros(256, dtype=torch.int32, device=dev)
                info1 = torch.zeros(1, dtype=torch.int32, device=dev)
                lw1 = r.rl_dgetrf_work_size(256, 256)
                wk1 = torch.empty(lw1, dtype=torch.uint8, device=dev)

                def per_matrix():
                    for b in range(nb):
                        n = int(sizes[b])
                        p = base + offs[b] * esz
                        if kind == "potrf":
                            r.check(r.rl_dpotrf("L", n, p, n, info1, None, 0, sp))
                        else:
                            r.check(r.rl_dgetrf(n, n, p, n, ipiv1, info1, wk1, lw1, sp))
                l0 = r.rl_launch_count()
                ms1 = timed(per_matrix, reps=1, before=restore)
                launches = r.rl_launch_count() - l0
                sub = float(np.sum(sizes[:nb].astype(np.float64) ** 3)) / float(np.sum(sizes.astype(np.float64) ** 3))
                res["per_matrix_path"] = {"matrices_timed": nb, "ms_for_timed": ms1,
                                          "ms_scaled_to_batch": ms1 / sub, "kernel_launches_timed": launches,
                                          "speedup_batched": (ms1 / sub) / ms}
            out[f"{kind}_{prec}"] = res
            del pristine, work_buf
            torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def routines_section(n, dev, sp):
    """The other recursive routines at order n (Section 5 list): GFLOP/s with
    LAPACK Working Note 41 counts, median of 3 after one warm-up, inputs
    restored before each timed call (outside its events)."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    def timed(fn, restore, reps=3):
        restore()
        fn()
        out = []
        for _ in range(reps):
            restore()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    info = torch.zeros(1, dtype=torch.int32, device=dev)
    S0 = inputs.spd_bbt_device(n, inputs.seed_for(2, 60), device=dev)
    L0 = S0.clone()
    r.check(r.rl_dpotrf("L", n, L0, n, info, None, 0, sp))
    G0 = inputs.uniform_device(n, n, inputs.seed_for(2, 61), device=dev)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    lw = r.rl_dgetrf_work_size(n, n)
    wk = torch.empty(lw, dtype=torch.uint8, device=dev)
    F0 = G0.clone()
    r.check(r.rl_dgetrf(n, n, F0, n, ipiv, info, wk, lw, sp))
    W = torch.empty_like(S0)
    out = {}
    n3 = float(n) ** 3
    cases = [
        ("dtrtri", n3 / 3.0, L0, lambda: r.check(r.rl_dtrtri("L", "N", n, W, n, info, None, 0, sp))),
        ("dlauum", n3 / 3.0, L0, lambda: r.check(r.rl_dlauum("L", n, W, n, info, None, 0, sp))),
        ("dpotri", 2.0 * n3 / 3.0, L0, lambda: r.check(r.rl_dpotri("L", n, W, n, info, None, 0, sp))),
    ]
    lg = r.rl_dgetri_work_size(n)
    wg = torch.empty(lg, dtype=torch.uint8, device=dev)
    cases.append(("dgetri", 4.0 * n3 / 3.0, F0,
                  lambda: r.check(r.rl_dgetri(n, W, n, ipiv, info, wg, lg, sp))))
    ls = r.rl_dsygst_work_size(n)
    ws = torch.empty(max(ls, 1), dtype=torch.uint8, device=dev)
    for it in (1, 2):
        cases.append((f"dsygst_itype{it}", n3, S0,
                      lambda it=it: r.check(r.rl_dsygst(it, "L", n, W, n, L0, n, ws, ls, sp))))
    for name, flops, src, fn in cases:
        ms = timed(fn, lambda src=src: W.copy_(src))
        out[name] = {"gflops": flops / (ms * 1e-3) / 1e9, "ms": ms}
    out["n"] = n
    out["flop_counts"] = "trtri, lauum n^3/3; potri 2n^3/3; getri 4n^3/3; sygst n^3"
    return out


def large_section(n, dev, sp):
    """The large FP64 case at order n (32768): dgetrf on the general matrix
    U diag(sigma) V^T with sigma log-spaced 1..1e4 (the matrix the large
    precision-form case solves), dpotrf and then POTRI (dtrtri + dlauum on the
    Cholesky factor, Section 5: xpotri from xtrtri and xlauum) on the SPD
    Q diag(sigma) Q^T with sigma log-spaced 1..1e6; 64 Householder
    reflectors per side.  One timed call each (a call takes seconds, far
    above any launch or clock effect), GFLOP/s with LAPACK Working Note 41
    counts and % of the derived FP64 peak, and a random-probe residual of
    each result in units of n eps ||A||_1 ||x||_1, computed with plain FP64
    torch products on the device: ||P A x - L (U x)||, ||A x - L (L^T x)||,
    ||A (X x) - x|| / ||X||_1 for the inverse X (symmetric, lower stored)."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    eps = 2.0 ** -53
    out = {"n": n}
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(inputs.seed_for(4, 90))
    x = torch.rand(n, 1, generator=g, device=dev, dtype=torch.float64) * 2 - 1

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def entry(name, flops, ms, res):
        out[name] = {"ms": round(ms, 2), "gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                     "pct_fp64_peak": round(100.0 * flops / (ms * 1e-3) / (FP64_PEAK_TFLOPS * 1e12), 1),
                     "info": int(info[0]), "probe_residual": res}

    # general, sigma 1..1e4: dgetrf
    A0 = inputs.spectrum_device(n, 1e4, inputs.seed_for(4, 91), spd=False, device=dev)
    A = A0.clone()
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    lw = r.rl_dgetrf_work_size(n, n)
    wk = torch.empty(lw, dtype=torch.uint8, device=dev)
    ms = timed(lambda: r.check(r.rl_dgetrf(n, n, A, n, ipiv, info, wk, lw, sp), "rl_dgetrf"))
    # the library reads the buffers column-major: its matrices are the transposes of the torch views
    Ft, Gt = A.t(), A0.t()
    b = (Gt @ x).squeeze(1)
    p = ipiv.cpu().numpy() - 1
    perm = list(range(n))
    for i in range(n):
        perm[i], perm[p[i]] = perm[p[i]], perm[i]
    b = b[torch.tensor(perm, device=dev)]
    y = torch.triu(Ft) @ x
    y = (torch.tril(Ft, -1) @ y + y).squeeze(1)
    res = float((b - y).abs().sum() / (n * eps * Gt.abs().sum(0).max() * x.abs().sum()))
    entry("dgetrf", flops_getrf(n), ms, res)
    del A, A0, Ft, Gt, y, wk
    torch.cuda.empty_cache()

    # SPD, sigma 1..1e6: dpotrf, then dtrtri + dlauum = dpotri on the factor
    S0 = inputs.spectrum_device(n, 1e6, inputs.seed_for(4, 92), spd=True, device=dev)
    L = S0.clone()
    ms = timed(lambda: r.check(r.rl_dpotrf("L", n, L, n, info, None, 0, sp), "rl_dpotrf"))
    Lt = torch.tril(L.t())
    St = S0.t()
    y = St @ x - Lt @ (Lt.t() @ x)
    anorm = St.abs().sum(0).max()
    res = float(y.abs().sum() / (n * eps * anorm * x.abs().sum()))
    entry("dpotrf", flops_potrf(n), ms, res)
    del Lt, y
    torch.cuda.empty_cache()
    X = L
    ms1 = timed(lambda: r.check(r.rl_dtrtri("L", "N", n, X, n, info, None, 0, sp), "rl_dtrtri"))
    ms2 = timed(lambda: r.check(r.rl_dlauum("L", n, X, n, info, None, 0, sp), "rl_dlauum"))
    Xl = torch.tril(X.t())
    Xx = Xl @ x + torch.tril(X.t(), -1).t() @ x
    xnorm = (Xl.abs().sum(0) + torch.tril(X.t(), -1).abs().sum(1)).max()
    del Xl
    y = St @ Xx - x
    res = float(y.abs().sum() / (n * eps * anorm * xnorm * x.abs().sum()))
    n3 = float(n) ** 3
    out["dtrtri"] = {"ms": round(ms1, 2), "gflops": round(n3 / 3.0 / (ms1 * 1e-3) / 1e9, 1)}
    out["dlauum"] = {"ms": round(ms2, 2), "gflops": round(n3 / 3.0 / (ms2 * 1e-3) / 1e9, 1)}
    entry("dpotri", 2.0 * n3 / 3.0, ms1 + ms2, res)
    out["inputs"] = "dgetrf: U diag(sigma) V^T, sigma 1..1e4; dpotrf/dpotri: Q diag(sigma) Q^T, sigma 1..1e6"
    del X, L, S0, St, Xx, y
    torch.cuda.empty_cache()
    return out


def lowprec_section(n, dev, sp):
    """The precision form's factorization step alone: rl_sgetrf_tc /
    rl_spotrf_tc (FP32 storage, tcgen05 updates in each operand precision)
    and the SIMT FP32 rl_sgetrf / rl_spotrf, GFLOP/s at order n (median of 2
    after a warm-up, inputs restored outside the events)."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    G0 = inputs.uniform_device(n, n, inputs.seed_for(2, 70), device=dev).to(torch.float32)
    S0 = inputs.spd_bbt_device(n, inputs.seed_for(2, 71), device=dev).to(torch.float32)
    A = torch.empty_like(G0)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {"n": n}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        bf = float(pk.get("bf16_tflops") or 0.0)
        peaks = {"bf16": bf, "fp16": bf, "tf32": bf / 2.0, "tf32x3": bf / 2.0 / 3.0}
    except Exception:
        pass
    for name in ("fp32", "tf32", "bf16", "fp16", "tf32x3"):
        res = {}
        for kind, src, flops in (("getrf", G0, 2.0 * n ** 3 / 3.0), ("potrf", S0, n ** 3 / 3.0)):
            if name == "fp32":
                lw = r.rl_dgetrf_work_size(n, n)
                w = torch.empty(lw, dtype=torch.uint8, device=dev)
                if kind == "getrf":
                    call = lambda: r.check(r.rl_sgetrf(n, n, A, n, ipiv, info, w, lw, sp))
                else:
                    call = lambda: r.check(r.rl_spotrf("L", n, A, n, info, None, 0, sp))
            else:
                p = {"tf32": r.RL_PREC_TF32, "bf16": r.RL_PREC_BF16, "fp16": r.RL_PREC_FP16S,
                     "tf32x3": r.RL_PREC_TF32X3}[name]
                if kind == "getrf":
                    lw = r.rl_sgetrf_tc_work_size(n, n, p)
                    w = torch.empty(lw, dtype=torch.uint8, device=dev)
                    call = lambda: r.check(r.rl_sgetrf_tc(p, n, n, A, n, ipiv, info, w, lw, sp))
                else:
                    lw = r.rl_spotrf_tc_work_size(n, p)
                    w = torch.empty(lw, dtype=torch.uint8, device=dev)
                    call = lambda: r.check(r.rl_spotrf_tc(p, "L", n, A, n, info, w, lw, sp))
            ts = []
            for rep in range(3):
                A.copy_(src)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                call()
                b.record()
                torch.cuda.synchronize()
                if rep:
                    ts.append(a.elapsed_time(b))
            ms = statistics.median(ts)
            res[kind] = {"ms": ms, "gflops": flops / (ms * 1e-3) / 1e9, "info": int(info[0])}
            del w
        if name in peaks and peaks[name] > 0:
            res["update_peak_tflops"] = peaks[name]
        out[name] = res
    out["peaks"] = "tensor peaks from MEASURED_PEAKS.json bf16 burst (tf32 = bf16/2, 3xtf32 = tf32/3, nominal ratios)"
    return out


def emulated_section(n, slices, dev, sp):
    """FP64 factorizations with the updates emulated on the BF16 tensor cores
    (rl_dpotrf_oz / rl_dgetrf_oz, `slices` digit planes) next to the native
    FP64 ones on the same inputs: GFLOP/s (LAWN 41 counts, median of 2 after
    a warm-up) and a random-probe residual of each result,
    ||A x - L (L^T x)|| or ||P A x - L (U x)|| / (n eps ||A||_1 ||x||_1)
    (O(n^2) FP64 work), and an 8192^3 GEMM both ways."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs

    eps = 2.0 ** -53
    S0 = inputs.spd_bbt_device(n, inputs.seed_for(2, 80), device=dev)
    G0 = inputs.uniform_device(n, n, inputs.seed_for(2, 81), device=dev)
    A = torch.empty_like(S0)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(inputs.seed_for(2, 82))
    x = torch.rand(n, 1, generator=gen, device=dev, dtype=torch.float64) * 2 - 1

    # the library reads each buffer column-major: its matrix is the transpose of the torch view
    def probe_chol(F):
        L = torch.tril(F.transpose(0, 1))
        A0 = S0.transpose(0, 1)
        y = A0 @ x - L @ (L.transpose(0, 1) @ x)
        return float(y.abs().sum() / (n * eps * A0.abs().sum(0).max() * x.abs().sum()))

    def probe_lu(F, piv):
        Ft = F.transpose(0, 1)
        L = torch.tril(Ft, -1) + torch.eye(n, device=dev, dtype=torch.float64)
        U = torch.triu(Ft)
        b = (G0.transpose(0, 1) @ x).squeeze(1)
        p = piv.cpu().numpy() - 1
        perm = list(range(n))
        for i in range(n):
            perm[i], perm[p[i]] = perm[p[i]], perm[i]
        b = b[torch.tensor(perm, device=dev)]
        y = b - (L @ (U @ x)).squeeze(1)
        return float(y.abs().sum() / (n * eps * G0.transpose(0, 1).abs().sum(0).max() * x.abs().sum()))

    def timed(call, src):
        ts = []
        for rep in range(3):
            A.copy_(src)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            call()
            b.record()
            torch.cuda.synchronize()
            if rep:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {"n": n, "slices": slices}
    lw = r.rl_dgetrf_work_size(n, n)
    wn = torch.empty(lw, dtype=torch.uint8, device=dev)
    lpo = r.rl_dpotrf_oz_work_size(n, slices)
    lgo = r.rl_dgetrf_oz_work_size(n, n, slices)
    wo = torch.empty(max(lpo, lgo), dtype=torch.uint8, device=dev)
    for kind, emu in (("dpotrf", False), ("dpotrf", True), ("dgetrf", False), ("dgetrf", True)):
        if kind == "dpotrf":
            call = ((lambda: r.check(r.rl_dpotrf_oz(slices, "L", n, A, n, info, wo, lpo, sp))) if emu else
                    (lambda: r.check(r.rl_dpotrf("L", n, A, n, info, None, 0, sp))))
            ms = timed(call, S0)
            res = probe_chol(A)
            flops = n ** 3 / 3.0
        else:
            call = ((lambda: r.check(r.rl_dgetrf_oz(slices, n, n, A, n, ipiv, info, wo, lgo, sp))) if emu else
                    (lambda: r.check(r.rl_dgetrf(n, n, A, n, ipiv, info, wn, lw, sp))))
            ms = timed(call, G0)
            res = probe_lu(A, ipiv)
            flops = 2.0 * n ** 3 / 3.0
        out[kind + ("_emulated" if emu else "_native")] = {
            "ms": ms, "gflops": flops / (ms * 1e-3) / 1e9, "info": int(info[0]), "probe_residual": res}
    del wo, wn
    g = 8192
    Ag = torch.rand(g, g, generator=gen, device=dev, dtype=torch.float64)
    Bg = torch.rand(g, g, generator=gen, device=dev, dtype=torch.float64)
    Cg = torch.zeros(g, g, device=dev, dtype=torch.float64)
    lz = r.rl_oz_work_size(g, g, g, slices)
    wz = torch.empty(lz, dtype=torch.uint8, device=dev)
    for emu in (False, True):
        call = ((lambda: r.check(r.rl_dgemm_oz(slices, "N", "N", g, g, g, 1.0, Ag, g, Bg, g, 0.0, Cg, g, wz, lz, sp)))
                if emu else (lambda: r.check(r.rl_dgemm("N", "N", g, g, g, 1.0, Ag, g, Bg, g, 0.0, Cg, g, sp))))
        call()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out["dgemm_8192_" + ("emulated" if emu else "native")] = {"ms": ms, "gflops": 2.0 * g ** 3 / (ms * 1e-3) / 1e9}
    out["note"] = ("not in the paper: the FP64 updates as BF16 digit products on tcgen05 (Ozaki scheme); "
                   "the headline value stays native FP64")
    return out


def cusolver_section(n, dev):
    """Context only: the vendor library (cuSOLVER through torch.linalg) on the
    same GPU and inputs (FP64), median of 3 after one warm-up."""
    import torch
    from paper_1602_06763_gb300 import inputs
    res = {}
    S = inputs.spd_bbt_device(n, inputs.seed_for(2, 10), device=dev).reshape(n, n)
    G = inputs.uniform_device(n, n, inputs.seed_for(2, 20), device=dev).reshape(n, n)
    for name, fn, flops in (("cholesky", lambda: torch.linalg.cholesky(S), n ** 3 / 3.0),
                            ("lu_factor", lambda: torch.linalg.lu_factor(G), 2.0 * n ** 3 / 3.0)):
        try:
            fn()
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                y = fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
                del y
            ms = statistics.median(ts)
            res[name] = {"gflops": flops / (ms * 1e-3) / 1e9, "ms": ms}
        except Exception as e:          # context figure: report, do not fail the bench
            res[name] = {"unavailable": str(e).splitlines()[0][:200]}
    res["what"] = "torch.linalg (cuSOLVER) FP64 on the same inputs; context, not the target"
    return res


def probe_chol_dev(S0, F, x):
    """||A x - L (L^T x)||_1 / (n eps ||A||_1 ||x||_1) for the Cholesky factor
    in F; S0 and F are column-major buffers (their torch views are the
    transposes), plain FP64 torch products."""
    import torch
    n = S0.shape[0]
    L = torch.tril(F.t())
    A0 = S0.t()
    y = A0 @ x - L @ (L.t() @ x)
    return float(y.abs().sum() / (n * 2.0 ** -53 * A0.abs().sum(0).max() * x.abs().sum()))


def probe_lu_dev(G0, F, piv, x):
    """||P A x - L (U x)||_1 / (n eps ||A||_1 ||x||_1) for the LU factors in F
    with the 1-based interchanges piv (column-major buffers, as above)."""
    import torch
    n = G0.shape[0]
    Ft = F.t()
    b = (G0.t() @ x).squeeze(1)
    p = piv.cpu().numpy() - 1
    perm = list(range(n))
    for i in range(n):
        perm[i], perm[p[i]] = perm[p[i]], perm[i]
    b = b[torch.tensor(perm, device=b.device)]
    y = torch.triu(Ft) @ x
    y = (torch.tril(Ft, -1) @ y + y).squeeze(1)
    return float((b - y).abs().sum() / (n * 2.0 ** -53 * G0.t().abs().sum(0).max() * x.abs().sum()))


def graph_section(n, dev, sp):
    """dpotrf and dgetrf captured once into CUDA graphs and replayed: the
    launch overhead of the ~2000 launches per factorization, measured."""
    import torch
    from paper_1602_06763_gb300 import relgpu as r, inputs
    res = {}
    S0 = inputs.spd_bbt_device(n, inputs.seed_for(2, 10), device=dev)
    G0 = inputs.uniform_device(n, n, inputs.seed_for(2, 20), device=dev)
    A = torch.empty_like(S0)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    lw = r.rl_dgetrf_work_size(n, n)
    wk = torch.empty(lw, dtype=torch.uint8, device=dev)
    for name, src, flops, call in (
            ("dpotrf", S0, n ** 3 / 3.0, lambda s: r.check(r.rl_dpotrf("L", n, A, n, info, None, 0, s))),
            ("dgetrf", G0, 2.0 * n ** 3 / 3.0, lambda s: r.check(r.rl_dgetrf(n, n, A, n, ipiv, info, wk, lw, s)))):
        try:
            A.copy_(src)
            call(sp)                                   # first call outside capture (one-time set-up)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            with torch.cuda.stream(cs):
                A.copy_(src)
                torch.cuda.synchronize()
                with torch.cuda.graph(g, stream=cs):
                    call(cs.cuda_stream)
            ts = []
            for _ in range(3):
                A.copy_(src)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                g.replay()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            if int(info[0]) != 0:
                raise RuntimeError(f"info {int(info[0])} after replay")
            ms = statistics.median(ts)
            gen = torch.Generator(device=dev)
            gen.manual_seed(inputs.seed_for(2, 11))
            x = torch.rand(n, 1, generator=gen, device=dev, dtype=torch.float64) * 2 - 1
            res[name] = {"gflops": flops / (ms * 1e-3) / 1e9, "ms": ms,
                         "probe_residual_of_replayed_factors": probe_chol_dev(src, A, x) if name == "dpotrf"
                         else probe_lu_dev(src, A, ipiv, x)}
            del g
        except Exception as e:
            res[name] = {"unavailable": str(e).splitlines()[0][:200]}
    return res


def summarize_mixed(*sections):
    """Per precision-form case: order, condition, right-hand sides, the FP64
    time, and per variant the refinement iterations (negative: the FP64
    fallback ran) and the speedup over FP64."""
    out = []
    for sec in sections:
        if not sec:
            continue
        for kind in ("general", "spd"):
            res = sec.get(kind)
            if not res:
                continue
            row = {"case": f"{kind} n={sec['n']} cond={sec['cond']:g} nrhs={sec['nrhs']}",
                   "fp64_ms": round(res["fp64"]["ms"], 1), "best": res.get("best"),
                   "speedup_at_equal_error": res.get("speedup_at_equal_error")}
            for k, v in res.items():
                if isinstance(v, dict) and "iters" in v:
                    row[k] = [v["iters"], v["speedup_vs_fp64"]]
            out.append(row)
    return {"format": "variant: [iterations (negative: FP64 fallback), speedup vs FP64]", "cases": out} if out else None


def summarize_batched(sec):
    if not sec:
        return None
    out = {}
    for k, v in sec.items():
        if isinstance(v, dict) and "ms" in v:
            out[k] = {"ms": round(v["ms"], 2), "pct_flop_peak": v.get("pct_flop_peak"), "pct_hbm": v.get("pct_hbm")}
    return out


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1602_06763_gb300 import relgpu as r, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    spd0 = inputs.spd_bbt_device(n, inputs.seed_for(2, 10 + rank), device=dev)
    gen0 = inputs.uniform_device(n, n, inputs.seed_for(2, 20 + rank), device=dev)
    spd = torch.empty_like(spd0)
    gen = torch.empty_like(gen0)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    lw = r.rl_dgetrf_work_size(n, n)
    work = torch.empty(lw, dtype=torch.uint8, device=dev)

    def step():
        spd.copy_(spd0)
        gen.copy_(gen0)
        r.check(r.rl_dpotrf("L", n, spd.data_ptr(), n, info.data_ptr(), None, 0, sp), "rl_dpotrf")
        r.check(r.rl_dgetrf(n, n, gen.data_ptr(), n, ipiv.data_ptr(), info.data_ptr() + 4,
                            work.data_ptr(), lw, sp), "rl_dgetrf")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    inf = info.cpu().tolist()
    if inf != [0, 0]:
        raise RuntimeError(f"factorization info {inf} on the benchmark inputs")

    def barrier():
        if world > 1:
            dist.barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(physical_gpu_id(local_rank))

    barrier()
    torch.cuda.synchronize()
    sampler.start()
    r.rl_trace_enable(1)
    launches0 = r.rl_launch_count()
    t_start.record(stream)
    for k in range(args.steps):
        spd.copy_(spd0)
        gen.copy_(gen0)
        ev[k][0].record(stream)
        r.check(r.rl_dpotrf("L", n, spd.data_ptr(), n, info.data_ptr(), None, 0, sp), "rl_dpotrf")
        ev[k][1].record(stream)
        r.check(r.rl_dgetrf(n, n, gen.data_ptr(), n, ipiv.data_ptr(), info.data_ptr() + 4,
                            work.data_ptr(), lw, sp), "rl_dgetrf")
        ev[k][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = r.rl_launch_count() - launches0
    trace = r.trace_summary()
    r.rl_trace_enable(0)
    clocks = sampler.stop()

    ms_total = t_start.elapsed_time(t_end)
    ms_potrf = [e[0].elapsed_time(e[1]) for e in ev]
    ms_getrf = [e[1].elapsed_time(e[2]) for e in ev]
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    step_flops = flops_potrf(n) + flops_getrf(n)
    value = aggregate_gflops(step_flops, ms_step, world)

    # dominant kernel by device time over the timed region
    dom_name = max(trace, key=lambda k: trace[k]["ms"]) if trace else None
    roofline = None
    if dom_name:
        d = trace[dom_name]
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        alg_bytes = d["bytes"] / d["launches"] if d["launches"] else None
        roofline = {
            "bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": GEMM_DRAM_BYTES_PER_LAUNCH if dom_name == "gemm" else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "traffic_source": GEMM_DRAM_SOURCE if dom_name == "gemm" else None,
            "algorithmic_bytes_per_launch": alg_bytes,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2070 MHz",
            "launches_per_step": d["launches"] / args.steps,
            "share_of_step": d["ms"] / ms_total,
        }

    # end to end through the host-buffer entry points (pinned host memory)
    e2e = None
    if args.e2e_steps > 0:
        import numpy as np
        h_spd0 = spd0.cpu().numpy().copy()
        h_gen0 = gen0.cpu().numpy().copy()
        h_spd = torch.empty(n * n, dtype=torch.float64).pin_memory()
        h_gen = torch.empty(n * n, dtype=torch.float64).pin_memory()
        h_piv = torch.empty(n, dtype=torch.int32).pin_memory()
        h_inf = torch.empty(2, dtype=torch.int32).pin_memory()
        del spd, gen
        lw_p = r.rl_host_work_size("dpotrf", n, n, n)
        lw_g = r.rl_host_work_size("dgetrf", n, n, n)
        w_p = torch.empty(lw_p, dtype=torch.uint8, device=dev)
        w_g = torch.empty(lw_g, dtype=torch.uint8, device=dev)
        ts = []
        for k in range(args.e2e_steps + 1):
            np.copyto(h_spd.numpy(), h_spd0.reshape(-1))
            np.copyto(h_gen.numpy(), h_gen0.reshape(-1))
            barrier()
            t0 = time.perf_counter()
            r.check(r.rl_dpotrf_host("L", n, h_spd.data_ptr(), n, h_inf.data_ptr(), w_p.data_ptr(),
                                     lw_p, sp), "rl_dpotrf_host")
            r.check(r.rl_dgetrf_host(n, n, h_gen.data_ptr(), n, h_piv.data_ptr(), h_inf.data_ptr() + 4,
                                     w_g.data_ptr(), lw_g, sp), "rl_dgetrf_host")
            t1 = time.perf_counter()
            if k > 0:          # the first pass is a warm-up
                ts.append(t1 - t0)
            if h_inf.tolist() != [0, 0]:
                raise RuntimeError("host-buffer factorization failed")
        t_e2e = max_over_ranks(statistics.median(ts), world, dev)
        e2e = {"value": aggregate_gflops(step_flops, 1e3 * t_e2e, world), "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * n * 8,
               "d2h_bytes_per_step": 2 * n * n * 8 + n * 4 + 2 * 4,
               "ms_per_step": 1e3 * t_e2e, "steps": len(ts)}

    if rank != 0:
        return 0

    secs = {}

    def section(name, fn):
        t0 = time.perf_counter()
        out = fn()
        secs[name] = round(time.perf_counter() - t0, 1)
        return out

    del spd0, gen0
    torch.cuda.empty_cache()
    mixed = section("mixed_solve", lambda: mixed_section(
        args.mixed_n, args.mixed_nrhs, args.mixed_cond, [p for p in args.mixed_precs.split(",") if p], dev, sp,
        gmres_budget=args.gmres_budget, oz_precs=[p for p in args.mixed_oz.split(",") if p])) \
        if args.mixed_n > 0 else None
    torch.cuda.empty_cache()
    mixed_large = section("mixed_solve_large", lambda: mixed_section(
        args.mixed4_n, args.mixed4_nrhs, args.mixed4_cond, [p for p in args.mixed4_precs.split(",") if p], dev,
        sp, reps=1, gmres_budget=args.gmres_budget)) if args.mixed4_n > 0 else None
    torch.cuda.empty_cache()
    large = section("large", lambda: large_section(args.large_n, dev, sp)) if args.large_n > 0 else None
    batched = section("batched", lambda: batched_section(args.batch_count, args.batch_baseline, dev, sp)) \
        if args.batch_count > 0 else None
    others = section("other_routines", lambda: routines_section(args.others_n, dev, sp)) if args.others_n > 0 else None
    lowprec = section("lowprec", lambda: lowprec_section(args.lowprec_n, dev, sp)) if args.lowprec_n > 0 else None
    emulated = section("fp64_emulated", lambda: emulated_section(args.oz_n, args.oz_slices, dev, sp)) \
        if args.oz_n > 0 else None
    graphs = section("graph_replay", lambda: graph_section(n, dev, sp)) if args.graph else None
    cusolver = section("cusolver", lambda: cusolver_section(n, dev)) if args.cusolver else None

    cpu = None
    if world == 1 and args.cpu_n > 0:
        from oracle import build as obuild
        obuild.build()
        t0 = time.perf_counter()
        gfl, dt = oracle_sample(args.cpu_n)
        cpu = {"value": gfl, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle dpotrf+dgetrf once at n={args.cpu_n} (same recipes as the n={n} workload), "
                         f"c=24, {dt:.1f} s; GFLOP/s of that order",
               "sample_n": args.cpu_n, "cpu_model": cpu_model(),
               "lapack_context": cpu_lapack_context(min(args.cpu_n, 4096))}
        secs["cpu_baseline"] = round(time.perf_counter() - t0, 1)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(n),
        "pct_fp64_peak": 100.0 * (value / world) / (FP64_PEAK_TFLOPS * 1e3),
        "routines": {
            "dpotrf": {"gflops": flops_potrf(n) / (statistics.median(ms_potrf) * 1e-3) / 1e9,
                       "ms": statistics.median(ms_potrf)},
            "dgetrf": {"gflops": flops_getrf(n) / (statistics.median(ms_getrf) * 1e-3) / 1e9,
                       "ms": statistics.median(ms_getrf)},
        },
        "roofline": roofline,
        "kernels": {k: {"launches_per_step": v["launches"] / args.steps,
                        "ms_per_step": v["ms"] / args.steps,
                        "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["flops"] else None,
                        "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["bytes"] else None}
                    for k, v in trace.items()},
        "gpu_launches": launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
        # detailed sections, then (last, so that they stay in view at the end
        # of the line) compact summaries of the precision, batching and
        # large-order sections
        "mixed_solve": mixed,
        "mixed_solve_large": mixed_large,
        "batched": batched,
        "other_routines": others,
        "lowprec_factorization": lowprec,
        "fp64_emulated": emulated,
        "graph_replay": graphs,
        "cusolver_context": cusolver,
        "section_seconds": secs,
        "summary_mixed": summarize_mixed(mixed, mixed_large),
        "summary_batched": summarize_batched(batched),
        "large": large,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--cpu-n", type=int, default=6144,
                    help="order of the oracle's timed sample for cpu_baseline (about 15 s on 16 cores)")
    ap.add_argument("--ref-n", type=int, default=3072,
                    help="order of the oracle's sample per step in the reference arm")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--mixed-n", type=int, default=16384,
                    help="order of the precision-form comparison (0 skips it)")
    ap.add_argument("--mixed-nrhs", type=int, default=16)
    ap.add_argument("--mixed-cond", type=float, default=1e6)
    ap.add_argument("--mixed-precs", default="fp32,tf32x3,tf32,bf16,fp16s")
    ap.add_argument("--mixed-oz", default="fp32,tf32x3",
                    help="precisions also run with emulated FP64 residual products (+oz) in the n=16384 case")
    ap.add_argument("--mixed4-n", type=int, default=32768,
                    help="order of the large precision-form case, 1 RHS (0 skips it)")
    ap.add_argument("--mixed4-nrhs", type=int, default=1)
    ap.add_argument("--mixed4-cond", type=float, default=1e4)
    ap.add_argument("--mixed4-precs", default="fp32,bf16,fp16s")
    ap.add_argument("--large-n", type=int, default=32768,
                    help="order of the large FP64 section: dgetrf, dpotrf, dpotri (0 skips it)")
    ap.add_argument("--gmres-budget", type=int, default=300,
                    help="GMRES iterations allowed to the '+gmres' precision-form variants (0 skips them)")
    ap.add_argument("--batch-count", type=int, default=20000,
                    help="matrices per kind in the batching-form comparison (0 skips it)")
    ap.add_argument("--batch-baseline", type=int, default=2000,
                    help="matrices timed through the single-matrix path for the comparison")
    ap.add_argument("--others-n", type=int, default=8192,
                    help="order of the trtri/lauum/potri/getri/sygst section (0 skips it)")
    ap.add_argument("--lowprec-n", type=int, default=16384,
                    help="order of the low-precision factorization section (0 skips it)")
    ap.add_argument("--oz-n", type=int, default=16384,
                    help="order of the FP64-emulation section (0 skips)")
    ap.add_argument("--oz-slices", type=int, default=7)
    ap.add_argument("--graph", type=int, default=1, help="time CUDA-graph replay of dpotrf/dgetrf (0 skips)")
    ap.add_argument("--cusolver", type=int, default=1, help="time torch.linalg (cuSOLVER) as context (0 skips)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank)

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group(backend="nccl")
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

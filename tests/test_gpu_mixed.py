"""Precision form (rl_dsgesv / rl_dsposv) and the FP64 solves (rl_dgetrs /
rl_dpotrs) against the oracle.

The bar: a converged refinement returns X whose normwise backward error
eta = max_j ||b_j - A x_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf),
computed by the oracle with compensated sums, is <= the requested tol
(1e-14); the forward error against the oracle's FP64 solution is within
kappa(A) * (tol + n eps), the first-order perturbation bound.  When the
refinement cannot converge the FP64 fallback runs and its result meets the
FP64 solve's own bound (eta <= 10 n eps).
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def run_mixed(A, B, spd=False, prec=0, tol=1e-14, maxiter=30):
    r = G.lib()
    t = G.torch()
    n = A.shape[0]
    nrhs = B.shape[1]
    dA, dB = G.DevMat(A), G.DevMat(B)
    dX = G.DevMat(np.zeros_like(B))
    ipiv = G.int_buf(n, -5)
    it = G.int_buf(1, -99)
    info = G.int_buf(1, -77)
    if spd:
        lw = r.rl_dsposv_work_size(n, nrhs, prec)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsposv("L", n, nrhs, dA.ptr(), dA.lda, dB.ptr(), dB.lda, dX.ptr(), dX.lda, prec, tol,
                         maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    else:
        lw = r.rl_dsgesv_work_size(n, nrhs, prec)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsgesv(n, nrhs, dA.ptr(), dA.lda, ipiv.data_ptr(), dB.ptr(), dB.lda, dX.ptr(), dX.lda,
                         prec, tol, maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert dA.canaries_intact() and dX.canaries_intact() and dB.canaries_intact()
    return dX.get(), dA.get(), int(it[0].item()), int(info[0].item()), ipiv.cpu().numpy()[:n]


def ref_solution(A, B, spd):
    if spd:
        L, _ = oracle.potrf(A, c=24)
        return oracle.potrs(L, B)
    F, piv, _ = oracle.getrf(A, c=24)
    return oracle.getrs(F, piv, B)


@pytest.mark.parametrize("spd", [False, True])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 3), (300, 16), (700, 9)])
def test_mixed_fp32_converges(spd, n, nrhs):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(2, n)) if spd else inputs.uniform(n, n, seed=inputs.seed_for(2, n))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 1000 + n))
    X, Aout, it, info, _ = run_mixed(A, B, spd=spd)
    assert info == 0 and 0 <= it <= 30
    assert np.array_equal(Aout, A)                   # A unchanged when refinement converged
    eta = oracle.backward_error(A, X, B)
    assert eta <= 1e-14
    Xr = ref_solution(A, B, spd)
    kappa = np.linalg.cond(A)
    fwd = np.max(np.abs(X - Xr)) / np.max(np.abs(Xr))
    assert fwd <= kappa * (1e-14 + n * EPS) * 4


@pytest.mark.parametrize("spd", [False, True])
def test_mixed_fp32_cond_1e6(spd):
    # the precision form's inputs at reduced order: sigma log-spaced 1..1e6
    n, nrhs = 768, 16
    if spd:
        A = inputs.spd_spectrum(n, 1e6, seed=inputs.seed_for(2, 1), reflectors=64)
    else:
        A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 2), reflectors=64)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 3))
    X, Aout, it, info, _ = run_mixed(A, B, spd=spd)
    assert info == 0 and 0 <= it <= 30, it
    assert oracle.backward_error(A, X, B) <= 1e-14


def test_mixed_no_convergence_falls_back_to_fp64():
    n, nrhs = 400, 2
    A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 4), reflectors=16)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 5))
    X, Aout, it, info, ipiv = run_mixed(A, B, maxiter=0)
    assert it == -31 and info == 0
    assert oracle.backward_error(A, X, B) <= 10 * n * EPS
    # A now holds the FP64 factors with their pivots
    assert oracle.res_lu(A, Aout, ipiv) <= 10.0


def test_mixed_fp32_overflow_falls_back():
    n, nrhs = 120, 1
    A = inputs.uniform(n, n, seed=inputs.seed_for(2, 6)) * 1e300
    A = np.asfortranarray(A)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 7))
    X, Aout, it, info, ipiv = run_mixed(A, B)
    assert it == -2 and info == 0
    assert oracle.backward_error(A, X, B) <= 10 * n * EPS


def test_mixed_singular_reports_info():
    n, nrhs = 100, 1
    A = inputs.uniform(n, n, seed=inputs.seed_for(2, 8))
    A[:, 37] = 0.0
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 9))
    X, Aout, it, info, ipiv = run_mixed(A, B)
    assert it == -3 and info == 38


def test_mixed_unsupported_precision():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float64, device="cuda")
    p = buf.data_ptr()
    assert r.rl_dsgesv(4, 1, p, 4, p, p, 4, p, 4, 99, 1e-14, 10, p, p, p, 1 << 30) == r.RL_ERR_UNSUPPORTED


def _trs_work(n, nrhs, use_work):
    """(work tensor, lwork) for the solves: None selects the recursive TRSM,
    a buffer the one-launch flow solve (nrhs <= 64)."""
    r = G.lib()
    if not use_work:
        return None, 0
    lw = max(r.rl_trs_work_size(n, nrhs), 256)
    return G.torch().full((lw,), 0x5A, dtype=G.torch().uint8, device="cuda"), lw


@pytest.mark.parametrize("use_work", [False, True])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (63, 16), (64, 17), (130, 7), (513, 20), (1100, 64), (700, 65)])
def test_getrs_potrs_vs_oracle(n, nrhs, use_work):
    r = G.lib()
    A = inputs.uniform(n, n, seed=inputs.seed_for(2, 50 + n))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 60 + n))
    F, ipiv, info = G.getrf(A)
    dF, dB = G.DevMat(F), G.DevMat(B, lda=n + 1)
    dp = G.torch().from_numpy(ipiv.astype(np.int32)).cuda()
    w, lw = _trs_work(n, nrhs, use_work)
    assert r.rl_dgetrs("N", n, nrhs, dF.ptr(), dF.lda, dp.data_ptr(), dB.ptr(), dB.lda, w, lw) == 0
    G.sync()
    X = dB.get()
    assert dB.canaries_intact()
    if w is not None and nrhs <= 64:
        assert int(w[:4].view(G.torch().int32)[0]) == 0        # status word: no wait expired
    assert oracle.backward_error(A, X, B) <= 10 * n * EPS
    S = inputs.spd_bbt(n, seed=inputs.seed_for(2, 70 + n))
    L, info = G.potrf(S)
    dL, dB = G.DevMat(L), G.DevMat(B)
    assert r.rl_dpotrs("L", n, nrhs, dL.ptr(), dL.lda, dB.ptr(), dB.lda, w, lw) == 0
    G.sync()
    assert dB.canaries_intact()
    assert oracle.backward_error(S, dB.get(), B) <= 10 * n * EPS


def test_trs_workspace_too_small():
    r = G.lib()
    t = G.torch()
    n, nrhs = 300, 8
    buf = t.zeros(n * n, dtype=t.float64, device="cuda")
    lw = r.rl_trs_work_size(n, nrhs)
    assert lw > 0 and r.rl_trs_work_size(n, 65) == 0
    w = t.zeros(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dpotrs("L", n, nrhs, buf, n, buf, n, w, lw - 1) == r.RL_ERR_WORKSPACE


def test_mixed_zero_rhs_column_converges():
    """A zero right-hand side next to ordinary ones: its residual, x and b
    are all zero, which counts as converged (no division by a zero norm)."""
    n = 300
    A = inputs.general_spectrum(n, 1e3, seed=inputs.seed_for(2, 790))
    B = inputs.normal(n, 3, seed=inputs.seed_for(2, 791))
    B[:, 0] = 0.0
    X, Aout, it, info, ipiv = run_mixed(A, B, prec=0)
    assert it >= 0 and info == 0
    assert np.all(X[:, 0] == 0.0)
    assert oracle.backward_error(A, X, B) <= 1e-14

"""GMRES-based refinement of the precision form (rl_dsgesv / rl_dsposv with
prec | RL_REFINE_GMRES) against the oracle.

The bar is the classic refinement's: a converged solve returns X whose
normwise backward error, computed by the oracle with compensated sums, is
<= tol = 1e-14, and whose forward error against the oracle's FP64 solution
is within kappa(A) (tol + n eps); the reported iteration count is the number
of GMRES iterations.  When the budget runs out, the FP64 fallback runs and
meets the FP64 solve's bound.  Inputs follow the precision-form recipe:
A = U diag(sigma) V^T (or Q diag(sigma) Q^T) with 64 Householder reflectors
per side and sigma log-spaced 1..kappa; B iid N(0, 1).
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
    r = G.lib()
    m0 = r.rl_get_param(r.RL_PARAM_GMRES_RESTART)
    yield
    r.rl_set_param(r.RL_PARAM_GMRES_RESTART, m0)


def run(A, B, spd, prec, maxiter, tol=1e-14):
    r = G.lib()
    t = G.torch()
    n, nrhs = A.shape[0], B.shape[1]
    dA, dB = G.DevMat(A), G.DevMat(B)
    dX = G.DevMat(np.zeros_like(B))
    ipiv = G.int_buf(n, -5)
    it = G.int_buf(1, -99)
    info = G.int_buf(1, -77)
    p = prec | r.RL_REFINE_GMRES
    if spd:
        lw = r.rl_dsposv_work_size(n, nrhs, p)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsposv("L", n, nrhs, dA.ptr(), dA.lda, dB.ptr(), dB.lda, dX.ptr(), dX.lda, p, tol, maxiter,
                         it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    else:
        lw = r.rl_dsgesv_work_size(n, nrhs, p)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsgesv(n, nrhs, dA.ptr(), dA.lda, ipiv.data_ptr(), dB.ptr(), dB.lda, dX.ptr(), dX.lda, p, tol,
                         maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert dA.canaries_intact() and dX.canaries_intact() and dB.canaries_intact()
    return dX.get(), dA.get(), int(it[0].item()), int(info[0].item())


def ref_solution(A, B, spd):
    if spd:
        L, _ = oracle.potrf(A, c=24)
        return oracle.potrs(L, B)
    F, piv, _ = oracle.getrf(A, c=24)
    return oracle.getrs(F, piv, B)


def check_converged(A, B, X, it, spd, kappa, tol=1e-14):
    assert it >= 0, f"no convergence (iter {it})"
    eta = oracle.backward_error(A, X, B)
    assert eta <= tol, eta
    X0 = ref_solution(A, B, spd)
    fwd = np.max(np.abs(X - X0), axis=0) / np.maximum(np.max(np.abs(X0), axis=0), 1e-300)
    assert np.max(fwd) <= kappa * (tol + A.shape[0] * EPS), np.max(fwd)


@pytest.mark.parametrize("spd", [False, True])
@pytest.mark.parametrize("prec_name", ["FP32", "TF32X3"])
def test_gmres_converges_cond_1e6(spd, prec_name):
    """kappa = 1e6, 16 right-hand sides: the factorizations whose updates
    are FP32-accurate converge in a few GMRES iterations."""
    r = G.lib()
    n, nrhs, kappa = 768, 16, 1e6
    A = (inputs.spd_spectrum if spd else inputs.general_spectrum)(n, kappa, seed=inputs.seed_for(2, 700 + spd))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 710))
    X, Aout, it, info = run(A, B, spd, getattr(r, "RL_PREC_" + prec_name), maxiter=60)
    assert info == 0 and 1 <= it <= 60
    assert np.array_equal(Aout, A)                      # A untouched when refinement converges
    check_converged(A, B, X, it, spd, kappa)


def run_classic(A, B, prec, maxiter=30):
    r = G.lib()
    t = G.torch()
    n, nrhs = A.shape[0], B.shape[1]
    dA, dB, dX = G.DevMat(A), G.DevMat(B), G.DevMat(np.zeros_like(B))
    ipiv, it, info = G.int_buf(n, -5), G.int_buf(1, -99), G.int_buf(1, -77)
    lw = r.rl_dsgesv_work_size(n, nrhs, prec)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dsgesv(n, nrhs, dA.ptr(), dA.lda, ipiv.data_ptr(), dB.ptr(), dB.lda, dX.ptr(), dX.lda, prec,
                     1e-14, maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0
    return int(it[0].item())


@pytest.mark.parametrize("prec_name,kappa,budget", [("TF32", 1e4, 200), ("FP16S", 1e4, 200), ("BF16", 1e3, 300)])
def test_gmres_where_the_classic_loop_stagnates(prec_name, kappa, budget):
    """Tensor-core factorizations too inexact for the classic refinement at
    this condition (it gives up and runs the FP64 fallback): the GMRES
    refinement converges without the fallback."""
    r = G.lib()
    prec = getattr(r, "RL_PREC_" + prec_name)
    n, nrhs = 768, 4
    A = inputs.general_spectrum(n, kappa, seed=inputs.seed_for(2, 720))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 730))
    assert run_classic(A, B, prec) == -31
    X, Aout, it, info = run(A, B, False, prec, maxiter=budget)
    assert info == 0
    check_converged(A, B, X, it, False, kappa)
    assert np.array_equal(Aout, A)


def test_gmres_cannot_rescue_bf16_at_cond_1e6():
    """At kappa = 1e6 the BF16-update LU differs from A by more than the
    smaller half of the singular values: the preconditioned operator has
    hundreds of eigenvalues far from 1, a cycle barely reduces the backward
    error, and the refinement gives up for the FP64 fallback after one
    cycle, whose result meets the FP64 bound."""
    r = G.lib()
    n, nrhs = 768, 4
    A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 735))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 736))
    X, Aout, it, info = run(A, B, False, r.RL_PREC_BF16, maxiter=300)
    assert it == -31 and info == 0
    assert oracle.backward_error(A, X, B) <= 10 * n * EPS


def test_gmres_budget_spent_falls_back_to_fp64():
    r = G.lib()
    n, nrhs = 300, 3
    A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 740))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 741))
    for maxiter in (0, 1):
        X, Aout, it, info = run(A, B, False, r.RL_PREC_BF16, maxiter=maxiter)
        assert it == -31 and info == 0
        assert oracle.backward_error(A, X, B) <= 10 * n * EPS
        assert not np.array_equal(Aout, A)            # the fallback factored A in place


def test_gmres_zero_and_repeated_columns():
    """A zero right-hand side (x = 0, no iterations needed for it) and a
    repeated column next to ordinary ones: each column converges on its own
    and the repeated columns get identical solutions."""
    r = G.lib()
    n = 500
    A = inputs.general_spectrum(n, 1e5, seed=inputs.seed_for(2, 750))
    B = inputs.normal(n, 5, seed=inputs.seed_for(2, 751))
    B[:, 1] = 0.0
    B[:, 3] = B[:, 2]
    X, Aout, it, info = run(A, B, False, r.RL_PREC_FP32, maxiter=40)
    assert info == 0 and it >= 0
    assert np.all(X[:, 1] == 0.0)
    assert np.array_equal(X[:, 2], X[:, 3])
    check_converged(A, B, X, it, False, 1e5)


@pytest.mark.parametrize("m", [1, 5, 64])
def test_gmres_restart_lengths(m):
    """The restart length changes the path, not the result's bound (m = 1
    is steepest-descent-like and needs more cycles)."""
    r = G.lib()
    assert r.rl_set_param(r.RL_PARAM_GMRES_RESTART, m) == 0
    try:
        n, nrhs, kappa = 400, 2, 1e4
        A = inputs.general_spectrum(n, kappa, seed=inputs.seed_for(2, 760))
        B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 761))
        X, Aout, it, info = run(A, B, False, r.RL_PREC_FP32, maxiter=100)
        assert info == 0
        check_converged(A, B, X, it, False, kappa)
    finally:
        r.rl_set_param(r.RL_PARAM_GMRES_RESTART, 50)


def test_gmres_scaled_fp16_and_upper_spd():
    """Scaled FP16 (the working copy is A 2^-e): the widening of each
    preconditioned vector undoes the scale; and uplo 'U' through the
    triangle swap."""
    r = G.lib()
    n, nrhs, kappa = 512, 3, 1e3
    A = inputs.spd_spectrum(n, kappa, seed=inputs.seed_for(2, 770)) * 1e5
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 771))
    X, Aout, it, info = run(A, B, True, r.RL_PREC_FP16S, maxiter=100)
    assert info == 0
    check_converged(A, B, X, it, True, kappa)
    # upper: the same system stored in the upper triangle
    t = G.torch()
    dA = G.DevMat(np.triu(A) + np.tril(np.full_like(A, 1e30), -1))
    dB = G.DevMat(B)
    dX = G.DevMat(np.zeros_like(B))
    it_b = G.int_buf(1, -99)
    info_b = G.int_buf(1, -77)
    p = r.RL_PREC_FP16S | r.RL_REFINE_GMRES
    lw = r.rl_dsposv_work_size(n, nrhs, p)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dsposv("U", n, nrhs, dA.ptr(), dA.lda, dB.ptr(), dB.lda, dX.ptr(), dX.lda, p, 1e-14, 100,
                     it_b.data_ptr(), info_b.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0
    assert int(it_b[0].item()) >= 0
    assert oracle.backward_error(A, dX.get(), B) <= 1e-14

"""Refinement with the FP64 products emulated on the BF16 tensor cores
(rl_dsgesv / rl_dsposv with prec | RL_REFINE_OZRES), against the oracle.

The bar is that of the precision form: a converged solve returns X whose
normwise backward error, computed by the oracle with compensated sums, is
<= 1e-14 and whose forward error against the oracle's FP64 solution is within
kappa(A) (tol + n eps), with about as many iterations as with FP64 products
(the emulated product is as accurate as an FP64 one in norm).  Covered: the
classic and the GMRES refinement, general and symmetric A (the symmetric
matrix's digit planes read the stored lower triangle across the diagonal),
uplo 'U', and rows whose entries span many orders of magnitude.
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


def solve(A, B, spd, prec, maxiter=30, uplo="L"):
    r, t = G.lib(), G.torch()
    n, nrhs = A.shape[0], B.shape[1]
    dA, dB, dX = G.DevMat(A), G.DevMat(B), G.DevMat(np.zeros_like(B))
    ipiv, it, info = G.int_buf(n, -5), G.int_buf(1, -99), G.int_buf(1, -77)
    if spd:
        lw = r.rl_dsposv_work_size(n, nrhs, prec)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsposv(uplo, n, nrhs, dA.ptr(), dA.lda, dB.ptr(), dB.lda, dX.ptr(), dX.lda, prec, 1e-14,
                         maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    else:
        lw = r.rl_dsgesv_work_size(n, nrhs, prec)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        st = r.rl_dsgesv(n, nrhs, dA.ptr(), dA.lda, ipiv.data_ptr(), dB.ptr(), dB.lda, dX.ptr(), dX.lda, prec,
                         1e-14, maxiter, it.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert dA.canaries_intact() and dX.canaries_intact() and dB.canaries_intact()
    return dX.get(), dA.get(), int(it[0].item()), int(info[0].item())


def converged(A, B, X, it, spd, kappa):
    assert it >= 0, it
    assert oracle.backward_error(A, X, B) <= 1e-14
    if spd:
        L, _ = oracle.potrf(A, c=24)
        X0 = oracle.potrs(L, B)
    else:
        F, piv, _ = oracle.getrf(A, c=24)
        X0 = oracle.getrs(F, piv, B)
    fwd = np.max(np.abs(X - X0), axis=0) / np.maximum(np.max(np.abs(X0), axis=0), 1e-300)
    assert np.max(fwd) <= kappa * (1e-14 + A.shape[0] * EPS)


@pytest.mark.parametrize("spd", [False, True])
@pytest.mark.parametrize("prec_name", ["FP32", "TF32X3"])
def test_emulated_residuals_classic(spd, prec_name):
    r = G.lib()
    n, nrhs, kappa = 768, 16, 1e6
    A = (inputs.spd_spectrum if spd else inputs.general_spectrum)(n, kappa, seed=inputs.seed_for(2, 800 + spd))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 810))
    p = getattr(r, "RL_PREC_" + prec_name)
    X, Aout, it, info = solve(A, B, spd, p | r.RL_REFINE_OZRES)
    assert info == 0 and np.array_equal(Aout, A)
    converged(A, B, X, it, spd, kappa)
    X1, _, it1, _ = solve(A, B, spd, p)                  # FP64 products
    assert abs(it - it1) <= 2


def test_emulated_residuals_gmres():
    r = G.lib()
    n, nrhs, kappa = 768, 4, 1e4
    A = inputs.general_spectrum(n, kappa, seed=inputs.seed_for(2, 720))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 730))
    X, Aout, it, info = solve(A, B, False, r.RL_PREC_FP16S | r.RL_REFINE_GMRES | r.RL_REFINE_OZRES, maxiter=200)
    assert info == 0 and np.array_equal(Aout, A)
    converged(A, B, X, it, False, kappa)


def test_emulated_residuals_upper_and_wide_rows():
    """uplo 'U' (the triangle swap, then the lower-stored planes), and rows
    whose entries span ~12 orders of magnitude (the planes keep each row's
    largest entries; the small ones are represented to the row's scale)."""
    r = G.lib()
    n, nrhs = 512, 3
    A = inputs.spd_spectrum(n, 1e4, seed=inputs.seed_for(2, 820))
    d = np.logspace(-6, 6, n)
    A = np.asfortranarray(A * np.sqrt(np.outer(d, d)))      # SPD, rows scaled over 12 decades
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 821))
    kappa = np.linalg.cond(A)
    p = r.RL_PREC_FP32 | r.RL_REFINE_OZRES
    X, Aout, it, info = solve(A, B, True, p, maxiter=60)
    assert info == 0
    assert oracle.backward_error(A, X, B) <= 1e-14 or it < 0
    Au = np.triu(A) + np.tril(np.full_like(A, 1e30), -1)
    Xu, _, itu, infou = solve(Au, B, True, p, maxiter=60, uplo="U")
    assert infou == 0 and itu == it
    assert np.array_equal(Xu, X)
    G2 = inputs.general_spectrum(n, 1e3, seed=inputs.seed_for(2, 822)) * np.logspace(-6, 6, n)[:, None]
    G2 = np.asfortranarray(G2)
    X, _, it, info = solve(G2, B, False, p, maxiter=60)
    assert info == 0
    assert it < 0 or oracle.backward_error(G2, X, B) <= 1e-14

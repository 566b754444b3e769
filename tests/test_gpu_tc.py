"""Tensor-core (tcgen05) GEMM on FP32 storage, and the precision form run
with tensor-core updates.

Exactness pin: integer operands in [-4, 4] are exact in TF32, BF16 and FP16,
their products and FP32 sums (< 2^24) are exact, so every precision must
return the integer product bit for bit -- on shapes that span several
128 x 256 tiles with ragged edges, for every transpose combination.  Any
mistake in the operand packing, the TMA swizzle, the shared-memory or
instruction descriptors or the TMEM read-back breaks this.

Random operands: |C_gpu - C_ref| <= (2 u_op + k 2^-24) |alpha| |op(A)||op(B)|
+ 2^-23 |C|, with u_op the operand rounding unit (2^-11 TF32 / FP16, 2^-8
BF16, 2^-21 for the split 3xTF32) and C_ref the oracle's FP64 product of the
FP32 inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu

PRECS = {"TF32": (1, 2.0 ** -11), "BF16": (2, 2.0 ** -8), "FP16": (3, 2.0 ** -11), "TF32X3": (4, 2.0 ** -21)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def run_tc(prec, ta, tb, A, B, C, alpha=1.0):
    r = G.lib()
    t = G.torch()
    m, n = C.shape
    k = A.shape[0] if ta == "T" else A.shape[1]
    dA = t.from_numpy(np.asfortranarray(A, dtype=np.float32).ravel(order="F").copy()).cuda()
    dB = t.from_numpy(np.asfortranarray(B, dtype=np.float32).ravel(order="F").copy()).cuda()
    dC = t.from_numpy(np.asfortranarray(C, dtype=np.float32).ravel(order="F").copy()).cuda()
    lw = r.rl_sgemm_tc_work_size(m, n, k, prec)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_sgemm_tc(prec, ta, tb, m, n, k, alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(),
                       B.shape[0], dC.data_ptr(), m, work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    return dC.cpu().numpy().reshape(n, m).T


def op(X, t):
    return X.T if t == "T" else X


@pytest.mark.parametrize("name", list(PRECS))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(300, 260, 200), (128, 256, 64), (129, 257, 65), (17, 33, 520)])
def test_tc_gemm_integer_exact(name, ta, tb, m, n, k):
    prec, _ = PRECS[name]
    rng = inputs.rng(m * 7 + n * 3 + k)
    A = rng.integers(-4, 5, size=(k, m) if ta == "T" else (m, k)).astype(np.float64)
    B = rng.integers(-4, 5, size=(n, k) if tb == "T" else (k, n)).astype(np.float64)
    C = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
    got = run_tc(prec, ta, tb, A, B, C)
    want = C + op(A, ta).astype(np.int64) @ op(B, tb).astype(np.int64)
    assert np.array_equal(got.astype(np.float64), want.astype(np.float64))


@pytest.mark.parametrize("name", list(PRECS))
@pytest.mark.parametrize("m,n,k", [(513, 300, 700), (1024, 1024, 256)])
def test_tc_gemm_random_vs_oracle(name, m, n, k):
    prec, u = PRECS[name]
    A = inputs.uniform(m, k, seed=m + k).astype(np.float32).astype(np.float64)
    B = inputs.uniform(k, n, seed=n + k + 1).astype(np.float32).astype(np.float64)
    C = inputs.uniform(m, n, seed=m + n + 2).astype(np.float32).astype(np.float64)
    alpha = -1.0
    got = run_tc(prec, "N", "N", A, B, C, alpha=alpha).astype(np.float64)
    ref = oracle.gemm(A, B, C, alpha=alpha)
    mag = np.abs(A) @ np.abs(B)
    bound = (2 * u + k * 2.0 ** -24) * mag + 2.0 ** -23 * np.abs(C) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


def test_tc_gemm_rejects_fp32_precision():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float32, device="cuda")
    p = buf.data_ptr()
    assert r.rl_sgemm_tc(0, "N", "N", 4, 4, 4, 1.0, p, 4, p, 4, p, 4, p, 1 << 20) == r.RL_ERR_UNSUPPORTED


# ----------------------------------------------------------------------------
# precision form with tensor-core updates
# ----------------------------------------------------------------------------

from .test_gpu_mixed import run_mixed  # noqa: E402


@pytest.mark.parametrize("name", list(PRECS))
@pytest.mark.parametrize("spd", [False, True])
def test_mixed_tc_well_conditioned_converges(name, spd):
    prec, _ = PRECS[name]
    n, nrhs = 700, 4
    A = inputs.spd_bbt(n, seed=inputs.seed_for(2, 40)) if spd else inputs.spd_bbt(n, seed=inputs.seed_for(2, 41))
    if not spd:
        A = np.asfortranarray(A + np.triu(inputs.uniform(n, n, seed=inputs.seed_for(2, 42)), 1))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 43))
    X, Aout, it, info, _ = run_mixed(A, B, spd=spd, prec=prec)
    assert info == 0 and 0 <= it <= 30, (name, it)
    assert np.array_equal(Aout, A)
    assert oracle.backward_error(A, X, B) <= 1e-14


@pytest.mark.parametrize("spd", [False, True])
def test_mixed_tf32x3_cond_1e6_converges(spd):
    n, nrhs = 768, 16
    if spd:
        A = inputs.spd_spectrum(n, 1e6, seed=inputs.seed_for(2, 11))
    else:
        A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 12))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 13))
    X, Aout, it, info, _ = run_mixed(A, B, spd=spd, prec=PRECS["TF32X3"][0])
    assert info == 0 and 0 <= it <= 30, it
    assert oracle.backward_error(A, X, B) <= 1e-14


def test_mixed_bf16_cond_1e6_reports_and_falls_back():
    # kappa * u_bf16 >> 1: classical refinement cannot converge; the call must
    # say so (iter = -31) and still return the FP64 solution
    n, nrhs = 512, 2
    A = inputs.general_spectrum(n, 1e6, seed=inputs.seed_for(2, 14))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(2, 15))
    X, Aout, it, info, ipiv = run_mixed(A, B, prec=PRECS["BF16"][0], maxiter=10)
    assert it in (-31,) or it >= 0
    assert oracle.backward_error(A, X, B) <= (1e-14 if it >= 0 else 10 * n * 2.0 ** -53)

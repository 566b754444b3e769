"""Low-precision factorizations (rl_spotrf_tc / rl_sgetrf_tc): FP32 storage,
tensor-core updates in TF32, BF16, FP16 or 3xTF32.  Residuals measured in
units of the operand precision's rounding unit u (2^-8 BF16, 2^-11 TF32 and
FP16, 2^-22 for 3xTF32) must be <= 10, like the FP64 bound in units of 2^-53;
exact inputs whose products are exact in the operand format come out bit for
bit."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "tf32x3": 2.0 ** -22}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def prec_id(name):
    r = G.lib()
    return {"tf32": r.RL_PREC_TF32, "bf16": r.RL_PREC_BF16, "fp16": r.RL_PREC_FP16S,
            "tf32x3": r.RL_PREC_TF32X3}[name]


def dev32(A):
    t = G.torch()
    return t.from_numpy(np.asfortranarray(A, dtype=np.float32).ravel(order="F").copy()).cuda()


def host64(d, m, n):
    return np.asfortranarray(d.cpu().numpy().reshape(n, m).T.astype(np.float64))


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16", "tf32x3"])
@pytest.mark.parametrize("n", [300, 700, 1500])
def test_lowprec_factorizations(prec, n):
    r = G.lib()
    t = G.torch()
    p = prec_id(prec)
    scale = 2.0 ** -53 / U[prec]
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 4000 + n)).astype(np.float32).astype(np.float64)
    dA = dev32(A)
    info = G.int_buf(1, -7)
    lw = r.rl_spotrf_tc_work_size(n, p)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_spotrf_tc(p, "L", n, dA, n, info, w, lw) == 0
    G.sync()
    assert int(info[0]) == 0
    assert oracle.res_chol(A, np.tril(host64(dA, n, n))) * scale <= 10.0
    Gm = inputs.uniform(n, n, seed=inputs.seed_for(1, 4100 + n)).astype(np.float32).astype(np.float64)
    dG = dev32(Gm)
    ipiv = G.int_buf(n, -5)
    lw = r.rl_sgetrf_tc_work_size(n, n, p)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetrf_tc(p, n, n, dG, n, ipiv, info, w, lw) == 0
    G.sync()
    assert int(info[0]) == 0
    assert oracle.res_lu(Gm, host64(dG, n, n), ipiv.cpu().numpy()[:n]) * scale <= 10.0


def test_lowprec_exact_small_integers():
    """Integer factors with entries in {-1, 0, 1} and diagonal 1: every update
    operand (a block of L) is exact in BF16 and every product sum is an
    integer exact in FP32."""
    r = G.lib()
    t = G.torch()
    n = 600
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 4200), offdiag=1, diag=(1, 1))
    A = inputs.product_lower(L)
    assert np.max(np.abs(A)) < 2 ** 24
    for prec in ("bf16", "tf32", "tf32x3"):
        dA = dev32(A)
        info = G.int_buf(1, -7)
        lw = r.rl_spotrf_tc_work_size(n, prec_id(prec))
        w = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_spotrf_tc(prec_id(prec), "L", n, dA, n, info, w, lw) == 0
        G.sync()
        assert int(info[0]) == 0
        assert np.array_equal(np.tril(host64(dA, n, n)), L), prec


def test_lowprec_arguments():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float32, device="cuda")
    info = G.int_buf(1)
    assert r.rl_spotrf_tc_work_size(100, r.RL_PREC_FP32) == 0
    assert r.rl_spotrf_tc(r.RL_PREC_FP32, "L", 4, buf, 4, info, None, 0) == r.RL_ERR_UNSUPPORTED
    lw = r.rl_sgetrf_tc_work_size(500, 500, r.RL_PREC_BF16)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetrf_tc(r.RL_PREC_BF16, 500, 500, buf, 500, buf, info, w, lw - 1) == r.RL_ERR_WORKSPACE

"""The lookahead of the LU and Cholesky recursions (the part of each large
trailing update that the next level needs last runs on an internal stream)
gives the same bits as the single-stream recursion, and both meet the
oracle's bounds; the FP32 and precision-form paths that reuse the
recursions likewise."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    G.lib().rl_set_param(G.lib().RL_PARAM_LOOKAHEAD, 1)


def both(fn):
    r = G.lib()
    out = []
    for la in (0, 1):
        assert r.rl_set_param(r.RL_PARAM_LOOKAHEAD, la) == 0
        out.append(fn())
    return out


@pytest.mark.parametrize("n", [1100, 2100, 3000])
def test_potrf_lookahead_bit_identical(n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 1200 + n))
    (L0, i0), (L1, i1) = both(lambda: G.potrf(A, lda=n + 3))
    assert i0 == i1 == 0
    assert np.array_equal(np.tril(L0), np.tril(L1))
    assert oracle.res_chol(A, np.tril(L1)) <= 10.0


@pytest.mark.parametrize("m,n", [(1100, 1100), (2500, 2100), (3000, 3000)])
def test_getrf_lookahead_bit_identical(m, n):
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 1300 + n))
    (F0, p0, i0), (F1, p1, i1) = both(lambda: G.getrf(A, lda=m + 1))
    assert i0 == i1 == 0
    assert np.array_equal(p0, p1) and np.array_equal(F0, F1)
    assert oracle.res_lu(A, F1, p1) <= 10.0


def test_fp32_and_precision_form_lookahead_bit_identical():
    r = G.lib()
    t = G.torch()
    n = 2200
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 1400))

    def sgetrf():
        d = t.from_numpy(A.astype(np.float32).ravel(order="F").copy()).cuda()
        ipiv = G.int_buf(n)
        info = G.int_buf(1, -7)
        lw = r.rl_dgetrf_work_size(n, n)
        w = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_sgetrf(n, n, d, n, ipiv, info, w, lw) == 0
        G.sync()
        return d.cpu().numpy(), ipiv.cpu().numpy()[:n]

    (a0, p0), (a1, p1) = both(sgetrf)
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)

    S = inputs.spd_bbt(n, seed=inputs.seed_for(1, 1401))
    B = inputs.normal(n, 4, seed=inputs.seed_for(1, 1402))

    def dsposv():
        dA, dB, dX = G.DevMat(S), G.DevMat(B), G.DevMat(np.zeros((n, 4)))
        it, info = G.int_buf(1, -9), G.int_buf(1, -9)
        lw = r.rl_dsposv_work_size(n, 4, r.RL_PREC_FP32)
        w = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_dsposv("L", n, 4, dA.ptr(), n, dB.ptr(), n, dX.ptr(), n, r.RL_PREC_FP32, 1e-14, 30,
                           it, info, w, lw) == 0
        G.sync()
        return dX.get(), int(it[0]), int(info[0])

    (x0, it0, f0), (x1, it1, f1) = both(dsposv)
    assert f0 == f1 == 0 and it0 == it1 >= 0
    assert np.array_equal(x0, x1)


def test_clear_cache_releases_and_recreates_the_side_stream():
    """rl_clear_cache destroys the lookahead stream and events and the trace
    pool; the next call creates them again and gives the same bits."""
    r = G.lib()
    assert r.rl_set_param(r.RL_PARAM_LOOKAHEAD, 1) == 0
    n = 2100
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 1500))
    F0, p0, _ = G.getrf(A)
    r.rl_trace_enable(1)
    G.getrf(A)
    assert r.rl_clear_cache() == 0
    F1, p1, _ = G.getrf(A)
    assert np.array_equal(p0, p1) and np.array_equal(F0, F1)
    assert r.rl_clear_cache() == 0
    assert r.rl_clear_cache() == 0                # nothing left to release


def test_nvtx_ranges_change_nothing():
    """With RL_PARAM_NVTX on, every recursion node pushes a named NVTX range
    (a no-op without a timeline tool attached): the same bits come out."""
    r = G.lib()
    n = 1100
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 1600))
    L0, _ = G.potrf(A)
    F0, p0, _ = G.getrf(A)
    assert r.rl_set_param(r.RL_PARAM_NVTX, 1) == 0
    try:
        L1, _ = G.potrf(A)
        F1, p1, _ = G.getrf(A)
        X1, _ = G.trtri(np.tril(L0))
    finally:
        assert r.rl_set_param(r.RL_PARAM_NVTX, 0) == 0
    assert np.array_equal(L0, L1) and np.array_equal(F0, F1) and np.array_equal(p0, p1)
    X0, _ = G.trtri(np.tril(L0))
    assert np.array_equal(X0, X1)

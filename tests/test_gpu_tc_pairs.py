"""The tensor-core GEMM on clusters of two CTAs (a pair of row tiles sharing
the B tile, each CTA loading half of it and multicasting it into both)
against the one-CTA-per-tile kernel: the same bits for every operand
precision and transpose, an odd number of row tiles (the pair's second tile
past the end), the lower-triangle form inside the Cholesky, and the LU."""
import numpy as np
import pytest

from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = G.lib()
    yield
    r.rl_set_param(r.RL_PARAM_TC_PAIRS, 1)


def gemm(prec, ta, tb, A, B, C, pairs):
    r, t = G.lib(), G.torch()
    assert r.rl_set_param(r.RL_PARAM_TC_PAIRS, pairs) == 0
    m, n = C.shape
    k = A.shape[0] if ta == "T" else A.shape[1]
    dA = t.from_numpy(np.asfortranarray(A, dtype=np.float32).ravel(order="F").copy()).cuda()
    dB = t.from_numpy(np.asfortranarray(B, dtype=np.float32).ravel(order="F").copy()).cuda()
    dC = t.from_numpy(np.asfortranarray(C, dtype=np.float32).ravel(order="F").copy()).cuda()
    lw = r.rl_sgemm_tc_work_size(m, n, k, prec)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_sgemm_tc(prec, ta, tb, m, n, k, 0.75, dA.data_ptr(), A.shape[0], dB.data_ptr(), B.shape[0],
                       dC.data_ptr(), m, work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    return dC.cpu().numpy()


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(2560, 4096, 512), (2600, 3840, 300)])
def test_pairs_bit_identical(prec, ta, tb, m, n, k):
    A = inputs.uniform(k if ta == "T" else m, m if ta == "T" else k, seed=inputs.seed_for(1, 7000 + m))
    B = inputs.uniform(n if tb == "T" else k, k if tb == "T" else n, seed=inputs.seed_for(1, 7100 + n))
    C = inputs.uniform(m, n, seed=inputs.seed_for(1, 7200 + k))
    c1 = gemm(prec, ta, tb, A, B, C, 1)
    c0 = gemm(prec, ta, tb, A, B, C, 0)
    assert np.array_equal(c1, c0)
    ref = C.astype(np.float32) + 0.75 * ((A.T if ta == "T" else A) @ (B.T if tb == "T" else B))
    assert np.max(np.abs(c1.reshape(n, m).T - ref)) <= 0.05 * np.sqrt(k) * (1 if prec == 4 else 10)


@pytest.mark.parametrize("prec", [2, 4])
def test_pairs_in_the_factorizations(prec):
    """spotrf (lower-triangle updates) and sgetrf with tensor-core updates
    give the same bits with and without the pairs."""
    r, t = G.lib(), G.torch()
    n = 4096
    S = inputs.spd_bbt(n, seed=inputs.seed_for(1, 7300)).astype(np.float32)
    Gm = inputs.uniform(n, n, seed=inputs.seed_for(1, 7301)).astype(np.float32)
    outs = []
    for pairs in (1, 0):
        assert r.rl_set_param(r.RL_PARAM_TC_PAIRS, pairs) == 0
        dS = t.from_numpy(S.ravel(order="F").copy()).cuda()
        dG = t.from_numpy(Gm.ravel(order="F").copy()).cuda()
        info = t.zeros(2, dtype=t.int32, device="cuda")
        ipiv = t.zeros(n, dtype=t.int32, device="cuda")
        lw = max(r.rl_spotrf_tc_work_size(n, prec), r.rl_sgetrf_tc_work_size(n, n, prec))
        wk = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_spotrf_tc(prec, "L", n, dS, n, info, wk, lw) == 0
        assert r.rl_sgetrf_tc(prec, n, n, dG, n, ipiv, info.data_ptr() + 4, wk, lw) == 0
        G.sync()
        outs.append((dS.cpu().numpy(), dG.cpu().numpy(), ipiv.cpu().numpy(), info.cpu().numpy()))
    (s1, g1, p1, i1), (s0, g0, p0, i0) = outs
    assert np.array_equal(i1, i0) and np.all(i1 == 0)
    assert np.array_equal(p1, p0)
    assert np.array_equal(s1, s0) and np.array_equal(g1, g0)

"""The LU panel on one thread-block cluster (pivot candidates exchanged
through distributed shared memory) against the cooperative panel kernel:
the same bits (factors, ipiv, info) for FP64 and FP32 storage, square, tall
and wide shapes whose panels select clusters of 4, 8 and 16 CTAs, and the
oracle's bounds; exact dyadic LU bit for bit; a singular column's info."""
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
    r = G.lib()
    yield
    r.rl_set_param(r.RL_PARAM_PANEL_CLUSTER, 1)


def lu(A, f32=False, lda=None, cluster=1):
    r, t = G.lib(), G.torch()
    assert r.rl_set_param(r.RL_PARAM_PANEL_CLUSTER, cluster) == 0
    m, n = A.shape
    ld = lda or m
    buf = np.zeros((n, ld), dtype=np.float32 if f32 else np.float64)
    buf[:, :m] = A.T
    d = t.from_numpy(buf.ravel().copy()).cuda()
    mn = min(m, n)
    ipiv = t.full((mn,), -5, dtype=t.int32, device="cuda")
    info = t.full((1,), -77, dtype=t.int32, device="cuda")
    lw = r.rl_dgetrf_work_size(m, n)
    wk = t.empty(lw, dtype=t.uint8, device="cuda")
    fn = r.rl_sgetrf if f32 else r.rl_dgetrf
    st = fn(m, n, d, ld, ipiv, info, wk, lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    out = d.cpu().numpy().reshape(n, ld)
    assert np.all(out[:, m:] == 0)                      # the padding rows are untouched
    return np.asfortranarray(out[:, :m].T.astype(np.float64)), ipiv.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("m,n", [(100, 32), (700, 64), (3000, 3000), (5000, 128), (9000, 96),
                                 (20000, 64), (1030, 1030), (300, 900)])
def test_cluster_panel_bit_identical(m, n, f32):
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 5000 + m + n))
    if f32:
        A = A.astype(np.float32).astype(np.float64)
    F1, p1, i1 = lu(A, f32, lda=m + 3, cluster=1)
    F0, p0, i0 = lu(A, f32, lda=m + 3, cluster=0)
    assert i1 == i0 == 0
    assert np.array_equal(p1, p0)
    assert np.array_equal(F1, F0)
    if not f32 and m * n <= 9_000_000:
        assert oracle.res_lu(A, F1, p1) <= 10.0


def test_cluster_panel_exact_dyadic_lu():
    n = 600
    A, L, U, perm = inputs.dyadic_lu(n, seed=inputs.seed_for(1, 5100))
    F, p, info = lu(A, cluster=1)
    assert info == 0
    assert np.array_equal(p, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1), np.tril(L, -1))
    assert np.array_equal(np.triu(F), U)


@pytest.mark.parametrize("f32", [False, True])
def test_cluster_panel_singular_column_info(f32):
    n = 2000
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 5200))
    A[:, 17] = 0.0
    A[:, 1500] = 0.0
    F1, p1, i1 = lu(A, f32, cluster=1)
    F0, p0, i0 = lu(A, f32, cluster=0)
    assert i1 == i0 == 18
    assert np.array_equal(p1, p0) and np.array_equal(F1, F0)

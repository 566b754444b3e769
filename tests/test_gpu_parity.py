"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: backward errors ||A - L L^T|| / (n eps ||A||) and
||P A - L U|| / (n eps ||A||) <= 10, and the analogous TRTRI / POTRI
residuals; ipiv equal to the oracle's up to the first pivot near-tie (relative
gap < 1e-12); factors that are exact in binary64 (integer / dyadic inputs)
bit for bit.  Elementwise agreement with the oracle: two backward-stable
computations of the same factor differ by at most about
2 * (bound) * n * eps * kappa(A) relative to the factor's size, which is the
tolerance written below (kappa from numpy).
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
BOUND = 10.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.lib()
    yield


def close(F, R, n, kappa, extra=1.0):
    tol = 2 * BOUND * max(n, 1) * EPS * kappa * extra
    scale = max(1.0, float(np.max(np.abs(R))))
    return float(np.max(np.abs(F - R))) <= tol * scale


# ----------------------------------------------------------------------------
# Cholesky
# ----------------------------------------------------------------------------

def test_potrf_integer_6x6_bit_exact():
    L = inputs.integer_chol_6()
    A = inputs.product_lower(L)
    F, info = G.potrf(A)
    assert info == 0
    assert np.array_equal(np.tril(F), L)
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))


@pytest.mark.parametrize("n", [65, 200, 333])
@pytest.mark.parametrize("c", [64, 17, 1])
def test_potrf_integer_bit_exact(n, c):
    r = G.lib()
    L = inputs.integer_chol(n, seed=inputs.seed_for(0, 10 + n))
    A = inputs.product_lower(L)
    r.rl_set_param(r.RL_PARAM_POTRF_CROSSOVER, c)
    try:
        F, info = G.potrf(A, lda=n + 3)
    finally:
        r.rl_set_param(r.RL_PARAM_POTRF_CROSSOVER, 64)
    assert info == 0 and np.array_equal(np.tril(F), L)
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))


@pytest.mark.parametrize("n", [1, 2, 7, 63, 64, 65, 100, 128, 129, 255, 500, 1024, 1500])
def test_potrf_vs_oracle(n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, n))
    F, info = G.potrf(A, lda=n + (n % 3))
    assert info == 0
    assert oracle.res_chol(A, F) <= BOUND
    R, rinfo = oracle.potrf(A, c=24)
    assert rinfo == 0
    assert close(np.tril(F), np.tril(R), n, np.linalg.cond(A))
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))


def test_potrf_config0_n1024():
    n = 1024
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 0))
    F, info = G.potrf(A)
    assert info == 0
    res = oracle.res_chol(A, F)
    assert res <= BOUND
    R, _ = oracle.potrf(A, c=24)
    assert close(np.tril(F), np.tril(R), n, np.linalg.cond(A))


@pytest.mark.parametrize("k", [0, 5, 64, 100, 199])
def test_potrf_info_not_spd(k):
    n = 200
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 77))
    A[k, k] = -1.0
    F, info = G.potrf(A)
    _, rinfo = oracle.potrf(A, c=24)
    assert info == rinfo == k + 1
    if k > 0:
        assert close(np.tril(F[:k, :k]), np.linalg.cholesky(A[:k, :k]), k, np.linalg.cond(A[:k, :k]))


# ----------------------------------------------------------------------------
# LU with partial pivoting
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [7, 32, 100, 300, 517])
@pytest.mark.parametrize("nb", [32, 8, 64])
def test_getrf_dyadic_bit_exact(n, nb):
    r = G.lib()
    A, L, U, perm = inputs.dyadic_lu(n, seed=inputs.seed_for(1, 20 + n))
    r.rl_set_param(r.RL_PARAM_GETRF_PANEL, nb)
    try:
        F, ipiv, info = G.getrf(A, lda=n + 1)
    finally:
        r.rl_set_param(r.RL_PARAM_GETRF_PANEL, 32)
    assert info == 0
    assert np.array_equal(ipiv, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L)
    assert np.array_equal(np.triu(F), U)


def _check_lu(A, F, ipiv, info):
    m, n = A.shape
    assert info == 0
    assert oracle.res_lu(A, F, ipiv) <= BOUND
    R, rpiv, rinfo = oracle.getrf(A, c=24)
    assert rinfo == 0
    t = G.first_near_tie(R)
    assert np.array_equal(ipiv[:t], rpiv[:t])
    if t == min(m, n):
        kappa = np.linalg.cond(A) if m == n else np.linalg.cond(A.T @ A) ** 0.5
        assert close(F, R, max(m, n), kappa)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 65, 100, 255, 300, 1000])
def test_getrf_square_vs_oracle(n):
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, n))
    F, ipiv, info = G.getrf(A, lda=n + (n % 5))
    _check_lu(A, F, ipiv, info)


@pytest.mark.parametrize("m,n", [(300, 100), (100, 300), (1000, 37), (37, 1000), (129, 64), (2000, 40)])
def test_getrf_rectangular_vs_oracle(m, n):
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 3 * m + n))
    F, ipiv, info = G.getrf(A)
    assert info == 0
    assert oracle.res_lu(A, F, ipiv) <= BOUND
    R, rpiv, rinfo = oracle.getrf(A, c=24)
    t = G.first_near_tie(R)
    assert np.array_equal(ipiv[:t], rpiv[:t])


@pytest.mark.parametrize("k", [0, 31, 32, 150, 299])
def test_getrf_info_singular(k):
    n = 300
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 88))
    A[:, k] = 0.0
    F, ipiv, info = G.getrf(A)
    R, rpiv, rinfo = oracle.getrf(A, c=24)
    assert info == rinfo == k + 1
    assert oracle.res_lu(A, F, ipiv) <= BOUND


def test_getrf_tall_panel_multi_cta():
    # one panel spread over many CTAs (grid barrier path), ragged last slab
    m, n = 5000, 32
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 99))
    F, ipiv, info = G.getrf(A)
    assert info == 0
    R, rpiv, rinfo = oracle.getrf(A, c=32)
    t = G.first_near_tie(R)
    assert np.array_equal(ipiv[:t], rpiv[:t])
    assert close(F, R, m, np.linalg.cond(A))


# ----------------------------------------------------------------------------
# TRTRI / LAUUM / POTRI
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [5, 64, 65, 150, 300])
def test_trtri_integer_bit_exact(n):
    L = inputs.integer_trtri(n, seed=inputs.seed_for(1, 40 + n))
    X, info = G.trtri(L, lda=n + 2)
    assert info == 0
    assert np.array_equal(np.tril(L) @ np.tril(X), np.eye(n))
    assert np.array_equal(np.triu(X, 1), np.triu(L, 1))


@pytest.mark.parametrize("n", [3, 64, 129, 333])
def test_lauum_integer_bit_exact(n):
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 60 + n))
    P, info = G.lauum(L)
    Li = np.tril(L).astype(np.int64)
    assert info == 0
    assert np.array_equal(np.tril(P), np.tril((Li.T @ Li).astype(np.float64)))
    assert np.array_equal(np.triu(P, 1), np.triu(L, 1))


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 200, 513, 1000])
def test_trtri_lauum_potri_vs_oracle(n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 200 + n))
    L, _ = oracle.potrf(A, c=24)
    L = np.asfortranarray(np.tril(L))
    X, info = G.trtri(L)
    assert info == 0 and oracle.res_trtri(L, X) <= BOUND
    RX, _ = oracle.trtri(L, c=24)
    assert close(np.tril(X), np.tril(RX), n, np.linalg.cond(L))
    P, info = G.lauum(L)
    RP = oracle.lauum(L, c=24)
    assert close(np.tril(P), np.tril(RP), n, 1.0)
    Ai, info = G.potri(L)
    assert info == 0 and oracle.res_potri(A, Ai) <= BOUND


def test_trtri_info_zero_diagonal():
    n = 300
    L = np.tril(inputs.uniform(n, n, seed=inputs.seed_for(1, 55))) + 3 * np.eye(n)
    L = np.asfortranarray(L)
    L[170, 170] = 0.0
    L[250, 250] = 0.0
    X, info = G.trtri(L)
    assert info == 171
    assert np.array_equal(X, L)
    Y, info = G.potri(L)
    assert info == 171 and np.array_equal(Y, L)


# ----------------------------------------------------------------------------
# the first full-size workloads (n = 4096 / 8192)
# ----------------------------------------------------------------------------

def test_config1_getrf_4096_vs_oracle():
    n = 4096
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 0))
    F, ipiv, info = G.getrf(A)
    assert info == 0
    R, rpiv, rinfo = oracle.getrf(A, c=24)
    t = G.first_near_tie(R)
    assert np.array_equal(ipiv[:t], rpiv[:t])
    x = inputs.normal(n, 4, seed=1)
    for j in range(4):
        assert oracle.probe_lu(A, F, ipiv, x[:, j]) <= BOUND
    if t == n:
        assert close(F, R, n, np.linalg.cond(A))


def test_config1_potrf_8192_probe():
    n = 8192
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 1))
    F, info = G.potrf(A)
    assert info == 0
    x = inputs.normal(n, 4, seed=2)
    for j in range(4):
        assert oracle.probe_chol(A, F, x[:, j]) <= BOUND


def test_config1_trtri_lauum_4096_probe():
    n = 4096
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 2))
    L, info = G.potrf(A)
    assert info == 0
    L = np.asfortranarray(np.tril(L))
    X, info = G.trtri(L)
    assert info == 0
    Ai, info = G.potri(L)
    assert info == 0
    x = inputs.normal(n, 3, seed=3)
    for j in range(3):
        assert oracle.probe_trtri(L, X, x[:, j]) <= BOUND
        assert oracle.probe_potri(A, Ai, x[:, j]) <= BOUND


# ----------------------------------------------------------------------------
# C ABI behaviour on the device
# ----------------------------------------------------------------------------

def test_argument_errors_and_quick_returns():
    r = G.lib()
    t = G.torch()
    info = G.int_buf(1, -3)
    buf = t.zeros(16, dtype=t.float64, device="cuda")
    assert r.rl_dpotrf("X", 4, buf.data_ptr(), 4, info.data_ptr()) == -1
    assert r.rl_dpotrf("L", -1, buf.data_ptr(), 4, info.data_ptr()) == -2
    assert r.rl_dpotrf("L", 4, buf.data_ptr(), 3, info.data_ptr()) == -4
    assert r.rl_dgetrf(-1, 4, buf.data_ptr(), 4, info.data_ptr(), info.data_ptr(), None, 0) == -1
    assert r.rl_dgetrf(4, 4, buf.data_ptr(), 2, info.data_ptr(), info.data_ptr(), None, 0) == -4
    assert r.rl_dgetrf(4, 4, buf.data_ptr(), 4, info.data_ptr(), info.data_ptr(), None, 0) == r.RL_ERR_WORKSPACE
    assert r.rl_dtrtri("L", "Q", 4, buf.data_ptr(), 4, info.data_ptr()) == -2
    assert r.rl_dlauum("L", 4, buf.data_ptr(), 1, info.data_ptr()) == -4
    assert r.rl_dpotrf("X", 4, buf.data_ptr(), 4, info.data_ptr()) == -1
    G.sync()
    assert int(info[0].item()) == -3          # never written on argument errors
    # n = 0 quick return writes info = 0
    assert r.rl_dpotrf("L", 0, buf.data_ptr(), 1, info.data_ptr()) == 0
    G.sync()
    assert int(info[0].item()) == 0


def test_host_buffer_forms():
    r = G.lib()
    t = G.torch()
    n = 300
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 5))
    h = t.from_numpy(np.asfortranarray(A).ravel(order="F").copy()).pin_memory()
    hinfo = t.full((1,), -9, dtype=t.int32).pin_memory()
    lw = r.rl_host_work_size("dpotrf", n, n, n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dpotrf_host("L", n, h.data_ptr(), n, hinfo.data_ptr(), work.data_ptr(), lw) == 0
    F = h.numpy().reshape(n, n).T
    assert int(hinfo[0]) == 0 and oracle.res_chol(A, F) <= BOUND
    G_ = inputs.uniform(n, n, seed=inputs.seed_for(1, 5))
    h = t.from_numpy(np.asfortranarray(G_).ravel(order="F").copy()).pin_memory()
    hpiv = t.zeros(n, dtype=t.int32).pin_memory()
    lw = r.rl_host_work_size("dgetrf", n, n, n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dgetrf_host(n, n, h.data_ptr(), n, hpiv.data_ptr(), hinfo.data_ptr(), work.data_ptr(), lw) == 0
    F = h.numpy().reshape(n, n).T
    assert int(hinfo[0]) == 0 and oracle.res_lu(G_, F, hpiv.numpy()) <= BOUND


@pytest.mark.parametrize("m,n", [(1500, 1500), (2000, 1300), (700, 1900)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_split_copies_bit_identical(m, n, pinned):
    """Above order 512 the host-buffer calls copy the columns right of the
    top-level split on a copy stream (and the Cholesky's left columns back
    early): the results equal the device-buffer calls' bit for bit, with
    pinned and pageable host memory, tall and wide, and with a non-SPD
    matrix (info, and the leading block before the failure)."""
    r = G.lib()
    t = G.torch()

    def host(X):
        h = t.from_numpy(np.asfortranarray(X).ravel(order="F").copy())
        return h.pin_memory() if pinned else h

    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 9000 + m + n))
    F_dev, p_dev, i_dev = G.getrf(A)
    h = host(A)
    hpiv = t.zeros(min(m, n), dtype=t.int32)
    hinfo = t.full((1,), -9, dtype=t.int32)
    lw = r.rl_host_work_size("dgetrf", m, n, m)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dgetrf_host(m, n, h.data_ptr(), m, hpiv.data_ptr(), hinfo.data_ptr(), work.data_ptr(), lw) == 0
    assert int(hinfo[0]) == i_dev
    assert np.array_equal(h.numpy().reshape(n, m).T, F_dev)
    assert np.array_equal(hpiv.numpy(), p_dev)
    if m != n:
        return
    for bad in (False, True):
        S = inputs.spd_bbt(n, seed=inputs.seed_for(1, 9100 + n))
        if bad:
            S[1200, 1200] = -1.0
        L_dev, li_dev = G.potrf(S)
        h = host(S)
        lw = r.rl_host_work_size("dpotrf", n, n, n)
        work = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_dpotrf_host("L", n, h.data_ptr(), n, hinfo.data_ptr(), work.data_ptr(), lw) == 0
        assert int(hinfo[0]) == li_dev == (1201 if bad else 0)
        L_host = h.numpy().reshape(n, n).T
        if bad:   # the leading 1200 x 1200 block is final; what follows depends on when kernels saw info
            assert np.array_equal(np.tril(L_host[:1200, :1200]), np.tril(L_dev[:1200, :1200]))
        else:
            assert np.array_equal(L_host, L_dev)


def test_bounded_wait_reports_timeout_and_context_survives():
    # A zero spin limit makes the panel's grid barrier give up at once: the
    # kernel must return with info = RL_INFO_DEVICE_TIMEOUT, not hang, and the
    # context must stay usable.
    r = G.lib()
    m, n = 4000, 32
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 7))
    r.rl_set_param(r.RL_PARAM_SPIN_LIMIT_NS, 0)
    try:
        _, _, info = G.getrf(A)
    finally:
        r.rl_set_param(r.RL_PARAM_SPIN_LIMIT_NS, 2_000_000_000)
    assert info == r.RL_INFO_DEVICE_TIMEOUT
    F, ipiv, info = G.getrf(A)
    assert info == 0 and oracle.res_lu(A, F, ipiv) <= BOUND


def test_launch_counter_advances():
    r = G.lib()
    before = r.rl_launch_count()
    G.potrf(inputs.spd_bbt(300, seed=1))
    assert r.rl_launch_count() > before

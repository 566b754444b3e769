"""The BLAS-3 layer (rl_dgemm / rl_dsyrk / rl_dtrsm / rl_dtrmm) against the
oracle's plain definitions, on ragged shapes that cross the 64-wide tiles and
the 64-order triangle blocks.

Tolerances follow the standard elementwise error bounds of the operations:
  GEMM/SYRK/TRMM: |C_gpu - C_ref| <= 2 k eps (|alpha| |op(A)| |op(B)| + |beta| |C|)
  TRSM:           |op(T) X - alpha B| <= 4 n eps |op(T)| |X|  (backward error)
where k (or n) is the inner dimension and eps = 2^-53.
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


def op(X, t):
    return X.T if t == "T" else X


@pytest.mark.parametrize("ta", ["N", "T"])
@pytest.mark.parametrize("tb", ["N", "T"])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 65, 130), (64, 64, 64), (130, 33, 300), (300, 200, 7), (5, 129, 0)])
def test_dgemm(ta, tb, m, n, k):
    r = G.lib()
    A = inputs.uniform(k if ta == "T" else m, m if ta == "T" else k, seed=m + 7 * n + 13 * k)
    B = inputs.uniform(n if tb == "T" else k, k if tb == "T" else n, seed=m + 3 * n + 11 * k + 1)
    C = inputs.uniform(m, n, seed=2 * m + n + k + 2)
    alpha, beta = -0.75, 1.25
    dA, dB, dC = G.DevMat(A, lda=A.shape[0] + 3), G.DevMat(B), G.DevMat(C, lda=m + 1)
    assert r.rl_dgemm(ta, tb, m, n, k, alpha, dA.ptr(), dA.lda, dB.ptr(), dB.lda, beta, dC.ptr(), dC.lda) == 0
    G.sync()
    assert dA.canaries_intact() and dC.canaries_intact()
    got = dC.get()
    ref = oracle.gemm(A, B, beta * C, alpha=alpha, ta=(ta == "T"), tb=(tb == "T"))
    bound = 2 * max(k, 1) * EPS * (abs(alpha) * np.abs(op(A, ta)) @ np.abs(op(B, tb)) + abs(beta) * np.abs(C)) + 1e-300
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("n,k", [(1, 5), (65, 64), (200, 130), (64, 1)])
def test_dsyrk_lower(trans, n, k):
    r = G.lib()
    A = inputs.uniform(k if trans == "T" else n, n if trans == "T" else k, seed=5 * n + k)
    C = inputs.uniform(n, n, seed=n + 3 * k)
    dA, dC = G.DevMat(A), G.DevMat(C, lda=n + 2)
    assert r.rl_dsyrk("L", trans, n, k, -1.0, dA.ptr(), dA.lda, 1.0, dC.ptr(), dC.lda) == 0
    G.sync()
    assert dC.canaries_intact()
    got = dC.get()
    ref = oracle.syrk_lower(A, C, alpha=-1.0, trans=(trans == "T"))
    oa = op(A, "T" if trans == "T" else "N")
    bound = 2 * k * EPS * (np.abs(oa) @ np.abs(oa).T + np.abs(C)) + 1e-300
    lower = np.tril(np.ones((n, n), dtype=bool))
    assert np.all((np.abs(got - ref) <= bound)[lower])
    assert np.array_equal(np.triu(got, 1), np.triu(C, 1))      # upper triangle untouched


def _tri(n, seed, lower=True, unit=False):
    T = inputs.uniform(n, n, seed=seed)
    T = np.tril(T) if lower else np.triu(T)
    T[np.diag_indices(n)] = 2.0 + np.abs(T[np.diag_indices(n)])
    if unit:
        T[np.diag_indices(n)] = 1.0
    return np.asfortranarray(T)


@pytest.mark.parametrize("case", ["LLNN", "LLNU", "LLTN", "RLTN", "LUNN"])
@pytest.mark.parametrize("m,n", [(1, 1), (16, 33), (64, 64), (65, 130), (200, 17), (33, 200)])
def test_dtrsm(case, m, n):
    r = G.lib()
    side, uplo, tr, diag = case
    nt = m if side == "L" else n
    T = _tri(nt, seed=m * 31 + n, lower=(uplo == "L"), unit=(diag == "U"))
    B = inputs.uniform(m, n, seed=m + n * 17)
    alpha = -1.5
    dT, dB = G.DevMat(T, lda=nt + 1), G.DevMat(B, lda=m + 2)
    assert r.rl_dtrsm(side, uplo, tr, diag, m, n, alpha, dT.ptr(), dT.lda, dB.ptr(), dB.lda) == 0
    G.sync()
    assert dB.canaries_intact() and dT.canaries_intact()
    X = dB.get()
    oT = op(T, tr)
    lhs = oT @ X if side == "L" else X @ oT
    bound = 4 * nt * EPS * (np.abs(oT) @ np.abs(X) if side == "L" else np.abs(X) @ np.abs(oT)) + 1e-300
    assert np.all(np.abs(lhs - alpha * B) <= bound)
    # against the oracle's substitution as well
    if case == "LLNN":
        ref = oracle.trsm_lln(T, B, alpha=alpha)
    elif case == "LLNU":
        ref = oracle.trsm_lln(T, B, alpha=alpha, unit=True)
    elif case == "LLTN":
        ref = alpha * oracle.trsm_llt(T, B)
    elif case == "RLTN":
        ref = alpha * oracle.trsm_rlt(T, B)
    else:
        ref = alpha * oracle.trsm_lun(T, B)
    kappa = np.linalg.cond(T)
    assert np.max(np.abs(X - ref)) <= 8 * nt * EPS * kappa * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("case", ["RLNN", "RLNU", "LLTN"])
@pytest.mark.parametrize("m,n", [(1, 1), (16, 33), (64, 64), (65, 130), (200, 17), (33, 200)])
def test_dtrmm(case, m, n):
    r = G.lib()
    side, uplo, tr, diag = case
    nt = m if side == "L" else n
    T = _tri(nt, seed=m * 7 + n, unit=(diag == "U"))
    B = inputs.uniform(m, n, seed=m + n * 5)
    alpha = 0.5
    dT, dB = G.DevMat(T), G.DevMat(B, lda=m + 1)
    assert r.rl_dtrmm(side, uplo, tr, diag, m, n, alpha, dT.ptr(), dT.lda, dB.ptr(), dB.lda) == 0
    G.sync()
    assert dB.canaries_intact()
    got = dB.get()
    if case == "LLTN":
        ref = alpha * oracle.trmm_llt(T, B)
        mag = np.abs(T.T) @ np.abs(B)
    else:
        ref = alpha * oracle.trmm_rln(T, B)
        mag = np.abs(B) @ np.abs(T)
    assert np.all(np.abs(got - ref) <= 2 * nt * EPS * abs(alpha) * mag + 1e-300)


def test_blas3_unsupported_options():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float64, device="cuda")
    p = buf.data_ptr()
    assert r.rl_dsyrk("U", "N", 4, 4, 1.0, p, 4, 1.0, p, 4) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dtrsm("R", "L", "N", "N", 4, 4, 1.0, p, 4, p, 4) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dtrmm("L", "L", "N", "N", 4, 4, 1.0, p, 4, p, 4) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dgemm("X", "N", 4, 4, 4, 1.0, p, 4, p, 4, 1.0, p, 4) == -1
    assert r.rl_dgemm("N", "N", 4, 4, 4, 1.0, p, 3, p, 4, 1.0, p, 4) == -8
    assert r.rl_dtrsm("L", "L", "N", "N", 4, 4, 1.0, p, 3, p, 4) == -9


# ---- the two triangle-kernel layouts give bit-identical results ---------------

@pytest.fixture
def tri_lanes_reset():
    yield
    G.lib().rl_set_param(G.lib().RL_PARAM_TRI_LANES, 0)


@pytest.mark.parametrize("case,m,n", [("RLTN", 13000, 64), ("RLTN", 300, 40), ("LLNN", 64, 12500),
                                      ("LLNU", 50, 700), ("LLTN", 64, 12400), ("LUNN", 33, 900),
                                      ("RLNN", 12300, 64), ("RLNU", 200, 17), ("LLTM", 64, 12300)])
def test_triangle_kernels_bit_identical(case, m, n, tri_lanes_reset):
    r = G.lib()
    side, uplo, tr, diag = case[0], case[1], case[2], case[3] if case[3] != "M" else "N"
    trmm = case in ("RLNN", "RLNU", "LLTM")
    nt = m if side == "L" else n
    T = _tri(nt, seed=nt * 13 + 5, lower=(uplo == "L"), unit=(diag == "U"))
    B = inputs.uniform(m, n, seed=m * 3 + n)
    outs = []
    for lanes in (4, 2):
        assert r.rl_set_param(r.RL_PARAM_TRI_LANES, lanes) == 0
        dT, dB = G.DevMat(T), G.DevMat(B, lda=m + 1)
        fn = r.rl_dtrmm if trmm else r.rl_dtrsm
        assert fn(side, uplo, tr, diag, m, n, 0.75, dT.ptr(), dT.lda, dB.ptr(), dB.lda) == 0
        G.sync()
        assert dB.canaries_intact()
        outs.append(dB.get())
    assert np.array_equal(outs[0], outs[1])


# ---- FP32 peers of GEMM / SYRK (both SIMT tile shapes) -------------------------

EPS32 = 2.0 ** -24


class DevMat32:
    """FP32 column-major device matrix with a canary tail."""

    def __init__(self, A, lda=None):
        t = G.torch()
        A = np.asarray(A, dtype=np.float32)
        self.m, self.n = A.shape
        self.lda = max(1, self.m) if lda is None else lda
        buf = np.full(self.lda * max(1, self.n) + 64, np.float32(-7.25), dtype=np.float32)
        buf[: self.lda * self.n].reshape(self.n, self.lda)[:, : self.m] = A.T
        self.t = t.from_numpy(buf).cuda()

    def ptr(self):
        return self.t.data_ptr()

    def get(self):
        buf = self.t.cpu().numpy()
        return np.asfortranarray(buf[: self.lda * self.n].reshape(self.n, self.lda)[:, : self.m].T.astype(np.float64))

    def tail_intact(self):
        return bool(np.all(self.t.cpu().numpy()[self.lda * self.n:] == np.float32(-7.25)))


def f32(X):
    return np.asarray(X, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("ta", ["N", "T"])
@pytest.mark.parametrize("tb", ["N", "T"])
@pytest.mark.parametrize("m,n,k", [(130, 33, 300), (1700, 1650, 100), (1601, 1999, 37)])
def test_sgemm(ta, tb, m, n, k):
    r = G.lib()
    A = f32(inputs.uniform(k if ta == "T" else m, m if ta == "T" else k, seed=m + 7 * n + 13 * k))
    B = f32(inputs.uniform(n if tb == "T" else k, k if tb == "T" else n, seed=m + 3 * n + 11 * k + 1))
    C = f32(inputs.uniform(m, n, seed=2 * m + n + k + 2))
    alpha, beta = -0.75, 1.25
    dA, dB, dC = DevMat32(A, lda=A.shape[0] + 3), DevMat32(B), DevMat32(C, lda=m + 1)
    assert r.rl_sgemm(ta, tb, m, n, k, alpha, dA.ptr(), dA.lda, dB.ptr(), dB.lda, beta, dC.ptr(), dC.lda) == 0
    G.sync()
    assert dC.tail_intact()
    got = dC.get()
    ref = oracle.gemm(A, B, beta * C, alpha=alpha, ta=(ta == "T"), tb=(tb == "T"))
    bound = 2 * (k + 2) * EPS32 * (abs(alpha) * np.abs(op(A, ta)) @ np.abs(op(B, tb)) + abs(beta) * np.abs(C)) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("n,k", [(200, 130), (2200, 64)])
def test_ssyrk_lower(trans, n, k):
    r = G.lib()
    A = f32(inputs.uniform(k if trans == "T" else n, n if trans == "T" else k, seed=5 * n + k))
    C = f32(inputs.uniform(n, n, seed=n + 3 * k))
    dA, dC = DevMat32(A), DevMat32(C, lda=n + 2)
    assert r.rl_ssyrk("L", trans, n, k, -1.0, dA.ptr(), dA.lda, 1.0, dC.ptr(), dC.lda) == 0
    G.sync()
    assert dC.tail_intact()
    got = dC.get()
    ref = oracle.syrk_lower(A, C, alpha=-1.0, trans=(trans == "T"))
    oa = op(A, "T" if trans == "T" else "N")
    bound = 2 * (k + 2) * EPS32 * (np.abs(oa) @ np.abs(oa).T + np.abs(C)) + 1e-30
    lower = np.tril(np.ones((n, n), dtype=bool))
    assert np.all((np.abs(got - ref) <= bound)[lower])
    assert np.array_equal(np.triu(got, 1), np.triu(C, 1))


def test_dlaswp_vs_oracle():
    r = G.lib()
    t = G.torch()
    m, ncols, k1, k2 = 5000, 300, 3, 4700
    rng = np.random.default_rng(inputs.seed_for(1, 5000))
    piv = np.array([rng.integers(j + 1, m + 1) for j in range(m)], dtype=np.int32)
    A = inputs.uniform(m, ncols, seed=inputs.seed_for(1, 5001))
    dA = G.DevMat(A, lda=m + 2)
    dp = t.from_numpy(piv).cuda()
    assert r.rl_dlaswp(m, ncols, dA.ptr(), dA.lda, k1, k2, dp) == 0
    G.sync()
    assert dA.canaries_intact()
    ref = oracle.laswp(A, k1 - 1, k2, piv)
    assert np.array_equal(dA.get(), ref)
    assert r.rl_dlaswp(m, ncols, dA.ptr(), dA.lda, 0, k2, dp) == -5

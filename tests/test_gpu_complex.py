"""Complex double peers (rl_zpotrf / rl_zgetrf) against the oracle: residuals
||A - L L^H|| and ||P A - L U|| in units of n eps ||A|| (<= 10), factors that
are exact in binary64 bit for bit (Gaussian-integer Cholesky, dyadic
complex LU with a planted permutation), ipiv equal to the oracle's up to the
first near-tie of the |Re| + |Im| pivot search, info on singular and
indefinite inputs, and canaries around every buffer; the inversions
(ztrtri lower/upper/unit, zlauum, zpotri) bit for bit on Gaussian-integer
triangles whose inverses are Gaussian integers, zgetri by ||A X - I||."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
CANARY = complex(-7.25e300, 3.5e299)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


class ZMat:
    """Column-major complex128 matrix in a canary-padded device buffer."""

    def __init__(self, A, lda=None):
        t = G.torch()
        A = np.asarray(A, dtype=np.complex128)
        self.m, self.n = A.shape
        self.lda = max(1, self.m) if lda is None else lda
        buf = np.full(self.lda * max(1, self.n) + G.TAIL, CANARY, dtype=np.complex128)
        v = buf[: self.lda * self.n].reshape(self.n, self.lda)
        v[:, : self.m] = A.T
        self.t = t.from_numpy(buf).cuda()

    def ptr(self):
        return self.t.data_ptr()

    def get(self):
        buf = self.t.cpu().numpy()
        v = buf[: self.lda * self.n].reshape(self.n, self.lda)
        return np.asfortranarray(v[:, : self.m].T)

    def canaries_intact(self):
        buf = self.t.cpu().numpy()
        v = buf[: self.lda * self.n].reshape(self.n, self.lda)
        pad_ok = np.all(v[:, self.m:] == CANARY) if self.lda > self.m else True
        return bool(pad_ok and np.all(buf[self.lda * self.n:] == CANARY))


def zpotrf(A, lda=None):
    r = G.lib()
    d = ZMat(A, lda)
    info = G.int_buf(1, -77)
    st = r.rl_zpotrf("L", d.n, d.ptr(), d.lda, info.data_ptr())
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0].item())


def zgetrf(A, lda=None):
    r = G.lib()
    t = G.torch()
    d = ZMat(A, lda)
    mn = min(d.m, d.n)
    ipiv = G.int_buf(mn, -5)
    info = G.int_buf(1, -77)
    lw = r.rl_dgetrf_work_size(d.m, d.n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_zgetrf(d.m, d.n, d.ptr(), d.lda, ipiv.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    iv = ipiv.cpu().numpy()
    assert np.all(iv[max(1, mn):] == -5)
    return d.get(), iv[:mn].copy(), int(info[0].item())


def abs1(z):
    return np.abs(z.real) + np.abs(z.imag)


def first_near_tie(LU, rel=1e-12):
    """First step j whose pivot choice was a near-tie: the candidates there
    were l_ij u_jj (i > j) against the chosen u_jj, compared by |Re| + |Im|."""
    m, n = LU.shape
    mn = min(m, n)
    for j in range(mn):
        if j + 1 < m:
            best = abs1(LU[j, j])
            if np.max(abs1(LU[j + 1:, j] * LU[j, j])) > (1.0 - rel) * best:
                return j
    return mn


@pytest.mark.parametrize("n", [1, 2, 33, 64, 65, 200, 700, 1100])
def test_zpotrf_vs_oracle(n):
    A = inputs.herm_spd(n, inputs.seed_for(1, 5000 + n))
    L, info = zpotrf(A)
    assert info == 0
    assert oracle.res_zchol(A, np.tril(L)) <= 10.0
    # the strictly upper triangle is not touched
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))
    ref, oinfo = oracle.zpotrf(A)
    assert oinfo == 0
    scale = np.max(np.abs(np.tril(ref)))
    assert np.max(np.abs(np.tril(L) - np.tril(ref))) <= 64 * n * 2.0 ** -53 * scale


@pytest.mark.parametrize("n", [5, 130, 300, 600])
def test_zpotrf_gaussian_integers_exact(n):
    Lx = inputs.gaussian_int_chol(n, inputs.seed_for(1, 5100 + n))
    A = np.asfortranarray(Lx @ Lx.conj().T)
    L, info = zpotrf(A, lda=n + 3)
    assert info == 0
    assert np.array_equal(np.tril(L), Lx)


def test_zpotrf_not_definite_info():
    n = 300
    A = inputs.herm_spd(n, inputs.seed_for(1, 5200))
    A[170, 170] = -1e6
    _, info = zpotrf(A)
    _, oinfo = oracle.zpotrf(A)
    assert info == oinfo == 171


@pytest.mark.parametrize("m,n", [(1, 1), (31, 31), (33, 33), (200, 200), (700, 700), (1100, 1100),
                                 (500, 130), (130, 500), (1000, 37)])
def test_zgetrf_vs_oracle(m, n):
    A = inputs.complex_uniform(m, n, inputs.seed_for(1, 5300 + m + 7 * n))
    F, ipiv, info = zgetrf(A)
    assert info == 0
    ref, opiv, oinfo = oracle.zgetrf(A)
    assert oinfo == 0
    assert oracle.res_zlu(A, F, ipiv) <= 10.0
    t = min(first_near_tie(F), first_near_tie(ref))
    assert np.array_equal(ipiv[:t], opiv[:t])
    if t == min(m, n):
        kappa = np.linalg.cond(A) if m == n else 1e3
        assert np.max(np.abs(F - ref)) <= 64 * max(m, n) * 2.0 ** -53 * kappa * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [6, 150, 300, 520])
def test_zgetrf_dyadic_exact(n):
    A, L, U, perm = inputs.complex_dyadic_lu(n, inputs.seed_for(1, 5400 + n))
    F, ipiv, info = zgetrf(A, lda=n + 1)
    assert info == 0
    assert np.array_equal(ipiv, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L)
    assert np.array_equal(np.triu(F), U)


def test_zgetrf_singular_info():
    n = 200
    A = inputs.complex_uniform(n, n, inputs.seed_for(1, 5500))
    A[:, 77] = 0.0
    F, ipiv, info = zgetrf(A)
    _, opiv, oinfo = oracle.zgetrf(A)
    assert info == oinfo == 78
    assert np.all(np.isfinite(F.real)) and np.all(np.isfinite(F.imag))


def test_complex_argument_errors():
    r = G.lib()
    info = G.int_buf(1, -77)
    assert r.rl_zpotrf("X", 4, 0, 4, info.data_ptr()) == -1
    assert r.rl_zpotrf("L", -1, 0, 4, info.data_ptr()) == -2
    assert r.rl_zpotrf("L", 4, 0, 4, info.data_ptr()) == -3
    d = ZMat(np.eye(4))
    assert r.rl_zpotrf("L", 4, d.ptr(), 3, info.data_ptr()) == -4
    ipiv = G.int_buf(4)
    assert r.rl_zgetrf(4, 4, d.ptr(), 4, ipiv.data_ptr(), info.data_ptr(), 0, 0) == r.RL_ERR_WORKSPACE
    assert r.rl_zgetrf(-1, 4, d.ptr(), 4, ipiv.data_ptr(), info.data_ptr(), 0, 0) == -1
    assert r.rl_zpotrf("L", 0, 0, 1, info.data_ptr()) == 0


# ----------------------------------------------------------------------------
# inversions: ztrtri, zlauum, zpotri, zgetri
# ----------------------------------------------------------------------------

def zcall(fn, *args):
    st = fn(*args)
    G.sync()
    assert st == 0, G.lib().rl_status_string(st)


@pytest.mark.parametrize("n", [1, 31, 33, 130, 300])
def test_ztrtri_exact(n):
    r = G.lib()
    L, Linv = inputs.gaussian_unit_trtri(n, inputs.seed_for(1, 5600 + n))
    info = G.int_buf(1, -77)
    d = ZMat(L, lda=n + 1)
    zcall(r.rl_ztrtri, "L", "N", n, d.ptr(), d.lda, info.data_ptr())
    assert int(info[0]) == 0 and d.canaries_intact()
    assert np.array_equal(np.tril(d.get()), Linv)
    # unit diagonal: L's off-diagonal part with ones on the diagonal
    Lu = np.tril(np.diag(1.0 / np.diag(L)) @ L)
    Lu_inv = np.asfortranarray(np.tril(Linv @ np.diag(np.diag(L))))
    d = ZMat(Lu)
    zcall(r.rl_ztrtri, "L", "U", n, d.ptr(), d.lda, info.data_ptr())
    assert np.array_equal(np.tril(d.get(), -1), np.tril(Lu_inv, -1))
    # upper: U = L^H, U^{-1} = (L^{-1})^H
    U = np.asfortranarray(L.conj().T)
    d = ZMat(U)
    zcall(r.rl_ztrtri, "U", "N", n, d.ptr(), d.lda, info.data_ptr())
    assert np.array_equal(np.triu(d.get()), np.triu(Linv.conj().T))


def test_ztrtri_zero_diagonal_info():
    r = G.lib()
    n = 200
    L, _ = inputs.gaussian_unit_trtri(n, inputs.seed_for(1, 5700))
    L[120, 120] = 0.0
    d = ZMat(L)
    info = G.int_buf(1, -77)
    zcall(r.rl_ztrtri, "L", "N", n, d.ptr(), d.lda, info.data_ptr())
    assert int(info[0]) == 121
    assert np.array_equal(d.get(), L)


@pytest.mark.parametrize("n", [7, 64, 250])
def test_zlauum_zpotri_exact(n):
    r = G.lib()
    L, Linv = inputs.gaussian_unit_trtri(n, inputs.seed_for(1, 5800 + n))
    info = G.int_buf(1, -77)
    d = ZMat(L)
    zcall(r.rl_zlauum, "L", n, d.ptr(), d.lda, info.data_ptr())
    assert np.array_equal(np.tril(d.get()), np.tril(L.conj().T @ L))
    d = ZMat(np.asfortranarray(L.conj().T))
    zcall(r.rl_zlauum, "U", n, d.ptr(), d.lda, info.data_ptr())
    assert np.array_equal(np.triu(d.get()), np.triu(L.conj().T @ L))
    # zpotri on the factor L of A = L L^H: A^{-1} = L^{-H} L^{-1}
    d = ZMat(L)
    zcall(r.rl_zpotri, "L", n, d.ptr(), d.lda, info.data_ptr())
    assert int(info[0]) == 0
    assert np.array_equal(np.tril(d.get()), np.tril(Linv.conj().T @ Linv))


@pytest.mark.parametrize("n", [1, 40, 300, 700])
def test_zgetri(n):
    r = G.lib()
    t = G.torch()
    A = inputs.complex_uniform(n, n, inputs.seed_for(1, 5900 + n))
    F, ipiv, info = zgetrf(A)
    assert info == 0
    d = ZMat(F)
    dp = t.from_numpy(ipiv.astype(np.int32)).cuda()
    inf = G.int_buf(1, -77)
    lw = r.rl_zgetri_work_size(n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    zcall(r.rl_zgetri, n, d.ptr(), d.lda, dp.data_ptr(), inf.data_ptr(), w.data_ptr(), lw)
    assert int(inf[0]) == 0 and d.canaries_intact()
    X = d.get()
    Al, Xl = A.astype(np.clongdouble), X.astype(np.clongdouble)
    R = (Al @ Xl - np.eye(n)).astype(np.complex128)
    # ||A X - I|| / (||A|| ||X|| n eps), 1-norms
    res = np.abs(R).sum(0).max() / (np.abs(A).sum(0).max() * np.abs(X).sum(0).max() * n * 2.0 ** -53)
    assert res <= 10.0


@pytest.mark.parametrize("n", [65, 300])
def test_complex_inversions_vs_oracle(n):
    """Random well-conditioned inputs against the oracle's definitions (the
    tolerances the oracle itself meets against LAPACK)."""
    r = G.lib()
    t = G.torch()
    tol = 64 * n * 2.0 ** -53
    H = inputs.herm_spd(n, inputs.seed_for(1, 6000 + n))
    L = np.asfortranarray(np.tril(oracle.zpotrf(H)[0]))
    info = G.int_buf(1, -77)
    for fn, ref in ((lambda d: r.rl_ztrtri("L", "N", n, d.ptr(), n, info.data_ptr()), oracle.ztrtri(L)[0]),
                    (lambda d: r.rl_zlauum("L", n, d.ptr(), n, info.data_ptr()), oracle.zlauum(L)),
                    (lambda d: r.rl_zpotri("L", n, d.ptr(), n, info.data_ptr()), oracle.zpotri(L)[0])):
        d = ZMat(L)
        zcall(fn, d)
        assert int(info[0]) == 0
        assert np.max(np.abs(np.tril(d.get()) - np.tril(ref))) <= tol * 8 * np.max(np.abs(ref))
    A = inputs.complex_uniform(n, n, inputs.seed_for(1, 6100 + n))
    F, ipiv, _ = zgetrf(A)
    d = ZMat(F)
    dp = t.from_numpy(ipiv.astype(np.int32)).cuda()
    lw = r.rl_zgetri_work_size(n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    zcall(r.rl_zgetri, n, d.ptr(), n, dp.data_ptr(), info.data_ptr(), w.data_ptr(), lw)
    ref = oracle.zgetri(F, ipiv)
    assert np.max(np.abs(d.get() - ref)) <= tol * 8 * np.linalg.cond(A) * np.max(np.abs(ref))

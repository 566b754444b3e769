"""uplo = 'U' through the C ABI: every upper routine against the oracle on
the transposed storage (the identity pinned against LAPACK's upper routines
in the oracle tests), exact inputs bit for bit, the strictly lower triangle
(filled with a marker pattern) unchanged, inputs that are transposed in
place for the call (sygst's B, potrs' A) restored bit for bit, and LAPACK's
info on indefinite and singular inputs."""
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


def marked_upper(U, seed):
    """U's upper triangle with a random marker pattern below the diagonal."""
    r = np.random.default_rng(seed)
    n = U.shape[0]
    return np.asfortranarray(np.triu(U) + np.tril(r.uniform(-9, 9, (n, n)), -1))


def tT(X):
    return np.asfortranarray(X.T)


def call(fn, *args):
    st = fn(*args)
    G.sync()
    assert st == 0, G.lib().rl_status_string(st)


@pytest.mark.parametrize("n", [1, 2, 65, 300, 1000])
def test_dpotrf_upper(n):
    r = G.lib()
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6000 + n))
    A0 = marked_upper(A, 6001 + n)
    d = G.DevMat(A0, lda=n + 2)
    info = G.int_buf(1, -77)
    call(r.rl_dpotrf, "U", n, d.ptr(), d.lda, info.data_ptr())
    assert int(info[0]) == 0 and d.canaries_intact()
    X = d.get()
    assert np.array_equal(np.tril(X, -1), np.tril(A0, -1))
    U = np.triu(X)
    assert oracle.res_chol(A, tT(U)) <= 10.0
    L, _ = oracle.potrf(tT(A))
    ref = np.triu(np.tril(L).T)
    assert np.max(np.abs(U - ref)) <= 64 * n * EPS * np.max(np.abs(ref))


def test_dpotrf_upper_exact_and_info():
    r = G.lib()
    n = 260
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 6100))
    A = inputs.product_lower(L)
    X, info = None, None
    d = G.DevMat(marked_upper(A, 6101))
    inf = G.int_buf(1, -77)
    call(r.rl_dpotrf, "U", n, d.ptr(), n, inf.data_ptr())
    assert int(inf[0]) == 0
    assert np.array_equal(np.triu(d.get()), np.triu(L.T))
    B = A.copy(order="F")
    B[150, 150] = -1.0
    d = G.DevMat(marked_upper(B, 6102))
    call(r.rl_dpotrf, "U", n, d.ptr(), n, inf.data_ptr())
    assert int(inf[0]) == 151
    X = d.get()
    # the leading 150 x 150 block of U is complete, as LAPACK leaves it
    assert np.array_equal(np.triu(X)[:150, :150], np.triu(L.T)[:150, :150])


def test_spotrf_zpotrf_upper():
    r = G.lib()
    t = G.torch()
    n = 400
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6200)).astype(np.float32).astype(np.float64)
    dA = t.from_numpy(np.asfortranarray(marked_upper(A, 6201), dtype=np.float32).ravel(order="F").copy()).cuda()
    info = G.int_buf(1, -77)
    call(r.rl_spotrf, "U", n, dA.data_ptr(), n, info.data_ptr())
    assert int(info[0]) == 0
    U = np.triu(dA.cpu().numpy().reshape(n, n).T.astype(np.float64))
    assert oracle.res_chol(A, tT(U)) * 2.0 ** -53 / 2.0 ** -24 <= 10.0
    # complex: A = U^H U, U = L^H; Gaussian-integer factors are exact
    Lz = inputs.gaussian_int_chol(n, inputs.seed_for(1, 6210))
    H = np.asfortranarray(Lz @ Lz.conj().T)
    M = np.triu(H) + np.tril(np.full((n, n), 3.0 - 5.0j), -1)
    dz = t.from_numpy(np.asfortranarray(M).ravel(order="F").copy()).cuda()
    call(r.rl_zpotrf, "U", n, dz.data_ptr(), n, info.data_ptr())
    assert int(info[0]) == 0
    X = dz.cpu().numpy().reshape(n, n).T
    assert np.array_equal(np.triu(X), np.triu(Lz.conj().T))
    assert np.array_equal(np.tril(X, -1), np.tril(M, -1))
    Hr = inputs.herm_spd(300, inputs.seed_for(1, 6220))
    dz = t.from_numpy(np.asfortranarray(Hr).ravel(order="F").copy()).cuda()
    call(r.rl_zpotrf, "U", 300, dz.data_ptr(), 300, info.data_ptr())
    U = np.triu(dz.cpu().numpy().reshape(300, 300).T)
    assert oracle.res_zchol(Hr, np.asfortranarray(U.conj().T)) <= 10.0


@pytest.mark.parametrize("n", [1, 70, 333])
@pytest.mark.parametrize("unit", [False, True])
def test_dtrtri_upper(n, unit):
    r = G.lib()
    L = inputs.integer_trtri(n, seed=inputs.seed_for(1, 6300 + n))
    U0 = marked_upper(L.T, 6301 + n)
    if unit:
        U0[np.diag_indices(n)] = 5.0          # not referenced
    d = G.DevMat(U0)
    info = G.int_buf(1, -77)
    call(r.rl_dtrtri, "U", "U" if unit else "N", n, d.ptr(), n, info.data_ptr())
    assert int(info[0]) == 0
    X = d.get()
    assert np.array_equal(np.tril(X, -1), np.tril(U0, -1))
    Lu = np.tril(L, -1) + np.eye(n) if unit else L
    ref, _ = oracle.trtri(np.asfortranarray(Lu), unit=unit)
    k = 1 if unit else 0
    assert np.array_equal(np.triu(X, k), np.triu(np.tril(ref).T, k))     # exact dyadic inverse


def test_dlauum_dpotri_upper():
    r = G.lib()
    n = 500
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6400))
    Lf, _ = oracle.potrf(A)
    U = np.triu(np.tril(Lf).T)
    U0 = marked_upper(U, 6401)
    info = G.int_buf(1, -77)
    d = G.DevMat(U0)
    call(r.rl_dlauum, "U", n, d.ptr(), n, info.data_ptr())
    X = d.get()
    assert np.array_equal(np.tril(X, -1), np.tril(U0, -1))
    ref = oracle.lauum(np.asfortranarray(np.tril(U.T)))
    ref = np.triu(np.tril(ref).T)
    assert np.max(np.abs(np.triu(X) - ref)) <= 64 * n * EPS * np.max(np.abs(ref))
    d = G.DevMat(U0)
    call(r.rl_dpotri, "U", n, d.ptr(), n, info.data_ptr())
    assert int(info[0]) == 0
    X = d.get()
    assert np.array_equal(np.tril(X, -1), np.tril(U0, -1))
    ref, _ = oracle.potri(np.asfortranarray(np.tril(U.T)))
    ref = np.triu(np.tril(ref).T)
    assert np.max(np.abs(np.triu(X) - ref)) <= 64 * n * EPS * np.linalg.cond(A) * np.max(np.abs(ref))
    # a zero on U's diagonal: info, A unchanged
    Z = U0.copy(order="F")
    Z[77, 77] = 0.0
    d = G.DevMat(Z)
    call(r.rl_dpotri, "U", n, d.ptr(), n, info.data_ptr())
    assert int(info[0]) == 78
    assert np.array_equal(d.get(), Z)


@pytest.mark.parametrize("itype", [1, 2])
def test_dsygst_upper(itype):
    r = G.lib()
    t = G.torch()
    n = 420
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6500))
    Lf, _ = oracle.potrf(Bm)
    U = np.triu(np.tril(Lf).T)
    M = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6501))
    A0 = marked_upper(M, 6502)
    B0 = marked_upper(U, 6503)
    dA, dB = G.DevMat(A0), G.DevMat(B0)
    lw = r.rl_dsygst_work_size(n)
    w = t.zeros(lw, dtype=t.uint8, device="cuda")
    call(r.rl_dsygst, itype, "U", n, dA.ptr(), n, dB.ptr(), n, w, lw)
    assert np.array_equal(dB.get(), B0)                    # B restored bit for bit
    X = dA.get()
    assert np.array_equal(np.tril(X, -1), np.tril(A0, -1))
    ref = oracle.sygst(itype, tT(M), np.asfortranarray(np.tril(U.T)))
    ref = np.triu(np.tril(ref).T)
    assert np.max(np.abs(np.triu(X) - ref)) <= 64 * n * EPS * np.max(np.abs(ref)) * (8 if itype == 1 else 1)


@pytest.mark.parametrize("use_work", [False, True])
def test_dpotrs_upper(use_work):
    r = G.lib()
    t = G.torch()
    n, nrhs = 700, 5
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6600))
    Lf, _ = oracle.potrf(A)
    U0 = marked_upper(np.tril(Lf).T, 6601)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(1, 6602))
    dA, dB = G.DevMat(U0), G.DevMat(B)
    lw = r.rl_trs_work_size(n, nrhs) if use_work else 0
    w = t.zeros(max(lw, 1), dtype=t.uint8, device="cuda") if use_work else None
    call(r.rl_dpotrs, "U", n, nrhs, dA.ptr(), n, dB.ptr(), n, w, lw)
    assert np.array_equal(dA.get(), U0)                    # A restored bit for bit
    X = dB.get()
    res = np.linalg.norm(A @ X - B, 1) / (np.linalg.norm(A, 1) * np.linalg.norm(X, 1) * n * EPS)
    assert res <= 10.0


def test_dsposv_upper():
    r = G.lib()
    t = G.torch()
    n, nrhs = 1000, 2
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6700))
    A0 = marked_upper(A, 6701)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(1, 6702))
    dA, dB, dX = G.DevMat(A0), G.DevMat(B), G.DevMat(np.zeros((n, nrhs)))
    lw = r.rl_dsposv_work_size(n, nrhs, r.RL_PREC_FP32)
    w = t.zeros(lw, dtype=t.uint8, device="cuda")
    it, info = G.int_buf(1, -9), G.int_buf(1, -77)
    call(r.rl_dsposv, "U", n, nrhs, dA.ptr(), n, dB.ptr(), n, dX.ptr(), n, r.RL_PREC_FP32, 0.0, 30,
         it.data_ptr(), info.data_ptr(), w, lw)
    assert int(info[0]) == 0 and int(it[0]) > 0
    assert np.array_equal(dA.get(), A0)                    # refinement converged: A untouched
    X = dX.get()
    ref = np.linalg.solve(A, B)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_batched_dpotrf_upper():
    r = G.lib()
    t = G.torch()
    sizes = [1, 8, 31, 32, 33, 100, 255, 256, 17, 64]
    mats, ptrs, bufs = [], [], []
    for k, n in enumerate(sizes):
        A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6800 + k))
        A0 = marked_upper(A, 6900 + k)
        b = t.from_numpy(A0.ravel(order="F").copy()).cuda()
        mats.append((A, A0))
        bufs.append(b)
        ptrs.append(b.data_ptr())
    nb = len(sizes)
    dn = t.tensor(sizes, dtype=t.int32, device="cuda")
    dld = t.tensor(sizes, dtype=t.int32, device="cuda")
    dp = t.tensor(ptrs, dtype=t.int64, device="cuda")
    info = t.full((nb,), -5, dtype=t.int32, device="cuda")
    lw = r.rl_potrf_vbatched_work_size(nb)
    w = t.zeros(lw, dtype=t.uint8, device="cuda")
    call(r.rl_dpotrf_vbatched, "U", nb, dn.data_ptr(), dp.data_ptr(), dld.data_ptr(), info.data_ptr(),
         max(sizes), w, lw)
    assert np.all(info.cpu().numpy() == 0)
    for (A, A0), b, n in zip(mats, bufs, sizes):
        X = b.cpu().numpy().reshape(n, n).T
        assert np.array_equal(np.tril(X, -1), np.tril(A0, -1))
        assert oracle.res_chol(A, tT(np.triu(X))) <= 10.0


@pytest.mark.parametrize("prec", ["FP32", "BF16"])
def test_dsposv_lower_ignores_the_upper_triangle(prec):
    """LAPACK's dsposv references only the uplo triangle: a marker pattern in
    the other one changes neither the solution nor the iteration count."""
    r = G.lib()
    t = G.torch()
    n, nrhs = 900, 3
    p = getattr(r, "RL_PREC_" + prec)
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 6750))
    rng = np.random.default_rng(6751)
    Am = np.asfortranarray(np.tril(A) + np.triu(rng.uniform(-1e30, 1e30, (n, n)), 1))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(1, 6752))
    out = []
    for M in (A, Am):
        dA, dB, dX = G.DevMat(M), G.DevMat(B), G.DevMat(np.zeros((n, nrhs)))
        lw = r.rl_dsposv_work_size(n, nrhs, p)
        w = t.zeros(lw, dtype=t.uint8, device="cuda")
        it, info = G.int_buf(1, -9), G.int_buf(1, -77)
        call(r.rl_dsposv, "L", n, nrhs, dA.ptr(), n, dB.ptr(), n, dX.ptr(), n, p, 0.0, 30,
             it.data_ptr(), info.data_ptr(), w, lw)
        assert int(info[0]) == 0 and int(it[0]) > 0
        assert np.array_equal(dA.get(), M)
        out.append((dX.get(), int(it[0])))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])

"""Batching form (rl_[ds]potrf_vbatched, rl_[ds]getrf_vbatched) against the
oracle, matrix by matrix.

FP64: the pass bound (residual / (n eps ||A||) <= 10, eps = 2^-53) and
ipiv equal to the oracle's up to the first near-tie; integer / dyadic
matrices bit-exact.  FP32: the same residual measured in units of the FP32
rounding unit 2^-24 on the FP32-rounded input.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


class Batch:
    """Matrices packed in one device buffer, each 256-byte aligned, with
    device arrays of orders, pointers, leading dimensions and pivots."""

    def __init__(self, mats, dtype, pad=0):
        t = G.torch()
        self.dtype = dtype
        self.esz = 8 if dtype == t.float64 else 4
        self.sizes = [m.shape[0] for m in mats]
        self.ldas = [max(1, n + pad) for n in self.sizes]
        align = 256 // self.esz
        offs, off = [], 0
        for n, ld in zip(self.sizes, self.ldas):
            offs.append(off)
            off += ((ld * max(n, 1) + align - 1) // align) * align
        self.offs = offs
        host = np.full(off + align, -3.5, dtype=np.float64 if self.esz == 8 else np.float32)
        for m, o, ld in zip(mats, offs, self.ldas):
            n = m.shape[0]
            if n:
                v = host[o:o + ld * n].reshape(n, ld)
                v[:, :n] = m.T
        self.buf = t.from_numpy(host).cuda()
        base = self.buf.data_ptr()
        self.ptrs = t.tensor([base + o * self.esz for o in offs], dtype=t.int64, device="cuda")
        self.n = t.tensor(self.sizes, dtype=t.int32, device="cuda")
        self.lda = t.tensor(self.ldas, dtype=t.int32, device="cuda")
        self.info = t.full((len(mats),), -77, dtype=t.int32, device="cuda")
        self.piv_store = t.full((max(1, sum(self.sizes)),), -5, dtype=t.int32, device="cuda")
        pofs, p = [], 0
        for n in self.sizes:
            pofs.append(p)
            p += n
        self.pofs = pofs
        self.ipiv = t.tensor([self.piv_store.data_ptr() + 4 * q for q in pofs], dtype=t.int64, device="cuda")

    def get(self, b):
        host = self.buf.cpu().numpy()
        n, ld, o = self.sizes[b], self.ldas[b], self.offs[b]
        return np.asfortranarray(host[o:o + ld * n].reshape(n, ld)[:, :n].T.astype(np.float64))

    def piv(self, b):
        p = self.piv_store.cpu().numpy()
        return p[self.pofs[b]:self.pofs[b] + self.sizes[b]]


def run(kind, batch, max_n=256):
    r = G.lib()
    t = G.torch()
    lw = r.rl_potrf_vbatched_work_size(len(batch.sizes))
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    f64 = batch.esz == 8
    if kind == "potrf":
        fn = r.rl_dpotrf_vbatched if f64 else r.rl_spotrf_vbatched
        st = fn("L", len(batch.sizes), batch.n, batch.ptrs, batch.lda, batch.info, max_n, work, lw)
    else:
        fn = r.rl_dgetrf_vbatched if f64 else r.rl_sgetrf_vbatched
        st = fn(len(batch.sizes), batch.n, batch.ptrs, batch.lda, batch.ipiv, batch.info, max_n, work, lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    return batch.info.cpu().numpy()


SIZES = [1, 2, 7, 8, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256]


def sizes_mix(count, seed):
    return list(SIZES) + list(inputs.bucket_sizes(count, 8, 256, seed))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_potrf_vbatched_vs_oracle(prec):
    t = G.torch()
    sizes = sizes_mix(60, seed=inputs.seed_for(3, 1))
    mats = [inputs.spd_bbt(n, seed=inputs.seed_for(3, 100 + i)) for i, n in enumerate(sizes)]
    if prec == "f32":
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
    B = Batch(mats, t.float64 if prec == "f64" else t.float32, pad=3)
    info = run("potrf", B)
    assert np.all(info == 0)
    scale = 1.0 if prec == "f64" else EPS64 / EPS32
    for b, (A, n) in enumerate(zip(mats, sizes)):
        L = B.get(b)
        assert oracle.res_chol(A, L) * scale <= 10.0, (b, n)
        assert np.array_equal(np.triu(L, 1), np.triu(A, 1).astype(L.dtype))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_getrf_vbatched_vs_oracle(prec):
    t = G.torch()
    sizes = sizes_mix(60, seed=inputs.seed_for(3, 2))
    mats = [inputs.uniform(n, n, seed=inputs.seed_for(3, 300 + i)) for i, n in enumerate(sizes)]
    if prec == "f32":
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
    B = Batch(mats, t.float64 if prec == "f64" else t.float32)
    info = run("getrf", B)
    assert np.all(info == 0)
    scale = 1.0 if prec == "f64" else EPS64 / EPS32
    for b, (A, n) in enumerate(zip(mats, sizes)):
        F, piv = B.get(b), B.piv(b)
        assert oracle.res_lu(A, F, piv) * scale <= 10.0, (b, n)
        if prec == "f64":
            R, rpiv, _ = oracle.getrf(A, c=24)
            tie = G.first_near_tie(R)
            assert np.array_equal(piv[:tie], rpiv[:tie]), (b, n)


def test_vbatched_exact_inputs_bit_exact():
    t = G.torch()
    Ls = [inputs.integer_chol(n, seed=inputs.seed_for(3, 500 + n)) for n in (6, 40, 97, 256)]
    As = [inputs.product_lower(L) for L in Ls]
    B = Batch(As, t.float64)
    assert np.all(run("potrf", B) == 0)
    for b, L in enumerate(Ls):
        assert np.array_equal(np.tril(B.get(b)), L)
    cases = [inputs.dyadic_lu(n, seed=inputs.seed_for(3, 600 + n)) for n in (5, 33, 130, 256)]
    B = Batch([c[0] for c in cases], t.float64)
    assert np.all(run("getrf", B) == 0)
    for b, (A, L, U, perm) in enumerate(cases):
        F = B.get(b)
        n = A.shape[0]
        assert np.array_equal(B.piv(b), inputs.expected_ipiv(perm))
        assert np.array_equal(np.tril(F, -1) + np.eye(n), L) and np.array_equal(np.triu(F), U)


def test_vbatched_info_per_matrix():
    t = G.torch()
    mats = [inputs.spd_bbt(n, seed=inputs.seed_for(3, 700 + n)) for n in (50, 120, 200)]
    mats[1][70, 70] = -1.0
    B = Batch(mats, t.float64)
    info = run("potrf", B)
    assert list(info) == [0, 71, 0]
    gm = [inputs.uniform(n, n, seed=inputs.seed_for(3, 800 + n)) for n in (40, 90, 150)]
    gm[2][:, 33] = 0.0
    B = Batch(gm, t.float64)
    info = run("getrf", B)
    assert list(info) == [0, 0, 34]
    F, piv = B.get(2), B.piv(2)
    assert oracle.res_lu(gm[2], F, piv) <= 10.0


def test_vbatched_argument_checks():
    r = G.lib()
    t = G.torch()
    p = t.zeros(8, dtype=t.int64, device="cuda")
    w = t.zeros(1024, dtype=t.uint8, device="cuda")
    assert r.rl_dpotrf_vbatched("X", 1, p, p, p, p, 8, w, 1024) == -1
    assert r.rl_dpotrf_vbatched("L", -1, p, p, p, p, 8, w, 1024) == -2
    assert r.rl_dpotrf_vbatched("L", 1, p, p, p, p, 300, w, 1024) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dgetrf_vbatched(2, p, p, p, p, p, 8, w, 4) == r.RL_ERR_WORKSPACE
    assert r.rl_dgetrf_vbatched(0, p, p, p, p, p, 8, w, 1024) == 0


# ---- the autotuner and every configuration it chooses from -------------------

@pytest.fixture
def batch_cfg_reset():
    yield
    r = G.lib()
    for k in "PG":
        for eb in (4, 8):
            r.rl_vbatched_set_config(k, eb, 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_every_batched_config_vs_oracle(prec, batch_cfg_reset):
    r = G.lib()
    t = G.torch()
    sizes = [1, 15, 16, 17, 31, 33, 64, 100, 129, 200, 256]
    eb = 8 if prec == "f64" else 4
    dt = t.float64 if prec == "f64" else t.float32
    scale = 1.0 if prec == "f64" else EPS64 / EPS32
    S = [inputs.spd_bbt(n, seed=inputs.seed_for(3, 700 + i)) for i, n in enumerate(sizes)]
    U_ = [inputs.uniform(n, n, seed=inputs.seed_for(3, 800 + i)) for i, n in enumerate(sizes)]
    if prec == "f32":
        S = [m.astype(np.float32).astype(np.float64) for m in S]
        U_ = [m.astype(np.float32).astype(np.float64) for m in U_]
    for cfg in range(r.RL_BATCH_CONFIGS):
        assert r.rl_vbatched_set_config("P", eb, cfg) == 0 and r.rl_vbatched_set_config("G", eb, cfg) == 0
        B = Batch(S, dt, pad=1)
        info = run("potrf", B)
        assert np.all(info == 0)
        for b, A in enumerate(S):
            assert oracle.res_chol(A, B.get(b)) * scale <= 10.0, (cfg, b)
        B = Batch(U_, dt)
        info = run("getrf", B)
        assert np.all(info == 0)
        for b, A in enumerate(U_):
            assert oracle.res_lu(A, B.get(b), B.piv(b)) * scale <= 10.0, (cfg, b)


def test_autotuner_restores_the_batch_and_picks_a_config(batch_cfg_reset):
    r = G.lib()
    t = G.torch()
    sizes = list(inputs.bucket_sizes(300, 8, 256, inputs.seed_for(3, 900)))
    mats = [inputs.uniform(n, n, seed=inputs.seed_for(3, 1000 + i)) for i, n in enumerate(sizes)]
    B = Batch(mats, t.float64)
    before = B.buf.clone()
    lw = r.rl_vbatched_tune_work_size(len(sizes), int(sum(n * n for n in sizes)), 8)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    st, best, ms = r.rl_vbatched_tune("G", 8, len(sizes), B.n, B.ptrs, B.lda, B.ipiv, B.info, 256, w, lw)
    assert st == 0, r.rl_status_string(st)
    assert 0 <= best < r.RL_BATCH_CONFIGS and all(m > 0 for m in ms)
    assert ms[best] == min(ms)
    assert r.rl_vbatched_config("G", 8)[0] == best
    assert t.equal(B.buf, before)                    # the caller's matrices are back
    info = run("getrf", B)
    assert np.all(info == 0)
    for b, A in enumerate(mats):
        assert oracle.res_lu(A, B.get(b), B.piv(b)) <= 10.0
    assert r.rl_vbatched_tune("G", 8, len(sizes), B.n, B.ptrs, B.lda, B.ipiv, B.info, 256, w, lw - 1)[0] \
        == r.RL_ERR_WORKSPACE


@pytest.mark.parametrize("kind", ["potrf", "getrf"])
def test_out_of_range_orders_report_argument_errors(kind):
    """A matrix whose order is negative or above 256, or whose leading
    dimension is below its order, gets LAPACK's argument error in its info
    entry (-3 / -5 for potrf's order and lda arrays, -2 / -4 for getrf's) and
    is not touched; the rest of the batch is factored as usual."""
    t = G.torch()
    sizes = [40, 12, 60, 33]
    mats = [inputs.spd_bbt(n, seed=inputs.seed_for(3, 1500 + i)) if kind == "potrf"
            else inputs.uniform(n, n, seed=inputs.seed_for(3, 1600 + i)) for i, n in enumerate(sizes)]
    B = Batch(mats, t.float64)
    before = B.buf.cpu().numpy().copy()
    # matrix 1: order 300 (> 256); matrix 3: order -1; matrix 2: lda 59 < 60
    B.n[1] = 300
    B.n[3] = -1
    B.lda[2] = 59
    info = run(kind, B)
    e_n, e_lda = (-3, -5) if kind == "potrf" else (-2, -4)
    assert info.tolist() == [0, e_n, e_lda, e_n]
    after = B.buf.cpu().numpy()
    for b in (1, 2, 3):
        o, n = B.offs[b], sizes[b]
        assert np.array_equal(after[o:o + n * n], before[o:o + n * n]), b
    F = B.get(0)
    if kind == "potrf":
        assert oracle.res_chol(mats[0], F) <= 10.0
    else:
        assert oracle.res_lu(mats[0], F, B.piv(0)) <= 10.0

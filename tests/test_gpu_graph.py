"""Calls captured into a CUDA graph and replayed give the eager call's bits.

The recursion schedules its kernels on the host (Section 3, Fig. 4: split,
recurse on the first half, update, recurse on the second half); a graph
captured from one call must replay exactly that schedule.  At orders of 1024
and more the LU and Cholesky recursions also put part of each large trailing
update on the library's internal stream, joined by events, so the capture
spans two streams.  Each replay runs on inputs restored from a pristine copy
and must equal the eager result bit for bit (factors, ipiv, info), twice in a
row, and meet the oracle's residual bound.
"""
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
    assert r.rl_get_param(r.RL_PARAM_LOOKAHEAD) == 1
    yield


def _capture(call):
    """Capture call(stream_handle) into a graph on a side stream (after one
    eager call, which does the library's one-time set-up)."""
    t = G.torch()
    g = t.cuda.CUDAGraph()
    cs = t.cuda.Stream()
    t.cuda.synchronize()
    with t.cuda.stream(cs):
        with t.cuda.graph(g, stream=cs):
            call(cs.cuda_stream)
    t.cuda.synchronize()
    return g


def _replays(g, restore, read, times=2):
    out = []
    for _ in range(times):
        restore()
        G.sync()
        g.replay()
        G.sync()
        out.append(read())
    return out


@pytest.mark.parametrize("n", [1024, 2050])
def test_dpotrf_graph_replay_bit_identical(n):
    r, t = G.lib(), G.torch()
    A0 = inputs.spd_bbt(n, seed=inputs.seed_for(1, 3100 + n))
    src = t.from_numpy(A0.ravel(order="F").copy()).cuda()
    A = src.clone()
    info = t.full((1,), -77, dtype=t.int32, device="cuda")

    def call(s):
        r.check(r.rl_dpotrf("L", n, A, n, info, None, 0, s), "rl_dpotrf")

    call(0)
    G.sync()
    eager = (A.cpu().numpy().copy(), int(info.item()))
    A.copy_(src)
    info.fill_(-77)
    g = _capture(call)
    # the capture itself ran nothing
    assert np.array_equal(A.cpu().numpy(), src.cpu().numpy()) and int(info.item()) == -77

    def restore():
        A.copy_(src)
        info.fill_(-77)

    got = _replays(g, restore, lambda: (A.cpu().numpy().copy(), int(info.item())))
    for Fa, inf in got:
        assert inf == eager[1] == 0
        assert np.array_equal(Fa, eager[0])
    L = np.tril(got[-1][0].reshape(n, n).T)
    assert oracle.res_chol(A0, L) <= 10.0


@pytest.mark.parametrize("m,n", [(1024, 1024), (2100, 1800)])
def test_dgetrf_graph_replay_bit_identical(m, n):
    r, t = G.lib(), G.torch()
    A0 = inputs.uniform(m, n, seed=inputs.seed_for(1, 3200 + n))
    src = t.from_numpy(A0.ravel(order="F").copy()).cuda()
    A = src.clone()
    mn = min(m, n)
    ipiv = t.full((mn,), -5, dtype=t.int32, device="cuda")
    info = t.full((1,), -77, dtype=t.int32, device="cuda")
    lw = r.rl_dgetrf_work_size(m, n)
    wk = t.empty(lw, dtype=t.uint8, device="cuda")

    def call(s):
        r.check(r.rl_dgetrf(m, n, A, m, ipiv, info, wk, lw, s), "rl_dgetrf")

    def read():
        return A.cpu().numpy().copy(), ipiv.cpu().numpy().copy(), int(info.item())

    call(0)
    G.sync()
    eager = read()

    def restore():
        A.copy_(src)
        ipiv.fill_(-5)
        info.fill_(-77)

    restore()
    g = _capture(call)
    got = _replays(g, restore, read)
    for Fa, p, inf in got:
        assert inf == eager[2] == 0
        assert np.array_equal(p, eager[1])
        assert np.array_equal(Fa, eager[0])
    F = np.asfortranarray(got[-1][0].reshape(n, m).T)
    assert oracle.res_lu(A0, F, got[-1][1]) <= 10.0


def test_dgetrf_graph_replay_singular_info():
    """A singular column: info is written by the replayed kernels too."""
    r, t = G.lib(), G.torch()
    n = 1100
    A0 = inputs.uniform(n, n, seed=inputs.seed_for(1, 3300))
    A0[:, 700] = 0.0
    src = t.from_numpy(A0.ravel(order="F").copy()).cuda()
    A = src.clone()
    ipiv = t.zeros(n, dtype=t.int32, device="cuda")
    info = t.full((1,), -77, dtype=t.int32, device="cuda")
    lw = r.rl_dgetrf_work_size(n, n)
    wk = t.empty(lw, dtype=t.uint8, device="cuda")

    def call(s):
        r.check(r.rl_dgetrf(n, n, A, n, ipiv, info, wk, lw, s), "rl_dgetrf")

    call(0)
    G.sync()
    eager = (A.cpu().numpy().copy(), int(info.item()))
    assert eager[1] == 701

    def restore():
        A.copy_(src)
        info.fill_(-77)

    restore()
    g = _capture(call)
    for Fa, inf in _replays(g, restore, lambda: (A.cpu().numpy().copy(), int(info.item()))):
        assert inf == 701 and np.array_equal(Fa, eager[0])


@pytest.mark.parametrize("kind", ["potrf", "getrf"])
def test_vbatched_graph_replay_bit_identical(kind):
    r, t = G.lib(), G.torch()
    sizes = [1, 8, 31, 64, 65, 129, 256] + list(inputs.bucket_sizes(200, 8, 256, inputs.seed_for(3, 3400)))
    if kind == "potrf":
        mats = [inputs.spd_bbt(n, seed=inputs.seed_for(3, 3500 + i)) for i, n in enumerate(sizes)]
    else:
        mats = [inputs.uniform(n, n, seed=inputs.seed_for(3, 3600 + i)) for i, n in enumerate(sizes)]
    offs, off = [], 0
    for n in sizes:
        offs.append(off)
        off += ((n * n + 31) // 32) * 32
    host = np.zeros(off + 32)
    for M, o in zip(mats, offs):
        host[o:o + M.size] = M.ravel(order="F")
    src = t.from_numpy(host).cuda()
    buf = src.clone()
    batch = len(sizes)
    ptrs = t.tensor([buf.data_ptr() + 8 * o for o in offs], dtype=t.int64, device="cuda")
    nd = t.tensor(sizes, dtype=t.int32, device="cuda")
    lda = t.tensor(sizes, dtype=t.int32, device="cuda")
    info = t.full((batch,), -77, dtype=t.int32, device="cuda")
    piv = t.full((sum(sizes),), -5, dtype=t.int32, device="cuda")
    pofs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    ipiv = t.tensor([piv.data_ptr() + 4 * int(q) for q in pofs], dtype=t.int64, device="cuda")
    lw = r.rl_getrf_vbatched_work_size(batch) if kind == "getrf" else r.rl_potrf_vbatched_work_size(batch)
    wk = t.empty(lw, dtype=t.uint8, device="cuda")

    def call(s):
        if kind == "potrf":
            r.check(r.rl_dpotrf_vbatched("L", batch, nd, ptrs, lda, info, 256, wk, lw, s), "potrf_vbatched")
        else:
            r.check(r.rl_dgetrf_vbatched(batch, nd, ptrs, lda, ipiv, info, 256, wk, lw, s), "getrf_vbatched")

    def read():
        return buf.cpu().numpy().copy(), piv.cpu().numpy().copy(), info.cpu().numpy().copy()

    def restore():
        buf.copy_(src)
        piv.fill_(-5)
        info.fill_(-77)

    call(0)
    G.sync()
    eager = read()
    assert np.all(eager[2] == 0)
    restore()
    g = _capture(call)
    for hb, p, inf in _replays(g, restore, read):
        assert np.array_equal(inf, eager[2])
        assert np.array_equal(hb, eager[0])
        if kind == "getrf":
            assert np.array_equal(p, eager[1])
    hb = eager[0]
    for b in (0, 3, 6, batch - 1):
        n, o = sizes[b], offs[b]
        F = np.asfortranarray(hb[o:o + n * n].reshape(n, n).T)
        if kind == "potrf":
            assert oracle.res_chol(mats[b], np.tril(F)) <= 10.0
        else:
            assert oracle.res_lu(mats[b], F, eager[1][pofs[b]:pofs[b] + n]) <= 10.0

"""rl_dgetrf_vbatched_noalloc (library-owned static scratch, nothing
allocated) against rl_dgetrf_vbatched with a caller workspace: the same
factors (bit for bit), pivots and info on two calls in a row, and the
oracle's residual bound on each.  Collected last on purpose: it must pass after the other GPU
tests as well as alone in a fresh process."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
EDGE = [1, 2, 8, 31, 32, 33, 64, 65, 128, 129, 255, 256]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


class Packed:
    """One copy of the batch: matrices packed 256-byte aligned in one device
    buffer, with device arrays of orders, pointers, leading dimensions,
    pivot pointers and info."""

    def __init__(self, mats):
        t = G.torch()
        self.sizes = [m.shape[0] for m in mats]
        offs, off = [], 0
        for n in self.sizes:
            offs.append(off)
            off += ((n * n + 31) // 32) * 32
        self.offs = offs
        host = np.zeros(off + 32)
        for m, o in zip(mats, offs):
            host[o:o + m.size] = np.asfortranarray(m).ravel(order="F")
        self.buf = t.from_numpy(host).cuda()
        base = self.buf.data_ptr()
        self.ptrs = t.tensor([base + 8 * o for o in offs], dtype=t.int64, device="cuda")
        self.n = t.tensor(self.sizes, dtype=t.int32, device="cuda")
        self.lda = t.tensor([max(1, n) for n in self.sizes], dtype=t.int32, device="cuda")
        self.info = t.full((len(mats),), -77, dtype=t.int32, device="cuda")
        self.piv = t.full((sum(self.sizes),), -5, dtype=t.int32, device="cuda")
        pofs = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.pofs = pofs
        self.ipiv = t.tensor([self.piv.data_ptr() + 4 * int(q) for q in pofs], dtype=t.int64, device="cuda")

    def factors(self, b):
        n, o = self.sizes[b], self.offs[b]
        return self.buf[o:o + n * n].cpu().numpy().reshape(n, n).T.copy()

    def pivots(self, b):
        return self.piv[int(self.pofs[b]):int(self.pofs[b]) + self.sizes[b]].cpu().numpy()


def test_noalloc_matches_workspace_form_twice():
    r = G.lib()
    t = G.torch()
    sizes = EDGE + list(inputs.bucket_sizes(120, 8, 256, inputs.seed_for(3, 900)))
    mats = [inputs.uniform(n, n, seed=inputs.seed_for(3, 1000 + i)) for i, n in enumerate(sizes)]
    batch = len(mats)

    ref = Packed(mats)
    lw = r.rl_getrf_vbatched_work_size(batch)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dgetrf_vbatched(batch, ref.n, ref.ptrs, ref.lda, ref.ipiv, ref.info, 256, work, lw) == 0
    G.sync()
    ref_info = ref.info.cpu().numpy()

    for call in range(2):                       # two calls in a row share the static scratch
        got = Packed(mats)
        st = r.rl_dgetrf_vbatched_noalloc(batch, got.n, got.ptrs, got.lda, got.ipiv, got.info, 256)
        assert st == 0, r.rl_status_string(st)
        G.sync()
        assert np.array_equal(got.info.cpu().numpy(), ref_info)
        for b, (A, n) in enumerate(zip(mats, sizes)):
            F, Fr = got.factors(b), ref.factors(b)
            p = got.pivots(b)
            assert np.array_equal(p, ref.pivots(b)), (call, b, n)
            # same kernel, same configuration, same inputs: bit for bit
            assert np.array_equal(F, Fr), (call, b, n)
            assert oracle.res_lu(A, F, p) <= 10.0, (call, b, n)


def test_noalloc_rejects_batch_beyond_limit():
    r = G.lib()
    dummy = G.torch().zeros(8, dtype=G.torch().int64, device="cuda")
    st = r.rl_dgetrf_vbatched_noalloc(65537, dummy, dummy, dummy, dummy, dummy, 256)
    assert st == r.RL_ERR_UNSUPPORTED
    assert r.rl_dgetrf_vbatched_noalloc(-1, dummy, dummy, dummy, dummy, dummy, 256) == -1

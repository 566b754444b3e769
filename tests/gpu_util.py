"""Helpers for the GPU tests: move column-major matrices to canary-padded
device buffers, call the C ABI through the binding, and read results back.

Every device buffer has a leading dimension >= m (the rows between m and lda
and a tail after the last column hold a canary value) so that out-of-bounds
writes are caught after each call.
"""
import numpy as np

CANARY = -7.25e300
TAIL = 64


def torch():
    import torch as _t
    return _t


def lib():
    from paper_1602_06763_gb300 import relgpu
    return relgpu


class DevMat:
    def __init__(self, A, lda=None):
        t = torch()
        A = np.asarray(A, dtype=np.float64)
        if A.ndim == 1:
            A = A.reshape(-1, 1)
        self.m, self.n = A.shape
        self.lda = max(1, self.m) if lda is None else lda
        buf = np.full(self.lda * max(1, self.n) + TAIL, CANARY)
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


def int_buf(n, fill=0):
    t = torch()
    return t.full((max(1, n) + TAIL,), fill, dtype=t.int32, device="cuda")


def sync():
    torch().cuda.synchronize()


def potrf(A, lda=None):
    r = lib()
    d = DevMat(A, lda)
    info = int_buf(1, -77)
    st = r.rl_dpotrf("L", d.n, d.ptr(), d.lda, info.data_ptr())
    sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0].item())


def getrf(A, lda=None):
    r = lib()
    t = torch()
    d = DevMat(A, lda)
    mn = min(d.m, d.n)
    ipiv = int_buf(mn, -5)
    info = int_buf(1, -77)
    lw = r.rl_dgetrf_work_size(d.m, d.n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dgetrf(d.m, d.n, d.ptr(), d.lda, ipiv.data_ptr(), info.data_ptr(), work.data_ptr(), lw)
    sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    iv = ipiv.cpu().numpy()
    assert np.all(iv[max(1, mn):] == -5)
    return d.get(), iv[:mn].copy(), int(info[0].item())


def trtri(L, unit=False, lda=None):
    r = lib()
    d = DevMat(L, lda)
    info = int_buf(1, -77)
    st = r.rl_dtrtri("L", "U" if unit else "N", d.n, d.ptr(), d.lda, info.data_ptr())
    sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0].item())


def lauum(L, lda=None):
    r = lib()
    d = DevMat(L, lda)
    info = int_buf(1, -77)
    st = r.rl_dlauum("L", d.n, d.ptr(), d.lda, info.data_ptr())
    sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0].item())


def potri(L, lda=None):
    r = lib()
    d = DevMat(L, lda)
    info = int_buf(1, -77)
    st = r.rl_dpotri("L", d.n, d.ptr(), d.lda, info.data_ptr())
    sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0].item())


def first_near_tie(LU, rel=1e-12):
    """First column j whose pivot decision was a near-tie: the candidates at
    step j are |l_ij u_jj| (i > j) against |u_jj|, so a relative gap below
    `rel` means max_{i>j} |l_ij| > 1 - rel.  Returns min(m,n) if none."""
    m, n = LU.shape
    mn = min(m, n)
    for j in range(mn):
        if j + 1 < m and np.max(np.abs(LU[j + 1:, j])) > 1.0 - rel:
            return j
    return mn

"""Seeded synthetic inputs shared by the tests, the oracle checks and the
benchmark.

This module holds none of the factorizations' arithmetic: it only draws random
numbers and assembles test matrices from them.  Both the CUDA path and the CPU
oracle are fed from here, so a parity comparison always sees the same bytes.

The paper measures synthetic matrices only (Section 6: n from 24 to 6168 in
steps of 128, random operands), so no dataset is replaced by these recipes.

Random numbers come from numpy's Philox counter-based generator, whose stream
is fixed by the seed on every platform.  Seeds follow 20260000 + 100*config + k.
All matrices are float64 numpy arrays in Fortran (column-major) order.
"""
from __future__ import annotations

import numpy as np


def seed_for(config: int, k: int = 0) -> int:
    return 20260000 + 100 * int(config) + int(k)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _fortran(a):
    return np.asfortranarray(a, dtype=np.float64)


def spd_bbt(n: int, seed: int, shift=None):
    """A = B B^T + n I with B iid N(0,1) (n x n).  B B^T's lower triangle is
    mirrored so A is exactly symmetric; its condition number is below ~5."""
    B = rng(seed).standard_normal((n, n))
    G = B @ B.T
    A = np.tril(G) + np.tril(G, -1).T
    A[np.diag_indices(n)] += float(n if shift is None else shift)
    return _fortran(A)


def uniform(m: int, n: int, seed: int, lo=-1.0, hi=1.0):
    """Entries iid Uniform(lo, hi)."""
    return _fortran(rng(seed).uniform(lo, hi, size=(m, n)))


def normal(m: int, n: int, seed: int):
    return _fortran(rng(seed).standard_normal((m, n)))


def integer_chol_6():
    """A 6x6 integer lower factor with positive diagonal (our own example).
    A = L L^T is exact in binary64 and every step of a Cholesky factorization
    of A is exact, so the factor must come back bit for bit."""
    L = np.array([[2, 0, 0, 0, 0, 0],
                  [1, 3, 0, 0, 0, 0],
                  [-2, 1, 1, 0, 0, 0],
                  [0, 2, -1, 2, 0, 0],
                  [3, -1, 2, 1, 1, 0],
                  [1, 0, -3, 2, -1, 4]], dtype=np.float64)
    return _fortran(L)


def integer_chol(n: int, seed: int, offdiag=2, diag=(1, 4)):
    """Random integer lower factor L: off-diagonal entries uniform in
    [-offdiag, offdiag], diagonal in [diag[0], diag[1]].  A = L L^T is
    integer-exact and so is every intermediate value of its Cholesky
    factorization (all below 2^53 for the sizes used)."""
    r = rng(seed)
    L = np.tril(r.integers(-offdiag, offdiag + 1, size=(n, n)).astype(np.float64), -1)
    L[np.diag_indices(n)] = r.integers(diag[0], diag[1] + 1, size=n).astype(np.float64)
    return _fortran(L)


def product_lower(L):
    """A = L L^T for an integer L, mirrored to be exactly symmetric."""
    G = L @ L.T
    return _fortran(np.tril(G) + np.tril(G, -1).T)


def dyadic_lu(n: int, seed: int):
    """A = P^T L U built so that partial pivoting reproduces P, L and U exactly.

    L is unit lower with off-diagonal entries in {0, +-1/4, +-1/2, +-3/4}, so at
    every elimination step the row carrying L's unit diagonal is the unique
    largest candidate; U is upper with integer entries in [-4, 4] and a
    diagonal in {+-1, ..., +-4}.  All values are dyadic rationals of small
    magnitude, so every operation of an LU factorization is exact.
    Returns (A, L, U, perm) with A[perm[i], :] = (L U)[i, :]."""
    r = rng(seed)
    L = np.tril(r.integers(-3, 4, size=(n, n)).astype(np.float64) / 4.0, -1)
    L[np.diag_indices(n)] = 1.0
    U = np.triu(r.integers(-4, 5, size=(n, n)).astype(np.float64), 1)
    d = r.integers(1, 5, size=n).astype(np.float64) * r.choice([-1.0, 1.0], size=n)
    U[np.diag_indices(n)] = d
    perm = r.permutation(n)
    LU = L @ U
    A = np.empty_like(LU)
    A[perm, :] = LU
    return _fortran(A), _fortran(L), _fortran(U), perm


def expected_ipiv(perm):
    """The LAPACK swap sequence (1-based) whose application to the rows of A
    brings row perm[i] to position i, i = 0..n-1, in order (bookkeeping only)."""
    n = len(perm)
    pos = list(range(n))          # pos[r] = current position of original row r
    at = list(range(n))           # at[p] = original row currently at position p
    ipiv = np.zeros(n, dtype=np.int32)
    for i in range(n):
        p = pos[perm[i]]
        ipiv[i] = p + 1
        ri, rp = at[i], at[p]
        at[i], at[p] = rp, ri
        pos[rp], pos[ri] = i, p
    return ipiv


def herm_spd(n: int, seed: int):
    """Complex A = B B^H + n I with Re B, Im B iid N(0,1), mirrored so that A
    is exactly Hermitian (real diagonal).  Complex128, column-major."""
    r = rng(seed)
    B = r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))
    G = B @ B.conj().T
    A = np.tril(G, -1) + np.tril(G, -1).conj().T + np.diag(G.diagonal().real + n)
    return np.asfortranarray(A, dtype=np.complex128)


def complex_uniform(m: int, n: int, seed: int):
    """Re and Im iid Uniform(-1, 1).  Complex128, column-major."""
    r = rng(seed)
    return np.asfortranarray(r.uniform(-1, 1, (m, n)) + 1j * r.uniform(-1, 1, (m, n)))


def gaussian_int_chol(n: int, seed: int):
    """Unit lower L with Gaussian-integer off-diagonal entries a + bi,
    a, b in {-1, 0, 1}.  A = L L^H then has Gaussian-integer entries and its
    Cholesky factor is L exactly (every square root is sqrt(1))."""
    r = rng(seed)
    L = np.tril(r.integers(-1, 2, size=(n, n)) + 1j * r.integers(-1, 2, size=(n, n)), -1) + np.eye(n)
    return np.asfortranarray(L, dtype=np.complex128)


def gaussian_unit_trtri(n: int, seed: int, factors=3):
    """A lower triangular L = D (I + N_1)(I + N_2)... with N_k a block below
    the diagonal (rows >= s_k, columns < s_k) of Gaussian integers a + bi,
    a, b in {-1, 0, 1} (so N_k^2 = 0), and D = diag of units {1, -1, i, -i}.
    Returns (L, L^{-1}) with L^{-1} = ... (I - N_2)(I - N_1) D^{-1}, both
    exact Gaussian-integer matrices in complex128."""
    r = rng(seed)
    L = np.eye(n, dtype=np.complex128)
    Linv = np.eye(n, dtype=np.complex128)
    for _ in range(factors):
        sk = int(r.integers(1, max(2, n)))
        N = np.zeros((n, n), dtype=np.complex128)
        N[sk:, :sk] = r.integers(-1, 2, size=(n - sk, sk)) + 1j * r.integers(-1, 2, size=(n - sk, sk))
        L = L @ (np.eye(n) + N)
        Linv = (np.eye(n) - N) @ Linv
    d = r.choice(np.array([1, -1, 1j, -1j]), size=n)
    L = np.diag(d) @ L
    Linv = Linv @ np.diag(1.0 / d)
    return np.asfortranarray(np.tril(L)), np.asfortranarray(np.tril(Linv))


def complex_dyadic_lu(n: int, seed: int):
    """A = P^T L U with L unit lower, off-diagonal (a + bi)/4 (a, b in -1..1,
    so |Re| + |Im| <= 1/2) and U upper with Gaussian-integer entries and a
    diagonal in {+-1, +-2, +-i, +-2i}: partial pivoting on |Re| + |Im|
    reproduces P, and every operation (divisions by U's diagonal included)
    is exact.  Returns (A, L, U, perm) with A[perm[i], :] = (L U)[i, :]."""
    r = rng(seed)
    L = np.tril((r.integers(-1, 2, size=(n, n)) + 1j * r.integers(-1, 2, size=(n, n))) / 4.0, -1) + np.eye(n)
    U = np.triu(r.integers(-3, 4, size=(n, n)) + 1j * r.integers(-3, 4, size=(n, n)), 1).astype(complex)
    U[np.diag_indices(n)] = r.choice(np.array([1, -1, 2, -2, 1j, -1j, 2j, -2j]), size=n)
    perm = r.permutation(n)
    A = np.empty((n, n), dtype=complex)
    A[perm, :] = L @ U
    return np.asfortranarray(A), L, U, perm


def integer_trtri(n: int, seed: int, factors=3):
    """A lower triangular L whose inverse is exact in binary64:
    L = D (I + N_1) (I + N_2) ... with N_k = a block below the diagonal (rows
    >= s_k, columns < s_k, entries in {-1, 0, 1}) so N_k^2 = 0 and
    (I + N_k)^{-1} = I - N_k, and D = diag(+-1, +-2).  L^{-1} has dyadic
    entries of moderate size."""
    r = rng(seed)
    L = np.eye(n)
    for _ in range(factors):
        s = int(r.integers(1, max(2, n)))
        N = np.zeros((n, n))
        N[s:, :s] = r.integers(-1, 2, size=(n - s, s))
        L = L @ (np.eye(n) + N)
    d = r.choice([1.0, 2.0], size=n) * r.choice([-1.0, 1.0], size=n)
    L = np.diag(d) @ L
    return _fortran(np.tril(L))


def householder_product_apply(A, k: int, seed: int, side: str):
    """Apply k random Householder reflectors H_i = I - 2 v_i v_i^T / v_i^T v_i
    (v_i iid N(0,1), drawn in order from `seed`) to A: side='L' gives
    Q A with Q = H_k ... H_1, side='R' gives A Q^T = A H_1 ... H_k for the
    same seed.  Used to build matrices with a prescribed singular spectrum."""
    r = rng(seed)
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0] if side == "L" else A.shape[1]
    for _ in range(k):
        v = r.standard_normal(n)
        beta = 2.0 / float(v @ v)
        if side == "L":
            w = v @ A                        # w = v^T A
            A -= beta * np.outer(v, w)
        else:
            w = A @ v                        # A v
            A -= beta * np.outer(w, v)
    return A


def sigma_logspace(n: int, cond: float):
    """sigma_i = cond^(i/(n-1)), i = 0..n-1 (log-spaced from 1 to cond)."""
    if n == 1:
        return np.ones(1)
    return cond ** (np.arange(n) / (n - 1))


def spd_spectrum(n: int, cond: float, seed: int, reflectors=64):
    """SPD A = Q diag(sigma) Q^T, Q a product of `reflectors` random
    Householder reflectors, sigma log-spaced from 1 to cond."""
    D = np.diag(sigma_logspace(n, cond))
    QD = householder_product_apply(D, reflectors, seed, "L")        # Q D
    A = householder_product_apply(QD, reflectors, seed, "R")        # Q D Q^T
    A = np.tril(A) + np.tril(A, -1).T
    return _fortran(A)


def general_spectrum(n: int, cond: float, seed: int, reflectors=64):
    """General A = U diag(sigma) V^T, U and V products of random Householder
    reflectors (independent seeds), sigma log-spaced from 1 to cond."""
    D = np.diag(sigma_logspace(n, cond))
    UD = householder_product_apply(D, reflectors, seed, "L")
    return _fortran(householder_product_apply(UD, reflectors, seed + 1, "R"))


def spd_bbt_device(n: int, seed: int, device="cuda"):
    """Large-n form of spd_bbt generated on the GPU with torch (input
    generation only): B iid N(0,1) from torch's seeded Philox generator, the
    product B B^T formed in FP32 (the FP32 rounding of B B^T is far below the
    n I shift, so A stays SPD with condition number below ~5), widened to
    FP64, the lower triangle mirrored for exact symmetry, plus n I.
    Returns a torch float64 tensor holding A in column-major order (A is
    symmetric, so the row-major buffer is the same matrix)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    B = torch.randn(n, n, generator=g, device=device, dtype=torch.float32)
    G = torch.matmul(B, B.T).double()
    del B
    A = torch.tril(G)
    A = A + torch.tril(G, -1).T
    del G
    A.diagonal().add_(float(n))
    return A.contiguous()


def uniform_device(m: int, n: int, seed: int, device="cuda"):
    """Entries iid Uniform(-1, 1) drawn on the GPU (torch Philox), returned as
    a float64 tensor of n*m elements holding an m x n column-major matrix."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return (torch.rand(n, m, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0).contiguous()


def spectrum_device(n: int, cond: float, seed: int, spd: bool, reflectors=64, device="cuda"):
    """Large-n form of spd_spectrum / general_spectrum generated on the GPU
    with torch in FP64 (input generation only): diag(sigma), sigma
    log-spaced 1..cond, multiplied from the left by `reflectors` random
    Householder reflectors and from the right by the same (SPD) or an
    independent set (general).  Returns an n x n float64 tensor read as a
    column-major matrix."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    den = max(n - 1, 1)
    sig = torch.pow(torch.tensor(float(cond), dtype=torch.float64, device=device),
                    torch.arange(n, device=device, dtype=torch.float64) / den)
    A = torch.diag(sig)
    VL = torch.randn(reflectors, n, generator=g, device=device, dtype=torch.float64)
    VR = VL if spd else torch.randn(reflectors, n, generator=g, device=device, dtype=torch.float64)
    for i in range(reflectors):
        v = VL[i]
        w = v @ A                                    # v^T A
        A.addr_(v, w, alpha=-2.0 / float(v @ v))     # (I - 2 v v^T / v^T v) A
    for i in range(reflectors):
        v = VR[i]
        w = A @ v                                    # A v
        A.addr_(w, v, alpha=-2.0 / float(v @ v))     # A (I - 2 v v^T / v^T v)
    if spd:
        L = torch.tril(A)
        A = L + torch.tril(A, -1).T
    return A.contiguous()


def bucket_sizes(count: int, lo: int, hi: int, seed: int):
    """Matrix orders drawn uniformly from lo..hi inclusive (batched form)."""
    return rng(seed).integers(lo, hi + 1, size=count).astype(np.int64)

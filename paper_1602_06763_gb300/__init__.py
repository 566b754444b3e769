"""GB300-native recursive dense factorizations (Peise & Bientinesi, "Recursive
Algorithms for Dense Linear Algebra: The ReLAPACK Collection", arXiv
1602.06763): recursive Cholesky (dpotrf), LU with partial pivoting (dgetrf),
triangular inverse (dtrtri) and the product L^T L (dlauum), on one GPU.

The compute path is the C-ABI library ``librelgpu.so`` (declared in
``include/relgpu.h``, built from ``csrc/`` by ``_build.py``).  The Python
binding in ``relgpu.py`` only marshals arguments; it is loaded on first use so
that ``inputs`` (the seeded generators) can be imported without a GPU.
"""

__all__ = ["relgpu", "inputs"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

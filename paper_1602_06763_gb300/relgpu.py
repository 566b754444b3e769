"""Thin ctypes binding of librelgpu.so (the C ABI declared in include/relgpu.h).

Argument marshalling only: every function forwards to the C entry point of
the same name.  Buffers may be given as integers (raw device or host
addresses) or as torch tensors (their ``data_ptr()``); streams as integers,
``torch.cuda.Stream`` objects or None (the current torch stream).  The library
must have been built (``_build.build()``); if it is missing, importing this
module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librelgpu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with paper_1602_06763_gb300._build.build() "
        "(the factorizations run only in the CUDA library; there is no fallback)")

_lib = ctypes.CDLL(LIB_PATH)

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_ch = ctypes.c_char

_SIGS = {
    "rl_dpotrf": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_dgetrf": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_dgetrf_work_size": (_sz, [_i64, _i64]),
    "rl_dtrtri": (ctypes.c_int, [_ch, _ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_dlauum": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_dpotri": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_strtri": (ctypes.c_int, [_ch, _ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_slauum": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_spotri": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_host_work_size": (_sz, [ctypes.c_char_p, _i64, _i64, _i64]),
    "rl_dpotrf_host": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_dgetrf_host": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_set_param": (ctypes.c_int, [ctypes.c_int, _i64]),
    "rl_get_param": (_i64, [ctypes.c_int]),
    "rl_launch_count": (ctypes.c_uint64, []),
    "rl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rl_dgemm": (ctypes.c_int, [_ch, _ch, _i64, _i64, _i64, ctypes.c_double, _vp, _i64, _vp, _i64,
                                ctypes.c_double, _vp, _i64, _vp]),
    "rl_dsyrk": (ctypes.c_int, [_ch, _ch, _i64, _i64, ctypes.c_double, _vp, _i64, ctypes.c_double,
                                _vp, _i64, _vp]),
    "rl_sgemm": (ctypes.c_int, [_ch, _ch, _i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp, _i64,
                                ctypes.c_float, _vp, _i64, _vp]),
    "rl_ssyrk": (ctypes.c_int, [_ch, _ch, _i64, _i64, ctypes.c_float, _vp, _i64, ctypes.c_float,
                                _vp, _i64, _vp]),
    "rl_dtrsm": (ctypes.c_int, [_ch, _ch, _ch, _ch, _i64, _i64, ctypes.c_double, _vp, _i64, _vp,
                                _i64, _vp]),
    "rl_dtrmm": (ctypes.c_int, [_ch, _ch, _ch, _ch, _i64, _i64, ctypes.c_double, _vp, _i64, _vp,
                                _i64, _vp]),
    "rl_trs_work_size": (ctypes.c_size_t, [_i64, _i64]),
    "rl_dlaswp": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _vp, _vp]),
    "rl_zpotrf": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_zgetrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]),
    "rl_ztrtri": (ctypes.c_int, [_ch, _ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_zlauum": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_zpotri": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_zgetri_work_size": (_sz, [_i64]),
    "rl_zgetri": (ctypes.c_int, [_i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_zpotrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_zgetrf": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_spotrf_tc_work_size": (ctypes.c_size_t, [_i64, ctypes.c_int]),
    "rl_sgetrf_tc_work_size": (ctypes.c_size_t, [_i64, _i64, ctypes.c_int]),
    "rl_spotrf_tc": (ctypes.c_int, [ctypes.c_int, _ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_clear_cache": (ctypes.c_int, []),
    "rl_oz_work_size": (_sz, [_i64, _i64, _i64, ctypes.c_int]),
    "rl_dgemm_oz": (ctypes.c_int, [ctypes.c_int, _ch, _ch, _i64, _i64, _i64, ctypes.c_double, _vp, _i64, _vp,
                                   _i64, ctypes.c_double, _vp, _i64, _vp, _sz, _vp]),
    "rl_dpotrf_oz_work_size": (_sz, [_i64, ctypes.c_int]),
    "rl_dgetrf_oz_work_size": (_sz, [_i64, _i64, ctypes.c_int]),
    "rl_dpotrf_oz": (ctypes.c_int, [ctypes.c_int, _ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_dgetrf_oz": (ctypes.c_int, [ctypes.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_sgetrf_tc": (ctypes.c_int, [ctypes.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_dgetri_work_size": (ctypes.c_size_t, [_i64]),
    "rl_dgetri": (ctypes.c_int, [_i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_sgetri_work_size": (ctypes.c_size_t, [_i64]),
    "rl_sgetri": (ctypes.c_int, [_i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_dsygst_work_size": (ctypes.c_size_t, [_i64]),
    "rl_ssygst_work_size": (ctypes.c_size_t, [_i64]),
    "rl_ssygst": (ctypes.c_int, [ctypes.c_int, _ch, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_dsygst": (ctypes.c_int, [ctypes.c_int, _ch, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_dgetrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]),
    "rl_dpotrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_dsgesv_work_size": (_sz, [_i64, _i64, ctypes.c_int]),
    "rl_dsposv_work_size": (_sz, [_i64, _i64, ctypes.c_int]),
    "rl_dsgesv": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
    "rl_dsposv": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]),
    "rl_sgemm_tc_work_size": (_sz, [_i64, _i64, _i64, ctypes.c_int]),
    "rl_sgemm_tc": (ctypes.c_int, [ctypes.c_int, _ch, _ch, _i64, _i64, _i64, ctypes.c_float, _vp, _i64,
                                   _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_potrf_vbatched_work_size": (_sz, [_i64]),
    "rl_getrf_vbatched_work_size": (_sz, [_i64]),
    "rl_dpotrf_vbatched": (ctypes.c_int, [_ch, _i64, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _sz, _vp]),
    "rl_spotrf_vbatched": (ctypes.c_int, [_ch, _i64, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _sz, _vp]),
    "rl_dgetrf_vbatched": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _sz, _vp]),
    "rl_sgetrf_vbatched": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _sz, _vp]),
    "rl_vbatched_tune_work_size": (ctypes.c_size_t, [_i64, _i64, ctypes.c_int]),
    "rl_vbatched_tune": (ctypes.c_int, [_ch, ctypes.c_int, _i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp,
                                        _sz, _vp, _vp, _vp]),
    "rl_vbatched_config": (ctypes.c_int, [_ch, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "rl_vbatched_set_config": (ctypes.c_int, [_ch, ctypes.c_int, ctypes.c_int32]),
    "rl_dgetrf_vbatched_noalloc": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp]),
    "rl_spotrf": (ctypes.c_int, [_ch, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rl_sgetrf": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rl_sgetrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]),
    "rl_spotrs": (ctypes.c_int, [_ch, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rl_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "rl_trace_kinds": (ctypes.c_int, []),
    "rl_trace_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                     ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

RL_SUCCESS = 0
RL_ERR_CUDA = 1
RL_ERR_WORKSPACE = 2
RL_ERR_UNSUPPORTED = 3
RL_ERR_NULL_POINTER = 4
RL_ERR_PARAM = 5
RL_INFO_DEVICE_TIMEOUT = -1000

RL_PREC_FP32 = 0
RL_PREC_TF32 = 1
RL_PREC_BF16 = 2
RL_PREC_FP16S = 3
RL_PREC_TF32X3 = 4
RL_PREC_MASK = 0xFF
RL_REFINE_GMRES = 0x100
RL_REFINE_OZRES = 0x200

RL_PARAM_POTRF_CROSSOVER = 1
RL_PARAM_GETRF_PANEL = 2
RL_PARAM_TRTRI_CROSSOVER = 3
RL_PARAM_SPIN_LIMIT_NS = 4
RL_PARAM_BATCH_CTAS = 5
RL_PARAM_TRI_LANES = 6
RL_PARAM_LOOKAHEAD = 7
RL_PARAM_PANEL_CTAS = 8
RL_PARAM_OZ_MIN = 9
RL_PARAM_NVTX = 10
RL_PARAM_GMRES_RESTART = 11
RL_PARAM_PANEL_CLUSTER = 12
RL_PARAM_TC_PAIRS = 13


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _c(ch):
    return ch.encode() if isinstance(ch, str) else ch


def rl_dpotrf(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_dpotrf(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dgetrf(m, n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_dgetrf(m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork,
                          _stream(stream))


def rl_dgetrf_work_size(m, n):
    return int(_lib.rl_dgetrf_work_size(m, n))


def rl_dtrtri(uplo, diag, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_dtrtri(_c(uplo), _c(diag), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork,
                          _stream(stream))


def rl_dlauum(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_dlauum(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dpotri(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_dpotri(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))

def rl_strtri(uplo, diag, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_strtri(_c(uplo), _c(diag), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork,
                          _stream(stream))


def rl_slauum(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_slauum(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_spotri(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_spotri(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    return _lib.rl_dgemm(_c(transa), _c(transb), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                         _ptr(C), ldc, _stream(stream))


def rl_dsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, stream=None):
    return _lib.rl_dsyrk(_c(uplo), _c(trans), n, k, alpha, _ptr(A), lda, beta, _ptr(C), ldc,
                         _stream(stream))


def rl_sgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    return _lib.rl_sgemm(_c(transa), _c(transb), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                         _ptr(C), ldc, _stream(stream))


def rl_ssyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, stream=None):
    return _lib.rl_ssyrk(_c(uplo), _c(trans), n, k, alpha, _ptr(A), lda, beta, _ptr(C), ldc,
                         _stream(stream))


def rl_dtrsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, stream=None):
    return _lib.rl_dtrsm(_c(side), _c(uplo), _c(transa), _c(diag), m, n, alpha, _ptr(A), lda,
                         _ptr(B), ldb, _stream(stream))


def rl_dtrmm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, stream=None):
    return _lib.rl_dtrmm(_c(side), _c(uplo), _c(transa), _c(diag), m, n, alpha, _ptr(A), lda,
                         _ptr(B), ldb, _stream(stream))


def rl_zpotrf(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_zpotrf(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_ztrtri(uplo, diag, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_ztrtri(_c(uplo), _c(diag), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_zlauum(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_zlauum(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_zpotri(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_zpotri(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_zgetri_work_size(n):
    return int(_lib.rl_zgetri_work_size(n))


def rl_zgetri(n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_zgetri(n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_zgetrs(trans, n, nrhs, A, lda, ipiv, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_zgetrs(_c(trans), n, nrhs, _ptr(A), lda, _ptr(ipiv), _ptr(B), ldb, _ptr(work), lwork,
                          _stream(stream))


def rl_zpotrs(uplo, n, nrhs, A, lda, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_zpotrs(_c(uplo), n, nrhs, _ptr(A), lda, _ptr(B), ldb, _ptr(work), lwork, _stream(stream))


def rl_zgetrf(m, n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_zgetrf(m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_clear_cache():
    return _lib.rl_clear_cache()


def rl_oz_work_size(m, n, k, slices):
    return int(_lib.rl_oz_work_size(m, n, k, slices))


def rl_dgemm_oz(slices, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, work, lwork, stream=None):
    return _lib.rl_dgemm_oz(slices, _c(transa), _c(transb), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                            _ptr(C), ldc, _ptr(work), lwork, _stream(stream))


def rl_dpotrf_oz_work_size(n, slices):
    return int(_lib.rl_dpotrf_oz_work_size(n, slices))


def rl_dgetrf_oz_work_size(m, n, slices):
    return int(_lib.rl_dgetrf_oz_work_size(m, n, slices))


def rl_dpotrf_oz(slices, uplo, n, A, lda, info, work, lwork, stream=None):
    return _lib.rl_dpotrf_oz(slices, _c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dgetrf_oz(slices, m, n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_dgetrf_oz(slices, m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork,
                             _stream(stream))


def rl_spotrf_tc_work_size(n, prec):
    return int(_lib.rl_spotrf_tc_work_size(n, prec))


def rl_sgetrf_tc_work_size(m, n, prec):
    return int(_lib.rl_sgetrf_tc_work_size(m, n, prec))


def rl_spotrf_tc(prec, uplo, n, A, lda, info, work, lwork, stream=None):
    return _lib.rl_spotrf_tc(prec, _c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_sgetrf_tc(prec, m, n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_sgetrf_tc(prec, m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork,
                             _stream(stream))


def rl_sgetri_work_size(n):
    return int(_lib.rl_sgetri_work_size(n))


def rl_sgetri(n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_sgetri(n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dgetri_work_size(n):
    return int(_lib.rl_dgetri_work_size(n))


def rl_dgetri(n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_dgetri(n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_ssygst_work_size(n):
    return int(_lib.rl_ssygst_work_size(n))


def rl_ssygst(itype, uplo, n, A, lda, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_ssygst(itype, _c(uplo), n, _ptr(A), lda, _ptr(B), ldb, _ptr(work), lwork, _stream(stream))


def rl_dsygst_work_size(n):
    return int(_lib.rl_dsygst_work_size(n))


def rl_dsygst(itype, uplo, n, A, lda, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_dsygst(itype, _c(uplo), n, _ptr(A), lda, _ptr(B), ldb, _ptr(work), lwork, _stream(stream))


def rl_dlaswp(m, ncols, A, lda, k1, k2, ipiv, stream=None):
    return _lib.rl_dlaswp(m, ncols, _ptr(A), lda, k1, k2, _ptr(ipiv), _stream(stream))


def rl_trs_work_size(n, nrhs):
    return int(_lib.rl_trs_work_size(n, nrhs))


def rl_dgetrs(trans, n, nrhs, A, lda, ipiv, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_dgetrs(_c(trans), n, nrhs, _ptr(A), lda, _ptr(ipiv), _ptr(B), ldb, _ptr(work), lwork,
                           _stream(stream))


def rl_dpotrs(uplo, n, nrhs, A, lda, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_dpotrs(_c(uplo), n, nrhs, _ptr(A), lda, _ptr(B), ldb, _ptr(work), lwork, _stream(stream))


def rl_dsgesv_work_size(n, nrhs, prec):
    return int(_lib.rl_dsgesv_work_size(n, nrhs, prec))


def rl_dsposv_work_size(n, nrhs, prec):
    return int(_lib.rl_dsposv_work_size(n, nrhs, prec))


def rl_dsgesv(n, nrhs, A, lda, ipiv, B, ldb, X, ldx, prec, tol, maxiter, iter_, info, work, lwork,
              stream=None):
    return _lib.rl_dsgesv(n, nrhs, _ptr(A), lda, _ptr(ipiv), _ptr(B), ldb, _ptr(X), ldx, prec, tol,
                          maxiter, _ptr(iter_), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_dsposv(uplo, n, nrhs, A, lda, B, ldb, X, ldx, prec, tol, maxiter, iter_, info, work, lwork,
              stream=None):
    return _lib.rl_dsposv(_c(uplo), n, nrhs, _ptr(A), lda, _ptr(B), ldb, _ptr(X), ldx, prec, tol,
                          maxiter, _ptr(iter_), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_sgemm_tc_work_size(m, n, k, prec):
    return int(_lib.rl_sgemm_tc_work_size(m, n, k, prec))


def rl_sgemm_tc(prec, transa, transb, m, n, k, alpha, A, lda, B, ldb, C, ldc, work, lwork,
                stream=None):
    return _lib.rl_sgemm_tc(prec, _c(transa), _c(transb), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb,
                            _ptr(C), ldc, _ptr(work), lwork, _stream(stream))


def rl_potrf_vbatched_work_size(batch):
    return int(_lib.rl_potrf_vbatched_work_size(batch))


def rl_getrf_vbatched_work_size(batch):
    return int(_lib.rl_getrf_vbatched_work_size(batch))


def rl_dpotrf_vbatched(uplo, batch, n, A, lda, info, max_n, work, lwork, stream=None):
    return _lib.rl_dpotrf_vbatched(_c(uplo), batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(info), max_n,
                                   _ptr(work), lwork, _stream(stream))


def rl_spotrf_vbatched(uplo, batch, n, A, lda, info, max_n, work, lwork, stream=None):
    return _lib.rl_spotrf_vbatched(_c(uplo), batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(info), max_n,
                                   _ptr(work), lwork, _stream(stream))


def rl_dgetrf_vbatched(batch, n, A, lda, ipiv, info, max_n, work, lwork, stream=None):
    return _lib.rl_dgetrf_vbatched(batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(ipiv), _ptr(info), max_n,
                                   _ptr(work), lwork, _stream(stream))


def rl_sgetrf_vbatched(batch, n, A, lda, ipiv, info, max_n, work, lwork, stream=None):
    return _lib.rl_sgetrf_vbatched(batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(ipiv), _ptr(info), max_n,
                                   _ptr(work), lwork, _stream(stream))


RL_BATCH_CONFIGS = 8


def rl_vbatched_tune_work_size(batch, sum_n2, elem_bytes):
    return int(_lib.rl_vbatched_tune_work_size(batch, sum_n2, elem_bytes))


def rl_vbatched_tune(routine, elem_bytes, batch, n, A, lda, ipiv, info, max_n, work, lwork, stream=None):
    """Returns (status, best configuration, list of ms per configuration)."""
    best = ctypes.c_int32(-1)
    ms = (ctypes.c_float * RL_BATCH_CONFIGS)()
    st = _lib.rl_vbatched_tune(_c(routine), elem_bytes, batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(ipiv),
                               _ptr(info), max_n, _ptr(work), lwork, ctypes.byref(best),
                               ctypes.cast(ms, ctypes.c_void_p), _stream(stream))
    return st, best.value, list(ms)


def rl_vbatched_set_config(routine, elem_bytes, cfg):
    return _lib.rl_vbatched_set_config(_c(routine), elem_bytes, cfg)


def rl_vbatched_config(routine, elem_bytes):
    """(cfg, nb, threads, per_sm) in use for the routine and element size."""
    v = [ctypes.c_int32(0) for _ in range(4)]
    st = _lib.rl_vbatched_config(_c(routine), elem_bytes, *[ctypes.byref(x) for x in v])
    check(st, "rl_vbatched_config")
    return tuple(x.value for x in v)


def rl_dgetrf_vbatched_noalloc(batch, n, A, lda, ipiv, info, max_n, stream=None):
    """rl_dgetrf_vbatched with the library's static scratch (no workspace
    argument, nothing allocated): for callers that cannot allocate device
    memory at the call; overlapping calls on one device race on the scratch."""
    return _lib.rl_dgetrf_vbatched_noalloc(batch, _ptr(n), _ptr(A), _ptr(lda), _ptr(ipiv), _ptr(info), max_n,
                                           _stream(stream))


def rl_spotrf(uplo, n, A, lda, info, work=None, lwork=0, stream=None):
    return _lib.rl_spotrf(_c(uplo), n, _ptr(A), lda, _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_sgetrf(m, n, A, lda, ipiv, info, work, lwork, stream=None):
    return _lib.rl_sgetrf(m, n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(work), lwork, _stream(stream))


def rl_sgetrs(trans, n, nrhs, A, lda, ipiv, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_sgetrs(_c(trans), n, nrhs, _ptr(A), lda, _ptr(ipiv), _ptr(B), ldb, _ptr(work), lwork,
                           _stream(stream))


def rl_spotrs(uplo, n, nrhs, A, lda, B, ldb, work=None, lwork=0, stream=None):
    return _lib.rl_spotrs(_c(uplo), n, nrhs, _ptr(A), lda, _ptr(B), ldb, _ptr(work), lwork, _stream(stream))


def rl_host_work_size(routine, m, n, lda):
    return int(_lib.rl_host_work_size(routine.encode(), m, n, lda))


def rl_dpotrf_host(uplo, n, A_host, lda, info_host, work, lwork, stream=None):
    return _lib.rl_dpotrf_host(_c(uplo), n, _ptr(A_host), lda, _ptr(info_host), _ptr(work), lwork,
                               _stream(stream))


def rl_dgetrf_host(m, n, A_host, lda, ipiv_host, info_host, work, lwork, stream=None):
    return _lib.rl_dgetrf_host(m, n, _ptr(A_host), lda, _ptr(ipiv_host), _ptr(info_host),
                               _ptr(work), lwork, _stream(stream))


def rl_set_param(key, value):
    return _lib.rl_set_param(key, value)


def rl_get_param(key):
    return int(_lib.rl_get_param(key))


def rl_launch_count():
    return int(_lib.rl_launch_count())


def rl_status_string(status):
    return _lib.rl_status_string(status).decode()


def rl_trace_enable(on):
    return _lib.rl_trace_enable(1 if on else 0)


def rl_trace_kinds():
    return int(_lib.rl_trace_kinds())


def rl_trace_read(kind):
    """Returns (name, launches, ms, flops, bytes) for one kernel kind."""
    name = ctypes.c_char_p()
    launches = ctypes.c_uint64()
    ms = ctypes.c_double()
    flops = ctypes.c_double()
    nbytes = ctypes.c_double()
    st = _lib.rl_trace_read(kind, ctypes.byref(name), ctypes.byref(launches), ctypes.byref(ms),
                            ctypes.byref(flops), ctypes.byref(nbytes))
    if st != RL_SUCCESS:
        raise ValueError(f"bad trace kind {kind}")
    return name.value.decode(), int(launches.value), ms.value, flops.value, nbytes.value


def trace_summary():
    """All kinds with at least one traced launch, as a dict keyed by name."""
    out = {}
    for k in range(rl_trace_kinds()):
        name, launches, ms, flops, nbytes = rl_trace_read(k)
        if launches:
            out[name] = {"launches": launches, "ms": ms, "flops": flops, "bytes": nbytes}
    return out


def check(status, what="call"):
    """Raise RuntimeError for a nonzero return value of an entry point."""
    if status != RL_SUCCESS:
        raise RuntimeError(f"{what} failed: status {status} ({rl_status_string(status)})")
    return status

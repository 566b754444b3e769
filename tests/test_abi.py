"""The C-ABI library loads on a machine without a GPU, exports every symbol
that include/relgpu.h declares, and its host-side logic (argument checking,
size queries, parameters, status strings) works without touching the device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "relgpu.h")


@pytest.fixture(scope="module")
def built():
    from paper_1602_06763_gb300 import _build
    return _build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_routines():
    names = declared_functions()
    for want in ("rl_dpotrf", "rl_dgetrf", "rl_dtrtri", "rl_dlauum", "rl_dpotri",
                 "rl_dgetrf_work_size", "rl_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_logic_without_gpu(built):
    from paper_1602_06763_gb300 import relgpu as r
    # argument errors are detected on the host before any CUDA call
    assert r.rl_dpotrf("X", 4, 0, 4, 0, None, 0, 0) == -1
    assert r.rl_dpotrf("L", -2, 0, 4, 0, None, 0, 0) == -2
    assert r.rl_dpotrf("L", 4, 0, 4, 0, None, 0, 0) == -3
    assert r.rl_dpotrf("L", 4, 8, 3, 0, None, 0, 0) == -4
    assert r.rl_dgetrf(-1, 1, 8, 1, 8, 8, None, 0, 0) == -1
    assert r.rl_dgetrf(3, -1, 8, 3, 8, 8, None, 0, 0) == -2
    assert r.rl_dgetrf(3, 3, 8, 2, 8, 8, None, 0, 0) == -4
    assert r.rl_dgetrf(3, 3, 8, 3, 8, 8, None, 0, 0) == r.RL_ERR_WORKSPACE
    assert r.rl_dtrtri("L", "X", 3, 8, 3, 8, None, 0, 0) == -2
    assert r.rl_dtrtri("L", "N", 3, 8, 2, 8, None, 0, 0) == -5
    assert r.rl_dlauum("Q", 3, 8, 3, 8, None, 0, 0) == -1
    assert r.rl_dpotri("L", 3, 8, 3, 0, None, 0, 0) == r.RL_ERR_NULL_POINTER
    assert r.rl_dpotrf("U", 3, 8, 2, 8, None, 0, 0) == -4      # 'U' accepted; lda checked
    assert r.rl_dgetrf_work_size(16384, 16384) > 0
    assert r.rl_host_work_size("dpotrf", 10, 10, 12) >= 10 * 12 * 8
    assert r.rl_host_work_size("nope", 10, 10, 10) == 0
    # parameters
    assert r.rl_get_param(r.RL_PARAM_POTRF_CROSSOVER) == 64
    assert r.rl_set_param(r.RL_PARAM_POTRF_CROSSOVER, 65) == r.RL_ERR_PARAM
    assert r.rl_set_param(99, 1) == r.RL_ERR_PARAM
    assert r.rl_get_param(99) == -1
    assert r.rl_set_param(r.RL_PARAM_GETRF_PANEL, 16) == 0
    assert r.rl_get_param(r.RL_PARAM_GETRF_PANEL) == 16
    assert r.rl_set_param(r.RL_PARAM_GETRF_PANEL, 32) == 0
    assert "workspace" in r.rl_status_string(r.RL_ERR_WORKSPACE)
    assert "illegal" in r.rl_status_string(-3)


def test_host_logic_of_the_other_routines(built):
    from paper_1602_06763_gb300 import relgpu as r
    # size queries are pure host arithmetic
    assert r.rl_trs_work_size(16384, 16) > 0 and r.rl_trs_work_size(100, 65) == 0
    assert r.rl_trs_work_size(0, 4) == 0
    assert r.rl_dsygst_work_size(64) == 0 and r.rl_dsygst_work_size(1000) == 8 * 512 * 488   # split 512 + 488
    assert r.rl_dgetri_work_size(1000) >= 8 * 1000
    # argument errors come back before any device work
    assert r.rl_dsygst(0, "L", 4, 8, 4, 8, 4, stream=0) == -1
    assert r.rl_dsygst(1, "Q", 4, 8, 4, 8, 4, stream=0) == -2
    assert r.rl_dsygst(1, "L", -1, 8, 4, 8, 4, stream=0) == -3
    assert r.rl_dsygst(1, "L", 4, 8, 3, 8, 4, stream=0) == -5
    assert r.rl_dsygst(2, "U", 4, 8, 4, 8, 3, stream=0) == -7
    assert r.rl_dgetri(-1, 8, 1, 8, 8, None, 0, stream=0) == -1
    assert r.rl_dgetri(4, 8, 3, 8, 8, None, 0, stream=0) == -3
    assert r.rl_dgetri(4, 8, 4, 8, None, None, 0, stream=0) == r.RL_ERR_NULL_POINTER
    assert r.rl_strtri("L", "X", 4, 8, 4, 8, stream=0) == -2
    assert r.rl_slauum("U", 4, 8, 3, 8, stream=0) == -4
    assert r.rl_spotri("L", 4, 8, 3, 8, stream=0) == -4
    assert r.rl_sgemm("X", "N", 4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, stream=0) == -1
    assert r.rl_ssyrk("U", "N", 4, 4, 1.0, 8, 4, 0.0, 8, 4, stream=0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dgetrs("X", 4, 1, 8, 4, 8, 8, 4, stream=0) == -1
    assert r.rl_dpotrs("L", 4, 1, 8, 3, 8, 4, stream=0) == -5
    assert r.rl_set_param(r.RL_PARAM_TRI_LANES, 3) == r.RL_ERR_PARAM
    assert r.rl_get_param(r.RL_PARAM_TRI_LANES) == 0


def test_host_logic_of_the_tuning_and_lowprec_calls(built):
    from paper_1602_06763_gb300 import relgpu as r
    assert r.rl_spotrf_tc_work_size(1000, r.RL_PREC_FP32) == 0
    assert r.rl_spotrf_tc_work_size(1000, r.RL_PREC_BF16) > 0
    assert r.rl_sgetrf_tc_work_size(1000, 1000, r.RL_PREC_TF32X3) > r.rl_sgetrf_tc_work_size(1000, 1000,
                                                                                           r.RL_PREC_TF32)
    assert r.rl_spotrf_tc(r.RL_PREC_FP32, "L", 4, 8, 4, 8, None, 0, stream=0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_spotrf_tc(r.RL_PREC_BF16, "L", 4, 8, 4, 8, None, 0, stream=0) == r.RL_ERR_WORKSPACE
    assert r.rl_sgetrf_tc(r.RL_PREC_BF16, 4, 4, 8, 3, 8, 8, None, 0, stream=0) == -5
    assert r.rl_dlaswp(10, 4, 8, 10, 0, 5, 8, stream=0) == -5
    assert r.rl_dlaswp(10, 4, 8, 10, 1, 11, 8, stream=0) == -6
    assert r.rl_vbatched_set_config("G", 8, r.RL_BATCH_CONFIGS) == -3
    assert r.rl_vbatched_set_config("X", 8, 0) == -1
    assert r.rl_vbatched_set_config("P", 4, 3) == 0
    assert r.rl_vbatched_config("P", 4)[:2] == (3, 32)
    assert r.rl_vbatched_set_config("P", 4, 0) == 0
    assert r.rl_vbatched_tune_work_size(10, 1000, 8) >= 1000 * 8
    assert r.rl_vbatched_tune_work_size(10, 1000, 3) == 0


def test_host_logic_of_the_complex_upper_and_emulated_calls(built):
    """Argument checks and size queries of the complex, transposed-solve and
    emulated-FP64 entry points return before any device work."""
    from paper_1602_06763_gb300 import relgpu as r
    # complex: LAPACK argument numbering
    assert r.rl_zpotrf("X", 4, 8, 4, 8, stream=0) == -1
    assert r.rl_zgetrf(4, -1, 8, 4, 8, 8, None, 0, stream=0) == -2
    assert r.rl_ztrtri("L", "Q", 4, 8, 4, 8, stream=0) == -2
    assert r.rl_zlauum("L", 4, 8, 3, 8, stream=0) == -4
    assert r.rl_zpotri("Q", 4, 8, 4, 8, stream=0) == -1
    assert r.rl_zgetri(-1, 8, 1, 8, 8, None, 0, stream=0) == -1
    assert r.rl_zgetri_work_size(1000) == r.rl_dgetri_work_size(1000)
    assert r.rl_zgetrs("Q", 4, 1, 8, 4, 8, 8, 4, stream=0) == -1
    assert r.rl_zgetrs("N", 4, 1, 8, 3, 8, 8, 4, stream=0) == -5
    assert r.rl_zgetrs("T", 4, 1, 8, 4, 8, 8, 4, stream=0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_zpotrs("L", 4, 1, 8, 4, 8, 3, stream=0) == -7
    # transposed real solves: argument checks
    assert r.rl_sgetrs("Q", 4, 1, 8, 4, 8, 8, 4, stream=0) == -1
    assert r.rl_dgetrs("T", 4, -1, 8, 4, 8, 8, 4, stream=0) == -3
    # emulated FP64: slices, arguments, workspace queries
    assert r.rl_oz_work_size(100, 100, 100, 5) == 0 and r.rl_oz_work_size(100, 100, 100, 9) == 0
    w7 = r.rl_oz_work_size(1000, 500, 300, 7)
    # digit planes: 7 planes x 2 bytes x (rows padded to 128 + columns padded to 64) x k padded to 64
    assert w7 >= 7 * 2 * (1024 + 512) * 320
    assert r.rl_oz_work_size(1000, 500, 300, 8) > w7 > r.rl_oz_work_size(1000, 500, 300, 6)
    assert r.rl_dpotrf_oz_work_size(4096, 7) >= 2 * r.rl_oz_work_size(2112, 2112, 2112, 7)
    assert r.rl_dgetrf_oz_work_size(4096, 4096, 7) > r.rl_oz_work_size(4096, 4096, 2112, 7)
    assert r.rl_dgemm_oz(7, "N", "X", 4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, None, 0, stream=0) == -3
    assert r.rl_dgemm_oz(7, "N", "N", -1, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, None, 0, stream=0) == -4
    assert r.rl_dgemm_oz(7, "N", "N", 4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 3, None, 0, stream=0) == -14
    assert r.rl_dgemm_oz(7, "N", "N", 4, 4, 1 << 22, 1.0, 8, 4, 8, 1 << 22, 0.0, 8, 4, None, 0,
                         stream=0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dpotrf_oz(9, "L", 4, 8, 4, 8, None, 0, stream=0) == -1
    assert r.rl_dpotrf_oz(7, "L", 4, 8, 3, 8, None, 0, stream=0) == -5
    assert r.rl_dgetrf_oz(7, 4, 4, 8, 4, 8, 8, None, 0, stream=0) == r.RL_ERR_WORKSPACE
    assert r.rl_set_param(r.RL_PARAM_OZ_MIN, 0) == r.RL_ERR_PARAM
    assert r.rl_get_param(r.RL_PARAM_OZ_MIN) == 128
    assert r.rl_get_param(r.RL_PARAM_NVTX) == 0
    assert r.rl_set_param(r.RL_PARAM_NVTX, 2) == r.RL_ERR_PARAM
    assert r.rl_set_param(r.RL_PARAM_NVTX, 1) == 0 and r.rl_get_param(r.RL_PARAM_NVTX) == 1
    assert r.rl_set_param(r.RL_PARAM_NVTX, 0) == 0


def test_binding_has_every_declared_entry_point(built):
    """The Python binding carries the same names as the C ABI: a ctypes
    signature and a wrapper function for each declared routine."""
    from paper_1602_06763_gb300 import relgpu as r
    src = open(os.path.join(ROOT, "paper_1602_06763_gb300", "relgpu.py")).read()
    for name in declared_functions():
        assert f'"{name}"' in src, name
        assert callable(getattr(r, name, None)), name


def test_host_logic_of_the_gmres_refinement(built):
    from paper_1602_06763_gb300 import relgpu as r
    g = r.RL_REFINE_GMRES
    n, nrhs = 1000, 16
    for prec in (r.RL_PREC_FP32, r.RL_PREC_BF16, r.RL_PREC_TF32X3):
        base = r.rl_dsgesv_work_size(n, nrhs, prec)
        gm = r.rl_dsgesv_work_size(n, nrhs, prec | g)
        m = r.rl_get_param(r.RL_PARAM_GMRES_RESTART)
        # the basis V (m + 1 vectors) and Z (m vectors) per right-hand side, FP64
        assert gm - base >= nrhs * (2 * m + 1) * n * 8
        assert r.rl_dsposv_work_size(n, nrhs, prec | g) > r.rl_dsposv_work_size(n, nrhs, prec)
    assert r.rl_dsgesv_work_size(n, nrhs, 0x400) == 0                # unknown flag bits
    # emulated residual products: A's digit planes (7 x 2 bytes per element) in the workspace
    oz = r.rl_dsgesv_work_size(n, nrhs, r.RL_REFINE_OZRES) - r.rl_dsgesv_work_size(n, nrhs, 0)
    assert oz >= 14 * n * n
    assert r.rl_dsposv_work_size(n, nrhs, r.RL_REFINE_OZRES | g) > r.rl_dsposv_work_size(n, nrhs, g)
    assert r.rl_dsgesv_work_size(n, nrhs, 7 | g) == 0                # unknown precision
    # the restart length sizes the workspace and is range-checked
    assert r.rl_get_param(r.RL_PARAM_GMRES_RESTART) == 50
    w50 = r.rl_dsgesv_work_size(n, nrhs, g)
    assert r.rl_set_param(r.RL_PARAM_GMRES_RESTART, 10) == 0
    assert r.rl_dsgesv_work_size(n, nrhs, g) < w50
    assert r.rl_set_param(r.RL_PARAM_GMRES_RESTART, 0) == r.RL_ERR_PARAM
    assert r.rl_set_param(r.RL_PARAM_GMRES_RESTART, 65) == r.RL_ERR_PARAM
    assert r.rl_set_param(r.RL_PARAM_GMRES_RESTART, 50) == 0
    # more than 64 right-hand sides with the GMRES refinement: unsupported
    # (checked on the host before any launch)
    assert r.rl_dsgesv(n, 65, 8, n, 8, 8, n, 8, n, g, 1e-14, 30, 8, 8, 8, 1 << 40, 0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dsposv("L", n, 65, 8, n, 8, n, 8, n, g, 1e-14, 30, 8, 8, 8, 1 << 40, 0) == r.RL_ERR_UNSUPPORTED
    assert r.rl_dsgesv(n, 65, 8, n, 8, 8, n, 8, n, 0, 1e-14, 30, 8, 8, None, 0, 0) == r.RL_ERR_WORKSPACE


def test_host_logic_of_the_cluster_parameters(built):
    from paper_1602_06763_gb300 import relgpu as r
    for key in (r.RL_PARAM_PANEL_CLUSTER, r.RL_PARAM_TC_PAIRS):
        assert r.rl_get_param(key) == 1                  # on by default
        assert r.rl_set_param(key, 0) == 0 and r.rl_get_param(key) == 0
        assert r.rl_set_param(key, 2) == r.RL_ERR_PARAM
        assert r.rl_set_param(key, -1) == r.RL_ERR_PARAM
        assert r.rl_set_param(key, 1) == 0 and r.rl_get_param(key) == 1

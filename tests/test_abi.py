"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"\b(mvgd_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1603_04100_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mvgd_knn", "mvgd_assemble", "mvgd_spmv", "mvgd_solve", "mvgd_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = C.CDLL(str(lib_path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_only_the_abi(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_path)], capture_output=True, text=True).stdout
    ours = sorted({line.split()[-1] for line in out.splitlines() if line.split()[-1].startswith("mvgd_")})
    assert ours == declared_functions()


def test_host_side_queries(lib_path):
    from paper_1603_04100_gb300 import _lib as LB
    L = LB.load(lib_path)
    assert L.mvgd_version() >= 100
    assert LB.status_string(LB.EINVAL).startswith("MVGD_EINVAL")
    n, k = 1000, 20
    assert L.mvgd_knn_workspace_bytes(n, k) > 16 * n
    assert L.mvgd_ell_bytes(n, k, LB.FP64, LB.ELL_VAL) == 1024 * 21 * 8
    assert L.mvgd_ell_bytes(n, k, LB.FP32_REFINE, LB.ELL_VAL_LO) == 1024 * 21 * 4
    assert L.mvgd_ell_bytes(n, k, LB.FP64, LB.ELL_VAL_LO) == 0
    assert L.mvgd_solve_workspace_bytes(n, k, 2, LB.FP32_REFINE, 1) > 9 * 4 * 2 * n
    # the multigrid hierarchy and its per-level vectors come on top
    assert L.mvgd_solve_workspace_bytes(n, k, 2, LB.FP32_REFINE, 2) > (L.mvgd_solve_workspace_bytes(
        n, k, 2, LB.FP32_REFINE, 1) + L.mvgd_amg_workspace_bytes(n, k))
    assert L.mvgd_amg_workspace_bytes(n, k) > 4 * (k + 1) * n
    assert L.mvgd_amg_workspace_bytes(n, 4) == 0 and L.mvgd_amg_workspace_bytes(0, k) == 0
    assert L.mvgd_amg_apply_workspace_bytes(n, 2) >= 2 * 4 * 2 * n
    assert L.mvgd_request_workspace_bytes(n, k, 1, LB.FP64, 3) == 0


def test_argument_errors_are_reported_before_any_launch(lib_path):
    """Null or misaligned pointers and bad sizes return MVGD_EINVAL without touching the device."""
    from paper_1603_04100_gb300 import _lib as LB
    L = LB.load(lib_path)
    assert L.mvgd_knn(None, 100, 10, None, None, 0.0, None, 0, None) == LB.EINVAL
    assert L.mvgd_knn(C.c_void_p(256), 100, 40, C.c_void_p(512), None, 0.0, C.c_void_p(1024), 1 << 20,
                      None) == LB.EINVAL                      # k > 31
    assert L.mvgd_knn(C.c_void_p(257), 100, 10, C.c_void_p(512), None, 0.0, C.c_void_p(1024), 1 << 20,
                      None) == LB.EINVAL                      # misaligned
    assert L.mvgd_knn(C.c_void_p(256), 100, 10, C.c_void_p(512), None, 0.0, C.c_void_p(1024), 16,
                      None) == LB.EWORKSPACE
    e = LB.Ell(100, 4, LB.FP64, None, C.c_void_p(256), C.c_void_p(512), None)
    rule = LB.DeltaRule(LB.DELTA_MEAN_NN, 6, 1.0)
    assert L.mvgd_assemble(C.c_void_p(256), 100, 4, C.c_void_p(512), rule, C.byref(e), None, None, None, None, 0,
                           None) == LB.EINVAL                 # k < 5
    e = LB.Ell(100, 10, LB.FP64, None, C.c_void_p(256), C.c_void_p(512), None)
    bad = LB.DeltaRule(LB.DELTA_MEAN_NN, 11, 1.0)
    assert L.mvgd_assemble(C.c_void_p(256), 100, 10, C.c_void_p(512), bad, C.byref(e), None, None, None, None, 0,
                           None) == LB.EINVAL                 # m > k
    bad = LB.DeltaRule(LB.DELTA_MEAN_NN, 6, 1.0, 2)
    assert L.mvgd_assemble(C.c_void_p(256), 100, 10, C.c_void_p(512), bad, C.byref(e), None, None, None, None, 0,
                           None) == LB.EINVAL                 # unknown row variant
    assert L.mvgd_row_signs(None, C.c_void_p(256), None) == LB.EINVAL
    assert L.mvgd_row_signs(C.byref(e), C.c_void_p(260), None) == LB.EINVAL  # counts not 8-byte aligned
    # block sets: p not a multiple of w, X == Y, null mask
    assert L.mvgd_block_gram(C.c_void_p(256), 7, C.c_void_p(512), 8, 100, 8, C.c_void_p(1024), C.c_void_p(2048),
                             1 << 20, None) == LB.EINVAL
    assert L.mvgd_block_combine(C.c_void_p(256), 8, C.c_void_p(1024), 8, 100, 8, C.c_void_p(256),
                                None) == LB.EINVAL
    assert L.mvgd_block_zero_rows(C.c_void_p(256), 8, 100, 8, None, None) == LB.EINVAL
    assert L.mvgd_dirichlet_rows(None, C.c_void_p(256), None, None) == LB.EINVAL
    # Gauss-Seidel power iteration: no steps, no status word, a NaN shift, too small a workspace
    assert L.mvgd_gs_power_workspace_bytes(100, 0) == 0
    assert L.mvgd_gs_power_workspace_bytes(100, 10) >= 2 * 8 * 100 + 4 * 100 + 4 * 10
    gs = (C.c_void_p(256), 10, C.c_void_p(512), C.c_void_p(768), C.c_void_p(1024), C.c_void_p(2048), 1 << 20, None)
    assert L.mvgd_gs_power(C.byref(e), 1.0, gs[0], 0, *gs[2:]) == LB.EINVAL
    assert L.mvgd_gs_power(C.byref(e), 1.0, *gs[:4], None, *gs[5:]) == LB.EINVAL
    assert L.mvgd_gs_power(C.byref(e), float("nan"), *gs) == LB.EINVAL
    assert L.mvgd_gs_power(C.byref(e), 1.0, *gs[:6], 64, None) == LB.EWORKSPACE
    # Neumann ghosts: kb below 2, no counts word, too small a workspace; fold: k or order mismatch
    assert L.mvgd_neumann_ghosts_workspace_bytes(1) == 0 and L.mvgd_neumann_ghosts_workspace_bytes(100) > 24 * 100
    ng = [C.c_void_p(256), 100, 10, C.c_void_p(512), C.c_void_p(768), 6] + [C.c_void_p(1024 * (i + 1)) for i in range(6)]
    assert L.mvgd_neumann_ghosts(*ng[:5], 1, *ng[6:], C.c_void_p(8192), 1 << 20, None) == LB.EINVAL
    assert L.mvgd_neumann_ghosts(*ng[:11], None, C.c_void_p(8192), 1 << 20, None) == LB.EINVAL
    assert L.mvgd_neumann_ghosts(*ng, C.c_void_p(8192), 64, None) == LB.EWORKSPACE
    eq = LB.Ell(120, 10, LB.FP64, None, C.c_void_p(256), C.c_void_p(512), None)
    ei = LB.Ell(100, 12, LB.FP64, C.c_void_p(4096), C.c_void_p(1024), C.c_void_p(2048), None)
    assert L.mvgd_neumann_fold(C.byref(eq), C.c_void_p(768), C.byref(ei), C.c_void_p(8192), 1 << 20,
                               None) == LB.EINVAL
    ei = LB.Ell(100, 10, LB.FP64, None, C.c_void_p(1024), C.c_void_p(2048), None)
    assert L.mvgd_neumann_fold(C.byref(eq), C.c_void_p(768), C.byref(ei), C.c_void_p(8192), 1 << 20,
                               None) == LB.EINVAL
    # the condition's term: more interior points than rows, a misaligned output
    assert L.mvgd_neumann_rhs(C.byref(eq), 121, C.c_void_p(256), C.c_void_p(512), C.c_void_p(768),
                              C.c_void_p(1024), None) == LB.EINVAL
    assert L.mvgd_neumann_rhs(C.byref(eq), 100, C.c_void_p(256), C.c_void_p(512), C.c_void_p(768),
                              C.c_void_p(1032), None) == LB.EINVAL
    e4 = LB.Ell(100, 4, LB.FP64, None, C.c_void_p(256), C.c_void_p(512), None)
    assert L.mvgd_row_signs(C.byref(e4), C.c_void_p(256), None) == LB.EINVAL  # k < 5
    assert L.mvgd_spmv(C.byref(e), LB.SPMV_F32, 1, 1.0, 1.0, C.c_void_p(256), 0.0, C.c_void_p(512),
                       None) == LB.EINVAL                     # FP32 mode on an FP64 operator
    opts = LB.SolveOpts(0.0, 10, 10, 1e-5, 5, 0)
    info = (LB.SolveInfo * 1)()
    assert L.mvgd_solve(C.byref(e), 1, 1.0, C.c_void_p(256), C.c_void_p(512), C.byref(opts),
                        C.cast(info, C.c_void_p), None, C.c_void_p(1024), 1 << 30, None) == LB.EINVAL  # rtol 0
    # multigrid: bad K, misaligned workspace, too small a workspace; an iterate with an unknown preconditioner
    e5 = LB.Ell(100, 4, LB.FP64, None, C.c_void_p(256), C.c_void_p(512), None)
    assert L.mvgd_amg_setup(C.byref(e5), 1.0, C.c_void_p(1024), 1 << 30, None) == LB.EINVAL
    assert L.mvgd_amg_setup(C.byref(e), 1.0, C.c_void_p(1025), 1 << 30, None) == LB.EINVAL
    assert L.mvgd_amg_setup(C.byref(e), 1.0, C.c_void_p(1024), 64, None) == LB.EWORKSPACE
    reqs = LB.requests([(256, 100, 1, 10)])
    assert L.mvgd_iterate(reqs, 1, LB.FP64, 3, 10, None, C.c_void_p(1024), 1 << 20, None) == LB.EINVAL
    assert L.mvgd_iterate(reqs, 1, LB.FP64, 0, 10, None, C.c_void_p(1024), 16, None) == LB.EWORKSPACE
    amg_opts = LB.SolveOpts(1e-8, 10, 10, 1e-5, 5, 2, C.c_void_p(0))
    assert L.mvgd_request_init(C.c_void_p(1024), 1 << 30, C.byref(e), 1, 1.0, C.c_void_p(256), None,
                               C.byref(amg_opts), None) == LB.EINVAL  # precond 2 needs a hierarchy


def test_binding_modules_import():
    # the Python layer imports without a GPU (the CUDA path is only reached on a call)
    import importlib
    for mod in ("api", "batch", "eigs", "pipeline", "serve", "inputs", "replicas"):
        importlib.import_module(f"paper_1603_04100_gb300.{mod}")


def test_wait_limit_controls_are_host_side(lib_path):
    # both controls only set host state read by the next launch: callable without a GPU
    from paper_1603_04100_gb300 import _lib as LB
    L = LB.load(lib_path)
    assert L.mvgd_set_wait_limit(-1) == LB.EINVAL
    assert L.mvgd_set_wait_limit(4096) == LB.OK
    assert L.mvgd_set_wait_limit(0) == LB.OK
    assert L.mvgd_test_withhold_arrival(1) == LB.OK
    assert L.mvgd_test_withhold_arrival(0) == LB.OK

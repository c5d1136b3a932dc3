"""The C-ABI library builds, loads and exports every entry point of include/ot.h (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ot.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2209_00315_gb300 import build

    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["ot_mesh_create", "ot_mesh_destroy", "ot_mesh_info", "ot_ipm_solve", "ot_newton_solve",
                 "ot_cost_grad", "ot_last_error", "ot_ipm_solve_batched"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ot_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors_without_gpu(lib_path):
    """Host-only calls work without a device: defaults, mesh creation, argument errors."""
    from paper_2209_00315_gb300 import capi

    lib = capi.load()
    o = capi.default_options()
    assert o.fgmres_max_iter == 400 and abs(o.eps_out - 1e-5) < 1e-20 and abs(o.eps_schur - 0.1) < 1e-15
    m = capi.Mesh(8)
    assert (m.n_coarse, m.n_fine, m.n_edges_fine) == (128, 512, 12 * 64 - 32)
    with pytest.raises(capi.OTError) as e:
        capi.Mesh(13)
    assert e.value.code == 1 and "2^a" in str(e.value)
    h = ctypes.c_void_p()
    assert lib.ot_mesh_create(None, ctypes.byref(h)) == 1
    assert b"NULL" in lib.ot_last_error()
    # batched: argument checks come before any device work
    assert lib.ot_ipm_solve_batched(0, None, None, None, None, 1.0, 1e-6, ctypes.byref(o), None, None, None,
                                    None, None, None, 4) == 0
    assert lib.ot_ipm_solve_batched(1, None, None, None, None, 1.0, 1e-6, ctypes.byref(o), None, None, None,
                                    None, None, None, 0) == 1
    assert b"n_streams" in lib.ot_last_error()
    assert lib.ot_ipm_solve_batched(1, None, None, None, None, 1.0, 1e-6, ctypes.byref(o), None, None, None,
                                    None, None, None, 2) == 1
    assert b"NULL" in lib.ot_last_error()


def test_package_does_not_import_the_oracle():
    """The CUDA path and the oracle share no code (the binding never imports oracle/)."""
    pkg = os.path.join(ROOT, "paper_2209_00315_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "__init__.py", f


def test_noalloc_entry_point_checks_arguments_before_device_work(lib_path):
    """ot_kkt_apply_noalloc rejects sizes beyond its static scratch, unsupported
    sides and NULL arrays with OT_ERR_INVALID_ARG before it touches a device."""
    from paper_2209_00315_gb300 import capi

    lib = capi.load()
    p = [ctypes.c_void_p(16)] * 7   # never dereferenced: every case fails its argument check first
    assert lib.ot_kkt_apply_noalloc(8, 4097, *p, None) == 1
    assert b"4096" in lib.ot_last_error()
    assert lib.ot_kkt_apply_noalloc(13, 4, *p, None) == 1
    assert lib.ot_kkt_apply_noalloc(8, 0, *p, None) == 1
    assert lib.ot_kkt_apply_noalloc(8, 4, None, *p[1:], None) == 1
    assert b"NULL" in lib.ot_last_error()


def test_cube_meshes_report_their_grid_and_refuse_the_solver_calls(lib_path):
    """The 3D Cartesian mesh (n^3 cubes, J = I) reports n^3 cells on both levels,
    3 n^2 (n - 1) faces and cell volumes 1/n^3; every solver entry point returns
    OT_ERR_INVALID_ARG for it before any device work."""
    from paper_2209_00315_gb300 import capi

    lib = capi.load()
    m = capi.Mesh(5, kind="cube")
    assert (m.n_coarse, m.n_fine, m.n_edges_fine) == (125, 125, 3 * 25 * 4)
    assert abs(float(m.coarse_areas.sum()) - 1.0) < 1e-14
    with pytest.raises(capi.OTError):
        capi.Mesh(0, kind="cube")
    o = capi.default_options()
    p = ctypes.c_void_p(16)   # never dereferenced
    st = capi.ot_stats()
    assert lib.ot_ipm_solve(m.handle, p, p, 4, 1.0, 1e-6, ctypes.byref(o), 0, p, p, p, None, ctypes.byref(st),
                            None) == 1
    assert b"3D Cartesian" in lib.ot_last_error()
    assert lib.ot_newton_solve(m.handle, 4, 0.1, p, p, p, p, p, ctypes.byref(o), p, p, p, None, None) == 1
    assert lib.ot_bb_apply(m.handle, 4, ctypes.byref(o), p, p, p, p, p, p, p, None) == 1
    assert b"3D Cartesian" in lib.ot_last_error()


def test_solver_entry_points_check_arguments_before_allocating(lib_path):
    """Bad scalars, sizes and NULL arrays are rejected before any workspace is
    allocated, so these calls return OT_ERR_INVALID_ARG without a device."""
    from paper_2209_00315_gb300 import capi

    lib = capi.load()
    o = capi.default_options()
    m = capi.Mesh(4)
    p = ctypes.c_void_p(16)   # never dereferenced
    st = capi.ot_stats()
    solve = lambda K, mu0, tol, r0, out: lib.ot_ipm_solve(  # noqa: E731
        m.handle, r0, r0, K, mu0, tol, ctypes.byref(o), 0, out, out, out, None, ctypes.byref(st), None)
    assert solve(4, 0.0, 1e-6, p, p) == 1 and b"mu0" in lib.ot_last_error()
    assert solve(4, 1.0, -1.0, p, p) == 1
    assert solve(0, 1.0, 1e-6, p, p) == 1 and b"K must be" in lib.ot_last_error()
    assert solve(5000, 1.0, 1e-6, p, p) == 1
    assert solve(4, 1.0, 1e-6, None, p) == 1 and b"NULL" in lib.ot_last_error()
    assert solve(4, 1.0, 1e-6, p, None) == 1 and b"NULL" in lib.ot_last_error()
    assert lib.ot_newton_solve(m.handle, 4, -1.0, p, p, p, p, p, ctypes.byref(o), p, p, p, None, None) == 1
    assert b"mu" in lib.ot_last_error()
    assert lib.ot_cost_grad(m.handle, 4, 1e-3, p, p, p, p, p, ctypes.byref(o), None, p, None) == 1
    assert b"NULL" in lib.ot_last_error()
    bad = capi.default_options(tau=1.5)
    assert lib.ot_ipm_solve(m.handle, p, p, 4, 1.0, 1e-6, ctypes.byref(bad), 0, p, p, p, None, None, None) == 1
    # the preconditioner choice: BB by default, SIMPLE after mu < 1e-5 in the hybrid; others rejected
    assert o.precond == capi.OT_PRECOND_BB and abs(o.simple_mu - 1e-5) < 1e-20
    for bad in (capi.default_options(precond=3), capi.default_options(precond="hybrid", simple_mu=-1.0)):
        assert lib.ot_ipm_solve(m.handle, p, p, 4, 1.0, 1e-6, ctypes.byref(bad), 0, p, p, p, None, None, None) == 1
        assert b"precond" in lib.ot_last_error() or b"simple_mu" in lib.ot_last_error()
    assert lib.ot_simple_apply(m.handle, 4, ctypes.byref(o), p, p, p, p, p, None, p, None) == 1
    assert b"NULL" in lib.ot_last_error()


def test_autotuner_checks_arguments_and_candidates_before_device_work(lib_path):
    """ot_tune_newton validates its options, state pointers and every candidate
    setting before its first trial solve."""
    from paper_2209_00315_gb300 import capi

    lib = capi.load()
    m = capi.Mesh(4)
    o = capi.default_options()
    p = ctypes.c_void_p(16)   # never dereferenced
    cand = (ctypes.c_int32 * 6)(2, 6, 2, 2, 6, 0)   # the second candidate has lap_cycles = 0
    tune = lambda mu, opt, n, c, phi=p: lib.ot_tune_newton(  # noqa: E731
        m.handle, 4, mu, phi, p, p, p, p, opt, n, c, None, None)
    assert tune(1e-3, None, 1, cand) == 1 and b"opt is NULL" in lib.ot_last_error()
    assert tune(0.0, ctypes.byref(o), 1, cand) == 1 and b"mu" in lib.ot_last_error()
    assert tune(1e-3, ctypes.byref(o), 1, cand, phi=None) == 1 and b"NULL" in lib.ot_last_error()
    assert tune(1e-3, ctypes.byref(o), 0, cand) == 1 and b"n_cand" in lib.ot_last_error()
    assert tune(1e-3, ctypes.byref(o), 2, cand) == 1 and b"cycle counts" in lib.ot_last_error()
    assert (o.smooth_sweeps, o.coarse_sweeps, o.lap_cycles) == (2, 6, 2)   # unchanged on error
    assert len(capi.TUNE_GRID) == 12 and (2, 6, 2) in capi.TUNE_GRID

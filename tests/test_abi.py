"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/rsg.h declares, builds meshes on the host identical (as point sets) to
the oracle's, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from paper_1501_05654_gb300 import rsg as binding
from tests._parity import perm_lib_to_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rsg.build()
    return binding.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rsg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SIGNATURES), set(names) ^ set(binding.SIGNATURES)


@pytest.mark.parametrize("case", [("cube", 13), ("box", (7, 11, 5)), ("sphere", 2.3)])
def test_mesh_point_sets_match_oracle(lib, case):
    kind, arg = case
    if kind == "cube":
        lm, om = rsg.Mesh(rsg.CUBE, arg, spacing=0.3), oracle.Mesh(oracle.CUBE, arg, h=0.3)
    elif kind == "box":
        lm, om = rsg.Mesh(rsg.BOX, arg, spacing=0.25), oracle.Mesh(oracle.BOX, arg, h=0.25)
    else:
        lm, om = rsg.Mesh(rsg.SPHERE, radius=arg, spacing=0.3), oracle.Mesh(oracle.SPHERE, radius=arg, h=0.3)
    assert lm.P == om.P
    idx = perm_lib_to_oracle(lm.ijk, om.ijk)
    assert np.abs(lm.xyz - om.xyz[idx]).max() < 1e-13


def test_library_point_order_is_rows(lib):
    """z slowest, then y, x fastest; each (y, z) row contiguous."""
    m = rsg.Mesh(rsg.SPHERE, radius=3.0, spacing=0.5)
    key = m.ijk[:, 2] * 10 ** 6 + m.ijk[:, 1] * 10 ** 3 + m.ijk[:, 0]
    assert np.all(np.diff(key) > 0)


def test_sphere_count_full_size(lib):
    assert rsg.Mesh(rsg.SPHERE, radius=18.0, spacing=0.2).P == 3053617


def _status(f, *args):
    return f(*args)


def test_argument_errors_without_device(lib):
    h = C.c_void_p()
    n = (C.c_int32 * 3)(4, 4, 4)
    assert lib.rsg_mesh_create(0, n, 0.0, -1.0, C.byref(h)) == -1
    assert b"spacing" in lib.rsg_last_error()
    big = (C.c_int32 * 3)(1025, 4, 4)
    assert lib.rsg_mesh_create(2, big, 0.0, 0.3, C.byref(h)) == -1
    assert lib.rsg_mesh_create(1, None, -2.0, 0.3, C.byref(h)) == -1
    assert lib.rsg_mesh_create(7, n, 0.0, 0.3, C.byref(h)) == -1
    assert lib.rsg_mesh_create(0, n, 0.0, 0.3, None) == -1
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m)
    with pytest.raises(rsg.RSGError, match="ARG"):
        H.set_option("rx", 3)
    with pytest.raises(rsg.RSGError, match="ARG"):
        H.set_option("nonsense", 1)
    with pytest.raises(rsg.RSGError, match="UNSUPPORTED"):
        H.set_projectors([[0, 0, 0]], [1.0], [3], [0.25], [np.eye(16)])
    # NULL state pointers and a missing potential are rejected on the host
    assert lib.rsg_hamiltonian_apply(H._h, None, None, 1, 2, None) == -1
    assert lib.rsg_propagate_steps(H._h, None, 1, 2, 1, 0.1, 0, 1, None, None, 0, None, None) == -1
    assert lib.rsg_ham_create(m._h, 5, C.byref(h)) == -1


def test_odd_ld_rejected_for_complex64(lib):
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m)
    fake = C.c_void_p(16)   # never dereferenced: the check fails first
    assert lib.rsg_hamiltonian_apply(H._h, fake, C.c_void_p(4096), 3, 3, None) == -1
    assert b"even ld" in lib.rsg_last_error()
    fake_mis = C.c_void_p(8)
    assert lib.rsg_hamiltonian_apply(H._h, fake_mis, C.c_void_p(4096), 2, 2, None) == -1
    assert b"aligned" in lib.rsg_last_error()


def test_solver_entry_points_argument_errors(lib):
    """Host-side checks of the eigensolver, shifted solver, control loop and
    absorber, which fail before any device work (no GPU needed)."""
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex128)
    fake, fake2 = C.c_void_p(4096), C.c_void_p(1 << 30)   # never dereferenced
    ev = np.zeros(2)
    it = C.c_int64()
    # NULL eigenvalue output, then no potential
    assert lib.rsg_eigensolve(H._h, fake, 2, 2, 2, 10, 8, 1e-8, None, None, None, None) == -1
    assert lib.rsg_eigensolve(H._h, fake, 2, 2, 2, 10, 8, 1e-8, ev.ctypes.data_as(C.c_void_p), None,
                              C.byref(it), None) == -7
    assert lib.rsg_shifted_solve(H._h, fake, None, 2, 2, 0.1, 0.1, 10, 1e-8, None, None, None) == -1
    assert lib.rsg_shifted_solve(H._h, fake, fake2, 2, 2, 0.1, 0.1, 10, 1e-8, None, None, None) == -7
    J = C.c_double()
    assert lib.rsg_control_optimize(H._h, fake, fake2, 4, 0.05, 1, 1, None, None, 50, 5, 1e-8, C.byref(J),
                                    None, None, None, None) == -1
    eps = np.zeros(4)
    assert lib.rsg_control_optimize(H._h, fake, fake2, 4, 0.05, 1, 1, eps.ctypes.data_as(C.c_void_p), None, 50,
                                    -1, 1e-8, C.byref(J), None, None, None, None) == -1
    bad = np.full(m.P, 2.0)
    assert lib.rsg_absorber_set(H._h, bad.ctypes.data_as(C.c_void_p), 0) == -1
    assert b"[0, 1]" in lib.rsg_last_error()
    assert lib.rsg_absorber_set(H._h, None, 0) == 0


def test_complex_scaling_argument_errors(lib):
    """Host-side checks of rsg_complex_scaling_set (no device work)."""
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex64)
    vt = np.zeros(2 * m.P)
    p = vt.ctypes.data_as(C.c_void_p)
    assert lib.rsg_complex_scaling_set(None, 0.3, p, 0) == -1
    assert lib.rsg_complex_scaling_set(H._h, -0.1, p, 0) == -1
    assert lib.rsg_complex_scaling_set(H._h, 0.8, p, 0) == -1
    assert b"pi/4" in lib.rsg_last_error()
    assert lib.rsg_complex_scaling_set(H._h, float("nan"), p, 0) == -1
    assert lib.rsg_complex_scaling_set(H._h, 0.3, None, 0) == 0     # removal
    d = np.array([1.0, 0.0, 0.0])
    assert lib.rsg_field_set(H._h, 0.05, d.ctypes.data_as(C.c_void_p)) == 0
    assert lib.rsg_complex_scaling_set(H._h, 0.3, p, 0) == -4
    assert b"dipole field" in lib.rsg_last_error()
    assert lib.rsg_field_set(H._h, 0.0, d.ctypes.data_as(C.c_void_p)) == 0
    vt[5] = np.inf
    assert lib.rsg_complex_scaling_set(H._h, 0.3, p, 0) == -1
    assert b"not finite" in lib.rsg_last_error()


def test_fourier_basis(lib):
    """Sine series at interval midpoints: the discrete sine transform's
    orthogonality (sum_k s_m s_m' = n/2 delta) and the field's zeros at the
    ends of [0, T] (values at the first and last midpoints shrink as
    sin(m pi / 2n))."""
    n, M = 40, 7
    B = rsg.fourier_basis(n, M)
    assert B.shape == (n, M)
    assert np.abs(B.T @ B - 0.5 * n * np.eye(M)).max() < 1e-12
    for m in range(1, M + 1):
        assert abs(abs(B[0, m - 1]) - np.sin(m * np.pi / (2 * n))) < 1e-13
        assert abs(abs(B[-1, m - 1]) - np.sin(m * np.pi / (2 * n))) < 1e-13
    assert lib.rsg_fourier_basis(0, 3, B.ctypes.data_as(C.c_void_p)) == -1
    assert lib.rsg_fourier_basis(4, 0, B.ctypes.data_as(C.c_void_p)) == -1
    assert lib.rsg_fourier_basis(4, 3, None) == -1
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex128)
    u = np.zeros(3)
    J = C.c_double()
    # NULL basis, nparam < 1 (both before any device work)
    assert lib.rsg_control_optimize_basis(H._h, None, None, 4, 0.05, 1, 1, 3, None, u.ctypes.data_as(C.c_void_p),
                                          None, 50, 5, 1e-8, C.byref(J), None, None, None, None) == -1
    assert lib.rsg_control_optimize_basis(H._h, None, None, 4, 0.05, 1, 1, 0, B.ctypes.data_as(C.c_void_p),
                                          u.ctypes.data_as(C.c_void_p), None, 50, 5, 1e-8, C.byref(J), None, None,
                                          None, None) == -1


def test_raw_projector_argument_errors(lib):
    """rsg_projectors_set_raw validates everything before any device work."""
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex128)

    def call(pts, vals, nproj, hm):
        npts = np.array([len(pts)], dtype=np.int64)
        pi = np.asarray(pts, dtype=np.int64)
        pv = np.asarray(vals, dtype=np.float64).ravel()
        npj = np.array([nproj], dtype=np.int32)
        hf = np.asarray(hm, dtype=np.float64).ravel()
        return lib.rsg_projectors_set_raw(H._h, 1, npts.ctypes.data_as(C.c_void_p), pi.ctypes.data_as(C.c_void_p),
                                          npj.ctypes.data_as(C.c_void_p), pv.ctypes.data_as(C.c_void_p),
                                          hf.ctypes.data_as(C.c_void_p))

    assert lib.rsg_projectors_set_raw(H._h, 1, None, None, None, None, None) == -1
    assert call([0, 1, 1], np.ones(3), 1, [1.0]) == -1
    assert b"twice" in lib.rsg_last_error()
    assert call([0, m.P], np.ones(2), 1, [1.0]) == -1
    assert b"outside" in lib.rsg_last_error()
    assert call([0, 1], np.ones(20), 10, np.eye(10)) == -4
    assert call([0, 1], np.ones(4), 2, [[1.0, 0.5], [0.4, 1.0]]) == -1
    assert b"symmetric" in lib.rsg_last_error()
    assert call([0, 1], [1.0, np.inf], 1, [1.0]) == -1
    assert call([0, 1], np.ones(2), 0, [1.0]) == -1
    assert lib.rsg_projectors_set_raw(H._h, 0, None, None, None, None, None) == 0


def test_failure_path_support_arguments(lib):
    """rsg_selftest_bounded_wait and rsg_debug_fail_allocations reject bad
    arguments before any device work; a simulated allocation failure is
    reported as RSG_ERR_OOM by the call that allocates (here the potential
    upload), and it is consumed."""
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex64)
    assert lib.rsg_selftest_bounded_wait(None, 10, None) == -1
    assert lib.rsg_selftest_bounded_wait(H._h, 0, None) == -1
    assert lib.rsg_selftest_bounded_wait(H._h, 65537, None) == -1
    assert lib.rsg_debug_fail_allocations(-1) == -1
    V = np.zeros(m.P)
    assert lib.rsg_debug_fail_allocations(1) == 0
    assert lib.rsg_potential_set(H._h, V.ctypes.data_as(C.c_void_p), 0) == -2
    assert b"memory" in lib.rsg_last_error().lower()
    assert lib.rsg_debug_fail_allocations(0) == 0


def test_mesh_boundary_rule(lib):
    """Image walls are for cubes and boxes; the rule is validated on the host."""
    sph = rsg.Mesh(rsg.SPHERE, radius=1.0, spacing=0.3)
    assert lib.rsg_mesh_set_boundary(sph._h, rsg.BC_ODD) == -4
    cube = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    assert lib.rsg_mesh_set_boundary(cube._h, 2) == -1
    assert lib.rsg_mesh_set_boundary(None, 0) == -1
    assert lib.rsg_mesh_set_boundary(cube._h, rsg.BC_ODD) == 0
    assert lib.rsg_mesh_set_boundary(cube._h, rsg.BC_ZERO) == 0


def test_log_level(lib):
    """Errors go to stderr at level >= 1 (RSG_LOG_LEVEL or rsg_set_log_level);
    the default level is silent."""
    import subprocess
    import sys
    code = ("import paper_1501_05654_gb300 as rsg; L = rsg.load(); "
            "L.rsg_mesh_set_boundary(None, 0)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RSG_LOG_LEVEL="1", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "rsg: error -1: NULL mesh" in r.stderr, r.stderr
    env["RSG_LOG_LEVEL"] = "0"
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "rsg:" not in r.stderr, r.stderr
    assert lib.rsg_set_log_level(3) == -1
    assert lib.rsg_set_log_level(0) == 0


def test_image_walls_refused_on_short_axes():
    """Image walls reflect a neighbour once, which reaches every neighbour's
    image only with at least 4 points along each axis: shorter boxes are
    refused by the library and by the oracle; 4 points are accepted."""
    import oracle
    lib = rsg.load()
    for n in ((3, 8, 8), (8, 2, 8), (8, 8, 1)):
        m = rsg.Mesh(rsg.BOX, n, spacing=0.3)
        assert lib.rsg_mesh_set_boundary(m._h, rsg.BC_ODD) == -1
        with pytest.raises(ValueError):
            oracle.Mesh(oracle.BOX, n, h=0.3, bc=oracle.ODD)
        assert lib.rsg_mesh_set_boundary(m._h, rsg.BC_ZERO) == 0
    m = rsg.Mesh(rsg.BOX, (4, 4, 4), spacing=0.3)
    assert lib.rsg_mesh_set_boundary(m._h, rsg.BC_ODD) == 0
    assert oracle.Mesh(oracle.BOX, (4, 4, 4), h=0.3, bc=oracle.ODD).P == 64


def test_batch_entry_points_argument_errors(lib):
    """Host-side checks of the batch calls, before any device work (no GPU
    needed): NULL handles and arguments, and batches of unsupported systems."""
    v = C.c_int64()
    ms = C.c_double()
    assert lib.rsg_batch_set_option(None, b"zseg", 64) == -1
    assert lib.rsg_batch_get_option(None, b"zseg", C.byref(v)) == -1
    assert lib.rsg_batch_autotune(None, None, 0.02, 1, None, C.byref(ms)) == -1
    assert lib.rsg_batch_propagate(None, None, 1, 0.02, 1, 0, None) == -1
    assert lib.rsg_batch_create(None, None, 0, None) == -1
    m = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(m, torch.complex128)
    arr = (C.c_void_p * 1)(H._h.value)
    S = np.ones(1, dtype=np.int64)
    b = C.c_void_p()
    # complex128 systems are refused before any allocation
    assert lib.rsg_batch_create(arr, S.ctypes.data_as(C.c_void_p), 1, C.byref(b)) == -4
    assert b"complex64" in lib.rsg_last_error()
    H2 = rsg.Hamiltonian(m)
    arr2 = (C.c_void_p * 1)(H2._h.value)
    S0 = np.zeros(1, dtype=np.int64)
    assert lib.rsg_batch_create(arr2, S0.ctypes.data_as(C.c_void_p), 1, C.byref(b)) == -1

"""FP64 CPU oracle (plain C, OpenMP `parallel for`) and its ctypes wrapper.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The CUDA library never
imports, links or calls anything here, and nothing here imports the library.

Functions map one-to-one onto ``rsg_oracle.c``; see that file for the method
passages each step follows.  Arrays are numpy, complex128 for states with
shape (P, S) (states fastest) in the ORACLE's point order (x-major), which
differs from the CUDA library's on purpose: callers match points by lattice
coordinates.

Parity pins: every function here is pinned by tests in
``tests/test_oracle_*.py`` against closed forms, library routines (LAPACK
eigh, scipy expm, numpy QR/FFT), brute force and the paper's printed
one-dimensional lithium table.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CUBE, SPHERE, BOX = 0, 1, 2
ZERO, ODD = 0, 1
EXPMID, ETRS = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = C.CDLL(_LIB)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        P = C.POINTER
        L.orc_mesh_new.restype = vp
        L.orc_mesh_new.argtypes = [C.c_int, P(i32), dbl, dbl, C.c_int]
        L.orc_mesh_npoints.restype = i64
        L.orc_mesh_npoints.argtypes = [vp]
        L.orc_mesh_ijk.argtypes = [vp, vp]
        L.orc_mesh_xyz.argtypes = [vp, vp]
        L.orc_mesh_free.argtypes = [vp]
        L.orc_ham_new.restype = vp
        L.orc_ham_new.argtypes = [vp, vp]
        L.orc_ham_free.argtypes = [vp]
        L.orc_ham_set_projectors.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
        L.orc_ham_set_projectors_raw.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
        L.orc_ham_atom_npoints.restype = i64
        L.orc_ham_atom_npoints.argtypes = [vp, C.c_int]
        L.orc_ham_atom_nproj.restype = C.c_int
        L.orc_ham_atom_nproj.argtypes = [vp, C.c_int]
        L.orc_ham_atom_values.argtypes = [vp, C.c_int, vp, vp]
        L.orc_apply.argtypes = [vp, dbl, vp, vp, vp, i64]
        L.orc_apply_scaled.argtypes = [vp, dbl, vp, vp, vp, i64]
        L.orc_apply_scaled_sampled.argtypes = [vp, dbl, vp, vp, i64, i64, vp, vp, vp]
        L.orc_apply_sampled.argtypes = [vp, dbl, vp, vp, i64, i64, vp, vp, vp]
        L.orc_taylor4.argtypes = [vp, dbl, vp, dbl, vp, vp, i64]
        L.orc_norms2.argtypes = [vp, vp, i64, vp]
        L.orc_taylor4_scaled.argtypes = [vp, dbl, vp, dbl, vp, vp, i64]
        L.orc_propagate_scaled.argtypes = [vp, dbl, vp, vp, i64, i64, dbl, C.c_int]
        L.orc_mgs.argtypes = [vp, vp, i64]
        L.orc_propagate.argtypes = [vp, vp, i64, i64, dbl, C.c_int, C.c_int, vp, vp,
                                    C.c_int, vp]
        L.orc_objective.restype = dbl
        L.orc_objective.argtypes = [vp, vp, vp, i64, dbl, C.c_int, C.c_int, vp, vp]
        L.orc_control_gradient.restype = dbl
        L.orc_control_gradient.argtypes = [vp, vp, vp, i64, dbl, C.c_int, C.c_int, vp, vp,
                                           C.c_int, vp]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        _lib = L
        return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


class Mesh:
    """Oracle mesh: cube (n), box (nx, ny, nz) or sphere (radius)."""

    def __init__(self, shape: int, n=(0, 0, 0), radius: float = 0.0, h: float = 0.3,
                 bc: int = ZERO):
        L = _load()
        if isinstance(n, int):
            n = (n, n, n)
        nn = (C.c_int32 * 3)(*[int(v) for v in n])
        self.h = float(h)
        self.shape = shape
        self._m = L.orc_mesh_new(int(shape), nn, float(radius), float(h), int(bc))
        if not self._m:
            raise ValueError("image walls need at least 4 points along every axis")
        self.P = int(L.orc_mesh_npoints(self._m))
        self.ijk = np.empty((self.P, 3), dtype=np.int32)
        L.orc_mesh_ijk(self._m, _p(self.ijk))
        self.xyz = np.empty((self.P, 3), dtype=np.float64)
        L.orc_mesh_xyz(self._m, _p(self.xyz))

    def __del__(self):
        if getattr(self, "_m", None) and _lib is not None:
            _lib.orc_mesh_free(self._m)
            self._m = None

    def norms2(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty(psi.shape[1])
        _load().orc_norms2(self._m, _p(psi), psi.shape[1], _p(out))
        return out

    def apply_scaled(self, psi, theta: float, vtheta):
        """Complex-scaled operator -1/2 e^{-2 i theta} lap + V(r e^{i theta})
        (vtheta: the caller's complex values of V(r e^{i theta}) per point)."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        vt = np.ascontiguousarray(vtheta, dtype=np.complex128)
        assert vt.shape == (self.P,)
        out = np.empty_like(psi)
        _load().orc_apply_scaled(self._m, float(theta), _p(vt), _p(psi), _p(out), psi.shape[1])
        return out

    def apply_scaled_sampled(self, psi, theta: float, vtheta, pidx, sidx):
        """(H_theta psi) at the (point, state) pairs (pidx[t], sidx[t])."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        vt = np.ascontiguousarray(vtheta, dtype=np.complex128)
        pidx = np.ascontiguousarray(pidx, dtype=np.int64)
        sidx = np.ascontiguousarray(sidx, dtype=np.int64)
        out = np.empty(pidx.shape[0], dtype=np.complex128)
        _load().orc_apply_scaled_sampled(self._m, float(theta), _p(vt), _p(psi), psi.shape[1], pidx.shape[0],
                                         _p(pidx), _p(sidx), _p(out))
        return out

    def taylor4_scaled(self, psi, theta: float, vtheta, tau: float):
        """sum_{n<=4} (-i tau H_theta)^n psi / n! by explicit terms."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        vt = np.ascontiguousarray(vtheta, dtype=np.complex128)
        out = np.empty_like(psi)
        _load().orc_taylor4_scaled(self._m, float(theta), _p(vt), float(tau), _p(psi), _p(out), psi.shape[1])
        return out

    def propagate_scaled(self, psi, theta: float, vtheta, nsteps: int, dt: float, scheme: int = 0):
        """nsteps steps of dt with H_theta (exponential midpoint, or ETRS)."""
        psi = np.array(psi, dtype=np.complex128, order="C", copy=True)
        vt = np.ascontiguousarray(vtheta, dtype=np.complex128)
        _load().orc_propagate_scaled(self._m, float(theta), _p(vt), _p(psi), psi.shape[1], int(nsteps),
                                     float(dt), int(scheme))
        return psi

    def mgs(self, psi):
        psi = np.array(psi, dtype=np.complex128, order="C", copy=True)
        _load().orc_mgs(self._m, _p(psi), psi.shape[1])
        return psi


class Hamiltonian:
    """Oracle H = -1/2 lap + V + eps dir.r + sum_a |p_a> h_a <p_a|."""

    def __init__(self, mesh: Mesh, V):
        self.mesh = mesh
        V = np.ascontiguousarray(V, dtype=np.float64)
        assert V.shape == (mesh.P,)
        self._h = _load().orc_ham_new(mesh._m, _p(V))
        self.natoms = 0

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_ham_free(self._h)
            self._h = None

    def set_projectors(self, centres, rcut, lmax, beta, hmats):
        centres = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        n = centres.shape[0]
        rcut = np.ascontiguousarray(rcut, dtype=np.float64)
        lmax = np.ascontiguousarray(lmax, dtype=np.int32)
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        hflat = np.ascontiguousarray(np.concatenate([np.asarray(h, dtype=np.float64).ravel()
                                                     for h in hmats]) if n else np.zeros(1))
        _load().orc_ham_set_projectors(self._h, n, _p(centres), _p(rcut), _p(lmax), _p(beta),
                                       _p(hflat))
        self.natoms = n

    def set_projectors_raw(self, points, values, hmats):
        """Projectors as sampled values: per atom the point indices (n_a,),
        values (n_a, nproj_a) and the matrix h_a (orc_ham_set_projectors_raw)."""
        n = len(points)
        npts = np.array([len(p) for p in points], dtype=np.int64)
        vals = [np.asarray(v, dtype=np.float64).reshape(len(p), -1) for p, v in zip(points, values)]
        nproj = np.array([v.shape[1] for v in vals], dtype=np.int32)
        pidx = np.ascontiguousarray(np.concatenate([np.asarray(p, np.int64) for p in points]) if n
                                    else np.zeros(1, np.int64))
        pv = np.ascontiguousarray(np.concatenate([v.ravel() for v in vals]) if n else np.zeros(1))
        hflat = np.ascontiguousarray(np.concatenate([np.asarray(h, dtype=np.float64).ravel() for h in hmats])
                                     if n else np.zeros(1))
        _load().orc_ham_set_projectors_raw(self._h, n, _p(npts), _p(pidx), _p(nproj), _p(pv), _p(hflat))
        self.natoms = n

    def atom(self, a: int):
        L = _load()
        n = int(L.orc_ham_atom_npoints(self._h, a))
        k = int(L.orc_ham_atom_nproj(self._h, a))
        pts = np.empty(n, dtype=np.int64)
        vals = np.empty((k, n), dtype=np.float64)
        L.orc_ham_atom_values(self._h, a, _p(pts), _p(vals))
        return pts, vals

    @staticmethod
    def _dir(d):
        return None if d is None else np.ascontiguousarray(d, dtype=np.float64)

    def apply(self, psi, eps: float = 0.0, dir=None):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(psi)
        d = self._dir(dir)
        _load().orc_apply(self._h, float(eps), _p(d), _p(psi), _p(out), psi.shape[1])
        return out

    def apply_sampled(self, psi, pidx, sidx, eps: float = 0.0, dir=None):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        pidx = np.ascontiguousarray(pidx, dtype=np.int64)
        sidx = np.ascontiguousarray(sidx, dtype=np.int64)
        out = np.empty(pidx.shape[0], dtype=np.complex128)
        d = self._dir(dir)
        _load().orc_apply_sampled(self._h, float(eps), _p(d), _p(psi), psi.shape[1],
                                  pidx.shape[0], _p(pidx), _p(sidx), _p(out))
        return out

    def taylor4(self, psi, tau: float, eps: float = 0.0, dir=None):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(psi)
        d = self._dir(dir)
        _load().orc_taylor4(self._h, float(eps), _p(d), float(tau), _p(psi), _p(out),
                            psi.shape[1])
        return out

    def propagate(self, psi, nsteps: int, dt: float, scheme: int = EXPMID, nsub: int = 1,
                  eps=None, dir=None, gs_every: int = 0):
        psi = np.array(psi, dtype=np.complex128, order="C", copy=True)
        S = psi.shape[1]
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        d = self._dir(dir)
        drift = np.zeros(S)
        _load().orc_propagate(self._h, _p(psi), S, int(nsteps), float(dt), int(scheme),
                              int(nsub), _p(e), _p(d), int(gs_every), _p(drift))
        return psi, drift

    def propagate_masked(self, psi, nsteps: int, dt: float, mask, scheme: int = EXPMID):
        """nsteps steps, each followed by the pointwise product with the mask
        M(r): the bounded part M psi of the mask split (Sec. "Photoemission",
        Eq. (mask_split)) is kept after every step."""
        mask = np.asarray(mask, dtype=np.float64)
        for _ in range(int(nsteps)):
            psi, _ = self.propagate(psi, 1, dt, scheme=scheme)
            psi = psi * mask[:, None]
        return psi

    def objective(self, psi0, target, eps, dt: float, scheme: int = ETRS, nsub: int = 1,
                  dir=(1.0, 0.0, 0.0)):
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128).reshape(-1)
        target = np.ascontiguousarray(target, dtype=np.complex128).reshape(-1)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        d = self._dir(dir)
        return float(_load().orc_objective(self._h, _p(psi0), _p(target), eps.shape[0],
                                           float(dt), int(scheme), int(nsub), _p(eps), _p(d)))

    def control_gradient(self, psi0, target, eps, dt: float, scheme: int = ETRS,
                         nsub: int = 1, dir=(1.0, 0.0, 0.0), checkpoint_every: int = 50):
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128).reshape(-1)
        target = np.ascontiguousarray(target, dtype=np.complex128).reshape(-1)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        d = self._dir(dir)
        g = np.empty(eps.shape[0])
        J = _load().orc_control_gradient(self._h, _p(psi0), _p(target), eps.shape[0],
                                         float(dt), int(scheme), int(nsub), _p(eps), _p(d),
                                         int(checkpoint_every), _p(g))
        return float(J), g

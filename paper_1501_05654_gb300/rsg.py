"""Thin ctypes binding over librsg.so (include/rsg.h).

Argument marshalling only: every step of the Hamiltonian application,
propagation, re-orthonormalisation and adjoint gradient runs in the CUDA
library.  PyTorch supplies device memory and the current CUDA stream.  There
is no CPU fallback: if the library is missing or fails to load, importing
this module's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsg.so")

CUBE, SPHERE, BOX = 0, 1, 2
C64, C128 = 0, 1
EXPMID, ETRS = 0, 1
BC_ZERO, BC_ODD = 0, 1

_STATUS = {0: "RSG_OK", -1: "RSG_ERR_ARG", -2: "RSG_ERR_OOM", -3: "RSG_ERR_CUDA",
           -4: "RSG_ERR_UNSUPPORTED", -5: "RSG_ERR_TIMEOUT", -6: "RSG_ERR_NONFINITE",
           -7: "RSG_ERR_STATE"}

# Every entry point of include/rsg.h with its ctypes signature.
_vp, _i64, _i32, _dbl, _int = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_int
SIGNATURES = {
    "rsg_mesh_create": [_int, _vp, _dbl, _dbl, _vp],
    "rsg_mesh_num_points": [_vp, _vp],
    "rsg_mesh_coords": [_vp, _vp],
    "rsg_mesh_geometry": [_vp, _vp, _vp],
    "rsg_mesh_destroy": [_vp],
    "rsg_ham_create": [_vp, _int, _vp],
    "rsg_ham_destroy": [_vp],
    "rsg_potential_set": [_vp, _vp, _int],
    "rsg_projectors_set": [_vp, _int, _vp, _vp, _vp, _vp, _vp],
    "rsg_field_set": [_vp, _dbl, _vp],
    "rsg_hamiltonian_apply": [_vp, _vp, _vp, _i64, _i64, _vp],
    "rsg_taylor_apply": [_vp, _vp, _vp, _i64, _i64, _dbl, _vp],
    "rsg_propagate_steps": [_vp, _vp, _i64, _i64, _i64, _dbl, _int, _int, _vp, _vp, _int, _vp, _vp],
    "rsg_orthonormalize": [_vp, _vp, _i64, _i64, _vp, _vp],
    "rsg_absorber_set": [_vp, _vp, _int],
    "rsg_states_save": [_vp, C.c_char_p, _vp, _i64, _i64, _int, _i64, _dbl, C.c_uint64],
    "rsg_states_load": [_vp, C.c_char_p, _vp, _i64, _i64, _int, _vp, _vp, _vp],
    "rsg_mesh_set_boundary": [_vp, _int],
    "rsg_projectors_set_raw": [_vp, _int, _vp, _vp, _vp, _vp, _vp],
    "rsg_complex_scaling_set": [_vp, _dbl, _vp, _int],
    "rsg_shifted_solve": [_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _i64, _dbl, _vp, _vp, _vp],
    "rsg_eigensolve": [_vp, _vp, _i64, _i64, _i64, _i64, _int, _dbl, _vp, _vp, _vp, _vp],
    "rsg_state_norms": [_vp, _vp, _i64, _i64, _vp, _vp],
    "rsg_state_norms_noalloc": [_vp, _vp, _i64, _i64, _vp, _vp],
    "rsg_control_gradient": [_vp, _vp, _vp, _i64, _dbl, _int, _int, _vp, _vp, _int, _vp, _vp, _vp],
    "rsg_control_optimize": [_vp, _vp, _vp, _i64, _dbl, _int, _int, _vp, _vp, _int, _i64, _dbl, _vp, _vp, _vp,
                             _vp, _vp],
    "rsg_control_optimize_basis": [_vp, _vp, _vp, _i64, _dbl, _int, _int, _i64, _vp, _vp, _vp, _int, _i64, _dbl,
                                   _vp, _vp, _vp, _vp, _vp],
    "rsg_fourier_basis": [_i64, _i64, _vp],
    "rsg_batch_create": [_vp, _vp, _int, _vp],
    "rsg_batch_propagate": [_vp, _vp, _i64, _dbl, _int, _int, _vp],
    "rsg_batch_destroy": [_vp],
    "rsg_batch_set_option": [_vp, C.c_char_p, _i64],
    "rsg_batch_get_option": [_vp, C.c_char_p, _vp],
    "rsg_batch_autotune": [_vp, _vp, _dbl, _int, _vp, _vp],
    "rsg_ham_set_option": [_vp, C.c_char_p, _i64],
    "rsg_ham_get_option": [_vp, C.c_char_p, _vp],
    "rsg_ham_autotune": [_vp, _vp, _vp, _i64, _i64, _vp, _vp],
    "rsg_ham_profile": [_vp, _int],
    "rsg_ham_kernel_stats": [_vp, _vp, _vp, _vp, _vp],
    "rsg_selftest_bounded_wait": [_vp, _int, _vp],
    "rsg_debug_fail_allocations": [_int],
    "rsg_set_log_level": [_int],
    "rsg_last_error": [],
}

_lock = threading.Lock()
_lib = None


class RSGError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Load librsg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"librsg.so is not built ({path}); run "
                              "paper_1501_05654_gb300.build.build() first")
        L = C.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "rsg_last_error" else C.c_int
        _lib = L
        return L


def _ck(status: int):
    if status != 0:
        msg = load().rsg_last_error().decode(errors="replace")
        raise RSGError(f"{_STATUS.get(status, status)}: {msg}")


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def padded_ld(S: int, dtype) -> int:
    """Leading dimension for S states: even for complex64 (16-byte rows)."""
    return S + (S % 2) if dtype == torch.complex64 else S


def empty_states(P: int, S: int, dtype=torch.complex64, device="cuda"):
    """Zero-filled (P, ld) state block with ld = padded_ld(S)."""
    return torch.zeros((P, padded_ld(S, dtype)), dtype=dtype, device=device)


class Mesh:
    """rsg_mesh: CUBE(n), BOX((nx,ny,nz)) or SPHERE(radius) at spacing h."""

    def __init__(self, shape: int, n=0, radius: float = 0.0, spacing: float = 0.3):
        L = load()
        if isinstance(n, int):
            n = (n, n, n)
        nn = (C.c_int32 * 3)(*[int(v) for v in n])
        h = C.c_void_p()
        _ck(L.rsg_mesh_create(int(shape), nn, float(radius), float(spacing), C.byref(h)))
        self._h = h
        P = C.c_int64()
        _ck(L.rsg_mesh_num_points(self._h, C.byref(P)))
        self.P = int(P.value)
        self.ijk = np.empty((self.P, 3), dtype=np.int32)
        _ck(L.rsg_mesh_coords(self._h, _ptr(self.ijk)))
        org = np.zeros(3)
        sp = C.c_double()
        _ck(L.rsg_mesh_geometry(self._h, _ptr(org), C.byref(sp)))
        self.origin = org
        self.h = float(sp.value)
        self.xyz = org[None, :] + self.h * self.ijk.astype(np.float64)

    def set_boundary(self, bc: int):
        """BC_ZERO (zero values outside the mesh) or BC_ODD (antisymmetric
        images about walls one spacing outside a cube or box)."""
        _ck(load().rsg_mesh_set_boundary(self._h, int(bc)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsg_mesh_destroy(self._h)
            self._h = None


class Hamiltonian:
    """rsg_ham bound to a mesh and a compute type (complex64 or complex128)."""

    def __init__(self, mesh: Mesh, dtype=torch.complex64):
        L = load()
        self.mesh = mesh
        self.dtype = dtype
        self._code = C64 if dtype == torch.complex64 else C128
        h = C.c_void_p()
        _ck(L.rsg_ham_create(mesh._h, self._code, C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsg_ham_destroy(self._h)
            self._h = None

    # -- set-up
    def set_potential(self, V):
        if isinstance(V, torch.Tensor) and V.is_cuda:
            V = V.to(torch.float64).contiguous()
            _ck(load().rsg_potential_set(self._h, C.c_void_p(V.data_ptr()), 1))
        else:
            V = _np(V if not isinstance(V, torch.Tensor) else V.numpy(), np.float64)
            _ck(load().rsg_potential_set(self._h, _ptr(V), 0))

    def set_projectors(self, centres, rcut, lmax, beta, hmats):
        centres = _np(centres, np.float64).reshape(-1, 3)
        n = centres.shape[0]
        rcut, beta = _np(rcut, np.float64), _np(beta, np.float64)
        lmax = _np(lmax, np.int32)
        hflat = _np(np.concatenate([np.asarray(h, np.float64).ravel() for h in hmats])
                    if n else np.zeros(1), np.float64)
        _ck(load().rsg_projectors_set(self._h, n, _ptr(centres), _ptr(rcut), _ptr(lmax),
                                      _ptr(beta), _ptr(hflat)))

    def set_projectors_raw(self, points, values, hmats):
        """Projectors as sampled values (rsg_projectors_set_raw): per atom a
        list of library point indices (n_a,), values of shape (n_a, nproj_a)
        and the nproj_a x nproj_a matrix h_a."""
        n = len(points)
        if not (len(values) == n and len(hmats) == n):
            raise ValueError("points, values and hmats: one entry per atom")
        npts = np.array([len(p) for p in points], dtype=np.int64)
        vals = [np.asarray(v, np.float64).reshape(len(p), -1) for p, v in zip(points, values)]
        nproj = np.array([v.shape[1] for v in vals], dtype=np.int32)
        pidx = _np(np.concatenate([np.asarray(p, np.int64) for p in points]) if n else np.zeros(1), np.int64)
        pv = _np(np.concatenate([v.ravel() for v in vals]) if n else np.zeros(1), np.float64)
        hflat = _np(np.concatenate([np.asarray(h, np.float64).ravel() for h in hmats]) if n else np.zeros(1),
                    np.float64)
        _ck(load().rsg_projectors_set_raw(self._h, n, _ptr(npts), _ptr(pidx), _ptr(nproj), _ptr(pv),
                                          _ptr(hflat)))

    def set_field(self, eps: float, dir=(1.0, 0.0, 0.0)):
        d = _np(dir, np.float64)
        _ck(load().rsg_field_set(self._h, float(eps), _ptr(d)))

    def set_absorber(self, mask):
        """Mask absorber M (P values in [0, 1], library point order) applied
        after every time step; None removes it (rsg_absorber_set)."""
        if mask is None:
            _ck(load().rsg_absorber_set(self._h, None, 0))
        elif isinstance(mask, torch.Tensor) and mask.is_cuda:
            m = mask.to(torch.float64).contiguous()
            _ck(load().rsg_absorber_set(self._h, C.c_void_p(m.data_ptr()), 1))
        else:
            m = _np(mask if not isinstance(mask, torch.Tensor) else mask.numpy(), np.float64)
            _ck(load().rsg_absorber_set(self._h, _ptr(m), 0))

    def set_complex_scaling(self, theta, v_theta):
        """Complex scaling: from now on H is -1/2 e^{-2i theta} lap + v_theta,
        v_theta the P complex values v(r e^{i theta}) in library point order;
        v_theta None removes it (rsg_complex_scaling_set)."""
        if v_theta is None:
            _ck(load().rsg_complex_scaling_set(self._h, float(theta), None, 0))
        elif isinstance(v_theta, torch.Tensor) and v_theta.is_cuda:
            v = torch.view_as_real(v_theta.to(torch.complex128).contiguous()).contiguous()
            _ck(load().rsg_complex_scaling_set(self._h, float(theta), C.c_void_p(v.data_ptr()), 1))
        else:
            a = v_theta.numpy() if isinstance(v_theta, torch.Tensor) else np.asarray(v_theta)
            v = np.ascontiguousarray(a.astype(np.complex128)).view(np.float64)
            _ck(load().rsg_complex_scaling_set(self._h, float(theta), _ptr(v), 0))

    def save_states(self, path, psi, S=None, step: int = 0, time: float = 0.0, seed: int = 0):
        """Write the S live columns of psi (cuda tensor or host array of
        shape (P, ld)) to path (.npy) and its metadata to path.json."""
        dev = isinstance(psi, torch.Tensor) and psi.is_cuda
        if dev:
            self._check(psi)
            ptr, ld = C.c_void_p(psi.data_ptr()), psi.shape[1]
        else:
            a = psi.numpy() if isinstance(psi, torch.Tensor) else psi
            a = np.ascontiguousarray(a, dtype=np.complex64 if self.dtype == torch.complex64 else np.complex128)
            ptr, ld = _ptr(a), a.shape[1]
        S = ld if S is None else S
        _ck(load().rsg_states_save(self._h, os.fsencode(str(path)), ptr, S, ld, int(dev), int(step), float(time),
                                   int(seed)))

    def load_states(self, path, psi, S=None):
        """Read path into psi (cuda tensor, or a writable C-contiguous host
        array of shape (P, ld)); returns (step, time, seed)."""
        dev = isinstance(psi, torch.Tensor) and psi.is_cuda
        if dev:
            self._check(psi)
            ptr, ld = C.c_void_p(psi.data_ptr()), psi.shape[1]
        else:
            a = psi.numpy() if isinstance(psi, torch.Tensor) else psi
            want = np.complex64 if self.dtype == torch.complex64 else np.complex128
            if not (a.dtype == want and a.flags.c_contiguous and a.flags.writeable and a.ndim == 2):
                raise ValueError("psi: writable C-contiguous (P, ld) array of the Hamiltonian's dtype")
            ptr, ld = _ptr(a), a.shape[1]
        S = ld if S is None else S
        st, t, sd = C.c_int64(), C.c_double(), C.c_uint64()
        _ck(load().rsg_states_load(self._h, os.fsencode(str(path)), ptr, S, ld, int(dev), C.byref(st), C.byref(t),
                                   C.byref(sd)))
        return int(st.value), float(t.value), int(sd.value)

    def set_option(self, key: str, value: int):
        _ck(load().rsg_ham_set_option(self._h, key.encode(), int(value)))

    def get_option(self, key: str) -> int:
        v = C.c_int64()
        _ck(load().rsg_ham_get_option(self._h, key.encode(), C.byref(v)))
        return int(v.value)

    TUNED_KEYS = ("kernel", "threads", "cv", "stages", "zseg", "blocks_per_sm", "wide_ty", "producers")

    def autotune(self, psi, S=None, cache_path=None, stream=None):
        """Choose the fastest stencil configuration for this mesh and block.

        With cache_path (a JSON file), a configuration tuned earlier for the
        same mesh size, state count, leading dimension and dtype is reused
        without timing, and new results are added to the file.
        """
        import json
        self._check(psi)
        S = psi.shape[1] if S is None else S
        key = f"{self.mesh.P}:{self.mesh.h:.6g}:{S}:{psi.shape[1]}:{self.dtype}"
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                for k in self.TUNED_KEYS:
                    self.set_option(k, cache[key][k])
                return cache[key]
        work = torch.empty_like(psi)
        best = C.c_double()
        _ck(load().rsg_ham_autotune(self._h, C.c_void_p(psi.data_ptr()), C.c_void_p(work.data_ptr()), S,
                                    psi.shape[1], _stream(stream), C.byref(best)))
        res = {k: self.get_option(k) for k in self.TUNED_KEYS}
        res["stage_ms"] = float(best.value)
        if cache_path:
            cache[key] = res
            tmp = cache_path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, cache_path)
        return res

    def profile(self, enable: bool):
        _ck(load().rsg_ham_profile(self._h, 1 if enable else 0))

    def kernel_stats(self):
        """(stencil ms, stencil launches, stencil algorithmic bytes, all launches)."""
        ms, nb = C.c_double(), C.c_double()
        nk, na = C.c_int64(), C.c_int64()
        _ck(load().rsg_ham_kernel_stats(self._h, C.byref(ms), C.byref(nk), C.byref(nb),
                                        C.byref(na)))
        return float(ms.value), int(nk.value), float(nb.value), int(na.value)

    # -- operations
    def _check(self, psi):
        if not (isinstance(psi, torch.Tensor) and psi.is_cuda and psi.dtype == self.dtype
                and psi.dim() == 2 and psi.shape[0] == self.mesh.P and psi.is_contiguous()):
            raise ValueError(f"expected a contiguous cuda {self.dtype} tensor of shape "
                             f"({self.mesh.P}, ld)")

    def apply(self, psi, out=None, S=None, stream=None):
        """out = H psi (device blocks of shape (P, ld))."""
        self._check(psi)
        if out is None:
            out = torch.empty_like(psi)
        self._check(out)
        S = psi.shape[1] if S is None else S
        _ck(load().rsg_hamiltonian_apply(self._h, C.c_void_p(psi.data_ptr()),
                                         C.c_void_p(out.data_ptr()), S, psi.shape[1],
                                         _stream(stream)))
        return out

    def taylor(self, psi, tau: float, out=None, S=None, stream=None):
        """out = T(tau) psi (Taylor-4 exponential); out may be psi."""
        self._check(psi)
        if out is None:
            out = torch.empty_like(psi)
        self._check(out)
        S = psi.shape[1] if S is None else S
        _ck(load().rsg_taylor_apply(self._h, C.c_void_p(psi.data_ptr()),
                                    C.c_void_p(out.data_ptr()), S, psi.shape[1], float(tau),
                                    _stream(stream)))
        return out

    def propagate(self, psi, nsteps: int, dt: float, scheme: int = ETRS, nsub: int = 1,
                  eps=None, dir=(1.0, 0.0, 0.0), gs_every: int = 0, S=None, stream=None,
                  want_drift: bool = True):
        """Propagates psi in place; returns the per-state norm drift (numpy) or None."""
        self._check(psi)
        S = psi.shape[1] if S is None else S
        e = None if eps is None else _np(eps, np.float64)
        d = _np(dir, np.float64)
        drift = np.zeros(S) if want_drift else None
        _ck(load().rsg_propagate_steps(self._h, C.c_void_p(psi.data_ptr()), S, psi.shape[1],
                                       int(nsteps), float(dt), int(scheme), int(nsub),
                                       None if e is None else _ptr(e), _ptr(d), int(gs_every),
                                       None if drift is None else _ptr(drift), _stream(stream)))
        return drift

    def eigensolve(self, psi, nwant=None, max_iter: int = 200, degree: int = 10, tol: float = 1e-8, S=None,
                   stream=None):
        """Lowest eigenpairs (rsg_eigensolve): psi (in, starting block of S
        states; out, Ritz vectors); the nwant lowest (default S) must reach
        tol.  Returns (eigenvalues, residual norms, iterations) for all S."""
        self._check(psi)
        S = psi.shape[1] if S is None else S
        nwant = S if nwant is None else nwant
        ev, res = np.zeros(S), np.zeros(S)
        it = C.c_int64()
        _ck(load().rsg_eigensolve(self._h, C.c_void_p(psi.data_ptr()), S, psi.shape[1], int(nwant), int(max_iter),
                                  int(degree), float(tol), _ptr(ev), _ptr(res), C.byref(it), _stream(stream)))
        return ev, res, int(it.value)

    def shifted_solve(self, b, x, z: complex, max_iter: int = 500, tol: float = 1e-10, S=None, stream=None):
        """Solve (H - z) x = b (rsg_shifted_solve); x holds the initial guess
        and receives the solution.  Returns (relative residuals, iterations)."""
        self._check(b)
        self._check(x)
        S = b.shape[1] if S is None else S
        res = np.zeros(S)
        it = C.c_int64()
        z = complex(z)
        _ck(load().rsg_shifted_solve(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), S, b.shape[1],
                                     z.real, z.imag, int(max_iter), float(tol), _ptr(res), C.byref(it),
                                     _stream(stream)))
        return res, int(it.value)

    def orthonormalize(self, psi, S=None, stream=None):
        self._check(psi)
        S = psi.shape[1] if S is None else S
        n2 = np.zeros(S)
        _ck(load().rsg_orthonormalize(self._h, C.c_void_p(psi.data_ptr()), S, psi.shape[1],
                                      _ptr(n2), _stream(stream)))
        return n2

    def norms(self, psi, S=None, stream=None):
        self._check(psi)
        S = psi.shape[1] if S is None else S
        n2 = np.zeros(S)
        _ck(load().rsg_state_norms(self._h, C.c_void_p(psi.data_ptr()), S, psi.shape[1],
                                   _ptr(n2), _stream(stream)))
        return n2

    def control_gradient(self, psi0, target, eps, dt: float, scheme: int = ETRS, nsub: int = 1,
                         dir=(1.0, 0.0, 0.0), checkpoint_every: int = 50, stream=None):
        """J = |<target|psi(T)>|^2 and dJ/d eps_k (numpy) for one state."""
        for t in (psi0, target):
            if not (t.is_cuda and t.dtype == self.dtype and t.numel() == self.mesh.P
                    and t.is_contiguous()):
                raise ValueError("psi0/target: contiguous cuda vectors of P values")
        e = _np(eps, np.float64)
        d = _np(dir, np.float64)
        g = np.zeros(e.shape[0])
        J = C.c_double()
        _ck(load().rsg_control_gradient(self._h, C.c_void_p(psi0.data_ptr()),
                                        C.c_void_p(target.data_ptr()), e.shape[0], float(dt),
                                        int(scheme), int(nsub), _ptr(e), _ptr(d),
                                        int(checkpoint_every), C.byref(J), _ptr(g),
                                        _stream(stream)))
        return float(J.value), g

    def control_optimize(self, psi0, target, eps, dt: float, scheme: int = ETRS, nsub: int = 1,
                         dir=(1.0, 0.0, 0.0), checkpoint_every: int = 50, max_iter: int = 50,
                         gtol: float = 1e-8, stream=None):
        """Maximise J over the control (rsg_control_optimize).  Returns
        (eps (numpy, the best field), J, J history, accepted steps, evaluations)."""
        for t in (psi0, target):
            if not (t.is_cuda and t.dtype == self.dtype and t.numel() == self.mesh.P
                    and t.is_contiguous()):
                raise ValueError("psi0/target: contiguous cuda vectors of P values")
        e = _np(eps, np.float64).copy()
        d = _np(dir, np.float64)
        hist = np.zeros(int(max_iter) + 1)
        J = C.c_double()
        it, ev = C.c_int64(), C.c_int64()
        _ck(load().rsg_control_optimize(self._h, C.c_void_p(psi0.data_ptr()), C.c_void_p(target.data_ptr()),
                                        e.shape[0], float(dt), int(scheme), int(nsub), _ptr(e), _ptr(d),
                                        int(checkpoint_every), int(max_iter), float(gtol), C.byref(J),
                                        _ptr(hist), C.byref(it), C.byref(ev), _stream(stream)))
        return e, float(J.value), hist[:it.value + 1], int(it.value), int(ev.value)

    def control_optimize_basis(self, psi0, target, basis, u, dt: float, scheme: int = ETRS, nsub: int = 1,
                               dir=(1.0, 0.0, 0.0), checkpoint_every: int = 50, max_iter: int = 50,
                               gtol: float = 1e-8, stream=None):
        """Maximise J over the coefficients u of eps = basis @ u
        (rsg_control_optimize_basis; basis of shape (nsteps, nparam)).
        Returns (u (numpy), J, J history, accepted steps, evaluations)."""
        for t in (psi0, target):
            if not (t.is_cuda and t.dtype == self.dtype and t.numel() == self.mesh.P
                    and t.is_contiguous()):
                raise ValueError("psi0/target: contiguous cuda vectors of P values")
        B = _np(basis, np.float64)
        if B.ndim != 2:
            raise ValueError("basis: (nsteps, nparam)")
        x = _np(u, np.float64).copy()
        if x.shape != (B.shape[1],):
            raise ValueError("u: nparam values")
        d = _np(dir, np.float64)
        hist = np.zeros(int(max_iter) + 1)
        J = C.c_double()
        it, ev = C.c_int64(), C.c_int64()
        _ck(load().rsg_control_optimize_basis(self._h, C.c_void_p(psi0.data_ptr()), C.c_void_p(target.data_ptr()),
                                              B.shape[0], float(dt), int(scheme), int(nsub), B.shape[1], _ptr(B),
                                              _ptr(x), _ptr(d), int(checkpoint_every), int(max_iter), float(gtol),
                                              C.byref(J), _ptr(hist), C.byref(it), C.byref(ev), _stream(stream)))
        return x, float(J.value), hist[:it.value + 1], int(it.value), int(ev.value)


def fourier_basis(nsteps: int, nparam: int) -> np.ndarray:
    """Sine-series basis sin(m pi t / T) at the interval midpoints,
    shape (nsteps, nparam) (rsg_fourier_basis)."""
    B = np.zeros((int(nsteps), int(nparam)))
    _ck(load().rsg_fourier_basis(int(nsteps), int(nparam), _ptr(B)))
    return B


class ControlObjective(torch.autograd.Function):
    """J(eps) = |<target|psi(T; eps)>|^2 with a hand-written adjoint backward.

    forward(eps, ham, psi0, target, dt, scheme, nsub, dir, checkpoint_every)
    takes eps as a CPU float64 tensor; backward returns grad_J * dJ/d eps from
    the library's discrete adjoint (rsg_control_gradient).
    """

    @staticmethod
    def forward(ctx, eps, ham, psi0, target, dt, scheme=ETRS, nsub=1, dir=(1.0, 0.0, 0.0),
                checkpoint_every=50):
        J, g = ham.control_gradient(psi0, target, eps.detach().cpu().numpy(), dt, scheme, nsub,
                                    dir, checkpoint_every)
        ctx.save_for_backward(torch.from_numpy(g))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return (gJ * g, None, None, None, None, None, None, None, None)


class Batch:
    """rsg_batch over several complex64 Hamiltonians."""

    def __init__(self, hams, S):
        self.hams = list(hams)
        self.S = [int(s) for s in S]
        arr = (C.c_void_p * len(self.hams))(*[h._h.value for h in self.hams])
        s = np.asarray(self.S, dtype=np.int64)
        h = C.c_void_p()
        _ck(load().rsg_batch_create(arr, _ptr(s), len(self.hams), C.byref(h)))
        self._h = h
        self._keep = (arr, s)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rsg_batch_destroy(self._h)
            self._h = None

    def propagate(self, psis, nsteps: int, dt: float, scheme: int = ETRS, gs_every: int = 0,
                  stream=None):
        ptrs = (C.c_void_p * len(psis))(*[p.data_ptr() for p in psis])
        _ck(load().rsg_batch_propagate(self._h, ptrs, int(nsteps), float(dt), int(scheme),
                                       int(gs_every), _stream(stream)))

    def set_option(self, key: str, value: int):
        _ck(load().rsg_batch_set_option(self._h, key.encode(), int(value)))

    def get_option(self, key: str) -> int:
        v = C.c_int64()
        _ck(load().rsg_batch_get_option(self._h, key.encode(), C.byref(v)))
        return int(v.value)

    def autotune(self, psis, dt: float, scheme: int = ETRS, stream=None) -> float:
        """Choose launch mode, segment length and tile variants by timing
        steps on copies of psis; returns the best time per step in ms."""
        ptrs = (C.c_void_p * len(psis))(*[p.data_ptr() for p in psis])
        ms = C.c_double()
        _ck(load().rsg_batch_autotune(self._h, ptrs, float(dt), int(scheme), _stream(stream), C.byref(ms)))
        return float(ms.value)

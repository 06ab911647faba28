"""Small helpers shared by the oracle pin tests (no method arithmetic)."""
import numpy as np
import scipy.sparse.linalg as sla


def dense_h(H, P, eps=0.0, dir=None):
    """Assemble the dense matrix of the oracle operator column by column."""
    eye = np.eye(P, dtype=np.complex128)
    return H.apply(eye, eps=eps, dir=dir)   # column j = H e_j (states fastest)


def lowest_eigs(H, P, k, seed=0, tol=1e-9, ncv=None):
    op = sla.LinearOperator(
        (P, P), dtype=np.float64,
        matvec=lambda v: H.apply(np.asarray(v, dtype=np.complex128).reshape(-1, 1)).real.ravel())
    v0 = np.random.default_rng(seed).standard_normal(P)
    w = sla.eigsh(op, k=k, which="SA", tol=tol, ncv=ncv, return_eigenvectors=False, v0=v0)
    return np.sort(w)


def wdot(h, a, b):
    """h^3-weighted inner product of two vectors."""
    return h ** 3 * np.vdot(a, b)

"""GPU: the optimal-control loop (rsg_control_optimize, limited-memory BFGS
on -J with the library's discrete-adjoint gradient) on the double-well
system of the adjoint tests.  Checks that do not trust the library:
the accepted objective values never decrease; the FP64 oracle evaluates the
same J at the returned field; and the oracle's own gradient there is far
smaller than at the starting field (the loop has found a stationary point
of the oracle's objective, not of its own)."""
import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests.test_gpu_adjoint import _setup

pytestmark = pytest.mark.gpu


def test_optimizer_complex128_against_oracle():
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=12, seed=6)
    J0o, g0o = p.O.control_gradient(a, b, eps, 0.05, checkpoint_every=4)
    e, J, hist, it, nev = p.H.control_optimize(psi0, phi, eps, 0.05, checkpoint_every=4, max_iter=40,
                                               gtol=1e-10)
    assert it >= 1 and nev >= it + 1
    assert np.all(np.diff(hist) >= -1e-14 * abs(hist).max()), hist
    assert J > 1.01 * hist[0] and abs(hist[0] - J0o) < 1e-12 * J0o
    Jo, go = p.O.control_gradient(a, b, e, 0.05, checkpoint_every=4)
    assert abs(J - Jo) < 1e-10 * Jo, (J, Jo)
    assert np.abs(go).max() < 0.05 * np.abs(g0o).max(), (np.abs(go).max(), np.abs(g0o).max())


def test_optimizer_complex64_increases_objective():
    p, a, b, psi0, phi, eps = _setup(torch.complex64, nsteps=12, seed=6)
    e, J, hist, it, nev = p.H.control_optimize(psi0, phi, eps, 0.05, checkpoint_every=4, max_iter=10,
                                               gtol=1e-9)
    assert it >= 1
    assert np.all(np.diff(hist) >= -1e-6 * abs(hist).max()), hist
    assert J > 1.01 * hist[0]
    Jo, _ = p.O.control_gradient(a, b, e, 0.05, checkpoint_every=4)
    assert abs(J - Jo) < 1e-4 * Jo


def test_optimizer_argument_errors():
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=4, seed=6)
    with pytest.raises(rsg.RSGError):
        p.H.control_optimize(psi0, phi, eps, 0.05, max_iter=-1)
    # max_iter = 0: one evaluation, the field unchanged
    e, J, hist, it, nev = p.H.control_optimize(psi0, phi, eps, 0.05, max_iter=0)
    assert it == 0 and nev == 1 and np.array_equal(e, eps)


def test_fourier_parametrised_optimizer_against_oracle():
    """eps = B u with the sine-series basis (rsg_control_optimize_basis): the
    oracle evaluates J at the returned field and its gradient projected on
    the basis, B^T dJ/deps, has shrunk well below its starting size."""
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=12, seed=6)
    B = rsg.fourier_basis(12, 4)
    u0 = np.linalg.lstsq(B, eps, rcond=None)[0]
    J0o, g0o = p.O.control_gradient(a, b, B @ u0, 0.05, checkpoint_every=4)
    u, J, hist, it, nev = p.H.control_optimize_basis(psi0, phi, B, u0, 0.05, checkpoint_every=4, max_iter=40,
                                                     gtol=1e-10)
    assert it >= 1 and nev >= it + 1 and u.shape == (4,)
    assert abs(hist[0] - J0o) < 1e-12 * J0o
    assert np.all(np.diff(hist) >= -1e-14 * abs(hist).max()), hist
    assert J > 1.01 * hist[0]
    Jo, go = p.O.control_gradient(a, b, B @ u, 0.05, checkpoint_every=4)
    assert abs(J - Jo) < 1e-10 * Jo, (J, Jo)
    assert np.abs(B.T @ go).max() < 0.05 * np.abs(B.T @ g0o).max(), (B.T @ go, B.T @ g0o)
    # the search space is the basis: with the full-rank interval basis
    # (B = I) the loop is the plain one
    e1, J1, h1, it1, _ = p.H.control_optimize(psi0, phi, eps, 0.05, checkpoint_every=4, max_iter=3)
    e2, J2, h2, it2, _ = p.H.control_optimize_basis(psi0, phi, np.eye(12), eps, 0.05, checkpoint_every=4,
                                                    max_iter=3)
    assert it1 == it2 and np.abs(e1 - e2).max() < 1e-12 and abs(J1 - J2) < 1e-14 * J1


def test_basis_optimizer_argument_errors():
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=4, seed=6)
    B = rsg.fourier_basis(4, 2)
    with pytest.raises(rsg.RSGError):
        p.H.control_optimize_basis(psi0, phi, B, np.zeros(2), 0.05, max_iter=-1)
    Bn = B.copy()
    Bn[1, 1] = np.nan
    with pytest.raises(rsg.RSGError):
        p.H.control_optimize_basis(psi0, phi, Bn, np.zeros(2), 0.05)
    with pytest.raises(ValueError):
        p.H.control_optimize_basis(psi0, phi, B, np.zeros(3), 0.05)

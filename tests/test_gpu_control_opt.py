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

"""GPU parity: discrete adjoint gradient of J = |<phi|psi(T)>|^2 against the
oracle adjoint (1e-9 relative, complex128), central finite differences of the
library's own forward objective (1e-4), and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._parity import round_c64
from tests._systems import double_well_system
from workloads import control_field, rng, wavepacket_params, wavepacket_states

pytestmark = pytest.mark.gpu


def _setup(dtype, n=14, h=0.5, nsteps=12, seed=0):
    p = double_well_system(n, h, dtype)
    g = rng(4, seed)
    a = wavepacket_states(p.om.xyz, wavepacket_params(g, 1, 1.5))
    b = wavepacket_states(p.om.xyz, wavepacket_params(g, 1, 1.5))
    a = a / np.sqrt(p.h ** 3 * np.vdot(a, a).real)
    b = b / np.sqrt(p.h ** 3 * np.vdot(b, b).real)
    if dtype == torch.complex64:
        a, b = round_c64(a), round_c64(b)
    eps = control_field(g, nsteps, 0.05, amax=0.3)
    npdt = np.complex64 if dtype == torch.complex64 else np.complex128
    psi0 = torch.from_numpy(p.to_lib(a[:, 0]).astype(npdt)).cuda()
    phi = torch.from_numpy(p.to_lib(b[:, 0]).astype(npdt)).cuda()
    return p, a[:, 0], b[:, 0], psi0, phi, eps


@pytest.mark.parametrize("keep,merge", [(-1, -1), (0, -1), (1, 0), (1, 1)])
@pytest.mark.parametrize("scheme,nsub,K", [(1, 1, 5), (0, 2, 3), (1, 2, 12)])
def test_adjoint_matches_oracle_c128(scheme, nsub, K, keep, merge):
    """keep 1, merge 1: the costate sweep of each checkpoint segment and the
    recompute sweep of the segment before it share two-column launches, each
    column with its own field and sign; with K = 5 the last segment is
    shorter than its partner, with K = 12 there is one segment."""
    p, a, b, psi0, phi, eps = _setup(torch.complex128)
    p.H.set_option("adjoint_keep_powers", keep)
    p.H.set_option("adjoint_merge", merge)
    Jw, gw = p.O.control_gradient(a, b, eps, 0.05, scheme=scheme, nsub=nsub, checkpoint_every=4)
    J, gr = p.H.control_gradient(psi0, phi, eps, 0.05, scheme=scheme, nsub=nsub,
                                 checkpoint_every=K)
    assert abs(J - Jw) < 1e-12 * abs(Jw)
    assert np.abs(gr - gw).max() < 1e-9 * np.abs(gw).max(), (gr, gw)


def test_adjoint_c64_error_reported():
    p, a, b, psi0, phi, eps = _setup(torch.complex64)
    Jw, gw = p.O.control_gradient(a, b, eps, 0.05, checkpoint_every=4)
    J, gr = p.H.control_gradient(psi0, phi, eps, 0.05, checkpoint_every=4)
    err = np.abs(gr - gw).max() / np.abs(gw).max()
    print(f"complex64 adjoint gradient error vs FP64 oracle: {err:.3e}")
    assert abs(J - Jw) < 1e-5 * abs(Jw)
    assert err < 1e-3


@pytest.mark.parametrize("kernel,merge", [(0, 0), (5, 0), (7, 0), (0, 1)])
def test_adjoint_c64_kernels_agree(kernel, merge):
    """The adjoint's power sums run through the stencil epilogue's running
    sum (acc, acc_base): the staged, register-blocked and tensor-copy kernels
    against the oracle; with merge 1 the shared two-column sweeps (which run
    on the one-thread-per-value kernel)."""
    p, a, b, psi0, phi, eps = _setup(torch.complex64, n=20, h=0.45)
    p.H.set_option("kernel", kernel)
    p.H.set_option("adjoint_merge", merge)
    Jw, gw = p.O.control_gradient(a, b, eps, 0.05, checkpoint_every=4)
    J, gr = p.H.control_gradient(psi0, phi, eps, 0.05, checkpoint_every=4)
    if merge == 0:
        assert p.H.get_option("last_kernel") == kernel
    assert abs(J - Jw) < 1e-5 * abs(Jw)
    assert np.abs(gr - gw).max() < 1e-3 * np.abs(gw).max()


def test_adjoint_vs_central_differences_on_device():
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=8, seed=3)
    J, g = p.H.control_gradient(psi0, phi, eps, 0.05, checkpoint_every=3)
    eta = 1e-5
    for k in range(len(eps)):
        e1, e2 = eps.copy(), eps.copy()
        e1[k] += eta
        e2[k] -= eta
        fd = (p.H.control_gradient(psi0, phi, e1, 0.05)[0]
              - p.H.control_gradient(psi0, phi, e2, 0.05)[0]) / (2 * eta)
        assert abs(fd - g[k]) < 1e-4 * np.abs(g).max()


def test_autograd_function():
    p, a, b, psi0, phi, eps = _setup(torch.complex128, nsteps=6, seed=4)
    e = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    J = rsg.ControlObjective.apply(e, p.H, psi0, phi, 0.05)
    (2.0 * J).backward()
    _, g = p.H.control_gradient(psi0, phi, eps, 0.05)
    assert torch.allclose(e.grad, torch.from_numpy(2.0 * g), rtol=0, atol=1e-15)
    _ = oracle

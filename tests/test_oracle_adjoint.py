"""Pins for the oracle's discrete adjoint gradient (no GPU).

The adjoint gradient is checked against central finite differences of the
oracle's forward objective, the second-order Taylor remainder, invariance to
the checkpoint spacing, and the continuum gradient formula
dJ/du = 2 Im int <chi| dH/du |psi> dt in the small-step limit.
"""
import numpy as np

import oracle
from workloads import control_field, potential_double_well, rng, wavepacket_params, wavepacket_states


def _problem(n=12, h=0.5, nsteps=12, seed=0):
    g = rng(4, seed)
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, potential_double_well(m.xyz, 0.02, 2.0, 0.5))
    a = wavepacket_states(m.xyz, wavepacket_params(g, 1, 1.5))
    b = wavepacket_states(m.xyz, wavepacket_params(g, 1, 1.5))
    a = a / np.sqrt(m.h ** 3 * np.vdot(a, a).real)
    b = b / np.sqrt(m.h ** 3 * np.vdot(b, b).real)
    eps = control_field(g, nsteps, 0.05, amax=0.3)
    return m, H, a[:, 0], b[:, 0], eps


def test_gradient_matches_central_differences():
    m, H, psi0, phi, eps = _problem()
    for scheme, nsub in ((oracle.ETRS, 1), (oracle.EXPMID, 2)):
        J, g = H.control_gradient(psi0, phi, eps, 0.05, scheme=scheme, nsub=nsub,
                                  checkpoint_every=5)
        assert abs(J - H.objective(psi0, phi, eps, 0.05, scheme=scheme, nsub=nsub)) < 1e-15
        fd = np.empty_like(g)
        eta = 1e-5
        for k in range(len(eps)):
            e1, e2 = eps.copy(), eps.copy()
            e1[k] += eta
            e2[k] -= eta
            fd[k] = (H.objective(psi0, phi, e1, 0.05, scheme=scheme, nsub=nsub)
                     - H.objective(psi0, phi, e2, 0.05, scheme=scheme, nsub=nsub)) / (2 * eta)
        assert np.abs(g - fd).max() < 1e-6 * np.abs(fd).max(), (g, fd)


def test_taylor_remainder_is_second_order():
    m, H, psi0, phi, eps = _problem(seed=1)
    J, g = H.control_gradient(psi0, phi, eps, 0.05, checkpoint_every=4)
    d = rng(4, 7).standard_normal(len(eps))
    rem = []
    for eta in (1e-2, 5e-3, 2.5e-3):
        rem.append(abs(H.objective(psi0, phi, eps + eta * d, 0.05) - J - eta * g @ d))
    assert 3.5 < rem[0] / rem[1] < 4.5 and 3.5 < rem[1] / rem[2] < 4.5, rem


def test_checkpoint_spacing_does_not_change_result():
    m, H, psi0, phi, eps = _problem(seed=2)
    res = [H.control_gradient(psi0, phi, eps, 0.05, checkpoint_every=k)[1] for k in (1, 5, 12)]
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[1], res[2])


def test_small_step_limit_matches_continuum_formula():
    """As dt -> 0 each component tends to 2 dt Im <chi(t_k)| x |psi(t_k)>
    (the paper's gradient integral restricted to one interval)."""
    m, H, psi0, phi, eps = _problem(n=10, h=0.6, nsteps=6, seed=3)
    dt = 0.004
    J, g = H.control_gradient(psi0, phi, eps, dt, checkpoint_every=6)
    # continuum estimate: forward psi(t_k), backward chi(t_{k+1}) with the same
    # propagator, midpoint quadrature over each interval
    x = m.xyz[:, 0]
    psis = [psi0.reshape(-1, 1)]
    for k in range(len(eps)):
        nxt, _ = H.propagate(psis[-1], 1, dt, scheme=oracle.ETRS, eps=eps[k:k + 1], dir=(1, 0, 0))
        psis.append(nxt)
    ov = m.h ** 3 * np.vdot(phi, psis[-1][:, 0])
    chi = (phi * ov).reshape(-1, 1)
    est = np.empty(len(eps))
    for k in range(len(eps) - 1, -1, -1):
        prev, _ = H.propagate(chi, 1, -dt, scheme=oracle.ETRS, eps=eps[k:k + 1], dir=(1, 0, 0))
        mid_chi = 0.5 * (chi + prev)
        mid_psi = 0.5 * (psis[k] + psis[k + 1])
        est[k] = 2 * dt * np.imag(m.h ** 3 * np.vdot(mid_chi[:, 0], x * mid_psi[:, 0]))
        chi = prev
    assert np.abs(g - est).max() < 1e-3 * np.abs(g).max(), (g, est)

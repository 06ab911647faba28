"""Pins for the oracle's Taylor-4 exponential, time-step schemes and MGS.

References that are not the oracle itself: the eigen-decomposition of the
dense operator (LAPACK), scipy's matrix exponential, the closed-form
spreading of a free Gaussian packet, numpy's QR and the exact shift of an
oscillator's ground level in a uniform field.
"""
import numpy as np
import scipy.linalg as sl

import oracle
from workloads import (potential_double_well, potential_harmonic, rng,
                       wavepacket_params, wavepacket_states, white_noise_states)
from tests._oracle_helpers import dense_h, lowest_eigs


def _small_system(seed=0, n=8, h=0.5):
    g = rng(90, seed)
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, potential_harmonic(m.xyz, 0.5))
    H.set_projectors([[0.2, -0.1, 0.3]], [1.2], [1], [0.3], [np.diag([0.4, -0.2, 0.3, 0.1])])
    return g, m, H


def _R(z):
    """The degree-4 truncated exponential as a scalar polynomial."""
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def test_taylor4_equals_eigen_expansion():
    """T(tau) psi = V R(-i tau E) V^H psi for the dense Hermitian operator."""
    g, m, H = _small_system()
    D = dense_h(H, m.P, eps=0.03, dir=(1, 0, 0))
    E, V = np.linalg.eigh(D)
    psi = white_noise_states(g, m.P, 2)
    tau = 0.02
    want = V @ (_R(-1j * tau * E)[:, None] * (V.conj().T @ psi))
    got = H.taylor4(psi, tau, eps=0.03, dir=(1, 0, 0))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_taylor4_local_error_is_fifth_order():
    """||T(tau) - expm(-i tau H)|| psi shrinks 32x when tau halves."""
    g, m, H = _small_system(1)
    D = dense_h(H, m.P)
    psi = white_noise_states(g, m.P, 1)
    errs = []
    for tau in (0.01, 0.005):
        exact = sl.expm(-1j * tau * D) @ psi
        errs.append(np.linalg.norm(H.taylor4(psi, tau) - exact))
    assert 25 < errs[0] / errs[1] < 40, errs


def test_backward_exponential_is_adjoint():
    """<T(-tau) chi, psi> = <chi, T(tau) psi>: T(tau)^dagger = T(-tau) for Hermitian H."""
    g, m, H = _small_system(2)
    a = white_noise_states(g, m.P, 1)
    b = white_noise_states(g, m.P, 1)
    tau = 0.03
    lhs = np.vdot(H.taylor4(a, -tau, eps=0.02, dir=(0, 1, 0)), b)
    rhs = np.vdot(a, H.taylor4(b, tau, eps=0.02, dir=(0, 1, 0)))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_norm_loss_matches_stability_polynomial():
    """For an eigenvector, one step scales the norm^2 by |R(i y)|^2 = 1 - y^6/72 + y^8/576."""
    g, m, H = _small_system(3)
    D = dense_h(H, m.P)
    E, V = np.linalg.eigh(D)
    k = len(E) - 1            # highest level: the largest y
    phi = V[:, k:k + 1]
    tau = 1.5 / E[k]
    y = tau * E[k]
    out = H.taylor4(phi, tau)
    n2 = np.vdot(out, out).real / np.vdot(phi, phi).real
    assert abs(n2 - (1 - y ** 6 / 72 + y ** 8 / 576)) < 1e-12


def test_free_gaussian_packet_spreads_as_closed_form():
    """|psi|^2 of a free packet: mean x0 + k0 t, variance s0^2 (1 + t^2/(4 s0^4))."""
    n, h = 40, 0.4
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    s0, k0, x0 = 1.0, 0.5, -0.5
    r = m.xyz - np.array([x0, 0.0, 0.0])
    psi = np.exp(-np.sum(r * r, axis=1) / (4 * s0 * s0) + 1j * k0 * m.xyz[:, 0])
    psi = (psi / np.sqrt(h ** 3 * np.vdot(psi, psi).real)).reshape(-1, 1)
    dt, nsteps = 0.04, 50
    out, _ = H.propagate(psi, nsteps, dt, scheme=oracle.EXPMID)
    t = dt * nsteps
    rho = np.abs(out[:, 0]) ** 2 * h ** 3
    mean = np.sum(rho * m.xyz[:, 0])
    var = np.sum(rho * (m.xyz[:, 0] - mean) ** 2)
    assert abs(mean - (x0 + k0 * t)) < 1e-4, mean
    assert abs(var - s0 ** 2 * (1 + t * t / (4 * s0 ** 4))) < 1e-4, var


def test_etrs_equals_two_half_exponentials_of_expmid():
    """With a linear H and a field constant over the interval, ETRS with nsub
    substeps performs the same exponentials as the midpoint rule with 2 nsub."""
    g, m, H = _small_system(4)
    psi = white_noise_states(g, m.P, 2)
    eps = np.array([0.01, -0.02, 0.03])
    a, _ = H.propagate(psi, 3, 0.02, scheme=oracle.ETRS, nsub=1, eps=eps, dir=(0, 0, 1))
    b, _ = H.propagate(psi, 3, 0.02, scheme=oracle.EXPMID, nsub=2, eps=eps, dir=(0, 0, 1))
    assert np.array_equal(a, b)


def test_propagation_of_eigenstate_is_a_phase():
    """An eigenvector evolves as R(-i tau E)^n phi: phase and norm as predicted."""
    m = oracle.Mesh(oracle.CUBE, 14, h=0.5)
    H = oracle.Hamiltonian(m, potential_double_well(m.xyz, 0.02, 2.0, 0.5))
    import scipy.sparse.linalg as sla
    op = sla.LinearOperator((m.P, m.P), dtype=np.float64,
                            matvec=lambda v: H.apply(np.asarray(v, np.complex128).reshape(-1, 1)).real.ravel())
    E, V = sla.eigsh(op, k=1, which="SA", tol=1e-13, v0=np.ones(m.P))
    phi = V[:, :1] / np.sqrt(m.h ** 3)
    dt, n = 0.05, 20
    out, _ = H.propagate(phi + 0j, n, dt, scheme=oracle.EXPMID)
    want = _R(-1j * dt * E[0]) ** n * phi
    assert np.abs(out - want).max() < 1e-9 * np.abs(phi).max()


def test_norm_drift_reporting_and_mgs():
    """Drift is |<psi|psi>-1| before each MGS; after MGS the block is orthonormal."""
    g = rng(91)
    m = oracle.Mesh(oracle.CUBE, 12, h=0.5)
    H = oracle.Hamiltonian(m, potential_harmonic(m.xyz, 0.5))
    psi = wavepacket_states(m.xyz, wavepacket_params(g, 3, 1.0))
    psi = m.mgs(psi)
    out, drift = H.propagate(psi, 10, 0.02, scheme=oracle.ETRS, gs_every=5)
    G = m.h ** 3 * out.conj().T @ out
    assert np.abs(G - np.eye(3)).max() < 1e-13
    assert np.all(drift < 1e-8) and np.all(drift >= 0)
    noGS, drift2 = H.propagate(psi, 10, 0.02, scheme=oracle.ETRS, gs_every=0)
    n2 = m.h ** 3 * np.sum(np.abs(noGS) ** 2, axis=0)
    assert np.allclose(drift2, np.abs(n2 - 1), rtol=0, atol=1e-15)


def test_mgs_matches_numpy_qr():
    """MGS in index order = QR with a positive real R diagonal (h^3-weighted)."""
    g = rng(92)
    m = oracle.Mesh(oracle.CUBE, 9, h=0.3)
    A = white_noise_states(g, m.P, 5)
    Q = m.mgs(A) * np.sqrt(m.h ** 3)
    q, r = np.linalg.qr(A * np.sqrt(m.h ** 3))
    ph = np.diag(r) / np.abs(np.diag(r))
    assert np.abs(Q - q * ph[None, :]).max() < 1e-12


def test_uniform_field_shifts_oscillator_ground_level():
    """H0 + eps x for V = w^2 r^2/2: E0 shifts by -eps^2/(2 w^2); <x> by -eps/w^2."""
    m = oracle.Mesh(oracle.CUBE, 36, h=0.35)
    H = oracle.Hamiltonian(m, potential_harmonic(m.xyz, 0.5))
    e0 = lowest_eigs(H, m.P, 1, tol=1e-12)[0]
    eps = 0.05
    import scipy.sparse.linalg as sla
    op = sla.LinearOperator(
        (m.P, m.P), dtype=np.float64,
        matvec=lambda v: H.apply(np.asarray(v, np.complex128).reshape(-1, 1), eps=eps,
                                 dir=(1, 0, 0)).real.ravel())
    E, V = sla.eigsh(op, k=1, which="SA", tol=1e-12, v0=np.ones(m.P))
    assert abs((E[0] - e0) - (-eps ** 2 / (2 * 0.25))) < 2e-6
    rho = V[:, 0] ** 2 / np.sum(V[:, 0] ** 2)
    assert abs(np.sum(rho * m.xyz[:, 0]) - (-eps / 0.25)) < 1e-4

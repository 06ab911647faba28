"""Pins of the oracle's complex-scaled operator (Sec. "Complex scaling and
resonances": H_theta = -1/2 e^{-2 i theta} lap + V(r e^{i theta})):

- closed form: with antisymmetric-image walls and V = v0 constant, products
  of sines are exact eigenvectors with eigenvalue e^{-2 i theta} E + v0, E
  the closed-form discrete free spectrum sum_d sigma(pi m_d / (N+1)) / (2 h^2),
  sigma(phi) = -c0 - 2 sum_k c_k cos(k phi);
- complex symmetry: x^T H_theta y = y^T H_theta x (no conjugate) on a sphere
  with random complex potential values;
- the paper's one-dimensional example v(x) = 3 (x^2 - 2) e^{-x^2/4}: its
  two bound-state energies do not move with theta (the rotated continuum
  does), checked between theta = 0 and theta = 0.5 on a 301-point line;
- the same example's lowest resonance (spectrum figure of the section: an
  isolated eigenvalue near the origin, imaginary part of order -1e-5): the
  first non-real eigenvalue that stays put between theta = 0.4 and 0.5 has
  0 < Re < 1 and -1e-4 < Im < -1e-6 (this discretisation converges in h
  to 0.35448 - 4.70e-5 i).

The scaled Taylor-4 exponential and propagation are pinned by the same
closed-form modes through the scalar polynomial R(-i tau lambda), and by
the plain exponential at theta = 0; the mask-absorber propagation (Sec.
"Photoemission", Eq. (mask_split)) by its reductions to the plain
propagation.
"""
import math

import numpy as np

import oracle
from workloads import rng, white_noise_states

C = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]


def _sigma(phi):
    return -C[0] - 2 * sum(C[k] * np.cos(k * phi) for k in range(1, 5))


def test_closed_form_rotated_spectrum():
    n, h, v0, theta = 9, 0.35, 0.7, 0.4
    m = oracle.Mesh(oracle.CUBE, n, h=h, bc=oracle.ODD)
    for modes in ((1, 1, 1), (2, 3, 1), (4, 1, 7)):
        f = np.ones(m.P)
        for d, md in enumerate(modes):
            f = f * np.sin(np.pi * md * (m.ijk[:, d] + 1) / (n + 1))
        E = sum(_sigma(np.pi * md / (n + 1)) for md in modes) / (2 * h * h)
        hf = m.apply_scaled(f.reshape(-1, 1).astype(np.complex128), theta, np.full(m.P, v0 + 0j))[:, 0]
        big = np.abs(f) > 0.1 * np.abs(f).max()
        ratio = hf[big] / f[big]
        want = np.exp(-2j * theta) * E + v0
        assert np.abs(ratio - want).max() < 1e-11 * abs(want), (ratio[:3], want)


def test_complex_symmetric():
    g = np.random.default_rng(21)
    m = oracle.Mesh(oracle.SPHERE, radius=2.0, h=0.3)
    vt = g.standard_normal(m.P) + 1j * g.standard_normal(m.P)
    x = g.standard_normal((m.P, 1)) + 1j * g.standard_normal((m.P, 1))
    y = g.standard_normal((m.P, 1)) + 1j * g.standard_normal((m.P, 1))
    a = (x[:, 0] * m.apply_scaled(y, 0.3, vt)[:, 0]).sum()
    b = (y[:, 0] * m.apply_scaled(x, 0.3, vt)[:, 0]).sum()
    assert abs(a - b) < 1e-12 * abs(a)
    # and not Hermitian once theta != 0
    c = (np.conj(x[:, 0]) * m.apply_scaled(y, 0.3, vt)[:, 0]).sum()
    d = np.conj((np.conj(y[:, 0]) * m.apply_scaled(x, 0.3, vt)[:, 0]).sum())
    assert abs(c - d) > 1e-3 * abs(c)


def test_paper_1d_example_bound_states_do_not_rotate():
    N, h = 301, 0.1
    m = oracle.Mesh(oracle.BOX, (N, 1, 1), h=h)
    x = m.xyz[:, 0]
    levels = []
    for theta in (0.0, 0.5):
        z = x * np.exp(1j * theta)
        vt = 3 * (z * z - 2) * np.exp(-z * z / 4)
        A = m.apply_scaled(np.eye(m.P, dtype=np.complex128), theta, vt)
        w = np.linalg.eigvals(A)
        # the single-point y and z directions add -1/2 e^{-2 i theta} 2 c0 / h^2
        w = w - np.exp(-2j * theta) * (-C[0] / h ** 2)
        levels.append(w)
    w0 = np.sort(levels[0].real)
    bound = w0[w0 < -0.05][:2]
    assert len(bound) == 2, w0[:5]
    for e in bound:
        near = levels[1][np.argmin(np.abs(levels[1] - e))]
        assert abs(near - e) < 1e-5, (e, near)
    # the continuum rotates into the lower half plane
    assert np.sum(levels[1].imag < -0.1) > N // 2


def _spectrum_1d(N, h, theta):
    m = oracle.Mesh(oracle.BOX, (N, 1, 1), h=h)
    z = m.xyz[:, 0] * np.exp(1j * theta)
    vt = 3 * (z * z - 2) * np.exp(-z * z / 4)
    w = np.linalg.eigvals(m.apply_scaled(np.eye(m.P, dtype=np.complex128), theta, vt))
    return w - np.exp(-2j * theta) * (-C[0] / h ** 2)


def test_paper_1d_example_lowest_resonance():
    a, b = _spectrum_1d(301, 0.1, 0.5), _spectrum_1d(301, 0.1, 0.4)
    stable = np.array(sorted((e for e in a if np.abs(b - e).min() < 1e-4 and e.real < 3), key=lambda e: e.real))
    assert len(stable) >= 3, stable
    assert np.all(np.abs(stable[:2].imag) < 1e-6) and np.all(stable[:2].real < 0)
    r = stable[2]
    assert 0 < r.real < 1 and -1e-4 < r.imag < -1e-6, r


def test_rotated_wells_generator():
    """workloads.potential_wells_scaled: theta = 0 gives the real wells, and
    for small theta v(r e^{i theta}) = v(r) + i theta r.grad v(r) + O(theta^2)."""
    from workloads import gaussian_wells, potential_wells, potential_wells_scaled, rng
    g = rng(40)
    c, d, w = gaussian_wells(g, 5, 2.0)
    xyz = g.uniform(-3, 3, size=(200, 3))
    assert np.abs(potential_wells_scaled(xyz, c, d, w, 0.0) - potential_wells(xyz, c, d, w)).max() < 1e-15
    t, dx = 1e-4, 1e-6
    v = potential_wells(xyz, c, d, w)
    rgrad = (potential_wells(xyz * (1 + dx), c, d, w) - potential_wells(xyz * (1 - dx), c, d, w)) / (2 * dx)
    want = v + 1j * t * rgrad
    got = potential_wells_scaled(xyz, c, d, w, t)
    assert np.abs(got - want).max() < 1e-7 * max(1.0, np.abs(v).max())


def _R4(z):
    return sum(z ** n / math.factorial(n) for n in range(5))


def test_scaled_taylor_and_propagation_on_closed_form_modes():
    """The scaled Taylor-4 exponential and propagation against the closed
    form: a product of sines between image walls is an eigenvector of H_theta
    with lambda = e^{-2i theta} E + v0 (E from the stencil's symbol), so one
    exponential multiplies it by R(-i tau lambda), R(z) = sum_{n<=4} z^n/n!,
    a scalar polynomial (a route other than repeated applications); an ETRS
    step by R(-i dt lambda / 2)^2 and an exponential-midpoint step by
    R(-i dt lambda)."""
    n, h, v0, theta, tau = 9, 0.35, 0.7 - 0.05j, 0.3, 0.04
    m = oracle.Mesh(oracle.CUBE, n, h=h, bc=oracle.ODD)
    vt = np.full(m.P, v0)
    for modes in ((1, 1, 1), (2, 3, 1)):
        f = np.ones(m.P, dtype=np.complex128)
        for d, md in enumerate(modes):
            f = f * np.sin(np.pi * md * (m.ijk[:, d] + 1) / (n + 1))
        E = sum(_sigma(np.pi * md / (n + 1)) for md in modes) / (2 * h * h)
        lam = np.exp(-2j * theta) * E + v0
        got = m.taylor4_scaled(f.reshape(-1, 1), theta, vt, tau)[:, 0]
        assert np.abs(got - _R4(-1j * tau * lam) * f).max() < 1e-12 * np.abs(f).max()
        et = m.propagate_scaled(f.reshape(-1, 1), theta, vt, 3, 2 * tau, scheme=oracle.ETRS)[:, 0]
        assert np.abs(et - _R4(-1j * tau * lam) ** 6 * f).max() < 1e-12 * np.abs(f).max()
        mid = m.propagate_scaled(f.reshape(-1, 1), theta, vt, 2, tau, scheme=oracle.EXPMID)[:, 0]
        assert np.abs(mid - _R4(-1j * tau * lam) ** 2 * f).max() < 1e-12 * np.abs(f).max()


def test_scaled_taylor_at_zero_angle_is_the_plain_exponential():
    """theta = 0 with a real v_theta: the plain operator's Taylor-4 exponential."""
    m = oracle.Mesh(oracle.SPHERE, radius=2.0, h=0.3)
    g = rng(31)
    V = g.uniform(-1.0, 1.0, m.P)
    psi = white_noise_states(g, m.P, 3)
    O = oracle.Hamiltonian(m, V)
    want = O.taylor4(psi, 0.03)
    got = m.taylor4_scaled(psi, 0.0, V.astype(np.complex128), 0.03)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_masked_propagation_reduces_to_plain_and_scales():
    """A mask of ones is the plain propagation; a constant mask c multiplies
    n steps by c^n (every step is linear); a mask vanishing outside a ball
    leaves zero there after the first step."""
    m = oracle.Mesh(oracle.CUBE, 12, h=0.35)
    g = rng(32)
    O = oracle.Hamiltonian(m, 0.5 * np.sum(m.xyz ** 2, axis=1))
    psi = white_noise_states(g, m.P, 2)
    plain, _ = O.propagate(psi, 4, 0.02, scheme=oracle.ETRS)
    ones = O.propagate_masked(psi, 4, 0.02, np.ones(m.P), scheme=oracle.ETRS)
    assert np.array_equal(ones, plain)
    half = O.propagate_masked(psi, 4, 0.02, np.full(m.P, 0.5), scheme=oracle.ETRS)
    assert np.abs(half - 0.0625 * plain).max() < 1e-15 * np.abs(plain).max() + 1e-300
    ball = (np.linalg.norm(m.xyz, axis=1) < 1.2).astype(np.float64)
    inside = O.propagate_masked(psi, 2, 0.02, ball, scheme=oracle.ETRS)
    assert not inside[ball == 0].any()

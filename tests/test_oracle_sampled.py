"""The oracle's sampled applications equal its full applications (no GPU)."""
import numpy as np

import oracle
from workloads import rng, white_noise_states


def test_sampled_equals_full():
    g = rng(96)
    m = oracle.Mesh(oracle.SPHERE, radius=3.0, h=0.3)
    H = oracle.Hamiltonian(m, g.standard_normal(m.P))
    H.set_projectors(g.uniform(-1, 1, (3, 3)), [1.2, 1.0, 1.4], [1, 0, 2], [0.3, 0.25, 0.35],
                     [np.diag(g.uniform(-1, 1, k)) for k in (4, 1, 9)])
    psi = white_noise_states(g, m.P, 3)
    full = H.apply(psi, eps=0.1, dir=(0, 1, 0))
    p = g.integers(0, m.P, 500)
    s = g.integers(0, 3, 500)
    got = H.apply_sampled(psi, p, s, eps=0.1, dir=(0, 1, 0))
    assert np.abs(got - full[p, s]).max() < 1e-13 * np.abs(full).max()   # summation order differs


def test_scaled_sampled_equals_full():
    g = rng(97)
    m = oracle.Mesh(oracle.SPHERE, radius=3.0, h=0.3)
    vt = g.standard_normal(m.P) + 1j * g.standard_normal(m.P)
    psi = white_noise_states(g, m.P, 3)
    full = m.apply_scaled(psi, 0.3, vt)
    p = g.integers(0, m.P, 500)
    s = g.integers(0, 3, 500)
    got = m.apply_scaled_sampled(psi, 0.3, vt, p, s)
    assert np.array_equal(got, full[p, s])          # the same per-point arithmetic

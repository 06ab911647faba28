"""Pins for the oracle's kinetic + local operator (no GPU).

Each test checks the oracle against something other than itself: exactness
of the finite-difference Laplacian on polynomials (a mathematical property of
an order-8 central difference), closed-form continuum eigenvalues, the
paper's printed lithium table, and symmetry invariants.
"""
import json
import os

import numpy as np
import pytest

import oracle
from workloads import (potential_harmonic, potential_soft_coulomb_li, rng,
                       white_noise_states)
from tests._oracle_helpers import lowest_eigs, wdot

HERE = os.path.dirname(os.path.abspath(__file__))


def _poly(xyz, a, b, c):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return x ** a * y ** b * z ** c


def _lap_poly(xyz, a, b, c):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    out = np.zeros(xyz.shape[0])
    if a >= 2:
        out += a * (a - 1) * x ** (a - 2) * y ** b * z ** c
    if b >= 2:
        out += b * (b - 1) * x ** a * y ** (b - 2) * z ** c
    if c >= 2:
        out += c * (c - 1) * x ** a * y ** b * z ** (c - 2)
    return out


@pytest.mark.parametrize("abc", [(2, 0, 0), (0, 5, 0), (0, 0, 9), (9, 0, 0), (3, 4, 2),
                                 (1, 7, 3), (9, 9, 0)])
def test_laplacian_exact_on_polynomials(abc):
    """An order-8 central second difference is exact for degree <= 9 per axis."""
    n, h = 18, 0.2
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    f = _poly(m.xyz, *abc)
    got = H.apply(f.reshape(-1, 1).astype(np.complex128)).real.ravel()
    want = -0.5 * _lap_poly(m.xyz, *abc)
    inner = np.all((m.ijk >= 4) & (m.ijk <= n - 5), axis=1)
    scale = np.abs(f[inner]).max() / h ** 2 + np.abs(want[inner]).max()
    err = np.abs(got[inner] - want[inner]).max() / scale
    assert err < 1e-13, err


def test_laplacian_not_exact_at_degree_10():
    """Degree 10 must leave a residual: the stencil is order 8, not higher."""
    n, h = 18, 0.2
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    f = _poly(m.xyz, 10, 0, 0)
    got = H.apply(f.reshape(-1, 1).astype(np.complex128)).real.ravel()
    want = -0.5 * _lap_poly(m.xyz, 10, 0, 0)
    inner = np.all((m.ijk >= 4) & (m.ijk <= n - 5), axis=1)
    # The truncation term of an order-8 second difference for x^10 is
    # -(2 / 9!)... h^8 * f^(10) / const: a constant offset, visibly nonzero.
    resid = got[inner] - want[inner]
    assert np.abs(resid).max() > 1e-6
    assert np.ptp(resid) < 1e-6 * np.abs(resid).max() + 1e-9   # constant, as f^(10) is


def _odd_box_level(n, h, modes):
    m = oracle.Mesh(oracle.CUBE, n, h=h, bc=oracle.ODD)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    f = np.ones(m.P)
    for d, md in enumerate(modes):
        f = f * np.sin(np.pi * md * (m.ijk[:, d] + 1) / (n + 1))
    hf = H.apply(f.reshape(-1, 1).astype(np.complex128)).real.ravel()
    big = np.abs(f) > 0.1 * np.abs(f).max()
    ratio = hf[big] / f[big]
    assert np.ptp(ratio) < 1e-10 * abs(ratio.mean())   # exact eigenvector
    return ratio.mean()


def test_particle_in_box_converges_at_order_8():
    """Antisymmetric-image walls at distance L: E -> pi^2 (nx^2+ny^2+nz^2)/(2 L^2)."""
    L = 4.0
    modes = (1, 2, 3)
    exact = np.pi ** 2 * sum(k * k for k in modes) / (2 * L * L)
    errs = []
    for n in (15, 31):
        h = L / (n + 1)
        errs.append(abs(_odd_box_level(n, h, modes) - exact))
    rate = np.log2(errs[0] / errs[1])
    assert 7.5 < rate < 8.6, (errs, rate)
    assert errs[1] < 1e-7


def test_zero_boundary_box_converges_at_first_order():
    """With zero ghosts the box levels converge only at O(h), not O(h^8)."""
    L = 4.0
    exact = 3 * np.pi ** 2 / (2 * L * L)
    errs = []
    for n in (15, 31):
        h = L / (n + 1)
        m = oracle.Mesh(oracle.CUBE, n, h=h)
        H = oracle.Hamiltonian(m, np.zeros(m.P))
        errs.append(abs(lowest_eigs(H, m.P, 1, tol=1e-12)[0] - exact))
    rate = np.log2(errs[0] / errs[1])
    assert 0.7 < rate < 1.3, (errs, rate)


def test_harmonic_oscillator_levels_cfg1():
    """32^3 at h=0.3, w=0.5: levels 3/2 w, 5/2 w (x3), up to box truncation."""
    m = oracle.Mesh(oracle.CUBE, 32, h=0.3)
    H = oracle.Hamiltonian(m, potential_harmonic(m.xyz, 0.5))
    w = lowest_eigs(H, m.P, 5, tol=1e-10)
    assert abs(w[0] - 0.75) < 1e-4, w
    assert np.all(np.abs(w[1:4] - 1.25) < 5e-4), w


def test_harmonic_oscillator_bigger_box_converges():
    """Box truncation dominates at 32^3; a wider box at the same h shrinks it."""
    h = 0.3
    errs = []
    for n in (32, 44):
        m = oracle.Mesh(oracle.CUBE, n, h=h)
        H = oracle.Hamiltonian(m, potential_harmonic(m.xyz, 0.5))
        errs.append(abs(lowest_eigs(H, m.P, 1, tol=1e-12)[0] - 0.75))
    assert errs[1] < errs[0] / 10, errs
    assert errs[1] < 1e-6, errs


@pytest.mark.slow
def test_lithium_1d_table_from_paper():
    """The paper's 1-D lithium eigenvalues as a 3-D one-particle problem."""
    with open(os.path.join(HERE, "golden", "li_1d_table.json")) as f:
        gold = json.load(f)
    L, h = 12.0, 0.4
    n = int(round(2 * L / h)) + 1
    m = oracle.Mesh(oracle.CUBE, n, h=h)
    H = oracle.Hamiltonian(m, potential_soft_coulomb_li(m.xyz))
    # Lanczos finds a degenerate pair only with room to spare: ask for 6
    # with a wide Krylov space and pin the lowest 4.
    w = lowest_eigs(H, m.P, 6, seed=3, tol=1e-8, ncv=40)[:4]
    want = np.array(gold["energies_hartree"])
    assert np.all(np.abs(w - want) < 1.5 * gold["printed_precision"]), (w, want)


def test_hermitian_with_projectors_and_field():
    """<phi|H psi> = conj <psi|H phi> on a sphere with wells, atoms and a field."""
    g = rng(99)
    m = oracle.Mesh(oracle.SPHERE, radius=3.0, h=0.3)
    V = g.standard_normal(m.P)
    H = oracle.Hamiltonian(m, V)
    c = g.uniform(-1.5, 1.5, size=(2, 3))
    hm = [np.diag(g.uniform(-1, 1, 9)), g.uniform(-1, 1, (4, 4))]
    hm[1] = hm[1] + hm[1].T
    H.set_projectors(c, [1.5, 1.2], [2, 1], [0.4, 0.3], hm)
    a = white_noise_states(g, m.P, 2)
    d = (0.3, -0.5, 0.8)
    ha = H.apply(a, eps=0.07, dir=d)
    lhs = wdot(m.h, a[:, 0], ha[:, 1])
    rhs = np.conj(wdot(m.h, a[:, 1], ha[:, 0]))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_sphere_mesh_counts():
    """Integer-ball lattice counts: known values of #{i^2+j^2+k^2 <= r^2}."""
    # r^2 = 1 -> 7 points, r^2 = 2 -> 19, r^2 = 4 -> 33 (lattice points in a ball)
    assert oracle.Mesh(oracle.SPHERE, radius=1.0, h=1.0).P == 7
    assert oracle.Mesh(oracle.SPHERE, radius=np.sqrt(2.0), h=1.0).P == 19
    assert oracle.Mesh(oracle.SPHERE, radius=2.0, h=1.0).P == 33
    # the sphere of the large single-system workload, R/h = 90
    assert oracle.Mesh(oracle.SPHERE, radius=18.0, h=0.2).P == 3053617

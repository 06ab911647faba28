"""GPU: lowest eigenpairs by Chebyshev-filtered subspace iteration
(rsg_eigensolve) against references independent of the library:

- the harmonic oscillator on a cube: the operator separates, so its exact
  discrete spectrum is the sums of LAPACK eigenvalues of the 1-D 8th-order
  operator (the lowest ten: one level, a triple and a six-fold multiplet);
- ARPACK (scipy eigsh) on the FP64 oracle operator for a sphere with wells,
  projectors and a dipole field, and the residuals |H x - lambda x| of the
  returned vectors recomputed by the oracle;
- the one-dimensional lithium table of the paper's few-electron section
  (three soft-Coulomb electrons in 1-D as one particle in 3-D).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as sla
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._oracle_helpers import lowest_eigs
from tests._systems import Pair, wells_system
from workloads import potential_harmonic, potential_soft_coulomb_li, white_noise_states

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
C = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]


def _levels_1d(x, h, v):
    n = len(x)
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(-4, 5):
            if 0 <= i + k < n:
                A[i, i + k] += -0.5 * C[abs(k)] / h ** 2
        A[i, i] += v[i]
    return np.linalg.eigvalsh(A)


def _start(p, S, seed=0):
    """Seeded white-noise starting block on the device."""
    psi = white_noise_states(np.random.default_rng(seed), p.P, S)
    return p.states_to_gpu(psi if p.dtype == torch.complex128 else psi.astype(np.complex64))


@pytest.mark.parametrize("dtype,tol,etol", [(torch.complex128, 1e-8, 1e-9), (torch.complex64, 2e-3, 2e-5)])
def test_harmonic_oscillator_exact_discrete_levels(dtype, tol, etol):
    n, h, omega = 32, 0.3, 0.5
    p = Pair("cube", n, h=h, dtype=dtype)
    p.set_potential(potential_harmonic(p.om.xyz, omega))
    x1 = (np.arange(n) - (n - 1) / 2) * h
    e1 = _levels_1d(x1, h, 0.5 * omega ** 2 * x1 ** 2)[:4]
    lv = np.sort([a + b + c for a in e1 for b in e1 for c in e1])
    want = lv[:10]
    assert lv[10] - lv[9] > 0.3          # a gap after the ten lowest: the block is well defined
    # ten wanted states and four buffer states from the next multiplet
    x = _start(p, 14)
    ev, res, it = p.H.eigensolve(x, nwant=10, max_iter=300, degree=12, tol=tol)
    assert np.all(res[:10] <= tol), (res, it)
    assert np.abs(ev[:10] - want).max() < etol * np.abs(want).max(), (ev, want)
    # the vectors are orthonormal in the h^3 inner product
    got = p.states_from_gpu(x, 14)
    G = h ** 3 * got.conj().T @ got
    assert np.abs(G - np.eye(14)).max() < (1e-12 if dtype == torch.complex128 else 1e-5)


def test_sphere_with_projectors_and_field_against_arpack():
    p, g = wells_system("sphere", radius=4.0, h=0.3, dtype=torch.complex128, seed=11, natoms=3, lmax=1)
    eps, dirv = 0.03, (0.0, 0.6, 0.8)
    p.H.set_field(eps, dirv)
    P = p.P
    op = sla.LinearOperator((P, P), dtype=np.float64, matvec=lambda v: p.O.apply(
        np.asarray(v, dtype=np.complex128).reshape(-1, 1), eps=eps, dir=dirv).real.ravel())
    want = np.sort(sla.eigsh(op, k=6, which="SA", tol=1e-11, ncv=40, v0=np.ones(P),
                             return_eigenvectors=False))[:4]
    x = _start(p, 8, seed=2)
    # four wanted states and four buffer states
    ev, res, it = p.H.eigensolve(x, nwant=4, max_iter=300, degree=12, tol=1e-10)
    assert np.all(res[:4] <= 1e-10), (res, it)
    assert np.abs(ev[:4] - want).max() < 1e-9 * np.abs(want).max(), (ev[:4], want)
    # residuals of the returned pairs, recomputed by the FP64 oracle
    got = p.states_from_gpu(x, 8)
    r = p.O.apply(got, eps=eps, dir=dirv) - got * ev[None, :]
    rn = np.sqrt(p.h ** 3 * (np.abs(r) ** 2).sum(0))
    assert np.abs(rn - res).max() < 1e-10 and rn[:4].max() < 1e-9, (rn, res)


def test_lithium_table():
    with open(os.path.join(HERE, "golden", "li_1d_table.json")) as f:
        gold = json.load(f)
    L, h = 12.0, 0.4
    n = int(round(2 * L / h)) + 1
    p = Pair("cube", n, h=h, dtype=torch.complex128)
    p.set_potential(potential_soft_coulomb_li(p.om.xyz))
    x = _start(p, 8, seed=5)
    ev, res, it = p.H.eigensolve(x, nwant=4, max_iter=300, degree=16, tol=1e-8)
    assert np.all(res[:4] <= 1e-8), (res, it)
    want = np.array(gold["energies_hartree"])
    assert np.all(np.abs(ev[:4] - want) < 1.5 * gold["printed_precision"]), (ev[:4], want)
    # the same discrete operator through the oracle (ARPACK)
    ref = lowest_eigs(p.O, p.P, 6, seed=3, tol=1e-10, ncv=40)[:4]
    assert np.abs(ev[:4] - ref).max() < 1e-7, (ev[:4], ref)


def test_argument_errors():
    p = Pair("cube", 10, h=0.3, dtype=torch.complex128)
    p.set_potential(potential_harmonic(p.om.xyz, 0.5))
    x = _start(p, 2)
    with pytest.raises(rsg.RSGError):
        p.H.eigensolve(x, degree=0)
    with pytest.raises(rsg.RSGError):
        p.H.eigensolve(x, tol=0.0)
    with pytest.raises(rsg.RSGError):
        p.H.eigensolve(x, nwant=3)
    _ = oracle

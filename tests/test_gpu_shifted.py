"""GPU: shifted linear solves (H - z) x = b (rsg_shifted_solve, COCG for the
complex symmetric H - z) against references independent of the library:
dense LAPACK solves with the oracle's assembled FP64 matrix on a small cube
(wells, projectors and a field), and on a larger sphere the true residual
recomputed by the oracle's FP64 operator.  complex64 solves stop near the
FP32 floor of applying H - z (|H| eps_32 |x| / |b|, ~1e-5 for a shift 0.05
from the real axis), so their tolerance is 1e-4."""
import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._oracle_helpers import dense_h
from tests._parity import rel_err
from tests._systems import wells_system
from workloads import white_noise_states

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol,etol", [(torch.complex128, 1e-11, 1e-9), (torch.complex64, 1e-4, 1e-3)])
@pytest.mark.parametrize("z", [-0.4 + 0.05j, 1.3 + 0.1j])
def test_small_cube_against_dense_solve(dtype, tol, etol, z):
    p, g = wells_system("cube", 10, h=0.4, dtype=dtype, seed=12, natoms=2, lmax=1)
    eps, dirv = 0.02, (0.0, 0.0, 1.0)
    p.H.set_field(eps, dirv)
    A = dense_h(p.O, p.P, eps=eps, dir=dirv) - z * np.eye(p.P)
    b = white_noise_states(g, p.P, 3)
    if dtype == torch.complex64:
        b = b.astype(np.complex64).astype(np.complex128)
    want = np.linalg.solve(A, b)
    bd = p.states_to_gpu(b)
    x = torch.zeros_like(bd)
    res, it = p.H.shifted_solve(bd, x, z, max_iter=2000, tol=tol, S=3)
    assert np.all(res <= 10 * tol), (res, it)
    got = p.states_from_gpu(x, 3)
    assert rel_err(got, want) < etol, rel_err(got, want)
    # started at the solution: no iteration needed
    res2, it2 = p.H.shifted_solve(bd, x, z, max_iter=10, tol=max(10 * tol, 1e-9), S=3)
    assert it2 == 0 and np.all(res2 <= max(10 * tol, 1e-9))


def test_sphere_residual_by_oracle():
    p, g = wells_system("sphere", radius=4.0, h=0.3, dtype=torch.complex128, seed=13, natoms=3, lmax=2)
    z = -0.8 + 0.05j
    b = white_noise_states(g, p.P, 4)
    bd = p.states_to_gpu(b)
    x = torch.zeros_like(bd)
    res, it = p.H.shifted_solve(bd, x, z, max_iter=3000, tol=1e-10)
    assert np.all(res <= 1e-9), (res, it)
    got = p.states_from_gpu(x, 4)
    r = b - (p.O.apply(got) - z * got)
    rel = np.sqrt((np.abs(r) ** 2).sum(0) / (np.abs(b) ** 2).sum(0))
    assert rel.max() < 1e-9 and np.abs(rel - res).max() < 1e-11, (rel, res)


def test_argument_errors():
    p, g = wells_system("cube", 8, h=0.4, dtype=torch.complex128, seed=1, natoms=0)
    bd = p.states_to_gpu(white_noise_states(g, p.P, 2))
    with pytest.raises(rsg.RSGError):
        p.H.shifted_solve(bd, bd, 0.1 + 0.1j)          # b and x overlap
    with pytest.raises(rsg.RSGError):
        p.H.shifted_solve(bd, torch.zeros_like(bd), 0.1 + 0.1j, tol=0.0)

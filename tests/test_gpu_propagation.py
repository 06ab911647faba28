"""GPU parity: Taylor-4 exponential, time-step schemes, norms and Cholesky-QR
against the FP64 oracle.

Tolerances: one exponential as H|psi> (1e-12 complex128, 2e-5 complex64).
Propagation accumulates one rounding error per Hamiltonian application, so
n_apply x 1e-13 bounds the complex128 result: 1e-10 for the 400 applications
of the 100-step oscillator run; complex64 runs are kept short (<= 80
applications, bound 2e-5).  Norm drift of smooth complex64 states over 1000
steps with re-orthonormalisation every 50 steps stays below 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from tests._parity import rel_err, round_c64
from tests._systems import ho_system, wells_system
from workloads import rng, wavepacket_params, wavepacket_states, white_noise_states

pytestmark = pytest.mark.gpu

TOL1 = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _smooth_states(p, S, seed=0, radius=1.5):
    g = rng(1, seed)
    psi = wavepacket_states(p.om.xyz, wavepacket_params(g, S, radius))
    psi = p.om.mgs(psi)
    if p.dtype == torch.complex64:
        psi = round_c64(psi)
    return psi


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("inplace", [False, True])
def test_taylor_exponential(dtype, inplace):
    p, g = wells_system("sphere", radius=3.6, h=0.3, dtype=dtype, seed=11, natoms=3, lmax=2, rcut=1.4)
    p.H.set_field(0.03, (0.0, 1.0, 0.0))
    psi = white_noise_states(g, p.P, 5)
    if dtype == torch.complex64:
        psi = round_c64(psi)
    tau = 0.01
    want = p.O.taylor4(psi, tau, eps=0.03, dir=(0.0, 1.0, 0.0))
    x = p.states_to_gpu(psi)
    y = p.H.taylor(x, tau, out=x if inplace else None, S=5)
    torch.cuda.synchronize()
    assert rel_err(p.states_from_gpu(y, 5), want) < TOL1[dtype]


def test_oscillator_cube_100_steps_expmid_c128():
    """32^3 at h=0.3, w=0.5, 4 smooth states, exponential midpoint, dt=0.01."""
    p = ho_system(32, 0.3, torch.complex128)
    psi = _smooth_states(p, 4)
    want, wdrift = p.O.propagate(psi, 100, 0.01, scheme=oracle.EXPMID)
    x = p.states_to_gpu(psi)
    drift = p.H.propagate(x, 100, 0.01, scheme=0)
    torch.cuda.synchronize()
    assert rel_err(p.states_from_gpu(x, 4), want) < 1e-10
    assert np.abs(drift - wdrift).max() < 1e-12


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_etrs_field_projectors_nsub(dtype):
    p, g = wells_system("sphere", radius=3.3, h=0.3, dtype=dtype, seed=12, natoms=2, lmax=1)
    psi = _smooth_states(p, 3, seed=1, radius=1.0)
    eps = g.uniform(-0.05, 0.05, 5)
    want, _ = p.O.propagate(psi, 5, 0.02, scheme=oracle.ETRS, nsub=2, eps=eps, dir=(1, 1, 0))
    x = p.states_to_gpu(psi)
    p.H.propagate(x, 5, 0.02, scheme=1, nsub=2, eps=eps, dir=(1, 1, 0))
    torch.cuda.synchronize()
    tol = 1e-10 if dtype == torch.complex128 else 2e-5
    assert rel_err(p.states_from_gpu(x, 3), want) < tol


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_orthonormalize_matches_mgs(dtype):
    p, g = wells_system("cube", 21, h=0.3, dtype=dtype, seed=13, natoms=0)
    S = 7
    psi = white_noise_states(g, p.P, S) * np.sqrt(1.0 / (p.h ** 3 * p.P))
    if dtype == torch.complex64:
        psi = round_c64(psi)
    want = p.om.mgs(psi)
    n2_want = p.om.norms2(psi)
    x = p.states_to_gpu(psi)
    n2 = p.H.orthonormalize(x, S=S)
    got = p.states_from_gpu(x, S)
    assert np.abs(n2 - n2_want).max() < 1e-12 * n2_want.max()
    assert rel_err(got, want) < (1e-12 if dtype == torch.complex128 else 2e-5)
    G = p.h ** 3 * got.conj().T @ got
    assert np.abs(G - np.eye(S)).max() < (1e-12 if dtype == torch.complex128 else 1e-5)


def test_gs_drift_matches_oracle_c128():
    p = ho_system(20, 0.4, torch.complex128)
    psi = _smooth_states(p, 3)
    want, wdrift = p.O.propagate(psi, 12, 0.02, scheme=oracle.ETRS, gs_every=4)
    x = p.states_to_gpu(psi)
    drift = p.H.propagate(x, 12, 0.02, scheme=1, gs_every=4)
    assert rel_err(p.states_from_gpu(x, 3), want) < 1e-10
    assert np.abs(drift - wdrift).max() < 1e-12


def test_norm_drift_1000_steps_c64():
    """Smooth complex64 states, 1000 ETRS steps, FP64 Cholesky-QR every 50:
    the drift just before each re-orthonormalisation stays below 1e-6."""
    p = ho_system(32, 0.3, torch.complex64)
    psi = _smooth_states(p, 4)
    x = p.states_to_gpu(psi)
    drift = p.H.propagate(x, 1000, 0.01, scheme=1, gs_every=50)
    assert np.all(drift < 1e-6), drift
    # and the FP64 norms after the last re-orthonormalisation
    n2 = p.H.norms(x, S=4)
    assert np.abs(n2 - 1).max() < 1e-6


def test_norms_against_numpy():
    p, g = wells_system("sphere", radius=2.5, h=0.3, dtype=torch.complex64, natoms=0)
    psi = round_c64(white_noise_states(g, p.P, 9))
    x = p.states_to_gpu(psi)
    n2 = p.H.norms(x, S=9)
    want = p.h ** 3 * np.sum(np.abs(psi) ** 2, axis=0)
    assert np.abs(n2 - want).max() < 1e-12 * want.max()


def test_projector_coefficients_on_a_side_stream_give_the_same_step():
    """Option proj_overlap: the coefficients run on an internal side stream
    next to the stencil; the step is bit-for-bit the one on one stream."""
    import paper_1501_05654_gb300 as rsg_
    from tests._systems import wells_system
    from tests._parity import round_c64
    from workloads import white_noise_states
    p, g = wells_system("sphere", 0, radius=4.0, h=0.2, dtype=torch.complex64, seed=2, natoms=3, lmax=1)
    psi = round_c64(white_noise_states(g, p.P, 16))
    p.H.set_option("kernel", 7)      # the stencil that leaves the projector terms to the scatter
    x = p.states_to_gpu(psi)
    y = x.clone()
    p.H.propagate(x, 3, 0.01, scheme=rsg_.ETRS, S=16)
    assert p.H.get_option("last_kernel") == 7
    p.H.set_option("proj_overlap", 1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p.H.propagate(y, 3, 0.01, scheme=rsg_.ETRS, S=16)
    s.synchronize()
    assert p.H.get_option("proj_overlap") == 1
    assert torch.equal(x, y)

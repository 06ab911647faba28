"""GPU: the mask absorber (rsg_absorber_set; after every time step each state
is multiplied by M(r), keeping the bounded part of Eq. (mask_split)) against
the FP64 oracle propagating one step at a time followed by the same pointwise
product; the absorbed norm; clearing the mask; and the refusals of the
calls whose adjoint or batch does not include it."""
import numpy as np
import pytest
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err
from tests._systems import Pair
from workloads import potential_harmonic, rng, wavepacket_params, wavepacket_states

pytestmark = pytest.mark.gpu


def _mask(xyz, r0, r1):
    """1 inside r0, cos^2 down to 0 at r1, 0 beyond."""
    r = np.linalg.norm(xyz, axis=1)
    m = np.ones(len(r))
    mid = (r > r0) & (r < r1)
    m[mid] = np.cos(0.5 * np.pi * (r[mid] - r0) / (r1 - r0)) ** 2
    m[r >= r1] = 0.0
    return m


def _system():
    p = Pair("cube", 24, h=0.3, dtype=torch.complex128)
    p.set_potential(potential_harmonic(p.om.xyz, 0.1))
    psi = wavepacket_states(p.om.xyz, wavepacket_params(rng(9), 3, 1.5))
    psi = p.om.mgs(psi)
    return p, psi


def test_absorber_matches_oracle_step_then_mask():
    p, psi = _system()
    M = _mask(p.om.xyz, 1.5, 3.3)
    p.H.set_absorber(p.to_lib(M))
    x = p.states_to_gpu(psi)
    p.H.propagate(x, 30, 0.05, scheme=rsg.ETRS)
    ref = p.O.propagate_masked(psi, 30, 0.05, M, scheme=oracle.ETRS)
    got = p.states_from_gpu(x, 3)
    assert rel_err(got, ref) < 1e-10, rel_err(got, ref)
    n2 = p.h ** 3 * (np.abs(got) ** 2).sum(0)
    assert np.all(n2 < 1.0 - 1e-6) and np.all(n2 > 0.0), n2     # some charge absorbed
    # cleared: one plain step again
    p.H.set_absorber(None)
    y = p.states_to_gpu(psi)
    p.H.propagate(y, 1, 0.05, scheme=rsg.ETRS)
    want, _ = p.O.propagate(psi, 1, 0.05, scheme=oracle.ETRS)
    assert rel_err(p.states_from_gpu(y, 3), want) < 1e-12


def test_absorber_refusals():
    p, psi = _system()
    with pytest.raises(rsg.RSGError):
        p.H.set_absorber(np.full(p.P, 1.5))
    p.H.set_absorber(np.ones(p.P))
    a = torch.from_numpy(p.to_lib(psi[:, 0])).cuda()
    with pytest.raises(rsg.RSGError):
        p.H.control_gradient(a, a, np.zeros(3), 0.05)
    H64 = rsg.Hamiltonian(p.lm, torch.complex64)
    H64.set_potential(np.zeros(p.P))
    H64.set_absorber(np.ones(p.P))
    with pytest.raises(rsg.RSGError):
        rsg.Batch([H64], [1])

"""GPU failure paths, made without faulting, trapping or hanging the GPU:

- a bounded device wait that runs out (an mbarrier phase that nothing
  completes) is reported as RSG_ERR_TIMEOUT within milliseconds, and the
  Hamiltonian and the context stay usable;
- a NaN in the input block is caught by the FP64 Gram check of the
  re-orthonormalisation (RSG_ERR_NONFINITE);
- a simulated allocation failure surfaces as RSG_ERR_OOM from the call that
  needed the memory, and the next call succeeds.
"""
import time

import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err
from tests._systems import ho_system
from workloads import rng, white_noise_states

pytestmark = pytest.mark.gpu


def _check_apply(p, S=3, seed=0):
    psi = white_noise_states(rng(50, seed), p.P, S)
    y = p.H.apply(p.states_to_gpu(psi), S=S)
    assert rel_err(p.states_from_gpu(y, S), p.O.apply(psi)) < 1e-12


def test_bounded_wait_times_out_and_context_survives():
    p = ho_system(n=12, dtype=torch.complex128)
    lib = rsg.load()
    t0 = time.perf_counter()
    assert lib.rsg_selftest_bounded_wait(p.H._h, 4096, None) == -5
    assert time.perf_counter() - t0 < 5.0
    assert b"bounded device wait" in lib.rsg_last_error()
    # the status was read and cleared; the Hamiltonian still applies exactly
    _check_apply(p)
    assert lib.rsg_selftest_bounded_wait(p.H._h, 1, None) == -5
    _check_apply(p, seed=1)


def test_nan_input_is_reported_nonfinite():
    p = ho_system(n=12, dtype=torch.complex128)
    psi = p.om.mgs(white_noise_states(rng(51), p.P, 4))
    psi[17, 2] = np.nan
    x = p.states_to_gpu(psi)
    with pytest.raises(rsg.RSGError, match="not finite"):
        p.H.orthonormalize(x, S=4)
    with pytest.raises(rsg.RSGError, match="not finite"):
        p.H.propagate(p.states_to_gpu(psi), 2, 0.01, gs_every=1, S=4)
    _check_apply(p)


def test_simulated_allocation_failure():
    p = ho_system(n=12, dtype=torch.complex64)
    lib = rsg.load()
    psi = p.states_to_gpu(white_noise_states(rng(52), p.P, 2).astype(np.complex64))
    out = torch.zeros_like(psi)
    assert lib.rsg_debug_fail_allocations(1) == 0
    try:
        # the first Taylor stage needs the Hamiltonian's work blocks
        rc = lib.rsg_taylor_apply(p.H._h, psi.data_ptr(), out.data_ptr(), 2, psi.shape[1], 0.01, None)
        assert rc == -2, rc
        assert b"memory" in lib.rsg_last_error().lower()
    finally:
        lib.rsg_debug_fail_allocations(0)
    p.H.taylor(psi, 0.01, out=out, S=2)
    assert torch.isfinite(torch.view_as_real(out)).all()

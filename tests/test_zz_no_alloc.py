"""The allocation-free norm entry point, called through the C ABI, agrees
with the allocating rsg_state_norms on two calls in a row.

Collected last on purpose: if it fails, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from paper_1501_05654_gb300 import rsg as binding
from workloads import rng, white_noise_states

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_noalloc_norms_match_allocating_entry_point(dtype):
    rsg.build()
    lib = binding.load()
    g = rng(55)
    mesh = rsg.Mesh(rsg.SPHERE, radius=3.7, spacing=0.3)
    H = rsg.Hamiltonian(mesh, dtype)
    S = 7
    npdt = np.complex64 if dtype == torch.complex64 else np.complex128
    ld = rsg.padded_ld(S, dtype)
    out = torch.full((S,), -1.0, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        psi = torch.zeros((mesh.P, ld), dtype=dtype)
        psi[:, :S] = torch.from_numpy(white_noise_states(g, mesh.P, S, dtype=npdt) * (call + 1))
        psi = psi.cuda()
        want = H.norms(psi, S=S)                       # rsg_state_norms
        st = lib.rsg_state_norms_noalloc(H._h, C.c_void_p(psi.data_ptr()), S, ld,
                                         C.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.rsg_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0), (call, got, want)


def test_noalloc_rejects_more_states_than_its_workspace():
    rsg.build()
    lib = binding.load()
    mesh = rsg.Mesh(rsg.CUBE, 6, spacing=0.3)
    H = rsg.Hamiltonian(mesh, torch.complex128)
    psi = torch.zeros((mesh.P, 130), dtype=torch.complex128, device="cuda")
    out = torch.zeros(130, dtype=torch.float64, device="cuda")
    st = lib.rsg_state_norms_noalloc(H._h, C.c_void_p(psi.data_ptr()), 130, 130,
                                     C.c_void_p(out.data_ptr()), None)
    assert st == -4
    assert b"128" in lib.rsg_last_error()


def test_noalloc_large_block_while_library_allocations_fail():
    """373,248 points (more than 128 reduction blocks of 2048 points, so the
    block count is clamped to the array's 128 rows) and 128 states, on a
    Hamiltonian that has never allocated: two calls in a row succeed while
    every allocation the library attempts is made to fail, and their norms
    equal those of the allocating rsg_state_norms (called afterwards) and the
    FP64 oracle's."""
    import oracle
    rsg.build()
    lib = binding.load()
    mesh = rsg.Mesh(rsg.CUBE, 72, spacing=0.25)
    assert mesh.P > 128 * 2048
    H = rsg.Hamiltonian(mesh, torch.complex64)
    S = 128
    g = rng(56)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.full((S,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        host = white_noise_states(g, mesh.P, S, dtype=np.complex64) * (call + 1)
        psi = torch.from_numpy(host).cuda()
        torch.cuda.synchronize()
        assert lib.rsg_debug_fail_allocations(1 << 20) == 0
        try:
            st = lib.rsg_state_norms_noalloc(H._h, C.c_void_p(psi.data_ptr()), S, S,
                                             C.c_void_p(out.data_ptr()), stream)
            torch.cuda.synchronize()
        finally:
            assert lib.rsg_debug_fail_allocations(0) == 0
        assert st == 0, lib.rsg_last_error()
        got = out.cpu().numpy()
        want = H.norms(psi, S=S)                       # rsg_state_norms, allocating
        assert np.allclose(got, want, rtol=1e-12, atol=0), call
        om = oracle.Mesh(oracle.CUBE, 72, h=0.25)
        ref = om.norms2(host.astype(np.complex128))    # same points, any order: a sum over all of them
        assert np.allclose(got, ref, rtol=1e-9, atol=0), call

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

"""Checkpoint and resume of state blocks (rsg_states_save / rsg_states_load)
with host buffers, no GPU: the file is a standard .npy array of the live
columns (numpy reads it as is), the padding columns come back as zeros, the
metadata round-trips, and mismatched files are refused."""
import ctypes
import json

import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from workloads import rng, white_noise_states


@pytest.mark.parametrize("dtype,npdt,ld", [(torch.complex64, np.complex64, 4), (torch.complex128, np.complex128, 3)])
def test_round_trip_host(tmp_path, dtype, npdt, ld):
    m = rsg.Mesh(rsg.BOX, (7, 5, 6), spacing=0.3)
    H = rsg.Hamiltonian(m, dtype)
    S = 3
    psi = np.zeros((m.P, ld), dtype=npdt)
    psi[:, :S] = white_noise_states(rng(70), m.P, S).astype(npdt)
    psi[:, S:] = 7.0                                   # padding: not saved
    path = tmp_path / "psi.npy"
    H.save_states(path, psi, S=S, step=1234, time=61.7, seed=2 ** 63 + 5)
    on_disk = np.load(path)
    assert on_disk.dtype == npdt and on_disk.shape == (m.P, S)
    assert np.array_equal(on_disk, psi[:, :S])
    meta = json.loads((tmp_path / "psi.npy.json").read_text())
    assert meta["points"] == m.P and meta["states"] == S and meta["step"] == 1234
    back = np.full((m.P, ld), 9.0, dtype=npdt)
    step, t, seed = H.load_states(path, back, S=S)
    assert (step, t, seed) == (1234, 61.7, 2 ** 63 + 5)
    assert np.array_equal(back[:, :S], psi[:, :S]) and np.all(back[:, S:] == 0)


def test_mismatches_are_refused(tmp_path):
    m = rsg.Mesh(rsg.CUBE, 5, spacing=0.3)
    H64 = rsg.Hamiltonian(m, torch.complex64)
    H128 = rsg.Hamiltonian(m, torch.complex128)
    psi = white_noise_states(rng(71), m.P, 2).astype(np.complex64)
    path = tmp_path / "a.npy"
    H64.save_states(path, psi, S=2)
    with pytest.raises(rsg.RSGError):                  # other dtype
        H128.load_states(path, np.zeros((m.P, 2), np.complex128), S=2)
    with pytest.raises(rsg.RSGError):                  # other state count
        H64.load_states(path, np.zeros((m.P, 4), np.complex64), S=4)
    other = rsg.Hamiltonian(rsg.Mesh(rsg.CUBE, 6, spacing=0.3), torch.complex64)
    with pytest.raises(rsg.RSGError):                  # other mesh
        other.load_states(path, np.zeros((other.mesh.P, 2), np.complex64), S=2)
    with pytest.raises(rsg.RSGError):                  # missing file
        H64.load_states(tmp_path / "none.npy", np.zeros((m.P, 2), np.complex64), S=2)
    bad = tmp_path / "bad.npy"
    bad.write_bytes(b"not a numpy file at all")
    with pytest.raises(rsg.RSGError):
        H64.load_states(bad, np.zeros((m.P, 2), np.complex64), S=2)
    # a .npy without the metadata file: the data loads, the metadata request fails
    np.save(tmp_path / "plain.npy", psi)
    with pytest.raises(rsg.RSGError):
        H64.load_states(tmp_path / "plain.npy", np.zeros((m.P, 2), np.complex64), S=2)
    lib = rsg.load()
    out = np.zeros((m.P, 2), np.complex64)
    assert lib.rsg_states_load(H64._h, str(tmp_path / "plain.npy").encode(), out.ctypes.data_as(ctypes.c_void_p),
                               2, 2, 0, None, None, None) == 0
    assert np.array_equal(out, psi)

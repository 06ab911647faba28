"""GPU: resuming a propagation from a checkpoint (rsg_states_save /
rsg_states_load with device buffers) continues it bit for bit."""
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._systems import ho_system
from workloads import rng, wavepacket_params, wavepacket_states

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_resume_continues_bit_for_bit(tmp_path, dtype):
    p = ho_system(n=16, dtype=dtype)
    S = 3
    psi = p.om.mgs(wavepacket_states(p.om.xyz, wavepacket_params(rng(72), S, 1.5)))
    x = p.states_to_gpu(psi)
    p.H.propagate(x, 10, 0.01, scheme=rsg.ETRS, S=S)
    path = tmp_path / "ck.npy"
    p.H.save_states(path, x, S=S, step=10, time=0.1, seed=72)
    y = x.clone()
    p.H.propagate(y, 10, 0.01, scheme=rsg.ETRS, S=S)
    z = torch.full_like(x, 3.0)
    step, t, seed = p.H.load_states(path, z, S=S)
    assert (step, t, seed) == (10, 0.1, 72)
    assert torch.equal(z[:, :S], x[:, :S]) and not z[:, S:].any()
    p.H.propagate(z, 10, 0.01, scheme=rsg.ETRS, S=S)
    assert torch.equal(y, z)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_save_after_propagation_on_a_side_stream(tmp_path, dtype):
    """A propagation enqueued on a non-blocking stream and a save issued
    right after it, with no synchronisation by the caller: the checkpoint
    holds the propagated block, and a load followed by work on another side
    stream sees the restored values."""
    p = ho_system(n=24, dtype=dtype)
    S = 4
    psi = p.om.mgs(wavepacket_states(p.om.xyz, wavepacket_params(rng(73), S, 1.5)))
    x = p.states_to_gpu(psi)
    torch.cuda.synchronize()
    s1 = torch.cuda.Stream()
    with torch.cuda.stream(s1):
        p.H.propagate(x, 40, 0.01, scheme=rsg.ETRS, S=S, want_drift=False, stream=s1)
    path = tmp_path / "side.npy"
    p.H.save_states(path, x, S=S, step=40, time=0.4, seed=73)
    torch.cuda.synchronize()
    want = x.clone()
    z = torch.zeros_like(x)
    p.H.load_states(path, z, S=S)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        w = z * 1.0
    torch.cuda.synchronize()
    assert torch.equal(w[:, :S], want[:, :S])


def test_failed_save_keeps_the_previous_checkpoint(tmp_path):
    """The .npy and .json files are written under temporary names and moved
    into place; a save whose temporary file cannot be created (a folder of
    that name stands in the way) fails and leaves the checkpoint already at
    the path unchanged."""
    import os
    p = ho_system(n=12, dtype=torch.complex128)
    x = p.states_to_gpu(p.om.mgs(wavepacket_states(p.om.xyz, wavepacket_params(rng(74), 2, 1.5))))
    path = tmp_path / "a.npy"
    p.H.save_states(path, x, S=2, step=1, time=0.0, seed=1)
    before = (path.read_bytes(), (tmp_path / "a.npy.json").read_bytes())
    (tmp_path / f"a.npy.tmp{os.getpid()}").mkdir()
    with pytest.raises(rsg.RSGError):
        p.H.save_states(path, x * 2, S=2, step=2, time=0.1, seed=2)
    assert (path.read_bytes(), (tmp_path / "a.npy.json").read_bytes()) == before

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

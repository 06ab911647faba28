"""GPU: projectors given as sampled values (rsg_projectors_set_raw) against
the FP64 oracle fed the same values (orc_ham_set_projectors_raw, pinned by
the small-problem spectrum and by reproducing the oracle's own sampled
set):

- scattered point clusters with 1, 5 and 9 projectors per atom and full
  symmetric couplings, both precisions, through the default stencil path
  (separate projector scatter) and the one-thread-per-value kernel (fused
  in the epilogue);
- the raw form of the library's own Gaussian projectors equals the
  analytic call;
- argument errors.
"""
import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err, round_c64
from tests._systems import Pair
from workloads import gaussian_wells, potential_wells, rng, white_noise_states

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _lib_index(p):
    """oracle point index -> library point index"""
    inv = np.empty(p.P, dtype=np.int64)
    inv[p.idx] = np.arange(p.P)
    return inv


def _raw_set(p, g, nprojs, radius=1.1):
    """Clusters of points around random centres (oracle order) with random
    values under a smooth envelope, and random symmetric couplings."""
    xyz = p.om.xyz
    pts, vals, hs = [], [], []
    for k in nprojs:
        c = xyz[g.integers(p.P)]
        r2 = ((xyz - c) ** 2).sum(1)
        sel = np.nonzero(r2 <= radius ** 2)[0]
        sel = sel[g.random(len(sel)) < 0.8]          # holes: an arbitrary point set
        env = np.exp(-r2[sel] / 0.8)
        pts.append(sel)
        vals.append(g.standard_normal((len(sel), k)) * env[:, None])
        A = g.standard_normal((k, k))
        hs.append(0.25 * (A + A.T))
    return pts, vals, hs


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("kernel", [None, 1, 0])
def test_raw_projectors_match_oracle(dtype, kernel):
    p = Pair("sphere", radius=3.5, h=0.3, dtype=dtype)
    g = rng(43, 0 if kernel is None else kernel + 1)
    p.set_potential(potential_wells(p.om.xyz, *gaussian_wells(g, 3, 2.0)))
    pts, vals, hs = _raw_set(p, g, (1, 5, 9))
    if dtype == torch.complex64:
        vals = [v.astype(np.float32).astype(np.float64) for v in vals]   # the FP32 path stores float32
    p.O.set_projectors_raw(pts, vals, hs)
    lib = _lib_index(p)
    p.H.set_projectors_raw([lib[s] for s in pts], vals, hs)
    if kernel is not None:
        p.H.set_option("kernel", kernel)
    S = 5
    psi = white_noise_states(g, p.P, S)
    if dtype == torch.complex64:
        psi = round_c64(psi)
    y = p.H.apply(p.states_to_gpu(psi), S=S)
    if kernel is not None:
        assert p.H.get_option("last_kernel") == kernel
    err = rel_err(p.states_from_gpu(y, S), p.O.apply(psi))
    assert err < TOL[dtype], err


def test_raw_form_of_the_analytic_projectors():
    p = Pair("sphere", radius=3.2, h=0.3, dtype=torch.complex128)
    g = rng(44)
    p.set_potential(potential_wells(p.om.xyz, *gaussian_wells(g, 2, 2.0)))
    cen = [[0.3, -0.2, 0.4], [-0.8, 0.6, 0.1]]
    hm = [np.diag(g.uniform(-1, 1, 4)), np.diag(g.uniform(-1, 1, 9))]
    p.set_projectors(cen, [1.4, 1.7], [1, 2], [0.35, 0.42], hm)
    S = 3
    x = p.states_to_gpu(white_noise_states(g, p.P, S))
    want = p.states_from_gpu(p.H.apply(x, S=S), S)
    lib = _lib_index(p)
    pts, vals = zip(*(p.O.atom(a) for a in range(2)))
    p.H.set_projectors_raw([lib[s] for s in pts], [v.T for v in vals], hm)
    got = p.states_from_gpu(p.H.apply(x, S=S), S)
    assert rel_err(got, want) < 1e-14


def test_raw_projector_errors():
    p = Pair("cube", 8, h=0.3, dtype=torch.complex64)
    p.H.set_potential(np.zeros(p.P))
    ok = [np.arange(5)]
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors_raw([np.array([0, 3, 3])], [np.ones((3, 1))], [np.eye(1)])      # repeated point
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors_raw([np.array([0, p.P])], [np.ones((2, 1))], [np.eye(1)])       # outside the mesh
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors_raw(ok, [np.ones((5, 10))], [np.eye(10)])                       # more than 9
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors_raw(ok, [np.ones((5, 2))], [np.array([[1.0, 0.5], [0.4, 1.0]])])  # asymmetric
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors_raw(ok, [np.full((5, 1), np.nan)], [np.eye(1)])
    # a valid set, then removal
    p.H.set_projectors_raw(ok, [np.ones((5, 1))], [np.eye(1)])
    p.H.set_projectors_raw([], [], [])
    x = p.states_to_gpu(np.ones((p.P, 1), dtype=np.complex128))
    y = p.H.apply(x, S=1)
    assert torch.isfinite(torch.view_as_real(y)).all()

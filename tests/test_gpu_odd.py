"""GPU: the antisymmetric-image boundary of cube and box meshes
(rsg_mesh_set_boundary with RSG_BC_ODD) against the FP64 oracle's image
walls and against the closed form that the image rule makes exact:

- the application with wells, projectors and a field, both precisions;
- products of sines are eigenvectors of -1/2 lap with eigenvalues
  sum_d sigma(pi m_d / (n_d + 1)) / (2 h^2), sigma(phi) = -c0 - 2 sum_k c_k cos(k phi);
- the library's eigensolver on an empty box returns those closed-form
  levels (the particle in a box, converging at the stencil's order);
- complex scaling on image walls: e^{-2i theta} E + v0 on the same modes;
- batches refuse image-wall meshes.
"""
import itertools

import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err, round_c64
from tests._systems import Pair
from workloads import (gaussian_wells, potential_wells, projector_atoms, rng, white_noise_states)

pytestmark = pytest.mark.gpu

C = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _sigma(phi):
    return -C[0] - 2 * sum(C[k] * np.cos(k * phi) for k in range(1, 5))


def _modes(p, n3, modes):
    """Sine products (oracle order) and their closed-form levels of -1/2 lap."""
    f, E = [], []
    for md in modes:
        v = np.ones(p.P)
        for d in range(3):
            v = v * np.sin(np.pi * md[d] * (p.om.ijk[:, d] - p.om.ijk[:, d].min() + 1) / (n3[d] + 1))
        f.append(v)
        E.append(sum(_sigma(np.pi * md[d] / (n3[d] + 1)) for d in range(3)) / (2 * p.h ** 2))
    return np.array(f).T.astype(np.complex128), np.array(E)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("shape,n", [("box", (13, 9, 11)), ("cube", 12)])
def test_odd_apply_matches_oracle(dtype, shape, n):
    p = Pair(shape, n, h=0.3, dtype=dtype, odd=True)
    g = rng(60, 0 if shape == "box" else 1)
    half = 0.5 * 8 * 0.3
    p.set_potential(potential_wells(p.om.xyz, *gaussian_wells(g, 2, 0.0, cube_half=half)))
    p.set_projectors(*projector_atoms(g, 2, 1.0, 1, cube_half=half))
    eps, dirv = 0.03, (0.6, 0.0, 0.8)
    p.H.set_field(eps, dirv)
    for S in (1, 3):
        psi = white_noise_states(g, p.P, S)
        if dtype == torch.complex64:
            psi = round_c64(psi)
        y = p.H.apply(p.states_to_gpu(psi), S=S)
        assert p.H.get_option("last_kernel") == 1
        err = rel_err(p.states_from_gpu(y, S), p.O.apply(psi, eps=eps, dir=dirv))
        assert err < TOL[dtype], err


def test_odd_sine_modes_are_exact_eigenvectors():
    n3 = (12, 9, 10)
    p = Pair("box", n3, h=0.35, dtype=torch.complex128, odd=True)
    p.H.set_potential(np.zeros(p.P))
    f, E = _modes(p, n3, [(1, 1, 1), (2, 1, 3), (5, 4, 2), (12, 9, 10)])
    y = p.states_from_gpu(p.H.apply(p.states_to_gpu(f), S=4), 4)
    for s in range(4):
        assert np.abs(y[:, s] - E[s] * f[:, s]).max() < 1e-12 * abs(E[s]) * np.abs(f[:, s]).max()


def test_odd_box_eigensolver_gives_closed_form_levels():
    n3 = (14, 11, 9)
    h = 0.3
    p = Pair("box", n3, h=h, dtype=torch.complex128, odd=True)
    p.H.set_potential(np.zeros(p.P))
    lv = np.sort([sum(_sigma(np.pi * m[d] / (n3[d] + 1)) for d in range(3)) / (2 * h * h)
                  for m in itertools.product(range(1, 5), repeat=3)])
    x = p.states_to_gpu(white_noise_states(rng(61), p.P, 8))
    ev, res, it = p.H.eigensolve(x, nwant=4, max_iter=400, degree=16, tol=1e-9)
    assert np.all(res[:4] <= 1e-9), (res, it)
    assert np.abs(ev[:4] - lv[:4]).max() < 1e-9 * lv[3], (ev[:4], lv[:4])
    # and the ground level is the continuum particle in a box to the stencil's accuracy
    L = [(k + 1) * h for k in n3]
    e0 = 0.5 * np.pi ** 2 * sum(1 / Li ** 2 for Li in L)
    assert abs(ev[0] - e0) < 1e-4 * e0


def test_odd_complex_scaling_rotates_the_closed_form():
    n3 = (10, 10, 10)
    theta, v0 = 0.4, 0.7
    p = Pair("cube", 10, h=0.35, dtype=torch.complex128, odd=True)
    p.H.set_complex_scaling(theta, np.full(p.P, v0 + 0j))
    f, E = _modes(p, n3, [(1, 1, 1), (3, 2, 1), (4, 4, 7)])
    y = p.states_from_gpu(p.H.apply(p.states_to_gpu(f), S=3), 3)
    assert p.H.get_option("last_kernel") == 6
    for s in range(3):
        want = np.exp(-2j * theta) * E[s] + v0
        assert np.abs(y[:, s] - want * f[:, s]).max() < 1e-12 * abs(want) * np.abs(f[:, s]).max()


def test_batch_refuses_image_walls():
    p = Pair("cube", 10, h=0.3, dtype=torch.complex64, odd=True)
    p.H.set_potential(np.zeros(p.P))
    with pytest.raises(rsg.RSGError):
        rsg.Batch([p.H], [2])

"""Full-size checks in the launch configuration the benchmark uses: properties
that hold at any size, and sampled comparisons.

- Large cube (192^3, h = 0.18, 128 smooth complex64 states, 64 atoms x 9
  projectors): norm drift over 50 ETRS steps below 1e-6 and orthonormality
  after the Cholesky-QR, checked by an FP64 Gram matrix and by the library's
  own FP64 norms.
- Control workload's mesh and operator (64^3, h = 0.3, double well, 4 ETRS
  substeps per 0.05 au interval, 200 intervals): adjoint gradient against central differences of the library's
  own objective on seeded components, from the ground to the first excited
  state (exact discrete eigenvectors of the separable operator).
- Batch of 256 uneven systems: a seeded sample of systems against their
  single-system propagation.
"""
import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from workloads import (batch_systems, control_field, gaussian_wells, potential_double_well,
                       potential_wells, projector_atoms, rng)

pytestmark = pytest.mark.gpu


def test_large_cube_norm_drift_and_orthonormality():
    g = rng(5)
    m = rsg.Mesh(rsg.CUBE, 192, spacing=0.18)
    half = 0.5 * 191 * 0.18
    c, d, w = gaussian_wells(g, 64, 0.0, cube_half=half - 3.0)
    H = rsg.Hamiltonian(m, torch.complex64)
    H.set_potential(potential_wells(m.xyz, c, d, w))
    cen, rc, lm, beta, hm = projector_atoms(g, 64, 3.0, 2, cube_half=half - 3.0)
    cen[:] = c
    H.set_projectors(cen, rc, lm, beta, hm)
    xyz = torch.from_numpy(m.xyz).to("cuda", torch.float32)
    S = 128
    x = torch.empty((m.P, S), dtype=torch.complex64, device="cuda")
    cs = torch.from_numpy(g.uniform(-0.5 * half, 0.5 * half, (S, 3))).to("cuda", torch.float32)
    ks = torch.from_numpy(g.uniform(-0.5, 0.5, (S, 3))).to("cuda", torch.float32)
    sg = torch.from_numpy(g.uniform(1.0, 2.0, S)).to("cuda", torch.float32)
    for s in range(S):
        r2 = ((xyz - cs[s]) ** 2).sum(1)
        x[:, s] = torch.polar(torch.exp(-r2 / (4 * sg[s] ** 2)), xyz @ ks[s])
    H.orthonormalize(x)
    drift = H.propagate(x, 50, 0.01, scheme=rsg.ETRS, gs_every=50)
    assert np.all(drift < 1e-6), drift.max()
    # after the re-orthonormalisation at step 50: h^3 X^H X = I, summed in FP64
    G = torch.zeros((S, S), dtype=torch.complex128, device="cuda")
    for p0 in range(0, m.P, 1 << 20):
        xc = x[p0:p0 + (1 << 20)].to(torch.complex128)
        G += xc.conj().T @ xc
    G *= m.h ** 3
    eye = torch.eye(S, dtype=torch.complex128, device="cuda")
    assert (G - eye).abs().max().item() < 1e-5
    assert np.abs(H.norms(x) - 1).max() < 1e-5
    # the library's FP64 norms of x_a + x_b and x_a + i x_b give 2 + 2 Re/Im <x_a|x_b>
    for a, b in ((0, 1), (5, 77), (126, 127)):
        pair = rsg.empty_states(m.P, 1)
        for ph in (1.0, 1.0j):
            pair[:, 0] = x[:, a] + ph * x[:, b]
            nn = H.norms(pair, S=1)[0]
            assert abs(nn - 2.0) < 1e-5, (a, b, ph, nn)


def _dw_eigvecs_1d(n, h, pot):
    """Lowest eigenvectors of the 1-D operator -1/2 d2 + v on n points with
    zero values outside (the 8th-order second difference), via LAPACK."""
    c = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(-4, 5):
            j = i + k
            if 0 <= j < n:
                A[i, j] += -0.5 * c[abs(k)] / h ** 2
        A[i, i] += pot[i]
    return np.linalg.eigh(A)


def test_control_workload_full_mesh_against_finite_differences():
    n, h = 64, 0.3
    m = rsg.Mesh(rsg.CUBE, n, spacing=h)
    H = rsg.Hamiltonian(m, torch.complex128)
    H.set_potential(potential_double_well(m.xyz, 0.02, 2.0, 0.5))
    ijk = m.ijk - m.ijk.min(0)
    assert (ijk.max(0) == n - 1).all()
    x1 = m.origin[0] + m.h * (np.arange(n) + m.ijk[:, 0].min())
    y1 = m.origin[1] + m.h * (np.arange(n) + m.ijk[:, 1].min())
    assert np.allclose(m.origin, m.origin[0]) and np.allclose(m.ijk.min(0), m.ijk.min())
    # the operator separates: zero values outside the cube in every direction
    _, vx = _dw_eigvecs_1d(n, m.h, 0.02 * (x1 ** 2 - 4.0) ** 2)
    _, vy = _dw_eigvecs_1d(n, m.h, 0.5 * 0.5 ** 2 * y1 ** 2)
    # ground state phi_0 = vx0 vy0 vz0, first excited phi_1 = vx1 vy0 vz0
    i, j, k = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    phi0 = vx[i, 0] * vy[j, 0] * vy[k, 0] / h ** 1.5
    phi1 = vx[i, 1] * vy[j, 0] * vy[k, 0] / h ** 1.5
    psi0 = torch.from_numpy(phi0.astype(np.complex128)).cuda()
    tgt = torch.from_numpy(phi1.astype(np.complex128)).cuda()
    nsteps, dt = 200, 0.05
    eps = control_field(rng(4), nsteps, dt)
    J, grad = H.control_gradient(psi0, tgt, eps, dt, scheme=rsg.ETRS, nsub=4, checkpoint_every=50)
    assert 0 <= J <= 1
    ks = rng(4, 1).choice(nsteps, 5, replace=False)
    eta = 1e-5
    for kk in ks:
        e1, e2 = eps.copy(), eps.copy()
        e1[kk] += eta
        e2[kk] -= eta
        fd = (H.control_gradient(psi0, tgt, e1, dt, scheme=rsg.ETRS, nsub=4)[0]
              - H.control_gradient(psi0, tgt, e2, dt, scheme=rsg.ETRS, nsub=4)[0]) / (2 * eta)
        assert abs(fd - grad[kk]) < 1e-4 * np.abs(grad).max(), (kk, fd, grad[kk])


def test_batch_full_size_sample_against_single_systems():
    g = rng(3)
    ns, Ss, nas = batch_systems(g, 256)
    hams, psis = [], []
    gen = torch.Generator(device="cuda").manual_seed(7)
    for n, S, na in zip(ns, Ss, nas):
        mm = rsg.Mesh(rsg.CUBE, int(n), spacing=0.25)
        half = 0.5 * (n - 1) * 0.25
        c, d, w = gaussian_wells(g, int(na), 0.0, cube_half=0.6 * half)
        Hb = rsg.Hamiltonian(mm, torch.complex64)
        Hb.set_potential(potential_wells(mm.xyz, c, d, w))
        Hb.set_projectors(*projector_atoms(g, int(na), 2.5, 1, cube_half=0.6 * half))
        x = torch.randn((mm.P, rsg.padded_ld(int(S), torch.complex64)), dtype=torch.complex64,
                        device="cuda", generator=gen) * 1e-3
        hams.append(Hb)
        psis.append(x)
    sample = rng(3, 9).choice(256, 6, replace=False)
    ref = {i: psis[i].clone() for i in sample}
    batch = rsg.Batch(hams, [int(s) for s in Ss])
    batch.propagate(psis, 2, 0.02, scheme=rsg.ETRS)
    for i in sample:
        hams[i].propagate(ref[i], 2, 0.02, scheme=rsg.ETRS, S=int(Ss[i]))
    torch.cuda.synchronize()
    for i in sample:
        S = int(Ss[i])
        a, b = psis[i][:, :S], ref[i][:, :S]
        err = ((a - b).abs().amax(0) / b.abs().amax(0)).max().item()
        assert err < 2e-5, (i, err)

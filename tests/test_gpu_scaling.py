"""GPU: complex scaling (rsg_complex_scaling_set; Sec. "Complex scaling and
resonances": H_theta = -1/2 e^{-2i theta} lap + v(r e^{i theta})) against the
FP64 oracle's scaled operator (itself pinned by the closed-form rotated
spectrum, complex symmetry and the paper's one-dimensional example):

- the application on a sphere (ragged rows) and a box, complex128 and
  complex64, several state counts;
- a Taylor-4 stage and ETRS steps against the power series summed from
  oracle applications;
- shifted solves (H_theta - z) x = b (COCG: H_theta - z is complex
  symmetric) against a dense LAPACK solve of the oracle's matrix;
- the paper's one-dimensional example assembled column by column on the
  GPU: its two bound states stay real and the lowest resonance sits near the
  origin with an imaginary part of order -1e-5;
- the refusals while scaling is set, and its removal.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err
from tests._systems import Pair
from workloads import rng, white_noise_states

pytestmark = pytest.mark.gpu

C0 = -205 / 72


def _v_theta(xyz, theta):
    """v(r e^{i theta}) for a soft well v(r) = -2 exp(-r^2 / 2) plus a
    Gaussian bump 1.5 exp(-(r - a)^2) off the centre."""
    z2 = (xyz ** 2).sum(1) * np.exp(2j * theta)
    d = xyz - np.array([0.7, -0.4, 0.3])
    zd2 = (d ** 2).sum(1) * np.exp(2j * theta)
    return -2.0 * np.exp(-z2 / 2) + 1.5 * np.exp(-zd2)


def _scaled_pair(shape, n=0, radius=0.0, h=0.3, dtype=torch.complex128, theta=0.35):
    p = Pair(shape, n, radius, h, dtype)
    vt = _v_theta(p.om.xyz, theta)
    if dtype == torch.complex64:
        vt = vt.astype(np.complex64).astype(np.complex128)    # the FP32 path stores complex64
    p.H.set_complex_scaling(theta, p.to_lib(vt))
    return p, vt


def _states(p, S, seed):
    psi = white_noise_states(rng(31, seed), p.P, S)
    if p.dtype == torch.complex64:
        psi = psi.astype(np.complex64).astype(np.complex128)
    return psi


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("shape,n,radius", [("sphere", 0, 2.4), ("box", (13, 7, 9), 0.0)])
@pytest.mark.parametrize("S", [1, 3, 8])
def test_apply_matches_oracle(dtype, shape, n, radius, S):
    theta = 0.35
    p, vt = _scaled_pair(shape, n, radius, dtype=dtype, theta=theta)
    psi = _states(p, S, seed=S)
    x = p.states_to_gpu(psi)
    y = torch.zeros_like(x)
    p.H.apply(x, y, S)
    assert p.H.get_option("last_kernel") == 6
    got = p.states_from_gpu(y, S)
    want = p.om.apply_scaled(psi, theta, vt)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < (1e-13 if dtype == torch.complex128 else 2e-6), err
    # padding columns (zero input) stay zero
    if y.shape[1] > S:
        assert torch.count_nonzero(y[:, S:]) == 0


def test_taylor_stage_and_etrs_steps():
    theta, tau = 0.3, 0.02
    p, vt = _scaled_pair("sphere", radius=2.4, theta=theta)
    psi = _states(p, 4, seed=7)
    x = p.states_to_gpu(psi)
    out = torch.zeros_like(x)
    p.H.taylor(x, tau, out=out, S=4)
    want = p.om.taylor4_scaled(psi, theta, vt, tau)
    got = p.states_from_gpu(out, 4)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    # ETRS without a field: two half stages per step, the same operator
    nsteps, dt = 5, 0.04
    p.H.propagate(x, nsteps, dt, scheme=rsg.ETRS, S=4)
    want = p.om.propagate_scaled(psi, theta, vt, nsteps, dt, scheme=oracle.ETRS)
    got = p.states_from_gpu(x, 4)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("dtype,tol,etol", [(torch.complex128, 1e-11, 1e-9), (torch.complex64, 1e-4, 1e-3)])
def test_shifted_solve_against_dense(dtype, tol, etol):
    theta, z = 0.3, 0.4 + 0.15j
    p, vt = _scaled_pair("cube", 8, h=0.35, dtype=dtype, theta=theta)
    A = p.om.apply_scaled(np.eye(p.P, dtype=np.complex128), theta, vt) - z * np.eye(p.P)
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()       # complex symmetric
    assert np.abs(A - A.conj().T).max() > 1e-3                    # not Hermitian
    b = _states(p, 3, seed=11)
    want = np.linalg.solve(A, b)
    bd = p.states_to_gpu(b)
    x = torch.zeros_like(bd)
    res, it = p.H.shifted_solve(bd, x, z, max_iter=3000, tol=tol, S=3)
    assert np.all(res <= tol), (res, it)
    got = p.states_from_gpu(x, 3)
    assert np.abs(got - want).max() < etol * np.abs(want).max()


def test_paper_1d_example_spectrum():
    """v(x) = 3 (x^2 - 2) e^{-x^2/4} at theta = 0.5 on a 301-point line,
    h = 0.1 (the spectrum figure of the complex-scaling section)."""
    N, h = 301, 0.1
    mats = {}
    for theta in (0.4, 0.5):
        p = Pair("box", (N, 1, 1), h=h, dtype=torch.complex128)
        zc = p.om.xyz[:, 0] * np.exp(1j * theta)
        vt = 3 * (zc * zc - 2) * np.exp(-zc * zc / 4)
        p.H.set_complex_scaling(theta, p.to_lib(vt))
        eye = p.states_to_gpu(np.eye(N, dtype=np.complex128), ld=N)
        out = torch.zeros_like(eye)
        p.H.apply(eye, out, N)
        # column j = H_theta applied to the unit vector at oracle point j (oracle order on both axes)
        got = p.states_from_gpu(out, N)
        want = p.om.apply_scaled(np.eye(N, dtype=np.complex128), theta, vt)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()
        # the single-point y and z directions add -e^{-2i theta} c0 / h^2 to the diagonal
        mats[theta] = np.linalg.eigvals(got) - np.exp(-2j * theta) * (-C0 / h ** 2)
    a, b = mats[0.5], mats[0.4]
    stable = sorted((e for e in a if np.abs(b - e).min() < 1e-4 and e.real < 3), key=lambda e: e.real)
    assert len(stable) >= 3, stable
    bound, res = np.array(stable[:2]), stable[2]
    assert np.all(bound.real < 0) and np.all(np.abs(bound.imag) < 1e-6), bound
    assert 0 < res.real < 1 and -1e-4 < res.imag < -1e-6, res
    # the continuum turns into the lower half plane, by about -2 theta far out
    far = a[np.abs(a) > 50]
    assert np.all(far.imag < 0) and abs(np.median(np.angle(far)) + 1.0) < 0.05


def test_refusals_and_removal():
    p, vt = _scaled_pair("cube", 10, theta=0.2)
    S = 2
    x = p.states_to_gpu(_states(p, S, seed=1))
    with pytest.raises(rsg.RSGError):
        p.H.eigensolve(x, S=S)
    with pytest.raises(rsg.RSGError):
        p.H.set_field(0.05)
    with pytest.raises(rsg.RSGError):
        p.H.propagate(x, 2, 0.01, eps=[0.1, 0.0], S=S)
    one = x[:, :1].contiguous().reshape(-1)
    with pytest.raises(rsg.RSGError):
        p.H.control_gradient(one, one, np.zeros(3), 0.05)
    with pytest.raises(rsg.RSGError):
        p.H.set_projectors([[0.0, 0.0, 0.0]], [1.0], [0], [0.5], [1.0])
    q, _ = _scaled_pair("cube", 10, dtype=torch.complex64, theta=0.2)
    with pytest.raises(rsg.RSGError):
        rsg.Batch([q.H], [S])
    # removal: without a real potential the Hamiltonian is not ready;
    # with one it is the plain operator again
    p.H.set_complex_scaling(0.0, None)
    with pytest.raises(rsg.RSGError):
        p.H.apply(x, S=S)
    V = np.cos(p.om.xyz[:, 0])
    p.set_potential(V)
    y = p.H.apply(x, S=S)
    assert p.H.get_option("last_kernel") != 6
    got = p.states_from_gpu(y, S)
    want = p.O.apply(p.states_from_gpu(x, S))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    # theta = 0 with v_theta = v reproduces the plain operator through the scaled kernel
    p.H.set_complex_scaling(0.0, p.to_lib(V.astype(np.complex128)))
    y = p.H.apply(x, S=S)
    assert p.H.get_option("last_kernel") == 6
    assert np.abs(p.states_from_gpu(y, S) - want).max() < 1e-12 * np.abs(want).max()
    _ = oracle


@pytest.mark.parametrize("kernel", [5, 7])
@pytest.mark.parametrize("shape,n,radius,S", [("sphere", 0, 3.3, 4), ("box", (37, 23, 29), 0.0, 6),
                                              ("sphere", 0, 3.0, 64), ("sphere", 0, 2.7, 1),
                                              ("box", (21, 30, 17), 0.0, 13)])
def test_register_blocked_scaled_kernel(shape, n, radius, S, kernel):
    """complex64 with the register-blocked (5) or tensor-copy (7) kernel
    forced: the complex diagonal v_theta e^{2i theta} in shared memory and
    e^{-2i theta} folded into alpha; apply and a Taylor stage (alpha, base)."""
    theta = 0.35
    p, vt = _scaled_pair(shape, n, radius, dtype=torch.complex64, theta=theta)
    p.H.set_option("kernel", kernel)
    psi = _states(p, S, seed=S + 3)
    x = p.states_to_gpu(psi)
    y = p.H.apply(x, S=S)
    assert p.H.get_option("last_kernel") == kernel
    want = p.om.apply_scaled(psi, theta, vt)
    got = p.states_from_gpu(y, S)
    assert np.abs(got - want).max() < 2e-6 * np.abs(want).max()
    out = torch.zeros_like(x)
    p.H.taylor(x, 0.01, out=out, S=S)
    assert p.H.get_option("last_kernel") == kernel
    tw = p.om.taylor4_scaled(psi, theta, vt, 0.01)
    assert np.abs(p.states_from_gpu(out, S) - tw).max() < 2e-6 * np.abs(tw).max()
    # the same results as the one-thread-per-value kernel
    p.H.set_option("kernel", 1)
    y1 = p.H.apply(x, S=S)
    assert p.H.get_option("last_kernel") == 6
    assert np.abs(p.states_from_gpu(y1, S) - got).max() < 2e-6 * np.abs(want).max()


@pytest.mark.parametrize("kernel", [5, 7])
def test_register_blocked_scaled_shifted_solve(kernel):
    theta, z = 0.3, 0.4 + 0.15j
    p, vt = _scaled_pair("cube", 12, h=0.35, dtype=torch.complex64, theta=theta)
    p.H.set_option("kernel", kernel)
    A = p.om.apply_scaled(np.eye(p.P, dtype=np.complex128), theta, vt) - z * np.eye(p.P)
    b = _states(p, 3, seed=12)
    want = np.linalg.solve(A, b)
    x = torch.zeros_like(p.states_to_gpu(b))
    res, it = p.H.shifted_solve(p.states_to_gpu(b), x, z, max_iter=3000, tol=1e-4, S=3)
    assert p.H.get_option("last_kernel") == kernel
    assert np.all(res <= 1e-4), (res, it)
    assert np.abs(p.states_from_gpu(x, 3) - want).max() < 1e-3 * np.abs(want).max()


def test_full_size_sphere_sampled_register_blocked():
    """The benchmark's complex-scaled configuration: R = 18 bohr, h = 0.2
    (3,053,617 points), 64 complex64 states, 32 wells at r e^{0.3i}, the
    default kernel (tensor-copy staging with a complex diagonal); every state
    of 4096 sampled points against the oracle."""
    from workloads import gaussian_wells, potential_wells_scaled
    g = rng(2)
    theta = 0.3
    p = Pair("sphere", radius=18.0, h=0.2, dtype=torch.complex64)
    c, d, w = gaussian_wells(g, 32, 18.0 - 2.5)
    vt = potential_wells_scaled(p.om.xyz, c, d, w, theta).astype(np.complex64).astype(np.complex128)
    p.H.set_complex_scaling(theta, p.to_lib(vt))
    S = 64
    psi = white_noise_states(g, p.P, S, dtype=np.complex64).astype(np.complex128)
    y = p.H.apply(p.states_to_gpu(psi))
    torch.cuda.synchronize()
    assert p.H.get_option("last_kernel") == 7
    samp = g.choice(p.P, 4096, replace=False)
    pidx = np.repeat(samp, S)
    sidx = np.tile(np.arange(S), len(samp))
    want = p.om.apply_scaled_sampled(psi, theta, vt, pidx, sidx).reshape(len(samp), S)
    lib_rows = np.argsort(p.idx)[samp]     # library index of each sampled oracle point
    got = y[torch.from_numpy(lib_rows).cuda()].cpu().numpy().astype(np.complex128)
    assert rel_err(got, want) < 2e-5

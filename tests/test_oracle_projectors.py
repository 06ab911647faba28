"""Pins for the oracle's non-local (projector) term (no GPU).

The oracle's projector part is pinned by brute force (dense assembly of the
operator from unit vectors), by its spectrum computed through a different
route (the small nproj x nproj problem), and by the rank-one eigen relation
that the discrete normalisation implies.
"""
import numpy as np

import oracle
from workloads import rng, white_noise_states
from tests._oracle_helpers import dense_h, wdot


def _nonlocal_dense(m, centres, rcut, lmax, beta, hm):
    V = np.zeros(m.P)
    H0 = oracle.Hamiltonian(m, V)
    H1 = oracle.Hamiltonian(m, V)
    H1.set_projectors(centres, rcut, lmax, beta, hm)
    return dense_h(H1, m.P) - dense_h(H0, m.P), H1


def test_single_projector_eigenvector():
    """One s-projector: H_nl p = h_00 <p|p> p = h_00 p (discrete normalisation)."""
    m = oracle.Mesh(oracle.CUBE, 14, h=0.3)
    H0 = oracle.Hamiltonian(m, np.zeros(m.P))
    H1 = oracle.Hamiltonian(m, np.zeros(m.P))
    H1.set_projectors([[0.13, -0.21, 0.07]], [1.4], [0], [0.35], [np.array([[0.6]])])
    pts, vals = H1.atom(0)
    p = np.zeros(m.P)
    p[pts] = vals[0]
    assert abs(m.h ** 3 * np.sum(p * p) - 1.0) < 1e-13
    hnl = (H1.apply(p.reshape(-1, 1) + 0j) - H0.apply(p.reshape(-1, 1) + 0j)).ravel()
    assert np.abs(hnl - 0.6 * p).max() < 1e-12 * np.abs(p).max()


def test_sphere_membership():
    """Projector sphere = mesh points within r_c of the centre (inclusive)."""
    m = oracle.Mesh(oracle.SPHERE, radius=3.0, h=0.25)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    c = np.array([0.31, -0.42, 0.17])
    H.set_projectors([c], [1.3], [1], [0.325], [np.eye(4)])
    pts, _ = H.atom(0)
    d = np.linalg.norm(m.xyz - c, axis=1)
    assert set(pts.tolist()) == set(np.nonzero(d <= 1.3)[0].tolist())


def test_angular_parts_are_solid_harmonics():
    """p_i / p_s follows x, y, z, xy, yz, zx, x^2-y^2, 3z^2-r^2 up to a constant."""
    m = oracle.Mesh(oracle.CUBE, 16, h=0.25)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    c = np.array([0.05, -0.11, 0.09])
    H.set_projectors([c], [1.5], [2], [0.375], [np.eye(9)])
    pts, vals = H.atom(0)
    r = m.xyz[pts] - c
    x, y, z = r[:, 0], r[:, 1], r[:, 2]
    shapes = [np.ones_like(x), x, y, z, x * y, y * z, z * x, x * x - y * y,
              3 * z * z - (x * x + y * y + z * z)]
    for i, sh in enumerate(shapes):
        ok = np.abs(sh) > 0.2 * np.abs(sh).max()
        ratio = vals[i][ok] / (vals[0][ok] * sh[ok])
        assert np.ptp(ratio) < 1e-10 * np.abs(ratio).mean(), i


def test_dense_nonlocal_rank_and_spectrum():
    """Brute-force assembly: Hermitian, rank = total projectors, and spectrum
    equal to that of the small matrix h_a (h^3 P_a^T P_a) per atom pair block."""
    g = rng(98)
    m = oracle.Mesh(oracle.SPHERE, radius=2.2, h=0.4)
    c = np.array([[0.3, 0.1, -0.2], [-0.5, 0.4, 0.6]])
    A = g.uniform(-1, 1, (4, 4))
    hm = [np.diag(g.uniform(-1, 1, 9)), A + A.T]
    D, H1 = _nonlocal_dense(m, c, [1.6, 1.4], [2, 1], [0.4, 0.35], hm)
    assert np.abs(D - D.conj().T).max() < 1e-12 * np.abs(D).max()
    w = np.linalg.eigvalsh(D)
    tol = 1e-9 * np.abs(w).max()
    assert np.sum(np.abs(w) > tol) == 13
    # small-problem route: nonzero spectrum of B h B^T h^3 = spectrum of
    # h (h^3 B^T B), with B the P x 13 matrix of all projector columns.
    cols, blocks = [], []
    for a in range(2):
        pts, vals = H1.atom(a)
        for row in vals:
            col = np.zeros(m.P)
            col[pts] = row
            cols.append(col)
        blocks.append(hm[a])
    B = np.stack(cols, axis=1)
    Hb = np.zeros((13, 13))
    Hb[:9, :9] = blocks[0]
    Hb[9:, 9:] = blocks[1]
    small = np.linalg.eigvals(Hb @ (m.h ** 3 * B.T @ B))
    big = np.sort(w[np.abs(w) > tol])
    assert np.allclose(np.sort(small.real), big, rtol=1e-9, atol=1e-12)


def test_projectors_act_linearly_on_state_blocks():
    """Applying to a block equals applying state by state (no cross-talk)."""
    g = rng(97)
    m = oracle.Mesh(oracle.CUBE, 10, h=0.4)
    H = oracle.Hamiltonian(m, g.standard_normal(m.P))
    H.set_projectors([[0.1, 0.2, -0.1]], [1.5], [1], [0.37], [np.diag([0.5, -0.3, 0.2, 0.9])])
    psi = white_noise_states(g, m.P, 3)
    blk = H.apply(psi)
    for s in range(3):
        one = H.apply(psi[:, s:s + 1].copy())
        assert np.array_equal(one.ravel(), blk[:, s])
    lin = H.apply(psi @ np.array([[1.0], [2.0 - 1j], [0.5j]]))
    assert np.abs(lin.ravel() - blk @ np.array([1.0, 2.0 - 1j, 0.5j])).max() < 1e-11 * np.abs(blk).max()
    _ = wdot  # keep the helper import used across the suite


def test_raw_projectors_reproduce_the_sampled_set():
    """Feeding the oracle's own sampled projectors back as raw values gives
    the same operator."""
    m = oracle.Mesh(oracle.SPHERE, radius=2.5, h=0.3)
    g = rng(41)
    V = g.standard_normal(m.P)
    Ha = oracle.Hamiltonian(m, V)
    hm = [np.diag(g.uniform(-1, 1, 4)), np.diag(g.uniform(-1, 1, 9))]
    Ha.set_projectors([[0.2, -0.1, 0.3], [-0.6, 0.5, -0.2]], [1.3, 1.6], [1, 2], [0.33, 0.4], hm)
    pts, vals = zip(*(Ha.atom(a) for a in range(2)))
    Hr = oracle.Hamiltonian(m, V)
    Hr.set_projectors_raw(list(pts), [v.T for v in vals], hm)
    psi = white_noise_states(g, m.P, 3)
    assert np.abs(Ha.apply(psi) - Hr.apply(psi)).max() == 0.0


def test_raw_projectors_spectrum_from_small_problem():
    """Arbitrary sampled projectors on scattered point sets: the non-local
    operator h^3 sum_a P_a h_a P_a^T is real symmetric with rank
    sum nproj_a, and (disjoint supports) its nonzero eigenvalues are those of
    the small problems h_a G_a, G_a = h^3 P_a^T P_a (similar matrices)."""
    m = oracle.Mesh(oracle.CUBE, 6, h=0.4)
    g = rng(42)
    perm = g.permutation(m.P)
    sets = [np.sort(perm[:40]), np.sort(perm[40:95])]
    vals = [g.standard_normal((40, 3)), g.standard_normal((55, 2))]
    hs = []
    for k in (3, 2):
        A = g.standard_normal((k, k))
        hs.append(A + A.T)
    H0 = oracle.Hamiltonian(m, np.zeros(m.P))
    H1 = oracle.Hamiltonian(m, np.zeros(m.P))
    H1.set_projectors_raw(sets, vals, hs)
    D = dense_h(H1, m.P) - dense_h(H0, m.P)
    assert np.abs(D.imag).max() == 0.0 and np.abs(D - D.T).max() < 1e-13 * np.abs(D).max()
    w = np.linalg.eigvalsh(D.real)
    big = np.sort(w[np.abs(w) > 1e-9 * np.abs(w).max()])
    assert len(big) == 5
    h3 = m.h ** 3
    small = np.sort(np.concatenate([np.linalg.eigvals(hh @ (h3 * v.T @ v)).real for hh, v in zip(hs, vals)]))
    assert np.abs(big - small).max() < 1e-10 * np.abs(small).max(), (big, small)


def test_radial_factor_is_gaussian_in_two_beta_squared():
    """The radial part of every projector is exp(-|r - R_a|^2 / (2 beta^2))
    (reading C-6 of the projector passage in Sec. "Magnetic response and
    gauge invariance in real-space grids").  The discrete normalisation is a
    constant per projector, so ratios between sphere points fix the radial
    factor independently of it: for the s-projector
    p(q) / p(q') = exp(-(d_q^2 - d_q'^2) / (2 beta^2)), and for the p- and
    d-projectors the same after dividing out the solid harmonic.  A radial
    factor exp(-d^2 / beta^2), or one in |r| instead of |r - R_a|, fails."""
    m = oracle.Mesh(oracle.CUBE, 18, h=0.25)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    c = np.array([0.17, -0.08, 0.11])
    rc, beta = 1.9, 0.55
    H.set_projectors([c], [rc], [2], [beta], [np.eye(9)])
    pts, vals = H.atom(0)
    r = m.xyz[pts] - c
    d2 = np.sum(r * r, axis=1)
    x, y, z = r[:, 0], r[:, 1], r[:, 2]
    shapes = [np.ones_like(x), x, y, z, x * y, y * z, z * x, x * x - y * y, 3 * z * z - d2]
    g = rng(91)
    for i, sh in enumerate(shapes):
        ok = np.nonzero(np.abs(sh) > 0.2 * np.abs(sh).max())[0]
        radial = vals[i][ok] / sh[ok]
        a, b = g.choice(len(ok), 40), g.choice(len(ok), 40)
        want = np.exp(-(d2[ok][a] - d2[ok][b]) / (2.0 * beta * beta))
        assert np.allclose(radial[a] / radial[b], want, rtol=1e-12, atol=0.0), i


def test_workload_projector_width_decays_to_e_minus_8_at_cutoff():
    """The workloads take beta = r_c / 4, so the radial factor at the cutoff
    sphere is exp(-r_c^2 / (2 (r_c/4)^2)) = e^-8; checked on the oracle's
    sampled s-projector against its value at the point nearest the centre."""
    _, rcut, lmax, beta, _ = projector_atoms_for_test()
    assert np.allclose(beta, rcut / 4.0)
    m = oracle.Mesh(oracle.CUBE, 24, h=0.2)
    H = oracle.Hamiltonian(m, np.zeros(m.P))
    c = np.zeros(3) + 0.1   # no mesh point at the centre
    H.set_projectors([c], [rcut[0]], [0], [beta[0]], [np.eye(1)])
    pts, vals = H.atom(0)
    d = np.linalg.norm(m.xyz[pts] - c, axis=1)
    i0, i1 = np.argmin(d), np.argmax(d)
    ratio = vals[0][i1] / vals[0][i0]
    assert abs(ratio - np.exp(-8.0 * (d[i1] ** 2 - d[i0] ** 2) / rcut[0] ** 2)) < 1e-13
    # the farthest sphere point lies within one spacing of r_c
    assert rcut[0] - m.h < d[i1] <= rcut[0]


def projector_atoms_for_test():
    from workloads import projector_atoms
    return projector_atoms(rng(3), 2, 2.5, 1, ball_radius=5.0)

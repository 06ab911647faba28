"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds NO arithmetic of the method itself (no stencil, no
projector construction, no propagator, no orthonormalisation).  It only draws
random numbers and evaluates the external potentials / control fields that
define a workload, as functions of positions the caller supplies.  Each side
(the CUDA library and the oracle) builds its own mesh and passes its own
point positions here, so the two never share mesh code.

Seeds follow one recipe: PCG64 with seed 1501056540 + workload index.

Workloads (positions in bohr, energies in hartree, times in au):
  1  HO cube:      32^3 at h=0.3, V = 1/2 w^2 r^2 (w=0.5), 4 smooth states.
  2  sphere:       R=18 at h=0.2 (3,053,617 points), 64 white-noise states,
                   32 Gaussian wells, 32 atoms x 4 projectors (r_c=2.5).
  3  batch:        256 cubes n in U{24..96} at h=0.25, S in U{1..16},
                   1..8 atoms x 4 projectors.
  4  control:      64^3 at h=0.3, double well, dipole field along x.
  5  large cube:   192^3 at h=0.18, 128 states, 64 atoms x 9 projectors.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1501056540


def rng(workload: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for a workload index (and an optional sub-stream)."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + int(workload), int(stream)]))


# ----------------------------------------------------------------------------
# external potentials, evaluated at caller-supplied positions (P x 3, bohr)
# ----------------------------------------------------------------------------

def potential_harmonic(xyz: np.ndarray, omega: float = 0.5) -> np.ndarray:
    """Isotropic oscillator 1/2 w^2 |r|^2."""
    xyz = np.asarray(xyz, dtype=np.float64)
    return 0.5 * omega * omega * np.einsum("pi,pi->p", xyz, xyz)


def potential_double_well(xyz: np.ndarray, a: float = 0.02, b: float = 2.0,
                          omega: float = 0.5) -> np.ndarray:
    """a (x^2 - b^2)^2 + 1/2 w^2 (y^2 + z^2)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return a * (x * x - b * b) ** 2 + 0.5 * omega * omega * (y * y + z * z)


def potential_soft_coulomb_li(xyz: np.ndarray) -> np.ndarray:
    """Three soft-Coulomb electrons in 1-D seen as one particle in 3-D.

    Coordinates (x1, x2, x3) are the three electron positions; the external
    potential is -3/sqrt(x_j^2+1) per electron and the interaction is
    1/sqrt((x_j-x_k)^2+1) per pair (the one-dimensional lithium model).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    v = np.zeros(xyz.shape[0])
    for j in range(3):
        v -= 3.0 / np.sqrt(xyz[:, j] ** 2 + 1.0)
    for j in range(3):
        for k in range(j + 1, 3):
            v += 1.0 / np.sqrt((xyz[:, j] - xyz[:, k]) ** 2 + 1.0)
    return v


def gaussian_wells(g: np.random.Generator, n: int, region_radius: float,
                   depth=(1.0, 4.0), width=(0.8, 1.5), cube_half=None):
    """Seeded well centres, depths and widths.

    Centres are uniform in a ball of radius ``region_radius`` (or, if
    ``cube_half`` is given, uniform in the cube [-cube_half, cube_half]^3).
    """
    if cube_half is None:
        c = _uniform_ball(g, n, region_radius)
    else:
        c = g.uniform(-cube_half, cube_half, size=(n, 3))
    d = g.uniform(depth[0], depth[1], size=n)
    w = g.uniform(width[0], width[1], size=n)
    return c, d, w


def potential_wells(xyz: np.ndarray, centres, depths, widths) -> np.ndarray:
    """Sum of Gaussian wells -D exp(-|r-R|^2 / (2 w^2))."""
    xyz = np.asarray(xyz, dtype=np.float64)
    v = np.zeros(xyz.shape[0])
    for c, d, w in zip(centres, depths, widths):
        r2 = np.einsum("pi,pi->p", xyz - c, xyz - c)
        v -= d * np.exp(-r2 / (2.0 * w * w))
    return v


def potential_wells_scaled(xyz: np.ndarray, centres, depths, widths, theta: float) -> np.ndarray:
    """The Gaussian wells of potential_wells at the rotated coordinates
    r e^{i theta} (complex values; the square |r e^{i theta} - R|^2 taken
    without conjugation, as the analytic continuation requires)."""
    z = np.asarray(xyz, dtype=np.float64) * np.exp(1j * theta)
    v = np.zeros(z.shape[0], dtype=np.complex128)
    for c, d, w in zip(centres, depths, widths):
        dz = z - np.asarray(c, dtype=np.float64)
        v -= d * np.exp(-np.einsum("pi,pi->p", dz, dz) / (2.0 * w * w))
    return v


def _uniform_ball(g: np.random.Generator, n: int, radius: float) -> np.ndarray:
    out = np.empty((n, 3))
    k = 0
    while k < n:
        p = g.uniform(-radius, radius, size=3)
        if p @ p <= radius * radius:
            out[k] = p
            k += 1
    return out


# ----------------------------------------------------------------------------
# pseudo-atoms carrying projectors (parameters only; projector values are
# built by each side from these parameters)
# ----------------------------------------------------------------------------

def projector_atoms(g: np.random.Generator, n: int, rcut: float, lmax: int,
                    ball_radius=None, cube_half=None):
    """Seeded atom centres, r_c, l_max, beta and diagonal h_ij in U[-1, 1].

    beta = r_c / 4, so the radial Gaussian has decayed to e^-8 at r_c.
    Returns (centres (n,3), rcut (n,), lmax (n,), beta (n,), hmat list of
    (nproj, nproj) arrays).
    """
    if cube_half is not None:
        c = g.uniform(-cube_half, cube_half, size=(n, 3))
    else:
        c = _uniform_ball(g, n, ball_radius)
    nproj = (lmax + 1) ** 2
    hs = [np.diag(g.uniform(-1.0, 1.0, size=nproj)) for _ in range(n)]
    return (c, np.full(n, float(rcut)), np.full(n, int(lmax), dtype=np.int32),
            np.full(n, rcut / 4.0), hs)


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------

def white_noise_states(g: np.random.Generator, P: int, S: int,
                       dtype=np.complex128) -> np.ndarray:
    """i.i.d. complex normal values, shape (P, S)."""
    re = g.standard_normal((P, S), dtype=np.float64 if dtype == np.complex128 else np.float32)
    im = g.standard_normal((P, S), dtype=re.dtype)
    out = np.empty((P, S), dtype=dtype)
    out.real = re
    out.imag = im
    return out


def wavepacket_params(g: np.random.Generator, S: int, centre_radius: float,
                      sigma=(0.8, 1.5), kmax: float = 1.0, max_terms: int = 3):
    """Per state: 1-3 Gaussians with seeded centres, widths and momenta."""
    params = []
    for _ in range(S):
        m = int(g.integers(1, max_terms + 1))
        terms = []
        for _ in range(m):
            c = _uniform_ball(g, 1, centre_radius)[0]
            s = g.uniform(sigma[0], sigma[1])
            k = _uniform_ball(g, 1, kmax)[0]
            a = complex(g.standard_normal(), g.standard_normal())
            terms.append((c, s, k, a))
        params.append(terms)
    return params


def wavepacket_states(xyz: np.ndarray, params) -> np.ndarray:
    """Evaluate smooth packets sum_m a_m exp(-|r-c|^2/(4 s^2) + i k.r)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    out = np.zeros((xyz.shape[0], len(params)), dtype=np.complex128)
    for s_idx, terms in enumerate(params):
        for c, s, k, a in terms:
            d = xyz - c
            r2 = np.einsum("pi,pi->p", d, d)
            out[:, s_idx] += a * np.exp(-r2 / (4.0 * s * s) + 1j * (xyz @ k))
    return out


# ----------------------------------------------------------------------------
# control field
# ----------------------------------------------------------------------------

def control_field(g: np.random.Generator, nsteps: int, dt: float,
                  amax: float = 0.05, nterms: int = 8,
                  wrange=(0.05, 0.6)) -> np.ndarray:
    """eps_k = sum of seeded sines sampled at t_k = k dt, scaled to max |eps| = amax."""
    t = np.arange(nsteps) * dt
    a = g.standard_normal(nterms)
    w = g.uniform(wrange[0], wrange[1], size=nterms)
    ph = g.uniform(0.0, 2.0 * np.pi, size=nterms)
    e = (a[None, :] * np.sin(w[None, :] * t[:, None] + ph[None, :])).sum(axis=1)
    m = np.abs(e).max()
    return e * (amax / m) if m > 0 else e


# ----------------------------------------------------------------------------
# batch of uneven systems
# ----------------------------------------------------------------------------

def batch_systems(g: np.random.Generator, nsys: int = 256, nmin: int = 24,
                  nmax: int = 96, smax: int = 16, amax: int = 8):
    """Per system: cube edge n, state count S, atom count."""
    n = g.integers(nmin, nmax + 1, size=nsys)
    S = g.integers(1, smax + 1, size=nsys)
    na = g.integers(1, amax + 1, size=nsys)
    return n, S, na

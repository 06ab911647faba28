"""GPU parity: H|psi> through the C ABI against the FP64 oracle.

Tolerances (normwise max relative error per state): 1e-12 for complex128;
2e-5 for complex64, with the oracle fed the complex64-rounded inputs.
"""
import numpy as np
import pytest
import torch

import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err, round_c64
from tests._systems import Pair, wells_system
from workloads import white_noise_states

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _check_apply(p, g, S, eps=0.0, dir=(1.0, 0.0, 0.0), opts=None, expect_kernel=None):
    psi = white_noise_states(g, p.P, S)
    if p.dtype == torch.complex64:
        psi = round_c64(psi)
    want = p.O.apply(psi, eps=eps, dir=dir)
    if eps:
        p.H.set_field(eps, dir)
    for k, v in (opts or {}).items():
        p.H.set_option(k, v)
    x = p.states_to_gpu(psi)
    y = p.H.apply(x, S=S)
    torch.cuda.synchronize()
    if expect_kernel is not None:
        assert p.H.get_option("last_kernel") == expect_kernel
    got = p.states_from_gpu(y, S)
    err = rel_err(got, want)
    assert err < TOL[p.dtype], err
    return err


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("S", [1, 3, 8, 19])
def test_cube_ragged_tiles(dtype, S):
    """37^3: several tiles plus a ragged tail in every direction."""
    p, g = wells_system("cube", 37, h=0.3, dtype=dtype, seed=S, natoms=3, lmax=2, rcut=1.5)
    _check_apply(p, g, S)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_sphere_with_projectors_and_field(dtype):
    p, g = wells_system("sphere", radius=4.1, h=0.3, dtype=dtype, seed=5, natoms=4, lmax=1)
    _check_apply(p, g, 6, eps=0.037, dir=(0.6, -0.8, 0.0))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_box_odd_extents(dtype):
    p, g = wells_system("box", (23, 9, 14), h=0.25, dtype=dtype, seed=6, natoms=1, lmax=0)
    _check_apply(p, g, 4, eps=-0.02, dir=(0.0, 0.0, 1.0))


@pytest.mark.parametrize("opts", [{"kernel": 1}, {"kernel": 0, "rx": 1}, {"kernel": 0, "rx": 2},
                                  {"kernel": 0, "ty": 2, "zseg": 5},
                                  {"kernel": 0, "ty": 16, "zseg": 64, "rx": 1},
                                  {"kernel": 2, "rx": 1}, {"kernel": 2, "rx": 2},
                                  {"kernel": 2, "rx": 4}, {"kernel": 2, "ty": 2, "zseg": 5},
                                  {"kernel": 2, "ty": 4, "rx": 4, "zseg": 3},
                                  {"kernel": 0, "threads": 256, "cv": 2}, {"kernel": 0, "threads": 256, "cv": 4},
                                  {"kernel": 0, "cv": 8, "zseg": 120, "threads": 512},
                                  {"kernel": 0, "cv": 1, "zseg": 11, "threads": 512},
                                  {"kernel": 0, "stages": 3, "blocks_per_sm": 3, "zseg": 40},
                                  {"kernel": 0, "stages": 3, "blocks_per_sm": 2, "cv": 4, "zseg": 9}])
def test_kernel_variants_agree(opts):
    p, g = wells_system("sphere", radius=3.3, h=0.25, dtype=torch.complex64, seed=7, natoms=2)
    _check_apply(p, g, 10, opts=opts, expect_kernel=opts["kernel"])


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("opts", [{"kernel": 3}, {"kernel": 3, "cv": 2}, {"kernel": 3, "cv": 8, "ty": 8},
                                  {"kernel": 3, "cv": 2, "ty": 4, "zseg": 7}])
def test_tma_gather_kernel(dtype, opts):
    """The TMA-gather stencil on a ragged sphere with projectors and a field."""
    p, g = wells_system("sphere", radius=4.6, h=0.25, dtype=dtype, seed=8, natoms=3, lmax=2)
    _check_apply(p, g, 13, eps=0.02, dir=(0.0, 0.6, 0.8), opts=opts, expect_kernel=3)
    # Horner stage through the same kernel (base stream gathered by the TMA)
    psi = white_noise_states(g, p.P, 5)
    if dtype == torch.complex64:
        psi = round_c64(psi)
    want = p.O.taylor4(psi, 0.01, eps=0.02, dir=(0.0, 0.6, 0.8))
    y = p.H.taylor(p.states_to_gpu(psi), 0.01, S=5)
    torch.cuda.synchronize()
    assert p.H.get_option("last_kernel") == 3
    assert rel_err(p.states_from_gpu(y, 5), want) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("opts", [{"kernel": 4}, {"kernel": 4, "stages": 5}, {"kernel": 4, "threads": 512},
                                  {"kernel": 4, "zseg": 7}, {"kernel": 4, "zseg": 1}])
@pytest.mark.parametrize("S", [4, 13])
def test_row_tma_kernel(dtype, opts, S):
    """Row-TMA staged stencil on a sphere: rows that end inside a tile and
    rows absent from the mesh (zeroed in shared memory), a partial last state
    chunk (S = 13: the copy box runs past the state columns), projectors, a
    field, and a Horner stage (base values by cp.async)."""
    p, g = wells_system("sphere", radius=4.6, h=0.25, dtype=dtype, seed=9, natoms=3, lmax=2)
    want_k = 0 if (dtype == torch.complex128 and opts.get("threads") == 512) else 4
    _check_apply(p, g, S, eps=0.02, dir=(0.0, 0.6, 0.8), opts=opts, expect_kernel=want_k)
    psi = white_noise_states(g, p.P, S)
    if dtype == torch.complex64:
        psi = round_c64(psi)
    want = p.O.taylor4(psi, 0.01, eps=0.02, dir=(0.0, 0.6, 0.8))
    y = p.H.taylor(p.states_to_gpu(psi), 0.01, S=S)
    torch.cuda.synchronize()
    assert p.H.get_option("last_kernel") == want_k
    assert rel_err(p.states_from_gpu(y, S), want) < TOL[dtype]


@pytest.mark.parametrize("opts", [{"kernel": 5}, {"kernel": 5, "threads": 256}, {"kernel": 5, "zseg": 7},
                                  {"kernel": 5, "threads": 256, "zseg": 1}, {"kernel": 5, "threads": 512},
                                  {"kernel": 5, "sync": 1}, {"kernel": 5, "sync": 2}, {"kernel": 5, "sync": 2, "zseg": 3},
                                  {"kernel": 5, "stages": 3, "zseg": 9}, {"kernel": 5, "threads": 160, "zseg": 96}])
@pytest.mark.parametrize("S", [1, 2, 5, 13, 16])
def test_quad_kernel(opts, S):
    """Register-blocked stencil (complex64): a sphere with projectors and a
    field; S = 1, 2 and 5 leave part of the last four-value chunk empty."""
    p, g = wells_system("sphere", radius=4.6, h=0.25, dtype=torch.complex64, seed=10, natoms=3, lmax=2)
    _check_apply(p, g, S, eps=0.02, dir=(0.0, 0.6, 0.8), opts=opts, expect_kernel=5)
    psi = round_c64(white_noise_states(g, p.P, S))
    want = p.O.taylor4(psi, 0.01, eps=0.02, dir=(0.0, 0.6, 0.8))
    y = p.H.taylor(p.states_to_gpu(psi), 0.01, S=S)
    torch.cuda.synchronize()
    assert p.H.get_option("last_kernel") == 5
    assert rel_err(p.states_from_gpu(y, S), want) < TOL[torch.complex64]


@pytest.mark.parametrize("opts", [{"kernel": 7}, {"kernel": 7, "wide_ty": 6}, {"kernel": 7, "zseg": 7},
                                  {"kernel": 7, "zseg": 1}, {"kernel": 7, "wide_ty": 6, "zseg": 3},
                                  {"kernel": 7, "wide_ty": 6, "zseg": 200}, {"kernel": 7, "wide_ty": 6, "producers": 4},
                                  {"kernel": 7, "wide_ty": 4, "stages": 4, "producers": 3},
                                  {"kernel": 7, "wide_ty": 8, "producers": 2, "zseg": 64}])
@pytest.mark.parametrize("S", [1, 2, 13, 16, 17, 40])
def test_wide_kernel(opts, S):
    """Warp-specialised tensor-copy stencil (complex64) on a sphere with
    projectors and a field: rows that end inside the window (partial boxes and
    zero-fill boxes), empty planes and columns, a partial last 16-value chunk
    (S = 1, 2, 13, 17, 40) and a Horner stage (base rows by tensor copy)."""
    p, g = wells_system("sphere", radius=4.6, h=0.25, dtype=torch.complex64, seed=10, natoms=3, lmax=2)
    _check_apply(p, g, S, eps=0.02, dir=(0.0, 0.6, 0.8), opts=opts, expect_kernel=7)
    psi = round_c64(white_noise_states(g, p.P, S))
    want = p.O.taylor4(psi, 0.01, eps=0.02, dir=(0.0, 0.6, 0.8))
    y = p.H.taylor(p.states_to_gpu(psi), 0.01, S=S)
    torch.cuda.synchronize()
    assert p.H.get_option("last_kernel") == 7
    assert rel_err(p.states_from_gpu(y, S), want) < TOL[torch.complex64]


def test_wide_kernel_cube_box_and_long_segments():
    """Full rows (one 24-record box per window row), ragged tile tails in x, y
    and z, extents below the stencil radius, and a 260-plane box in one
    segment; the same block reused across launches with different inputs."""
    for shape, n, zseg, wty in (("cube", 37, 150, 8), ("box", (23, 9, 14), 150, 8), ("box", (3, 2, 40), 150, 6),
                                ("box", (12, 10, 260), 150, 8), ("box", (12, 10, 260), 256, 6),
                                ("box", (40, 33, 5), 2, 8)):
        p, g = wells_system(shape, n, h=0.3, dtype=torch.complex64, seed=4, natoms=2, lmax=1)
        for S in (10, 64):
            _check_apply(p, g, S, opts={"kernel": 7, "zseg": zseg, "wide_ty": wty}, expect_kernel=7)


@pytest.mark.parametrize("opts", [{"kernel": 7, "wide_ty": 6, "producers": 4, "zseg": 190},
                                  {"kernel": 7, "wide_ty": 8, "producers": 1, "zseg": 5}])
def test_wide_kernel_taylor_in_place(opts):
    """A Taylor exponential written over its input: the last Horner stage's
    outputs (stored from shared memory by tensor copies) land on the base
    block they were computed from."""
    p, g = wells_system("sphere", radius=4.6, h=0.25, dtype=torch.complex64, seed=11, natoms=3, lmax=2)
    for k, v in opts.items():
        p.H.set_option(k, v)
    psi = round_c64(white_noise_states(g, p.P, 16))
    want = p.O.taylor4(psi, 0.01)
    x = p.states_to_gpu(psi)
    y = p.H.taylor(x, 0.01, out=x, S=16)
    torch.cuda.synchronize()
    assert y.data_ptr() == x.data_ptr()
    assert p.H.get_option("last_kernel") == 7
    assert rel_err(p.states_from_gpu(x, 16), want) < TOL[torch.complex64]


def test_wide_kernel_declines_oversized_segments():
    """8-row tiles with 256-plane segments need more shared memory than a
    block may have: the launcher declines and the staged kernel runs."""
    p, g = wells_system("box", (12, 10, 260), h=0.3, dtype=torch.complex64, seed=4, natoms=1, lmax=0)
    _check_apply(p, g, 6, opts={"kernel": 7, "zseg": 256, "wide_ty": 8, "stages": 3}, expect_kernel=0)


def test_quad_kernel_cube_box_and_complex128_fallback():
    for shape, n in (("cube", 37), ("box", (23, 9, 14)), ("box", (3, 2, 40))):
        p, g = wells_system(shape, n, h=0.3, dtype=torch.complex64, seed=4, natoms=2, lmax=1)
        _check_apply(p, g, 10, opts={"kernel": 5}, expect_kernel=5)
    # complex128 has no register-blocked kernel: the staged kernel runs
    p, g = wells_system("cube", 20, h=0.3, dtype=torch.complex128, seed=4, natoms=2, lmax=1)
    _check_apply(p, g, 3, opts={"kernel": 5}, expect_kernel=0)


@pytest.mark.parametrize("opts", [{"kernel": 5, "zseg": 256}, {"kernel": 5, "zseg": 200, "threads": 256},
                                  {"kernel": 0, "zseg": 200}, {"kernel": 4, "zseg": 256},
                                  {"kernel": 3, "zseg": 200}])
def test_long_z_segments(opts):
    """A 260-plane box: z segments beyond 120 planes (kernels 0, 4, 5 size
    their row tables dynamically; kernel 3 caps its segments at 120)."""
    p, g = wells_system("box", (12, 10, 260), h=0.3, dtype=torch.complex64, seed=14, natoms=2, lmax=1)
    _check_apply(p, g, 6, opts=opts, expect_kernel=opts["kernel"])


def test_row_tma_kernel_cube_and_box():
    """Full rows (no fix-ups inside the mesh), ragged tile tails in x, y, z."""
    for shape, n in (("cube", 37), ("box", (23, 9, 14))):
        p, g = wells_system(shape, n, h=0.3, dtype=torch.complex64, seed=3, natoms=2, lmax=1)
        _check_apply(p, g, 10, opts={"kernel": 4}, expect_kernel=4)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_degenerate_meshes(dtype):
    # one point: every neighbour is a ghost
    p, g = wells_system("cube", 1, h=0.3, dtype=dtype, natoms=0)
    _check_apply(p, g, 2)
    # sphere smaller than one spacing: the origin only
    p, g = wells_system("sphere", radius=0.1, h=0.3, dtype=dtype, natoms=0)
    assert p.P == 1
    _check_apply(p, g, 1)
    # thin slab: extents below the stencil radius
    p, g = wells_system("box", (3, 2, 40), h=0.3, dtype=dtype, natoms=1, lmax=0)
    _check_apply(p, g, 3)


def test_no_projectors_then_projectors_removed():
    p, g = wells_system("cube", 12, h=0.3, dtype=torch.complex128, natoms=2)
    _check_apply(p, g, 2)
    p.H.set_projectors(np.zeros((0, 3)), [], [], [], [])
    p.O.set_projectors(np.zeros((0, 3)), [], [], [], [])
    _check_apply(p, g, 2)


def test_linear_and_hermitian_on_device():
    """<a|H b> = conj <b|H a> with device results (sanity independent of the oracle)."""
    p, g = wells_system("sphere", radius=3.0, h=0.3, dtype=torch.complex128, natoms=2)
    a = p.states_to_gpu(white_noise_states(g, p.P, 1))
    b = p.states_to_gpu(white_noise_states(g, p.P, 1))
    ha, hb = p.H.apply(a), p.H.apply(b)
    l = torch.vdot(a[:, 0], hb[:, 0]).item()
    r = torch.vdot(b[:, 0], ha[:, 0]).conj().item()
    assert abs(l - r) < 1e-12 * abs(l)


def test_errors_on_device():
    p, g = wells_system("cube", 8, h=0.3, dtype=torch.complex64, natoms=0)
    x = torch.zeros((p.P, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(rsg.RSGError, match="overlap"):
        p.H.apply(x, out=x)
    with pytest.raises(ValueError):
        p.H.apply(x.to(torch.complex128))
    with pytest.raises(rsg.RSGError, match="ARG"):
        p.H.apply(x, S=5)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_full_size_sphere_sampled(dtype):
    """R = 18 bohr, h = 0.2 (3,053,617 points), 64 states, 32 wells and 32
    atoms x 4 projectors: every state of 4096 sampled points vs the oracle."""
    from workloads import gaussian_wells, potential_wells, projector_atoms, rng
    g = rng(2)
    p = Pair("sphere", radius=18.0, h=0.2, dtype=dtype)
    c, d, w = gaussian_wells(g, 32, 18.0 - 2.5)
    p.set_potential(potential_wells(p.om.xyz, c, d, w))
    cen, rc, lm, beta, hm = projector_atoms(g, 32, 2.5, 1, ball_radius=18.0 - 2.5)
    p.set_projectors(cen, rc, lm, beta, hm)
    S = 64
    psi = white_noise_states(g, p.P, S, dtype=np.complex64 if dtype == torch.complex64 else np.complex128)
    psi = psi.astype(np.complex128)
    x = p.states_to_gpu(psi)
    y = p.H.apply(x)
    torch.cuda.synchronize()
    # sample points: random, plus points inside projector spheres and on the surface
    samp = g.choice(p.P, 4096, replace=False)
    pidx = np.repeat(samp, S)
    sidx = np.tile(np.arange(S), len(samp))
    want = p.O.apply_sampled(psi, pidx, sidx).reshape(len(samp), S)
    lib_rows = np.argsort(p.idx)[samp]     # library index of each sampled oracle point
    got = y[torch.from_numpy(lib_rows).cuda()].cpu().numpy().astype(np.complex128)
    assert rel_err(got, want) < TOL[dtype]


def test_autotune_picks_a_working_configuration(tmp_path):
    p, g = wells_system("sphere", radius=6.0, h=0.25, dtype=torch.complex64, seed=9, natoms=2)
    psi = round_c64(white_noise_states(g, p.P, 12))
    x = p.states_to_gpu(psi)
    cache = str(tmp_path / "tune.json")
    res = p.H.autotune(x, S=12, cache_path=cache)
    assert res["stage_ms"] > 0
    # the tuned configuration still matches the oracle
    want = p.O.apply(psi)
    y = p.H.apply(x, S=12)
    torch.cuda.synchronize()
    assert rel_err(p.states_from_gpu(y, 12), want) < TOL[torch.complex64]
    # a second Hamiltonian reuses the cached choice without timing
    q, _ = wells_system("sphere", radius=6.0, h=0.25, dtype=torch.complex64, seed=9, natoms=2)
    res2 = q.H.autotune(q.states_to_gpu(psi), S=12, cache_path=cache)
    assert {k: res2[k] for k in q.H.TUNED_KEYS} == {k: res[k] for k in q.H.TUNED_KEYS}

"""GPU parity: a batch of uneven complex64 systems against single-system
propagation and against the FP64 oracle.  The default path is one persistent
launch per time step (k_batch_step: every Horner stage of every system from
one work queue); "persistent" = 0 is one launch per stage and kernel."""
import numpy as np
import pytest
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._parity import rel_err, round_c64
from tests._systems import Pair
from workloads import (gaussian_wells, potential_wells, projector_atoms, rng,
                       wavepacket_params, wavepacket_states)

pytestmark = pytest.mark.gpu

SPECS = [(9, 1, 1), (14, 3, 2), (20, 4, 0), (24, 6, 3), (11, 2, 1), (17, 5, 2)]   # (n, S, atoms)


def _systems(lmax_of=lambda i: 1, seed=0, atoms=True, specs=SPECS):
    g = rng(3, seed)
    out = []
    for i, (n, S, na) in enumerate(specs):
        na = na if atoms else 0
        p = Pair("cube", n, h=0.25, dtype=torch.complex64)
        half = 0.5 * (n - 1) * 0.25
        c, d, w = gaussian_wells(g, 2, 0.0, cube_half=0.6 * half)
        p.set_potential(potential_wells(p.om.xyz, c, d, w))
        if na:
            cen, rc, lm, beta, hm = projector_atoms(g, na, 1.0, lmax_of(i), cube_half=0.5 * half)
            p.set_projectors(cen, rc, lm, beta, hm)
        psi = p.om.mgs(wavepacket_states(p.om.xyz, wavepacket_params(g, S, 0.5 * half)))
        out.append((p, round_c64(psi), S))
    return out


def _run_batch(systems, nsteps, dt, scheme, gs_every=0, **opts):
    batch = rsg.Batch([p.H for p, _, _ in systems], [S for _, _, S in systems])
    for k, v in opts.items():
        batch.set_option(k, v)
    xs = [p.states_to_gpu(psi) for p, psi, _ in systems]
    batch.propagate(xs, nsteps, dt, scheme=scheme, gs_every=gs_every)
    torch.cuda.synchronize()
    return batch, xs


@pytest.mark.parametrize("persistent", [1, 0])
def test_batch_matches_single_system_and_oracle(persistent):
    systems = _systems()
    batch, xs = _run_batch(systems, 4, 0.02, rsg.ETRS, persistent=persistent)
    assert batch.get_option("launches_per_step") == (1 if persistent else 32)
    for (p, psi, S), x in zip(systems, xs):
        y = p.states_to_gpu(psi)
        p.H.propagate(y, 4, 0.02, scheme=rsg.ETRS)
        torch.cuda.synchronize()
        got, ref = p.states_from_gpu(x, S), p.states_from_gpu(y, S)
        assert rel_err(got, ref) < 2e-5
    p, psi, S = systems[3]
    want, _ = p.O.propagate(psi, 4, 0.02, scheme=oracle.ETRS)
    assert rel_err(p.states_from_gpu(xs[3], S), want) < 2e-5


def test_persistent_batch_bitwise_equals_single_wide_kernel():
    """Without projectors each stencil item of the persistent step computes
    every output with the same operations in the same order as the
    single-system tensor-copy kernel (kernel 7) with its Horner epilogue;
    tiles differ, results per point do not."""
    systems = _systems(seed=3, atoms=False)
    _, xs = _run_batch(systems, 3, 0.02, rsg.ETRS)
    for (p, psi, S), x in zip(systems, xs):
        p.H.set_option("kernel", 7)
        y = p.states_to_gpu(psi)
        p.H.propagate(y, 3, 0.02, scheme=rsg.ETRS)
        torch.cuda.synchronize()
        assert p.H.get_option("last_kernel") == 7
        assert torch.equal(x, y), (p.P, S, (x - y).abs().max().item())


def test_batch_bitwise_equals_single_register_blocked_systems():
    """Without projectors the batched stencil runs the same register-blocked
    block, tiles, plane order and epilogue constants as the single-system
    kernel 5, so each system's result is bit-for-bit that of its own run."""
    systems = _systems(seed=3, atoms=False)
    _, xs = _run_batch(systems, 3, 0.02, rsg.ETRS, persistent=0)
    for (p, psi, S), x in zip(systems, xs):
        p.H.set_option("kernel", 5)
        y = p.states_to_gpu(psi)
        p.H.propagate(y, 3, 0.02, scheme=rsg.ETRS)
        torch.cuda.synchronize()
        assert p.H.get_option("last_kernel") == 5
        assert torch.equal(x, y), (p.P, S, (x - y).abs().max().item())


def test_batch_expmid_and_recapture_on_new_buffers():
    systems = _systems(seed=1)
    batch, xs = _run_batch(systems, 2, 0.01, rsg.EXPMID)
    # a second call with fresh buffers must not reuse the old graph's pointers
    ys = [p.states_to_gpu(psi) for p, psi, _ in systems]
    batch.propagate(ys, 2, 0.01, scheme=rsg.EXPMID)
    torch.cuda.synchronize()
    for (p, psi, S), x, y in zip(systems, xs, ys):
        assert rel_err(p.states_from_gpu(y, S), p.states_from_gpu(x, S)) < 1e-6
        want, _ = p.O.propagate(psi, 2, 0.01, scheme=oracle.EXPMID)
        assert rel_err(p.states_from_gpu(y, S), want) < 2e-5


def test_batch_with_gram_schmidt():
    systems = _systems(seed=2)
    _, xs = _run_batch(systems, 4, 0.02, rsg.ETRS, gs_every=2)
    for (p, psi, S), x in zip(systems, xs):
        got = p.states_from_gpu(x, S)
        G = p.h ** 3 * got.conj().T @ got
        assert np.abs(G - np.eye(S)).max() < 1e-5


def test_batch_mixed_projector_counts_falls_back():
    """The per-stage path propagates the systems one by one when projector
    set sizes differ."""
    systems = _systems(lmax_of=lambda i: i % 2, seed=3)     # npmax 1 and 4 mixed
    batch, xs = _run_batch(systems, 2, 0.02, rsg.ETRS, persistent=0)
    assert batch.get_option("batched") == 0
    for (p, psi, S), x in zip(systems, xs):
        want, _ = p.O.propagate(psi, 2, 0.02, scheme=oracle.ETRS)
        assert rel_err(p.states_from_gpu(x, S), want) < 2e-5


# systems with more than 16 states (16-value chunks), and s, p and d
# projector sets mixed in one persistent step
WIDE_SPECS = [(12, 20, 2), (16, 3, 1), (10, 33, 1), (14, 16, 2), (9, 1, 1), (18, 7, 2)]


@pytest.mark.parametrize("persistent", [1, 0])
def test_batch_wide_blocks_and_mixed_lmax_against_oracle(persistent):
    systems = _systems(lmax_of=lambda i: i % 3, seed=5, specs=WIDE_SPECS)
    batch, xs = _run_batch(systems, 2, 0.02, rsg.ETRS, persistent=persistent)
    assert batch.get_option("batched") == (1 if persistent else 0)
    for (p, psi, S), x in zip(systems, xs):
        want, _ = p.O.propagate(psi, 2, 0.02, scheme=oracle.ETRS)
        assert rel_err(p.states_from_gpu(x, S), want) < 2e-5, (p.P, S)


@pytest.mark.parametrize("zseg", [8, 13, 40])
def test_persistent_batch_short_segments(zseg):
    """Several z segments per tile column (and segments shorter than the
    pipeline), EXPMID: the same result as the one-segment step."""
    systems = _systems(seed=6)
    _, xs = _run_batch(systems, 2, 0.02, rsg.EXPMID)
    _, ys = _run_batch(systems, 2, 0.02, rsg.EXPMID, zseg=zseg)
    for (p, psi, S), x, y in zip(systems, xs, ys):
        assert torch.equal(x, y), (zseg, p.P, S)


def test_persistent_batch_bounded_wait_times_out_and_recovers():
    """A dependency that is never met (debug_stall) makes the step's waits
    run out: the call returns RSG_ERR_TIMEOUT, and the next step on the same
    context is correct."""
    systems = _systems(seed=7)
    batch = rsg.Batch([p.H for p, _, _ in systems], [S for _, _, S in systems])
    xs = [p.states_to_gpu(psi) for p, psi, _ in systems]
    batch.set_option("wait_limit", 2000)
    batch.set_option("debug_stall", 1)
    with pytest.raises(rsg.RSGError, match="RSG_ERR_TIMEOUT"):
        batch.propagate(xs, 1, 0.02, scheme=rsg.ETRS)
    batch.set_option("debug_stall", 0)
    batch.set_option("wait_limit", 1 << 22)
    xs = [p.states_to_gpu(psi) for p, psi, _ in systems]
    batch.propagate(xs, 2, 0.02, scheme=rsg.ETRS)
    torch.cuda.synchronize()
    for (p, psi, S), x in zip(systems, xs):
        want, _ = p.O.propagate(psi, 2, 0.02, scheme=oracle.ETRS)
        assert rel_err(p.states_from_gpu(x, S), want) < 2e-5


def test_persistent_batch_falls_back_above_128_states():
    """Systems with more than 128 values per point are propagated one by one."""
    systems = _systems(seed=8, specs=[(8, 130, 1), (10, 4, 1)])
    batch, xs = _run_batch(systems, 1, 0.02, rsg.ETRS)
    assert batch.get_option("batched") == 0
    for (p, psi, S), x in zip(systems, xs):
        want, _ = p.O.propagate(psi, 1, 0.02, scheme=oracle.ETRS)
        assert rel_err(p.states_from_gpu(x, S), want) < 2e-5


def test_batch_tile_variants_and_autotune():
    """Both tile variants of every record length give the same step (the
    arithmetic per point does not depend on the tile), and the autotuner
    leaves the states it times untouched and keeps a valid configuration."""
    specs = [(12, 5, 1), (16, 7, 1), (10, 9, 1), (14, 11, 2), (9, 13, 1), (18, 3, 1)]
    systems = _systems(seed=9, specs=specs, atoms=False)
    _, xs = _run_batch(systems, 2, 0.02, rsg.ETRS, tile_variants=0)
    _, ys = _run_batch(systems, 2, 0.02, rsg.ETRS, tile_variants=255)
    for (p, psi, S), x, y in zip(systems, xs, ys):
        assert torch.equal(x, y), (p.P, S)
    systems = _systems(seed=10, specs=specs)
    batch = rsg.Batch([p.H for p, _, _ in systems], [S for _, _, S in systems])
    xs = [p.states_to_gpu(psi) for p, psi, _ in systems]
    before = [x.clone() for x in xs]
    ms = batch.autotune(xs, 0.02)
    assert ms > 0
    assert all(torch.equal(a, b) for a, b in zip(xs, before))
    batch.propagate(xs, 2, 0.02, scheme=rsg.ETRS)
    torch.cuda.synchronize()
    for (p, psi, S), x in zip(systems, xs):
        want, _ = p.O.propagate(psi, 2, 0.02, scheme=oracle.ETRS)
        assert rel_err(p.states_from_gpu(x, S), want) < 2e-5

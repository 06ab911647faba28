"""Benchmark: H|psi> throughput inside Taylor-4 ETRS propagation on one GB300.

Workload (the single large system): spherical mesh of radius 18 bohr at
spacing 0.2 bohr (3,053,617 points, row-indexed), 64 complex64 states of
white noise, V_loc = 32 Gaussian wells (depth U[1,4] Ha, width U[0.8,1.5]
bohr), 32 atoms x 4 projectors (s + p) on 2.5-bohr spheres, h_ij diagonal in
U[-1,1].  One step = one ETRS time step (dt = 0.01 au): two Taylor-4
exponentials = 8 Hamiltonian applications with the projector terms, each a
Horner stage u' = psi + (-i tau/k) H u.

metric: grid-point.states per second of H applications (x1e9), i.e.
P * S * 8 * steps / time.  Inputs (1.56 GB per state block) exceed L2
(129 MB), so no flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one H application to one state on the full
mesh per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "sphere R=18 bohr h=0.2 (3,053,617 pts), 64 states, 32 wells, 32 atoms x 4 projectors, ETRS Taylor-4 dt=0.01"
METRIC = "H|psi> grid-point.states/s (ETRS Taylor-4 step, sphere R=18 h=0.2, 64 states)"
UNIT = "Gpoint.states/s"
N_APPLY_PER_STEP = 8


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def reduce_max(value, ws, device="cpu"):
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ms_max, ws, units_per_rank_per_step, steps):
    """Whole-job throughput in 1e9 units/s: every rank did the same work in
    at most ms_max milliseconds (weak scaling)."""
    return ws * units_per_rank_per_step * steps / (ms_max * 1e-3) / 1e9


def build_inputs(g_seed=2):
    """Seeded inputs of the workload: potential, projector parameters."""
    from workloads import gaussian_wells, projector_atoms, rng
    g = rng(g_seed)
    c, d, w = gaussian_wells(g, 32, 18.0 - 2.5)
    cen, rc, lm, beta, hm = projector_atoms(g, 32, 2.5, 1, ball_radius=18.0 - 2.5)
    return g, (c, d, w), (cen, rc, lm, beta, hm)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# stencil kernel of each "kernel" option value (rsg_ham_get_option "last_kernel")
KERNEL_NAMES = {0: "k_apply_staged", 1: "k_apply_naive", 2: "k_apply_zmarch", 3: "k_apply_tma",
                4: "k_apply_rowtma", 5: "k_apply_quad", 7: "k_apply_wide"}
# the files the dominant stencil kernel (k_apply_wide) is compiled from; the
# public header it also includes holds only C declarations the kernel does
# not use
KERNEL_SOURCES = ("rsg_wide.cu", "rsg_vec.cuh", "rsg_async.cuh", "rsg_internal.h")


def traffic_record(kernel_src_hash, kernel_name):
    """DRAM bytes per launch of the stencil kernel from the committed ncu
    summary, if it was taken on the current kernel source and kernel."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_sha256") != kernel_src_hash or kernel_name not in d.get("kernel", ""):
        return None
    return d.get("bytes_per_launch_full_size")


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1501_05654_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: a temporary file unless RSG_CLOCK_LOG_DIR names a folder to keep them in
        folder = os.environ.get("RSG_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def lib_to_orc(lib_ijk, orc_ijk):
    """idx with library point i = oracle point idx[i] (matched by lattice coordinates)."""
    a = np.lexsort(np.asarray(lib_ijk).T[::-1])
    b = np.lexsort(np.asarray(orc_ijk).T[::-1])
    idx = np.empty(len(a), dtype=np.int64)
    idx[a] = b
    return idx


def rel_err(got, want):
    """Largest over states of max_p |got - want| / max_p |want|."""
    got, want = np.asarray(got), np.asarray(want)
    if got.ndim == 1:
        got, want = got[:, None], want[:, None]
    den = np.abs(want).max(axis=0)
    den[den == 0] = 1.0
    return float((np.abs(got - want).max(axis=0) / den).max())


def oracle_leg(chk, wells, proj, seconds=20.0):
    """The FP64 oracle, as it stands, on the host cores.

    Times it (the headline workload with all threads and with one thread,
    and bounded samples of the other workloads, extrapolated where stated)
    and compares every result collected in chk with it.  Returns
    (cpu_baseline, legs, errors)."""
    import oracle
    from workloads import (potential_double_well, potential_harmonic, potential_soft_coulomb_li,
                           potential_wells, potential_wells_scaled, rng, white_noise_states)
    errs, legs = {}, {}
    nthr = oracle.num_threads()
    om = oracle.Mesh(oracle.SPHERE, radius=18.0, h=0.2)
    O = oracle.Hamiltonian(om, potential_wells(om.xyz, *wells))
    O.set_projectors(*proj)
    # the headline timing: H applications to one state on the full mesh
    x1 = white_noise_states(rng(2, 5), om.P, 1)

    def timed_applies(secs, cap):
        n, t0 = 0, time.perf_counter()
        while True:
            O.apply(x1)
            n += 1
            dt = time.perf_counter() - t0
            if dt > secs or n >= cap:
                return n, dt
    n, dt = timed_applies(seconds, 5000)
    base = {"value": om.P * n / dt / 1e9, "unit": UNIT, "cores": nthr, "kind": "oracle",
            "sample": f"{n} FP64 H applications to 1 state on the full 3,053,617-point sphere "
                      f"(wells + projectors), {dt:.1f} s"}
    oracle.set_num_threads(1)
    try:
        n1, dt1 = timed_applies(seconds / 2, 5000)
    finally:
        oracle.set_num_threads(nthr)
    legs["sphere_R18_1_thread"] = {"value": om.P * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                                   "sample": f"{n1} H applications to 1 state, {dt1:.1f} s"}
    hd = chk.get("headline")
    if hd is not None:
        idx = lib_to_orc(hd["lib_ijk"], om.ijk)
        S = hd["psi"].shape[1]
        psi = np.empty((om.P, S), dtype=np.complex128)
        psi[idx] = hd["psi"]
        samp = idx[hd["samp"]]
        pidx, sidx = np.repeat(samp, S), np.tile(np.arange(S), len(samp))
        t0 = time.perf_counter()
        want = O.apply_sampled(psi, pidx, sidx).reshape(len(samp), S)
        legs["sphere_R18_sampled_apply_s"] = time.perf_counter() - t0
        errs["headline"] = {"h_apply_sampled": rel_err(hd["y"], want),
                            "sample": f"{len(samp)} random points x {S} states, one application, "
                                      f"kernel {hd['kernel']}"}
        for name in ("c64_plain_kernel", "c128_default", "c128_staged_kernel"):
            if name in chk:
                errs[name] = {"h_apply_sampled": rel_err(chk[name]["y"], want),
                              "sample": "the headline's sampled points and input"}
        if "complex_scaling_c64" in chk:
            c = chk["complex_scaling_c64"]
            vt = potential_wells_scaled(om.xyz, *wells, c["theta"])
            wz = om.apply_scaled_sampled(psi, c["theta"], vt, pidx, sidx).reshape(len(samp), S)
            errs["complex_scaling_c64"] = {"h_apply_sampled": rel_err(c["y"], wz),
                                           "sample": "the headline's sampled points and input"}
        del psi
    sm = chk.get("etrs_small")
    if sm is not None:
        o6 = oracle.Mesh(oracle.SPHERE, radius=sm["radius"], h=0.2)
        O6 = oracle.Hamiltonian(o6, potential_wells(o6.xyz, *sm["wells"]))
        O6.set_projectors(*sm["proj"])
        idx = lib_to_orc(sm["lib_ijk"], o6.ijk)
        psi = np.empty((o6.P, sm["psi"].shape[1]), dtype=np.complex128)
        psi[idx] = sm["psi"]
        t0 = time.perf_counter()
        got, _ = O6.propagate(psi, 1, 0.01, scheme=oracle.ETRS)
        legs["sphere_R6_etrs_step_s"] = time.perf_counter() - t0
        errs["headline"]["etrs_step"] = rel_err(sm["out"], got[idx])
        errs["headline"]["etrs_step_sample"] = (f"sphere R={sm['radius']:g} h=0.2 ({o6.P:,} points) with wells and "
                                                f"projectors, {sm['psi'].shape[1]} states, one ETRS step, kernel "
                                                f"{sm['kernel']}")
    if "batch_256_systems" in chk:
        e = []
        for sy in chk["batch_256_systems"]["systems"]:
            ob = oracle.Mesh(oracle.CUBE, sy["n"], h=0.25)
            Ob = oracle.Hamiltonian(ob, potential_wells(ob.xyz, *sy["wells"]))
            Ob.set_projectors(*sy["proj"])
            idx = lib_to_orc(sy["lib_ijk"], ob.ijk)
            psi = np.empty((ob.P, sy["psi"].shape[1]), dtype=np.complex128)
            psi[idx] = sy["psi"]
            got, _ = Ob.propagate(psi, 1, 0.02, scheme=oracle.ETRS)
            e.append(rel_err(sy["out"], got[idx]))
        errs["batch_256_systems"] = {"etrs_step": max(e), "sample": "the 3 smallest systems, one batched ETRS step"}
    if "batch_sample" in chk:
        bsm = chk["batch_sample"]
        ps, tb = 0, 0.0
        for n_, S_, (wl, pj) in zip(bsm["n"], bsm["S"], bsm["par"]):
            ob = oracle.Mesh(oracle.CUBE, n_, h=0.25)
            Ob = oracle.Hamiltonian(ob, potential_wells(ob.xyz, *wl))
            Ob.set_projectors(*pj)
            xb = white_noise_states(rng(9), ob.P, S_)
            t0 = time.perf_counter()
            Ob.apply(xb)
            tb += time.perf_counter() - t0
            ps += ob.P * S_
        legs["batch_256_systems"] = {"value": ps / tb / 1e9, "unit": UNIT, "cores": nthr,
                                     "step_s_extrapolated": N_APPLY_PER_STEP * bsm["point_states_all"] / (ps / tb),
                                     "sample": f"one H application on each of the first 16 systems ({ps:,} "
                                               f"point-states, {tb:.1f} s); the step time is extrapolated to all "
                                               f"256 systems by point-states"}
    if "large_cube_192" in chk:
        c5 = chk["large_cube_192"]
        o5 = oracle.Mesh(oracle.CUBE, 192, h=0.18)
        O5 = oracle.Hamiltonian(o5, potential_wells(o5.xyz, *c5["wells"]))
        O5.set_projectors(*c5["proj"])
        idx = lib_to_orc(c5["lib_ijk"], o5.ijk)
        psi = np.empty((o5.P, 8), dtype=np.complex128)
        psi[idx] = c5["psi"]
        t0 = time.perf_counter()
        got, _ = O5.propagate(psi, 1, 0.01, scheme=oracle.ETRS, gs_every=1)
        t5 = time.perf_counter() - t0
        errs["large_cube_192"] = {"etrs_step_with_gram_schmidt": rel_err(c5["out"], got[idx]),
                                  "sample": "states 0-7 of 128 (independent of 8-127 under index-order "
                                            "orthonormalisation), one ETRS step then Gram-Schmidt"}
        legs["large_cube_192"] = {"s_per_step_8_states": t5, "cores": nthr,
                                  "s_1000_steps_128_states_extrapolated": t5 * 1000 * 16,
                                  "sample": "states 0-7, one ETRS step with Gram-Schmidt; extrapolated to 128 "
                                            "states and 1000 steps"}
        del psi, got
    for dt_name in ("c128", "c64"):
        cg = chk.get(f"control_gradient_{dt_name}")
        if cg is None:
            continue
        o4 = oracle.Mesh(oracle.CUBE, 64, h=0.3)
        O4 = oracle.Hamiltonian(o4, potential_double_well(o4.xyz, 0.02, 2.0, 0.5))
        idx = lib_to_orc(cg["lib_ijk"], o4.ijk)
        a = np.empty(o4.P, dtype=np.complex128)
        b = np.empty(o4.P, dtype=np.complex128)
        a[idx], b[idx] = cg["psi0"], cg["target"]
        t0 = time.perf_counter()
        Jw, gw = O4.control_gradient(a, b, cg["eps"], 0.05, scheme=oracle.ETRS, nsub=4, checkpoint_every=50)
        t4 = time.perf_counter() - t0
        errs[f"control_gradient_{dt_name}"] = {
            "J": abs(cg["J"] - Jw) / abs(Jw), "gradient": float(np.abs(cg["grad"] - gw).max() / np.abs(gw).max()),
            "sample": "the first 5 intervals of the workload (its field, states and operator)"}
        if dt_name == "c128":
            nint = len(cg["eps"])
            legs["control_gradient"] = {"s_forward_and_gradient_5_intervals": t4, "cores": nthr,
                                        "s_2000_intervals_extrapolated": t4 * 2000 / nint,
                                        "sample": "oracle forward + discrete adjoint, 5 intervals of 4 ETRS "
                                                  "substeps, extrapolated to 2000"}
    ss = chk.get("shifted_solve_c64")
    if ss is not None and hd is not None:
        idx = lib_to_orc(hd["lib_ijk"], om.ijk)
        xs = np.empty_like(ss["x"])
        bs = np.empty_like(ss["b"])
        xs[idx], bs[idx] = ss["x"], ss["b"]
        r = bs - (O.apply(xs) - ss["z"] * xs)
        errs["shifted_solve_c64"] = {"true_relative_residual": float(
            (np.linalg.norm(r, axis=0) / np.linalg.norm(bs, axis=0)).max()),
            "sample": "all 8 right-hand sides, residual of the returned solutions under the oracle's operator"}
    eg = chk.get("eigensolve_li_model")
    if eg is not None:
        ol = oracle.Mesh(oracle.CUBE, 61, h=0.4)
        Ol = oracle.Hamiltonian(ol, potential_soft_coulomb_li(ol.xyz))
        idx = lib_to_orc(eg["lib_ijk"], ol.ijk)
        xe = np.empty_like(eg["x"])
        xe[idx] = eg["x"]
        r = Ol.apply(xe) - xe * eg["ev"][None, :]
        rel = np.linalg.norm(r, axis=0) / (np.abs(eg["ev"]) * np.linalg.norm(xe, axis=0))
        errs["eigensolve_li_model"] = {"relative_residual": float(rel.max()),
                                       "sample": "the four wanted pairs under the oracle's operator"}
    ho = chk.get("oscillator_32_c128")
    if ho is not None:
        o1 = oracle.Mesh(oracle.CUBE, 32, h=0.3)
        O1 = oracle.Hamiltonian(o1, potential_harmonic(o1.xyz, 0.5))
        idx = lib_to_orc(ho["lib_ijk"], o1.ijk)
        psi = np.empty_like(ho["psi"])
        psi[idx] = ho["psi"]
        t0 = time.perf_counter()
        got, _ = O1.propagate(psi, 100, 0.01, scheme=oracle.EXPMID)
        t1 = time.perf_counter() - t0
        errs["oscillator_32_c128"] = {"propagation_100_steps": rel_err(ho["out"], got[idx]),
                                      "sample": "the whole run: 4 states, 100 steps"}
        legs["oscillator_32_c128"] = {"s_100_steps": t1, "cores": nthr, "sample": "the whole run"}
    return base, legs, errs


def collect_headline_checks(H, mesh, psi_h, kname):
    """One application of the headline Hamiltonian to the headline input at
    4096 seeded points, and one ETRS step of a small sphere built the same
    way with the same stencil kernel (kept on the host for the oracle leg)."""
    import torch
    import paper_1501_05654_gb300 as rsg
    from workloads import gaussian_wells, potential_wells, projector_atoms, rng, white_noise_states
    chk = {}
    x = psi_h.to("cuda")
    y = H.apply(x)
    samp = rng(11).choice(mesh.P, 4096, replace=False)
    torch.cuda.synchronize()
    chk["headline"] = {"lib_ijk": mesh.ijk, "psi": psi_h.numpy(), "samp": samp, "kernel": kname,
                       "y": y[torch.from_numpy(samp).cuda()].cpu().numpy().astype(np.complex128)}
    del x, y
    g6 = rng(12)
    m6 = rsg.Mesh(rsg.SPHERE, radius=6.0, spacing=0.2)
    w6 = gaussian_wells(g6, 8, 3.5)
    p6 = projector_atoms(g6, 4, 2.5, 1, ball_radius=3.5)
    H6 = rsg.Hamiltonian(m6, torch.complex64)
    H6.set_potential(potential_wells(m6.xyz, *w6))
    H6.set_projectors(*p6)
    for k in ("kernel", "wide_ty", "producers", "zseg", "stages", "threads"):
        H6.set_option(k, H.get_option(k))
    x6 = white_noise_states(g6, m6.P, 64, dtype=np.complex64)
    t6 = torch.from_numpy(x6).cuda()
    H6.propagate(t6, 1, 0.01, scheme=rsg.ETRS, want_drift=False)
    torch.cuda.synchronize()
    chk["etrs_small"] = {"radius": 6.0, "wells": w6, "proj": p6, "lib_ijk": m6.ijk, "psi": x6.astype(np.complex128),
                         "out": t6.cpu().numpy().astype(np.complex128),
                         "kernel": KERNEL_NAMES.get(H6.get_option("last_kernel"), "unknown")}
    return chk


def time_steps(H, psi, steps, fn):
    import torch
    for _ in range(2):
        fn(psi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn(psi)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def batch_extra(chk, peak, steps=10, nsys=256, tune=True):
    """The batch of 256 uneven systems: ms per ETRS step through the batched
    launch, and (with chk) the host copies the oracle leg checks.  nsys < 256
    keeps the first nsys systems (profiler captures)."""
    import torch
    import paper_1501_05654_gb300 as rsg
    from workloads import potential_wells, projector_atoms, rng
    out = {}
    # batch of 256 uneven systems (cubes 24^3..96^3 at h = 0.25, 1..16 states,
    # 1..8 atoms x 4 projectors), autotuned, then timed through the batched step
    from workloads import batch_systems, gaussian_wells
    gb = rng(3)
    ns, Ss, nas = batch_systems(gb, 256)
    hams, psis, pst, bpar = [], [], 0, []
    for n, S_, na in list(zip(ns, Ss, nas))[:nsys]:
        m = rsg.Mesh(rsg.CUBE, int(n), spacing=0.25)
        half = 0.5 * (n - 1) * 0.25
        c, d, w = gaussian_wells(gb, int(na), 0.0, cube_half=0.6 * half)
        Hb = rsg.Hamiltonian(m, torch.complex64)
        Hb.set_potential(potential_wells(m.xyz, c, d, w))
        pj = projector_atoms(gb, int(na), 2.5, 1, cube_half=0.6 * half)
        Hb.set_projectors(*pj)
        bpar.append(((c, d, w), pj))
        hams.append(Hb)
        psis.append(torch.randn((m.P, rsg.padded_ld(int(S_), torch.complex64)), dtype=torch.complex64,
                                device="cuda") * 1e-3)
        pst += m.P * int(S_)
    batch = rsg.Batch(hams, [int(x) for x in Ss[:nsys]])
    tune_ms = batch.autotune(psis, 0.02, scheme=rsg.ETRS) if tune else None
    tuned = {k: batch.get_option(k) for k in ("persistent", "zseg", "tile_variants", "launches_per_step",
                                              "items_per_stage", "blocks")}
    ms = time_steps(None, psis, steps, lambda xs: batch.propagate(xs, 1, 0.02, scheme=rsg.ETRS))
    if chk is not None:
        # one more batched step; the three smallest systems are checked
        small = [int(i) for i in np.argsort(ns)[:3]]
        ins = [psis[i][:, :int(Ss[i])].cpu().numpy().astype(np.complex128) for i in small]
        batch.propagate(psis, 1, 0.02, scheme=rsg.ETRS)
        torch.cuda.synchronize()
        chk["batch_256_systems"] = {
            "kind": "batch", "systems": [
                {"n": int(ns[i]), "wells": bpar[i][0], "proj": bpar[i][1], "lib_ijk": hams[i].mesh.ijk,
                 "psi": x_in, "out": psis[i][:, :int(Ss[i])].cpu().numpy().astype(np.complex128)}
                for i, x_in in zip(small, ins)]}
        # the oracle leg times single applications on the first 16 systems
        chk["batch_sample"] = {"n": [int(v) for v in ns[:16]], "S": [int(v) for v in Ss[:16]],
                               "par": bpar[:16], "point_states_all": pst}
    # algorithmic stencil bytes of one step (read u, read psi, write, V per
    # Horner stage) over the whole step time: a lower bound on the batched
    # stencil's own fraction, since the step also holds the projector kernels
    sbytes = N_APPLY_PER_STEP * sum(h.mesh.P * (3 * x.shape[1] * 8 + 4) for h, x in zip(hams, psis))
    out["batch_256_systems"] = {"ms_per_step": ms, "point_states": pst, "autotuned": tuned,
                                "autotune_best_ms": tune_ms,
                                "value": pst * N_APPLY_PER_STEP / (ms * 1e-3) / 1e9, "unit": UNIT,
                                "step_stencil_GBps": sbytes / (ms * 1e-3) / 1e9,
                                "step_frac_of_measured_hbm": sbytes / (ms * 1e-3) / 1e9 / peak,
                                "workload": "256 cubes n~U{24..96} h=0.25, S~U{1..16}, 1..8 atoms x 4 "
                                            "projectors, ETRS dt=0.02, one captured graph per step "
                                            "(persistent: one launch per step)"}
    del batch, hams, psis
    torch.cuda.empty_cache()
    return out


def control_extra(chk, nint=2000, dtypes=None):
    """The optimal-control workload: time of one control gradient (discrete
    adjoint with checkpoints) against one forward propagation, 64^3 double
    well, nint intervals of 0.05 au, 4 ETRS substeps, checkpoints every 50."""
    import torch
    import paper_1501_05654_gb300 as rsg
    from workloads import control_field, potential_double_well, rng, white_noise_states
    if dtypes is None:
        dtypes = (torch.complex128, torch.complex64)
    out = {}
    cm = rsg.Mesh(rsg.CUBE, 64, spacing=0.3)
    gg = rng(4)
    eps = control_field(gg, nint, 0.05)
    for dtype in dtypes:
        H = rsg.Hamiltonian(cm, dtype)
        H.set_potential(potential_double_well(cm.xyz, 0.02, 2.0, 0.5))
        x = torch.from_numpy(white_noise_states(gg, cm.P, 1)[:, 0]).to(dtype).cuda()
        x /= torch.linalg.vector_norm(x) * cm.h ** 1.5
        tgt = torch.roll(x, 1).contiguous()
        ld = rsg.padded_ld(1, dtype)
        blk = torch.zeros((cm.P, ld), dtype=dtype, device="cuda")
        blk[:, 0] = x
        torch.cuda.synchronize()
        H.kernel_stats()                  # reset the library's counters
        t0 = time.perf_counter()
        H.propagate(blk, nint, 0.05, scheme=rsg.ETRS, nsub=4, eps=eps, want_drift=False, S=1)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        nf = H.kernel_stats()[1]          # Hamiltonian applications of the forward propagation
        t0 = time.perf_counter()
        J, grad = H.control_gradient(x, tgt, eps, 0.05, scheme=rsg.ETRS, nsub=4, checkpoint_every=50)
        tg = time.perf_counter() - t0
        ng = H.kernel_stats()[1]          # ... of the gradient (forward, recompute, costate)
        if chk is not None:
            # the first 5 intervals of the same problem, for the oracle
            J5, g5 = H.control_gradient(x, tgt, eps[:5], 0.05, scheme=rsg.ETRS, nsub=4, checkpoint_every=50)
            chk[f"control_gradient_{'c128' if dtype == torch.complex128 else 'c64'}"] = {
                "kind": "gradient", "lib_ijk": cm.ijk, "psi0": x.cpu().numpy().astype(np.complex128),
                "target": tgt.cpu().numpy().astype(np.complex128), "eps": np.array(eps[:5]), "J": J5,
                "grad": np.array(g5)}
        out[f"control_gradient_{'c128' if dtype == torch.complex128 else 'c64'}"] = {
            "forward_s": tf, "gradient_s": tg, "ratio": tg / tf,
            "h_applications_forward": nf, "h_applications_gradient": ng, "h_application_ratio": ng / nf,
            "workload": f"64^3 h=0.3 double well, {nint} intervals dt=0.05, ETRS nsub=4, K=50"}
        del H, blk
    return out


def extras(mesh, wells, proj, g, chk):
    """Side measurements on the same GPU: the FP64 (complex128) path with the
    default and the plain one-thread-per-value stencil, the FP32 plain
    stencil, and the optimal-control adjoint gradient against a forward
    propagation of the control workload (64^3 double well, dipole field,
    2000 intervals of dt = 0.05 au, 4 ETRS substeps, checkpoints every 50).

    chk (a dict, or None) collects host copies of inputs and results that the
    oracle leg compares against the FP64 oracle: for every workload a small
    sample (sampled points of one application, a short prefix of a
    propagation or of a gradient)."""
    import torch
    import paper_1501_05654_gb300 as rsg
    from workloads import (control_field, gaussian_wells, potential_double_well, potential_wells,
                           projector_atoms, rng, white_noise_states)
    out = {}
    hd = chk.get("headline") if chk is not None else None

    def sampled_apply(Hx, dtype_):
        """One application of Hx to the headline input, at the headline's sampled points."""
        x = torch.from_numpy(hd["psi"]).to(dtype_).cuda()
        y = Hx.apply(x)
        torch.cuda.synchronize()
        ys = y[torch.from_numpy(hd["samp"]).cuda()].cpu().numpy().astype(np.complex128)
        del x, y
        return ys
    peak, _ = peaks()
    P, S = mesh.P, 64
    # the headline step with the projector coefficients on a side stream next
    # to the stencil (option proj_overlap; the headline runs them in line so
    # that the stencil's CUDA-event time is its own)
    Ho = rsg.Hamiltonian(mesh, torch.complex64)
    Ho.set_potential(potential_wells(mesh.xyz, *wells))
    Ho.set_projectors(*proj)
    Ho.set_option("proj_overlap", 1)
    psi = torch.from_numpy(white_noise_states(g, P, S, dtype=np.complex64)).cuda()
    ms = time_steps(Ho, psi, 10, lambda x: Ho.propagate(x, 1, 0.01, scheme=rsg.ETRS, want_drift=False))
    out["headline_proj_overlap"] = {"ms_per_step": ms, "value": P * S * N_APPLY_PER_STEP / (ms * 1e-3) / 1e9,
                                    "unit": UNIT, "workload": "the headline step, proj_overlap = 1"}
    del psi, Ho
    torch.cuda.empty_cache()
    for name, dtype, kernel in (("c64_plain_kernel", torch.complex64, 1),
                                ("c128_default", torch.complex128, None),
                                ("c128_staged_kernel", torch.complex128, 0)):
        H = rsg.Hamiltonian(mesh, dtype)
        H.set_potential(potential_wells(mesh.xyz, *wells))
        H.set_projectors(*proj)
        if kernel is not None:
            H.set_option("kernel", kernel)
        npdt = np.complex64 if dtype == torch.complex64 else np.complex128
        psi = torch.from_numpy(white_noise_states(g, P, S, dtype=npdt)).cuda()
        ms = time_steps(H, psi, 2, lambda x: H.propagate(x, 1, 0.01, scheme=rsg.ETRS, want_drift=False))
        out[name] = {"ms_per_step": ms, "value": P * S * N_APPLY_PER_STEP / (ms * 1e-3) / 1e9,
                     "unit": UNIT}
        del psi
        if hd is not None:
            chk[name] = {"kind": "sampled_apply", "y": sampled_apply(H, dtype)}
        del H
        torch.cuda.empty_cache()
    # complex scaling on the headline mesh: the same wells at r e^{0.3 i}, no
    # projectors (refused while scaling is set), 64 complex64 states, ETRS
    from workloads import potential_wells_scaled
    Hz = rsg.Hamiltonian(mesh, torch.complex64)
    Hz.set_complex_scaling(0.3, potential_wells_scaled(mesh.xyz, *wells, 0.3))
    psi = torch.from_numpy(white_noise_states(g, P, S, dtype=np.complex64)).cuda()
    Hz.profile(True)
    ms = time_steps(Hz, psi, 2, lambda x: Hz.propagate(x, 1, 0.01, scheme=rsg.ETRS, want_drift=False))
    kms, kn, kbytes, _ = Hz.kernel_stats()
    Hz.profile(False)
    zk = Hz.get_option("last_kernel")
    if hd is not None:
        del psi
        chk["complex_scaling_c64"] = {"kind": "sampled_apply_scaled", "theta": 0.3,
                                      "y": sampled_apply(Hz, torch.complex64)}
        psi = None
    out["complex_scaling_c64"] = {"ms_per_step": ms, "value": P * S * N_APPLY_PER_STEP / (ms * 1e-3) / 1e9,
                                  "unit": UNIT,
                                  "kernel": {5: "k_apply_quad (complex diagonal)",
                                             7: "k_apply_wide (complex diagonal)"}.get(zk, "k_apply_scaled"),
                                  "kernel_GBps": kbytes / (kms * 1e-3) / 1e9 if kms > 0 else None,
                                  "kernel_frac_of_measured_hbm": kbytes / (kms * 1e-3) / 1e9 / peak if kms > 0 else None,
                                  "workload": "sphere R=18 h=0.2, 32 wells at r e^{0.3i}, 64 states, ETRS dt=0.01"}
    del psi, Hz
    torch.cuda.empty_cache()
    out.update(batch_extra(chk, peak))
    # large cube: 192^3 at h = 0.18, 128 smooth complex64 states, 64 atoms x 9
    # projectors (s, p, d) on 3-bohr spheres, ETRS dt = 0.01, FP64-checked
    # Cholesky-QR every 50 steps; drift = max |<psi|psi> - 1| before it
    gl = rng(5)
    cm5 = rsg.Mesh(rsg.CUBE, 192, spacing=0.18)
    half = 0.5 * 191 * 0.18
    c5, d5, w5 = gaussian_wells(gl, 64, 0.0, cube_half=half - 3.0)
    H5 = rsg.Hamiltonian(cm5, torch.complex64)
    H5.set_potential(potential_wells(cm5.xyz, c5, d5, w5))
    cen, rc, lm, beta, hm = projector_atoms(gl, 64, 3.0, 2, cube_half=half - 3.0)
    cen[:] = c5                                   # projectors sit on the wells
    H5.set_projectors(cen, rc, lm, beta, hm)
    xyz = torch.from_numpy(cm5.xyz).to("cuda", torch.float32)
    S5 = 128
    x5 = torch.empty((cm5.P, S5), dtype=torch.complex64, device="cuda")
    cs = torch.from_numpy(gl.uniform(-0.5 * half, 0.5 * half, (S5, 3))).to("cuda", torch.float32)
    ks = torch.from_numpy(gl.uniform(-0.5, 0.5, (S5, 3))).to("cuda", torch.float32)
    sg = torch.from_numpy(gl.uniform(1.0, 2.0, S5)).to("cuda", torch.float32)
    for s_ in range(S5):
        r2 = ((xyz - cs[s_]) ** 2).sum(1)
        x5[:, s_] = torch.polar(torch.exp(-r2 / (4 * sg[s_] ** 2)), xyz @ ks[s_])
    H5.orthonormalize(x5)
    H5.profile(True)
    ms5 = time_steps(None, x5, 3, lambda x: H5.propagate(x, 1, 0.01, scheme=rsg.ETRS, want_drift=False))
    k5_ms, _, k5_bytes, _ = H5.kernel_stats()
    H5.profile(False)
    k5_name = KERNEL_NAMES.get(H5.get_option("last_kernel"), "unknown")
    torch.cuda.synchronize()
    g0 = time.perf_counter()
    H5.orthonormalize(x5)
    gs_s = time.perf_counter() - g0
    if chk is not None:
        # one step with Gram-Schmidt after it; states 0-7 go to the oracle
        # (index-order orthonormalisation makes them independent of 8-127)
        x_in = x5[:, :8].cpu().numpy().astype(np.complex128)
        H5.propagate(x5, 1, 0.01, scheme=rsg.ETRS, gs_every=1, want_drift=False)
        torch.cuda.synchronize()
        chk["large_cube_192"] = {"kind": "propagate", "wells": (c5, d5, w5), "proj": (cen, rc, lm, beta, hm),
                                 "lib_ijk": cm5.ijk, "psi": x_in,
                                 "out": x5[:, :8].cpu().numpy().astype(np.complex128)}
    # the workload's full length: 1000 ETRS steps, Cholesky-QR every 50;
    # per state, the largest |<psi|psi> - 1| seen before a re-orthonormalisation
    t5 = time.perf_counter()
    drift = H5.propagate(x5, 1000, 0.01, scheme=rsg.ETRS, gs_every=50)
    torch.cuda.synchronize()
    t5 = time.perf_counter() - t5
    k5_gbs = k5_bytes / (k5_ms * 1e-3) / 1e9 if k5_ms > 0 else None
    out["large_cube_192"] = {"ms_per_step": ms5, "value": cm5.P * S5 * N_APPLY_PER_STEP / (ms5 * 1e-3) / 1e9,
                             "unit": UNIT, "kernel": k5_name, "kernel_GBps": k5_gbs,
                             "kernel_frac_of_measured_hbm": k5_gbs / peak if k5_gbs else None,
                             "gram_schmidt_s": gs_s, "run_1000_steps_s": t5,
                             "norm_drift_max_1000_steps": float(np.max(drift)),
                             "norm_drift_per_state": [float("%.3g" % v) for v in drift],
                             "workload": "192^3 h=0.18, 128 smooth states, 64 atoms x 9 projectors r_c=3, "
                                         "ETRS dt=0.01, Cholesky-QR every 50 steps, 1000 steps"}
    del H5, x5, xyz
    torch.cuda.empty_cache()
    out.update(control_extra(chk))
    cm = rsg.Mesh(rsg.CUBE, 64, spacing=0.3)
    # optimal control loop on the control workload's operator (64^3 double
    # well, 200 intervals of 0.05 au, 4 ETRS substeps): from the ground to the
    # first excited state of H_0 (both from the eigensolver), 8 L-BFGS steps
    Hc = rsg.Hamiltonian(cm, torch.complex128)
    Hc.set_potential(potential_double_well(cm.xyz, 0.02, 2.0, 0.5))
    xb = torch.from_numpy(white_noise_states(rng(7), cm.P, 4)).cuda()
    Hc.eigensolve(xb, nwant=2, max_iter=300, degree=16, tol=1e-9)
    phi0, phi1 = xb[:, 0].contiguous(), xb[:, 1].contiguous()
    eps0 = control_field(rng(4), 200, 0.05)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, Jopt, hist, nit, nev = Hc.control_optimize(phi0, phi1, eps0, 0.05, scheme=rsg.ETRS, nsub=4,
                                                  checkpoint_every=50, max_iter=8, gtol=1e-9)
    to = time.perf_counter() - t0
    out["control_optimize_c128"] = {"s": to, "steps": nit, "gradient_evaluations": nev, "J_start": float(hist[0]),
                                    "J_end": Jopt, "s_per_evaluation": to / nev,
                                    "workload": "64^3 h=0.3 double well, 200 intervals dt=0.05, ETRS nsub=4, K=50, "
                                                "ground -> first excited state, L-BFGS 8 steps"}
    del Hc, xb
    # shifted linear solves (H - z) x = b on the headline workload's operator:
    # 8 white-noise right-hand sides, z = -0.5 + 0.1 i, complex64, tol 1e-4
    Hs = rsg.Hamiltonian(mesh, torch.complex64)
    Hs.set_potential(potential_wells(mesh.xyz, *wells))
    Hs.set_projectors(*proj)
    bs = torch.from_numpy(white_noise_states(rng(8), mesh.P, 8, dtype=np.complex64)).cuda()
    xs = torch.zeros_like(bs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sres, sit = Hs.shifted_solve(bs, xs, -0.5 + 0.1j, max_iter=5000, tol=1e-4)
    torch.cuda.synchronize()
    tsv = time.perf_counter() - t0
    if chk is not None:
        chk["shifted_solve_c64"] = {"kind": "shifted", "z": -0.5 + 0.1j,
                                    "b": bs.cpu().numpy().astype(np.complex128),
                                    "x": xs.cpu().numpy().astype(np.complex128)}
    out["shifted_solve_c64"] = {"s": tsv, "iterations": sit, "ms_per_iteration": 1e3 * tsv / max(sit, 1),
                                "max_relative_residual": float(np.max(sres)),
                                "workload": "sphere R=18 h=0.2, wells + projectors, 8 right-hand sides, "
                                            "z = -0.5 + 0.1i, COCG, tol 1e-4"}
    del Hs, bs, xs
    # ground state (Chebyshev-filtered subspace iteration): the four lowest
    # levels of the 1-D lithium model as one particle in 3-D (61^3, h = 0.4,
    # complex128), four buffer states, residuals <= 1e-8
    from workloads import potential_soft_coulomb_li
    lm = rsg.Mesh(rsg.CUBE, 61, spacing=0.4)
    Hl = rsg.Hamiltonian(lm, torch.complex128)
    Hl.set_potential(potential_soft_coulomb_li(lm.xyz))
    x = torch.from_numpy(white_noise_states(rng(6), lm.P, 8)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, res, it = Hl.eigensolve(x, nwant=4, max_iter=300, degree=16, tol=1e-8)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    if chk is not None:
        chk["eigensolve_li_model"] = {"kind": "eigen", "lib_ijk": lm.ijk,
                                      "x": x[:, :4].cpu().numpy().astype(np.complex128),
                                      "ev": np.array([float(v) for v in ev[:4]])}
    out["eigensolve_li_model"] = {
        "s": te, "iterations": it, "h_applications": (it * 16 + it + 1) * 8,
        "levels": [float(v) for v in ev[:4]], "max_residual": float(np.max(res[:4])),
        "paper_table": [-4.721, -4.211, -4.211, -4.086],
        "workload": "61^3 h=0.4 soft-Coulomb Li model, c128, 8 states (4 wanted), degree 16, tol 1e-8"}
    del Hl, x
    # the plain-method workload: 32^3, h = 0.3, oscillator w = 0.5, 4 smooth
    # states, complex128, 100 exponential-midpoint steps of 0.01 au
    from workloads import potential_harmonic, wavepacket_params, wavepacket_states
    m1 = rsg.Mesh(rsg.CUBE, 32, spacing=0.3)
    H1 = rsg.Hamiltonian(m1, torch.complex128)
    H1.set_potential(potential_harmonic(m1.xyz, 0.5))
    x1 = torch.from_numpy(wavepacket_states(m1.xyz, wavepacket_params(rng(1), 4, 1.5))).cuda()
    H1.orthonormalize(x1)
    x1_in = x1.cpu().numpy()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    d1 = H1.propagate(x1, 100, 0.01, scheme=rsg.EXPMID)
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    out["oscillator_32_c128"] = {"ms_per_step": ms1 / 100, "s_100_steps": ms1 * 1e-3,
                                 "value": m1.P * 4 * 4 / (ms1 / 100 * 1e-3) / 1e9, "unit": UNIT,
                                 "norm_drift_max": float(np.max(d1)),
                                 "workload": "32^3 h=0.3 oscillator w=0.5, 4 smooth states, c128, 100 exponential "
                                             "midpoint steps dt=0.01"}
    if chk is not None:
        chk["oscillator_32_c128"] = {"kind": "propagate_ho", "lib_ijk": m1.ijk, "psi": x1_in,
                                     "out": x1.cpu().numpy()}
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    from workloads import potential_wells
    g, wells, proj = build_inputs()
    om = oracle.Mesh(oracle.SPHERE, radius=18.0, h=0.2)
    O = oracle.Hamiltonian(om, potential_wells(om.xyz, *wells))
    O.set_projectors(*proj)
    from workloads import rng, white_noise_states
    psi = white_noise_states(rng(2, 5), om.P, 1)
    for _ in range(args.warmup):
        O.apply(psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.apply(psi)
    dt = time.perf_counter() - t0
    val = om.P * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + " (oracle sample: 1 state, 1 H application per step)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "1 FP64 H application to 1 state on the full mesh per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel", type=int, default=None,
                    help="stencil variant (rsg_ham_set_option \"kernel\": 0 staged, 1 naive, 5 register-blocked, ...)")
    ap.add_argument("--threads", type=int, default=None, help="staged kernels: threads per block")
    ap.add_argument("--rx", type=int, default=None)
    ap.add_argument("--ty", type=int, default=None)
    ap.add_argument("--zseg", type=int, default=None)
    ap.add_argument("--wide-ty", type=int, default=None, help="kernel 7: tile rows (4, 6 or 8)")
    ap.add_argument("--producers", type=int, default=None, help="kernel 7: producer warps (1 to 4)")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the complex128 / plain-kernel / control-gradient side measurements")
    ap.add_argument("--only", default=None, choices=["batch", "adjoint"],
                    help="run one side measurement alone and print it (for profiler captures)")
    ap.add_argument("--batch-no-tune", action="store_true",
                    help="with --only batch: default batch options, no autotuning (profiler captures)")
    ap.add_argument("--adjoint-intervals", type=int, default=2000,
                    help="with --only adjoint: control intervals (2000 is the workload)")
    ap.add_argument("--batch-systems", type=int, default=256,
                    help="with --only batch: the first N systems of the batch (profiler captures)")
    ap.add_argument("--radius", type=float, default=18.0,
                    help="sphere radius (bohr); 18 is the benchmark workload, smaller radii "
                         "are for profiler captures only")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1501_05654_gb300 as rsg
    from workloads import potential_wells, white_noise_states

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rsg.build()
    if args.only == "batch":
        if rank == 0:
            print(json.dumps(batch_extra(None, peaks()[0], steps=args.steps, nsys=args.batch_systems,
                                         tune=not args.batch_no_tune)), flush=True)
        return
    if args.only == "adjoint":
        if rank == 0:
            dt_ = torch.complex64 if args.dtype == "c64" else torch.complex128
            print(json.dumps(control_extra(None, nint=args.adjoint_intervals, dtypes=(dt_,))), flush=True)
        return

    g, wells, proj = build_inputs()
    mesh = rsg.Mesh(rsg.SPHERE, radius=args.radius, spacing=0.2)
    dtype = torch.complex64 if args.dtype == "c64" else torch.complex128
    H = rsg.Hamiltonian(mesh, dtype)
    H.set_potential(potential_wells(mesh.xyz, *wells))
    H.set_projectors(*proj)
    for k in ("kernel", "threads", "rx", "ty", "zseg", "wide_ty", "producers"):
        if getattr(args, k) is not None:
            H.set_option(k, getattr(args, k))
    S = 64
    P = mesh.P
    npdt = np.complex64 if dtype == torch.complex64 else np.complex128
    psi_h = torch.from_numpy(white_noise_states(g, P, S, dtype=npdt)).pin_memory()
    psi = psi_h.to("cuda")
    dt = 0.01
    stream = torch.cuda.current_stream()

    def step(x):
        H.propagate(x, 1, dt, scheme=rsg.ETRS, want_drift=False)

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(psi)
    torch.cuda.synchronize()
    H.kernel_stats()                      # reset counters
    H.profile(True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_id = vis.split(",")[local] if vis else str(local)
    with ClockSampler(smi_id) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step(psi)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    H.profile(False)
    ms = e0.elapsed_time(e1)
    k_ms, k_n, k_bytes, n_launch = H.kernel_stats()
    ms_max = reduce_max(ms, ws, "cuda")
    value = whole_job_value(ms_max, ws, P * S * N_APPLY_PER_STEP, args.steps)

    # end to end through the public API with host buffers: every step copies
    # its input from pinned host memory, runs one ETRS step and copies the
    # result back.  The steps are independent (each propagates the same host
    # input), so they are pipelined over three device buffers and three
    # streams: step k+1's copy in and step k-1's copy out overlap step k's
    # compute, each on its own buffer (with two buffers a copy in would wait
    # for the previous copy out of its buffer, and the step would take the
    # sum of both copies).  The serial form (one stream, no overlap) is
    # reported beside it.
    e2e = None
    if not args.no_e2e:
        nbytes = psi_h.numel() * psi_h.element_size()
        NBUF = 3
        dev = [psi] + [torch.empty_like(psi) for _ in range(NBUF - 1)]
        out_h = [torch.empty_like(psi_h).pin_memory() for _ in range(NBUF)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_steps(n):
            ev_in = [torch.cuda.Event() for _ in range(NBUF)]
            ev_cmp = [torch.cuda.Event() for _ in range(NBUF)]
            ev_out = [torch.cuda.Event() for _ in range(NBUF)]
            used = [False] * NBUF
            for k in range(n):
                b = k % NBUF
                if used[b]:
                    s_in.wait_event(ev_out[b])          # buffer b's previous result is home
                with torch.cuda.stream(s_in):
                    dev[b].copy_(psi_h, non_blocking=True)
                    ev_in[b].record(s_in)
                s_cmp.wait_event(ev_in[b])
                H.propagate(dev[b], 1, dt, scheme=rsg.ETRS, want_drift=False, stream=s_cmp)
                ev_cmp[b].record(s_cmp)
                s_out.wait_event(ev_cmp[b])
                with torch.cuda.stream(s_out):
                    out_h[b].copy_(dev[b], non_blocking=True)
                    ev_out[b].record(s_out)
                used[b] = True

        e2e_steps(2)
        torch.cuda.synchronize()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s_in)
        e2e_steps(args.steps)
        s_out.wait_stream(s_in)
        s_out.wait_stream(s_cmp)
        f1.record(s_out)
        torch.cuda.synchronize()
        barrier()
        te = reduce_max(f0.elapsed_time(f1), ws, "cuda")
        # serial form: one stream, copy in, step, copy out
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            psi.copy_(psi_h, non_blocking=True)
            step(psi)
            out_h[0].copy_(psi, non_blocking=True)
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ts = reduce_max(g0.elapsed_time(g1), ws, "cuda")
        e2e = {"value": whole_job_value(te, ws, P * S * N_APPLY_PER_STEP, args.steps),
               "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "pipelining": "3 device buffers, copy-in / compute / copy-out streams",
               "serial_value": whole_job_value(ts, ws, P * S * N_APPLY_PER_STEP, args.steps)}
        del dev[1:]

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    achieved = (k_bytes / k_n) / (k_ms / k_n * 1e-3) / 1e9 if k_n else None
    per_launch_bytes = k_bytes / k_n if k_n else None
    kname = KERNEL_NAMES.get(H.get_option("last_kernel"), "unknown")
    traffic = traffic_record(kernel_hash(), kname)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if dtype == torch.complex64 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.radius == 18.0 else
                   f"sphere R={args.radius:g} bohr h=0.2 ({P:,} pts), 64 states, 32 wells, 32 atoms x 4 projectors, "
                   "ETRS Taylor-4 dt=0.01 (smaller than the headline workload)",
                   "points": P, "states": S, "state_dtype": args.dtype,
                   "h_applications_per_step": N_APPLY_PER_STEP,
                   "l2": "state blocks (1.56 GB) exceed L2; no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "kernel": f"{kname} (Horner stage: stencil + V, base and result streams)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes_per_launch": per_launch_bytes,
                     "avg_launch_ms": k_ms / k_n if k_n else None,
                     "traffic": traffic},
        "gpu_launches": n_launch,
        "e2e": e2e,
    }
    line["clocks"] = clk.summary()
    # host copies of results that the oracle leg checks against the FP64
    # oracle (only with the oracle leg, on the headline workload)
    chk = None
    if not args.no_cpu_baseline and ws == 1 and args.radius == 18.0 and dtype == torch.complex64:
        chk = collect_headline_checks(H, mesh, psi_h, kname)
    if not args.no_extras and ws == 1:
        line["extras"] = extras(mesh, wells, proj, g, chk)
    if not args.no_cpu_baseline and ws == 1:
        try:
            base, legs, errs = oracle_leg(chk or {}, wells, proj)
            line["cpu_baseline"] = base
            line["cpu_baseline"]["legs"] = legs
            line["error_vs_oracle"] = errs.get("headline")
            for name, e in errs.items():
                if name != "headline" and name in line.get("extras", {}):
                    line["extras"][name]["error_vs_oracle"] = e
        except Exception as ex:     # reported, never fatal
            line["cpu_baseline"] = {"error": repr(ex)}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

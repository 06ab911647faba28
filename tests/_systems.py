"""Builds matched (library, oracle) systems from the seeded workload recipes.

Inputs are generated in the oracle's point order and permuted into the
library's order; nothing here computes any part of the method.
"""
import numpy as np
import torch

import oracle
import paper_1501_05654_gb300 as rsg
from tests._parity import perm_lib_to_oracle
from workloads import (gaussian_wells, potential_double_well, potential_harmonic,
                       potential_wells, projector_atoms, rng)


class Pair:
    def __init__(self, shape, n=0, radius=0.0, h=0.3, dtype=torch.complex64, odd=False):
        self.lm = rsg.Mesh({"cube": rsg.CUBE, "box": rsg.BOX, "sphere": rsg.SPHERE}[shape], n,
                           radius=radius, spacing=h)
        if odd:
            self.lm.set_boundary(rsg.BC_ODD)
        self.om = oracle.Mesh({"cube": oracle.CUBE, "box": oracle.BOX,
                               "sphere": oracle.SPHERE}[shape], n, radius=radius, h=h,
                              bc=oracle.ODD if odd else oracle.ZERO)
        self.idx = perm_lib_to_oracle(self.lm.ijk, self.om.ijk)
        self.P = self.lm.P
        self.h = h
        self.dtype = dtype
        self.H = rsg.Hamiltonian(self.lm, dtype)
        self.O = None

    # oracle-order array -> library-order array
    def to_lib(self, a):
        return np.asarray(a)[self.idx]

    def to_orc(self, a):
        out = np.empty_like(np.asarray(a))
        out[self.idx] = a
        return out

    def set_potential(self, V_orc):
        self.V_orc = np.asarray(V_orc, np.float64)
        V_lib = self.to_lib(self.V_orc)
        if self.dtype == torch.complex64:
            # the FP32 path stores V in float32; feed the oracle the same values
            self.V_orc = self.V_orc.astype(np.float32).astype(np.float64)
        self.O = oracle.Hamiltonian(self.om, self.V_orc)
        self.H.set_potential(V_lib)

    def set_projectors(self, centres, rcut, lmax, beta, hm):
        self.H.set_projectors(centres, rcut, lmax, beta, hm)
        self.O.set_projectors(centres, rcut, lmax, beta, hm)

    def states_to_gpu(self, psi_orc, ld=None):
        """Oracle-order (P, S) complex128 -> library-order cuda block (P, ld)."""
        S = psi_orc.shape[1]
        ld = rsg.padded_ld(S, self.dtype) if ld is None else ld
        t = torch.zeros((self.P, ld), dtype=self.dtype)
        t[:, :S] = torch.from_numpy(self.to_lib(psi_orc).astype(
            np.complex64 if self.dtype == torch.complex64 else np.complex128))
        return t.cuda()

    def states_from_gpu(self, t, S):
        a = t[:, :S].cpu().numpy().astype(np.complex128)
        return self.to_orc(a)


def wells_system(shape="cube", n=0, radius=0.0, h=0.3, dtype=torch.complex64, seed=0,
                 nwells=4, natoms=2, lmax=1, rcut=1.2):
    g = rng(2, seed)
    p = Pair(shape, n, radius, h, dtype)
    ext = np.abs(p.om.xyz).max() if p.P else 1.0
    c, d, w = gaussian_wells(g, nwells, 0.6 * ext)
    p.set_potential(potential_wells(p.om.xyz, c, d, w))
    if natoms:
        cen, rc, lm, beta, hm = projector_atoms(g, natoms, rcut, lmax, ball_radius=0.5 * ext)
        p.set_projectors(cen, rc, lm, beta, hm)
    return p, g


def ho_system(n=32, h=0.3, dtype=torch.complex128, omega=0.5):
    p = Pair("cube", n, h=h, dtype=dtype)
    p.set_potential(potential_harmonic(p.om.xyz, omega))
    return p


def double_well_system(n=16, h=0.5, dtype=torch.complex128):
    p = Pair("cube", n, h=h, dtype=dtype)
    p.set_potential(potential_double_well(p.om.xyz, 0.02, 2.0, 0.5))
    return p

"""Helpers for GPU-vs-oracle parity tests (point matching and error metrics).

The library and the oracle order mesh points differently; every comparison
goes through the permutation built from their lattice coordinates.  Inputs
are generated once, in the oracle's order, by the seeded generators in
``workloads`` and permuted into the library's order.
"""
import numpy as np


def perm_lib_to_oracle(lib_ijk, orc_ijk):
    """idx such that lib point i is oracle point idx[i]."""
    assert lib_ijk.shape == orc_ijk.shape
    a = np.lexsort(lib_ijk.T[::-1])
    b = np.lexsort(orc_ijk.T[::-1])
    assert np.array_equal(lib_ijk[a], orc_ijk[b]), "meshes differ"
    idx = np.empty(len(a), dtype=np.int64)
    idx[a] = b
    return idx


def rel_err(got, want):
    """Normwise-max error per state: max_p |d| / max_p |want|, then max over states."""
    got = np.asarray(got)
    want = np.asarray(want)
    if got.ndim == 1:
        got, want = got[:, None], want[:, None]
    den = np.abs(want).max(axis=0)
    den[den == 0] = 1.0
    return float((np.abs(got - want).max(axis=0) / den).max())


def round_c64(a):
    """complex128 -> complex64 -> complex128 (what the FP32 path is fed)."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)

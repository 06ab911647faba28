"""Real-space-grid Hamiltonian application and Taylor-4 real-time propagation
on GB300 (sm_103a), behind the C ABI of include/rsg.h.

Public API: ``Mesh``, ``Hamiltonian``, ``Batch``, ``ControlObjective`` and
``empty_states`` from :mod:`paper_1501_05654_gb300.rsg`; ``build`` compiles
the CUDA library in-tree.
"""
from .build import build  # noqa: F401
from .rsg import (BC_ODD, BC_ZERO, BOX, C64, C128, CUBE, ETRS, EXPMID, SPHERE, Batch,  # noqa: F401
                  ControlObjective, Hamiltonian, Mesh, RSGError, empty_states, fourier_basis, load,
                  padded_ld)

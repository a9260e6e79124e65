"""GB300-native phase-field lattice Boltzmann solver for N-phase flow.

The solver (arXiv:1904.12553) runs in the CUDA library built from ``csrc/``
and is reached through the C ABI of ``include/lbm_nphase.h``; ``binding``
exposes the same functions to Python, ``workloads`` the seeded inputs.
"""
from .binding import (Batch, LbmError, Solver, lbm_nphase_create, lbm_nphase_derive,  # noqa: F401
                      lbm_nphase_destroy, lbm_nphase_diagnostics,
                      lbm_nphase_init, lbm_nphase_moments, lbm_nphase_step,
                      lbm_nphase_steps_taken, lbm_nphase_workspace_bytes,
                      load_library, make_params, strerror)

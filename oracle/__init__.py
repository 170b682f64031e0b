"""CPU oracle of the exact Gillespie simulation with Gumbel-max choice and its straight-through
gradient (arXiv 2602.19775, Sections 2-3, Eqs. 3-7, Figure 1).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. It shares no code with the CUDA library and never reads anything the
CUDA path produced.

Modules:
* ``native``   -- ctypes front end of ``ssa_oracle.c`` (FP64 simulation + hand adjoint), and the
                  gcc build of that file.
* ``cme``      -- chemical master equation tools (Eq. 1): finite generator matrices, transient
                  laws by matrix exponential and their bin averages, stationary laws, the Poisson law of
                  immigration-death, and exact enumeration of short jump chains.
* ``autodiff`` -- the literal straight-through graph of Eq. 5 in float64 PyTorch CPU autograd,
                  for small cases; it pins the hand adjoint.
* ``quadrature`` -- the expected one-step straight-through gradient for two reactions as a
                  one-dimensional integral over the logistic law of G_1 - G_2.
"""
from .native import (  # noqa: F401
    HOLD,
    LINEAR,
    BIN,
    STATUS,
    build,
    philox_blocks,
    uniforms,
    run,
    OracleResult,
    grn_run,
    GRNResult,
)

"""GB300 (sm_103a) library for exact Gillespie simulation with a Gumbel-max choice and its
Gumbel-Softmax straight-through gradient (arXiv 2602.19775).

The compute path is libssa.so (hand-written CUDA, C ABI in include/ssa.h); `ssa` is the thin
PyTorch front end. Importing this package does not load the library; the first call does, and
fails loudly if it is missing.
"""
from ._lib import SSAError, EXPORTS  # noqa: F401


def __getattr__(name):
    if name in ("Network", "forward", "backward", "simulate", "ensemble_mean", "philox_uniforms", "SSAFunction",
                "ForwardResult", "Run", "make_opts", "workspace_bytes", "Batch"):
        from . import ssa
        return getattr(ssa, name)
    raise AttributeError(name)

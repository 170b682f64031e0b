"""The C-ABI library loads and exports every function that include/ssa.h declares (no GPU needed:
no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ssa_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2602_19775_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_expected_entry_points():
    from paper_2602_19775_gb300._lib import EXPORTS
    assert _declared() == set(EXPORTS)


def test_library_exports_every_declared_symbol(built_lib):
    for name in _declared():
        assert hasattr(built_lib, name), name


def test_binding_declares_signatures_without_gpu():
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    assert lib.ssa_last_error() is not None
    # argument errors are reported without touching a device
    h = ctypes.c_void_p()
    st = lib.ssa_create_network(0, 1, None, None, None, None, 1, None, ctypes.byref(h))
    assert st == -1 and b"n_species" in lib.ssa_last_error()
    assert lib.ssa_forward_workspace_bytes(None, 1, 1, None) == 0


def test_grn_soft_path_rejects_shapes_beyond_shared_memory_without_gpu():
    """The soft GRN kernels keep W2 (n_out x n_hid floats) in shared memory: a 4096-1024 output layer
    (16 MiB) is refused with SSA_ERR_UNSUPPORTED before any device call, and so is a soft call at T = 0."""
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    g = ctypes.c_void_p()
    assert lib.ssa_grn_create(16, 4096, 1024, ctypes.c_float(1.0), ctypes.byref(g)) == 0
    try:
        opts = _lib.FwdOpts(_lib.SSA_READOUT_HOLD, 0, 0, 0, 64, 0, 0, _lib.SSA_SELECT_SOFT, 1.0)
        run = ctypes.c_void_p()
        args = [g] + [None] * 5 + [1, 1, 0, None, 1.0, None, 0, 0, ctypes.byref(opts), None, 0, None, None, None,
                                    None, ctypes.byref(run)]
        assert lib.ssa_grn_forward(*args) == -4
        assert b"shared memory" in lib.ssa_last_error()
        opts.temperature = 0.0  # the soft forward needs T > 0
        assert lib.ssa_grn_forward(*args) == -4
        assert b"T > 0" in lib.ssa_last_error()
    finally:
        lib.ssa_grn_destroy(g)


def _net_args(**over):
    """2A -> B, B -> 2A as host tables, with fields replaced by `over`."""
    a = dict(N=2, M=2, reactants=[0, 0, 1, -1], ptr=[0, 2, 4], sp=[0, 1, 0, 1], dl=[-2, 1, 2, -1], P=2, ri=[0, 1])
    a.update(over)
    arr = lambda v: None if v is None else (ctypes.c_int32 * len(v))(*v)
    return (a["N"], a["M"], arr(a["reactants"]), arr(a["ptr"]), arr(a["sp"]), arr(a["dl"]), a["P"], arr(a["ri"]))


@pytest.mark.parametrize("over, code, text", [
    (dict(N=0), -1, b"n_species"),
    (dict(M=0), -1, b"n_reactions"),
    (dict(M=65536), -4, b"65535"),
    (dict(P=0), -1, b"n_params"),
    (dict(ri=None), -1, b"NULL table"),
    (dict(ptr=[1, 2, 4]), -1, b"stoich_ptr[0]"),
    (dict(ptr=[0, 3, 2]), -1, b"monotone"),
    (dict(sp=None), -1, b"NULL stoichiometry"),
    (dict(reactants=[0, 2, 1, -1]), -1, b"reactant of reaction 0"),
    (dict(reactants=[0, 0, -2, -1]), -1, b"reactant of reaction 1"),
    (dict(ri=[0, 2]), -1, b"rate_index[1]"),
    (dict(sp=[0, 0, 0, 1]), -1, b"twice"),
    (dict(sp=[0, 1, 0, 2]), -1, b"stoich_species[3]"),
    (dict(dl=[-2, 1, 128, -1]), -1, b"stoich_delta[2]"),
])
def test_network_tables_are_validated_on_the_host(over, code, text):
    """ssa_create_network checks every table entry (Section 2's mass-action network: reactant slots,
    the CSR net change, rate indices) before it allocates anything on a device."""
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    h = ctypes.c_void_p(1)
    assert lib.ssa_create_network(*_net_args(**over), ctypes.byref(h)) == code
    assert text in lib.ssa_last_error(), lib.ssa_last_error()
    assert h.value is None  # the handle is cleared on failure


@pytest.mark.parametrize("args, code, text", [
    ((0, 4, 3, 1.0), -1, b"sizes"),
    ((5, 4097, 3, 1.0), -1, b"sizes"),
    ((5, 4, 1025, 1.0), -1, b"sizes"),
    ((1041, 4, 3, 1.0), -4, b"n_in above 1040"),
    ((5, 4, 3, 0.0), -1, b"k_max"),
    ((5, 4, 3, float("nan")), -1, b"k_max"),
])
def test_grn_sizes_are_validated_on_the_host(args, code, text):
    """ssa_grn_create: the layer sizes, the exactness bound of the tensor-core contraction (one 6-bit limb of
    W1 times 8-bit counts summed over n_in stays below 2^24) and k_max > 0."""
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    g = ctypes.c_void_p(1)
    n_in, n_hid, n_out, k_max = args
    assert lib.ssa_grn_create(n_in, n_hid, n_out, ctypes.c_float(k_max), ctypes.byref(g)) == code
    assert text in lib.ssa_last_error(), lib.ssa_last_error()
    assert g.value is None
    assert lib.ssa_grn_create(1040, 4096, 1024, ctypes.c_float(1.0), ctypes.byref(g)) == 0  # the largest accepted
    lib.ssa_grn_destroy(g)


def test_grn_workspace_sizes_on_the_host():
    """ssa_grn_workspace_bytes: a recorded soft run holds float checkpoints of all n_hid + n_out counts every 8
    steps for every trajectory (and the adjoint's scratch); a recorded hard run the 2-byte event log and int
    checkpoints every K steps; an unrecorded run neither. Invalid arguments give 0."""
    from paper_2602_19775_gb300 import _lib
    lib = _lib.lib()
    g = ctypes.c_void_p()
    assert lib.ssa_grn_create(784, 256, 10, ctypes.c_float(1.0), ctypes.byref(g)) == 0
    try:
        n_img, tpi, S, steps = 16, 64, 1, 4096
        n, nd = n_img * tpi, 266
        size = lambda sel, rec, T: lib.ssa_grn_workspace_bytes(
            g, n_img, tpi, S, ctypes.byref(_lib.FwdOpts(_lib.SSA_READOUT_HOLD, rec, 64, 0, steps, 0, 0, sel, T)))
        hard_fwd = size(_lib.SSA_SELECT_GUMBEL, 0, 0.0)
        hard_rec = size(_lib.SSA_SELECT_GUMBEL, 1, 0.0)
        soft_rec = size(_lib.SSA_SELECT_SOFT, 1, 1.0)
        assert 0 < hard_fwd < hard_rec < soft_rec
        assert hard_rec - hard_fwd >= n * (2 * steps + 4 * nd * (steps // 64 + 1))
        assert soft_rec - hard_fwd >= n * 4 * nd * (steps // 8 + 1)
        assert lib.ssa_grn_workspace_bytes(g, -1, tpi, S, ctypes.byref(_lib.FwdOpts(0, 0, 64, 0, steps))) == 0
        assert lib.ssa_grn_workspace_bytes(g, n_img, 0, S, ctypes.byref(_lib.FwdOpts(0, 0, 64, 0, steps))) == 0
        assert lib.ssa_grn_workspace_bytes(g, n_img, tpi, S, ctypes.byref(_lib.FwdOpts(0, 0, 64, 0, 0))) == 0
    finally:
        lib.ssa_grn_destroy(g)


def test_binding_bf16_weights_match_the_generators_rounding():
    """The binding hands the GRN its weights as bf16 (torch's round-to-nearest-even cast); the input
    generators' own bit-level rounding gives the same values, ties included, so the oracle and the GPU
    path see identical weights."""
    import numpy as np
    import torch
    from paper_2602_19775_gb300.ssa import _bf16_bits
    from ssa_workloads.grn import round_bf16
    rng = np.random.default_rng(4)
    w = np.concatenate([rng.normal(0, 0.05, 4096), rng.normal(0, 30.0, 4096)]).astype(np.float32)
    ties = (np.arange(1, 257, dtype=np.uint32) << 16 | 0x8000).view(np.float32)  # exactly half-way
    w = np.concatenate([w, ties, -ties])
    got = _bf16_bits(w).to(torch.float32).numpy()
    np.testing.assert_array_equal(got, round_bf16(w))


def test_start_point_fit_rejects_an_unknown_optimizer_on_the_host():
    import numpy as np
    from paper_2602_19775_gb300.fit import fit_start_point_map
    with pytest.raises(ValueError):
        fit_start_point_map(None, np.zeros(2), [0], np.zeros((1, 2), np.int32), np.zeros((1, 1)), [0], 0.1, 1, 1, 1,
                            0.1, optimizer="momentum")

"""ssa_ensemble_mean_static, the entry point for callers that cannot allocate device memory when
they call (graph capture, allocation-free real-time loops, libraries without the application's
allocator): it must give the same means as ssa_ensemble_mean, which takes a workspace, on
consecutive calls that reuse its fixed scratch array, and reject inputs that do not fit that array.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _mean_with_workspace(L, obs, is_int, stream):
    n, row = obs.shape[0], int(np.prod(obs.shape[1:]))
    need = int(L.ssa_ensemble_mean_workspace_bytes(n, row))
    ws = torch.empty(max(need, 4), dtype=torch.uint8, device="cuda")
    out = torch.empty(row, dtype=torch.float32, device="cuda")
    assert L.ssa_ensemble_mean(_p(obs), is_int, n, row, _p(ws), need, _p(out), stream) == 0
    return out


def _mean_static(L, obs, is_int, stream):
    n, row = obs.shape[0], int(np.prod(obs.shape[1:]))
    out = torch.full((row,), float("nan"), dtype=torch.float32, device="cuda")
    st = L.ssa_ensemble_mean_static(_p(obs), is_int, n, row, _p(out), stream)
    assert st == 0, L.ssa_last_error()
    return out


def test_static_scratch_mean_matches_workspace_mean_on_consecutive_calls():
    from paper_2602_19775_gb300 import _lib
    L = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(123)
    # first call: int32 observables (HOLD readout shape), large enough for many scratch chunks
    a = torch.randint(0, 500, (65536, 50, 2), dtype=torch.int32, device="cuda", generator=g)
    # second call: float observables of another shape, which reuse the same scratch entries
    b = torch.randn((40000, 37, 1), dtype=torch.float32, device="cuda", generator=g) * 100.0
    for obs, is_int in ((a, 1), (b, 0)):
        ref = _mean_with_workspace(L, obs, is_int, stream)
        got = _mean_static(L, obs, is_int, stream)
        torch.cuda.synchronize()
        torch.testing.assert_close(got, ref, rtol=1e-6, atol=1e-6)
        # both follow the same fixed summation order
        assert torch.equal(got, ref)
        # and a plain fp32 PyTorch mean agrees within fp32 rounding
        torch.testing.assert_close(got, obs.double().mean(0).reshape(-1).float(), rtol=1e-5, atol=1e-4)


def test_static_scratch_rejects_inputs_beyond_its_size():
    from paper_2602_19775_gb300 import _lib
    L = _lib.lib()
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    # ceil(n_traj / 256) * row_len = 4097 * 256 > 1,048,576 floats: refused before any launch
    st = L.ssa_ensemble_mean_static(_p(x), 0, 4097 * 256, 256, _p(out), None)
    assert st == -4
    assert b"static scratch" in L.ssa_last_error()

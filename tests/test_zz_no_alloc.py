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


@pytest.mark.parametrize("n_traj,row_len", [
    (1024 * 256, 1024),   # ceil(n_traj/256) * row_len = 1,048,576: the last entry of the scratch array
    (65537 * 256, 1),     # 65,537 chunks: more than gridDim.y can hold, so the chunks are strided
])
def test_static_scratch_boundary_shapes_match_workspace_mean(n_traj, row_len):
    from paper_2602_19775_gb300 import _lib
    L = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(n_traj + row_len)
    obs = torch.rand((n_traj, row_len), dtype=torch.float32, device="cuda", generator=g)
    ref = _mean_with_workspace(L, obs, 0, stream)
    got = _mean_static(L, obs, 0, stream)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    torch.testing.assert_close(got, obs.double().mean(0).float(), rtol=1e-5, atol=1e-5)
    del obs
    torch.cuda.empty_cache()


_FIRST_CALL_IN_CAPTURE = r"""
import ctypes, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2602_19775_gb300 import _lib
L = _lib.lib()
obs = torch.ones((256, 2), dtype=torch.float32, device="cuda")
out = torch.zeros(2, dtype=torch.float32, device="cuda")
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    st = L.ssa_ensemble_mean_static(ctypes.c_void_p(obs.data_ptr()), 0, 256, 2, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream))
print("STATUS", st, L.ssa_last_error().decode())
"""


def test_static_scratch_first_call_during_capture_is_refused():
    """In a fresh process, a first call made while the stream is being captured is refused with
    SSA_ERR_UNSUPPORTED and a message, before any CUDA call that a capture would not allow."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _FIRST_CALL_IN_CAPTURE, root], capture_output=True, text=True,
                         timeout=300)
    line = [ln for ln in res.stdout.splitlines() if ln.startswith("STATUS")]
    assert line, res.stdout + res.stderr
    assert line[0].split()[1] == "-4", line[0]
    assert "before capturing" in line[0]


def test_static_scratch_captured_call_replays_after_a_warm_up_call():
    """Once the address is known on the device, a call captured into a CUDA graph replays correctly."""
    from paper_2602_19775_gb300 import _lib
    L = _lib.lib()
    obs = torch.arange(512 * 3, dtype=torch.float32, device="cuda").reshape(512, 3)
    out = torch.zeros(3, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    # warm-up call outside capture: the address is then cached for this device
    with torch.cuda.stream(s):
        assert L.ssa_ensemble_mean_static(_p(obs), 0, 512, 3, _p(out), ctypes.c_void_p(s.cuda_stream)) == 0
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(graph, stream=s):
        st = L.ssa_ensemble_mean_static(_p(obs), 0, 512, 3, _p(out), ctypes.c_void_p(s.cuda_stream))
    assert st == 0, L.ssa_last_error()
    graph.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(out, obs.double().mean(0).float())

"""Argument checks of the Python binding (CPU).

The C ABI receives bare pointers, so it cannot tell a short or mistyped buffer from a good
one; the binding checks every per-cell buffer (device and host) before the call: a CUDA tensor
on the context's device, contiguous, of the expected dtype, with one element per grid cell.
A stand-in object plays the CUDA tensor here (no GPU needed); nothing reaches the library.
"""
import types

import numpy as np
import pytest
import torch

import paper_2112_10059_gb300 as sph


class FakeCudaTensor:
    def __init__(self, n, dtype, index=0, contiguous=True):
        self.n, self.dtype = n, dtype
        self.device = types.SimpleNamespace(index=index)
        self.is_cuda = True
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous

    def numel(self):
        return self.n

    def data_ptr(self):
        return 4096


def test_device_cells():
    f = sph._cells
    assert f(0, 8, None, torch.float32, "q") is None
    assert f(0, 8, FakeCudaTensor(8, torch.float32), torch.float32, "q").value == 4096
    with pytest.raises(TypeError):
        f(0, 8, FakeCudaTensor(8, torch.float64), torch.float32, "q")
    with pytest.raises(TypeError):
        f(0, 8, FakeCudaTensor(8, torch.bool), torch.uint8, "mask")
    with pytest.raises(ValueError):
        f(0, 8, FakeCudaTensor(7, torch.float32), torch.float32, "q")
    with pytest.raises(ValueError):
        f(0, 8, FakeCudaTensor(8, torch.float32, index=1), torch.float32, "q")
    with pytest.raises(ValueError):
        f(0, 8, FakeCudaTensor(8, torch.float32, contiguous=False), torch.float32, "q")
    with pytest.raises(ValueError):                       # host memory where a device pointer is due
        f(0, 8, torch.zeros(8), torch.float32, "q")
    # no grid yet: the size is left to the library's call-order check
    assert f(0, 0, FakeCudaTensor(5, torch.float32), torch.float32, "q").value == 4096


def test_host_cells():
    h = sph._hcells
    a = np.zeros(8, np.float32)
    assert h(8, a, np.float32, "q").value == a.ctypes.data
    assert h(8, None, np.float32, "q") is None
    with pytest.raises(TypeError):
        h(8, np.zeros(8, np.float64), np.float32, "q")
    with pytest.raises(ValueError):
        h(8, np.zeros(7, np.float32), np.float32, "q")
    with pytest.raises(ValueError):
        h(8, np.zeros(16, np.float32)[::2], np.float32, "q")


def _fake_ctx(calls, ncell=8):
    rec = lambda name: (lambda *a: calls.append((name, a)) or 0)
    lib = types.SimpleNamespace(set_sources=rec("set_sources"), set_targets=rec("set_targets"))
    return types.SimpleNamespace(device=0, ncell=ncell, h=None, lib=lib, _keep=[], _ck=lambda rc: rc)


def test_setters_check_before_the_library_call():
    calls = []
    ctx = _fake_ctx(calls)
    with pytest.raises(TypeError):
        sph.set_sources(ctx, FakeCudaTensor(8, torch.float64), 1.0)
    with pytest.raises(ValueError):
        sph.set_targets(ctx, emag=FakeCudaTensor(9, torch.float32))
    with pytest.raises(TypeError):
        sph.set_targets(ctx, mask=FakeCudaTensor(8, torch.float32))
    assert calls == []
    sph.set_sources(ctx, FakeCudaTensor(8, torch.float32), 1.0)
    sph.set_targets(ctx, mask=FakeCudaTensor(8, torch.uint8))
    assert [c[0] for c in calls] == ["set_sources", "set_targets"]
    assert calls[1][1][1] is None and calls[1][1][2].value == 4096    # no |E|, the mask


def test_batch_problem_checks_each_buffer():
    bp = sph.BatchProblem(2, 2, 2, 0.01, 150.0, FakeCudaTensor(8, torch.float32), 1.0,
                          out=FakeCudaTensor(8, torch.float32))
    assert bp.c_struct().nx == 2
    bp.emag = FakeCudaTensor(4, torch.float32)
    with pytest.raises(ValueError):
        bp.c_struct()

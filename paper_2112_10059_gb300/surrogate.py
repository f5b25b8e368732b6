"""Learned surrogate of the S_ph evaluation: binding of include/sph_nn.h and the trainer.

Argument marshalling only: the network's forward and backward passes, the optimiser,
the input preparation and the judge / fallback run in libsph's CUDA kernels.  BF16
tensors are torch.bfloat16 CUDA tensors; FP32 ones torch.float32.

* :class:`Net` owns one ``sph_nn`` (parameters, Adam state, activations).
* :func:`conv3d`, :func:`conv3d_wgrad`: the single convolution kernels.
* :func:`training_set` / :func:`train`: samples generated by the adaptive FMM
  itself (fine-grid S_ph pooled to the coarse grid, against a coarse FMM estimate),
  then Adam on the BF16 network.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import SphError, _ptr, load

N_PARAMS = None


def _ck(lib, h, rc, what="sph_nn"):
    if rc != 0:
        msg = lib.sph_nn_last_error(h).decode() if h is not None else what
        raise SphError(rc, msg or what)


def num_params():
    return int(load().sph_nn_num_params())


class Net:
    """One network for ``edge``^3 coarse inputs, batches of at most ``max_batch``."""

    def __init__(self, edge=64, max_batch=4, device=0, stream=None, seed=None):
        import torch
        self.lib = load()
        self.device = device
        self.edge = edge
        self.max_batch = max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        rc = self.lib.sph_nn_create(ctypes.byref(h), int(device), ctypes.c_void_p(self.stream.cuda_stream),
                                    int(edge), int(max_batch))
        if rc != 0:
            raise SphError(rc, "sph_nn_create failed")
        self.h = h
        self.P = num_params()
        if seed is not None:
            self.init(seed)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.sph_nn_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        _ck(self.lib, self.h, rc)

    def init(self, seed):
        self._ck(self.lib.sph_nn_init(self.h, ctypes.c_uint64(int(seed))))

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._ck(self.lib.sph_nn_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p), p.size))

    def get_params(self):
        p = np.empty(self.P, np.float32)
        self._ck(self.lib.sph_nn_get_params(self.h, p.ctypes.data_as(ctypes.c_void_p), p.size))
        return p

    def get_grads(self):
        g = np.empty(self.P, np.float32)
        self._ck(self.lib.sph_nn_get_grads(self.h, g.ctypes.data_as(ctypes.c_void_p), g.size))
        return g

    def voxels(self, batch):
        return batch * self.edge ** 3

    def forward(self, x, batch, y=None):
        """x: bfloat16 [batch * edge^3 * 16]; returns y float32 [batch * edge^3 * 2]."""
        import torch
        if y is None:
            y = torch.empty(self.voxels(batch) * 2, dtype=torch.float32, device=x.device)
        self._ck(self.lib.sph_nn_forward(self.h, int(batch), _ptr(x), _ptr(y)))
        return y

    def backward(self, x, t, batch):
        loss = ctypes.c_double()
        self._ck(self.lib.sph_nn_backward(self.h, int(batch), _ptr(x), _ptr(t), ctypes.byref(loss)))
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._ck(self.lib.sph_nn_adam(self.h, lr, beta1, beta2, eps))

    def train_step(self, x, t, batch, lr, want_loss=True):
        loss = ctypes.c_double()
        self._ck(self.lib.sph_nn_train_step(self.h, int(batch), _ptr(x), _ptr(t), lr,
                                            ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def make_inputs(self, I_fine, E_fine, S_coarse, factor, x=None):
        import torch
        if x is None:
            x = torch.empty(self.edge ** 3 * 16, dtype=torch.bfloat16, device=S_coarse.device)
        self._ck(self.lib.sph_nn_make_inputs(self.h, self.edge * factor, int(factor), _ptr(I_fine), _ptr(E_fine),
                                             _ptr(S_coarse), _ptr(x)))
        return x

    def make_target(self, S_fine, S_coarse, factor, t=None):
        import torch
        if t is None:
            t = torch.empty(self.edge ** 3, dtype=torch.float32, device=S_coarse.device)
        self._ck(self.lib.sph_nn_make_target(self.h, self.edge * factor, int(factor), _ptr(S_fine), _ptr(S_coarse),
                                             _ptr(t)))
        return t


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def conv3d(mode, C, N, edge, batch, x, w, bias=None, add=None, mask=None, relu=True, out=None, device=0, stream=None):
    """One convolution kernel (mode 0 forward [nvox][C] -> [nvox][N]; mode 1 data gradient [nvox][N] -> [nvox][C])."""
    import torch
    lib = load()
    nvox = batch * edge ** 3
    if out is None:
        out = torch.empty(nvox * (N if mode == 0 else C), dtype=torch.bfloat16, device=x.device)
    rc = lib.sph_nn_conv3d(int(device), _stream_ptr(stream), int(mode), int(C), int(N), int(edge), int(batch),
                           _ptr(x), _ptr(w), _ptr(bias), _ptr(add), _ptr(mask), 1 if relu else 0, _ptr(out))
    if rc != 0:
        raise SphError(rc, "sph_nn_conv3d failed")
    return out


def conv3d_wgrad(C, N, edge, batch, x, dz, out=None, device=0, stream=None):
    """Weight gradient: float32 [N*27*C + N] (w then b)."""
    import torch
    lib = load()
    if out is None:
        out = torch.empty(N * 27 * C + N, dtype=torch.float32, device=x.device)
    rc = lib.sph_nn_conv3d_wgrad(int(device), _stream_ptr(stream), int(C), int(N), int(edge), int(batch), _ptr(x),
                                 _ptr(dz), _ptr(out))
    if rc != 0:
        raise SphError(rc, "sph_nn_conv3d_wgrad failed")
    return out


def pool_avg(fine, n_fine, factor, out=None, device=0, stream=None):
    import torch
    m = n_fine // factor
    if out is None:
        out = torch.empty(m ** 3, dtype=torch.float32, device=fine.device)
    rc = load().sph_pool_avg(int(device), _stream_ptr(stream), int(n_fine), int(factor), _ptr(fine), _ptr(out))
    if rc != 0:
        raise SphError(rc, "sph_pool_avg failed")
    return out

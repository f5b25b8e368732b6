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

def _ck(lib, h, rc, what="sph_nn"):
    if rc != 0:
        msg = lib.sph_nn_last_error(h).decode() if h is not None else what
        raise SphError(rc, msg or what)


def num_params():
    return int(load().sph_nn_num_params())


# (in channels, out channels, level) of the 12 convolutions, as in include/sph_nn.h
LAYER_SHAPES = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 32, 2), (32, 32, 2), (32, 32, 3),
                (32, 32, 3), (32, 32, 2), (32, 32, 1), (32, 16, 0), (16, 16, 0)]


def forward_flops(edge, batch=1):
    """Multiply-add flops (2 per MAC) of the 12 convolutions of one forward pass."""
    return sum(2 * 27 * ci * co * batch * (edge >> lvl) ** 3 for ci, co, lvl in LAYER_SHAPES)


def train_flops(edge, batch=1):
    """Forward + data gradient (all but the first layer) + weight gradient of the convolutions."""
    first = 2 * 27 * 16 * 16 * batch * edge ** 3
    return 3 * forward_flops(edge, batch) - first


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


class SurrogateStats(ctypes.Structure):
    """Mirror of ``sph_surrogate_stats``."""
    _fields_ = [("n_blocks", ctypes.c_int32), ("n_fallback", ctypes.c_int32), ("n_judged_fail", ctypes.c_int32),
                ("n_predicted_fail", ctypes.c_int32), ("n_judge_targets", ctypes.c_int64),
                ("n_fallback_targets", ctypes.c_int64), ("judged_max_err", ctypes.c_float),
                ("ms_coarse", ctypes.c_float), ("ms_net", ctypes.c_float), ("ms_judge", ctypes.c_float),
                ("ms_fallback", ctypes.c_float), ("ms_total", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def evaluate(ctx, net, factor, tol=1e-3, samples=2, seed=1, use_net=True, out=None):
    """Coarse S_ph (float32 [D^3]) by the surrogate with the FMM as judge and fallback.

    ``ctx`` holds the fine grid, sources and criteria (see ``eval_sph_surrogate``).
    Returns (out, SurrogateStats)."""
    import torch
    lib = load()
    D = net.edge
    if out is None:
        out = torch.empty(D ** 3, dtype=torch.float32, device="cuda:%d" % ctx.device)
    st = SurrogateStats()
    rc = lib.eval_sph_surrogate(ctx.h, net.h, int(factor), float(tol), int(samples), ctypes.c_uint64(int(seed)),
                                1 if use_net else 0, _ptr(out), ctypes.byref(st))
    ctx._ck(rc)
    return out, st


# ---------------------------------------------------------------------------- training
def _configure(ctx, n, box, p_torr, q, em, source_scale, i_frac, leaf_size=64, chi=(0.035, 2.0)):
    """Fine or coarse FMM context: n^3 grid over a ``box`` cube, every cell a target."""
    import sph_inputs as si
    from . import M2L_BF16X3, set_criteria, set_grid, set_sources, set_targets
    set_grid(ctx, n, n, n, box / n, si.pO2_of(p_torr), chi[0], chi[1])
    set_sources(ctx, q, source_scale)
    set_targets(ctx)
    set_criteria(ctx, i_frac, 0.0, 0.0, 1, leaf_size, M2L_BF16X3)


def make_sample(net, geom, n_fine, factor, ctx_fine, ctx_coarse, box=1.5, p_torr=760.0, i_frac=1e-4, x=None,
                t=None):
    """One training pair from the adaptive FMM: input x (BF16 [D^3*16]) and target t = ln(pool(S_fine) / S_coarse).

    S_fine: the FMM on the n_fine^3 grid (every cell a target, sources by i_frac); S_coarse: the
    FMM on the factor^3-pooled source over the coarse grid.  Returns (x, t, S_coarse, S_fine)."""
    import sph_inputs as si
    from . import eval_sph
    q, em = si.fields_torch(n_fine, box, geom, device="cuda:%d" % ctx_fine.device)
    scale = si.scale_of(p_torr)
    _configure(ctx_fine, n_fine, box, p_torr, q, em, scale, i_frac)
    S_f, _ = eval_sph(ctx_fine)
    qc = pool_avg(q, n_fine, factor)
    _configure(ctx_coarse, n_fine // factor, box, p_torr, qc, None, scale, i_frac)
    S_c, _ = eval_sph(ctx_coarse)
    x = net.make_inputs(q, em, S_c, factor, x)
    t = net.make_target(S_f, S_c, factor, t)
    return x, t, S_c, S_f


def training_set(net, count, n_fine, factor, seed=1005, first=0, box=1.5, p_torr=760.0, i_frac=1e-4):
    """``count`` samples of :func:`make_sample` for geometries first..first+count-1 of
    ``sph_inputs.cloud_geometry``; returns (X [count, D^3*16] bf16, T [count, D^3] f32)."""
    import torch
    import sph_inputs as si
    from . import Context
    D = n_fine // factor
    dev = "cuda:%d" % net.device
    X = torch.empty((count, D ** 3 * 16), dtype=torch.bfloat16, device=dev)
    T = torch.empty((count, D ** 3), dtype=torch.float32, device=dev)
    cf, cc = Context(net.device), Context(net.device)
    for k in range(count):
        make_sample(net, si.cloud_geometry(first + k, seed), n_fine, factor, cf, cc, box, p_torr, i_frac,
                    x=X[k], t=T[k])
    torch.cuda.synchronize()
    cf.close()
    cc.close()
    return X, T


def train(net, X, T, epochs=10, batch=4, lr=1e-3, lr_final=1e-4, seed=0, X_val=None, T_val=None, log=None):
    """Adam on (X, T) in shuffled batches (cosine learning-rate decay); returns the history
    [(epoch, mean training loss, validation loss or None)]."""
    import math
    import torch
    count = X.shape[0]
    batch = min(batch, net.max_batch, count)
    steps_per_epoch = count // batch
    total = epochs * steps_per_epoch
    rng = np.random.default_rng(seed)
    xb = torch.empty((batch, X.shape[1]), dtype=X.dtype, device=X.device)
    tb = torch.empty((batch, T.shape[1]), dtype=T.dtype, device=T.device)
    hist = []
    step = 0
    for ep in range(epochs):
        order = rng.permutation(count)
        tot = 0.0
        for s in range(steps_per_epoch):
            idx = torch.from_numpy(order[s * batch:(s + 1) * batch]).to(X.device)
            torch.index_select(X, 0, idx, out=xb)
            torch.index_select(T, 0, idx, out=tb)
            lr_s = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / max(total, 1)))
            tot += net.train_step(xb.reshape(-1), tb.reshape(-1), batch, lr_s)
            step += 1
        val = validation_loss(net, X_val, T_val) if X_val is not None else None
        hist.append((ep, tot / max(steps_per_epoch, 1), val))
        if log:
            log(hist[-1])
    return hist


def validation_loss(net, X, T):
    """Mean loss over (X, T) (forward + loss only; the gradient is discarded)."""
    tot = 0.0
    b = net.max_batch
    n = 0
    for i in range(0, X.shape[0] - b + 1, b):
        tot += net.backward(X[i:i + b].reshape(-1), T[i:i + b].reshape(-1), b) * b
        n += b
    return tot / max(n, 1)

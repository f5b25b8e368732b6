"""Python binding of libsph (C ABI in include/sph.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
kernels of ``libsph.so``.  Device buffers are PyTorch CUDA tensors (torch is
used for device memory and streams); host buffers are numpy arrays.  The
library is loaded on first use and the import fails loudly if it is missing
or was not built: there is no CPU fallback.

The functions keep the C names: :func:`set_grid`, :func:`set_sources`,
:func:`set_targets`, :func:`set_criteria`, :func:`eval_sph`,
:func:`eval_sph_host`, :func:`eval_direct`, plus :class:`Context` and the
introspection calls :func:`get_selection` / :func:`get_tree`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["Context", "set_grid", "set_sources", "set_targets", "set_criteria", "set_far_field", "set_near_field", "set_skip_ratio",
           "eval_sph",
           "eval_sph_host", "eval_direct", "eval_sph_batch", "BatchProblem", "get_selection", "get_tree", "load",
           "SphError", "M2L_F32", "M2L_BF16X3", "Stats"]

M2L_F32 = 0
M2L_BF16X3 = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsph.so")
_lib = None
_lock = threading.Lock()

_STATUS = {0: "SPH_OK", -1: "SPH_EINVAL", -2: "SPH_ENOMEM", -3: "SPH_ECUDA", -4: "SPH_ESTATE",
           -5: "SPH_ECAPACITY", -6: "SPH_ETIMEOUT", -7: "SPH_EINTERNAL"}


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_STATUS.get(code, "?"), code, msg))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_int64), ("n_targets", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("max_level", ctypes.c_int32), ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_u", ctypes.c_int64), ("n_v", ctypes.c_int64), ("n_w", ctypes.c_int64),
                ("n_x", ctypes.c_int64), ("ms_select", ctypes.c_float), ("ms_tree", ctypes.c_float),
                ("ms_upward", ctypes.c_float), ("ms_vpairs", ctypes.c_float), ("ms_m2l", ctypes.c_float),
                ("ms_l2l", ctypes.c_float), ("ms_l2p", ctypes.c_float),
                ("ms_near", ctypes.c_float), ("ms_total", ctypes.c_float), ("n_launches", ctypes.c_int64),
                ("far_method", ctypes.c_int32), ("far_order", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("near_table", ctypes.c_int32), ("n_w_skipped", ctypes.c_int64), ("l2lp_fused", ctypes.c_int32),
                ("ms_l2lp", ctypes.c_float), ("m2l_tiles", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TreeView(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int64), ("n_u", ctypes.c_int64), ("n_v", ctypes.c_int64),
                ("n_w", ctypes.c_int64), ("n_x", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("level", ctypes.c_void_p), ("key", ctypes.c_void_p), ("src_begin", ctypes.c_void_p),
                ("src_end", ctypes.c_void_p), ("trg_begin", ctypes.c_void_p), ("trg_end", ctypes.c_void_p),
                ("parent", ctypes.c_void_p), ("is_leaf", ctypes.c_void_p), ("u_pairs", ctypes.c_void_p),
                ("v_pairs", ctypes.c_void_p), ("w_pairs", ctypes.c_void_p), ("x_pairs", ctypes.c_void_p)]


class Problem(ctypes.Structure):
    """Mirror of ``sph_problem`` (one snapshot of a batch)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h_cm", ctypes.c_double),
                ("pO2_torr", ctypes.c_double), ("chi_min", ctypes.c_double), ("chi_max", ctypes.c_double),
                ("q_dev", ctypes.c_void_p), ("source_scale", ctypes.c_double), ("emag_dev", ctypes.c_void_p),
                ("mask_dev", ctypes.c_void_p), ("i_frac", ctypes.c_double), ("e_frac", ctypes.c_double),
                ("e_applied", ctypes.c_double), ("s_dev", ctypes.c_void_p)]


EXPORTS = ["sph_create", "sph_destroy", "sph_last_error", "set_grid", "set_sources", "set_targets",
           "set_criteria", "sph_set_far_field", "sph_set_near_field", "sph_set_skip_ratio", "eval_sph", "eval_sph_batch", "eval_sph_host", "eval_direct",
           "sph_get_selection", "sph_get_tree", "sph_select_noalloc", "sph_scan_i32", "sph_measure_pipe_peaks",
           "sph_version",
           # learned surrogate (include/sph_nn.h)
           "sph_nn_create", "sph_nn_destroy", "sph_nn_last_error", "sph_nn_num_params", "sph_nn_init",
           "sph_nn_set_params", "sph_nn_get_params", "sph_nn_get_grads", "sph_nn_forward", "sph_nn_backward",
           "sph_nn_adam", "sph_nn_train_step", "sph_nn_make_inputs", "sph_nn_make_target", "sph_pool_avg",
           "sph_nn_conv3d", "sph_nn_conv3d_wgrad", "eval_sph_surrogate"]

FAR_CHEBYSHEV = 0
FAR_SURFACE = 1
NEAR_EXP, NEAR_TABLE, NEAR_AUTO = 0, 1, 2


def load(path: str | None = None):
    """Load libsph.so (built by ``paper_2112_10059_gb300.build``).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError("libsph.so not built at %s: run __graft_entry__.build()" % p)
        lib = ctypes.CDLL(p)
        V, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.sph_create.argtypes = [ctypes.POINTER(V), I, V]
        lib.sph_destroy.argtypes = [V]
        lib.sph_destroy.restype = None
        lib.sph_last_error.argtypes = [V]
        lib.sph_last_error.restype = ctypes.c_char_p
        lib.set_grid.argtypes = [V, I, I, I, V, D, D, D, D]
        lib.set_sources.argtypes = [V, V, D]
        lib.set_targets.argtypes = [V, V, V]
        lib.set_criteria.argtypes = [V, D, D, D, I, I, I]
        lib.sph_set_far_field.argtypes = [V, I, I]
        lib.sph_set_near_field.argtypes = [V, I]
        lib.sph_set_skip_ratio.argtypes = [V, D]
        lib.eval_sph.argtypes = [V, V, V]
        lib.eval_sph_batch.argtypes = [V, I, ctypes.POINTER(Problem), V]
        lib.eval_sph_host.argtypes = [V, V, V, V, V, V]
        lib.eval_direct.argtypes = [V, I, V]
        lib.sph_get_selection.argtypes = [V, V, ctypes.POINTER(I64), V, ctypes.POINTER(I64)]
        lib.sph_get_tree.argtypes = [V, ctypes.POINTER(TreeView)]
        lib.sph_version.restype = ctypes.c_char_p
        lib.sph_select_noalloc.argtypes = [I, V, I, I, I, V, V, V, D, D, D, V, V, V, V, V, V]
        lib.sph_select_noalloc.restype = I
        lib.sph_scan_i32.argtypes = [I, V, I64, V, V, V]
        lib.sph_measure_pipe_peaks.argtypes = [I, V, ctypes.POINTER(ctypes.c_double)]
        lib.sph_scan_i32.restype = I
        PD, PF = ctypes.POINTER(ctypes.c_double), ctypes.c_float
        lib.sph_nn_create.argtypes = [ctypes.POINTER(V), I, V, I, I]
        lib.sph_nn_destroy.argtypes = [V]
        lib.sph_nn_destroy.restype = None
        lib.sph_nn_last_error.argtypes = [V]
        lib.sph_nn_last_error.restype = ctypes.c_char_p
        lib.sph_nn_num_params.restype = I64
        lib.sph_nn_init.argtypes = [V, ctypes.c_uint64]
        lib.sph_nn_set_params.argtypes = [V, V, I64]
        lib.sph_nn_get_params.argtypes = [V, V, I64]
        lib.sph_nn_get_grads.argtypes = [V, V, I64]
        lib.sph_nn_forward.argtypes = [V, I, V, V]
        lib.sph_nn_backward.argtypes = [V, I, V, V, PD]
        lib.sph_nn_adam.argtypes = [V, PF, PF, PF, PF]
        lib.sph_nn_train_step.argtypes = [V, I, V, V, PF, PD]
        lib.sph_nn_make_inputs.argtypes = [V, I, I, V, V, V, V]
        lib.sph_nn_make_target.argtypes = [V, I, I, V, V, V]
        lib.sph_pool_avg.argtypes = [I, V, I, I, V, V]
        lib.sph_nn_conv3d.argtypes = [I, V, I, I, I, I, I, V, V, V, V, V, I, V]
        lib.sph_nn_conv3d_wgrad.argtypes = [I, V, I, I, I, I, V, V, V]
        lib.eval_sph_surrogate.argtypes = [V, V, I, D, I, ctypes.c_uint64, I, V, V]
        for f in ("sph_nn_create", "sph_nn_init", "sph_nn_set_params", "sph_nn_get_params", "sph_nn_get_grads",
                  "sph_nn_forward", "sph_nn_backward", "sph_nn_adam", "sph_nn_train_step", "sph_nn_make_inputs",
                  "sph_nn_make_target", "sph_pool_avg", "sph_nn_conv3d", "sph_nn_conv3d_wgrad", "eval_sph_surrogate"):
            getattr(lib, f).restype = I
        for f in ("sph_create", "set_grid", "set_sources", "set_targets", "set_criteria", "sph_set_far_field",
                  "sph_set_near_field", "sph_set_skip_ratio", "eval_sph",
                  "eval_sph_batch", "eval_sph_host", "eval_direct", "sph_get_selection", "sph_get_tree"):
            getattr(lib, f).restype = I
        _lib = lib
        return lib


def _ptr(t):
    """Device pointer of a CUDA tensor, or None."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return a.ctypes.data_as(ctypes.c_void_p)


def _cells(device, ncell, t, dtype, name):
    """Device pointer of a per-cell CUDA tensor, after the checks the C ABI cannot make from a
    bare pointer: on the context's device, contiguous, of ``dtype``, one element per grid cell.
    With no grid yet (ncell 0) the size is left to the library's own call-order check."""
    if t is None:
        return None
    p = _ptr(t)
    if t.dtype != dtype:
        raise TypeError("%s: expected %s, got %s" % (name, dtype, t.dtype))
    if device is not None and t.device.index is not None and t.device.index != device:
        raise ValueError("%s: tensor on cuda:%d, context on cuda:%d" % (name, t.device.index, device))
    if ncell and t.numel() != ncell:
        raise ValueError("%s: %d elements for a grid of %d cells" % (name, t.numel(), ncell))
    return p


def _hcells(ncell, a, dtype, name):
    """Host pointer of a per-cell numpy array, with the same checks as :func:`_cells`."""
    if a is None:
        return None
    if a.dtype != np.dtype(dtype):
        raise TypeError("%s: expected %s, got %s" % (name, np.dtype(dtype), a.dtype))
    if ncell and a.size != ncell:
        raise ValueError("%s: %d elements for a grid of %d cells" % (name, a.size, ncell))
    return _hptr(a)


class Context:
    """Owns one ``sph_ctx``: device memory, operator cache and the last tree."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.sph_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise SphError(rc, "sph_create failed")
        self.h = h
        self.nx = self.ny = self.nz = 0
        self._keep = []

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.sph_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != 0:
            raise SphError(rc, self.lib.sph_last_error(self.h).decode())
        return rc

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz


def set_grid(ctx: Context, nx, ny, nz, h, pO2, chi_min=0.035, chi_max=2.0, origin=(0.0, 0.0, 0.0)):
    org = (ctypes.c_double * 3)(*origin)
    ctx._ck(ctx.lib.set_grid(ctx.h, int(nx), int(ny), int(nz), ctypes.cast(org, ctypes.c_void_p),
                             float(h), float(pO2), float(chi_min), float(chi_max)))
    ctx.nx, ctx.ny, ctx.nz = int(nx), int(ny), int(nz)


def set_sources(ctx: Context, q, source_scale):
    """q: float32 CUDA tensor of nx*ny*nz cells (kept alive by the context)."""
    import torch
    qp = _cells(ctx.device, ctx.ncell, q, torch.float32, "q")
    ctx._keep = [k for k in ctx._keep if k[0] != "q"] + [("q", q)]
    ctx._ck(ctx.lib.set_sources(ctx.h, qp, float(source_scale)))


def set_targets(ctx: Context, emag=None, mask=None):
    import torch
    ep = _cells(ctx.device, ctx.ncell, emag, torch.float32, "emag")
    mp = _cells(ctx.device, ctx.ncell, mask, torch.uint8, "mask")
    ctx._keep = [k for k in ctx._keep if k[0] not in ("e", "m")] + [("e", emag), ("m", mask)]
    ctx._ck(ctx.lib.set_targets(ctx.h, ep, mp))


def set_criteria(ctx: Context, i_frac=0.0, e_frac=0.0, e_applied=0.0, self_mode=1, leaf_size=64,
                 m2l_precision=M2L_BF16X3):
    ctx._ck(ctx.lib.set_criteria(ctx.h, float(i_frac), float(e_frac), float(e_applied), int(self_mode),
                                 int(leaf_size), int(m2l_precision)))


def set_far_field(ctx: Context, method=FAR_CHEBYSHEV, order=5):
    """Far-field representation: FAR_CHEBYSHEV (order p, p^3 nodes) or FAR_SURFACE (order = points per edge)."""
    ctx._ck(ctx.lib.sph_set_far_field(ctx.h, int(method), int(order)))


def set_near_field(ctx: Context, mode=NEAR_EXP):
    """Near-field form: NEAR_EXP (kernel evaluated per pair), NEAR_TABLE (table of G over the
    integer squared cell offsets), NEAR_AUTO (timed on the first eval of a problem class)."""
    ctx._ck(ctx.lib.sph_set_near_field(ctx.h, int(mode)))


def set_skip_ratio(ctx: Context, r_s=0.0):
    """Strategy 3: skip W boxes whose bounded share of a target's S_ph is below r_s (0 = off)."""
    ctx._ck(ctx.lib.sph_set_skip_ratio(ctx.h, float(r_s)))


def eval_sph(ctx: Context, out=None, stats: bool = False):
    """S_ph on the grid (float32 CUDA tensor, 0 at non-targets).  Returns (out, Stats|None)."""
    import torch
    if out is None:
        out = torch.empty(ctx.ncell, dtype=torch.float32, device="cuda:%d" % ctx.device)
    st = Stats() if stats else None
    op = _cells(ctx.device, ctx.ncell, out, torch.float32, "out")
    ctx._ck(ctx.lib.eval_sph(ctx.h, op, ctypes.byref(st) if st is not None else None))
    return out, st


class BatchProblem:
    """One snapshot for :func:`eval_sph_batch`: grid, gas, CUDA-tensor fields and thresholds."""

    def __init__(self, nx, ny, nz, h, pO2, q, source_scale, emag=None, mask=None, i_frac=0.0, e_frac=0.0,
                 e_applied=0.0, chi_min=0.035, chi_max=2.0, out=None):
        import torch
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.h, self.pO2, self.chi_min, self.chi_max = float(h), float(pO2), float(chi_min), float(chi_max)
        self.q, self.emag, self.mask = q, emag, mask
        self.source_scale = float(source_scale)
        self.i_frac, self.e_frac, self.e_applied = float(i_frac), float(e_frac), float(e_applied)
        if out is None:
            out = torch.empty(self.nx * self.ny * self.nz, dtype=torch.float32, device=q.device)
        self.out = out

    @classmethod
    def from_problem(cls, problem, device="cuda", mask=None):
        """From a ``sph_inputs.Problem`` (fields copied to the device)."""
        import torch
        q = torch.from_numpy(problem.q).to(device)
        emag = None
        m = None
        if mask is not None:
            m = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to(device)
        elif not (problem.targets_all or problem.emag is None):
            emag = torch.from_numpy(problem.emag).to(device)
        return cls(problem.nx, problem.ny, problem.nz, problem.h, problem.pO2_torr, q, problem.source_scale,
                   emag=emag, mask=m, i_frac=problem.i_frac, e_frac=problem.e_frac, e_applied=problem.e_applied,
                   chi_min=problem.chi_min, chi_max=problem.chi_max)

    def c_struct(self):
        import torch
        n = self.nx * self.ny * self.nz
        dev = self.q.device.index if self.q is not None else None
        return Problem(self.nx, self.ny, self.nz, self.h, self.pO2, self.chi_min, self.chi_max,
                       _cells(dev, n, self.q, torch.float32, "q"), self.source_scale,
                       _cells(dev, n, self.emag, torch.float32, "emag"),
                       _cells(dev, n, self.mask, torch.uint8, "mask"), self.i_frac,
                       self.e_frac, self.e_applied, _cells(dev, n, self.out, torch.float32, "out"))


def eval_sph_batch(ctx: Context, problems, stats: bool = False):
    """S_ph for every snapshot of ``problems`` (list of :class:`BatchProblem`) in one call.

    Method options (self term, leaf size -- 0 autotunes --, M2L arithmetic, far field)
    come from ``set_criteria`` / ``set_far_field`` on ``ctx``.  Returns (list of outputs,
    Stats|None); the outputs are each problem's ``out`` tensor.
    """
    arr = (Problem * max(len(problems), 1))(*[p.c_struct() for p in problems])
    st = Stats() if stats else None
    ctx._ck(ctx.lib.eval_sph_batch(ctx.h, len(problems), arr, ctypes.byref(st) if st is not None else None))
    return [p.out for p in problems], st


def eval_sph_host(ctx: Context, q, emag=None, mask=None, out=None, stats: bool = False):
    """Host-buffer evaluation: numpy in, numpy out (copies inside the call)."""
    if out is None:
        out = np.empty(ctx.ncell, np.float32)
    st = Stats() if stats else None
    n = ctx.ncell
    ctx._ck(ctx.lib.eval_sph_host(ctx.h, _hcells(n, q, np.float32, "q"), _hcells(n, emag, np.float32, "emag"),
                                  _hcells(n, mask, np.uint8, "mask"), _hcells(n, out, np.float32, "out"),
                                  ctypes.byref(st) if st is not None else None))
    return out, st


def eval_direct(ctx: Context, fp64=False, out=None):
    """Direct sum over the selected sets; float32 (or float64 with fp64=True) CUDA tensor."""
    import torch
    if out is None:
        out = torch.empty(ctx.ncell, dtype=torch.float64 if fp64 else torch.float32,
                          device="cuda:%d" % ctx.device)
    op = _cells(ctx.device, ctx.ncell, out, torch.float64 if fp64 else torch.float32, "out")
    ctx._ck(ctx.lib.eval_direct(ctx.h, 1 if fp64 else 0, op))
    return out


def get_selection(ctx: Context):
    """(J, T): selected source and target linear indices of the last eval, ascending int32."""
    ns = ctypes.c_int64()
    nt = ctypes.c_int64()
    ctx._ck(ctx.lib.sph_get_selection(ctx.h, None, ctypes.byref(ns), None, ctypes.byref(nt)))
    J = np.empty(ns.value, np.int32)
    T = np.empty(nt.value, np.int32)
    ctx._ck(ctx.lib.sph_get_selection(ctx.h, _hptr(J), ctypes.byref(ns), _hptr(T), ctypes.byref(nt)))
    return J, T


def get_tree(ctx: Context):
    """Octree and lists of the last eval as numpy arrays (pairs sorted (target box, source box))."""
    tv = TreeView()
    ctx._ck(ctx.lib.sph_get_tree(ctx.h, ctypes.byref(tv)))
    nb = tv.n_boxes
    out = dict(depth=tv.depth, level=np.empty(nb, np.int32), key=np.empty(nb, np.uint32),
               src_begin=np.empty(nb, np.int32), src_end=np.empty(nb, np.int32),
               trg_begin=np.empty(nb, np.int32), trg_end=np.empty(nb, np.int32),
               parent=np.empty(nb, np.int32), leaf=np.empty(nb, np.uint8),
               U=np.empty((tv.n_u, 2), np.int32), V=np.empty((tv.n_v, 2), np.int32),
               W=np.empty((tv.n_w, 2), np.int32), X=np.empty((tv.n_x, 2), np.int32))
    if nb == 0:
        out["leaf"] = out["leaf"].astype(bool)
        return out
    tv.level = _hptr(out["level"])
    tv.key = _hptr(out["key"])
    tv.src_begin = _hptr(out["src_begin"])
    tv.src_end = _hptr(out["src_end"])
    tv.trg_begin = _hptr(out["trg_begin"])
    tv.trg_end = _hptr(out["trg_end"])
    tv.parent = _hptr(out["parent"])
    tv.is_leaf = _hptr(out["leaf"])
    tv.u_pairs = _hptr(out["U"])
    tv.v_pairs = _hptr(out["V"])
    tv.w_pairs = _hptr(out["W"])
    tv.x_pairs = _hptr(out["X"])
    ctx._ck(ctx.lib.sph_get_tree(ctx.h, ctypes.byref(tv)))
    out["leaf"] = out["leaf"].astype(bool)
    return out


def scan_i32(x):
    """Exclusive prefix sum of a CUDA int32 tensor through the library's device scan:
    (out, total) with out[i] = sum of x[:i] (int32 wrap-around) and total = sum of x."""
    import torch
    lib = load()
    if x.dtype != torch.int32:
        raise ValueError("expected an int32 tensor")
    out = torch.empty_like(x)
    total = torch.empty(1, dtype=torch.int32, device=x.device)
    st = torch.cuda.current_stream(x.device)
    rc = lib.sph_scan_i32(int(x.device.index or 0), ctypes.c_void_p(st.cuda_stream), x.numel(), _ptr(x),
                          _ptr(out), _ptr(total))
    if rc != 0:
        raise SphError(rc, "sph_scan_i32 failed")
    return out, int(total.item())


def pipe_peaks(device=0, stream=None):
    """Measured FP32 FMA and MUFU throughput of the device: dict with ffma_flops (flop/s),
    ex2_per_s, rsqrt_per_s (results/s) and n_sm.  Synchronises the stream."""
    lib = load()
    out = (ctypes.c_double * 4)()
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = lib.sph_measure_pipe_peaks(int(device), sp, out)
    if rc != 0:
        raise SphError(rc, "sph_measure_pipe_peaks failed")
    return {"ffma_flops": out[0], "ex2_per_s": out[1], "rsqrt_per_s": out[2], "n_sm": int(out[3])}


def solve(problem, ctx: Context | None = None, m2l_precision=M2L_BF16X3, leaf_size=None, stats=False,
          mask=None):
    """Convenience: evaluate S_ph for a ``sph_inputs.Problem`` (inputs copied to the GPU)."""
    import torch
    ctx = ctx or Context(0)
    set_grid(ctx, problem.nx, problem.ny, problem.nz, problem.h, problem.pO2_torr,
             problem.chi_min, problem.chi_max, problem.origin)
    dev = "cuda:%d" % ctx.device
    q = torch.from_numpy(problem.q).to(dev)
    set_sources(ctx, q, problem.source_scale)
    if mask is not None:
        set_targets(ctx, mask=torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to(dev))
    elif problem.targets_all or problem.emag is None:
        set_targets(ctx)
    else:
        set_targets(ctx, emag=torch.from_numpy(problem.emag).to(dev))
    set_criteria(ctx, problem.i_frac, problem.e_frac, problem.e_applied, 1,
                 problem.leaf_size if leaf_size is None else leaf_size, m2l_precision)
    out, st = eval_sph(ctx, stats=stats)
    return ctx, out, st

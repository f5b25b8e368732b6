"""FP64 CPU oracle of the learned surrogate's network (TEST INFRASTRUCTURE ONLY).

Plain numpy, float64, written from the definitions; it shares nothing with the CUDA
path.  Used by the tests to check the GPU BF16 kernels (forward, data gradient, weight
gradient, pooling, up-sampling, head and loss, Adam) and the whole network's gradient.

Definitions (the surrogate has no counterpart in the paper; it follows the
learned-surrogate design stated for this project: a 4-level U-Net-like BF16
convolutional network on a coarse grid whose output corrects a coarse
evaluation of Eq. summation, judged by the FMM):

* tensors are channels-last ``[B, D, D, D, C]`` with axes (batch, z, y, x, channel);
* a 3x3x3 "same" convolution with zero padding:
  ``y[b,z,y,x,n] = bias[n] + sum_t sum_c w[n,t,c] x[b,z+dz,y+dy,x+dx,c]``,
  tap ``t = 9 (dz+1) + 3 (dy+1) + (dx+1)``, ``dz, dy, dx in {-1, 0, 1}``;
* ``pool``: mean over 2x2x2 children; ``up``: nearest-neighbour copy to 2x2x2 children;
* the network (``LAYERS``; every convolution followed by ReLU):

    a00 = c00(x)          s0 = c01(a00)          p0 = pool(s0)
    a10 = c10(p0)         s1 = c11(a10)          p1 = pool(s1)
    a20 = c20(p1)         s2 = c21(a20)          p2 = pool(s2)
    a30 = c30(p2)         b3 = c31(a30)
    u2 = up(b3) + s2      d2 = c22(u2)
    u1 = up(d2) + s1      d1 = c12(u1)
    u0 = up(d1)           d0 = c02(u0)           v0 = d0 + s0
    f = c03(v0)           [r, e] = Wh f + bh      (1x1x1 head, no ReLU)

* loss over the M voxels with target t (log ratio of the fine-grid truth to the coarse
  evaluation): ``L = mean((r - t)^2) + LAMBDA * mean((e - log(|r - t| + EPS))^2)`` with
  the inner ``|r - t|`` held constant (e learns the log of r's error);
* Adam with bias correction.

Parity status: pinned by ``tests/test_nn_oracle.py`` (finite differences of every
backward, adjoint identities, shift and averaging special cases, Adam's first step).
"""
from __future__ import annotations

import numpy as np

LAMBDA = 0.01
EPS = 1e-4

# (name, in channels, out channels, level)
LAYERS = [("c00", 16, 16, 0), ("c01", 16, 16, 0), ("c10", 16, 32, 1), ("c11", 32, 32, 1),
          ("c20", 32, 32, 2), ("c21", 32, 32, 2), ("c30", 32, 32, 3), ("c31", 32, 32, 3),
          ("c22", 32, 32, 2), ("c12", 32, 32, 1), ("c02", 32, 16, 0), ("c03", 16, 16, 0)]
HEAD_IN, HEAD_OUT = 16, 2
IN_CH = 16


def taps():
    """(dz, dy, dx) of tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)."""
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def _shift(x, dz, dy, dx):
    """s[b,z,y,x] = x[b,z+dz,y+dy,x+dx], zero outside."""
    out = np.zeros_like(x)
    D = x.shape[1]
    zs = slice(max(0, -dz), D - max(0, dz))
    ys = slice(max(0, -dy), D - max(0, dy))
    xs = slice(max(0, -dx), D - max(0, dx))
    zt = slice(max(0, dz), D - max(0, -dz))
    yt = slice(max(0, dy), D - max(0, -dy))
    xt = slice(max(0, dx), D - max(0, -dx))
    out[:, zs, ys, xs] = x[:, zt, yt, xt]
    return out


def conv3d(x, w, b=None):
    """3x3x3 same convolution: x [B,D,D,D,C], w [N,27,C], b [N] -> [B,D,D,D,N]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(taps()):
        y += _shift(x, dz, dy, dx) @ w[:, t, :].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_dgrad(dy, w):
    """Gradient of sum(dy * conv3d(x, w)) with respect to x."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    dx = np.zeros(dy.shape[:4] + (w.shape[2],))
    for t, (dz, ddy, ddx) in enumerate(taps()):
        # y[p] uses x[p + o]; so x[q] receives dy[q - o]
        dx += _shift(dy, -dz, -ddy, -ddx) @ w[:, t, :]
    return dx


def conv3d_wgrad(x, dy):
    """Gradients of sum(dy * conv3d(x, w, b)) with respect to w [N,27,C] and b [N]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    C, N = x.shape[-1], dy.shape[-1]
    dw = np.zeros((N, 27, C))
    for t, (dz, ddy, ddx) in enumerate(taps()):
        xs = _shift(x, dz, ddy, ddx).reshape(-1, C)
        dw[:, t, :] = dy.reshape(-1, N).T @ xs
    return dw, dy.reshape(-1, N).sum(0)


def pool(x):
    B, D = x.shape[0], x.shape[1]
    C = x.shape[-1]
    return np.asarray(x, np.float64).reshape(B, D // 2, 2, D // 2, 2, D // 2, 2, C).mean(axis=(2, 4, 6))


def pool_back(g):
    """Adjoint of pool: every child receives 1/8 of its parent's gradient."""
    return up(g) / 8.0


def up(x):
    x = np.asarray(x, np.float64)
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def up_back(g):
    """Adjoint of up: the sum over the 8 children."""
    B, D = g.shape[0], g.shape[1]
    C = g.shape[-1]
    return np.asarray(g, np.float64).reshape(B, D // 2, 2, D // 2, 2, D // 2, 2, C).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def init_params(seed=0, scale=1.0):
    """He-normal weights, zero biases (numpy's generator; tests only)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _ in LAYERS:
        P[name + ".w"] = rng.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci)) * scale
        P[name + ".b"] = rng.standard_normal(co) * 0.01 * scale
    P["head.w"] = rng.standard_normal((HEAD_OUT, HEAD_IN)) * np.sqrt(1.0 / HEAD_IN) * scale
    P["head.b"] = np.zeros(HEAD_OUT)
    return P


def forward(P, x):
    """Network forward; returns (y [B,D,D,D,2], cache of every intermediate)."""
    A = {"x": np.asarray(x, np.float64)}

    def c(name, inp):
        return relu(conv3d(inp, P[name + ".w"], P[name + ".b"]))

    A["a00"] = c("c00", A["x"])
    A["s0"] = c("c01", A["a00"])
    A["p0"] = pool(A["s0"])
    A["a10"] = c("c10", A["p0"])
    A["s1"] = c("c11", A["a10"])
    A["p1"] = pool(A["s1"])
    A["a20"] = c("c20", A["p1"])
    A["s2"] = c("c21", A["a20"])
    A["p2"] = pool(A["s2"])
    A["a30"] = c("c30", A["p2"])
    A["b3"] = c("c31", A["a30"])
    A["u2"] = up(A["b3"]) + A["s2"]
    A["d2"] = c("c22", A["u2"])
    A["u1"] = up(A["d2"]) + A["s1"]
    A["d1"] = c("c12", A["u1"])
    A["u0"] = up(A["d1"])
    A["d0"] = c("c02", A["u0"])
    A["v0"] = A["d0"] + A["s0"]
    A["f"] = c("c03", A["v0"])
    y = A["f"] @ P["head.w"].T + P["head.b"]
    return y, A


def loss(y, t):
    """Loss and its gradient with respect to y (inner |r - t| held constant)."""
    r, e = y[..., 0], y[..., 1]
    M = r.size
    d = r - t
    le = np.log(np.abs(d) + EPS)
    L = np.mean(d * d) + LAMBDA * np.mean((e - le) ** 2)
    gy = np.zeros_like(y)
    gy[..., 0] = 2.0 * d / M
    gy[..., 1] = 2.0 * LAMBDA * (e - le) / M
    return L, gy


def backward(P, A, gy):
    """Gradients of every parameter given dL/dy."""
    G = {}
    f = A["f"]
    G["head.w"] = gy.reshape(-1, HEAD_OUT).T @ f.reshape(-1, HEAD_IN)
    G["head.b"] = gy.reshape(-1, HEAD_OUT).sum(0)
    g = (gy @ P["head.w"]) * (f > 0)                 # dL/d(pre-activation of c03)

    def layer(name, inp, gz):
        G[name + ".w"], G[name + ".b"] = conv3d_wgrad(inp, gz)
        return conv3d_dgrad(gz, P[name + ".w"])

    g_v0 = layer("c03", A["v0"], g)
    g_u0 = layer("c02", A["u0"], g_v0 * (A["d0"] > 0))
    g_u1 = layer("c12", A["u1"], up_back(g_u0) * (A["d1"] > 0))
    g_u2 = layer("c22", A["u2"], up_back(g_u1) * (A["d2"] > 0))
    g_a30 = layer("c31", A["a30"], up_back(g_u2) * (A["b3"] > 0))
    g_p2 = layer("c30", A["p2"], g_a30 * (A["a30"] > 0))
    g_a20 = layer("c21", A["a20"], (g_u2 + pool_back(g_p2)) * (A["s2"] > 0))
    g_p1 = layer("c20", A["p1"], g_a20 * (A["a20"] > 0))
    g_a10 = layer("c11", A["a10"], (g_u1 + pool_back(g_p1)) * (A["s1"] > 0))
    g_p0 = layer("c10", A["p0"], g_a10 * (A["a10"] > 0))
    g_a00 = layer("c01", A["a00"], (g_v0 + pool_back(g_p0)) * (A["s0"] > 0))
    layer("c00", A["x"], g_a00 * (A["a00"] > 0))
    return G


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1); returns the new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def flatten(P):
    """Parameters in the library's flat order: per layer w [N][27][C] then b [N]; head w, b."""
    parts = []
    for name, _, _, _ in LAYERS:
        parts += [P[name + ".w"].ravel(), P[name + ".b"].ravel()]
    parts += [P["head.w"].ravel(), P["head.b"].ravel()]
    return np.concatenate(parts)


def unflatten(flat):
    P = {}
    o = 0
    for name, ci, co, _ in LAYERS:
        P[name + ".w"] = flat[o:o + co * 27 * ci].reshape(co, 27, ci)
        o += co * 27 * ci
        P[name + ".b"] = flat[o:o + co]
        o += co
    P["head.w"] = flat[o:o + HEAD_OUT * HEAD_IN].reshape(HEAD_OUT, HEAD_IN)
    o += HEAD_OUT * HEAD_IN
    P["head.b"] = flat[o:o + HEAD_OUT]
    o += HEAD_OUT
    assert o == flat.size
    return P


def n_params():
    return sum(co * 27 * ci + co for _, ci, co, _ in LAYERS) + HEAD_OUT * HEAD_IN + HEAD_OUT


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)

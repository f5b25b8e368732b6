"""GPU checks of the surrogate network's BF16 kernels against the FP64 oracle (oracle/nn_oracle.py).

Inputs are BF16-representable, so the oracle sees exactly what the kernels see; the
kernels accumulate in FP32 and round BF16 outputs once (relative 2^-9), FP32 outputs
(weight gradients) are compared at FP32-accumulation accuracy.
"""
import numpy as np
import pytest

from oracle import nn_oracle as nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sur():
    import __graft_entry__ as g
    g.build()
    from paper_2112_10059_gb300 import surrogate as s
    return s


def _bf(a):
    return nn.bf16_round(a)


def _to_dev_bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda().to(torch.bfloat16)


def _to_dev_f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()


def _host(t):
    import torch
    return t.float().cpu().numpy().astype(np.float64) if t.dtype == torch.bfloat16 else t.cpu().numpy().astype(np.float64)


def _close_bf16(got, ref, label):
    scale = np.max(np.abs(ref)) + 1e-30
    err = np.abs(got - ref)
    bad = err > 2.0 ** -8 * np.abs(ref) + 2e-5 * scale
    assert not bad.any(), "%s: %d bad, worst %.3e (scale %.3e)" % (label, bad.sum(), err.max(), scale)


SHAPES = [(16, 16), (16, 32), (32, 16), (32, 32)]


@pytest.mark.parametrize("C,N", SHAPES)
@pytest.mark.parametrize("edge,batch", [(4, 1), (8, 2), (16, 1)])
def test_conv_forward(sur, C, N, edge, batch):
    rng = np.random.default_rng(100 + C + N + edge)
    x = _bf(rng.standard_normal((batch, edge, edge, edge, C)))
    w = _bf(rng.standard_normal((N, 27, C)) * 0.2)
    b = rng.standard_normal(N).astype(np.float32).astype(np.float64)
    out = sur.conv3d(0, C, N, edge, batch, _to_dev_bf16(x), _to_dev_f32(w), bias=_to_dev_f32(b), relu=True)
    ref = nn.relu(nn.conv3d(x, w, b))
    _close_bf16(_host(out).reshape(ref.shape), ref, "fwd C%d N%d e%d" % (C, N, edge))


@pytest.mark.parametrize("C,N", SHAPES)
def test_conv_forward_add_and_mask(sur, C, N):
    rng = np.random.default_rng(7 + C * N)
    edge, batch = 8, 1
    x = _bf(rng.standard_normal((batch, edge, edge, edge, C)))
    w = _bf(rng.standard_normal((N, 27, C)) * 0.2)
    add = _bf(rng.standard_normal((batch, edge, edge, edge, N)))
    mask = _bf(rng.standard_normal((batch, edge, edge, edge, N)))
    out = sur.conv3d(0, C, N, edge, batch, _to_dev_bf16(x), _to_dev_f32(w), add=_to_dev_bf16(add),
                     mask=_to_dev_bf16(mask), relu=False)
    ref = (nn.conv3d(x, w) + add) * (mask > 0)
    got = _host(out).reshape(ref.shape)
    # the addition is done in FP32 before the single rounding
    _close_bf16(got, ref, "fwd+add+mask")
    assert np.all(got[mask <= 0] == 0)


@pytest.mark.parametrize("C,N", SHAPES)
@pytest.mark.parametrize("edge,batch", [(4, 2), (8, 1), (16, 2)])
def test_conv_data_gradient(sur, C, N, edge, batch):
    rng = np.random.default_rng(200 + C + 3 * N + edge)
    g = _bf(rng.standard_normal((batch, edge, edge, edge, N)))
    w = _bf(rng.standard_normal((N, 27, C)) * 0.2)
    mask = _bf(rng.standard_normal((batch, edge, edge, edge, C)))
    out = sur.conv3d(1, C, N, edge, batch, _to_dev_bf16(g), _to_dev_f32(w), mask=_to_dev_bf16(mask))
    ref = nn.conv3d_dgrad(g, w) * (mask > 0)
    _close_bf16(_host(out).reshape(ref.shape), ref, "dgrad C%d N%d e%d" % (C, N, edge))


@pytest.mark.parametrize("C,N", SHAPES)
@pytest.mark.parametrize("edge,batch", [(4, 1), (8, 3), (32, 1)])
def test_conv_weight_gradient(sur, C, N, edge, batch):
    rng = np.random.default_rng(300 + C + 5 * N + edge)
    x = _bf(rng.standard_normal((batch, edge, edge, edge, C)))
    dz = _bf(rng.standard_normal((batch, edge, edge, edge, N)))
    out = _host(sur.conv3d_wgrad(C, N, edge, batch, _to_dev_bf16(x), _to_dev_bf16(dz)))
    dw, db = nn.conv3d_wgrad(x, dz)
    ref = np.concatenate([dw.ravel(), db])
    scale = np.sqrt(batch * edge ** 3)      # size of a sum of products of unit normals
    assert np.max(np.abs(out - ref)) <= 1e-5 * scale * 4, "wgrad C%d N%d e%d: %.3e" % (
        C, N, edge, np.max(np.abs(out - ref)))


def _net_inputs(edge, batch, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((batch, edge, edge, edge, nn.IN_CH))
    x[..., :3] = rng.random((batch, edge, edge, edge, 3))
    return _bf(x), rng.standard_normal((batch, edge, edge, edge)) * 0.05


def test_network_forward_and_gradient(sur):
    import torch
    edge, batch = 16, 2
    P = nn.init_params(seed=5)
    flat = nn.flatten(P)
    net = sur.Net(edge=edge, max_batch=batch)
    net.set_params(flat.astype(np.float32))
    # the device keeps FP32 master weights and BF16 images: compare with BF16 weights in the oracle
    Pb = nn.unflatten(flat.astype(np.float32).astype(np.float64))
    for name, _, _, _ in nn.LAYERS:
        Pb[name + ".w"] = _bf(Pb[name + ".w"])
    x, t = _net_inputs(edge, batch, 9)
    xd = _to_dev_bf16(x)
    td = _to_dev_f32(t)
    y = _host(net.forward(xd, batch)).reshape(batch, edge, edge, edge, 2)
    yr, A = nn.forward(Pb, x)
    e = np.linalg.norm(y - yr) / np.linalg.norm(yr)
    assert e < 2e-2, "forward rel-L2 %.3e" % e
    loss = net.backward(xd, td, batch)
    Lr, gy = nn.loss(yr, t)
    assert abs(loss - Lr) <= 2e-2 * Lr
    G = nn.backward(Pb, A, gy)
    g = nn.unflatten(net.get_grads().astype(np.float64))
    for k in G:
        d = np.linalg.norm(g[k] - G[k]) / max(np.linalg.norm(G[k]), 1e-30)
        assert d < 6e-2, "%s gradient rel-L2 %.3e" % (k, d)
    torch.cuda.synchronize()


def test_adam_step_matches_oracle(sur):
    edge, batch = 8, 1
    P = nn.init_params(seed=6)
    flat = nn.flatten(P).astype(np.float32)
    net = sur.Net(edge=edge, max_batch=batch)
    net.set_params(flat)
    x, t = _net_inputs(edge, batch, 10)
    xd, td = _to_dev_bf16(x), _to_dev_f32(t)
    p = flat.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in (1, 2, 3):
        net.backward(xd, td, batch)
        g = net.get_grads().astype(np.float64)
        net.adam(1e-3)
        p, m, v = nn.adam(p, g, m, v, step, 1e-3)
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - p)) <= 1e-6 * step, step


def test_training_reduces_loss(sur):
    edge, batch = 16, 4
    net = sur.Net(edge=edge, max_batch=batch, seed=1)
    x, _ = _net_inputs(edge, batch, 11)
    # a learnable target: a smooth function of the input channels
    t = 0.3 * x[..., 0] - 0.2 * x[..., 1] * x[..., 2]
    xd, td = _to_dev_bf16(x), _to_dev_f32(t)
    first = net.backward(xd, td, batch)
    for _ in range(60):
        last = net.train_step(xd, td, batch, 2e-3)
    assert last < 0.5 * first, (first, last)


def test_training_is_reproducible(sur):
    """The weight and head gradients are summed in a fixed order (per-CTA partials, then an
    ordered sum), so two trainings from the same initial weights on the same data end with the
    same weights, bit for bit; at 64^3 the weight gradient spans many voxel splits per layer."""
    edge, batch = 64, 2
    x, _ = _net_inputs(edge, batch, 12)
    t = 0.3 * x[..., 0] - 0.2 * x[..., 1] * x[..., 2]
    xd, td = _to_dev_bf16(x), _to_dev_f32(t)
    finals = []
    for _ in range(2):
        net = sur.Net(edge=edge, max_batch=batch, seed=3)
        for _ in range(12):
            net.train_step(xd, td, batch, 1e-3, want_loss=False)
        finals.append(net.get_params())
        g = net.get_grads()
        net.close()
    assert np.array_equal(finals[0], finals[1])
    assert np.any(g != 0)


def test_bad_arguments(sur):
    import torch
    with pytest.raises(Exception):
        sur.Net(edge=12)          # not a power of two
    net = sur.Net(edge=8, max_batch=1)
    with pytest.raises(Exception):
        net.set_params(np.zeros(3, np.float32))
    x = torch.zeros(2 * 8 ** 3 * 16, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(Exception):
        net.forward(x, 2)         # above max_batch

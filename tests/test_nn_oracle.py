"""CPU pins of the surrogate network's FP64 oracle (oracle/nn_oracle.py).

The convolution is checked against a brute-force loop and a shifted identity, each
backward against central finite differences and adjoint identities, pooling and
up-sampling against their definitions, Adam against its closed-form first step.
"""
import numpy as np
import pytest

from oracle import nn_oracle as nn


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_brute_force_loop():
    B, D, C, N = 1, 4, 3, 2
    x = _rand((B, D, D, D, C), 1)
    w = _rand((N, 27, C), 2)
    b = _rand(N, 3)
    y = nn.conv3d(x, w, b)
    ref = np.zeros((B, D, D, D, N))
    for z in range(D):
        for yy in range(D):
            for xx in range(D):
                for n in range(N):
                    s = b[n]
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                t = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
                                zz, y2, x2 = z + dz, yy + dy, xx + dx
                                if 0 <= zz < D and 0 <= y2 < D and 0 <= x2 < D:
                                    s += np.dot(w[n, t], x[0, zz, y2, x2])
                    ref[0, z, yy, xx, n] = s
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_conv_single_tap_is_a_shift():
    x = _rand((2, 5, 5, 5, 1), 4)
    w = np.zeros((1, 27, 1))
    t = 9 * 2 + 3 * 1 + 0          # dz = +1, dy = 0, dx = -1
    w[0, t, 0] = 1.0
    y = nn.conv3d(x, w)[..., 0]
    ref = np.zeros_like(y)
    ref[:, :-1, :, 1:] = x[:, 1:, :, :-1, 0]
    assert np.array_equal(y, ref)


def test_dgrad_is_the_adjoint():
    x = _rand((2, 6, 6, 6, 4), 5)
    w = _rand((3, 27, 4), 6)
    g = _rand((2, 6, 6, 6, 3), 7)
    lhs = np.sum(nn.conv3d(x, w) * g)
    rhs = np.sum(x * nn.conv3d_dgrad(g, w))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_wgrad_finite_differences_and_linearity():
    x = _rand((1, 4, 4, 4, 3), 8)
    w = _rand((2, 27, 3), 9)
    b = _rand(2, 10)
    g = _rand((1, 4, 4, 4, 2), 11)
    dw, db = nn.conv3d_wgrad(x, g)
    assert abs(np.sum(nn.conv3d(x, w) * g) - np.sum(w * dw)) <= 1e-11 * np.abs(np.sum(w * dw))
    f = lambda W, B_: np.sum(nn.conv3d(x, W, B_) * g)
    h = 1e-6
    for (n, t, c) in [(0, 0, 0), (1, 13, 2), (0, 26, 1), (1, 4, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[n, t, c] += h
        wm[n, t, c] -= h
        assert abs((f(wp, b) - f(wm, b)) / (2 * h) - dw[n, t, c]) <= 1e-6 * max(1.0, abs(dw[n, t, c]))
    bp = b.copy()
    bp[1] += h
    assert abs((f(w, bp) - f(w, b)) / h - db[1]) <= 1e-5


def test_pool_and_up_definitions_and_adjoints():
    x = _rand((1, 4, 4, 4, 2), 12)
    p = nn.pool(x)
    assert np.isclose(p[0, 1, 0, 1, 1], x[0, 2:4, 0:2, 2:4, 1].mean())
    assert np.array_equal(nn.pool(np.full((1, 4, 4, 4, 1), 3.0)), np.full((1, 2, 2, 2, 1), 3.0))
    u = nn.up(p)
    assert np.array_equal(u[0, 3, 1, 2], p[0, 1, 0, 1])
    g = _rand((1, 2, 2, 2, 2), 13)
    assert np.isclose(np.sum(nn.pool(x) * g), np.sum(x * nn.pool_back(g)))
    g4 = _rand((1, 4, 4, 4, 2), 14)
    assert np.isclose(np.sum(nn.up(p) * g4), np.sum(p * nn.up_back(g4)))


def test_network_gradient_finite_differences():
    P = nn.init_params(seed=3)
    x = _rand((1, 8, 8, 8, nn.IN_CH), 15) * 0.5
    t = _rand((1, 8, 8, 8), 16) * 0.1
    y, A = nn.forward(P, x)
    L, gy = nn.loss(y, t)
    G = nn.backward(P, A, gy)
    rng = np.random.default_rng(17)
    h = 1e-6

    def L_of(Pm):
        # the inner |r - t| of the error-head term is held constant: use the unperturbed one
        yy, _ = nn.forward(Pm, x)
        r, e = yy[..., 0], yy[..., 1]
        le = np.log(np.abs(y[..., 0] - t) + nn.EPS)
        return np.mean((r - t) ** 2) + nn.LAMBDA * np.mean((e - le) ** 2)

    checked = 0
    for key in list(P):
        arr = P[key]
        for _ in range(2):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[key][idx] += h
            Pm[key][idx] -= h
            fd = (L_of(Pp) - L_of(Pm)) / (2 * h)
            an = G[key][idx]
            assert abs(fd - an) <= 2e-5 * max(abs(an), 1e-3 * abs(L)), (key, idx, fd, an)
            checked += 1
    assert checked == 2 * len(P)


def test_adam_first_step_closed_form():
    g = np.array([1e-3, -2.0, 0.5, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = nn.adam(p, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_flatten_roundtrip_and_count():
    P = nn.init_params(seed=1)
    f = nn.flatten(P)
    assert f.size == nn.n_params()
    Q = nn.unflatten(f)
    assert all(np.array_equal(P[k], Q[k]) for k in P)


@pytest.mark.parametrize("v,expect", [(1.0, 1.0), (1.0 + 2 ** -8, 1.0), (1.0 + 3 * 2 ** -8, 1.0 + 2 ** -6),
                                      (-2.5, -2.5), (1.0 + 2 ** -7, 1.0 + 2 ** -7)])
def test_bf16_rounding(v, expect):
    assert nn.bf16_round(np.array([v]))[0] == expect

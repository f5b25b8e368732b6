"""The seeded input generator, pinned to its published definition (CPU).

SplitMix64 (Steele, Lea & Flood, 2014; the reference C form by Vigna): the state advances by
the golden-ratio increment 0x9E3779B97F4A7C15 and each output is the state mixed by two
xor-shift-multiply rounds and a final xor-shift.  The generator draws the n-th output directly
from the index (state = seed + (n + 1) * increment); these tests check it against the
sequential definition, against the published first outputs for seed 1234567, and the
properties the parity tests rely on (offsets, the 53-bit uniform deviate, determinism).
"""
import numpy as np

import sph_inputs as si

M64 = (1 << 64) - 1


def _splitmix_sequential(seed, n):
    x, out = seed, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & M64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_published_first_outputs():
    # the first five outputs of SplitMix64 seeded with 1234567
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    assert [int(v) for v in si.splitmix64(1234567, 5)] == ref


def test_indexed_draws_equal_the_sequential_stream():
    for seed in (0, 1, 42, 2 ** 63 + 12345, M64):
        assert [int(v) for v in si.splitmix64(seed, 300)] == _splitmix_sequential(seed, 300)


def test_offsets_continue_the_stream():
    full = si.splitmix64(77, 1000)
    assert np.array_equal(si.splitmix64(77, 400, offset=600), full[600:])
    assert np.array_equal(si.uniform01(77, 10, offset=990), si.uniform01(77, 1000)[990:])


def test_uniform_deviate_is_the_top_53_bits():
    x = si.splitmix64(5, 4096)
    u = si.uniform01(5, 4096)
    assert np.array_equal(u, (x >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    assert u.min() >= 0.0 and u.max() < 1.0
    # 53-bit values are exact in FP64: scaling back gives integers
    assert np.array_equal(u * 2.0 ** 53, np.floor(u * 2.0 ** 53))
    # roughly uniform: the mean of 4096 draws within 5 sigma of 1/2
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)


def test_streamer_inputs_are_deterministic():
    a = si.streamer(n=24, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.2, targets_all=False, seed=9, name="a")
    b = si.streamer(n=24, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.2, targets_all=False, seed=9, name="b")
    assert np.array_equal(a.q, b.q) and np.array_equal(a.emag, b.emag)
    assert a.q.dtype == np.float32 and a.q.size == 24 ** 3


def test_stratified_targets_ball_and_uniform_part():
    """The parity sample: exactly the targets within the radius (brute force over every cell
    centre), plus the requested number of distinct others, ascending, deterministic."""
    p = si.gaussian_box(20, 16, 12, sigma_cells=3.0, h=0.01)
    T = np.flatnonzero(si.uniform01(9, p.ncell) < 0.6).astype(np.int32)
    c, r = (0.1, 0.08, 0.05), 0.035
    s, b, w = si.stratified_targets(p, T, c, r, 300, seed=4)
    X, Y, Z = p.centres()
    d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2).ravel()
    ball = T[d[T] <= r]
    assert np.array_equal(s[b], ball)
    others = s[~b]
    assert others.size == 300 and np.unique(others).size == 300
    assert np.all(np.isin(others, T)) and not np.any(np.isin(others, ball))
    assert np.all(np.diff(s) > 0)
    assert w == (T.size - ball.size) / 300
    s2, b2, _ = si.stratified_targets(p, T, c, r, 300, seed=4)
    assert np.array_equal(s, s2) and np.array_equal(b, b2)
    s3, _, _ = si.stratified_targets(p, T, c, r, 300, seed=5)
    assert not np.array_equal(s, s3)
    # asking for more than there is gives every target
    s4, b4, w4 = si.stratified_targets(p, T, c, r, 10 ** 6)
    assert np.array_equal(s4, T) and w4 == 1.0

"""GPU tests of batched evaluation (eval_sph_batch) and of the leaf-size autotuner.

A batch evaluates independent snapshots (different grids, pressures, target
rules); each snapshot must equal its own eval_sph on an identically configured
context up to the summation order of the atomic reductions (rel 1e-5), and pass
the same accuracy gate against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import sph_inputs as si

pytestmark = pytest.mark.gpu

REL_L2 = 1e-3
MAX_REL = 1e-2
SAME = 1e-5


@pytest.fixture(scope="module")
def sph():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as m
    return m


def _snapshots():
    return [
        si.streamer(n=48, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.3, targets_all=False, leaf_size=32,
                    sigma_head=0.02, chan_radius=0.02, seed=21, name="b48"),
        si.streamer(n=40, box=0.4, p_torr=76.0, chan_len=0.2, i_frac=1e-4, targets_all=True, leaf_size=32,
                    sigma_head=0.015, chan_radius=0.015, seed=22, name="b40_76torr"),
        si.plain_24(),
        si.streamer(n=32, box=0.3, p_torr=380.0, chan_len=0.15, i_frac=0.0, e_frac=0.5, targets_all=False,
                    leaf_size=32, seed=23, name="b32_380torr"),
    ]


def _configure(sph, ctx, leaf, prec):
    sph.set_criteria(ctx, 0.0, 0.0, 0.0, 1, leaf, prec)


def _single(sph, p, leaf, prec):
    ctx = sph.Context(0)
    ctx2, out, _ = sph.solve(p, ctx, m2l_precision=prec, leaf_size=leaf)
    return out.cpu().numpy().astype(np.float64)


def _close(a, b, label):
    d = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    assert d <= SAME, "%s: batch vs single rel %.3e" % (label, d)
    assert np.array_equal(a == 0, b == 0), label


def _oracle_gate(p, S):
    ref, J, T = oracle.sph_problem(p)
    S = np.asarray(S, np.float64)
    assert oracle.rel_l2(S[T], ref) <= REL_L2
    assert oracle.max_rel(S[T], ref, 1e-3) <= MAX_REL
    others = np.ones(S.size, bool)
    others[T] = False
    assert np.all(S[others] == 0.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_individual(sph, prec):
    import torch
    probs = _snapshots()
    ctx = sph.Context(0)
    _configure(sph, ctx, 32, prec)
    bps = [sph.BatchProblem.from_problem(p) for p in probs]
    outs, st = sph.eval_sph_batch(ctx, bps, stats=True)
    torch.cuda.synchronize()
    assert st.ms_total > 0
    ntot = 0
    for p, o in zip(probs, outs):
        S = o.cpu().numpy().astype(np.float64)
        _close(S, _single(sph, p, 32, prec), p.name)
        ntot += int(np.count_nonzero(S))
    assert st.n_targets >= ntot
    _oracle_gate(probs[0], outs[0].cpu().numpy())
    _oracle_gate(probs[1], outs[1].cpu().numpy())


def test_batch_repeat_and_without_graph(sph, monkeypatch):
    import torch
    probs = _snapshots()
    ctx = sph.Context(0)
    _configure(sph, ctx, 32, 1)
    bps = [sph.BatchProblem.from_problem(p) for p in probs]
    first = [o.cpu().numpy().astype(np.float64) for o in sph.eval_sph_batch(ctx, bps)[0]]
    # second call: same shapes (graph executable updated in place), fields changed in one snapshot
    bps[2].q.mul_(2.0)
    second = [o.cpu().numpy().astype(np.float64) for o in sph.eval_sph_batch(ctx, bps)[0]]
    for i in (0, 1, 3):
        _close(second[i], first[i], "repeat %d" % i)
    _close(second[2], 2.0 * first[2], "scaled q")
    # reorder the snapshots (different graph topology), then without graph capture
    rev = list(reversed(bps))
    third = [o.cpu().numpy().astype(np.float64) for o in sph.eval_sph_batch(ctx, rev)[0]]
    for i, s in enumerate(reversed(third)):
        _close(s, second[i], "reordered %d" % i)
    monkeypatch.setenv("SPH_BATCH_GRAPH", "0")
    ctx2 = sph.Context(0)
    _configure(sph, ctx2, 32, 1)
    plain = [o.cpu().numpy().astype(np.float64) for o in sph.eval_sph_batch(ctx2, bps)[0]]
    torch.cuda.synchronize()
    for i in range(len(bps)):
        _close(plain[i], second[i], "no graph %d" % i)


def test_batch_with_empty_snapshot_and_zero_length(sph):
    import torch
    probs = _snapshots()[:2]
    bps = [sph.BatchProblem.from_problem(p) for p in probs]
    # a snapshot with no targets: every |E| below the threshold through an all-zero mask
    p0 = probs[0]
    zero_mask = np.zeros(p0.nx * p0.ny * p0.nz, np.uint8)
    bps.insert(1, sph.BatchProblem.from_problem(p0, mask=zero_mask))
    bps[1].out.fill_(7.0)
    ctx = sph.Context(0)
    _configure(sph, ctx, 32, 1)
    outs, st = sph.eval_sph_batch(ctx, bps, stats=True)
    torch.cuda.synchronize()
    assert torch.count_nonzero(outs[1]).item() == 0
    _close(outs[0].cpu().numpy().astype(np.float64), _single(sph, probs[0], 32, 1), "with empty neighbour")
    outs0, st0 = sph.eval_sph_batch(ctx, [], stats=True)
    assert outs0 == [] and st0.n_targets == 0


def test_batch_rejects_bad_problem(sph):
    import torch
    p = _snapshots()[2]
    bp = sph.BatchProblem.from_problem(p)
    ctx = sph.Context(0)
    _configure(sph, ctx, 32, 1)
    bp.pO2 = -1.0
    with pytest.raises(sph.SphError) as e:
        sph.eval_sph_batch(ctx, [bp])
    assert e.value.code == -1
    bp.pO2 = p.pO2_torr
    bp.emag = torch.ones_like(bp.q)
    bp.mask = torch.ones(bp.q.numel(), dtype=torch.uint8, device=bp.q.device)
    with pytest.raises(sph.SphError):
        sph.eval_sph_batch(ctx, [bp])
    with pytest.raises(sph.SphError):
        sph.eval_sph_batch(sph.Context(0), [sph.BatchProblem.from_problem(p)])   # no set_criteria


def test_autotuned_leaf_size(sph):
    p = _snapshots()[0]
    ctx = sph.Context(0)
    _, out, st = sph.solve(p, ctx, m2l_precision=1, leaf_size=0, stats=True)
    leaf = st.leaf_size
    assert leaf in (32, 64, 512)
    S = out.cpu().numpy().astype(np.float64)
    _oracle_gate(p, S)
    _close(S, _single(sph, p, leaf, 1), "autotuned vs fixed leaf %d" % leaf)
    # cached: the second evaluation keeps the choice and gives the same field
    _, out2, st2 = sph.solve(p, ctx, m2l_precision=1, leaf_size=0, stats=True)
    assert st2.leaf_size == leaf
    _close(out2.cpu().numpy().astype(np.float64), S, "autotune cache")


def test_stress_batch_millions_of_sources(sph):
    """The wide-channel batch (channel radius 0.2 .. 1 mm, source threshold 1e-5; the last
    snapshot selects about three million sources on a 256^3 grid) in one eval_sph_batch with the
    leaf size and the M2L form autotuned: every snapshot selects the oracle's sets (counted) and
    passes the gate on 200 seeded sampled targets, zero at sampled non-targets."""
    import torch
    probs = si.stress_batch(4)
    ctx = sph.Context(0)
    _configure(sph, ctx, 0, sph.M2L_BF16X3)
    bps = [sph.BatchProblem.from_problem(p) for p in probs]
    outs, st = sph.eval_sph_batch(ctx, bps, stats=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(29)
    ns_total = 0
    for p, o in zip(probs, outs):
        S = o.cpu().numpy().astype(np.float64)
        J, T = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
        ns_total += J.size
        samp = np.sort(rng.choice(T, size=min(T.size, 200), replace=False))
        a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
        ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
        assert oracle.rel_l2(S[samp], ref) <= REL_L2, p.name
        assert oracle.max_rel(S[samp], ref, 1e-3) <= MAX_REL, p.name
        others = np.setdiff1d(rng.choice(p.ncell, size=2000, replace=False), T)
        assert np.all(S[others] == 0.0), p.name
        assert np.count_nonzero(S) <= T.size, p.name
    assert st.n_sources == ns_total
    assert ns_total > 2_500_000
    ctx.close()


def test_m2l_form_autotuned(sph):
    """With the leaf size autotuned the M2L form is timed too (tiles of V pairs against
    target-stationary tiles); whichever is kept, the result passes the oracle gate and the
    choice is cached for the problem class."""
    p = si.streamer(n=64, box=1.0, chan_len=0.5, i_frac=0.0, targets_all=True, seed=42, name="tune64")
    ctx = sph.Context(0)
    _, out, st = sph.solve(p, ctx, m2l_precision=sph.M2L_BF16X3, leaf_size=0, stats=True)
    assert st.m2l_tiles in (0, 1)
    _, out2, st2 = sph.solve(p, ctx, m2l_precision=sph.M2L_BF16X3, leaf_size=0, stats=True)
    assert st2.m2l_tiles == st.m2l_tiles and st2.leaf_size == st.leaf_size
    S = out2.cpu().numpy().astype(np.float64)
    samp = np.sort(np.random.default_rng(4).choice(p.ncell, 2000, replace=False)).astype(np.int32)
    a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, np.arange(p.ncell, dtype=np.int32), samp)
    assert oracle.rel_l2(S[samp], ref) <= REL_L2
    ctx.close()

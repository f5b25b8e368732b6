"""GPU tests of the learned surrogate's pipeline: FMM-generated training pairs, training,
and the judge / fallback evaluation (the FMM decides which coarse blocks the network may keep).

Small scale: 64^3 fine grid in the 1.5 cm cube, 4^3 pooling to a 16^3 coarse grid (8 judge
blocks).  The full-scale figures (256^3 -> 64^3, 2000 samples) come from bench.py.
"""
import numpy as np
import pytest

import sph_inputs as si

pytestmark = pytest.mark.gpu

N_FINE, FACTOR = 64, 4
D = N_FINE // FACTOR


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph
    from paper_2112_10059_gb300 import surrogate as sur
    return sph, sur


def _pool(a, f):
    n = round(a.size ** (1 / 3))
    m = n // f
    return a.reshape(m, f, m, f, m, f).mean(axis=(1, 3, 5))


def _fine_ctx(sph, sur, geom, p_torr=760.0, i_frac=1e-4):
    q, em = si.fields_torch(N_FINE, 1.5, geom)
    ctx = sph.Context(0)
    sph.set_grid(ctx, N_FINE, N_FINE, N_FINE, 1.5 / N_FINE, si.pO2_of(p_torr))
    sph.set_sources(ctx, q, si.scale_of(p_torr))
    sph.set_targets(ctx, emag=em)
    sph.set_criteria(ctx, i_frac, 0.0, 0.0, 1, 64, sph.M2L_BF16X3)
    ctx._fields = (q, em)
    return ctx


def _truth(sph, geom, p_torr=760.0, i_frac=1e-4):
    """Pooled fine-grid FMM over every cell (what the surrogate estimates)."""
    q, _ = si.fields_torch(N_FINE, 1.5, geom)
    ctx = sph.Context(0)
    sph.set_grid(ctx, N_FINE, N_FINE, N_FINE, 1.5 / N_FINE, si.pO2_of(p_torr))
    sph.set_sources(ctx, q, si.scale_of(p_torr))
    sph.set_targets(ctx)
    sph.set_criteria(ctx, i_frac, 0.0, 0.0, 1, 64, sph.M2L_BF16X3)
    S, _ = sph.eval_sph(ctx)
    return _pool(S.cpu().numpy().astype(np.float64), FACTOR)


def test_training_pair_definition(mods):
    sph, sur = mods
    net = sur.Net(edge=D, max_batch=1, seed=1)
    cf, cc = sph.Context(0), sph.Context(0)
    x, t, S_c, S_f = sur.make_sample(net, si.cloud_geometry(0), N_FINE, FACTOR, cf, cc)
    Sf = S_f.cpu().numpy().astype(np.float64)
    Sc = S_c.cpu().numpy().astype(np.float64)
    assert np.all(Sf > 0) and np.all(Sc > 0)
    ref = np.log(_pool(Sf, FACTOR).ravel() / Sc)
    assert np.max(np.abs(t.cpu().numpy() - ref)) < 1e-5
    xs = x.float().cpu().numpy().reshape(-1, 16)
    assert np.all(xs[:, 4:] == 0) and xs[:, 0].max() <= 1.0 + 1e-2 and xs[:, 2].max() == 1.0
    assert xs[:, 3].max() == 1.0 and xs[:, 3].min() >= 0.0


def test_bad_network_falls_back_everywhere(mods):
    """A deliberately wrong network (head bias r = 0.5: S_pred off by 65%) is rejected by the
    judge in every block and the result is the FMM's."""
    sph, sur = mods
    geom = si.cloud_geometry(1)
    net = sur.Net(edge=D, max_batch=1, seed=2)
    p = net.get_params()
    p[-2] = 0.5          # head bias of r
    net.set_params(p)
    ctx = _fine_ctx(sph, sur, geom)
    out, st = sur.evaluate(ctx, net, FACTOR, tol=1e-3, samples=2, seed=3, use_net=True)
    assert st.n_blocks == (D // 8) ** 3
    assert st.n_fallback == st.n_blocks and st.n_judged_fail == st.n_blocks
    truth = _truth(sph, geom).ravel()
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - truth) / truth) < 1e-4
    assert st.n_fallback_targets == N_FINE ** 3


def test_coarse_only_and_judge_counts(mods):
    sph, sur = mods
    geom = si.cloud_geometry(2)
    net = sur.Net(edge=D, max_batch=1, seed=2)
    ctx = _fine_ctx(sph, sur, geom)
    out, st = sur.evaluate(ctx, net, FACTOR, tol=1e9, samples=3, seed=4, use_net=False)
    # nothing fails at an absurd tolerance: the output is the coarse FMM estimate
    assert st.n_fallback == 0 and st.n_fallback_targets == 0
    assert 0 < st.n_judge_targets <= st.n_blocks * 3 * FACTOR ** 3
    cc = sph.Context(0)
    q = ctx._fields[0]
    qc = sur.pool_avg(q, N_FINE, FACTOR)
    sph.set_grid(cc, D, D, D, 1.5 / D, si.pO2_of(760.0))
    sph.set_sources(cc, qc, si.scale_of(760.0))
    sph.set_targets(cc)
    sph.set_criteria(cc, 1e-4, 0.0, 0.0, 1, 64, sph.M2L_BF16X3)
    Sc, _ = sph.eval_sph(cc)
    # the same coarse evaluation twice: equal up to the order of the FP32 reductions
    d = np.max(np.abs(out.cpu().numpy() - Sc.cpu().numpy()) / Sc.cpu().numpy())
    assert d < 5e-5
    with pytest.raises(sph.SphError):
        sur.evaluate(ctx, net, 2, use_net=False)        # 64 != 2 * 16


def test_trained_network_gain(mods):
    """What training buys, at 128^3 -> 32^3: the trained network's S_pred error against the
    pooled fine FMM on held-out geometries, against the coarse FMM alone; and the judged
    result stays within the judge's tolerance."""
    sph, sur = mods
    nf, f = 128, 4
    d = nf // f
    net = sur.Net(edge=d, max_batch=8, seed=5)
    X, T = sur.training_set(net, 256, nf, f, first=0)
    Xv, Tv = sur.training_set(net, 16, nf, f, first=100000)
    before = sur.validation_loss(net, Xv, Tv)
    hist = sur.train(net, X, T, epochs=40, batch=8, lr=2e-3, lr_final=2e-4, X_val=Xv, T_val=Tv)
    after = hist[-1][2]
    assert after < 0.6 * before, (before, after)
    errs_n, errs_c = [], []
    for i in range(0, 16, 8):
        y = net.forward(Xv[i:i + 8].reshape(-1), 8).cpu().numpy().reshape(8, -1, 2)
        t = Tv[i:i + 8].cpu().numpy().reshape(8, -1)
        errs_n.append(np.abs(np.expm1(y[..., 0] - t)))
        errs_c.append(np.abs(np.expm1(-t)))
    err_net, err_coarse = np.mean(errs_n), np.mean(errs_c)
    assert err_net < 0.6 * err_coarse, (err_net, err_coarse)
    geom = si.cloud_geometry(100000)
    q, em = si.fields_torch(nf, 1.5, geom)
    ctx = sph.Context(0)
    sph.set_grid(ctx, nf, nf, nf, 1.5 / nf, si.pO2_of(760.0))
    sph.set_sources(ctx, q, si.scale_of(760.0))
    sph.set_targets(ctx, emag=em)
    sph.set_criteria(ctx, 1e-4, 0.0, 0.0, 1, 64, sph.M2L_BF16X3)
    full = sph.Context(0)
    sph.set_grid(full, nf, nf, nf, 1.5 / nf, si.pO2_of(760.0))
    sph.set_sources(full, q, si.scale_of(760.0))
    sph.set_targets(full)
    sph.set_criteria(full, 1e-4, 0.0, 0.0, 1, 64, sph.M2L_BF16X3)
    S, _ = sph.eval_sph(full)
    truth = sur.pool_avg(S, nf, f).cpu().numpy().astype(np.float64)
    out, st = sur.evaluate(ctx, net, f, tol=1e-2, samples=2, seed=6, use_net=True)
    e = np.linalg.norm(out.cpu().numpy() - truth) / np.linalg.norm(truth)
    assert e <= 1e-2, (e, st.as_dict())

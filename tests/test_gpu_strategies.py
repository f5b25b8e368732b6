"""GPU checks of the source-selection trade-off of Section 4.3 (Eq. sourcepct) at reduced size.

A spherical Gaussian (sigma = 8 cells) in a 2:2:1 box, every cell a target; the FMM with
sources I >= I_pct max I is compared with the full FP64 sum (no selection) on sampled
targets: E_V (relative L2 over the samples) grows with I_pct, and each run stays within the
FMM gate of the FP64 sum over its own selected sources.
"""
import numpy as np
import pytest

import oracle
import sph_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as m
    return m


def test_source_fraction_tradeoff(sph):
    p = si.gaussian_box(48, 48, 24, sigma_cells=8.0, h=1.25e-3, pO2_torr=150.0)
    a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    samp = np.sort(np.random.default_rng(7).choice(p.ncell, 1500, replace=False)).astype(np.int32)
    Jall = np.arange(p.ncell, dtype=np.int32)
    full = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, Jall, samp)
    ev = []
    for f in (1e-4, 1e-3, 1e-2, 1e-1):
        p.i_frac = f
        c = sph.Context(0)
        _, out, st = sph.solve(p, c, m2l_precision=sph.M2L_BF16X3, stats=True)
        S = out.cpu().numpy().astype(np.float64)[samp]
        Jf, _ = oracle.select(p.q, None, None, f)
        own = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, Jf, samp)
        assert oracle.rel_l2(S, own) <= 1e-3, f              # the FMM itself stays within its gate
        ev.append(oracle.rel_l2(S, full))
        assert st.n_sources == Jf.size
        c.close()
    assert ev[0] < ev[1] < ev[2] < ev[3], ev
    assert ev[0] < 1e-2 and ev[3] > 5e-2, ev

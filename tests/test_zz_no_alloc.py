"""The allocation-free selection entry point (sph_select_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory while they run; its scratch
lives in a fixed device array inside the library, shared by every call.  Two calls
in a row with different inputs must each give exactly the selection of the regular
entry point (eval_sph + sph_get_selection): the same index sets (selection is
integer work, so the comparison is bit-exact) and the same source values.

This file is collected last on purpose, and it passes both alone in a fresh process
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import sph_inputs as si

pytestmark = pytest.mark.gpu


def _lin(pc, nx, ny):
    pc = pc.astype(np.int64)
    return (pc & 1023) + nx * (((pc >> 10) & 1023) + ny * ((pc >> 20) & 1023))


def test_select_noalloc_matches_regular_path_twice():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph

    lib = sph.load()
    cases = [
        si.streamer(n=48, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.3, targets_all=False, seed=31,
                    name="first"),
        si.streamer(n=40, box=0.4, chan_len=0.2, i_frac=1e-2, e_frac=0.15, targets_all=False, seed=32,
                    sigma_head=0.01, name="second"),
    ]
    for p in cases:
        ctx, _, _ = sph.solve(p)
        J, T = sph.get_selection(ctx)
        ctx.close()

        n = p.ncell
        dev = torch.device("cuda", 0)
        q = torch.from_numpy(p.q).to(dev)
        em = torch.from_numpy(p.emag).to(dev)
        skey = torch.empty(n, dtype=torch.int32, device=dev)
        spc = torch.empty(n, dtype=torch.int32, device=dev)
        sq = torch.empty(n, dtype=torch.float32, device=dev)
        tkey = torch.empty(n, dtype=torch.int32, device=dev)
        tpc = torch.empty(n, dtype=torch.int32, device=dev)
        counts = torch.full((2,), -1, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        rc = lib.sph_select_noalloc(0, ctypes.c_void_p(stream.cuda_stream), p.nx, p.ny, p.nz, P(q), P(em), None,
                                    p.i_frac, p.e_frac, p.e_applied, P(skey), P(spc), P(sq), P(tkey), P(tpc),
                                    P(counts))
        assert rc == 0
        torch.cuda.synchronize()
        ns, nt = counts.cpu().numpy().tolist()
        assert ns == J.size and nt == T.size
        src = _lin(spc[:ns].cpu().numpy(), p.nx, p.ny)
        trg = _lin(tpc[:nt].cpu().numpy(), p.nx, p.ny)
        assert np.array_equal(np.sort(src), J)
        assert np.array_equal(np.sort(trg), T)
        # Morton order and the source values
        assert np.all(np.diff(skey[:ns].cpu().numpy().view(np.uint32).astype(np.int64)) > 0)
        assert np.array_equal(sq[:ns].cpu().numpy(), p.q[src])


def test_select_noalloc_rejects_oversized_grid():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph
    lib = sph.load()
    dummy = ctypes.c_void_p(16)
    rc = lib.sph_select_noalloc(0, None, 513, 4, 4, dummy, None, None, 0.0, 0.0, 0.0, dummy, dummy, dummy,
                                dummy, dummy, dummy)
    assert rc == -5   # SPH_ECAPACITY, before any work is queued

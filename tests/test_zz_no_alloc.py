"""The allocation-free selection entry point (sph_select_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory while they run; its scratch
lives in a fixed device array inside the library, shared by every call.  Calls in a
row with different inputs must each give exactly the selection of the regular entry
point (eval_sph + sph_get_selection) and of the FP64 oracle's selection rules: the
same index sets (selection is integer work, so the comparison is bit-exact), the
same source values, and a zero failure flag.  The cases cover the three target
modes (|E| rule, explicit mask, every cell), the capacity edge (512 cells on one
axis: the scratch's full 32768-brick layout) and bricks decided whole from the
maxima pass's per-brick statistics (their packed cells written without a read).

This file is collected last on purpose, and it passes both alone in a fresh process
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import sph_inputs as si

pytestmark = pytest.mark.gpu


def _lin(pc, nx, ny):
    pc = pc.astype(np.int64)
    return (pc & 1023) + nx * (((pc >> 10) & 1023) + ny * ((pc >> 20) & 1023))


def _edge_case():
    """512 x 8 x 8 cells (the largest axis the entry point takes), one Gaussian, |E| rule."""
    p = si.gaussian_box(512, 8, 8, sigma_cells=60.0, h=1e-3)
    p.i_frac = 1e-3
    x = np.arange(p.ncell) % 512
    p.emag = (30.0 + 120.0 * np.exp(-((x - 300.0) / 50.0) ** 2)).astype(np.float32)
    p.targets_all = False
    p.e_frac = 0.4
    return p, None


def _cases():
    first = si.streamer(n=48, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.3, targets_all=False, seed=31,
                        name="first")
    second = si.streamer(n=40, box=0.4, chan_len=0.2, i_frac=1e-2, e_frac=0.15, targets_all=False, seed=32,
                         sigma_head=0.01, name="second")
    masked = si.gaussian_box(40, 24, 33, sigma_cells=5.0)
    masked.i_frac = 1e-2
    masked_mask = si.random_mask(masked.ncell, 0.3, seed=33)
    every = si.gaussian_box(512, 8, 8, sigma_cells=40.0, h=1e-3)
    every.i_frac = 1e-2
    bricks = si.brick_structured(56, 48, 40)
    return [(first, None), (second, None), _edge_case(), (masked, masked_mask), (every, None), (bricks, None)]


def test_select_noalloc_matches_regular_path_and_oracle():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph

    lib = sph.load()
    dev = torch.device("cuda", 0)
    for p, mask in _cases():
        ctx, _, _ = sph.solve(p, mask=mask)
        J, T = sph.get_selection(ctx)
        ctx.close()
        emag = None if (p.targets_all or mask is not None) else p.emag
        Jo, To = oracle.select(p.q, emag, mask, p.i_frac, p.e_frac, p.e_applied)
        assert np.array_equal(J, Jo) and np.array_equal(T, To), p.name

        n = p.ncell
        q = torch.from_numpy(p.q).to(dev)
        em = torch.from_numpy(emag).to(dev) if emag is not None else None
        mk = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to(dev) if mask is not None else None
        skey = torch.empty(n, dtype=torch.int32, device=dev)
        spc = torch.empty(n, dtype=torch.int32, device=dev)
        sq = torch.empty(n, dtype=torch.float32, device=dev)
        tkey = torch.empty(n, dtype=torch.int32, device=dev)
        tpc = torch.empty(n, dtype=torch.int32, device=dev)
        counts = torch.full((3,), -7, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        rc = lib.sph_select_noalloc(0, ctypes.c_void_p(stream.cuda_stream), p.nx, p.ny, p.nz, P(q), P(em), P(mk),
                                    ctypes.c_double(p.i_frac), ctypes.c_double(p.e_frac),
                                    ctypes.c_double(p.e_applied), P(skey), P(spc), P(sq), P(tkey), P(tpc),
                                    P(counts))
        assert rc == 0, p.name
        torch.cuda.synchronize()
        ns, nt, failed = counts.cpu().numpy().tolist()
        assert failed == 0, p.name
        assert ns == Jo.size and nt == To.size, p.name
        src = _lin(spc[:ns].cpu().numpy(), p.nx, p.ny)
        trg = _lin(tpc[:nt].cpu().numpy(), p.nx, p.ny)
        assert np.array_equal(np.sort(src), Jo), p.name
        assert np.array_equal(np.sort(trg), To), p.name
        # Morton order and the source values
        assert np.all(np.diff(skey[:ns].cpu().numpy().view(np.uint32).astype(np.int64)) > 0)
        assert np.all(np.diff(tkey[:nt].cpu().numpy().view(np.uint32).astype(np.int64)) > 0)
        assert np.array_equal(sq[:ns].cpu().numpy(), p.q[src])


def test_select_noalloc_rejects_oversized_grid():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph
    lib = sph.load()
    dummy = ctypes.c_void_p(16)
    rc = lib.sph_select_noalloc(0, None, 513, 4, 4, dummy, None, None, ctypes.c_double(0.0), ctypes.c_double(0.0),
                                ctypes.c_double(0.0), dummy, dummy, dummy, dummy, dummy, dummy)
    assert rc == -5   # SPH_ECAPACITY, before any work is queued

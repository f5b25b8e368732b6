"""Failure paths of the library, made to happen on purpose without faulting the GPU.

* A bounded wait that runs out: the selection's decoupled look-back and the device scan poll
  their predecessors a limited number of times.  With the limit set to 0 from the environment
  every block after the first gives up at once (deterministically, with no spinning), the
  kernels still write only inside their outputs, and the host reports SPH_ETIMEOUT (the
  allocation-free selection reports it in its flag word).  A context created afterwards, with
  the default limits, gives the oracle's selection again.
* A failed allocation, injected on the host (SPH_FAULT=alloc): the call returns SPH_ENOMEM
  without poisoning the context, and the same context's next call succeeds with the same result
  as a fresh context.
"""
import ctypes

import numpy as np
import pytest

import oracle
import sph_inputs as si

pytestmark = pytest.mark.gpu

SPH_ENOMEM, SPH_ETIMEOUT = -2, -6


@pytest.fixture(scope="module")
def sph():
    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as m
    return m


def _case():
    return si.streamer(n=48, box=0.5, chan_len=0.25, i_frac=1e-3, e_frac=0.3, targets_all=False, seed=31,
                       name="fail48")


def test_selection_lookback_runs_out(sph, monkeypatch):
    p = _case()
    monkeypatch.setenv("SPH_SELECT_LOOKBACK", "1")      # the form whose CTAs wait on one another
    monkeypatch.setenv("SPH_WAIT_LIMIT_SELECT", "0")
    c = sph.Context(0)
    with pytest.raises(sph.SphError) as e:
        sph.solve(p, c)
    assert e.value.code == SPH_ETIMEOUT
    c.close()
    monkeypatch.delenv("SPH_WAIT_LIMIT_SELECT")
    c = sph.Context(0)
    sph.solve(p, c)
    J, T = sph.get_selection(c)
    c.close()
    Jo, To = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
    assert np.array_equal(J, Jo) and np.array_equal(T, To)


def test_noalloc_selection_reports_giving_up(sph, monkeypatch):
    import torch
    p = _case()
    lib = sph.load()
    dev = torch.device("cuda", 0)
    n = p.ncell
    q = torch.from_numpy(p.q).to(dev)
    em = torch.from_numpy(p.emag).to(dev)
    outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(4)]
    sq = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())

    def run():
        counts = torch.full((3,), -7, dtype=torch.int32, device=dev)
        rc = lib.sph_select_noalloc(0, ctypes.c_void_p(stream.cuda_stream), p.nx, p.ny, p.nz, P(q), P(em), None,
                                    ctypes.c_double(p.i_frac), ctypes.c_double(p.e_frac),
                                    ctypes.c_double(p.e_applied), P(outs[0]), P(outs[1]), P(sq), P(outs[2]),
                                    P(outs[3]), P(counts))
        torch.cuda.synchronize()
        return rc, counts.cpu().numpy().tolist()

    monkeypatch.setenv("SPH_SELECT_LOOKBACK", "1")
    monkeypatch.setenv("SPH_WAIT_LIMIT_SELECT", "0")
    rc, (ns, nt, failed) = run()
    assert rc == 0 and failed != 0 and ns == -1 and nt == -1
    monkeypatch.delenv("SPH_WAIT_LIMIT_SELECT")
    rc, (ns, nt, failed) = run()
    Jo, To = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
    assert rc == 0 and failed == 0 and ns == Jo.size and nt == To.size


def test_device_scan_runs_out(sph, monkeypatch):
    import torch
    x = torch.ones(1 << 20, dtype=torch.int32, device="cuda:0")
    monkeypatch.setenv("SPH_WAIT_LIMIT_SCAN", "0")
    with pytest.raises(sph.SphError) as e:
        sph.scan_i32(x)
    assert e.value.code == SPH_ETIMEOUT
    monkeypatch.delenv("SPH_WAIT_LIMIT_SCAN")
    out, total = sph.scan_i32(x)
    assert total == x.numel()
    assert np.array_equal(out.cpu().numpy(), np.arange(x.numel(), dtype=np.int32))


@pytest.mark.parametrize("k", [1, 5])
def test_injected_allocation_failure(sph, monkeypatch, k):
    p = _case()
    monkeypatch.setenv("SPH_FAULT", "alloc:%d" % k)
    c = sph.Context(0)
    monkeypatch.delenv("SPH_FAULT")
    with pytest.raises(sph.SphError) as e:
        sph.solve(p, c)
    assert e.value.code == SPH_ENOMEM
    _, out, _ = sph.solve(p, c)              # the same context, injection spent: succeeds
    got = out.cpu().numpy()
    c.close()
    fresh = sph.Context(0)
    _, ref, _ = sph.solve(p, fresh)
    ref = ref.cpu().numpy()
    fresh.close()
    assert oracle.rel_l2(got, ref) < 1e-5

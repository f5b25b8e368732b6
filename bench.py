"""Benchmark: S_ph targets/s of the adaptive FMM on one GB300 (or N replicas).

Workload (default): the 256^3 adaptive streamer case -- a 1 cm cube at 760 Torr,
Gaussian head + channel emission, sources with I >= 1e-4 max I, targets with
|E| >= 0.1 max|E| -- evaluated through the C ABI (eval_sph) with inputs resident
in device memory.  One step = one full evaluation: selection, octree and lists,
upward pass, M2L, downward pass, leaves.  L2 is flushed (256 MiB write) between
timed steps; each step is timed with CUDA events on the library's stream.

Printed: one JSON line (rank 0) with value = targets/s summed over ranks,
e2e = the same through eval_sph_host (host buffers, copies inside the timed
region), roofline of the dominant kernel, the FP32 direct sum on the same GPU,
accuracy against the FP64 oracle on sampled targets, and the CPU oracle baseline.

``--impl reference`` times the FP64 CPU oracle (the plain direct quadrature) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sph_inputs as si  # noqa: E402

MUFU_PER_SM_CLK = 16          # SFU (MUFU) results per SM per clock on sm_100-class parts
MUFU_PER_EVAL = 3             # rsqrt + 2 x ex2 per kernel evaluation
NSM = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid edge (cells)")
    ap.add_argument("--workload", default="adaptive", choices=["adaptive", "full"],
                    help="adaptive: sources I >= 1e-4 max I, targets |E| >= 0.1 max|E|; full: every cell a source "
                         "and a target (no adaptivity)")
    ap.add_argument("--p", type=float, default=760.0, help="pressure (Torr)")
    ap.add_argument("--m2l", default="bf16x3", choices=["f32", "bf16x3"])
    ap.add_argument("--order", type=int, default=5, help="Chebyshev order of the far field")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-snapshot batched evaluation")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-surrogate", action="store_true", help="skip training and judging the learned surrogate")
    ap.add_argument("--sweep", action="store_true",
                    help="Section 4.3 trade-off: FMM time and E_V against the full FP64 sum for I_pct 1e-4 .. 1e-1")
    ap.add_argument("--sur-samples", type=int, default=2000, help="FMM solves in the surrogate's training set")
    ap.add_argument("--sur-epochs", type=int, default=10)
    ap.add_argument("--acc-uniform", type=int, default=None,
                    help="uniform targets of the stratified oracle sample (plus every target within 5 sigma of the head); "
                         "default 100000 (adaptive workload), 1000 (every cell a source)")
    ap.add_argument("--no-decomp", action="store_true", help="skip the error decomposition (M2L arithmetic, fusion, order)")
    ap.add_argument("--no-full128", action="store_true",
                    help="skip the non-adaptive 128^3 FMM-vs-direct block (every cell a source and a target)")
    ap.add_argument("--no-pressures", action="store_true", help="skip the 76 and 380 Torr runs of the 256^3 workload")
    ap.add_argument("--fft256", action="store_true",
                    help="also time the FP64 FFT convolution of the 256^3 workload and check every target against it")
    a = ap.parse_args()
    if a.acc_uniform is None:
        a.acc_uniform = 100000 if a.workload == "adaptive" else 1000
    if a.workload == "full":
        a.no_full128 = True          # that block is this workload at 128^3
    return a


def workload(args):
    if args.workload == "full":
        p = si.streamer_full(args.n)
        if args.p != 760.0:
            p = si.streamer(n=args.n, box=1.0, p_torr=args.p, chan_len=0.5, i_frac=0.0, targets_all=True, seed=1001,
                            with_efield=False, name="streamer_%d_full" % args.n)
        return p
    return si.streamer_adaptive(n=args.n, p_torr=args.p)


def workload_cfg(p, args):
    if args.workload == "full":
        desc = "streamer %d^3 in 1 cm, %g Torr, every cell a source and a target" % (args.n, args.p)
    else:
        desc = "streamer %d^3 in 1 cm, %g Torr, sources I>=1e-4*max, targets |E|>=0.1*max|E|" % (args.n, args.p)
    return {"workload": desc,
            "grid": [p.nx, p.ny, p.nz], "pressure_torr": args.p, "i_frac": p.i_frac, "e_frac": p.e_frac,
            "leaf_size": p.leaf_size, "m2l": args.m2l, "far_field": "chebyshev order %d" % args.order,
            "l2_flush_between_steps": True,
            "inputs_resident_in_hbm": True}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    """Measured peaks of this GPU pool (HBM copy GB/s, dense BF16 TFLOP/s), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# DRAM bytes (read + write) per launch from one ncu capture each of the 256^3 adaptive workload
# (dram__bytes_read.sum + dram__bytes_write.sum of the kernel); valid for that workload and the
# kernels as profiled (removed once a kernel has changed since).
NCU_TRAFFIC = {"m2l": (97.748 + 2.976) * 1e6, "l2lp": (26.381 + 9.930) * 1e6}


def pipe_peaks(sph, dev, stream, f_mhz_nominal=2070.0):
    """FP32 FMA and MUFU throughput measured by the library's own kernels (sph_measure_pipe_peaks),
    with the nominal figures as a fallback if the measurement fails."""
    try:
        m = sph.pipe_peaks(dev.index or 0, stream)
        m["source"] = "measured (sph_measure_pipe_peaks: 8 independent chains per thread, 8 CTAs x 256 per SM)"
        return m
    except Exception as e:  # pragma: no cover - only without the library
        f = f_mhz_nominal * 1e6
        return {"ffma_flops": NSM * 128 * 2 * f, "ex2_per_s": NSM * MUFU_PER_SM_CLK * f,
                "rsqrt_per_s": NSM * MUFU_PER_SM_CLK * f, "n_sm": NSM,
                "source": "nominal (measurement failed: %s)" % e}


def rooflines(tree, step_stats, args, nt, ns, ncell, peaks, pipes, traffic_ok=True, order=None):
    """Achieved vs peak per kernel.  Work is ALGORITHMIC (what the method needs), not executed:
      m2l  (tensor, k_m2l_tc): 2 n^2 flops per V pair, n = order^3 (the BF16 x3 split executes
                     3 x 2 x 128^2);
      l2l  (tensor): 2 n^2 flops per child box with targets below level 2 (levels the separate
                     L2L kernels run: all but the deepest one when that level is fused);
      l2lp (HBM, k_l2lp_tc): fused L2L + L2P of the deepest level, parent terms: the parents'
                  local expansions read (npad x 4 B each) + S written (4 B per target there);
      l2p  (HBM, k_l2p_own + the separable L2P): the own local terms of the deepest leaves that
                  have V or X entries read (npad x 4 B each) with S read and written at their
                  targets (8 B per target), and the other levels' leaves (npad x 4 B per leaf
                  with targets + 4 B per target written) -- only where such leaves exist;
      near (MUFU, k_p2p): P2P pairs + M2P evaluations, 2 ex2 + 1 rsqrt each, against the measured
                  ex2 and rsqrt rates;
      select (HBM, k_brick_stats + k_select_onepass): 8 B per cell (q and |E| read once) + 4 B
                  per selected index (sources and targets) -- the minimum of the operation: the
                  maxima pass reads every cell, the rules re-read only the bricks that the
                  maxima pass's per-brick statistics leave undecided.
    Times are the medians of the library's CUDA-event phase timers; the step's dominant single
    kernel is the entry with the longest time among those timed as one kernel."""
    order = order or args.order
    n = order ** 3
    npad = (n + 15) // 16 * 16
    med = lambda k: statistics.median(x[k] for x in step_stats)
    fused = all(x["l2lp_fused"] for x in step_stats)
    lev = tree["level"]
    ntb = (tree["trg_end"] - tree["trg_begin"]).astype(np.int64)
    nsb = (tree["src_end"] - tree["src_begin"]).astype(np.int64)
    lmax = int(lev.max()) if lev.size else 0
    deep = (lev == lmax) if fused else np.zeros(lev.size, bool)
    n_child = int(np.sum((lev >= 3) & (ntb > 0) & ~deep))
    leaf_t = tree["leaf"] & (ntb > 0) & (lev >= 2)
    n_leaf_t = int(np.sum(leaf_t & ~deep))
    nt_other = int(np.sum(ntb[leaf_t & ~deep]))
    nV = len(tree["V"])
    U, W = tree["U"], tree["W"]
    p2p = int(np.sum(ntb[U[:, 0]] * nsb[U[:, 1]])) if len(U) else 0
    m2p = int(np.sum(ntb[W[:, 0]]) * n) if len(W) else 0
    fp32_peak = pipes["ffma_flops"] / 1e12
    mufu_evals = 1.0 / (2.0 / pipes["ex2_per_s"] + 1.0 / pipes["rsqrt_per_s"])
    tc = args.m2l == "bf16x3"
    tpk = peaks["bf16_tflops"]
    hbm = peaks["hbm_gbs"]
    hbm_basis = "measured HBM copy %.0f GB/s (%s)" % (hbm, peaks["source"])
    out = {}

    def add(name, kernel, single, bound, work, unit_work, ms, peak, unit, basis, traffic=None):
        ach = work / (ms * 1e-3) if ms > 0 else 0.0
        scale = 1e12 if unit == "TFLOP/s" else (1e9 if unit == "GB/s" else 1.0)
        out[name] = {"kernel": kernel, "single_kernel": single, "bound": bound, "achieved": ach / scale,
                     "peak": peak, "unit": unit, "frac": (ach / scale) / peak if peak else None,
                     "traffic": traffic, "ms_per_launch": ms, "work_per_launch": work, "work_unit": unit_work,
                     "peak_basis": basis}

    tiles = tc and all(x.get("m2l_tiles", 0) for x in step_stats)   # target-stationary form ran
    # pair tiles: the persistent tile loop unless SPH_M2L_LOOP=0 (one CTA per tile)
    pairs_k = "k_m2l_tc_loop" if os.environ.get("SPH_M2L_LOOP", "1") != "0" else "k_m2l_tc"
    add("m2l", ("k_m2l_groups + k_m2l_tiles" if tiles else pairs_k) if tc else "k_m2l_pairs", not tiles,
        "tensor" if tc else "alu", 2.0 * n * n * nV, "flop",
        med("ms_m2l"), tpk if tc else fp32_peak, "TFLOP/s",
        ("measured dense BF16 %.1f TFLOP/s burst (%s)" % (tpk, peaks["source"])) if tc else
        "measured FP32 FMA %.1f TFLOP/s (%s)" % (fp32_peak, pipes["source"]),
        traffic=NCU_TRAFFIC.get("m2l") if traffic_ok and tc and not tiles else None)
    if n_child > 0:
        add("l2l", "k_l2l_tc8 + k_l2l_tc" if tc else "k_l2l_gemm", False, "tensor" if tc else "alu",
            2.0 * n * n * n_child, "flop", med("ms_l2l"), tpk if tc else fp32_peak, "TFLOP/s", "as m2l")
    ms_lp = med("ms_l2lp") if fused else 0.0
    if fused:
        n_par = int(np.sum((lev == lmax - 1) & ~tree["leaf"] & (ntb > 0)))
        terms = np.zeros(lev.size, bool)
        for key in ("V", "X"):
            if len(tree.get(key, ())):
                terms[np.asarray(tree[key])[:, 0]] = True
        n_deep = int(np.sum(leaf_t & deep & terms))
        nt_own = int(np.sum(ntb[leaf_t & deep & terms]))
        nt_deep = int(np.sum(ntb[leaf_t & deep]))
        add("l2lp", "k_l2lp_tc", True, "hbm", 4.0 * npad * n_par + 4.0 * nt_deep, "bytes", ms_lp, hbm,
            "GB/s", hbm_basis, traffic=NCU_TRAFFIC.get("l2lp") if traffic_ok else None)
    else:
        n_deep = nt_own = 0
    if n_leaf_t + n_deep > 0:
        add("l2p", ("k_l2p_own + " if n_deep else "") + ("k_l2p_tc + " if tc and not fused else "") +
            "k_l2p_sep_small + k_l2p_sep", False, "hbm",
            4.0 * npad * (n_leaf_t + n_deep) + 4.0 * nt_other + 8.0 * nt_own, "bytes", med("ms_l2p") - ms_lp, hbm,
            "GB/s", hbm_basis)
    add("near", "k_p2p", True, "alu", float(p2p + m2p), "kernel-evals", med("ms_near"), mufu_evals, "evals/s",
        "MUFU: 2 ex2 + 1 rsqrt per evaluation at the measured %.3g ex2/s and %.3g rsqrt/s (%s)"
        % (pipes["ex2_per_s"], pipes["rsqrt_per_s"], pipes["source"]))
    add("select", "k_brick_stats + k_select_onepass", False, "hbm", 8.0 * ncell + 4.0 * (nt + ns),
        "bytes", med("ms_select"), hbm, "GB/s", hbm_basis)
    return out


def dominant_kernel(roof):
    """The entry of the longest-running single kernel."""
    singles = {k: v for k, v in roof.items() if v["single_kernel"]}
    return max(singles, key=lambda k: singles[k]["ms_per_launch"])


def oracle_sample(p, J, T, seconds, seed=5):
    """Time the FP64 oracle on a bounded random sample of targets; returns (targets/s, sample, seconds, cores).

    The sample grows geometrically until one timed run lasts at least half of ``seconds``
    (or covers every target), so that thread start-up does not dominate the figure.
    """
    import oracle
    a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    rng = np.random.default_rng(seed)
    n1 = max(8, min(T.size, 64))
    while True:
        samp = np.sort(rng.choice(T, size=n1, replace=False))
        t0 = time.perf_counter()
        oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds or n1 >= T.size:
            return n1 / dt, n1, dt, oracle.num_threads()
        n1 = int(min(T.size, max(2 * n1, n1 * 0.8 * seconds / max(dt, 1e-3))))


def whole_job_rate(ms_local, units_per_rank, world, dist=None, device=None):
    """Step time of the job = the maximum over the ranks (every rank calls this; a collective
    when dist is given), and the job's rate = the units all ranks processed per second of it."""
    ms = float(ms_local)
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms * 1e-3)


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = workload(args)
    J, T = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
    per_step = []
    nsamp = 0
    for k in range(args.warmup + args.steps):
        rate, n1, dt, cores = oracle_sample(p, J, T, max(1.0, min(args.cpu_seconds, 120.0 / (args.steps + args.warmup))),
                                            seed=100 + k)
        if k >= args.warmup:
            per_step.append(rate)
            nsamp = n1
    v = statistics.median(per_step)
    line = {"impl": "reference", "metric": "S_ph targets/s", "value": v, "unit": "targets/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T.size / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_cfg(p, args),
            "cpu_baseline": {"value": v, "unit": "targets/s", "cores": cores, "kind": "oracle",
                             "sample": "%d random targets of %d per step (FP64 direct sum over all %d sources), "
                                       "extrapolated to targets/s" % (nsamp, T.size, J.size)},
            "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(sph, torch, dev, stream, args, prec, flush=None):
    """24 independent snapshots through eval_sph_batch (autotuned leaf sizes), against the same
    snapshots evaluated one eval_sph call at a time on per-snapshot contexts."""
    import oracle
    probs = si.snapshot_batch(24)
    bps = [sph.BatchProblem.from_problem(p, device=dev) for p in probs]
    ctx = sph.Context(dev.index or 0, stream)
    sph.set_criteria(ctx, 0.0, 0.0, 0.0, 1, 0, prec)
    sph.set_far_field(ctx, sph.FAR_CHEBYSHEV, args.order)
    t0 = time.perf_counter()
    sph.eval_sph_batch(ctx, bps)          # first call: autotuner measurements, operator builds
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(2):
        sph.eval_sph_batch(ctx, bps)
    torch.cuda.synchronize()
    if flush is None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    wall, dev_ms, nt = [], [], 0
    for k in range(max(1, args.batch_steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        _, st = sph.eval_sph_batch(ctx, bps, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        wall.append(time.perf_counter() - t0)
        dev_ms.append(e0.elapsed_time(e1))
        nt = int(st.n_targets)
        launches = int(st.n_launches)
    # the same snapshots one call at a time (each on its own context, leaf sizes fixed to the tuned ones)
    seq_ctx = []
    for p, bp in zip(probs, bps):
        c = sph.Context(dev.index or 0, stream)
        sph.set_grid(c, p.nx, p.ny, p.nz, p.h, p.pO2_torr, p.chi_min, p.chi_max)
        sph.set_sources(c, bp.q, p.source_scale)
        sph.set_targets(c, emag=bp.emag)
        sph.set_criteria(c, p.i_frac, p.e_frac, p.e_applied, 1, 0, prec)
        sph.set_far_field(c, sph.FAR_CHEBYSHEV, args.order)
        seq_ctx.append(c)
    outs = [torch.empty_like(bp.out) for bp in bps]
    leaf = {}
    for i, c in enumerate(seq_ctx):
        _, st1 = sph.eval_sph(c, outs[i], stats=True)
        leaf[probs[i].name] = int(st1.leaf_size)
    torch.cuda.synchronize()
    seq = []
    for k in range(max(1, args.batch_steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, c in enumerate(seq_ctx):
            sph.eval_sph(c, outs[i])
        torch.cuda.synchronize()
        seq.append(time.perf_counter() - t0)
    same = max(float((o - bp.out).norm() / max(bp.out.norm(), 1e-30)) for o, bp in zip(outs, bps))
    # accuracy of the batch on sampled targets of the three smallest snapshots
    rng = np.random.default_rng(3)
    errs = []
    for i in sorted(range(len(probs)), key=lambda i: probs[i].ncell)[:3]:
        p = probs[i]
        J, T = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
        if T.size == 0:
            continue
        samp = np.sort(rng.choice(T, size=min(T.size, 200), replace=False))
        a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
        ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
        S = bps[i].out.cpu().numpy().astype(np.float64)[samp]
        errs.append(oracle.rel_l2(S, ref))
    bw, bd, sq = statistics.median(wall), statistics.median(dev_ms), statistics.median(seq)
    for c in seq_ctx:
        c.close()
    ctx.close()
    stress = run_stress(sph, torch, dev, stream, args, prec, flush)
    return {"workload": "24 streamer snapshots, grids %s, pressures %s Torr, i_frac 1e-5..1e-3, e_frac 0.05..0.2, "
                        "seed 1003" % (sorted({p.nx for p in probs}), sorted({int(p.p_torr) for p in probs})),
            "value": nt / bw, "unit": "targets/s", "ms_per_batch_wall": 1e3 * bw, "ms_per_batch_gpu": bd,
            "n_targets": nt, "gpu_launches": launches, "graph_captured": True,
            "sequential_ms_wall": 1e3 * sq, "speedup_vs_sequential": sq / bw,
            "max_rel_diff_vs_sequential": same, "first_call_s": first_s, "leaf_sizes": leaf,
            "rel_l2_sampled_smallest3": errs, "l2_flush": "256 MiB write before each batch", "stress": stress}


def run_stress(sph, torch, dev, stream, args, prec, flush):
    """The wide-channel batch (channel radius 0.2 .. 1 mm, source threshold 1e-5; about three
    million sources in its last, 256^3 snapshot) in one eval_sph_batch, leaf size and M2L form
    autotuned; accuracy on 200 sampled targets of every snapshot."""
    import oracle
    probs = si.stress_batch(4)
    bps = [sph.BatchProblem.from_problem(p, device=dev) for p in probs]
    ctx = sph.Context(dev.index or 0, stream)
    sph.set_criteria(ctx, 0.0, 0.0, 0.0, 1, 0, prec)
    sph.set_far_field(ctx, sph.FAR_CHEBYSHEV, args.order)
    t0 = time.perf_counter()
    sph.eval_sph_batch(ctx, bps)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    sph.eval_sph_batch(ctx, bps)
    dev_ms = []
    for k in range(3):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = sph.eval_sph_batch(ctx, bps, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
    rng = np.random.default_rng(29)
    snaps = []
    for p, bp in zip(probs, bps):
        J, T = oracle.select(p.q, p.emag, None, p.i_frac, p.e_frac, p.e_applied)
        samp = np.sort(rng.choice(T, size=min(T.size, 200), replace=False))
        a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
        ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
        S = bp.out.cpu().numpy().astype(np.float64)[samp]
        snaps.append({"name": p.name, "n_sources": int(J.size), "n_targets": int(T.size),
                      "rel_l2_sampled": oracle.rel_l2(S, ref), "max_rel_sampled": oracle.max_rel(S, ref, 1e-3)})
    ctx.close()
    md = statistics.median(dev_ms)
    return {"workload": "4 wide-channel snapshots (128^3, 192^3, 256^3, 256^3; channel radius 0.2 .. 1 mm, "
                        "i_frac 1e-5, seed 1006), leaf size and M2L form autotuned",
            "ms_per_batch_gpu": md, "targets_per_s": int(st.n_targets) / (md * 1e-3),
            "n_sources": int(st.n_sources), "n_targets": int(st.n_targets), "first_call_s": first_s,
            "snapshots": snaps}


def run_surrogate(sph, torch, dev, stream, args, peaks):
    """Learned surrogate at 256^3 -> 64^3 in the 1.5 cm cube: training set from the adaptive FMM,
    training by the library's BF16 kernels, then the judged evaluation of the streamer-and-cloud
    configuration against the FMM alone."""
    from paper_2112_10059_gb300 import surrogate as sur
    nf, f = 256, 4
    D = nf // f
    B = 4
    net = sur.Net(edge=D, max_batch=B, seed=11)
    t0 = time.perf_counter()
    X, T = sur.training_set(net, args.sur_samples, nf, f, first=0)
    gen_s = time.perf_counter() - t0
    Xv, Tv = sur.training_set(net, 16, nf, f, first=100000)
    before = sur.validation_loss(net, Xv, Tv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = sur.train(net, X, T, epochs=args.sur_epochs, batch=B, lr=1e-3, lr_final=1e-4, X_val=Xv, T_val=Tv)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    steps = args.sur_epochs * (args.sur_samples // B)
    # one training step and one forward pass timed alone (CUDA events on the network's stream)
    xb, tb = X[:B].reshape(-1), T[:B].reshape(-1)
    for _ in range(3):
        net.backward(xb, tb, B)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        net.backward(xb, tb, B)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 5
    y = net.forward(xb, B)
    e0.record(stream)
    for _ in range(5):
        net.forward(xb, B, y)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 5
    # prediction error on held-out geometries: network vs the coarse estimate alone
    def held_out_errors(nt):
        en, ec = [], []
        for i in range(0, 16, B):
            yy = nt.forward(Xv[i:i + B].reshape(-1), B).cpu().numpy().reshape(B, -1, 2)
            tt = Tv[i:i + B].cpu().numpy().reshape(B, -1)
            en.append(np.abs(np.expm1(yy[..., 0] - tt)))
            ec.append(np.abs(np.expm1(-tt)))
        return np.concatenate(en).ravel(), np.concatenate(ec).ravel()

    def err_stats(e):
        return {"mean": float(e.mean()), "median": float(np.median(e)), "p90": float(np.percentile(e, 90)),
                "frac_below_1e-3": float((e < 1e-3).mean())}

    en, ec = held_out_errors(net)
    # the spread over initial weights: the same training set and schedule from two more seeds
    # (training itself is deterministic: gradients are summed in a fixed order)
    seeds = [{"seed": 11, **err_stats(en)}]
    for sd in (12, 13):
        other = sur.Net(edge=D, max_batch=B, seed=sd)
        sur.train(other, X, T, epochs=args.sur_epochs, batch=B, lr=1e-3, lr_final=1e-4)
        seeds.append({"seed": sd, **err_stats(held_out_errors(other)[0])})
        other.close()
    # the streamer-and-cloud configuration: full FMM vs the judged surrogate
    p = si.streamer_cloud(nf)
    q = torch.from_numpy(p.q).to(dev)
    em = torch.from_numpy(p.emag).to(dev)
    full = sph.Context(dev.index or 0, stream)
    sph.set_grid(full, nf, nf, nf, p.h, p.pO2_torr, p.chi_min, p.chi_max)
    sph.set_sources(full, q, p.source_scale)
    sph.set_targets(full)
    sph.set_criteria(full, p.i_frac, 0.0, 0.0, 1, p.leaf_size, sph.M2L_BF16X3)
    S = torch.empty(nf ** 3, dtype=torch.float32, device=dev)
    pooled = torch.empty(D ** 3, dtype=torch.float32, device=dev)
    for _ in range(3):
        sph.eval_sph(full, S)
        sur.pool_avg(S, nf, f, pooled)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        sph.eval_sph(full, S)
        sur.pool_avg(S, nf, f, pooled)
    e1.record(stream)
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1) / 5
    truth = pooled.cpu().numpy().astype(np.float64)
    ctx = sph.Context(dev.index or 0, stream)
    sph.set_grid(ctx, nf, nf, nf, p.h, p.pO2_torr, p.chi_min, p.chi_max)
    sph.set_sources(ctx, q, p.source_scale)
    sph.set_targets(ctx, emag=em)
    sph.set_criteria(ctx, p.i_frac, 0.0, 0.0, 1, p.leaf_size, sph.M2L_BF16X3)
    judged = []
    for tol in (1e-3, 1e-2):
        for use in (True, False):
            for _ in range(2):
                o, st = sur.evaluate(ctx, net, f, tol=tol, samples=2, seed=7, use_net=use)
            o = o.cpu().numpy().astype(np.float64)
            rel = np.abs(o - truth) / truth
            judged.append({"tol": tol, "network": use, "fallback_blocks": st.n_fallback, "blocks": st.n_blocks,
                           "judged_fail": st.n_judged_fail, "predicted_fail": st.n_predicted_fail,
                           "rel_l2": float(np.linalg.norm(o - truth) / np.linalg.norm(truth)),
                           "max_rel": float(rel.max()), "ms": st.ms_total,
                           "ms_parts": {"coarse": st.ms_coarse, "network": st.ms_net, "judge": st.ms_judge,
                                        "fallback": st.ms_fallback}})
    full.close()
    ctx.close()
    peak = peaks.get("bf16_tflops", 1947.8)
    fl_step = sur.train_flops(D, B)
    fl_fwd = sur.forward_flops(D, B)
    return {"workload": "256^3 streamer + plasma cloud, 1.5 cm, 760 Torr; 4^3 pooling to 64^3; training set "
                        "%d seeded random geometries (FMM solves), %d epochs, batch %d" % (args.sur_samples,
                                                                                         args.sur_epochs, B),
            "params": int(net.P), "generate_s": gen_s, "train_s": train_s, "train_steps": steps,
            "val_loss_before": before, "val_loss_after": hist[-1][2], "train_loss_last": hist[-1][1],
            "pred_err_network": err_stats(en),
            "pred_err_network_seeds": seeds,
            "pred_err_coarse_only": err_stats(ec),
            "train_step_ms": step_ms, "forward_ms": fwd_ms,
            "conv_roofline": {"bound": "tensor", "achieved_train": fl_step / (step_ms * 1e-3) / 1e12,
                              "achieved_forward": fl_fwd / (fwd_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                              "frac_train": fl_step / (step_ms * 1e-3) / 1e12 / peak,
                              "frac_forward": fl_fwd / (fwd_ms * 1e-3) / 1e12 / peak,
                              "work": "2*27*Cin*Cout flop per voxel per convolution (%.1f GF forward, %.1f GF per "
                                      "training step)" % (fl_fwd / 1e9, fl_step / 1e9)},
            "full_fmm_ms": full_ms, "judged": judged}


def run_sweep(sph, torch, dev, stream, args):
    """I_pct trade-off (Eq. sourcepct): a spherical Gaussian (sigma = 8 cells, every cell a
    target) in a 2:2:1 box (128 x 128 x 64) and an elongated box (32 x 32 x 176), at pO2 = 150
    and 10 Torr.  Per I_pct: FMM step time (CUDA events, library timer) and E_V, the relative
    L2 error over 2000 sampled targets against the FP64 sum over every cell."""
    import oracle
    rows = []
    for shape in ((128, 128, 64), (32, 32, 176)):
        for po2 in (150.0, 10.0):
            p = si.gaussian_box(*shape, sigma_cells=8.0, h=1.25e-3, pO2_torr=po2)
            a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
            samp = np.sort(np.random.default_rng(11).choice(p.ncell, 2000, replace=False)).astype(np.int32)
            full = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale,
                              np.arange(p.ncell, dtype=np.int32), samp)
            for f in (0.0, 1e-4, 1e-3, 1e-2, 1e-1):
                p.i_frac = f
                c = sph.Context(dev.index or 0, stream)
                ctx_, out, st = sph.solve(p, c, m2l_precision=sph.M2L_BF16X3, stats=True)
                ms = []
                for _ in range(3):
                    _, st = sph.eval_sph(c, out, stats=True)
                    ms.append(st.ms_total)
                S = out.cpu().numpy().astype(np.float64)[samp]
                rows.append({"box": list(shape), "pO2_torr": po2, "I_pct": f, "n_sources": int(st.n_sources),
                             "ms": statistics.median(ms), "E_V_percent": 100.0 * oracle.rel_l2(S, full)})
                c.close()
    return rows


SIGMA_HEAD = 0.015      # cm: the streamer preset's head width (ball of E_delta: 5 sigma)


def make_ctx(sph, dev, stream, p, q, em, prec, order, leaf=None, env=None):
    """A context set up for problem p on device inputs q / em; ``env`` holds library switches
    read at context creation (set only for that call)."""
    saved = {}
    for k, v in (env or {}).items():
        saved[k] = os.environ.get(k)
        os.environ[k] = v
    try:
        ctx = sph.Context(dev.index or 0, stream)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    sph.set_grid(ctx, p.nx, p.ny, p.nz, p.h, p.pO2_torr, p.chi_min, p.chi_max)
    sph.set_sources(ctx, q, p.source_scale)
    if p.targets_all or em is None:
        sph.set_targets(ctx)
    else:
        sph.set_targets(ctx, emag=em)
    sph.set_criteria(ctx, p.i_frac, p.e_frac, p.e_applied, 1, p.leaf_size if leaf is None else leaf, prec)
    sph.set_far_field(ctx, sph.FAR_CHEBYSHEV, order)
    return ctx


def accuracy_block(p, J, T, S, n_uniform, cpu_seconds_single=3.0):
    """The FP64 oracle on a stratified target sample (every target within 5 sigma of the head
    + n_uniform seeded uniform others), timed on the host's cores; the FMM's errors there.
    Returns (accuracy dict, oracle reference, sample, in_ball, weight, cpu timing dict)."""
    import oracle
    samp, ball, w = si.stratified_targets(p, T, si.streamer_head(), 5 * SIGMA_HEAD, n_uniform, seed=17)
    a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    t0 = time.perf_counter()
    ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # single-thread rate on an evenly spaced part of the sample, about cpu_seconds_single long
    per = dt * cores / max(samp.size, 1)
    m = int(max(8, min(samp.size, cpu_seconds_single / max(per, 1e-9))))
    sub = samp[np.linspace(0, samp.size - 1, m).astype(np.int64)]
    prev = oracle.set_num_threads(1)
    t1 = time.perf_counter()
    oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, sub)
    dt1 = time.perf_counter() - t1
    oracle.set_num_threads(prev)
    cpu = {"value": samp.size / dt, "seconds": dt, "cores": cores, "n": int(samp.size),
           "single_thread_value": sub.size / dt1, "single_thread_n": int(sub.size), "single_thread_s": dt1}
    acc = errors_on_sample(S[samp].astype(np.float64), ref, samp, ball, w, p)
    return acc, ref, samp, ball, w, cpu


def errors_on_sample(got, ref, samp, ball, w, p):
    import oracle
    X = p.origin[0] + p.h * (samp % p.nx + 0.5)
    Y = p.origin[1] + p.h * ((samp // p.nx) % p.ny + 0.5)
    Z = p.origin[2] + p.h * (samp // (p.nx * p.ny) + 0.5)
    pts = np.stack([X, Y, Z], axis=1)
    return {"rel_l2_whole_set_estimate": oracle.rel_l2_weighted(got, ref, np.where(ball, 1.0, w)),
            "rel_l2_sample": oracle.rel_l2(got, ref),
            "rel_l2_ball": oracle.rel_l2(got[ball], ref[ball]),
            "rel_l2_uniform": oracle.rel_l2(got[~ball], ref[~ball]),
            "max_rel": oracle.max_rel(got, ref, 1e-3),
            "e_delta_5sigma": oracle.e_delta(got, ref, pts, si.streamer_head(), 5 * SIGMA_HEAD),
            "n_ball": int(ball.sum()), "n_uniform": int((~ball).sum()), "uniform_weight": w}


def error_decomposition(sph, torch, dev, stream, p, q, em, samp, ball, w, ref, args):
    """The same evaluation with one ingredient changed at a time, errors on the same sample:
    M2L arithmetic (FP32 SIMT vs BF16 x3), deepest level fused or separate, Chebyshev order."""
    variants = [("bf16x3_fused_order5", sph.M2L_BF16X3, 5, {}),
                ("bf16x3_separate_order5", sph.M2L_BF16X3, 5, {"SPH_L2LP_FUSED": "0"}),
                ("f32_order5", sph.M2L_F32, 5, {}),
                ("bf16x3_fused_order4", sph.M2L_BF16X3, 4, {}),
                ("bf16x3_fused_order6", sph.M2L_BF16X3, 6, {}),
                ("f32_order6", sph.M2L_F32, 6, {})]
    out = {}
    for name, prec, order, env in variants:
        c = make_ctx(sph, dev, stream, p, q, em, prec, order, env=env)
        o = torch.empty(p.ncell, dtype=torch.float32, device=dev)
        sph.eval_sph(c, o)
        _, st = sph.eval_sph(c, o, stats=True)
        got = o.cpu().numpy()[samp].astype(np.float64)
        e = errors_on_sample(got, ref, samp, ball, w, p)
        e["ms"] = st.ms_total
        e["fused"] = int(st.l2lp_fused)
        out[name] = e
        c.close()
    return out


def step_times(sph, torch, ctx, out, stream, flush, steps, warmup):
    """Device time of each step (CUDA events on the library's stream, L2 flushed before each)."""
    for _ in range(max(3, warmup)):
        sph.eval_sph(ctx, out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sph.eval_sph(ctx, out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def phase_stats(sph, ctx, out, flush, n):
    res = []
    for k in range(n):
        flush.fill_(float(k))
        _, st = sph.eval_sph(ctx, out, stats=True)
        res.append(st.as_dict())
    return res


def run_full128(sph, torch, dev, stream, args, peaks, pipes, flush):
    """FMM vs direct sum without adaptivity: the 128^3 streamer in a 1 cm cube at 760 Torr with
    every cell a source and a target (2.1 M points, 4.4e12 pairs), leaf size 64, FP32 and BF16 x3
    M2L.  Accuracy over EVERY target against the FP64 FFT convolution of the same discrete sum
    (timed on the host cores), itself checked against the FP64 direct oracle on sampled targets."""
    import oracle
    p = si.streamer_full(128)
    q = torch.from_numpy(p.q).to(dev)
    a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    Jall = np.arange(p.ncell, dtype=np.int32)
    t0 = time.perf_counter()
    fft = oracle.fft_convolution(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, Jall)
    fft_s = time.perf_counter() - t0
    chk = np.sort(np.random.default_rng(23).choice(p.ncell, 256, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    dref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, Jall, chk)
    direct_s = time.perf_counter() - t0
    res = {"workload": "streamer 128^3 in 1 cm, 760 Torr, every cell a source and a target (no adaptivity), "
                       "leaf 64, Chebyshev order %d" % args.order,
           "n_points": p.ncell, "pairs": p.ncell ** 2,
           "fft_oracle": {"seconds": fft_s, "cores": oracle.num_threads(),
                          "rel_l2_vs_direct_oracle_256_targets": oracle.rel_l2(fft[chk], dref),
                          "direct_oracle_targets_per_s": chk.size / direct_s}}
    for name, prec, m2l in (("bf16x3", sph.M2L_BF16X3, "bf16x3"), ("f32", sph.M2L_F32, "f32")):
        ctx = make_ctx(sph, dev, stream, p, q, None, prec, args.order, leaf=64)
        out = torch.empty(p.ncell, dtype=torch.float32, device=dev)
        ms = step_times(sph, torch, ctx, out, stream, flush, max(5, args.steps // 2), 3)
        st = phase_stats(sph, ctx, out, flush, 3)
        S = out.cpu().numpy().astype(np.float64)
        tree = sph.get_tree(ctx)
        sub_args = argparse.Namespace(order=args.order, m2l=m2l)
        roof = rooflines(tree, st, sub_args, p.ncell, p.ncell, p.ncell, peaks, pipes, traffic_ok=False)
        med = statistics.median(ms)
        res[name] = {"ms_per_step": med, "targets_per_s": p.ncell / (med * 1e-3),
                     "rel_l2_all_targets_vs_fft": oracle.rel_l2(S, fft),
                     "max_rel_all_targets_vs_fft": oracle.max_rel(S, fft, 1e-3),
                     "phases_ms": {k: statistics.median(x[k] for x in st)
                                   for k in ("ms_select", "ms_tree", "ms_upward", "ms_m2l", "ms_l2l", "ms_l2p",
                                             "ms_l2lp", "ms_near", "ms_total")},
                     "counts": {k: st[-1][k] for k in ("n_boxes", "n_u", "n_v", "n_w", "n_x", "max_level")},
                     "rooflines": {k: roof[k] for k in ("m2l", "near", "l2lp") if k in roof}}
        if name == "bf16x3" and not args.no_direct:
            d = sph.eval_direct(ctx, fp64=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d = sph.eval_direct(ctx, fp64=False)
            e1.record(stream)
            torch.cuda.synchronize()
            dms = e0.elapsed_time(e1)
            dd = d.cpu().numpy().astype(np.float64)
            res["direct_fp32"] = {"ms": dms, "targets_per_s": p.ncell / (dms * 1e-3),
                                  "pairs_per_s": float(p.ncell) ** 2 / (dms * 1e-3),
                                  "rel_l2_vs_fft": oracle.rel_l2(dd, fft),
                                  "fmm_speedup": dms / med}
        ctx.close()
    return res


def run_pressures(sph, torch, dev, stream, args, flush, pressures=(76.0, 380.0)):
    """The 256^3 adaptive workload at the other pressures of its configuration (Section 4.2):
    step time and the gate on a stratified oracle sample (ball + 20000 uniform targets)."""
    import oracle
    rows = []
    for pt in pressures:
        p = si.streamer_adaptive(n=args.n, p_torr=pt)
        q = torch.from_numpy(p.q).to(dev)
        em = torch.from_numpy(p.emag).to(dev)
        prec = sph.M2L_BF16X3 if args.m2l == "bf16x3" else sph.M2L_F32
        ctx = make_ctx(sph, dev, stream, p, q, em, prec, args.order)
        out = torch.empty(p.ncell, dtype=torch.float32, device=dev)
        ms = step_times(sph, torch, ctx, out, stream, flush, max(5, args.steps // 2), 3)
        _, st = sph.eval_sph(ctx, out, stats=True)
        J, T = sph.get_selection(ctx)
        samp, ball, w = si.stratified_targets(p, T, si.streamer_head(), 5 * SIGMA_HEAD, 20000, seed=19)
        a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
        ref = oracle.sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, samp)
        acc = errors_on_sample(out.cpu().numpy()[samp].astype(np.float64), ref, samp, ball, w, p)
        med = statistics.median(ms)
        rows.append({"pressure_torr": pt, "ms_per_step": med, "targets_per_s": int(st.n_targets) / (med * 1e-3),
                     "n_sources": int(st.n_sources), "n_targets": int(st.n_targets), "accuracy": acc})
        ctx.close()
    return rows


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import __graft_entry__ as g
    g.build()
    import paper_2112_10059_gb300 as sph

    p = workload(args)
    dev = torch.device("cuda", local)
    q = torch.from_numpy(p.q).to(dev)
    em = torch.from_numpy(p.emag).to(dev) if p.emag is not None and not p.targets_all else None
    stream = torch.cuda.current_stream(dev)
    pipes = pipe_peaks(sph, dev, stream)
    prec = sph.M2L_BF16X3 if args.m2l == "bf16x3" else sph.M2L_F32
    ctx = make_ctx(sph, dev, stream, p, q, em, prec, args.order)
    out = torch.empty(p.ncell, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(max(3, args.warmup)):
        sph.eval_sph(ctx, out)
    torch.cuda.synchronize()
    _, st0 = sph.eval_sph(ctx, out, stats=True)
    nt = int(st0.n_targets)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            sph.eval_sph(ctx, out)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # phase breakdown (library CUDA-event timers) from separate steps: the timers add event
    # records and a final synchronisation, which the timed steps above do without.  In the timed
    # steps the near field runs on a second stream beside the far-field passes, so its timer
    # spans the far field too; the per-kernel attribution (phases, rooflines) therefore comes
    # from a context with the near field after the far field, each kernel on the GPU alone
    nph = max(3, min(args.steps, 5))
    step_stats_overlapped = phase_stats(sph, ctx, out, flush, nph)
    ctx_seq = make_ctx(sph, dev, stream, p, q, em, prec, args.order, env={"SPH_NEAR_OVERLAP": "0"})
    for _ in range(2):
        sph.eval_sph(ctx_seq, out)
    step_stats = phase_stats(sph, ctx_seq, out, flush, nph)
    ctx_seq.close()
    torch.cuda.synchronize()
    ms, value = whole_job_rate(statistics.median(step_ms), nt, world, dist, dev)

    # e2e through the host-buffer entry point, inputs and output in pinned host memory
    qh = torch.from_numpy(p.q).pin_memory().numpy()
    eh = torch.from_numpy(p.emag).pin_memory().numpy() if em is not None else None
    sh = torch.empty(p.ncell, dtype=torch.float32).pin_memory().numpy()
    sph.eval_sph_host(ctx, qh, eh, out=sh)
    torch.cuda.synchronize()
    ne2e = max(3, min(args.steps, 5))
    e2e_t = []
    for _ in range(ne2e):
        t0 = time.perf_counter()
        sph.eval_sph_host(ctx, qh, eh, out=sh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms, e2e_value = whole_job_rate(1e3 * statistics.median(e2e_t), nt, world, dist, dev)
    # restore device inputs, and the device result of the last evaluation
    sph.set_sources(ctx, q, p.source_scale)
    if em is not None:
        sph.set_targets(ctx, emag=em)
    else:
        sph.set_targets(ctx)
    sph.eval_sph(ctx, out)
    torch.cuda.synchronize()

    # rooflines of the kernels, from the library's CUDA-event phase timers (medians)
    tree = sph.get_tree(ctx)
    clocks = clk.summary()
    peaks = measured_peaks()
    headline = args.n == 256 and args.p == 760.0 and args.order == 5 and args.workload == "adaptive"
    roof = rooflines(tree, step_stats, args, nt, int(st0.n_sources), p.ncell, peaks, pipes,
                     traffic_ok=headline)
    dominant = dominant_kernel(roof)

    # FP32 direct sum on the same GPU over the same selected sets
    direct = None
    if not args.no_direct:
        d = sph.eval_direct(ctx, fp64=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d = sph.eval_direct(ctx, fp64=False)
        e1.record(stream)
        torch.cuda.synchronize()
        dms = e0.elapsed_time(e1)
        direct = {"targets_per_s": nt / (dms * 1e-3), "ms": dms, "pairs": int(st0.n_sources) * nt,
                  "fmm_speedup": (nt / (ms * 1e-3)) / (nt / (dms * 1e-3))}

    # accuracy against the FP64 oracle on a stratified sample (every target within 5 sigma of the
    # head + seeded uniform targets), the same run timed as the CPU baseline
    J, T = sph.get_selection(ctx)
    S = out.cpu().numpy()
    acc, ref, samp, ball, w, cpu_t = accuracy_block(p, J, T, S, args.acc_uniform,
                                                    3.0 if args.workload == "adaptive" else 1.0)
    if not args.no_decomp:
        acc["decomposition"] = error_decomposition(sph, torch, dev, stream, p, q, em, samp, ball, w, ref, args)
    fft256 = None
    if args.fft256:
        import oracle
        a, b = oracle.alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
        t0 = time.perf_counter()
        full = oracle.fft_convolution(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J)
        fs = time.perf_counter() - t0
        fft256 = {"seconds": fs, "cores": oracle.num_threads(),
                  "rel_l2_all_targets": oracle.rel_l2(S[T].astype(np.float64), full[T]),
                  "max_rel_all_targets": oracle.max_rel(S[T].astype(np.float64), full[T], 1e-3),
                  "fft_vs_direct_oracle_on_sample": oracle.rel_l2(full[samp], ref)}

    full128 = None if args.no_full128 else run_full128(sph, torch, dev, stream, args, peaks, pipes, flush)
    pressures = None if args.no_pressures else run_pressures(sph, torch, dev, stream, args, flush)

    batch = None
    if not args.no_batch:
        batch = run_batch(sph, torch, dev, stream, args, prec, flush)

    sweep = run_sweep(sph, torch, dev, stream, args) if args.sweep else None

    surrogate = None
    if not args.no_surrogate:
        surrogate = run_surrogate(sph, torch, dev, stream, args, measured_peaks())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = {"value": cpu_t["value"], "unit": "targets/s", "cores": cpu_t["cores"], "kind": "oracle",
               "sample": "%d targets of %d -- every target within 5 sigma of the head (%d) + %d seeded uniform "
                         "others -- FP64 direct sum over all %d sources in %.1f s; the same run gives the "
                         "accuracy figures" % (cpu_t["n"], T.size, acc["n_ball"], acc["n_uniform"], J.size,
                                               cpu_t["seconds"]),
               "single_thread": {"value": cpu_t["single_thread_value"], "cores": 1,
                                 "sample": "%d of those targets in %.1f s" % (cpu_t["single_thread_n"],
                                                                             cpu_t["single_thread_s"])}}

    if rank == 0:
        last = step_stats[-1]
        line = {"metric": "S_ph targets/s", "value": value, "unit": "targets/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.m2l == "f32" else "f32+bf16x3",
                "data": "synthetic", "config": workload_cfg(p, args),
                "step_ms_stats": {"median": statistics.median(step_ms), "mean": statistics.mean(step_ms),
                                  "min": min(step_ms), "max": max(step_ms)},
                "e2e": {"value": e2e_value, "unit": "targets/s",
                        "h2d_bytes_per_step": int(qh.nbytes + (eh.nbytes if eh is not None else 0)),
                        "d2h_bytes_per_step": int(sh.nbytes)},
                "roofline": dict(roof[dominant], phase=dominant),
                "rooflines": roof, "pipe_peaks": pipes,
                "clocks": clocks, "gpu_launches": int(step_stats_overlapped[-1]["n_launches"]) * args.steps,
                "phases_overlapped_ms": {k: statistics.median(x[k] for x in step_stats_overlapped)
                                         for k in ("ms_select", "ms_tree", "ms_upward", "ms_m2l", "ms_l2l",
                                                   "ms_l2p", "ms_l2lp", "ms_near", "ms_total")},
                "phases_ms": {k: statistics.median(x[k] for x in step_stats)
                              for k in ("ms_select", "ms_tree", "ms_upward", "ms_vpairs", "ms_m2l", "ms_l2l",
                                        "ms_l2p", "ms_l2lp", "ms_near", "ms_total")},
                "counts": {k: last[k] for k in ("n_sources", "n_targets", "n_boxes", "n_u", "n_v", "n_w", "n_x",
                                                "max_level")},
                "direct_fp32": direct, "accuracy": acc, "fft256": fft256, "full128": full128,
                "pressures": pressures, "batch": batch, "surrogate": surrogate, "sweep": sweep,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

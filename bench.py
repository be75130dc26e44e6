#!/usr/bin/env python3
"""Benchmark of the fused leading-order integrand: one step = one Vegas
iteration of gg -> tt~gg (random numbers -> Vegas map -> x1,x2 -> phase space
-> cuts -> PDFs -> helicity amplitudes -> colour sum -> weight -> Vegas
accumulators -> grid refinement), 4e7 events per iteration, all on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is events/s of the mixed-precision path (f32
amplitudes, f64 kinematics and accumulators) over the whole job; the FP64 path
and the per-event agreement of the two are reported beside it.  With
--impl reference the oracle (CPU, numpy) is timed on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s of gg→tt̄g(g) LO integrand: mixed/batched vs FP64 at ≤1e-5 rel err"
# DRAM bytes per point of the fused integrand kernel, mixed precision:
# dram__bytes_read.sum + dram__bytes_write.sum of a one-pass ncu capture of
# one full-size 4e7-point gg->tt~gg iteration divided by its points (the
# capture's kernel is the one built from this source: vertex routines
# specialised on their couplings' phase)
KERNEL_DRAM_BYTES_PER_POINT = {("gg_ttxgg", "mixed"): (170401024 + 22289582336) / 4e7}
WORKLOAD = "gg_ttxgg"
# FP64 FLOPs per point executed by the gradient kernel (2 x DFMA + DADD +
# DMUL thread instructions of one ncu capture divided by its points)
GRAD_FP64_FLOPS_PER_POINT = {"gg_ttxgg": (2 * 53663185372 + 39529294092 + 38450987098) / 20000}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--events", type=int, default=0, help="events per step (default: the workload's 4e7)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp64-events", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-batch and variant measurements")
    ap.add_argument("--no-channels", action="store_true", help="skip the multichannel phase-space measurement")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_tc"],
                    help="arithmetic of the timed iterations (mixed_tc: colour sum on the tensor cores)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def measured_peaks(device):
    """The device's FP32 (FFMA and packed FFMA2), FP64 (DFMA) and TF32 MMA
    peaks from the library's own microbenchmarks (mf_measure_peak), with the
    SM clocks sampled while they run."""
    from paper_2106_10279_gb300 import api
    out = {}
    for kind in ("fp32_ffma", "fp32_ffma2", "fp64_dfma", "tf32_mma"):
        clk = Clocks(device)
        clk.start()
        tf, ms = api.mf_measure_peak(kind, reps=20)
        c = clk.stop()
        out[kind] = {"tflops": tf, "ms": ms, "sm_mhz": c["sm_mhz"] if c else None,
                     "reasons": c["reasons"] if c else None}
    return out


def cpu_baseline_oracle(wl, n_sample):
    """The oracle as it stands, single-threaded numpy, on n_sample points."""
    import numpy as np
    import workloads as W
    from oracle.integrand import Integrand
    from oracle import vegas
    from oracle.philox import vegas_uniforms
    I = Integrand(wl)
    I.proc.colour_matrix()                      # one-time set-up, not timed
    grid = vegas.uniform_grid(wl.ndim, wl.n_bins)
    t0 = time.perf_counter()
    y = vegas_uniforms(1, 0, 0, 0, n_sample, wl.ndim)
    x, jac, bins = vegas.vegas_map(grid, y)
    w = I(x) * jac
    vegas.accumulate(w, bins, wl.n_bins)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


_ORACLE = {}


def _oracle_worker_init(name):
    # one process per host core, one numpy thread each; the oracle's one-time
    # set-up (colour matrix) happens here, outside the timed work
    import workloads as W
    from oracle.integrand import Integrand
    I = Integrand(W.WORKLOADS[name])
    I.proc.colour_matrix()
    _ORACLE["I"] = I


def _oracle_chunk(args):
    seed, first, n, name = args
    import workloads as W
    from oracle import vegas
    from oracle.philox import vegas_uniforms
    wl = W.WORKLOADS[name]
    grid = vegas.uniform_grid(wl.ndim, wl.n_bins)
    y = vegas_uniforms(seed, 0, 0, first, n, wl.ndim)
    x, jac, bins = vegas.vegas_map(grid, y)
    w = _ORACLE["I"](x) * jac
    vegas.accumulate(w, bins, wl.n_bins)
    return n


def cpu_baseline_oracle_all_cores(wl, n_per_core):
    """The oracle on every host core: one spawned worker process per core
    (one numpy thread each) evaluating its own n_per_core points of the
    same Vegas iteration; events/s over the wall time of the timed map."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(wl.name,)) as pool:
            pool.map(_oracle_chunk, [(1, 10 ** 9 + i * 16, 16, wl.name) for i in range(cores)])   # warm
            jobs = [(1, i * n_per_core, n_per_core, wl.name) for i in range(cores)]
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_chunk, jobs, chunksize=1))
            dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return done / dt, dt, cores, done


def workload_config(wl, n_events, precision, n_diagrams, n_hel, n_jamp):
    """The `config` object of the bench line (shared by both arms)."""
    return {"workload": f"{wl.name}: {' '.join(l.particle for l in wl.legs[:2])} -> "
                        f"{' '.join(l.particle for l in wl.legs[2:])} at 13 TeV, {n_events:.0e} events per Vegas "
                        f"iteration per GPU, {wl.ndim} dims, 50 bins, cuts pT(g)>{wl.pt_min_gluon:g} GeV and "
                        f"dR(g,g)>{wl.dr_min_gluon:g}, synthetic PDF table; f32 amplitudes/colour sum, f64 "
                        f"kinematics and accumulators",
            "precision": precision + (" (colour sum on the tensor cores)" if precision == "mixed_tc" else ""),
            "events_per_step_per_gpu": n_events, "diagrams": n_diagrams, "helicities": n_hel,
            "colour_flows": n_jamp,
            "l2": "random numbers generated in-kernel; per-step outputs (w, bins) "
                  f"{n_events * (8 + wl.ndim) / 1e6:.0f} MB > 129 MB L2"}


def run_reference(args):
    import workloads as W
    from oracle.integrand import Integrand, oracle_process
    rank, world, _ = _dist()
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    sample = 64 if wl.name in ("gg_ttxgg", "gg_ttxggg") else 1000
    # the same workload description as the native arm, structural counts
    # from the oracle's own process
    oproc = oracle_process(wl)
    n_hel = len(Integrand(wl, process=oproc).nonzero_helicities())
    config = workload_config(wl, args.events or wl.n_events, args.precision, len(oproc.diagrams), n_hel,
                             oproc.string_basis().shape[1])
    # the oracle on every host core: one spawned process per core (one numpy
    # thread each, its set-up outside the timed steps); each step evaluates
    # `sample` fresh points per core of the same Vegas iteration
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    times = []
    try:
        with mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=(wl.name,)) as pool:
            for i in range(args.warmup + args.steps):
                first = i * cores * sample
                jobs = [(1, first + c * sample, sample, wl.name) for c in range(cores)]
                t0 = time.perf_counter()
                pool.map(_oracle_chunk, jobs, chunksize=1)
                if i >= args.warmup:
                    times.append(time.perf_counter() - t0)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dt = statistics.median(times)
    value = cores * sample / dt
    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} x {sample} points of one {wl.name} Vegas iteration per step "
                                       f"(Philox, map, integrand, accumulate; numpy), one spawned process per "
                                       f"host core (nproc = {cores}), one numpy thread each"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    import workloads as W
    from paper_2106_10279_gb300 import api

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = W.WORKLOADS[args.workload]
    n_events = args.events or wl.n_events
    proc = api.Process.from_workload(wl)
    info = proc.info
    stream = torch.cuda.current_stream()
    vg = api.Vegas(wl.ndim, wl.n_bins, wl.alpha_vegas)
    seed = 1000
    K = api.mf_vegas_partial_size(vg.handle)

    def step(prec, n, refine=True):
        """One Vegas iteration of n points per GPU.  On one GPU a single call;
        on N GPUs each rank evaluates its whole chunks of the N n points, the
        ranks exchange their partial-sum tree nodes (one all-gather) and every
        rank finishes the iteration to the same bits."""
        if dist is None:
            return api.mf_vegas_iterate([vg.handle], [proc.handle], [n], seed, prec, refine, stream)[0]
        n_total = world * n
        c0, c1 = api.shard_chunks(n_total, rank, world)
        mine = vg.iterate_shard(proc, n_total, c0, c1, seed, 0, prec, stream)
        buf = torch.from_numpy(api.pack_nodes(mine, K)).cuda()
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        return vg.finish_shards(n_total, api.unpack_nodes(torch.stack(parts).cpu().numpy(), K), refine, stream)

    # warm-up (also JIT-compiles the mixed kernel)
    for _ in range(max(args.warmup, 3)):
        step(args.precision, n_events)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    kernel_ms, results = [], []
    start_state = vg.save()          # the e2e leg below replays these same iterations
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        results.append(step(args.precision, n_events))
        kernel_ms.append(api.mf_process_last_kernel_ms(proc.handle))
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * n_events * args.steps / (total_ms / 1e3)

    # FP64 path on a sample of the same iteration
    n64 = args.fp64_events or min(n_events, 2_000_000)
    step("fp64", n64, refine=False)
    torch.cuda.synchronize()
    t64, k64, r64 = [], [], None
    for _ in range(2):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r64 = step("fp64", n64, refine=False)
        b.record(stream)
        torch.cuda.synchronize()
        t64.append(a.elapsed_time(b))
        k64.append(api.mf_process_last_kernel_ms(proc.handle))
    fp64_rate = n64 / (min(t64) / 1e3)
    # the FP64 kernel's achieved FLOP rate (against the measured DFMA peak below)
    fl64 = r64["n_nonzero"] / world * info["flops_helicity_sum"] + n64 * info["flops_kinematics"]
    fp64_tflops = fl64 / (min(k64) / 1e3) / 1e12

    # per-event agreement of the mixed path with the FP64 path
    x = torch.from_numpy(W.uniform_points(wl.ndim, 20000, 77)).cuda()
    f64 = proc.integrand(x, "fp64").cpu().numpy()
    fmx = proc.integrand(x, "mixed").cpu().numpy()
    nz = f64 != 0
    rel = np.abs(fmx[nz] - f64[nz]) / np.abs(f64[nz])

    # end to end through the public API with host buffers, replaying the
    # timed iterations from the same grid state: each step uploads the grid
    # from pinned host memory, runs the iteration and reads the result and
    # the refined grid back
    vg.load(start_state)
    grid_host = torch.from_numpy(vg.grid).pin_memory()
    h2d = grid_host.numel() * 8
    d2h = 7 * 8 + grid_host.numel() * 8
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vg.grid = grid_host.numpy()
        r = step(args.precision, n_events)
        grid_host.copy_(torch.from_numpy(vg.grid))
    barrier()
    t_e2e = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e_value = world * n_events * args.steps / t_e2e

    # variants of the same kernel on a sample of the workload, each over 5
    # seeds of 2e6 points on the adapted grid: the colour sum on the tensor
    # cores, and the Monte Carlo estimators over helicities (one helicity or
    # helicity pair per point), over colour (one colour flow per point) and
    # over both: different unbiased estimators with more variance, compared
    # by efficiency = 1 / (error^2 x kernel time) relative to the full sum
    variants = {}
    if not args.no_batch:
        nv = min(n_events, 2_000_000)
        gv = api.Vegas(wl.ndim, wl.n_bins, wl.alpha_vegas)
        gv.load(start_state)
        estimators = (("mixed", "mixed", 0, False), ("mixed_tc", "mixed_tc", 0, False),
                      ("mixed_helicity_sampling", "mixed", 1, False),
                      ("mixed_helicity_pair_sampling", "mixed", 2, False),
                      ("mixed_colour_sampling", "mixed", 0, True),
                      ("mixed_colour_and_pair_sampling", "mixed", 2, True))
        for tag, prec, sample, colour in estimators:
            proc.set_helicity_sampling(sample, seed=5)
            proc.set_colour_sampling(colour)
            api.mf_vegas_iterate([gv.handle], [proc.handle], [nv], seed, prec, False, stream)
            torch.cuda.synchronize()
            kms_s, err_s, int_s = [], [], []
            for s_ in range(5):
                r = api.mf_vegas_iterate([gv.handle], [proc.handle], [nv], seed + 101 + s_, prec, False, stream)[0]
                kms_s.append(api.mf_process_last_kernel_ms(proc.handle))
                err_s.append(r["error"])
                int_s.append(r["integral"])
            variants[tag] = {"events": nv, "seeds": 5, "kernel_ms": statistics.median(kms_s),
                             "events_per_s": nv / (statistics.median(kms_s) / 1e3),
                             "integral_pb": statistics.mean(int_s),
                             "error_pb_rms": math.sqrt(statistics.mean([e * e for e in err_s])),
                             "launch": proc.kernel_info(prec)}
        proc.set_helicity_sampling(False)
        proc.set_colour_sampling(False)
        ref = variants["mixed"]
        for v_ in variants.values():
            v_["efficiency_vs_full"] = (ref["error_pb_rms"] ** 2 * ref["kernel_ms"]) / (v_["error_pb_rms"] ** 2
                                                                                        * v_["kernel_ms"])

    # the multichannel phase space against the flat one on the same
    # workload: equal points per iteration, five adapting iterations each
    # (the grids, and the channels' Neyman allocation), then five seeds
    # without adaptation: the error and the device time of the whole
    # iteration (every channel's launches and accumulation); efficiency =
    # 1 / (error^2 x time) relative to the flat phase space
    phase_space = None
    if not args.no_channels and proc.n_channels > 0 and rank == 0:
        nps = min(n_events, 2_000_000)

        def timed_iter(fn):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            r = fn()
            b.record(stream)
            torch.cuda.synchronize()
            return r, a.elapsed_time(b)
        gf = api.Vegas(wl.ndim, wl.n_bins, wl.alpha_vegas)
        mc = api.MultiChannel(proc, wl.n_bins, wl.alpha_vegas)
        for it in range(5):
            gf.iterate(proc, nps, seed + 500 + it, "mixed", True, stream)
            mc.iterate(nps, seed + 500 + it, "mixed", True, True, stream=stream)
        legs = {"flat": ([], [], []), "multichannel": ([], [], [])}
        for s_ in range(5):
            r, ms = timed_iter(lambda: gf.iterate(proc, nps, seed + 600 + s_, "mixed", False, stream))
            for lst, v_ in zip(legs["flat"], (ms, r["error"], r["integral"])):
                lst.append(v_)
            r, ms = timed_iter(lambda: mc.iterate(nps, seed + 600 + s_, "mixed", False, False, stream=stream))
            for lst, v_ in zip(legs["multichannel"], (ms, r["error"], r["integral"])):
                lst.append(v_)
        phase_space = {"events_per_iteration": nps, "adapt_iterations": 5, "seeds": 5, "channels": proc.n_channels,
                       "regulators_gev2": (4.0 * max(wl.pt_min_gluon, 1.0)) ** 2}
        for tag, (ms_l, err_l, int_l) in legs.items():
            phase_space[tag] = {"iteration_ms": statistics.median(ms_l),
                                "events_per_s": nps / (statistics.median(ms_l) / 1e3),
                                "error_pb_rms": math.sqrt(statistics.mean([e * e for e in err_l])),
                                "integral_pb": statistics.mean(int_l)}
        f_, m_ = phase_space["flat"], phase_space["multichannel"]
        phase_space["efficiency_vs_flat"] = (f_["error_pb_rms"] ** 2 * f_["iteration_ms"]) / (
            m_["error_pb_rms"] ** 2 * m_["iteration_ms"])
        phase_space["allocation_min_max"] = [min(mc.allocation(nps)), max(mc.allocation(nps))]
        # unweighting efficiency <W> / max W of one iteration's event weights
        # (the paper puts the flat phase space's at about 5 %, Sec. 2.5); a
        # channel-k point weighs W = w N / n_k in the combined sample
        gf.iterate(proc, nps, seed + 700, "mixed", False, stream)
        wf = api.read_weights(proc, np.arange(nps))
        rm = mc.iterate(nps, seed + 700, "mixed", False, False, stream=stream)
        alloc = rm["allocation"]
        wm = api.read_weights(proc, np.arange(sum(alloc))) * np.repeat([sum(alloc) / k for k in alloc], alloc)
        phase_space["flat"]["unweighting_efficiency"] = float(wf.mean() / np.abs(wf).max())
        phase_space["multichannel"]["unweighting_efficiency"] = float(wm.mean() / np.abs(wm).max())
        mc.close()

    # the mixed batch of five subprocesses (gg->tt~, uu~->tt~, gg->tt~g,
    # uu~->tt~g, gg->tt~gg; 4e7 points per iteration in all), each with its own
    # grid: one persistent launch per iteration against one launch per
    # subprocess, same points and results
    batch = None
    if not args.no_batch:
        names = [name for name, _ in W.MIXED_BATCH]
        nb_ev = [nev for _, nev in W.MIXED_BATCH]
        procs = [proc if name == wl.name else api.Process.from_workload(W.WORKLOADS[name]) for name in names]
        bt = api.Batch(procs, "mixed")

        def timed(run, reps=3):
            for _ in range(2):
                run()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                out = run()
            b.record(stream)
            torch.cuda.synchronize()
            return sum(nb_ev) * reps / (a.elapsed_time(b) / 1e3), out
        gb = [api.Vegas(p.ndim) for p in procs]
        rate_b, res_b = timed(lambda: bt.iterate(gb, nb_ev, 4242, True, stream))
        gs = [api.Vegas(p.ndim) for p in procs]
        rate_s, res_s = timed(lambda: api.mf_vegas_iterate([g.handle for g in gs], [p.handle for p in procs],
                                                           nb_ev, 4242, "mixed", True, stream))
        # the same batch as one CUDA-graph replay per iteration
        gg_ = [api.Vegas(p.ndim) for p in procs]
        rate_g, res_g = timed(lambda: bt.iterate(gg_, nb_ev, 4242, True, stream, graph=True))
        # the four short programs as one batch (their own register budget)
        # and gg -> tt~gg on its own
        heavy = [i for i, (name, _) in enumerate(W.MIXED_BATCH) if name == "gg_ttxgg"]
        light = [i for i in range(len(procs)) if i not in heavy]
        bt_l = api.Batch([procs[i] for i in light], "mixed")
        gl = [api.Vegas(procs[i].ndim) for i in light]
        gh = [api.Vegas(procs[i].ndim) for i in heavy]

        def split():
            a_ = bt_l.iterate(gl, [nb_ev[i] for i in light], 4242, True, stream)
            b_ = api.mf_vegas_iterate([g.handle for g in gh], [procs[i].handle for i in heavy],
                                      [nb_ev[i] for i in heavy], 4242, "mixed", True, stream)
            return a_ + b_
        rate_split, _ = timed(split)
        # the same five subprocesses at 1/1000 of the points (an iteration of
        # 4e4 points: latency-bound, where one launch and one graph replay
        # per iteration count)
        small = [max(1024, e // 1000) for e in nb_ev]
        gs_s = [api.Vegas(p.ndim) for p in procs]
        gb_s = [api.Vegas(p.ndim) for p in procs]
        gg_s = [api.Vegas(p.ndim) for p in procs]

        def timed_small(run, reps=20):
            for _ in range(3):
                run()
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            for _ in range(reps):
                run()
            torch.cuda.synchronize()
            return sum(small) * reps / (time.perf_counter() - t0_)
        small_rates = {
            "separate_launches": timed_small(lambda: api.mf_vegas_iterate([g.handle for g in gs_s],
                                                                          [p.handle for p in procs], small, 4343,
                                                                          "mixed", True, stream)),
            "batch": timed_small(lambda: bt.iterate(gb_s, small, 4343, True, stream)),
            "graph_replay": timed_small(lambda: bt.iterate(gg_s, small, 4343, True, stream, graph=True))}
        batch = {"workload": "mixed batch " + ", ".join(f"{n} {e:.0e}" for n, e in W.MIXED_BATCH),
                 "value": rate_b, "unit": "events/s", "separate_launches": rate_s, "graph_replay": rate_g,
                 "light_batch_plus_heavy_alone": rate_split,
                 "sigma_total_pb": sum(r["sigma"] for r in res_b),
                 "same_sigma_as_separate": all(a["sigma"] == b["sigma"] for a, b in zip(res_b, res_s)),
                 "same_sigma_graph": all(a["sigma"] == b["sigma"] for a, b in zip(res_b, res_g)),
                 "kernel_ms": bt.info()["last_kernel_ms"], "registers": bt.info().get("regs"),
                 "light_batch_registers": bt_l.info().get("regs"),
                 "small_iterations": {"points": small, "unit": "events/s (host wall clock, synchronous calls)",
                                      **small_rates}}

    # the gradient kernel (mf_grad: f, df/dm_t, df/dalpha_s, df/dx in FP64) on
    # uniform points of the same process: points/s and, from the FP64
    # arithmetic ncu counted per point of that kernel, its FP64 rate
    grad = None
    if not args.no_batch:
        ng = min(n_events, 200_000)
        xg = torch.from_numpy(W.uniform_points(wl.ndim, ng, 91)).cuda()
        proc.grad(xg[:, :1024].contiguous(), stream=stream)     # compiles the gradient kernel
        torch.cuda.synchronize()
        gts, out = [], None
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = proc.grad(xg, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            gts.append(a.elapsed_time(b))
        gms = min(gts)
        fg, dpg, _ = out
        grad = {"events": ng, "ms": gms, "events_per_s": ng / (gms / 1e3),
                "dsigma_dmt_pb_per_gev_pathwise": float(dpg[0].mean()),
                "dsigma_dalphas_pb": float(dpg[1].mean()), "sigma_pb": float(fg.mean())}
        fl = GRAD_FP64_FLOPS_PER_POINT.get(wl.name)
        if fl:
            grad["roofline"] = {"bound": "alu", "achieved": fl * ng / (gms / 1e3) / 1e12, "unit": "TFLOP/s",
                                "flops_per_point": fl, "flops_source": "executed FP64 FMA x2 + add + mul per point "
                                                                      "of mf_grad_kernel (ncu counters)"}

    # roofline of the dominant kernel: algorithmic FLOPs / its device time
    kms = statistics.median(kernel_ms)
    # (an iteration's counts cover all ranks; the kernel timed is this rank's)
    passing = statistics.median([r["n_nonzero"] for r in results]) / world
    info = proc.info                   # FLOP counts of the program as compiled
    # (the helicity sum as evaluated: a helicity pair computes the
    # wavefunctions that do not depend on its pair leg once)
    flops = passing * info["flops_helicity_sum"] + n_events * info["flops_kinematics"]
    achieved = flops / (kms / 1e3) / 1e12
    # the roofline denominators, measured here by the library's own
    # microbenchmarks (FP32: the faster of scalar and packed-pair FMAs)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    mp = measured_peaks(local)
    fp32_kind = max(("fp32_ffma", "fp32_ffma2"), key=lambda k: mp[k]["tflops"])
    fp32_peak = mp[fp32_kind]["tflops"]
    fp64_peak = mp["fp64_dfma"]["tflops"]
    if grad and "roofline" in grad:
        grad["roofline"].update(peak=fp64_peak, frac=grad["roofline"]["achieved"] / fp64_peak,
                                peak_source="measured: mf_measure_peak fp64_dfma")

    cpu = cpu1 = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = 2000 if wl.name == "gg_ttxgg" else 20000
        rate, dt = cpu_baseline_oracle(wl, sample)
        cpu1 = {"value": rate, "unit": "events/s", "cores": 1, "kind": "oracle",
                "sample": f"{sample} points of one {wl.name} Vegas iteration (Philox, map, integrand, "
                          f"accumulate), {dt:.1f} s"}
        per_core = max(100, int(rate * 12))          # about 12 s of work per core
        rate_all, dt_all, cores, done = cpu_baseline_oracle_all_cores(wl, per_core)
        cpu = {"value": rate_all, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} points of one {wl.name} Vegas iteration (Philox, map, integrand, accumulate) "
                         f"split over {cores} spawned processes, one per host core (nproc = {cores}), "
                         f"one numpy thread each, {dt_all:.1f} s wall"}
    launches_per_step = 5          # integrand, accumulate, tree reduction, finalize, refine
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "parallelism": "one Vegas iteration of N x events_per_step_per_gpu points split in whole 4096-point "
                       "chunks; one all-gather of partial-sum tree nodes per iteration" if world > 1 else "1 GPU",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(wl, n_events, args.precision, proc.n_diagrams, info["n_hel"], info["n_jamp"]),
        "fp64": {"value": fp64_rate, "unit": "events/s", "events": n64,
                 "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": fp64_tflops / fp64_peak,
                              "peak_source": "measured: mf_measure_peak fp64_dfma (DFMA chains, all SMs)"}},
        "peaks": {"sms": n_sm, "measured": mp},
        "batch": batch,
        "grad": grad,
        "kernel_variants": variants,
        "phase_space": phase_space,
        "accuracy": {"median_rel_mixed_vs_fp64": float(np.median(rel)), "max_rel_mixed_vs_fp64": float(rel.max()),
                     "points": int(nz.sum())},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": (KERNEL_DRAM_BYTES_PER_POINT[(wl.name, args.precision)] * n_events
                                 if (wl.name, args.precision) in KERNEL_DRAM_BYTES_PER_POINT else None),
                     "traffic_note": "bytes per launch from a one-pass ncu capture of a full-size launch, "
                                     "scaled by points; mostly write-back of register spills; "
                                     f"algorithmic output {n_events * (8 + wl.ndim) / 1e6:.0f} MB; "
                                     "DRAM is not the bound (see traffic_gbs against the HBM peak)",
                     "traffic_gbs": (KERNEL_DRAM_BYTES_PER_POINT[(wl.name, args.precision)] * n_events / (kms / 1e3)
                                     / 1e9 if (wl.name, args.precision) in KERNEL_DRAM_BYTES_PER_POINT else None),
                     "hbm_peak_gbs": _peaks().get("hbm_gbs"),
                     "kernel": "mf_kernel (fused integrand)", "kernel_ms": kms,
                     "flops_per_passing_point": info["flops_helicity_sum"], "helicity_pairs": info["n_pairs"],
                     "peak_source": f"measured: mf_measure_peak {fp32_kind} ({n_sm} SMs, FMA chains, "
                                    f"{mp[fp32_kind]['sm_mhz']} MHz median SM clock)"},
        "cpu_baseline": cpu,
        "cpu_baseline_single_thread": cpu1,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "sigma_pb": results[-1]["sigma"], "sigma_err_pb": results[-1]["sigma_error"],
        "accepted_events_per_s": value * statistics.median([r["n_nonzero"] for r in results]) / (world * n_events),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the pulse-profile likelihood on GB300.

One step = one full likelihood evaluation (ring templates, shift-and-add with
atmosphere interpolation, ISM, response contraction, Poisson logL) of the
workload's parameter vectors.  Default workload: two hotspots (cap + ring)
x 128x128 elements, 128 phases, 256 energies, 300 channels, synthetic
35x11x67x166 atmosphere table, oblate Schwarzschild, one parameter vector.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank evaluates
its own copies of the workload (replicas, weak scaling; no collective on the
data path).  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PPM likelihood evals/s (ms/eval) at 1e-3 rel. accuracy; batched & grad evals/s"
FLOP_PER_TRIPLE = 14          # algorithmic FP32 flops per (element, phase, energy) triple
# backward shift-and-add: five interval cubics per triple (I, dI/dt, dI/dmu and the
# two cell-weight derivatives), each Horner + accumulate, plus the amortised mu
# contraction of four stencils: 18 FMA + 4 x 4 FMA x 0.48 nodes per energy
FLOP_PER_TRIPLE_BWD = 50
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_shift_add_atm_two_spot.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2510_07764_gb300", "csrc", "shift_add.cu")
REF_RING_STRIDE = 64
CPU_RING_STRIDE = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # defaults: 10 warm-up and 200 timed single-evaluation steps (about 0.2 s
    # timed on the two-spot workload, so that the clock sampler sees the
    # region); 5 and 50 for the CPU reference arm; 3 and 3 for the
    # multi-second batch workloads
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="atm_two_spot",
                    choices=["atm_two_spot", "bb_small", "crescent_extreme", "batch", "grad_batch",
                             "healpix_map"])
    ap.add_argument("--interp", choices=["d", "a", "b", "c"], default=None,
                    help="atmosphere interpolation strategy of Sect. 4 (default: the method's, d)")
    ap.add_argument("--phase-sub", type=int, default=None,
                    help="point samples per output phase bin (ppm_res.phase_sub)")
    ap.add_argument("--batch", type=int, default=None,
                    help="parameter vectors of the batch / grad_batch workloads")
    ap.add_argument("--flush-mib", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action="store_true",
                    help="capture one step in a CUDA graph and time its replays")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the shift-and-add tiles with ppm_autotune before timing")
    ap.add_argument("--walk", type=int, choices=[0, 1], default=0,
                    help="energy walk of the atmosphere shift-and-add: 0 node-major where "
                         "the energy grid allows it, 1 energy walk (ppm_tiles.walk)")
    return ap.parse_args()


def make_workload(args, rank: int = 0):
    """The workload of one rank.  Batched workloads draw their own parameter
    vectors per rank (seed offset by the rank: weak scaling over independent
    instances); single-instance workloads are replicas."""
    from paper_2510_07764_gb300 import synth
    if args.workload in ("batch", "grad_batch"):
        kw = {"seed": synth.SEED + (1 if args.workload == "grad_batch" else 0) + rank}
        if args.batch is not None:
            kw["B"] = args.batch
        w = synth.WORKLOADS[args.workload](**kw)
    else:
        w = synth.WORKLOADS[args.workload]()
    if getattr(args, "interp", None):
        w.interp = args.interp
    if getattr(args, "phase_sub", None):
        w.inst.phase_sub = int(args.phase_sub)
    return w


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (the job's
    time is its slowest rank's); identity without torch.distributed."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def workload_desc(w):
    inst = w.inst
    return {
        "workload": w.name,
        "B": int(inst.B),
        "spots": int(inst.n_spots),
        "elements_per_spot": ("%d pixels" % (12 * int(inst.n_theta[0]) ** 2) if inst.grid == 1
                              else "%dx%d" % (int(inst.n_theta[0]), int(inst.n_phi[0]))),
        "phases": int(inst.n_phase[0]),
        "energies": int(len(w.E_keV)),
        "channels": int(w.nc),
        "n_fp": int(inst.n_fp),
        "spacetime": "oblate Schwarzschild" if inst.oblate else "Schwarzschild+Doppler",
        "emission": "atmosphere table 35x11x67x166" if inst.emission else "analytic blackbody",
        "interp": getattr(w, "interp", "d"),
        "phase_sub": int(inst.phase_sub),
        "grid": ("HEALPix N_side %d, temperature map" % int(inst.n_theta[0])
                 if inst.grid == 1 else "spot-bounding"),
    }


class Clocks:
    """nvidia-smi sampling of the SM clock and the throttle reasons.  Sampling
    is live (its first sample has arrived) before the timed region starts;
    only the samples time-stamped inside the region [t0, t1] are reported."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", "ppm_clocks_%d.csv" % os.getpid())

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
               "-lms", str(self.PERIOD_MS)]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 10.0
        while time.time() < deadline and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    @staticmethod
    def _stamp(text):
        from datetime import datetime
        try:
            return datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            rows.append((self._stamp(parts[0]), sm, smax,
                         {n for n, v in zip(names, parts[6:10]) if v.lower().startswith("active")}))
        os.unlink(self.path)
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        used = inside if inside else rows
        return {"sm_mhz": statistics.median(r[1] for r in used) if used else None,
                "sm_max_mhz": max(r[2] for r in used) if used else None,
                "samples": len(inside), "sample_ms": self.PERIOD_MS,
                "window": "timed region" if inside else "whole run (no sample inside)",
                "reasons": sorted(set().union(*[r[3] for r in used])) if used else []}


def forward_kernel_name(w):
    """The shift-and-add kernel that dominates a forward evaluation of w."""
    if not w.inst.emission:
        return "k_shift_add<blackbody>"
    if getattr(w.inst, "logT_map", None) is not None:
        return "k_shift_add_map<atmosphere>"
    return "k_shift_add<atmosphere>"


def profiled_config(args):
    """Whether this run launches the kernel configuration of the committed ncu
    summary (the default two-spot workload, default interpolation, point
    phases, node-major walk and default tiles), whose DRAM bytes per launch
    may then be reported as this run's traffic."""
    return (args.workload == "atm_two_spot" and args.interp in (None, "d")
            and args.phase_sub in (None, 1) and not args.walk and not args.autotune)


def profile_traffic():
    """dram bytes per launch of the shift-and-add kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    txt = open(PROFILE_SUMMARY).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not (m and t):
        return None
    sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    return float(t.group(1)) if m.group(1) == sha else None


def _work(inst, b, nE):
    return float(inst.n_spots) * inst.n_theta[b] * inst.n_phi[b] * inst.n_phase[b] * nE


def _rings(inst, b):
    """Rings per spot in the oracle's loop (4 N_side - 1 on the HEALPix mesh)."""
    n = int(inst.n_theta[b])
    return 4 * n - 1 if getattr(inst, "grid", 0) == 1 else n


def sample_factor(inst, stride, nE):
    """Work of the whole workload over the work of instance 0's sample
    (every stride-th ring, ring 0 first)."""
    total = sum(_work(inst, b, nE) for b in range(inst.B))
    R = _rings(inst, 0)
    return total / _work(inst, 0, nE) * R / math.ceil(R / stride)


def oracle_sample(w, stride):
    """Time the FP64 oracle on instance 0, every `stride`-th ring (profile,
    response and logL); returns (seconds, extrapolation factor to the whole
    workload by element x phase x energy work)."""
    import numpy as np
    import oracle
    oracle.build()
    oracle.lens(w.lens)   # table build is not part of an evaluation
    w0 = w if w.inst.B == 1 else _single(w, 0)
    t0 = time.perf_counter()
    Ft = oracle.profile(w0, ring_stride=stride)
    if w.R is not None:
        C = oracle.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
        oracle.loglike(C, w0.counts, w.tau)
    dt = time.perf_counter() - t0
    return dt, sample_factor(w.inst, stride, len(w.E_keV))


def _single(w, b):
    from paper_2510_07764_gb300 import synth
    inst = w.inst.select(b)
    r0 = int(sum(w.inst.n_phase[:b]))
    return synth.Workload(w.name, inst, w.lens, w.E_keV, atm=w.atm, R=w.R,
                          sigma_ism=w.sigma_ism,
                          counts=w.counts[r0:r0 + int(inst.n_phase[0])], tau=w.tau)


_W = None


def _oracle_pool_init(w):
    """Worker set-up (not timed): the workload, the oracle and its lens table."""
    global _W
    import oracle
    oracle.build()
    oracle.lens(w.lens)
    _W = w


def _oracle_phase_chunk(job):
    import oracle
    jsel, stride = job
    return oracle.profile(_W, jsel=jsel, ring_stride=stride)


def oracle_sample_parallel(w, stride, workers):
    """The same bounded sample as oracle_sample on `workers` processes, split
    by output phase (spawned pool: no GPU state is forked); returns the wall
    time of the profile + response + logL and the extrapolation factor."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    w0 = w if w.inst.B == 1 else _single(w, 0)
    n = int(w0.inst.n_phase[0])
    chunks = [c for c in np.array_split(np.arange(n, dtype=np.int32), workers) if len(c)]
    with mp.get_context("spawn").Pool(len(chunks), initializer=_oracle_pool_init,
                                      initargs=(w0,)) as pool:
        pool.map(_oracle_phase_chunk, [(c[:1], stride) for c in chunks])  # warm
        t0 = time.perf_counter()
        parts = pool.map(_oracle_phase_chunk, [(c, stride) for c in chunks])
        Ft = np.concatenate(parts, axis=0)
        if w.R is not None:
            C = oracle.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
            oracle.loglike(C, w0.counts, w.tau)
        dt = time.perf_counter() - t0
    return dt, sample_factor(w.inst, stride, len(w.E_keV))


def fd_evals(w):
    """Oracle evaluations per gradient by central differences (logL + 2 per parameter)."""
    return 1 + 2 * (5 + 4 * int(w.inst.n_spots))


def cpu_baseline(w, grad_mode=False):
    """The FP64 oracle (single thread) on a bounded sample, extrapolated; for
    gradients, the cost of central differences with the oracle."""
    dt, factor = oracle_sample(w, CPU_RING_STRIDE)
    per_eval = dt * factor / w.inst.B
    mult = fd_evals(w) if grad_mode else 1
    unit = "grad-evals/s" if grad_mode else ("evals/s" if w.R is not None else "profile evals/s")
    cores = os.cpu_count() or 1
    all_core = None
    if cores > 1:
        try:
            dtp, fp = oracle_sample_parallel(w, CPU_RING_STRIDE, cores)
            all_core = {"value": 1.0 / (dtp * fp / w.inst.B * mult), "cores": cores,
                        "measured_s": round(dtp, 3)}
        except Exception as exc:  # the single-thread figure stands alone
            all_core = {"value": None, "cores": cores, "error": str(exc)[:200]}
    best = all_core["value"] if all_core and all_core.get("value") else 1.0 / (per_eval * mult)
    return {"value": best, "unit": unit,
            "cores": all_core["cores"] if all_core and all_core.get("value") else 1,
            "kind": "oracle",
            "single_thread": {"value": 1.0 / (per_eval * mult), "cores": 1,
                              "measured_s": round(dt, 3)},
            "all_core": all_core,
            "sample": "instance 0, every %dth ring, all phases x energies, response and logL; "
                      "single thread %.1f s measured, extrapolated x%.4g by element x phase x "
                      "energy work; all-core: the same sample split by output phase over a "
                      "process pool%s"
                      % (CPU_RING_STRIDE, dt, factor,
                         "; x%d evaluations per central-difference gradient" % mult
                         if grad_mode else "")}


REF_BUDGET_S = 120.0


def reference_stride(first_s, stride, n_steps, budget_s=REF_BUDGET_S, max_stride=1 << 30):
    """Ring stride of the reference arm's per-step sample: the stride of the
    first step, widened in proportion when n_steps samples of that size
    would exceed the budget (the sample's cost scales as 1 / stride), and at
    most the number of rings of a spot."""
    if n_steps * first_s <= budget_s:
        return stride
    return int(min(max_stride, math.ceil(stride * n_steps * first_s / budget_s)))


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2510_07764_gb300 import synth
    import oracle
    w = make_workload(args)
    grad_mode = args.workload == "grad_batch"
    mult = fd_evals(w) if grad_mode else 1
    times = []
    stride = REF_RING_STRIDE
    for k in range(args.warmup + args.steps):
        dt, factor = oracle_sample(w, stride)
        if k == 0:
            # widen the sample stride so that the whole run stays near the budget
            stride = reference_stride(dt, stride, args.warmup + args.steps,
                                      max_stride=max(1, int(w.inst.n_theta[0])))
        if k >= args.warmup:
            times.append(dt * factor * mult)
    if not times:
        times.append(dt * factor * mult)
    per_step = sum(times) / len(times)
    value = w.inst.B / per_step
    per_eval = per_step / w.inst.B
    sample = ("instance 0, every %dth ring per step, extrapolated by element x phase x energy "
              "work to the whole workload" % stride)
    unit = "evals/s" if w.R is not None else "profile evals/s"
    if grad_mode:
        sample += "; x%d evaluations per central-difference gradient" % mult
        unit = "grad-evals/s"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_eval * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(w),
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = make_workload(args, rank)
    grad_mode = args.workload == "grad_batch"
    ctx = ppm.Context(local_rank)
    t0 = time.perf_counter()
    ctx.setup(w)
    setup_s = time.perf_counter() - t0
    dp = ppm.DeviceParams(w.inst, device=dev)
    B = dp.B
    # workloads without a response (the small blackbody one) time the
    # forward profile alone; its result F_t is what the end-to-end leg reads
    profile_mode = w.R is None
    counts = None if profile_mode else torch.from_numpy(w.counts).to(dev)
    Ft = torch.empty((dp.rows, len(w.E_keV)), dtype=torch.float32, device=dev)
    logL = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty((B, ppm.N_GRAD), dtype=torch.float64, device=dev)
    flush = torch.empty(args.flush_mib * (1 << 20) // 4, dtype=torch.float32, device=dev)
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()

    def step(stream=None):
        if profile_mode:
            ctx.profile(dp, out=Ft, stream=stream)
        elif grad_mode:
            ctx.loglike_grad(dp, counts, w.tau, out=logL, grad=grad, stream=stream)
        else:
            ctx.loglike(dp, counts, w.tau, out=logL, stream=stream)

    tuned = None
    if args.walk:
        ctx.set_tiles(walk=args.walk)
    if args.autotune:
        tuned = ctx.autotune(dp)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = None
    if args.graph:
        # one step captured once; replays re-read parameters and counts from
        # the same device buffers (the plan and workspace are settled above)
        s_cap = torch.cuda.Stream()
        s_cap.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s_cap):
            step(s_cap)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM; L2 flushed before each)
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id)
    clocks.start()
    ctx.set_timing(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record()
        if graph is not None:
            graph.replay()
        else:
            step()
        evs[k][1].record()
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    clk = clocks.stop(t0, t1)
    if graph is not None:
        # graph replays record no stage events: three direct calls for the breakdown
        for _ in range(3):
            step()
        torch.cuda.synchronize()
    timing = ctx.get_timing()
    ctx.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_ms = sum(step_ms)
    n_bad = 0 if profile_mode else int((~np.isfinite(logL.cpu().numpy())).sum())
    fwd_ms = None
    if grad_mode:
        # the forward alone on the same inputs, for the backward / forward ratio
        evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            evf[k][0].record()
            ctx.loglike(dp, counts, w.tau, out=logL)
            evf[k][1].record()
        torch.cuda.synchronize()
        fwd_ms = sum(a.elapsed_time(b) for a, b in evf)

    # ---- end to end through host buffers (params + counts in, logL out)
    pin = {f: torch.from_numpy(np.ascontiguousarray(getattr(w.inst, f), dtype=np.float64)
                               .reshape(-1)).pin_memory() for f in ppm._abi.PARAM_FIELDS}
    host_inst = w.inst.replace()
    for f, t in pin.items():
        setattr(host_inst, f, t)
    counts_pin = None if profile_mode else torch.from_numpy(w.counts).pin_memory()
    out_pin = torch.empty(B, dtype=torch.float64).pin_memory()
    grad_pin = torch.empty((B, ppm.N_GRAD), dtype=torch.float64).pin_memory()
    ft_pin = torch.empty(tuple(Ft.shape), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 8 for t in pin.values()) + (0 if profile_mode else counts_pin.numel() * 4)
    d2h = Ft.numel() * 4 if profile_mode else B * 8 * (1 + (ppm.N_GRAD if grad_mode else 0))
    evs2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs2[k][0].record()
        dp.upload(host_inst, non_blocking=True)
        if not profile_mode:
            counts.copy_(counts_pin, non_blocking=True)
        if graph is not None:
            graph.replay()
        else:
            step()
        if profile_mode:
            ft_pin.copy_(Ft, non_blocking=True)
        else:
            out_pin.copy_(logL, non_blocking=True)
        if grad_mode:
            grad_pin.copy_(grad, non_blocking=True)
        evs2[k][1].record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in evs2)

    dev_ms, e2e_ms = max_over_ranks([dev_ms, e2e_ms], device=dev)
    if rank != 0:
        return
    units = world * args.steps * B
    value = units / (dev_ms / 1e3)
    e2e_value = units / (e2e_ms / 1e3)

    calls = max(timing["calls"], 1)
    triples = timing["triples"] / calls
    stages = {"ring_template": timing["ms_ring"] / calls,
              "shift_add": timing["ms_shift_add"] / calls,
              "reduce": timing["ms_reduce"] / calls,
              "response_loglike": timing["ms_loglike"] / calls}
    if grad_mode:
        stages.update({"grad_response": timing["ms_grad_resp"] / calls,
                       "shift_add_bwd": timing["ms_shift_add_bwd"] / calls,
                       "template_bwd_final": timing["ms_template_bwd"] / calls})
        kernel, k_ms, fpt, traffic = ("k_shift_add_bwd<atmosphere>", stages["shift_add_bwd"],
                                      FLOP_PER_TRIPLE_BWD, None)
    else:
        kernel, k_ms, fpt = (forward_kernel_name(w), stages["shift_add"], FLOP_PER_TRIPLE)
        traffic = profile_traffic() if profiled_config(args) else None
    achieved = triples * fpt / (k_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "kernel": kernel, "kernel_ms": k_ms,
                "triples_per_launch": triples, "flop_per_triple": fpt,
                "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (derived)",
                "stage_ms_per_eval": stages}
    cfg = workload_desc(w)
    cfg["l2"] = "flushed before every timed step (%d MiB write)" % args.flush_mib
    cfg["parallelism"] = "replicas x%d" % world
    cfg["setup_s"] = round(setup_s, 3)
    cfg["launch"] = "CUDA graph replay" if graph is not None else "direct calls"
    cfg["tiles"] = ctx.get_tiles()
    if tuned is not None:
        cfg["autotuned"] = tuned
    unit = "grad-evals/s" if grad_mode else ("profile evals/s" if profile_mode else "evals/s")
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / args.steps},
            "gpu_launches": int(timing["launches"]),
            "instances_logL_minus_inf": n_bad,
            "roofline": roofline, "clocks": clk}
    # measured FP32 FMA throughput (context for the derived peak above)
    meas = {}
    for name, paired in (("ffma", 0), ("ffma2", 1)):
        st_, v_ = ppm._abi.ppm_fp32_peak(local_rank, paired,
                                         ppm._stream_handle(torch.cuda.current_stream()))
        meas[name] = v_ if st_ == 0 else None
    line["roofline"]["fp32_measured_tflops"] = meas
    if grad_mode:
        line["forward_ms_per_step"] = fwd_ms / args.steps
        line["backward_over_forward"] = (dev_ms - fwd_ms) / fwd_ms
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, grad_mode)
    print(json.dumps(line), flush=True)
    ctx.close()


def default_steps(args):
    """Timed and warm-up steps when --steps / --warmup are not given."""
    batch = args.workload in ("batch", "grad_batch")
    if args.steps is None:
        args.steps = 50 if args.impl == "reference" else 3 if batch else 200
    if args.warmup is None:
        args.warmup = 5 if args.impl == "reference" else 3 if batch else 10
    return args


def main():
    args = default_steps(parse())
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

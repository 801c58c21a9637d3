#!/usr/bin/env python
"""Benchmark of the pulse-profile likelihood on GB300.

One step = one full likelihood evaluation (ring templates, shift-and-add with
atmosphere interpolation, ISM, response contraction, Poisson logL) of the
workload's parameter vectors.

Default (``--workload suite``): the headline is the high-fidelity crescent
(one crescent spot, 512 x 512 elements, 256 phases, 300 energies and
channels, M = 2.0, R = 11 km, i = 85 deg, 346 Hz), timed for --steps steps
after --warmup warm-up steps; the same JSON line carries sub-records of the
other workloads, each with its own fixed step counts:
  two_spot  two hotspots (cap + ring), 2 x 128 x 128 elements, 128 phases,
            256 energies, 300 channels;
  batched   4096 mixed-resolution parameter vectors in one call: tiles
            autotuned on a 256-instance sample, one CUDA graph replayed per
            batch, and the same 4096 instances timed one call at a time;
  grad      the log-likelihood and its 13-parameter gradient, 1024 instances
            at 128 x 128 elements, 128 phases, 256 energies, 300 channels.
Every record has its roofline, its clock record and its accuracy against the
FP64 oracle on sampled outputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload suite|atm_two_spot|crescent_extreme|...]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank evaluates
its own copies of the workloads (batched ones draw their own instances;
weak scaling, no collective on the data path).  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the headline workload.
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
PROFILE_DIR = os.path.join(ROOT, "profiles")
KERNEL_SRC = os.path.join(ROOT, "paper_2510_07764_gb300", "csrc", "shift_add.cu")
GRAD_GOLDEN = os.path.join(ROOT, "tests", "golden", "grad_batch_full.json")
HEADLINE = "crescent_extreme"
# one config description shared by both arms
L2_NOTE = ("GPU arm: L2 flushed before every timed step (512 MiB write); "
           "CPU reference arm: not applicable")
# CPU samples: every RING_STRIDE-th ring and PHASE_STRIDE-th output phase
CPU_SAMPLE = {"crescent_extreme": (64, 4), "atm_two_spot": (16, 1), "bb_small": (1, 1)}
REF_SAMPLE = {"crescent_extreme": (64, 8), "atm_two_spot": (64, 1), "bb_small": (1, 1)}
REF_BUDGET_S = 120.0
# sub-record step counts (timed, warm-up)
SUB_STEPS = {"two_spot": (100, 10), "batched": (3, 1), "grad": (2, 1)}
BATCH_TUNE_STRIDE = 16


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # defaults: 20 timed and 5 warm-up steps for the suite (the headline's
    # steps; sub-records use their own counts); 200 and 10 for single-instance
    # workloads; 3 and 3 for the batch workloads; 20 and 5 for the CPU arm
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="suite",
                    choices=["suite", "atm_two_spot", "bb_small", "crescent_extreme", "batch",
                             "grad_batch", "healpix_map"])
    ap.add_argument("--interp", choices=["d", "a", "b", "c"], default=None,
                    help="atmosphere interpolation strategy of Sect. 4 (default: the method's, d)")
    ap.add_argument("--phase-sub", type=int, default=None,
                    help="point samples per output phase bin (ppm_res.phase_sub)")
    ap.add_argument("--batch", type=int, default=None,
                    help="parameter vectors of the batch / grad_batch workloads")
    ap.add_argument("--flush-mib", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (CPU baseline and accuracy against the oracle)")
    ap.add_argument("--graph", action="store_true",
                    help="capture one step in a CUDA graph and time its replays")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the shift-and-add tiles with ppm_autotune before timing")
    ap.add_argument("--walk", type=int, choices=[0, 1, 2], default=0,
                    help="walk of the atmosphere shift-and-add: 0 moment walk, else "
                         "node-major walk, where they apply; 1 energy walk; 2 node-major walk "
                         "where it applies (ppm_tiles.walk)")
    return ap.parse_args(argv)


def default_steps(args):
    """Timed and warm-up steps when --steps / --warmup are not given."""
    batch = args.workload in ("batch", "grad_batch")
    suite = args.workload == "suite"
    if args.steps is None:
        args.steps = 20 if (args.impl == "reference" or suite) else 3 if batch else 200
    if args.warmup is None:
        args.warmup = 5 if (args.impl == "reference" or suite) else 3 if batch else 10
    return args


def headline_name(args):
    return HEADLINE if args.workload == "suite" else args.workload


def make_workload(name, args=None, rank: int = 0, B=None):
    """A workload of one rank.  Batched workloads draw their own parameter
    vectors per rank (seed offset by the rank: weak scaling over independent
    instances); single-instance workloads are replicas."""
    from paper_2510_07764_gb300 import synth
    if name in ("batch", "grad_batch"):
        kw = {"seed": synth.SEED + (1 if name == "grad_batch" else 0) + rank}
        if B is not None:
            kw["B"] = B
        w = synth.WORKLOADS[name](**kw)
    else:
        w = synth.WORKLOADS[name]()
    if args is not None and getattr(args, "interp", None):
        w.interp = args.interp
    if args is not None and getattr(args, "phase_sub", None):
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


def workload_desc(w, world: int = 1):
    """The workload's configuration (the same keys and values in both arms)."""
    inst = w.inst
    mixed = inst.B > 1 and len(set(map(int, inst.n_theta))) > 1
    return {
        "workload": w.name,
        "B": int(inst.B),
        "spots": int(inst.n_spots),
        "elements_per_spot": ("mixed %s" % "/".join("%dx%d" % (n, n) for n in
                                                   sorted(set(map(int, inst.n_theta))))
                              if mixed else
                              "%d pixels" % (12 * int(inst.n_theta[0]) ** 2) if inst.grid == 1
                              else "%dx%d" % (int(inst.n_theta[0]), int(inst.n_phi[0]))),
        "phases": ("mixed %s" % "/".join(map(str, sorted(set(map(int, inst.n_phase)))))
                   if len(set(map(int, inst.n_phase))) > 1 else int(inst.n_phase[0])),
        "energies": int(len(w.E_keV)),
        "channels": int(w.nc),
        "n_fp": int(inst.n_fp),
        "spacetime": "oblate Schwarzschild" if inst.oblate else "Schwarzschild+Doppler",
        "emission": "atmosphere table 35x11x67x166" if inst.emission else "analytic blackbody",
        "interp": getattr(w, "interp", "d"),
        "phase_sub": int(inst.phase_sub),
        "grid": ("HEALPix N_side %d, temperature map" % int(inst.n_theta[0])
                 if inst.grid == 1 else "spot-bounding"),
        "l2": L2_NOTE,
        "parallelism": "replicas x%d" % world,
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
        self.path = os.path.join("/tmp", "ppm_clocks_%d_%d.csv" % (os.getpid(), id(self)))

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


def profiled_config(args, name=None):
    """Whether this run launches the kernel configuration of a committed ncu
    summary (default interpolation, point phases, default walk, default
    tiles), whose DRAM bytes per launch may then be reported as traffic."""
    name = name or headline_name(args)
    return (name in ("atm_two_spot", "crescent_extreme") and args.interp in (None, "d")
            and args.phase_sub in (None, 1) and not args.walk and not args.autotune)


def profile_traffic(name):
    """DRAM bytes per launch of the shift-and-add kernel from the committed ncu
    summary of workload `name`, if it was taken on the current kernel source."""
    path = os.path.join(PROFILE_DIR, "k_shift_add_%s.md" % name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not (m and t):
        return None
    sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    return float(t.group(1)) if m.group(1) == sha else None


# ---------------------------------------------------------------------------
# CPU leg: the FP64 oracle timed on a bounded sample, and the accuracy of the
# GPU outputs against it on sampled bins
# ---------------------------------------------------------------------------
def _work(inst, b, nE):
    return float(inst.n_spots) * inst.n_theta[b] * inst.n_phi[b] * inst.n_phase[b] * nE


def _rings(inst, b):
    """Rings per spot in the oracle's loop (4 N_side - 1 on the HEALPix mesh)."""
    n = int(inst.n_theta[b])
    return 4 * n - 1 if getattr(inst, "grid", 0) == 1 else n


def sample_factor(inst, stride, nE, phase_stride: int = 1):
    """Work of the whole workload over the work of instance 0's sample
    (every stride-th ring, ring 0 first; every phase_stride-th phase, phase 0
    first)."""
    total = sum(_work(inst, b, nE) for b in range(inst.B))
    R = _rings(inst, 0)
    P = int(inst.n_phase[0])
    return total / _work(inst, 0, nE) * R / math.ceil(R / stride) * P / math.ceil(P / phase_stride)


def _single(w, b):
    from paper_2510_07764_gb300 import synth
    inst = w.inst.select(b)
    r0 = int(sum(w.inst.n_phase[:b]))
    return synth.Workload(w.name, inst, w.lens, w.E_keV, atm=w.atm, R=w.R,
                          sigma_ism=w.sigma_ism,
                          counts=None if w.counts is None
                          else w.counts[r0:r0 + int(inst.n_phase[0])], tau=w.tau,
                          interp=getattr(w, "interp", "d"))


def profile_only(w, idx):
    """The instances idx of w with what the oracle's profile needs (no
    response or counts): what the accuracy workers receive."""
    from paper_2510_07764_gb300 import synth
    return synth.Workload(w.name, w.inst.select(idx), w.lens, w.E_keV, atm=w.atm,
                          interp=getattr(w, "interp", "d"))


def oracle_sample(w, stride, phase_stride: int = 1):
    """Time the FP64 oracle on instance 0: every `stride`-th ring and every
    `phase_stride`-th output phase (profile, then the response and logL of
    those rows); returns (seconds, extrapolation factor to the whole workload
    by element x phase x energy work)."""
    import numpy as np
    import oracle
    oracle.build()
    oracle.lens(w.lens)   # table build is not part of an evaluation
    w0 = w if w.inst.B == 1 else _single(w, 0)
    js = np.arange(0, int(w0.inst.n_phase[0]), phase_stride, dtype=np.int32)
    t0 = time.perf_counter()
    Ft = oracle.profile(w0, jsel=None if phase_stride == 1 else js, ring_stride=stride)
    if w.R is not None:
        C = oracle.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
        oracle.loglike(C, w0.counts[js], w.tau)
    dt = time.perf_counter() - t0
    return dt, sample_factor(w.inst, stride, len(w.E_keV), phase_stride)


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


def _oracle_bins(job):
    """Oracle F_t of instance b of _W at the selected phases and energies."""
    import oracle
    b, js, ks = job
    w0 = _W if _W.inst.B == 1 else _single(_W, b)
    return oracle.profile(w0, jsel=js, ksel=ks)


def oracle_sample_parallel(w, stride, workers, phase_stride: int = 1):
    """The same bounded sample as oracle_sample on `workers` processes, split
    by output phase (spawned pool: no GPU state is forked); returns the wall
    time of the profile + response + logL and the extrapolation factor."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    w0 = w if w.inst.B == 1 else _single(w, 0)
    js = np.arange(0, int(w0.inst.n_phase[0]), phase_stride, dtype=np.int32)
    chunks = [c for c in np.array_split(js, workers) if len(c)]
    with mp.get_context("spawn").Pool(len(chunks), initializer=_oracle_pool_init,
                                      initargs=(w0,)) as pool:
        pool.map(_oracle_phase_chunk, [(c[:1], stride) for c in chunks])  # warm
        t0 = time.perf_counter()
        parts = pool.map(_oracle_phase_chunk, [(c, stride) for c in chunks])
        Ft = np.concatenate(parts, axis=0)
        if w.R is not None:
            C = oracle.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
            oracle.loglike(C, w0.counts[js], w.tau)
        dt = time.perf_counter() - t0
    return dt, sample_factor(w.inst, stride, len(w.E_keV), phase_stride)


def fd_evals(w):
    """Oracle evaluations per gradient by central differences (logL + 2 per parameter)."""
    return 1 + 2 * (5 + 4 * int(w.inst.n_spots))


def cpu_baseline(w, grad_mode=False):
    """The FP64 oracle (single thread, and all cores split by phase) on a
    bounded sample, extrapolated; for gradients, the cost of central
    differences with the oracle."""
    stride, pstride = CPU_SAMPLE.get(w.name, (16, 1))
    dt, factor = oracle_sample(w, stride, pstride)
    per_eval = dt * factor / w.inst.B
    mult = fd_evals(w) if grad_mode else 1
    unit = "grad-evals/s" if grad_mode else ("evals/s" if w.R is not None else "profile evals/s")
    cores = os.cpu_count() or 1
    all_core = None
    if cores > 1:
        try:
            dtp, fp = oracle_sample_parallel(w, stride, cores, pstride)
            all_core = {"value": 1.0 / (dtp * fp / w.inst.B * mult), "cores": cores,
                        "measured_s": round(dtp, 3)}
        except Exception as exc:  # the single-thread figure stands alone
            all_core = {"value": None, "cores": cores, "error": str(exc)[:200]}
    best = all_core["value"] if all_core and all_core.get("value") else 1.0 / (per_eval * mult)
    return {"value": best, "unit": unit,
            "cores": all_core["cores"] if all_core and all_core.get("value") else 1,
            "kind": "oracle", "extrapolated": bool(factor > 1.0),
            "single_thread": {"value": 1.0 / (per_eval * mult), "cores": 1,
                              "measured_s": round(dt, 3)},
            "all_core": all_core,
            "sample": "instance 0, every %dth ring%s, all energies, response and logL of "
                      "those rows; single thread %.1f s measured, extrapolated x%.4g by "
                      "element x phase x energy work; all-core: the same sample split by "
                      "output phase over a process pool%s"
                      % (stride, "" if pstride == 1 else " and every %dth phase" % pstride,
                         dt, factor,
                         "; x%d evaluations per central-difference gradient" % mult
                         if grad_mode else "")}


def oracle_accuracy(w, picks, workers=None):
    """Max relative error of GPU F_t values against the FP64 oracle.

    picks: list of (instance b, phase indices, energy indices, GPU values
    [len(js), len(ks)]).  The error is taken per bin where the oracle flux is
    at least 1e-6 of its maximum over the sampled bins of that instance (the
    paper's non-negligible flux criterion), as in the parity tests."""
    import multiprocessing as mp
    import numpy as np
    idx = [b for b, _, _, _ in picks]
    wsub = profile_only(w, idx)
    jobs = [(i, np.asarray(js, np.int32), np.asarray(ks, np.int32))
            for i, (_, js, ks, _) in enumerate(picks)]
    workers = max(1, min(len(jobs), workers or (os.cpu_count() or 1)))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(workers, initializer=_oracle_pool_init,
                                      initargs=(wsub,)) as pool:
        refs = pool.map(_oracle_bins, jobs, chunksize=1)
    worst, n = 0.0, 0
    for (_, _, _, got), ref in zip(picks, refs):
        got = np.asarray(got, np.float64)
        m = np.abs(ref) >= 1e-6 * np.max(np.abs(ref))
        if m.any():
            worst = max(worst, float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))))
            n += int(m.sum())
    return {"max_rel_err": worst, "bins": n, "instances": len(picks),
            "vs": "FP64 oracle, per bin with flux >= 1e-6 of the sampled maximum",
            "oracle_s": round(time.perf_counter() - t0, 2)}


def grad_accuracy(g):
    """Gradient of the timed batch against the oracle's forward-mode values
    stored in tests/golden/grad_batch_full.json (instances of the same seeded
    workload): max relative error per component, components below 1e-5 of
    the largest scale-weighted one taking that floor."""
    import numpy as np
    if not os.path.exists(GRAD_GOLDEN):
        return None
    gold = json.load(open(GRAD_GOLDEN))
    sc = np.array([1.0, 10.0, 1.0, 0.3, 1.0, 1.0, 1.0, 0.2, 6.0, 1.0, 1.0, 0.2, 6.0])
    worst, worst_dir = 0.0, 0.0
    recs = [r for r in gold["instances"] if np.isfinite(r["logL"])]
    for rec in recs:
        ref = np.asarray(rec["grad"], np.float64)
        got = np.asarray(g[rec["b"]], np.float64)[:len(ref)]
        floor = 1e-5 * np.max(np.abs(ref) * sc[:len(ref)]) / sc[:len(ref)]
        worst = max(worst, float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor))))
        for v, dv in zip(rec["directions"], rec["directional"]):
            gv = float(np.dot(got, np.asarray(v)[:len(got)]))
            worst_dir = max(worst_dir, abs(gv - dv) / max(abs(dv), 1e-300))
    return {"max_rel_err": worst, "max_rel_err_directional": worst_dir,
            "instances": [r["b"] for r in recs],
            "vs": "FP64 oracle forward mode (tests/golden/grad_batch_full.json)"}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host
# ---------------------------------------------------------------------------
def reference_stride(first_s, stride, n_steps, budget_s=REF_BUDGET_S, max_stride=1 << 30):
    """Stride of the reference arm's per-step sample: the stride of the first
    step, widened in proportion when n_steps samples of that size would
    exceed the budget (the sample's cost scales as 1 / stride), and at most
    max_stride."""
    if n_steps * first_s <= budget_s:
        return stride
    return int(min(max_stride, math.ceil(stride * n_steps * first_s / budget_s)))


def run_reference(args, rank, world):
    if rank != 0:
        return
    name = headline_name(args)
    w = make_workload(name, args)
    grad_mode = name == "grad_batch"
    mult = fd_evals(w) if grad_mode else 1
    stride, pstride = REF_SAMPLE.get(name, (64, 1))
    times, measured = [], 0.0
    n = args.warmup + args.steps
    for k in range(n):
        dt, factor = oracle_sample(w, stride, pstride)
        measured += dt
        if k == 0:
            # widen the sample (phases first, then rings) so that the whole
            # run stays near the budget
            P = int(w.inst.n_phase[0])
            new_p = reference_stride(dt, pstride, n, max_stride=P)
            rest = dt * pstride / new_p
            stride = reference_stride(rest, stride, n, max_stride=max(1, _rings(w.inst, 0)))
            pstride = new_p
        if k >= args.warmup:
            times.append(dt * factor * mult)
    if not times:
        times.append(dt * factor * mult)
    per_step = sum(times) / len(times)
    value = w.inst.B / per_step
    per_eval = per_step / w.inst.B
    sample = ("instance 0, every %dth ring%s per step, extrapolated by element x phase x "
              "energy work to the whole workload"
              % (stride, "" if pstride == 1 else " and every %dth phase" % pstride))
    unit = "evals/s" if w.R is not None else "profile evals/s"
    if grad_mode:
        sample += "; x%d evaluations per central-difference gradient" % mult
        unit = "grad-evals/s"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_eval * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(w, args.gpus),
            "extrapolated": True,
            "sample_measured_s": round(measured, 2),
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": sample, "extrapolated": True,
                             "measured_s": round(measured, 2)},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Bench:
    """One library context on this rank's GPU, the L2 flush buffer and the
    timing helpers shared by every record."""

    def __init__(self, args, rank, world, local_rank):
        import torch
        import paper_2510_07764_gb300 as ppm
        self.args, self.rank, self.world = args, rank, world
        torch.cuda.set_device(local_rank)
        self.dev = torch.device("cuda", local_rank)
        self.local_rank = local_rank
        self.ppm = ppm
        self.ctx = ppm.Context(local_rank)
        self.lens_key = None
        self.flush = torch.empty(args.flush_mib * (1 << 20) // 4, dtype=torch.float32,
                                 device=self.dev)
        try:
            gid = str(torch.cuda.get_device_properties(self.dev).uuid)
            self.gpu_id = gid if gid.startswith("GPU-") else "GPU-" + gid
        except Exception:
            self.gpu_id = None

    def barrier(self):
        import torch
        if self.world > 1:
            torch.distributed.barrier()

    def setup(self, w):
        t0 = time.perf_counter()
        key = tuple(sorted(vars(w.lens).items()))
        self.ctx.setup(w, build_lens=key != self.lens_key)
        self.lens_key = key
        self.ctx.set_tiles()
        return time.perf_counter() - t0

    def timed(self, step, n, clocks=False):
        """n steps bracketed by a barrier and synchronize on both sides, L2
        flushed before each; returns (per-step ms, clock record or None)."""
        import torch
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n)]
        clk = None
        if clocks:
            clk = Clocks(self.gpu_id)
            clk.start()
        self.barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        for k in range(n):
            self.flush.fill_(float(k))
            evs[k][0].record()
            step()
            evs[k][1].record()
        torch.cuda.synchronize()
        t1 = time.time()
        self.barrier()
        rec = clk.stop(t0, t1) if clk is not None else None
        return [a.elapsed_time(b) for a, b in evs], rec

    def e2e(self, w, dp, step, outs, n, counts=None):
        """The same steps through host buffers: per step the parameters (and
        counts) are copied from pinned host memory and the outputs read back."""
        import numpy as np
        import torch
        ppm = self.ppm
        pin = {f: torch.from_numpy(np.ascontiguousarray(getattr(w.inst, f), dtype=np.float64)
                                   .reshape(-1)).pin_memory() for f in ppm._abi.PARAM_FIELDS}
        host_inst = w.inst.replace()
        for f, t in pin.items():
            setattr(host_inst, f, t)
        counts_pin = None if counts is None else torch.from_numpy(w.counts).pin_memory()
        out_pin = [torch.empty(tuple(o.shape), dtype=o.dtype).pin_memory() for o in outs]
        h2d = sum(t.numel() * 8 for t in pin.values()) + (
            0 if counts is None else counts_pin.numel() * 4)
        d2h = sum(o.numel() * o.element_size() for o in outs)

        def one():
            dp.upload(host_inst, non_blocking=True)
            if counts is not None:
                counts.copy_(counts_pin, non_blocking=True)
            step()
            for o, p in zip(outs, out_pin):
                p.copy_(o, non_blocking=True)

        ms, _ = self.timed(one, n)
        return ms, int(h2d), int(d2h)

    def stage_times(self, step, n=1):
        """Per-evaluation stage times, kernel launches and triples of n direct
        calls (library CUDA events on the launch stream)."""
        import torch
        self.ctx.set_timing(True)  # resets the accumulators
        for _ in range(n):
            step()
        torch.cuda.synchronize()
        t = self.ctx.get_timing()
        self.ctx.set_timing(False)
        return t

    def roofline(self, t, w, grad_mode=False, traffic=None):
        calls = max(t["calls"], 1)
        stages = {"ring_template": t["ms_ring"] / calls, "shift_add": t["ms_shift_add"] / calls,
                  "reduce": t["ms_reduce"] / calls, "response_loglike": t["ms_loglike"] / calls}
        if grad_mode:
            stages.update({"grad_response": t["ms_grad_resp"] / calls,
                           "shift_add_bwd": t["ms_shift_add_bwd"] / calls,
                           "template_bwd_final": t["ms_template_bwd"] / calls})
            kernel, k_ms, fpt = ("k_shift_add_bwd<atmosphere>", stages["shift_add_bwd"],
                                 FLOP_PER_TRIPLE_BWD)
        else:
            kernel, k_ms, fpt = forward_kernel_name(w), stages["shift_add"], FLOP_PER_TRIPLE
        triples = t["triples"] / calls
        achieved = triples * fpt / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
        return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "kernel": kernel, "kernel_ms": k_ms, "triples_per_launch": triples,
                "flop_per_triple": fpt,
                "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (derived)",
                "stage_ms_per_eval": stages}

    # ---- one workload ------------------------------------------------------
    def forward_record(self, w, steps, warmup, graph=False, tune=None, e2e_steps=None,
                       grad_mode=False, traffic=None):
        """Time `steps` evaluations of w (likelihood; the profile alone when w
        has no response; likelihood and gradient in grad mode).  Returns the
        record and the device state the accuracy check reads afterwards."""
        import numpy as np
        import torch
        ppm, ctx, dev = self.ppm, self.ctx, self.dev
        setup_s = self.setup(w)
        dp = ppm.DeviceParams(w.inst, device=dev)
        B = dp.B
        profile_mode = w.R is None
        counts = None if profile_mode else torch.from_numpy(w.counts).to(dev)
        Ft = torch.empty((dp.rows, len(w.E_keV)), dtype=torch.float32, device=dev)
        logL = torch.empty(B, dtype=torch.float64, device=dev)
        grad = torch.empty((B, ppm.N_GRAD), dtype=torch.float64, device=dev)

        def step(stream=None):
            if profile_mode:
                ctx.profile(dp, out=Ft, stream=stream)
            elif grad_mode:
                ctx.loglike_grad(dp, counts, w.tau, out=logL, grad=grad, stream=stream)
            else:
                ctx.loglike(dp, counts, w.tau, out=logL, stream=stream)

        tuned = None
        if self.args.walk:
            ctx.set_tiles(walk=self.args.walk)
        if tune is not None:
            # tiles timed on a sample of the problem, kept for the whole of it
            tuned = ctx.autotune(ppm.DeviceParams(w.inst.select(tune), device=dev))
            tuned["tuned_on_instances"] = int(len(tune))
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        g = None
        if graph:
            # one step captured once; replays re-read parameters and counts from
            # the same device buffers (the plan and workspace are settled above)
            s_cap = torch.cuda.Stream(device=dev)
            s_cap.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s_cap):
                step(s_cap)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
        run = g.replay if g is not None else step
        # launches counted over the timed steps (graph replays record no
        # stage events: the same count as direct calls)
        step_ms, clk = self.timed(run, steps, clocks=True)
        t = self.stage_times(step, n=1 if g is not None or B > 1 else min(steps, 20))
        launches = int(round(t["launches"] / max(t["calls"], 1))) * steps
        fwd_ms = None
        if grad_mode:
            fwd_ms, _ = self.timed(lambda: ctx.loglike(dp, counts, w.tau, out=logL), steps)
        outs = [Ft] if profile_mode else [logL] + ([grad] if grad_mode else [])
        ms2, h2d, d2h = self.e2e(w, dp, run, outs, e2e_steps or steps, counts=counts)
        dev_ms, e2e_ms, fsum = max_over_ranks(
            [sum(step_ms), sum(ms2), sum(fwd_ms) if fwd_ms else 0.0], device=dev)
        units = self.world * steps * B
        unit = "grad-evals/s" if grad_mode else ("profile evals/s" if profile_mode else "evals/s")
        rec = {"value": units / (dev_ms / 1e3), "unit": unit,
               "steps": steps, "warmup": warmup, "ms_per_step": dev_ms / steps,
               "ms_per_step_median": statistics.median(step_ms),
               "e2e": {"value": self.world * len(ms2) * B / (e2e_ms / 1e3), "unit": unit,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": e2e_ms / len(ms2)},
               "gpu_launches": launches,
               "roofline": self.roofline(t, w, grad_mode, traffic),
               "clocks": clk,
               "config": workload_desc(w, self.world),
               "run": {"setup_s": round(setup_s, 3),
                       "launch": "CUDA graph replay" if g is not None else "direct calls",
                       "tiles": ctx.get_tiles()}}
        if tuned is not None:
            rec["run"]["autotuned"] = tuned
        if not profile_mode:
            rec["instances_logL_minus_inf"] = int((~torch.isfinite(logL)).sum())
        if grad_mode:
            rec["forward_ms_per_step"] = fsum / steps
            rec["backward_over_forward"] = (dev_ms - fsum) / fsum
        state = {"dp": dp, "counts": counts, "logL": logL, "grad": grad, "graph": g}
        return rec, state

    def profile_picks(self, w, dp, picks_of):
        """GPU F_t values at the bins the accuracy check samples: picks_of
        lists (instance, phase indices, energy indices)."""
        import numpy as np
        Ft = self.ctx.profile(dp).cpu().numpy()
        row0 = np.concatenate([[0], np.cumsum(w.inst.n_phase)])
        return [(b, js, ks, Ft[row0[b] + np.asarray(js)][:, np.asarray(ks)])
                for b, js, ks in picks_of]

    def single_calls(self, w, state):
        """The batch's instances one ppm_loglike call each, in batch order,
        on the same device arrays (instance views): wall time of the loop
        between two synchronizes, with the L2 flushed once before."""
        import numpy as np
        import torch
        dp, counts = state["dp"], state["counts"]
        out = torch.empty(dp.B, dtype=torch.float64, device=self.dev)
        row0 = np.concatenate([[0], np.cumsum(w.inst.n_phase)])
        views = [dp.instance(b) for b in range(dp.B)]

        def loop():
            for b, v in enumerate(views):
                self.ctx.loglike(v, counts[row0[b]:row0[b + 1]], w.tau, out=out[b:b + 1])

        loop()  # warm: plans and workspace of every resolution
        ms, _ = self.timed(loop, 1)
        ll_b = state["logL"]
        fin = torch.isfinite(ll_b) & torch.isfinite(out)
        diff = float(((out - ll_b).abs() / ll_b.abs().clamp_min(1.0))[fin].max()) if fin.any() else 0.0
        return {"value": dp.B / (ms[0] / 1e3), "unit": "evals/s", "ms": ms[0],
                "launch": "one direct ppm_loglike call per instance, batch order",
                "max_rel_diff_logL_vs_batched": diff}


def run_suite(bench, args):
    """Headline (crescent) plus the two-spot, batched and gradient sub-records."""
    import numpy as np
    B = bench
    w = make_workload(HEADLINE, args, bench.rank)
    line, st = B.forward_record(w, args.steps, args.warmup,
                                traffic=profile_traffic(HEADLINE) if profiled_config(args) else None)
    acc_jobs = []
    line_js = np.array([0, 63, 127, 128, 200, 255])
    line_ks = np.array([0, 37, 150, 299])
    acc_jobs.append(("headline", w, B.profile_picks(w, st["dp"], [(0, line_js, line_ks)])))

    sub = {}
    # two hotspots
    w2 = make_workload("atm_two_spot", args, bench.rank)
    n, wu = SUB_STEPS["two_spot"]
    sub["two_spot"], st2 = B.forward_record(
        w2, n, wu, traffic=profile_traffic("atm_two_spot") if profiled_config(args, "atm_two_spot")
        else None)
    rng = np.random.default_rng(3)
    acc_jobs.append(("two_spot", w2, B.profile_picks(
        w2, st2["dp"], [(0, np.sort(rng.choice(128, 6, replace=False)),
                         np.sort(rng.choice(256, 10, replace=False)))])))
    # batched: autotuned tiles, one CUDA graph per batch, and the same
    # instances one call at a time
    wb = make_workload("batch", args, bench.rank)
    n, wu = SUB_STEPS["batched"]
    tune = np.arange(0, wb.inst.B, BATCH_TUNE_STRIDE)
    rec, stb = B.forward_record(wb, n, wu, graph=True, tune=tune, e2e_steps=2)
    rec["single_calls"] = B.single_calls(wb, stb)
    rec["batched_over_single"] = rec["value"] / rec["single_calls"]["value"]
    sub["batched"] = rec
    rng = np.random.default_rng(5)
    picks = []
    for b in np.sort(rng.choice(wb.inst.B, 8, replace=False)):
        P = int(wb.inst.n_phase[b])
        picks.append((int(b), np.sort(rng.choice(P, 4, replace=False)),
                      np.sort(rng.choice(len(wb.E_keV), 6, replace=False))))
    acc_jobs.append(("batched", wb, B.profile_picks(wb, stb["dp"], picks)))
    del stb
    # gradient
    wg = make_workload("grad_batch", args, bench.rank)
    n, wu = SUB_STEPS["grad"]
    rec, stg = B.forward_record(wg, n, wu, grad_mode=True, e2e_steps=1)
    if bench.rank == 0:
        rec["accuracy"] = grad_accuracy(stg["grad"].cpu().numpy())
    sub["grad"] = rec
    return line, sub, acc_jobs, w


def run_ours(args, rank, world, local_rank):
    import torch
    bench = Bench(args, rank, world, local_rank)
    if args.workload == "suite":
        line, sub, acc_jobs, w = run_suite(bench, args)
    else:
        w = make_workload(args.workload, args, rank, B=args.batch)
        grad_mode = args.workload == "grad_batch"
        line, st = bench.forward_record(
            w, args.steps, args.warmup, graph=args.graph,
            tune=(list(range(w.inst.B)) if args.autotune else None), grad_mode=grad_mode,
            traffic=profile_traffic(args.workload) if profiled_config(args) else None)
        sub, acc_jobs = {}, []
        if not grad_mode and w.inst.B == 1:
            import numpy as np
            rng = np.random.default_rng(3)
            P, K = int(w.inst.n_phase[0]), len(w.E_keV)
            acc_jobs.append(("headline", w, bench.profile_picks(
                w, st["dp"], [(0, np.sort(rng.choice(P, min(P, 6), replace=False)),
                               np.sort(rng.choice(K, min(K, 10), replace=False)))])))
    if rank != 0:
        bench.ctx.close()
        return
    out = {"metric": METRIC, "value": line["value"], "unit": line["unit"], "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": line["ms_per_step"], "ms_per_step_median": line["ms_per_step_median"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": line["config"], "run": line["run"],
           "e2e": line["e2e"], "gpu_launches": line["gpu_launches"],
           "roofline": line["roofline"], "clocks": line["clocks"]}
    for k in ("instances_logL_minus_inf", "forward_ms_per_step", "backward_over_forward"):
        if k in line:
            out[k] = line[k]
    # measured FP32 FMA throughput (context for the derived peak)
    ppm = bench.ppm
    meas = {}
    for name, paired in (("ffma", 0), ("ffma2", 1)):
        st_, v_ = ppm._abi.ppm_fp32_peak(local_rank, paired,
                                         ppm._stream_handle(torch.cuda.current_stream()))
        meas[name] = v_ if st_ == 0 else None
    out["roofline"]["fp32_measured_tflops"] = meas
    out.update(sub)
    bench.ctx.close()
    if world == 1 and not args.no_cpu_baseline:
        # the oracle leg: CPU baseline of the headline workload and the
        # accuracy of every timed workload on sampled outputs
        out["cpu_baseline"] = cpu_baseline(w, args.workload == "grad_batch")
        for name, wk, picks in acc_jobs:
            acc = oracle_accuracy(wk, picks)
            if name == "headline":
                out["accuracy"] = acc
            else:
                out[name]["accuracy"] = acc
    print(json.dumps(out), flush=True)


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

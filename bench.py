#!/usr/bin/env python3
"""Throughput of the Epstein-Nesbet second-order energy on B300.

Metric: E2 perturber couplings/s (FP64).  A coupling is one external
determinant K (per root) whose V_K = <K|H|Psi> is formed and whose
|V_K|^2 / (E0 - H_KK) is reduced.  One step = one full e2_forward over every
external class of the workload (all of Q), inputs resident in HBM.

The headline runs the library's default arithmetic, IEEE FP64 throughout
(`--arith fp64`).  The opt-in emulated arithmetic (bf16 slices on the tensor
pipe with float-float epilogues, `e2_set_contraction`) is measured on the
same workload after it and reported under "alt_arithmetic" with its own
dtype label; `--arith sliced` makes it the headline instead.

Default workload: the Ar-shaped DCB DAS problem (8 core spinors, three
active subspaces of 8 spinors holding 10 electrons, N_P = 40,608, 400 virtual
spinors, 600 Coulomb + 300 Breit factors, one root): 1.59e11 couplings per
step, the largest of the five shapes whose K forwards fit a run of minutes in
FP64 (the Kr- and Xe-shaped ones take hours per forward at the FP64 rate).
The fwd+bwd, end-to-end and other-arithmetic timings take fewer steps when a
step is long (--aux-seconds); each says how many.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--config NAME]

Under torchrun (N > 1) the external space is sharded over the ranks: each
rank takes an even share of every class's units, the per-tile partials are
summed by one NCCL all-reduce and reduced in the fixed order, so E2 is
bitwise the N = 1 value (strong scaling).  --replicas runs N independent
copies instead (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E2 perturber couplings/s (FP64, |ΔE2|≤1e-9 Eh); fwd+bwd vs fwd time"
WORKLOADS = {
    "ne_dcg": "Ne-shaped DCG: 2 core + CAS(8e,16) + 200 virtual spinors, 400 Coulomb + 200 Gaunt factors, 1 root",
    "dc_small": "DC: 4 core + CAS(6e,12) + 40 virtual spinors, 60 Coulomb factors, 1 root",
    "ar_dcb_das": "Ar-shaped DCB: 8 core + DAS 3x8 spinors (10e, N_P = 40,608) + 400 virtual spinors, 600 Coulomb + "
            "300 Breit factors, 1 root",
    "kr_dcb": "Kr-shaped DCB: 16 core + CAS(8e,24) + 600 virtual spinors, 900 Coulomb + 450 Breit factors, 4 roots",
    "xe_dcb": "Xe-shaped DCB: 46 core + CAS(8e,24) + 1000 virtual spinors, 1400 Coulomb + 700 Breit factors, 1 root",
}
GEMM_CLASSES = {2: "ntp", 5: "na", 7: "na", 4: "na2p1", 6: "ntp"}
CLASS_NAMES = ["(0,0)", "(0,1)", "(0,2)", "(1,0)", "(1,1)", "(1,2)", "(2,0)", "(2,1)", "(2,2)"]
KERNEL_OF_CLASS = {c: "k_class_gemm" for c in GEMM_CLASSES} | {8: "k_class22", 1: "k_class01", 3: "k_class10",
                                                                0: "k_class00"}


def max_over_ranks(ms, ws, dist, device):
    """The whole job's step time: the slowest rank's.  Every rank brackets its
    timed region with barriers, so the regions overlap; with one rank this is
    ms itself (no collective)."""
    if ws <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _rows(prob, cls):
    """External rows of class cls (correlated core / virtual indices)."""
    nc = sum(1 for k in range(prob.n_core) if not prob.frozen[k])
    nv = sum(1 for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v])
    pair = lambda n: n * (n - 1) // 2
    return {0: 1, 1: nv, 2: pair(nv), 3: nc, 4: nc * nv, 5: nc * pair(nv), 6: pair(nc), 7: pair(nc) * nv,
            8: pair(nc) * pair(nv)}[cls]


def _ncols(prob, plan, cls):
    """Strings of a class (its coupling-table columns)."""
    return plan.q_per_class[cls] / max(_rows(prob, cls), 1)


def _kpad(prob, cls):
    return (_kdim(prob, cls) + 7) // 8 * 8


def _kdim(prob, cls):
    na = prob.n_act
    return {"ntp": na * (na - 1) // 2, "na": na, "na2p1": 1 + na * na}[GEMM_CLASSES[cls]]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.gpu), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCE = {"k_class_gemm": "e2_kernels.cu", "k_class_oz": "e2_ozaki.cu"}


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCE:
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    src = open(os.path.join(ROOT, "paper_2608_11529_b300", "csrc", KERNEL_SOURCE[kernel]), "rb").read()
    if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    # the sliced kernel's roofline is over a step's launches: bytes per step
    return rec.get("bytes_per_step", rec.get("bytes_per_launch"))


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def _sample_ks(prob, n, rng, chunk=1 << 19):
    """n random external determinants of the workload, drawn with the class
    sizes as weights: (holes, particles, active string), as arrays.  Holes
    (particles) are distinct correlated core (virtual) spinors; the active
    string holds the class's electron count on uniformly chosen active
    spinors."""
    from math import comb
    nc = np.array([k for k in range(prob.n_core) if not prob.frozen[k]], np.int32)
    nv = np.array([v for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v]], np.int32)
    cls, w = [], []
    for h in range(3):
        for p in range(3):
            ne = prob.n_elec + h - p
            if (h, p) == (0, 0) or ne < 0 or ne > prob.n_act:
                continue
            cls.append((h, p, ne))
            w.append(comb(len(nc), h) * comb(len(nv), p) * comb(prob.n_act, ne))
    w = np.array(w, float) / sum(w)
    cls = np.array(cls, np.int32)
    pick = rng.choice(len(cls), size=n, p=w)
    nh, npp, ne = cls[pick, 0], cls[pick, 1], cls[pick, 2]

    def tuples(pool, k):   # k[i] distinct members of pool, ascending, padded with 0
        out = np.zeros((n, 2), np.int32)
        m = len(pool)
        if m == 0:
            return out
        i1 = rng.integers(0, m, n)
        i2 = rng.integers(0, max(m - 1, 1), n)
        i2 = i2 + (i2 >= i1)
        lo, hi = np.minimum(i1, i2), np.minimum(np.maximum(i1, i2), m - 1)
        out[:, 0] = np.where(k == 2, pool[lo], np.where(k == 1, pool[i1], 0))
        out[:, 1] = np.where(k == 2, pool[hi], 0)
        return out

    hs, ps = tuples(nc, nh), tuples(nv, npp)
    acts = np.zeros(n, np.uint64)
    na = prob.n_act
    for a in range(0, n, chunk):   # a random permutation of the active spinors per determinant, first ne kept
        b = min(n, a + chunk)
        order = np.argsort(rng.random((b - a, na)), axis=1).astype(np.uint64)
        keep = np.arange(na)[None, :] < ne[a:b, None]
        acts[a:b] = np.where(keep, np.left_shift(np.uint64(1), order), np.uint64(0)).sum(axis=1, dtype=np.uint64)
    return nh, hs, npp, ps, acts


class OracleSampler:
    """The oracle (V_K from the explicit Q H P row, H_KK from the diagonal
    rule) on bounded random samples of the workload's external determinants,
    on all host cores.  The sample size is calibrated once, to about
    `seconds` of oracle work; each timed sample is drawn before its clock
    starts."""

    def __init__(self, prob, seconds, seed=0):
        from oracle import Oracle
        self.prob = prob
        self.o = Oracle(prob, use_eri_cache=False)
        c = prob.X0[:1] / np.linalg.norm(prob.X0[:1])
        self.o.set_c(c)
        self.E0 = np.zeros(1)
        self.rng = np.random.default_rng(seed)
        n = 256
        while True:
            dt = self._time(n)
            if dt >= 0.2 * seconds or n >= 1 << 21:
                break
            n *= 4
        self.n = int(max(256, min(4_000_000, n * seconds / max(dt, 1e-3))))

    def _time(self, n, reuse=False):
        if not (reuse and getattr(self, "_ks", None) is not None and len(self._ks[0]) == n):
            self._ks = _sample_ks(self.prob, n, self.rng)
        t0 = time.perf_counter()
        self.o.couplings(self.E0, *self._ks)
        return time.perf_counter() - t0

    def step(self, reuse=False):
        """(couplings, seconds) of one timed sample (a fresh draw, or the last
        one again with reuse)."""
        return self.n, self._time(self.n, reuse)


def oracle_rate(prob, seconds=15.0, seed=0):
    """Couplings/s of the oracle on a calibrated sample (see OracleSampler),
    timed over and over until about `seconds` of oracle work have passed (the
    sample is capped at 4 million determinants, which many host cores clear
    in under a second)."""
    s = OracleSampler(prob, seconds, seed)
    n, dt = s.step()
    reps = 1
    while dt < seconds:
        n1, dt1 = s.step(reuse=True)
        n, dt, reps = n + n1, dt + dt1, reps + 1
    return n / dt, n, dt, reps


def run_reference(args):
    """The oracle arm: each step times the oracle on a bounded sample of the
    workload (calibrated once, in the first warm-up step)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from e2_inputs import make_problem
    prob = make_problem(args.config)
    cores = os.cpu_count()
    sampler = OracleSampler(prob, args.ref_seconds, seed=1)
    for _ in range(args.warmup):
        sampler.step()
    ns, dts = [], []
    for _ in range(args.steps):
        n, dt = sampler.step()
        ns.append(n), dts.append(dt)
    value = sum(ns) / sum(dts)
    sample = (f"{sampler.n} random external determinants per step (class-size weighted), V_K from the explicit "
              f"Q H P row and H_KK each, about {args.ref_seconds:.0f} s of oracle work per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "couplings/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "couplings_per_step": sampler.n},
            "cpu_baseline": {"value": value, "unit": "couplings/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "couplings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched evidence run: the 3 Hamiltonians x 3 frozen cutoffs of a workload
    shape (all roots of each) in one e2_batch_forward -- every class of every
    job-root in one persistent launch, or one per group of --roots-per-launch
    roots -- captured in a CUDA graph and replayed, against the same jobs'
    e2_forward calls one after another.  Prints one JSON line with
    "mode": "batch"."""
    # the batch keeps every job's layout in one large workspace: let freed
    # memory of the set-up go back to the device (set before CUDA starts)
    os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    import torch
    import paper_2608_11529_b300 as e2
    from e2_inputs import make_problem
    from e2_inputs.synth import CONFIGS
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    over = dict(Lc=args.factors, Lx=args.factors // 2) if args.factors else {}
    if args.virt:
        over["n_virt"] = args.virt
    if args.core:
        over["n_core"] = args.core
    if args.roots:
        over["n_roots"] = args.roots
    nv = over.get("n_virt", CONFIGS[args.config]["n_virt"])
    nc = over.get("n_core", CONFIGS[args.config]["n_core"])
    # frozen (core, virtual) cutoffs: none, a core pair + 20%, more core + 40% of the virtuals
    cutoffs = [(0, 0), (min(2, nc), nv // 5), (min(6, nc), 2 * nv // 5)]
    jobs = []
    for ham in ("DC", "DCG", "DCB"):
        for fc, fv in cutoffs:
            prob = make_problem(args.config, ham=ham, n_frozen_core=fc, n_frozen_virt=fv, **over)
            plan = e2.E2Problem.from_problem(prob)
            t = e2.device_inputs(prob, prob.X0, device=dev)
            c, _, _ = plan.reference_solve(t["h"], t["B_c"], t["c"], t["B_x"], t["w_x"], lam=t["lam"], tol=1e-10)
            t["c"] = c
            if not args.no_autotune:
                plan.autotune(**t)
            jobs.append((ham, fc, fv, plan, t))
    couplings = sum(float(p.q_per_class.sum()) * p.n_roots for *_, p, _ in jobs)
    for *_, p, _ in jobs:   # the solve / tuning workspaces of every job
        p.release()
    torch.cuda.empty_cache()
    # the batch's workspace first (all jobs' layouts at once); the sequential
    # forwards then take one job's workspace at a time beside it
    batch = e2.E2Batch([p for *_, p, _ in jobs], roots_per_launch=args.roots_per_launch)
    batch.prepare(dev)
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def seq():   # one job at a time, each job's workspace released after its forward
        out = []
        for *_, p, t in jobs:
            E2, E2c, _ = p.forward(**t)
            out.append((E2.clone(), E2c.clone(), None))
            p.release()
        return out

    for _ in range(args.warmup):
        seq()
    torch.cuda.synchronize()
    a, z = ev(), ev()
    a.record(stream)
    for _ in range(args.steps):
        ref = seq()
    z.record(stream)
    torch.cuda.synchronize()
    ms_seq = a.elapsed_time(z) / args.steps
    ref = [(E2, E2c) for E2, E2c, _ in ref]
    torch.cuda.empty_cache()
    inputs = [t for *_, t in jobs]
    for _ in range(args.warmup):
        batch.forward(inputs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            out = batch.forward(inputs)
    stream.wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        g.replay()
    z.record(stream)
    torch.cuda.synchronize()
    ms_batch = a.elapsed_time(z) / args.steps
    same = all(torch.equal(x[0], y[0]) and torch.equal(x[1], y[1]) for x, y in zip(ref, out))
    line = {"mode": "batch", "metric": METRIC, "value": couplings / (ms_batch * 1e-3), "unit": "couplings/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config] + (f" [variant {over}]" if over else ""),
                       "jobs": [{"ham": h, "frozen_core": fc, "frozen_virt": fv, "roots": p.n_roots,
                                 "couplings": float(p.q_per_class.sum()) * p.n_roots} for h, fc, fv, p, _ in jobs],
                       "couplings_per_step": couplings},
            "sequential_ms": ms_seq, "sequential_couplings_per_s": couplings / (ms_seq * 1e-3),
            "graph_replay": True, "bitwise_equal_to_sequential": same,
            "job_roots": sum(p.n_roots for *_, p, _ in jobs),
            "persistent_launches": (-(-max(p.n_roots for *_, p, _ in jobs) // args.roots_per_launch)
                                    if args.roots_per_launch else 1),
            "batch_workspace_gb": batch.workspace_bytes / 1e9,
            "gpu_launches": batch.launch_count()}
    print(json.dumps(line), flush=True)
    return 0


ARITH_DTYPE = {"fp64": "f64", "sliced": "f64-emulated (bf16x5 slices, float-float epilogue)"}


def _arith_parts(plan, present):
    """The arithmetic each part of the path ran in."""
    return {**{CLASS_NAMES[k]: ("sliced bf16 + float-float epilogue" if plan.contraction(k)[0] else "fp64")
               for k in present if k in GEMM_CLASSES},
            **({"(2,2)": "float-float" if plan.contraction(8)[0] else "fp64"} if 8 in present else {}),
            "gather classes": "fp64",
            "integral products": "sliced bf16" if plan.contraction(-1)[0] else "fp64",
            "adjoint products": "sliced bf16 (4 slices)" if plan.contraction(-2)[0] else "fp64"}


def _forward_fn(plan, t, shard, dist):
    """One step: the forward over all of Q; with shards, this rank's share,
    the ranks' partials summed (NCCL) and the fixed-order reduction."""
    if shard:
        return lambda: plan.sharded_forward(dist, **t)
    return lambda: plan.forward(**t)


def _timed_forward(plan, t, steps, warmup, stream, ws, dist, dev, clocks=None, shard=False):
    """warmup + steps forwards; the timed region is barrier-bracketed and the
    step time is the slowest rank's.  Per-class kernel times (root 0) come
    from event pairs the library records around each class kernel."""
    import torch
    step = _forward_fn(plan, t, shard, dist)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches = plan.launch_count()
    evs = []
    for _ in range(steps):
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(9)]
        for a, b in pairs:
            a.record()
            b.record()
        evs.append(pairs)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    torch.cuda.nvtx.range_push("forward")   # ncu --nvtx --nvtx-include "forward/" selects these launches
    start.record(stream)
    for s in range(steps):
        plan.set_events(evs[s])
        E2, E2c, E0 = step()
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    if ws > 1:
        dist.barrier()
    plan.set_events(None)
    ms = max_over_ranks(start.elapsed_time(end) / steps, ws, dist, dev)
    present = [k for k in range(9) if plan.q_per_class[k] > 0]
    ktime = {k: sum(evs[s][k][0].elapsed_time(evs[s][k][1]) for s in range(steps)) / steps for k in present}
    return dict(ms=ms, ktime=ktime, present=present, E2=E2.clone(), E2c=E2c.clone(), E0=E0.clone(),
                launches=launches, clocks=clk)


def _kernels(plan, present):
    sliced = {k for k in GEMM_CLASSES if k in present and plan.contraction(k)[0]}
    kern = {k: ("k_class_oz" if k in sliced else KERNEL_OF_CLASS[k]) for k in present}
    if 8 in present and plan.contraction(8)[0]:
        kern[8] = "k_class22_df"  # class (2,2) in float-float
    return kern


def _roofline(prob, plan, fw, peak_dmma, peak_dfma):
    """Roofline of the dominant kernel over the timed steps (root 0's launches)."""
    present, ktime = fw["present"], fw["ktime"]
    kern = _kernels(plan, present)
    ksum = {}
    for k in present:
        ksum[kern[k]] = ksum.get(kern[k], 0.0) + ktime[k]
    dom_kernel = max(ksum, key=ksum.get)
    classes = [k for k in present if kern[k] == dom_kernel]
    t_ms = sum(ktime[k] for k in classes)
    couplings = sum(plan.q_per_class[k] for k in classes)
    if dom_kernel == "k_class_oz":
        # the emulation's tensor work: 15 slice pairs (levels 2..6 of five
        # slices per operand), each a real product of length 2K into the two
        # real outputs (Re V, Im V) of a coupling: 120 K bf16 flops per
        # coupling; peak: the measured bf16 rate, sustained (the kernel runs
        # inside a long step)
        mp = _measured_peaks()
        peak_bf16 = mp.get("bf16_tflops_sustained") or 1400.0
        flops = sum(120.0 * plan.q_per_class[k] * _kdim(prob, k) for k in classes)
        achieved = flops / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_bf16, "unit": "TFLOP/s",
                "frac": achieved / peak_bf16, "traffic": _traffic("k_class_oz"),
                "traffic_scope": "DRAM bytes per step over the kernel's launches (ncu)",
                "kernel": "k_class_oz classes " + " ".join(CLASS_NAMES[k] for k in classes),
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop), "
                                "of measured" if mp.get("bf16_tflops_sustained") else
                                "fallback 1.4 PFLOP/s sustained bf16, of fallback"),
                "algorithmic_flops_per_step": flops, "flops_per_coupling": "120 K bf16 (15 slice pairs x 2 real "
                                                                          "outputs x real length 2K x 2)"}
    elif dom_kernel == "k_class_gemm":
        # algorithmic: 8 K real flops per coupling (one complex multiply-add
        # per contraction index, K = the class's contraction length); the
        # kernel executes fewer: Gauss's three real products per complex
        # product (6 real flops) and, with column tiles, only each tile's
        # compacted rows (the structural zeros of the coupling tables skipped)
        flops = sum(8.0 * plan.q_per_class[k] * _kdim(prob, k) for k in classes)
        exe = 0.0
        for k in classes:
            f = 6.0 * plan.q_per_class[k] * _kpad(prob, k)
            tiles, krows, used = plan.class_tiles(k)
            if used:
                f = 6.0 * (plan.q_per_class[k] / _ncols(prob, plan, k)) * krows * 64
            exe += f
        achieved = flops / (t_ms * 1e-3) / 1e12
        executed = exe / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_dmma, "unit": "TFLOP/s",
                "frac": achieved / peak_dmma, "traffic": _traffic("k_class_gemm"),
                "traffic_scope": "DRAM bytes read + written per step over the kernel's class launches (ncu, one "
                                 "pass, full-size capture of the benchmark workload)",
                "kernel": "k_class_gemm classes " + " ".join(CLASS_NAMES[k] for k in classes),
                "peak_source": "FP64 tensor pipe (mma.sync m16n8k8 f64) measured on this GPU in this run "
                               "(e2_fp64_peak, burst), of measured; MEASURED_PEAKS.json has no FP64 figure",
                "peak_nominal_ratio_tflops": (_measured_peaks().get("bf16_tflops") or 1810.3) * 1.25 / 2250.0,
                "algorithmic_flops_per_step": flops,
                "flops_per_coupling": "8 K real (complex multiply-add per contraction index)",
                "executed_tflops": executed, "executed_frac": executed / peak_dmma,
                "executed_flops_per_step": exe,
                "executed_note": "6 real flops per complex product (Gauss) over each column tile's compacted "
                                 "rows; frac above 1 = the algorithmic count includes work the kernel skips"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": peak_dfma, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": dom_kernel}
    roof.update({"ms_per_step": t_ms, "launches_per_step": len(classes),
                 "couplings_per_s": couplings / (t_ms * 1e-3), "kernel_ms_per_step": ksum})
    return roof


def _per_class(prob, plan, fw, peak_dmma, peak_dfma):
    """Per class: couplings, event-timed ms, couplings/s; the dense classes'
    achieved FP64 tensor rate (8 K real flops per coupling, and the executed
    6 K' of the compacted Gauss products) against the measured DMMA peak;
    class (2,2)'s FP64 ALU rate (7 FP64 arithmetic instructions per
    coupling: two adds for the denominator, a quarter of the 15-operation
    four-way inversion, one FMA; compares and conversions not counted, so the
    fraction is a lower bound) against the measured FP64 FMA instruction
    rate."""
    out = {}
    for k in fw["present"]:
        ms, q = fw["ktime"][k], float(plan.q_per_class[k]) * plan.n_roots
        row = {"couplings": q, "ms": ms, "couplings_per_s": q / (ms * 1e-3) if ms > 0 else None}
        if k in GEMM_CLASSES and not plan.contraction(k)[0] and ms > 0:
            alg = 8.0 * q * _kdim(prob, k) / (ms * 1e-3) / 1e12
            tiles, krows, used = plan.class_tiles(k)
            kx = krows * 64 / (tiles * 64) if used and tiles else _kpad(prob, k)
            exe = 6.0 * q * kx / (ms * 1e-3) / 1e12
            row.update({"kernel": "k_class_gemm", "algorithmic_tflops": alg, "executed_tflops": exe,
                        "executed_frac_of_dmma_peak": exe / peak_dmma})
        elif k == 8 and not plan.contraction(8)[0] and ms > 0:
            ops = 7.0 * q / (ms * 1e-3)
            row.update({"kernel": "k_class22", "fp64_instructions_per_s": ops,
                        "frac_of_fp64_fma_instruction_peak": ops / (peak_dfma * 1e12 / 2.0)})
        out[CLASS_NAMES[k]] = row
    return out


def _timed_fwd_bwd(plan, t, steps, warmup, stream, ws, dist, dev):
    import torch
    for _ in range(warmup):
        plan.value_and_grad(**t)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("fwd_bwd")   # ncu --nvtx --nvtx-include "fwd_bwd/" selects these launches
    b0.record(stream)
    for _ in range(steps):
        vg = plan.value_and_grad(**t)
    b1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    return max_over_ranks(b0.elapsed_time(b1) / steps, ws, dist, dev), vg[0].clone()


def _integral_flops(prob, plan):
    """Algorithmic work of the integral formation (step a5): every
    antisymmetrised integral <pq||rs> = (pr|qs) - (ps|qr) that the classes
    contract, two complex dot products of length L over the factors each:
    16 L real flops per integral."""
    from math import comb
    nc = sum(1 for k in range(prob.n_core) if not prob.frozen[k])
    nv = sum(1 for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v])
    na = prob.n_act
    ntp, npv, npc = comb(na, 2), comb(nv, 2), comb(nc, 2)
    q = plan.q_per_class
    blocks = {2: npv * ntp, 5: nc * npv * na, 7: npc * nv * na, 4: nc * nv * na * na, 6: npc * ntp, 8: npc * npv,
              1: nv * na * ntp, 3: nc * ntp * na, 0: ntp * ntp}
    L = prob.Bc.shape[0] + (prob.Bx.shape[0] if prob.ham != "DC" else 0)
    n_int = sum(v for k, v in blocks.items() if q[k] > 0) + ntp * ntp   # <tu||vw> enters E0 always
    return 16.0 * L * n_int, n_int


def _timed_integrals(plan, prob, t, steps, warmup, stream, ws, dist, dev, peak_dmma):
    import torch
    tin = {k: v for k, v in t.items() if k != "c"}
    for _ in range(warmup):
        plan.form_integrals(**tin)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        plan.form_integrals(**tin)
    z.record(stream)
    torch.cuda.synchronize()
    ims = max_over_ranks(a.elapsed_time(z) / steps, ws, dist, dev)
    flops, n_int = _integral_flops(prob, plan)
    ach = flops / (ims * 1e-3) / 1e12
    return {"ms_per_step": ims, "steps": steps, "warmup": warmup, "integrals_formed": n_int,
            "algorithmic_flops": flops, "flops_per_integral": "16 L real (two complex dot products over the factors)",
            "achieved_tflops": ach, "frac_of_fp64_tensor_peak": ach / peak_dmma,
            "arithmetic": "sliced bf16" if plan.contraction(-1)[0] else "fp64",
            "what": "e2_form_integrals: compact factors, G, eps^, f^(O), string tables, every integral block "
                    "of the classes from the factors (step a5; the paper's T_int)"}


def _aux_steps(args, ms):
    """Steps of the secondary timings (fwd+bwd, end to end, the other
    arithmetic): the headline's K where a step is short, else as many as fit
    about --aux-seconds (at least 1)."""
    if args.aux_steps > 0:
        return args.aux_steps, 1
    n = int(max(1, min(args.steps, args.aux_seconds * 1e3 / max(ms, 1e-3))))
    return n, (2 if ms < 5e3 else 1)


def run(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    # N > 1: the external space is sharded over the ranks (each class's units
    # split evenly; partials summed by NCCL, E2 bitwise equal to N = 1); total
    # work fixed.  --replicas: N independent copies of the whole job instead.
    shard = ws > 1 and not args.replicas
    import paper_2608_11529_b300 as e2
    from e2_inputs import make_problem
    over = dict(Lc=args.factors, Lx=args.factors // 2) if args.factors else {}
    if args.virt:
        over["n_virt"] = args.virt
    if args.core:
        over["n_core"] = args.core
    prob = make_problem(args.config, **over)
    plan = e2.E2Problem.from_problem(prob)
    plan.set_arithmetic(args.arith == "sliced")
    couplings = float(plan.q_per_class.sum()) * plan.n_roots
    fbytes = 16.0 * (prob.Bc.shape[0] + (prob.Bx.shape[0] if prob.ham != "DC" else 0)) * prob.n * prob.n
    t = e2.device_inputs(prob, prob.X0, device=dev)
    c, E0_ref, iters = plan.reference_solve(t["h"], t["B_c"], t["c"], t["B_x"], t["w_x"], lam=t["lam"], tol=1e-10)
    t["c"] = c
    torch.cuda.synchronize()
    peak_dmma, peak_dfma = e2.fp64_peak(dev)
    # column tiles: time plain against compacted per class once, keep the faster
    tune = plan.autotune(**t) if not args.no_autotune else {}
    col_tiles = {}
    for k in (2, 4, 5, 6):
        tiles, krows, used = plan.class_tiles(k)
        if tiles:
            col_tiles[CLASS_NAMES[k]] = {"used": used, "compacted_share": krows / (tiles * _kpad(prob, k)),
                                         "autotune_ms": list(tune.get(k, ()))}
    stream = torch.cuda.current_stream(dev)

    fw = _timed_forward(plan, t, args.steps, args.warmup, stream, ws, dist, dev, clocks=ClockSampler(local),
                        shard=shard)
    ms = fw["ms"]
    jobs = 1 if shard else ws   # whole-job work per step: one job split over the ranks, or ws replicas
    roof = _roofline(prob, plan, fw, peak_dmma, peak_dfma)
    aux, aux_warm = _aux_steps(args, ms)

    # forward + backward in one pass (E2 and dE2/d(h, c, B, lambda), V formed
    # once) against forward alone
    fwdbwd = None
    if not args.no_backward and shard:
        fwdbwd = {"skipped": "the adjoint runs unsharded; fwd+bwd is measured at N = 1"}
    elif not args.no_backward:
        bms, E2vg = _timed_fwd_bwd(plan, t, aux, aux_warm, stream, ws, dist, dev)
        fwdbwd = {"ms_fwd": ms, "ms_fwd_bwd": bms, "ratio_fwd_bwd_over_fwd": bms / ms, "steps": aux,
                  "warmup": aux_warm, "E2_bitwise_equal_to_forward": bool(torch.equal(E2vg, fw["E2"])),
                  "gradients": "E2 with dE2/dh, dE2/dB (all factors, Hermitian), dE2/dc, dE2/dlambda from one "
                               "e2_backward call; V recomputed, never stored"}

    # end to end through the public API: pinned host inputs -> device, forward, E2 -> host
    e2e = None
    if not args.no_e2e:
        host = {k: (v.cpu().pin_memory() if torch.is_tensor(v) else v) for k, v in t.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values() if torch.is_tensor(v))
        dev_in = {k: (torch.empty_like(v, device=dev) if torch.is_tensor(v) else v) for k, v in host.items()}
        out_host = torch.empty(plan.n_roots, dtype=torch.float64).pin_memory()

        fwd_in = _forward_fn(plan, dev_in, shard, dist)

        def e2e_step():
            for k, v in host.items():
                if torch.is_tensor(v):
                    dev_in[k].copy_(v, non_blocking=True)
            E2_, _, _ = fwd_in()
            out_host.copy_(E2_, non_blocking=True)

        for _ in range(aux_warm):
            e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(aux):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ems = max_over_ranks(s0.elapsed_time(s1) / aux, ws, dist, dev)
        e2e = {"value": jobs * couplings / (ems * 1e-3), "unit": "couplings/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(out_host.numel() * 8), "ms_per_step": ems, "steps": aux}
        del dev_in, host

    # integral formation alone (step a5 as a workload of its own)
    integ = None
    if not args.no_integrals:
        integ = _timed_integrals(plan, prob, t, aux, aux_warm, stream, ws, dist, dev, peak_dmma)

    # the other arithmetic on the same workload (emulated when the headline is FP64)
    alt = None
    other = "sliced" if args.arith == "fp64" else "fp64"
    if not args.no_alt:
        plan.set_arithmetic(other == "sliced")
        if plan.arithmetic() == other:
            fa = _timed_forward(plan, t, aux, aux_warm, stream, ws, dist, dev, shard=shard)
            alt = {"arith": other, "dtype": ARITH_DTYPE[other], "value": jobs * couplings / (fa["ms"] * 1e-3),
                   "unit": "couplings/s", "ms_per_step": fa["ms"], "steps": aux, "warmup": aux_warm,
                   "arithmetic": _arith_parts(plan, fa["present"]),
                   "E2": float(fa["E2"].cpu()[0]),
                   "max_abs_dE2_class_vs_headline": float((fa["E2c"] - fw["E2c"]).abs().max()),
                   "class_ms": {CLASS_NAMES[k]: fa["ktime"][k] for k in fa["present"]},
                   "roofline": _roofline(prob, plan, fa, peak_dmma, peak_dfma)}
            if not args.no_backward and not shard:
                abms, _ = _timed_fwd_bwd(plan, t, aux, aux_warm, stream, ws, dist, dev)
                alt["fwd_bwd"] = {"ms_fwd_bwd": abms, "ratio_fwd_bwd_over_fwd": abms / fa["ms"], "steps": aux}
        plan.set_arithmetic(args.arith == "sliced")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, n, dt, reps = oracle_rate(prob, seconds=args.cpu_seconds)
        cpu = {"value": r, "unit": "couplings/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n // reps} random external determinants of this workload (class-size weighted), "
                         f"V_K from the explicit Q H P row and H_KK each, timed {reps} times: {n} couplings "
                         f"in {dt:.1f} s"}

    if rank == 0:
        present = fw["present"]
        line = {"metric": METRIC, "value": jobs * couplings / (ms * 1e-3), "unit": "couplings/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": ARITH_DTYPE[args.arith],
                "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config] + (f" [profiling variant {over}]" if over else ""),
                           "couplings_per_step": int(couplings),
                           "roots": plan.n_roots, "reference": f"device Davidson, {iters} iterations",
                           "l2": f"inputs larger than L2: the {fbytes / 1e6:.0f} MB factor set is re-read every step",
                           "arithmetic": _arith_parts(plan, present),
                           "column_tiles": col_tiles,
                           "E2": float(fw["E2"].cpu()[0]), "E2_hex": float(fw["E2"].cpu()[0]).hex(),
                           "E0": float(fw["E0"].cpu()[0]),
                           "parallelism": (f"external space sharded over {ws} GPUs (NCCL sum of the partials)"
                                           if shard else f"{ws} independent replica(s)"),
                           "class_ms": {CLASS_NAMES[k]: fw["ktime"][k] for k in present},
                           "per_class": _per_class(prob, plan, fw, peak_dmma, peak_dfma)},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fwd_bwd": fwdbwd, "alt_arithmetic": alt,
                "integrals": integ,
                "gpu_launches": fw["launches"] * args.steps,
                "clocks": fw["clocks"], "fp64_peaks_tflops": {"dmma": peak_dmma, "dfma": peak_dfma}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--config", default="ar_dcb_das", choices=sorted(WORKLOADS),
                    help="ar_dcb_das (the largest workload whose K forwards fit the run) is the benchmark workload; "
                         "the others run as evidence / profiling variants")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plan's default column tiles")
    ap.add_argument("--arith", default="fp64", choices=["fp64", "sliced"],
                    help="arithmetic of the headline: fp64 (the library default) or the emulated sliced form")
    ap.add_argument("--no-alt", action="store_true", help="skip the timing of the other arithmetic")
    ap.add_argument("--no-integrals", action="store_true", help="skip the timing of the integral formation alone")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: N independent replicas of the whole job instead of one sharded job")
    ap.add_argument("--aux-steps", type=int, default=0,
                    help="steps of the fwd+bwd, end-to-end and other-arithmetic timings (0: automatic)")
    ap.add_argument("--aux-seconds", type=float, default=30.0,
                    help="automatic aux steps: the headline's K, capped at about this much timed work")
    ap.add_argument("--roots", type=int, default=0, help="override the root count (batch evidence runs)")
    ap.add_argument("--batch", action="store_true",
                    help="evidence run: the 3 Hamiltonians x 3 frozen cutoffs of --config batched in one "
                         "graph-captured launch against sequential forwards")
    ap.add_argument("--roots-per-launch", type=int, default=0,
                    help="batch evidence run: roots of every job per persistent launch (0: all in one)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="oracle work per cpu_baseline sample (the sample is sized to about this long)")
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    ap.add_argument("--core", type=int, default=0, help="override the core spinor count (slices)")
    ap.add_argument("--virt", type=int, default=0,
                    help="override the virtual spinor count: a smaller variant with the same tile shapes, for "
                         "profiler captures of the backward (its workspace scales with the virtual pairs)")
    ap.add_argument("--factors", type=int, default=0,
                    help="override the Coulomb factor count (extra set = half); a small-memory variant with the "
                         "same class shapes, for profiler captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())

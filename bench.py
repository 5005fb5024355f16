#!/usr/bin/env python3
"""Throughput of the Epstein-Nesbet second-order energy on B300.

Metric: E2 perturber couplings/s (FP64).  A coupling is one external
determinant K (per root) whose V_K = <K|H|Psi> is formed and whose
|V_K|^2 / (E0 - H_KK) is reduced.  One step = one full e2_forward over every
external class of the workload (all of Q), inputs resident in HBM.

Default workload: the Ne-shaped DCG problem (2 core spinors, CAS 8e in 16
active spinors = 12,870 reference determinants, 200 virtual spinors,
400 Coulomb + 200 Gaunt factors, one root), 880,539,088 couplings per step.
Its factor inputs (456 MB) are larger than L2 and every step re-reads them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own GPU (independent
replicas, weak scaling); no data crosses between ranks.
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


def _sample_ks(prob, n, rng):
    """n random external determinants of the workload, drawn with the class
    sizes as weights: (holes, particles, active string)."""
    from math import comb
    nc = [k for k in range(prob.n_core) if not prob.frozen[k]]
    nv = [v for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v]]
    cls, w = [], []
    for h in range(3):
        for p in range(3):
            ne = prob.n_elec + h - p
            if (h, p) == (0, 0) or ne < 0 or ne > prob.n_act:
                continue
            cls.append((h, p, ne))
            w.append(comb(len(nc), h) * comb(len(nv), p) * comb(prob.n_act, ne))
    w = np.array(w, float) / sum(w)
    pick = rng.choice(len(cls), size=n, p=w)
    nh, hs, npp, ps, acts = [], [], [], [], []
    for k in pick:
        h, p, ne = cls[k]
        I = sorted(rng.choice(nc, size=h, replace=False).tolist()) if h else []
        S = sorted(rng.choice(nv, size=p, replace=False).tolist()) if p else []
        A = rng.choice(prob.n_act, size=ne, replace=False)
        nh.append(h), npp.append(p)
        hs.append(I + [0] * (2 - h)), ps.append(S + [0] * (2 - p))
        acts.append(int(sum(1 << int(t) for t in A)))
    return nh, hs, npp, ps, acts


def oracle_rate(prob, seconds=15.0, seed=0):
    """Couplings/s of the oracle on a bounded random sample of the workload's
    external determinants (V_K from the explicit Q H P row and H_KK), on all
    host cores."""
    from oracle import Oracle
    o = Oracle(prob, use_eri_cache=False)
    c = prob.X0[:1] / np.linalg.norm(prob.X0[:1])
    o.set_c(c)
    rng = np.random.default_rng(seed)
    E0 = np.zeros(1)
    n = 256
    while True:   # calibrate the sample size to about `seconds` of work
        ks = _sample_ks(prob, n, rng)
        t0 = time.perf_counter()
        o.couplings(E0, *ks)
        dt = time.perf_counter() - t0
        if dt >= 0.2 * seconds or n >= 2_000_000:
            break
        n *= 4
    n = int(max(256, min(4_000_000, n * seconds / max(dt, 1e-3))))
    args = _sample_ks(prob, n, rng)
    t0 = time.perf_counter()
    o.couplings(E0, *args)
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    """The oracle arm: each step times the oracle on a bounded sample of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from e2_inputs import make_problem
    prob = make_problem(args.config)
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_rate(prob, seconds=args.ref_seconds, seed=1)
    rates, ns, dts = [], [], []
    for s in range(args.steps):
        r, n, dt = oracle_rate(prob, seconds=args.ref_seconds, seed=100 + s)
        rates.append(r), ns.append(n), dts.append(dt)
    value = sum(ns) / sum(dts)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "couplings/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "couplings_per_step": int(sum(ns) / len(ns))},
            "cpu_baseline": {"value": value, "unit": "couplings/s", "cores": cores, "kind": "oracle",
                             "sample": f"{int(sum(ns) / len(ns))} random external determinants per step "
                                       f"(class-size weighted), V_K and H_KK each"},
            "e2e": {"value": value, "unit": "couplings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched evidence run: the 3 Hamiltonians x 3 frozen cutoffs of a workload
    shape (all roots of each) in one e2_batch_forward, captured in a CUDA
    graph and replayed, against the same jobs' e2_forward calls one after
    another.  Prints one JSON line with "mode": "batch"."""
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
    torch.cuda.empty_cache()   # the batch holds all jobs' layouts in one workspace
    batch = e2.E2Batch([p for *_, p, _ in jobs])
    batch.prepare(dev)
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
            "gpu_launches": sum(p.launch_count() for *_, p, _ in jobs)}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    import paper_2608_11529_b300 as e2
    from e2_inputs import make_problem
    over = dict(Lc=args.factors, Lx=args.factors // 2) if args.factors else {}
    if args.virt:
        over["n_virt"] = args.virt
    if args.core:
        over["n_core"] = args.core
    prob = make_problem(args.config, **over)
    plan = e2.E2Problem.from_problem(prob)
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

    # warm-up
    for _ in range(args.warmup):
        plan.forward(**t)
    torch.cuda.synchronize()
    launches = plan.launch_count()

    # per-step event pairs around each class kernel (handles materialised here)
    evs = []
    for _ in range(args.steps):
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(9)]
        for a, b in pairs:
            a.record()
            b.record()
        evs.append(pairs)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream(dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("forward")   # ncu --nvtx --nvtx-include "forward/" selects these launches
    start.record(stream)
    for s in range(args.steps):
        plan.set_events(evs[s])
        E2, E2c, E0 = plan.forward(**t)
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    plan.set_events(None)
    ms = max_over_ranks(start.elapsed_time(end) / args.steps, ws, dist, dev)
    E2dev = E2.clone()

    # per-class kernel times (root 0) over the timed region, summed per kernel
    present = [k for k in range(9) if plan.q_per_class[k] > 0]
    ktime = {k: sum(evs[s][k][0].elapsed_time(evs[s][k][1]) for s in range(args.steps)) / args.steps for k in present}
    sliced = {k for k in GEMM_CLASSES if k in present and plan.contraction(k)[0]}
    kern = {k: ("k_class_oz" if k in sliced else KERNEL_OF_CLASS[k]) for k in present}
    if 8 in present and plan.contraction(8)[0]:
        kern[8] = "k_class22_df"  # class (2,2) in float-float
    ksum = {}
    for k in present:
        ksum[kern[k]] = ksum.get(kern[k], 0.0) + ktime[k]
    dom_kernel = max(ksum, key=ksum.get)
    classes = [k for k in present if kern[k] == dom_kernel]
    if dom_kernel == "k_class_oz":
        # the sliced method's tensor work: 15 slice pairs (levels 2..6 of five
        # slices per operand), each a real product of length 2K into the two
        # real outputs (Re V, Im V) of a coupling: 15 * 2 * 2K * 2 = 120 K bf16
        # flops per coupling; peak: the measured bf16 rate, sustained (the
        # kernel runs inside a long step)
        mp = _measured_peaks()
        peak_bf16 = mp.get("bf16_tflops_sustained") or 1400.0
        flops = sum(120.0 * plan.q_per_class[k] * _kdim(prob, k) for k in classes)
        t_ms = sum(ktime[k] for k in classes)
        achieved = flops / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_bf16, "unit": "TFLOP/s",
                "frac": achieved / peak_bf16, "traffic": _traffic("k_class_oz"),
                "traffic_scope": "DRAM bytes per step over the kernel's launches (ncu, the (0,2) and (1,2) launches)",
                "kernel": "k_class_oz classes " + " ".join(CLASS_NAMES[k] for k in classes),
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"
                                if mp.get("bf16_tflops_sustained") else "fallback 1.4 PFLOP/s sustained bf16"),
                "algorithmic_flops_per_step": flops, "ms_per_step": t_ms,
                "launches_per_step": len(classes),
                "couplings_per_s": sum(plan.q_per_class[k] for k in classes) / (t_ms * 1e-3),
                "flops_per_coupling": "120 K bf16 (15 slice pairs x 2 real outputs x real length 2K x 2)"}
    elif dom_kernel == "k_class_gemm":
        # complex products by Gauss's three real products: 6 real flops per
        # complex multiply-add, K of them per coupling; with column tiles K is
        # each tile's compacted length (the products the kernel executes)
        flops = 0.0
        for k in classes:
            f = 6.0 * plan.q_per_class[k] * _kdim(prob, k)
            tiles, krows, used = plan.class_tiles(k)
            if used:
                f = 6.0 * (plan.q_per_class[k] / _ncols(prob, plan, k)) * krows * 64
            flops += f
        t_ms = sum(ktime[k] for k in classes)
        achieved = flops / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_dmma, "unit": "TFLOP/s",
                "frac": achieved / peak_dmma, "traffic": _traffic("k_class_gemm"),
                "kernel": "k_class_gemm classes " + " ".join(CLASS_NAMES[k] for k in classes), "peak_source":
                "measured on this GPU: mma.sync m16n8k8 f64 burst (e2_fp64_peak)",
                "algorithmic_flops_per_step": flops, "ms_per_step": t_ms, "launches_per_step": len(classes),
                "flops_per_coupling": "6 K (3 real products per complex product, K = contraction length; "
                                      "with column tiles, each tile's compacted K)"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": peak_dfma, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": dom_kernel}
    roof["kernel_ms_per_step"] = ksum

    # forward + backward in one pass (E2 and dE2/d(h, c, B, lambda), V formed
    # once) against forward alone
    fwdbwd = None
    if not args.no_backward:
        for _ in range(2):
            plan.value_and_grad(**t)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("fwd_bwd")   # ncu --nvtx --nvtx-include "fwd_bwd/" selects these launches
        b0.record(stream)
        for _ in range(args.steps):
            vg = plan.value_and_grad(**t)
        b1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        bms = max_over_ranks(b0.elapsed_time(b1) / args.steps, ws, dist, dev)
        same = bool(torch.equal(vg[0], E2dev)) if E2dev is not None else None
        fwdbwd = {"ms_fwd": ms, "ms_fwd_bwd": bms, "ratio_fwd_bwd_over_fwd": bms / ms,
                  "E2_bitwise_equal_to_forward": same,
                  "gradients": "E2 with dE2/dh, dE2/dB (all factors, Hermitian), dE2/dc, dE2/dlambda from one "
                               "e2_backward call; V recomputed, never stored"}

    # end to end through the public API: pinned host inputs -> device, forward, E2 -> host
    e2e = None
    if not args.no_e2e:
        host = {k: (v.cpu().pin_memory() if torch.is_tensor(v) else v) for k, v in t.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values() if torch.is_tensor(v))
        dev_in = {k: (torch.empty_like(v, device=dev) if torch.is_tensor(v) else v) for k, v in host.items()}
        out_host = torch.empty(plan.n_roots, dtype=torch.float64).pin_memory()

        def e2e_step():
            for k, v in host.items():
                if torch.is_tensor(v):
                    dev_in[k].copy_(v, non_blocking=True)
            E2_, _, _ = plan.forward(**dev_in)
            out_host.copy_(E2_, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ems = max_over_ranks(s0.elapsed_time(s1) / args.steps, ws, dist, dev)
        e2e = {"value": ws * couplings / (ems * 1e-3), "unit": "couplings/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(out_host.numel() * 8), "ms_per_step": ems}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, n, dt = oracle_rate(prob, seconds=args.cpu_seconds)
        cpu = {"value": r, "unit": "couplings/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} random external determinants of this workload (class-size weighted), "
                         f"V_K from the explicit Q H P row and H_KK each, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": ws * couplings / (ms * 1e-3), "unit": "couplings/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config] + (f" [profiling variant {over}]" if over else ""),
                           "couplings_per_step": int(couplings),
                           "roots": plan.n_roots, "reference": f"device Davidson, {iters} iterations",
                           "l2": f"inputs larger than L2: the {fbytes / 1e6:.0f} MB factor set is re-read every step",
                           "arithmetic": {
                               **{CLASS_NAMES[k]: ("sliced bf16 + float-float epilogue" if plan.contraction(k)[0]
                                                   else "fp64") for k in present if k in GEMM_CLASSES},
                               **({"(2,2)": "float-float" if plan.contraction(8)[0] else "fp64"} if 8 in present
                                  else {}),
                               "gather classes": "fp64",
                               "integral products": "sliced bf16" if plan.contraction(-1)[0] else "fp64",
                               "adjoint products": "sliced bf16 (4 slices)" if plan.contraction(-2)[0] else "fp64"},
                           "column_tiles": col_tiles,
                           "E2": float(E2.cpu()[0]), "E0": float(E0.cpu()[0]),
                           "class_ms": {CLASS_NAMES[k]: ktime[k] for k in present}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fwd_bwd": fwdbwd,
                "gpu_launches": launches * args.steps,
                "clocks": clk, "fp64_peaks_tflops": {"dmma": peak_dmma, "dfma": peak_dfma}}
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
    ap.add_argument("--config", default="ne_dcg", choices=sorted(WORKLOADS),
                    help="ne_dcg is the benchmark workload; the others run as evidence / profiling variants")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plan's default column tiles")
    ap.add_argument("--roots", type=int, default=0, help="override the root count (batch evidence runs)")
    ap.add_argument("--batch", action="store_true",
                    help="evidence run: the 3 Hamiltonians x 3 frozen cutoffs of --config batched in one "
                         "graph-captured launch against sequential forwards")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="oracle work per cpu_baseline sample (the sample is sized to about this long)")
    ap.add_argument("--ref-seconds", type=float, default=6.0)
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

"""Benchmark of the GB300 local-trace path (one JSON line on rank 0).

One step = one evaluation of the whole batch: sector walk and level-0
bounds, the chain products with fused propagators, renormalisation,
per-segment refined bounds and early rejects, final traces and the
per-chain combine.

Default workload: the uneven mixed batch -- 2048 seeded chains drawn
uniformly from the 3-orbital t2g, 5-orbital d-shell and 7-orbital f-shell
impurities, orders uniform in 10..200, lazy bounds on with half the chains
rejected early -- in three-term split bf16 (BF16X3) on the tensor cores,
captured once as a CUDA graph and replayed per step.  `value` is
evaluations/s with the inputs resident in HBM; `e2e` is the same steps
timed from the host->device copy of the inputs (pinned host memory) to the
device->host copy of the results; `fp64` times the plain float64 path and
the mixed path on the same named subset of the batch (the like-for-like
speedup); `roofline` is the dominant kernel (k_trace_big) timed with CUDA
events captured inside the graph.  L2 is flushed (a 256 MiB write) between
steps, outside the timed region.  Multi-GPU (torchrun): every rank
evaluates its own batch (no collective on the data path; weak scaling);
timing is max over ranks.

--workload t2g|d5|f7|hubbard2|f45 times one impurity's batch instead, and
--impl reference times the FP64 CPU oracle (the reference arm here) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# --precision names and their ctq precision codes (ctq.FP64 = 0, TF32 = 1, BF16X3 = 2, TF32X3 = 3).
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16x3": 2, "tf32x3": 3, "f32x2": 4}
METRIC = "local-trace evals/s and TFLOP/s vs peak, FP64 vs mixed at stated error, 1×GB300"
WORKLOAD_TEXT = {
    "t2g": "3-orbital t2g Kanamori (6 spin-orbitals, Fock dim 64, 16 (N_dn,N_up) sectors, blocks<=9), "
           "U=5, J=0.7, beta=50, real FP64; 4096 chains, order ~Poisson(40), tau uniform",
    "hubbard2": "2-orbital Kanamori (4 spin-orbitals, 9 sectors), U=4, J=0.5, mu=U/2, beta=10; 64 chains, k in 8..20",
    "d5": "5-orbital d-shell Slater-Condon (10 spin-orbitals, 36 sectors, largest block 100), U=8, J=1, "
          "real CF sigma=0.1, beta=40; 1024 chains, order ~Poisson(60)",
    "mixed": "uneven mixed batch: 2048 chains over the t2g, d5 and f7 models (uniform), orders uniform in 10-200, "
             "lazy bounds on, fair coin per chain: threshold +inf (reject at level 0) or -inf (full trace, accepted)",
    "f7": "7-orbital f-shell Slater-Condon with SOC 0.3 and complex CF sigma=0.05 (14 spin-orbitals, N in {4,5,6}, "
          "sectors 1001/2002/3003, complex), U=4.5, J=0.5, beta=40; 256 chains, order ~Poisson(80)",
}
WORKLOAD_TEXT["f45"] = ("f shell of the f7 model restricted to N in {4,5} (sectors 1001/2002, complex), mu where "
                        "E_gs(4) = E_gs(5); 2 chains of 80 operators, width-1 particle-number walk (profiling case)")
CPU_SAMPLE = {"t2g": 4096, "hubbard2": 64, "d5": 24, "f7": 1, "mixed": 4096}  # cpu_baseline: chains cycled >= 10 s
CPU_SAMPLE_REF = {"t2g": 64, "hubbard2": 64, "d5": 2, "f7": 1, "mixed": 24}  # per step of --impl reference
FLUSH_BYTES = 256 << 20
DEFAULT_PRECISION = {"mixed": "bf16x3"}  # every other workload: fp64
# Chains of the mixed batch on which the float64 path and the mixed path are
# timed side by side (the first N of the batch).
FP64_SUBSET = 8


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def algorithmic_flops(imp, batch):
    """Real FP64-equivalent flops of the surviving strings (complex x4):
    for each surviving (c, q0): sum_{i=1}^{n-2} 2 d_{q_{i+1}} d_{q_i} d_{q0}
    + 2 d_{q0} d_{q_{n-1}} (the first operator only scales; the last needs only
    a diagonal).  Host accounting from the library's sector table."""
    dims, _, _, s = imp.sectors()
    if imp.n_alpha > s.shape[0]:  # Bulla operators 2 n_flav + f map sectors as c_f (code 2 f)
        s = s[[a if a < s.shape[0] else 2 * (a - s.shape[0]) for a in range(imp.n_alpha)]]
    C = batch.n_chains
    lens = np.diff(batch.offsets)
    nmax = int(lens.max()) if C else 0
    ops = np.full((C, max(nmax, 1)), -1, np.int64)
    for c in range(C):
        a, b = batch.offsets[c], batch.offsets[c + 1]
        ops[c, : b - a] = batch.op[a:b]
    total = 0.0
    n_items = 0
    for q0 in range(len(dims)):
        q = np.full(C, q0, np.int64)
        alive = np.ones(C, bool)
        fl = np.zeros(C)
        d0 = dims[q0]
        for i in range(nmax):
            act = alive & (i < lens)
            a = np.where(act, ops[:, i], 0)
            qn = np.where(act, s[a, np.maximum(q, 0)], q)
            alive &= ~(act & (qn < 0))
            qn = np.where(alive, qn, 0)
            mid = act & alive & (i >= 1) & (i <= lens - 2)
            fl += np.where(mid, 2.0 * dims[qn] * dims[q] * d0, 0.0)
            last = act & alive & (i == lens - 1) & (lens >= 2)
            fl += np.where(last, 2.0 * d0 * dims[q], 0.0)
            q = np.where(act & alive, qn, q)
        surv = alive & (q == q0)
        total += float(fl[surv].sum())
        n_items += int(surv.sum())
    return total * (4.0 if imp.is_complex else 1.0), n_items


def density_flops(imp, batch):
    """Real FP64-equivalent flops of the density-matrix estimator over the
    surviving strings (complex x4): the forward products A_i (the first
    operator only scales), the backward products B_i (the last only scales)
    and the interval products A_i B_i for 1 <= i <= n-1 (G_0 = B_0, G_n = A_n)."""
    dims, _, _, s = imp.sectors()
    total = 0.0
    for c in range(batch.n_chains):
        a, b = batch.offsets[c], batch.offsets[c + 1]
        ops = batch.op[a:b]
        n = len(ops)
        for q0 in range(len(dims)):
            path, q = [q0], q0
            for al in ops:
                q = int(s[al, q])
                if q < 0:
                    break
                path.append(q)
            if q < 0 or q != q0:
                continue
            d0 = float(dims[q0])
            d = [float(dims[x]) for x in path]
            if n == 0:
                continue
            total += d[1] * d0 + sum(2.0 * d[i] * d[i - 1] * d0 for i in range(2, n + 1))
            total += d0 * d[n - 1] + sum(2.0 * d0 * d[i + 1] * d[i] for i in range(0, n - 1))
            total += sum(2.0 * d[i] * d[i] * d0 for i in range(1, n))
    return total * (4.0 if imp.is_complex else 1.0)


def one_pass_ratio_flops(imp, batch):
    """Real FP64-equivalent flops of the one-pass static ratios over the
    surviving strings (complex x4): the forward products A_i (the first
    operator only scales), the backward products (the last only scales) and,
    per annihilator, the product Y Q and its trace against P A."""
    dims, _, _, s = imp.sectors()
    nf2 = s.shape[0]
    total = 0.0
    for c in range(batch.n_chains):
        a, b = batch.offsets[c], batch.offsets[c + 1]
        ops = batch.op[a:b]
        n = len(ops)
        for q0 in range(len(dims)):
            path, q = [q0], q0
            for al in ops:
                q = int(s[al, q])
                if q < 0:
                    break
                path.append(q)
            if q < 0 or q != q0 or n == 0:
                continue
            d0 = float(dims[q0])
            d = [float(dims[x]) for x in path]
            total += d[1] * d0 + sum(2.0 * d[i] * d[i - 1] * d0 for i in range(2, n + 1))
            total += d0 * d[n - 1] + sum(2.0 * d0 * d[i + 1] * d[i] for i in range(0, n - 1))
            total += sum(2.0 * d0 * d[i + 1] * d[i] + 2.0 * d0 * d[i] for i in range(n)
                         if ops[i] < nf2 and ops[i] % 2 == 0)
    return total * (4.0 if imp.is_complex else 1.0)


def run_density(args, world, rank, local):
    """The reduced-density-matrix estimator (ctq_eval_density_matrices) on a
    workload: trace evaluation plus the estimator of every chain, float64."""
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mf, bf = w.WORKLOADS[args.workload]
    batch = bf(rank=rank)
    if args.chains:
        batch = batch.subset(range(min(args.chains, batch.n_chains)))
    imp = ctq.build_impurity(mf(), device=local)
    db = ctq.DeviceBatch(batch, device=dev)
    ev = ctq.DensityEvaluator(imp, batch.n_chains, db.max_ops, device=dev)
    flops = density_flops(imp, batch) + algorithmic_flops(imp, batch)[0]
    fp64_peak = ctq.probe_fma_rate(local, 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ev(db)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev(db)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks.stop()
    mean = statistics.mean(ms)
    achieved = flops / (mean * 1e-3) / 1e12
    line = {"metric": "density-matrix estimator evals/s (trace + rho per chain), FP64, 1xGB300",
            "value": batch.n_chains / (mean * 1e-3), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "n_chains": batch.n_chains,
                       "estimator": "reduced density matrix (Eq. ImpurityDensityMatrix)",
                       "l2": "flushed (256 MiB write) between steps"},
            "tflops": achieved, "algorithmic_flops_per_step": flops,
            "roofline": {"kernel": "k_trace<fp64> + k_rho", "bound": "alu", "achieved": achieved,
                         "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / (fp64_peak / 1e12),
                         "peak_source": "measured FP64 FMA rate (ctq_probe_fma_rate, this run)", "traffic": None},
            "gpu_launches": args.steps * 4, "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_improved(args, world, rank, local):
    """The static improved estimator for the self-energy (Eq.
    PImprovedEstimatorStatic) on a workload: every chain and, for each of its
    annihilators, the chain with that operator replaced by its Bulla operator
    [c_f, U] (ctq_eval_traces on both batches), then h^st = w^U / w
    (ctq_static_ratios).  The replaced sequences are built on the host once,
    before timing (they are the caller's input)."""
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mf, bf = w.WORKLOADS[args.workload]
    batch = bf(rank=rank)
    if args.chains:
        batch = batch.subset(range(min(args.chains, batch.n_chains)))
    imp = ctq.build_impurity(mf(), device=local)
    imp.add_bulla_operators()
    bu, chain, _ = w.bulla_sequences(batch, imp.n_flav)
    db = ctq.DeviceBatch(batch, device=dev)
    prec = PRECISIONS[args.precision]
    one_pass = args.estimator == "hst"
    if one_pass:
        if args.precision != "fp64":
            raise SystemExit("--estimator hst runs in fp64 (use hst-seq for the other precisions)")
        fe = ctq.FusedStaticEvaluator(imp, batch.n_chains, max(db.max_ops, 1), db.n_ops, device=dev)
        flops = algorithmic_flops(imp, batch)[0] + one_pass_ratio_flops(imp, batch)

        def step():
            fe(db)
        launches = ctq.launches_per_eval(imp, prec) + 1
        kernel = "k_trace<fp64> + k_rho<hst>"
    else:
        dbu = ctq.DeviceBatch(bu, device=dev)
        ev = ctq.StaticImprovedEvaluator(imp, batch.n_chains, bu.n_chains, max(db.max_ops, 1), precision=prec,
                                         device=dev)
        ch = torch.as_tensor(chain, device=dev)
        flops = algorithmic_flops(imp, batch)[0] + algorithmic_flops(imp, bu)[0]

        def step():
            ev(db, dbu, ch)
        launches = 2 * ctq.launches_per_eval(imp, prec) + 1
        kernel = "k_trace<fp64>" if args.precision == "fp64" else "trace kernels<" + args.precision + ">"
    fp64_peak = ctq.probe_fma_rate(local, 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks.stop()
    mean = statistics.mean(ms)
    achieved = flops / (mean * 1e-3) / 1e12
    line = {"metric": "static improved-estimator ratios h^st per second (Eq. PImprovedEstimatorStatic), 1xGB300",
            "value": bu.n_chains / (mean * 1e-3), "unit": "ratios/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision,
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "n_chains": batch.n_chains,
                       "replaced_sequences": bu.n_chains, "precision": args.precision,
                       "estimator": "static improved estimator, Bulla operators [c_f, U], "
                                    + ("one pass (forward / backward products)" if one_pass else "replaced sequences"),
                       "l2": "flushed (256 MiB write) between steps"},
            "tflops": achieved, "algorithmic_flops_per_step": flops,
            "roofline": {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / (fp64_peak / 1e12),
                         "peak_source": "measured FP64 FMA rate (ctq_probe_fma_rate, this run)", "traffic": None},
            "gpu_launches": args.steps * launches, "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_skiplist(args, world, rank, local):
    """The skip-list incremental trace (ctq_skiplist) on one configuration of
    a workload: W warm-up and K timed random pair moves (workloads.pair_move),
    each followed by ctq_skiplist_evaluate, against a fresh float64
    ctq_eval_traces of the same configuration (timed on the first and last
    configurations)."""
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mf, bf = w.WORKLOADS[args.workload]
    batch = bf(rank=rank)
    imp = ctq.build_impurity(mf(), device=local)
    tau, op = (np.asarray(x) for x in batch.chain(0))
    rng = np.random.default_rng(2010084820 + rank)
    if args.precision not in ("fp64", "bf16x3"):
        raise SystemExit("--estimator skiplist runs its products in fp64 or bf16x3")
    sl = ctq.SkipListTrace(imp, batch.beta, seed=11, precision=PRECISIONS[args.precision])
    stream = torch.cuda.current_stream()
    s_tab = imp.sectors()[3]

    def n_live(o):
        """Starting sectors whose string survives (integer walk on the sector table)."""
        q = np.arange(s_tab.shape[1])
        for a in o:
            q = np.where(q >= 0, s_tab[int(a), np.maximum(q, 0)], -1)
        return int(np.sum(q == np.arange(s_tab.shape[1])))

    def move(t, o):
        """A pair move whose configuration keeps a surviving string (a move
        that kills every string has weight 0 and would be rejected anyway;
        the N-truncated f shell rejects most moves this way)."""
        for _ in range(10000):
            mv = w.pair_move(rng, t, o, imp.n_flav, batch.beta)
            t2, o2 = w.apply_pair_move(mv, t, o)
            if n_live(o2) > 0:
                return mv, t2, o2
        raise RuntimeError("no surviving pair move found")

    def fresh(t, o):
        b = w.Batch(beta=batch.beta, offsets=np.array([0, len(t)], np.int32), tau=t, op=o)
        db = ctq.DeviceBatch(b, device=dev)
        ev = ctq.TraceEvaluator(imp, 1, max(1, len(t)), device=dev, precision=PRECISIONS[args.precision])
        ev(db)  # warm (first-call set-up)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev(db)
        e1.record(stream)
        e1.synchronize()
        r = ev.results(1)
        return e0.elapsed_time(e1) * 1e-3, float(r["log_abs"][0]), complex(*r["phase"][0])

    t0 = time.perf_counter()
    sl.set(tau, op)
    la, ph, st = sl.evaluate()
    build_s = time.perf_counter() - t0
    build_products = st["products"]
    fresh_first = fresh(tau, op)
    diffs = [abs(ph * math.exp(la - fresh_first[1]) - fresh_first[2])] if np.isfinite(fresh_first[1]) else []
    for _ in range(args.warmup):
        mv, tau, op = move(tau, op)
        (sl.remove(mv[1]) if mv[0] == "rem" else sl.insert(mv[1], mv[2]))
        sl.evaluate()
    clocks = ClockSampler(local)
    clocks.start()
    secs, prods, flops, n_ops, full, launches, rounds = [], [], [], [], [], [], []
    for _ in range(args.steps):
        mv, tau, op = move(tau, op)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        (sl.remove(mv[1]) if mv[0] == "rem" else sl.insert(mv[1], mv[2]))
        la, ph, st = sl.evaluate()  # synchronises the stream
        secs.append(time.perf_counter() - t1)
        prods.append(st["products"])
        flops.append(st["flops"])
        n_ops.append(len(tau))
        full.append((len(tau) - 1) * st["n_strings"])  # a full evaluation's products
        launches.append(st["launches"])
        rounds.append(st["rounds"])
    clocks.stop()
    fresh_last = fresh(tau, op)
    if np.isfinite(fresh_last[1]):
        diffs.append(abs(ph * math.exp(la - fresh_last[1]) - fresh_last[2]))
    per_move = statistics.mean(secs)
    fresh_s = 0.5 * (fresh_first[0] + fresh_last[0])
    fp64_peak = ctq.probe_fma_rate(local, 0)
    achieved = sum(flops) / sum(secs) / 1e12
    if args.precision == "fp64":
        sl_roofline = {"kernel": "k_sl_gemm (float64 SIMT)", "bound": "alu", "achieved": achieved,
                       "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / (fp64_peak / 1e12),
                       "peak_source": "measured FP64 FMA rate (ctq_probe_fma_rate, this run); achieved counts "
                                      "the products' flops over the whole move time", "traffic": None}
    else:
        sl_roofline = dict(roofline("bf16x3", achieved, fp64_peak, None), kernel="k_sl_tc (tcgen05 BF16X3)",
                           note="achieved counts the products' algorithmic flops over the whole move time")
    line = {"metric": f"skip-list incremental local trace: seconds per pair move, {args.precision.upper()}, 1xGB300",
            "value": per_move, "unit": "s/move", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * per_move, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else DTYPE_TEXT[args.precision], "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload] + " (first chain, random pair moves)",
                       "moves": "workloads.pair_move: insert or remove a pair between consecutive operators of "
                                "one flavour (Pauli-aware), redrawn until some string survives",
                       "mean_operators": statistics.mean(n_ops)},
            "products_per_move": statistics.mean(prods),
            "full_products": statistics.mean(full),  # (operators - 1) x surviving strings
            "build": {"seconds": build_s, "products": build_products},
            "fresh_eval_s": fresh_s, "fresh_eval": f"ctq_eval_traces, {args.precision}, the same configuration",
            "speedup_vs_fresh_eval": fresh_s / per_move,
            "max_rel_diff_vs_fresh": max(diffs) if diffs else None,
            "roofline": sl_roofline,
            "launches_per_move": statistics.mean(launches), "rounds_per_move": statistics.mean(rounds),
            "gpu_launches": int(sum(launches)), "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(x[1]) for x in self.samples if x[1].replace(".", "").isdigit()]
        mx = [float(x[2]) for x in self.samples if x[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for x in self.samples for i in range(4) if len(x) > 5 + i and "Active" in x[5 + i]
                          and "Not" not in x[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


KERNEL_SOURCES = {
    "small": ("trace_fp64.cu", "device_common.cuh", "two_float.cuh", "exp_tang.cuh"),
    "big": ("trace_big.cu", "big_common.cuh", "tc_ptx.cuh", "device_common.cuh"),
}


def source_hash(kind: str = "small") -> str:
    """Hash of a dominant kernel's code: the shared-memory FP64 kernel
    ("small") or the large-block tensor-core kernel ("big"), with the
    headers it includes."""
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2010_08482_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_traffic(kernel: str, workload: str, kind: str = "small"):
    """DRAM bytes per launch from a committed ncu summary
    (profiles/<kernel>_<workload>.md, lines "- key: value"), if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("source_sha256", "")[:16] != source_hash(kind)[:16]:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def host_cpu():
    """(logical core count, CPU model name) of this host."""
    n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return n, model or "unknown"


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
               "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_subprocess(spec: dict, threads: int, timeout: float = 1200.0) -> dict:
    """Runs oracle_worker(spec) in a child interpreter whose BLAS / OpenMP
    thread counts are fixed to `threads` through its environment (set before
    numpy loads) and which sees no GPU; returns the worker's JSON result."""
    env = dict(os.environ)
    for v in THREAD_VARS:
        env[v] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", json.dumps(spec)],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError("oracle worker failed: " + out.stderr[-2000:])
    for line in out.stdout.splitlines():
        if line.startswith("ORACLE "):
            return json.loads(line[len("ORACLE "):])
    raise RuntimeError("oracle worker printed no result: " + out.stdout[-500:])


MIXED_ORACLE_NOTE = ("the t2g and d5 chains of the mixed batch in batch order (the f-shell chains are left out: the "
                     "oracle's f-shell model takes minutes to build and about a minute per chain), each decided "
                     "as the method does: level-0 bound against the threshold, then the full trace")


def oracle_worker(spec: dict) -> dict:
    """The FP64 oracle, as it stands, on chains of a workload (runs in the
    child process of oracle_subprocess).  spec: workload; then either
    per_step + n_steps (per-step rates, the reference arm) or min_s + n_min
    (one rate over at least n_min evaluations and min_s seconds, cycling
    through the chains, and the first pass's results).  Chains with a
    threshold are decided as the method does: the level-0 bound first, the
    full trace only if the bound reaches the threshold."""
    from oracle import atom
    from oracle import trace as OT
    from paper_2010_08482_gb300 import workloads as w
    name = spec["workload"]
    if name == "mixed":
        batch, coin = w.batch_mixed()
        ps = {0: w.model_t2g(), 1: w.model_d5()}
        ms = {mi: atom.Model(p) for mi, p in ps.items()}
        chains = [c for c in range(batch.n_chains) if int(batch.model[c]) in ps]

        def job(c):
            mi = int(batch.model[c])
            return ms[mi], ps[mi].beta, (math.inf if coin[c] else -math.inf)
    else:
        mf, bf = w.WORKLOADS[name]
        batch = bf()
        m = atom.Model(mf())
        chains = list(range(batch.n_chains))

        def job(c):
            return m, batch.beta, None
    if spec.get("first"):
        chains = chains[: int(spec["first"])]

    def one(c):
        m, beta, T = job(c)
        tau, ops = batch.chain(c)
        if T is not None:
            logs = [OT.level0_bound(m, tau, ops, q0, beta) for q0 in range(m.n_sec)]
            logs = [x for x in logs if x != -math.inf]
            if not logs:
                return ["zero", -math.inf, 0.0, 0.0]
            mx = max(logs)
            if mx + math.log(sum(math.exp(x - mx) for x in logs)) < T:
                return ["rejected_early", None, None, None]
        r = OT.trace_chain(m, tau, ops, beta=beta)
        ph = complex(r["phase"])
        st = "ok" if T is None else ("accepted" if OT.decide(r["log_abs"], T) else "rejected")
        return [st, r["log_abs"], ph.real, ph.imag]

    out = {"chains_in_sample": len(chains), "blas_threads": {v: os.environ.get(v) for v in THREAD_VARS}}
    if "per_step" in spec:
        rates, pos = [], 0
        for _ in range(int(spec["n_steps"])):
            t0 = time.perf_counter()
            for _ in range(int(spec["per_step"])):
                one(chains[pos % len(chains)])
                pos += 1
            rates.append(int(spec["per_step"]) / (time.perf_counter() - t0))
        out["step_rates"] = rates
        return out
    results = {}
    count, t0 = 0, time.perf_counter()
    n_min = int(spec.get("n_min", len(chains)))
    while True:
        c = chains[count % len(chains)]
        r = one(c)
        if count < len(chains):
            results[str(c)] = r
        count += 1
        dt = time.perf_counter() - t0
        if count >= min(n_min, len(chains)) and dt >= float(spec.get("min_s", 0.0)):
            break
    out.update({"rate": count / dt, "count": count, "seconds": dt, "results": results})
    return out


def cpu_baseline_leg(workload: str, n_first: int, min_s: float = 10.0, n_min: int = 0):
    """The oracle on a bounded sample of the workload (at least min_s seconds
    and n_min evaluations, default one pass over the first n_first chains),
    once on one thread and once on every host core (BLAS / OpenMP threads
    fixed per child process).  Returns (cpu_baseline dict, the one-thread
    run's per-chain results)."""
    ncpu, model = host_cpu()
    spec = {"workload": workload, "first": n_first, "min_s": min_s, "n_min": n_min or n_first}
    one = oracle_subprocess(spec, threads=1)
    allc = oracle_subprocess(dict(spec, min_s=min_s), threads=ncpu)
    what = MIXED_ORACLE_NOTE if workload == "mixed" else f"the first {one['chains_in_sample']} chains of the workload"
    base = {"value": allc["rate"], "unit": "evals/s", "cores": ncpu, "kind": "oracle",
            "sample": f"{allc['count']} chain evaluations ({allc['seconds']:.1f} s) cycling over {what}; NumPy FP64 "
                      f"with BLAS / OpenMP threads = {ncpu} (all host cores)",
            "one_thread": {"value": one["rate"], "cores": 1,
                           "sample": f"{one['count']} evaluations ({one['seconds']:.1f} s) of the same chains, "
                                     "BLAS / OpenMP threads = 1"},
            "host": {"cpu_count": ncpu, "cpu_model": model}}
    return base, one["results"]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle, as it stands, on the host cores
    (BLAS / OpenMP threads = all cores), a bounded sample of the workload per
    step; rank 0 only."""
    if rank != 0:
        return
    workload = args.workload
    per_step = CPU_SAMPLE_REF.get(workload, 8)
    ncpu, model = host_cpu()
    res = oracle_subprocess({"workload": workload, "per_step": per_step, "n_steps": args.warmup + args.steps},
                            threads=ncpu)
    rates = res["step_rates"][args.warmup:]
    value = statistics.mean(rates)
    what = MIXED_ORACLE_NOTE if workload == "mixed" else f"the {res['chains_in_sample']} chains of the workload"
    sample = (f"{per_step} chain evaluations per step cycling over {what}; NumPy FP64, BLAS / OpenMP threads = "
              f"{ncpu} (all host cores of a {model})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_step / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[workload], "parallelism": "host cores, 1 process"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": ncpu, "kind": "oracle", "sample": sample,
                         "host": {"cpu_count": ncpu, "cpu_model": model}},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class _Group:
    """One impurity's share of the mixed batch: its chains, device batch,
    evaluator, timing events (captured inside the graph) and pinned host
    copies of its inputs and results."""


def _err_stats(errs):
    if not errs:
        return None
    e = np.asarray(errs)
    return {"n": int(e.size), "max": float(e.max()), "p90": float(np.quantile(e, 0.9)), "median": float(np.median(e))}


def _rel_err(la, ph, la_ref, ph_ref):
    """|w - w_ref| / |w_ref| for values held as (log|w|, phase)."""
    if la_ref == -math.inf:
        return 0.0 if la == -math.inf else math.inf
    if not np.isfinite(la):
        return math.inf
    return abs(complex(ph[0], ph[1]) * math.exp(la - la_ref) - complex(ph_ref[0], ph_ref[1]))


def run_mixed(args, world, rank, local):
    """The uneven mixed batch (the default workload): chains of the t2g, d5
    and f7 impurities, one ctq_eval_traces per impurity, lazy bounds on,
    captured once as a CUDA graph and replayed per step.  The coin of each
    chain sets its threshold to +inf (every bound falls below it: rejected
    at level 0, before any product) or -inf (never rejected: full trace,
    accepted), which gives the workload's 50 % early rejects with known
    decisions."""
    import ctypes

    import torch
    from paper_2010_08482_gb300 import autotune
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.perf_counter()
    batch, coin = w.batch_mixed(rank=rank)
    if args.chains:
        keep = np.arange(min(args.chains, batch.n_chains))
        batch, coin = batch.subset(keep), coin[keep]
    params = [w.model_t2g(), w.model_d5(), w.model_f7()]
    prec = PRECISIONS[args.precision]
    stream = torch.cuda.current_stream()
    groups = []
    for mi, p in enumerate(params):
        idx = np.nonzero(batch.model == mi)[0]
        if idx.size == 0:
            continue
        g = _Group()
        g.name, g.idx = p.name, idx
        g.sub = batch.subset(idx)
        g.sub.beta = p.beta  # the mixed batch draws each chain's times in [0, beta) of its own model
        g.thr = np.where(coin[idx] == 1, np.inf, -np.inf)
        g.imp = ctq.build_impurity(p, device=local)
        g.db = ctq.DeviceBatch(g.sub, device=dev, log_threshold=g.thr)
        g.tuning = {}
        acc = np.nonzero(coin[idx] == 0)[0]
        if not args.no_autotune and acc.size:
            eng = autotune.engine(g.imp, prec)
            if eng != "fp64big":  # the float64 large-block kernel is FP64-pipe bound: nothing to tune
                piece = acc[:8] if eng == "big" else acc[:512]
                tdb = ctq.DeviceBatch(g.sub.subset(piece), device=dev, log_threshold=np.full(piece.size, -np.inf))
                g.tuning = autotune.tune(g.imp, tdb, prec, lazy=True, cache_path=args.autotune_cache,
                                         reps=2 if eng == "big" else 3)
        g.ev = ctq.TraceEvaluator(g.imp, g.sub.n_chains, g.db.max_ops, precision=prec, device=dev, tune=g.tuning)
        g.flops, g.items = algorithmic_flops(g.imp, g.sub.subset(acc))
        g.launches = ctq.launches_per_eval(g.imp, prec)
        g.events = [torch.cuda.Event(enable_timing=True) for _ in range(g.launches + 1)]
        for e in g.events:
            e.record(stream)  # materialise the cudaEvent_t handles
        g.ev_arr = (ctypes.c_void_p * len(g.events))(*[e.cuda_event for e in g.events])
        g.ev_ptr = ctypes.cast(g.ev_arr, ctypes.c_void_p).value
        n, n_ops = g.sub.n_chains, len(g.sub.tau)
        g.h_off = torch.as_tensor(np.asarray(g.sub.offsets, np.int32)).pin_memory()
        g.h_tau = torch.as_tensor(np.asarray(g.sub.tau, np.float64)).pin_memory()
        g.h_op = torch.as_tensor(np.asarray(g.sub.op, np.int32)).pin_memory()
        g.h_thr = torch.as_tensor(g.thr.astype(np.float64)).pin_memory()
        g.h_la = torch.empty(n, dtype=torch.float64).pin_memory()
        g.h_ph = torch.empty(2 * n, dtype=torch.float64).pin_memory()
        g.h_st = torch.empty(n, dtype=torch.int32).pin_memory()
        g.n_ops = n_ops
        g.kern_ms = []
        groups.append(g)
    n_chains = sum(g.sub.n_chains for g in groups)

    def step():
        for g in groups:
            g.ev(g.db, lazy=True, events=g.ev_ptr)

    step()  # eager first evaluation (also the library's first-call set-up)
    torch.cuda.synchronize()
    # The whole mixed evaluation (every impurity's memsets and plan / trace /
    # combine launches, with the timing events as event-record nodes) is
    # captured once as a CUDA graph and replayed per step.
    graph, graph_note = None, "captured once, replayed per step"
    try:
        cap_stream = torch.cuda.Stream(device=dev)
        cap_stream.wait_stream(stream)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=cap_stream):
            step()
        torch.cuda.synchronize()
        graph = gr
    except Exception as exc:  # capture refused: the same launches eagerly
        torch.cuda.synchronize()
        graph_note = f"eager ({type(exc).__name__}: {str(exc)[:80]})"
    run = graph.replay if graph is not None else step
    for _ in range(max(args.warmup - 1, 0)):
        run()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    e_start, e0, e1, e_end = (torch.cuda.Event(enable_timing=True) for _ in range(4))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms, e2e_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e_start.record(stream)
        for g in groups:  # this step's inputs, host (pinned) -> device
            g.db.offsets.copy_(g.h_off, non_blocking=True)
            g.db.tau[: g.n_ops].copy_(g.h_tau, non_blocking=True)
            g.db.op[: g.n_ops].copy_(g.h_op, non_blocking=True)
            g.db.log_threshold.copy_(g.h_thr, non_blocking=True)
        e0.record(stream)
        run()
        e1.record(stream)
        for g in groups:  # results, device -> host (pinned)
            n = g.sub.n_chains
            g.h_la.copy_(g.ev.log_abs[:n], non_blocking=True)
            g.h_ph.copy_(g.ev.phase[: 2 * n], non_blocking=True)
            g.h_st.copy_(g.ev.status[:n], non_blocking=True)
        e_end.record(stream)
        e_end.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        e2e_ms.append(e_start.elapsed_time(e_end))
        for g in groups:
            g.kern_ms.append([g.events[k].elapsed_time(g.events[k + 1]) for k in range(g.launches)])
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    clocks.stop()
    h2d = sum(g.h_off.numel() * 4 + g.h_tau.numel() * 8 + g.h_op.numel() * 4 + g.h_thr.numel() * 8 for g in groups)
    d2h = sum(g.h_la.numel() * 8 + g.h_ph.numel() * 8 + g.h_st.numel() * 4 for g in groups)

    ms = max_over_ranks(world, statistics.mean(step_ms), dev)
    e2e = max_over_ranks(world, statistics.mean(e2e_ms), dev)
    flops = sum(g.flops for g in groups)
    # decisions of the last step: coin 1 rejected at level 0, coin 0 accepted (or exactly zero)
    status, decisions_ok = {}, True
    for g in groups:
        st = g.h_st.numpy()
        status[g.name] = np.bincount(st + 1, minlength=6)[1:].tolist()
        c1 = coin[g.idx] == 1
        decisions_ok &= bool(np.all(st[c1] == ctq.CHAIN_REJECTED_EARLY))
        decisions_ok &= bool(np.all(np.isin(st[~c1], [ctq.CHAIN_ACCEPTED, ctq.CHAIN_ZERO])))
    # dominant kernel: the trace kernel of the group with the most work
    dom = max(groups, key=lambda g: g.flops)
    dom_ms = statistics.mean(k[1] for k in dom.kern_ms)
    big = dom.imp.is_complex or dom.imp.max_dim > 112
    achieved = dom.flops / (dom_ms * 1e-3) / 1e12
    fp64_peak = ctq.probe_fma_rate(local, 0)
    fp32_rate = ctq.probe_fma_rate(local, 1) if args.precision == "f32x2" else None
    kname = kernel_name(args.precision, big)
    # DRAM bytes per launch from a committed ncu summary of this kernel on the
    # f shell (profiles/k_trace_big_<precision>_f7.md), if current
    traffic = profile_traffic(f"k_trace_big_{args.precision}", "f7", "big") if big else None
    roof = roofline(args.precision, achieved, fp64_peak, traffic, big=big, fp32_rate=fp32_rate, sustained=True)
    roof["kernel"] = kname
    per_group = {g.name: {"chains": int(g.sub.n_chains), "evaluated": int(np.sum(coin[g.idx] == 0)),
                          "surviving_strings": int(g.items), "algorithmic_flops": g.flops,
                          "kernel_ms": {"plan": statistics.mean(k[0] for k in g.kern_ms),
                                        "trace": statistics.mean(k[1] for k in g.kern_ms),
                                        "combine": statistics.mean(k[2] for k in g.kern_ms)},
                          "launch_tuning": g.tuning or "library default"} for g in groups}
    line = {
        "metric": METRIC, "value": world * n_chains / (ms * 1e-3), "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_TEXT[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["mixed"] + (f" (first {n_chains} chains)" if args.chains else ""),
                   "n_chains": n_chains, "precision": args.precision, "groups": per_group,
                   "thresholds": "coin 1: +inf (rejected on the level-0 bound), coin 0: -inf (full trace, "
                                 "accepted)", "cuda_graph": graph_note,
                   "group_order": "one after another on one stream (t2g, d5, f7)",
                   "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "tflops": flops / (ms * 1e-3) / 1e12, "algorithmic_flops_per_step": flops,
        "roofline": roof,
        "e2e": {"value": world * n_chains / (e2e * 1e-3), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "timed": "the same steps, from the host->device copy of every group's offsets, times, operator "
                         "codes and thresholds (pinned) to the device->host copy of log|w|, phase and status"},
        "status_counts [ok, zero, rejected_early, accepted, rejected]": status,
        "decisions_as_expected": decisions_ok,
        "gpu_launches": args.steps * sum(g.launches for g in groups),
        "clocks": clocks.summary(), "wall_s_timed_region": wall, "setup_s": setup_s,
    }
    if rank == 0 and world == 1 and not args.no_fp64_subset:
        line["fp64"] = fp64_subset_leg(args, batch, coin, groups, dev, fp64_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, oracle_res = cpu_baseline_leg("mixed", CPU_SAMPLE["mixed"], min_s=10.0, n_min=1)
        line["cpu_baseline"] = base
        errs = {}
        for g in groups:
            e = []
            la, ph = g.h_la.numpy(), g.h_ph.numpy().reshape(-1, 2)
            for k, c in enumerate(g.idx):
                r = oracle_res.get(str(int(c)))
                if r is None or r[0] != "accepted":
                    continue
                e.append(_rel_err(la[k], ph[k], r[1], (r[2], r[3])))
            if e:
                errs[g.name] = _err_stats(e)
        line["error_vs_oracle"] = dict(errs, note="relative error |w - w_oracle| / |w_oracle| of the accepted chains "
                                                  "of the oracle's sample (t2g and d5; the f shell is compared with "
                                                  "the float64 GPU path in fp64)")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def fp64_subset_leg(args, batch, coin, groups, dev, fp64_peak):
    """The plain float64 path and the mixed path on the same chains: the first
    FP64_SUBSET chains of the mixed batch, one ctq_eval_traces per impurity
    on one stream, eager; also the mixed path's error on them against the
    float64 path."""
    import torch
    from paper_2010_08482_gb300 import ctq
    stream = torch.cuda.current_stream()
    n_sub = min(args.fp64_subset, batch.n_chains)
    legs = []
    for g in groups:
        loc = np.nonzero(g.idx < n_sub)[0]
        if loc.size == 0:
            continue
        sub = g.sub.subset(loc)
        db = ctq.DeviceBatch(sub, device=dev, log_threshold=g.thr[loc])
        acc = loc[coin[g.idx[loc]] == 0]
        legs.append((g, loc, db, algorithmic_flops(g.imp, g.sub.subset(acc))[0]))

    def timed(precision, reps):
        evs = [ctq.TraceEvaluator(g.imp, db.n_chains, max(1, db.max_ops), precision=precision, device=dev,
                                  tune=g.tuning if precision != ctq.FP64 else None) for g, _, db, _ in legs]

        def once():
            for ev, (_, _, db, _) in zip(evs, legs):
                ev(db, lazy=True)
        once()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            once()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        res = [ev.results(db.n_chains) for ev, (_, _, db, _) in zip(evs, legs)]
        return statistics.mean(ms), res

    prec = PRECISIONS[args.precision]
    ms64, r64 = timed(ctq.FP64, 1)
    msm, rm = timed(prec, 3)
    errs = {}
    for (g, loc, db, _), a, b in zip(legs, r64, rm):
        e = [_rel_err(b["log_abs"][k], b["phase"][k], a["log_abs"][k], a["phase"][k])
             for k in range(len(loc)) if a["status"][k] == ctq.CHAIN_ACCEPTED]
        if e:
            errs[g.name] = _err_stats(e)
    flops = sum(f for *_, f in legs)
    return {"subset": f"first {n_sub} chains of the mixed batch ("
                      + ", ".join(f"{g.name}: {len(loc)} chains, {int(np.sum(coin[g.idx[loc]] == 0))} evaluated"
                                  for g, loc, _, _ in legs) + "), same thresholds, eager launches",
            "fp64_evals_per_s": n_sub / (ms64 * 1e-3), "fp64_ms": ms64,
            "fp64_tflops": flops / (ms64 * 1e-3) / 1e12,
            "fp64_frac_of_fp64_rate": flops / (ms64 * 1e-3) / fp64_peak,
            "mixed_precision": args.precision, "mixed_evals_per_s": n_sub / (msm * 1e-3), "mixed_ms": msm,
            "speedup_mixed_over_fp64": ms64 / msm,
            "mixed_error_vs_fp64": dict(errs, note="relative error of the accepted chains against the float64 "
                                                   "path (itself held to 1e-12 of the oracle by the tests, plus "
                                                   "the eigensolver term for library-built impurities)")}


def f45_impurity(ctq, w, device: int):
    """The profiling case's impurity: the f shell with N in {4, 5}, mu at the
    point where the N = 4 and N = 5 ground states are degenerate, computed
    from a first build at mu = 0."""
    p0 = w.model_f45(0.0)
    imp0 = ctq.build_impurity(p0, device=device)
    _, N, Emin, _ = imp0.sectors()
    e4, e5 = float(Emin[N == 4].min()), float(Emin[N == 5].min())
    del imp0
    return ctq.build_impurity(w.model_f45(e5 - e4), device=device)


def main():
    if len(sys.argv) >= 3 and sys.argv[1] == "--oracle-worker":
        print("ORACLE " + json.dumps(oracle_worker(json.loads(sys.argv[2]))), flush=True)
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 6 for the mixed batch, about a minute of timed work; 20 otherwise)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default: 3 mixed, 5 otherwise)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default=None, choices=["fp64", "tf32", "tf32x3", "bf16x3", "f32x2"],
                    help="default: bf16x3 for the mixed batch, fp64 otherwise")
    ap.add_argument("--fp64-subset", type=int, default=FP64_SUBSET,
                    help="mixed batch: chains (the first N) timed in float64 and in the mixed precision")
    ap.add_argument("--no-fp64-subset", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chains", type=int, default=0, help="evaluate only the first N chains of the workload")
    ap.add_argument("--no-autotune", action="store_true", help="library-default launch configuration")
    ap.add_argument("--estimator", default="trace", choices=["trace", "rho", "hst", "hst-seq", "skiplist"],
                    help="trace: local traces (default); rho: traces plus the reduced-density-matrix estimator; "
                         "hst: the static improved-estimator ratio of every annihilator in one pass; "
                         "hst-seq: the same from traces of the replaced sequences; "
                         "skiplist: incremental traces of one configuration under random pair moves")
    ap.add_argument("--autotune-cache", default=None, help="JSON cache of tuned launch configurations")
    args = ap.parse_args()
    long_steps = args.workload == "mixed" and args.estimator == "trace"
    if args.steps is None:
        args.steps = 6 if long_steps else 20
    if args.warmup is None:
        args.warmup = 3 if long_steps else 5
    args.warmup = max(args.warmup, 3)
    if args.precision is None:
        args.precision = DEFAULT_PRECISION.get(args.workload, "fp64")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    if args.workload == "mixed" and args.estimator != "trace":
        raise SystemExit("--estimator needs a single-impurity --workload (t2g, d5, f7, hubbard2)")
    if args.workload == "mixed":
        run_mixed(args, world, rank, local)
        return
    if args.estimator == "rho":
        run_density(args, world, rank, local)
        return
    if args.estimator in ("hst", "hst-seq"):
        run_improved(args, world, rank, local)
        return
    if args.estimator == "skiplist":
        run_skiplist(args, world, rank, local)
        return
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "f45":
        batch = w.batch_f45()
        imp = f45_impurity(ctq, w, local)
    else:
        mf, bf = w.WORKLOADS[args.workload]
        batch = bf(rank=rank)  # each rank evaluates its own independent batch (weak scaling)
        imp = ctq.build_impurity(mf(), device=local)
    if args.chains:
        batch = batch.subset(range(min(args.chains, batch.n_chains)))
    db = ctq.DeviceBatch(batch, device=dev)
    prec = PRECISIONS[args.precision]
    tuning = {}
    if not args.no_autotune:  # launch configuration picked by the package's autotuner, before any timing
        from paper_2010_08482_gb300 import autotune
        eng = autotune.engine(imp, prec)
        if eng != "fp64big":  # the float64 large-block kernel is FP64-pipe bound: nothing worth seconds of tuning
            big = eng == "big"
            tdb = ctq.DeviceBatch(batch.subset(range(min(batch.n_chains, 4))), device=dev) if big else db
            tuning = autotune.tune(imp, tdb, prec, cache_path=args.autotune_cache, reps=1 if big else 3)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, db.max_ops, precision=prec, device=dev, tune=tuning)
    flops, n_items = algorithmic_flops(imp, batch)
    launches = ctq.launches_per_eval(imp)
    stream = torch.cuda.current_stream()
    events = [torch.cuda.Event(enable_timing=True) for _ in range(launches + 1)]
    for e in events:
        e.record(stream)  # materialise the cudaEvent_t handles
    ev_handles = (ctypes_void_array(len(events)))(*[e.cuda_event for e in events])
    import ctypes
    ev_ptr = ctypes.cast(ev_handles, ctypes.c_void_p).value
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        ev(db, events=ev_ptr)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms, kern_ms = [], [[] for _ in range(launches)]
    for _ in range(args.steps):
        flush.zero_()
        ev(db, events=ev_ptr)
        events[-1].synchronize()
        step_ms.append(events[0].elapsed_time(events[-1]))
        for k in range(launches):
            kern_ms[k].append(events[k].elapsed_time(events[k + 1]))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0

    # end to end: pinned host batch in, results out, inside the timed region
    h_off = torch.as_tensor(np.asarray(batch.offsets, np.int32)).pin_memory()
    h_tau = torch.as_tensor(np.asarray(batch.tau, np.float64)).pin_memory()
    h_op = torch.as_tensor(np.asarray(batch.op, np.int32)).pin_memory()
    h_la = torch.empty(batch.n_chains, dtype=torch.float64).pin_memory()
    h_ph = torch.empty(2 * batch.n_chains, dtype=torch.float64).pin_memory()
    h_st = torch.empty(batch.n_chains, dtype=torch.int32).pin_memory()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    n_ops = len(batch.tau)
    e2e_warm = min(args.warmup, 2)
    for i in range(e2e_warm + args.steps):
        flush.zero_()
        e_start.record(stream)
        db.offsets.copy_(h_off, non_blocking=True)
        db.tau[:n_ops].copy_(h_tau, non_blocking=True)
        db.op[:n_ops].copy_(h_op, non_blocking=True)
        ev(db)
        h_la.copy_(ev.log_abs, non_blocking=True)
        h_ph.copy_(ev.phase, non_blocking=True)
        h_st.copy_(ev.status, non_blocking=True)
        e_end.record(stream)
        e_end.synchronize()
        if i >= e2e_warm:
            e2e_ms.append(e_start.elapsed_time(e_end))
    clocks.stop()
    h2d = h_off.numel() * 4 + h_tau.numel() * 8 + h_op.numel() * 4
    d2h = h_la.numel() * 8 + h_ph.numel() * 8 + h_st.numel() * 4

    ms = statistics.mean(step_ms)
    ms = max_over_ranks(world, ms, dev)
    e2e = max_over_ranks(world, statistics.mean(e2e_ms), dev)
    trace_ms = statistics.mean(kern_ms[1])
    value = world * batch.n_chains / (ms * 1e-3)
    fp64_peak = ctq.probe_fma_rate(local, 0)
    fp32_rate = ctq.probe_fma_rate(local, 1) if args.precision == "f32x2" else None
    achieved_tf = flops / (trace_ms * 1e-3) / 1e12
    big = imp.is_complex or imp.max_dim > 112
    # ncu DRAM counters are committed for the shared-memory FP64 kernel only
    traffic = profile_traffic("k_trace", args.workload) if (args.precision == "fp64" and not big) else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE_TEXT[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload] + (f" (first {batch.n_chains} chains)" if args.chains else ""),
                   "n_chains": batch.n_chains,
                   "surviving_strings": n_items, "precision": args.precision,
                   "l2": "flushed (256 MiB write) between steps",
                   "launch_tuning": tuning or "library default",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "tflops": flops / (ms * 1e-3) / 1e12,
        "algorithmic_flops_per_step": flops,
        "kernel_ms": {"plan": statistics.mean(kern_ms[0]), "trace": trace_ms, "combine": statistics.mean(kern_ms[2])},
        "roofline": roofline(args.precision, achieved_tf, fp64_peak, traffic, big=big, fp32_rate=fp32_rate),
        "e2e": {"value": world * batch.n_chains / (e2e * 1e-3), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * launches,
        "clocks": clocks.summary(),
        "wall_s_timed_region": wall,
    }
    if args.precision == "fp64":
        # the float64 pipe two ways: DFMA (the roofline's peak) and the warp-level MMA
        line["fp64_rates_tflops"] = {"dfma": fp64_peak / 1e12,
                                     "mma_sync_m8n8k4": ctq.probe_fma_rate(local, 2, 4000) / 1e12}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in w.WORKLOADS:
        n_first = min(CPU_SAMPLE.get(args.workload, 64), batch.n_chains)
        line["cpu_baseline"], _ = cpu_baseline_leg(args.workload, n_first, min_s=10.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# FP32 instructions per two-float multiply-add of the product loop
# (trace_fp64.cu): df_fma is one FMUL, three FFMA and eight FADD / FSUB, and
# the accumulator is renormalised (three FADD / FSUB) every four terms.
F32X2_INSTR_PER_FMA = 12.75

DTYPE_TEXT = {"fp64": "f64", "tf32": "tf32 (fp32 accumulate, f64 log scale)",
              "tf32x3": "3xtf32 (fp32 accumulate, f64 log scale)",
              "bf16x3": "3xbf16 (fp32 accumulate, f64 log scale)",
              "f32x2": "two-float f32 pairs (~48-bit products, f64 propagators and log scale)"}


def kernel_name(precision: str, big: bool) -> str:
    if precision == "f32x2":
        return "k_trace_big64<f32x2>" if big else "k_trace<f32x2>"
    if precision == "fp64":
        return "k_trace_big64<fp64>" if big else "k_trace<fp64>"
    return f"k_trace_big<{precision}>" if big else f"k_trace_tc<{precision}>"


def roofline(precision, achieved_tf, fp64_peak, traffic, big=False, fp32_rate=None, sustained=False):
    """Roofline of the dominant kernel: the FP64 pipe for the FP64 path
    (measured FMA rate), the FP32 pipe for the two-float path (measured FP32
    FMA rate / 12.75 instructions per two-float multiply-add, in
    FP64-equivalent flops), the tensor pipe of the operand type for the mixed
    paths: measured bf16 dense peak for bf16 operands, x 1/2 (the nominal
    TF32:BF16 ratio) for tf32 operands; the sustained bf16 figure when the
    kernel runs for seconds inside a long step, else the burst figure."""
    kernel = kernel_name(precision, big)
    if precision == "f32x2":
        peak = fp32_rate / F32X2_INSTR_PER_FMA / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": achieved_tf, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved_tf / peak,
                "peak_source": "measured FP32 FMA rate (ctq_probe_fma_rate, this run) / 12.75 FP32 "
                               "instructions per two-float multiply-add", "traffic": traffic}
    if precision == "fp64":
        return {"kernel": kernel, "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved_tf / (fp64_peak / 1e12),
                "peak_source": "measured FP64 FMA rate (ctq_probe_fma_rate, this run)", "traffic": traffic}
    peaks, src = load_peaks()
    bf16 = precision == "bf16x3"
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    peak = peaks[key] * (1.0 if bf16 else 0.5)
    passes = 1 if precision == "tf32" else 3
    which = "sustained" if sustained else "burst"
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved_tf, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved_tf / peak, "hardware_passes": passes,
            "tensor_pipe_frac_of_hardware_passes": passes * achieved_tf / peak,
            "peak_source": (f"{src} bf16 dense, {which} (MEASURED_PEAKS.json {key})" if bf16 else
                            f"{src} bf16 dense, {which}, x 0.5 (nominal TF32:BF16 ratio; MEASURED_PEAKS.json {key})"),
            "traffic": traffic}


def ctypes_void_array(n):
    import ctypes
    return ctypes.c_void_p * n


if __name__ == "__main__":
    main()

"""Benchmark of the GB300 local-trace path (one JSON line on rank 0).

One step = one ctq_eval_traces call over the whole batch: sector walk and
level-0 bounds, the chain products with fused propagators, renormalisation,
per-segment refined bounds, final traces and the per-chain combine.

Default workload: the 3-orbital t2g Kanamori impurity (U=5, J=0.7, beta=50,
16 sectors by (N_dn, N_up), blocks <= 9), 4096 seeded chains with orders
~ Poisson(40), FP64.  `value` is evaluations/s with inputs resident in HBM;
L2 is flushed (a 256 MiB write) between timed steps, outside the timed
kernels.  `e2e` repeats the measurement through the same C-ABI call with the
batch copied from pinned host memory and the results copied back inside the
timed region.  Multi-GPU (torchrun): every rank evaluates its own batch (no
collective on the data path; weak scaling); timing is max over ranks.

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
CPU_SAMPLE = {"t2g": 4096, "hubbard2": 64, "d5": 24, "f7": 1}  # cpu_baseline leg: chains cycled for >= 10 s
CPU_SAMPLE_REF = {"t2g": 64, "hubbard2": 64, "d5": 2, "f7": 1}  # per step of --impl reference
FLUSH_BYTES = 256 << 20


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


def profile_traffic(kernel: str, workload: str, src_hash: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("source_sha256", "")[:16] != src_hash[:16]:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def source_hash() -> str:
    """Hash of the dominant kernel's code (trace_fp64.cu and the headers it
    includes)."""
    h = hashlib.sha256()
    for fn in ("trace_fp64.cu", "device_common.cuh", "two_float.cuh", "ctq_internal.h"):
        with open(os.path.join(ROOT, "paper_2010_08482_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


_ORACLE_CACHE = {}


def cpu_oracle_rate(workload: str, n_chains: int, min_s: float = 0.0):
    """The FP64 oracle, as it stands, on the first n_chains of the workload,
    cycled through again until at least min_s seconds of CPU work (the
    cpu_baseline leg asks for 10-30 s).  Returns (evals/s, evaluations, s)."""
    from oracle import atom
    from oracle import trace as OT
    from paper_2010_08482_gb300 import workloads as w
    if workload not in _ORACLE_CACHE:
        mf, bf = w.WORKLOADS[workload]
        _ORACLE_CACHE[workload] = (atom.Model(mf()), bf())
    m, b = _ORACLE_CACHE[workload]
    n = min(n_chains, b.n_chains)
    t0 = time.perf_counter()
    count = 0
    while True:
        OT.trace_chain(m, *b.chain(count % n), beta=b.beta)
        count += 1
        dt = time.perf_counter() - t0
        if count >= n and dt >= min_s:
            break
    return count / dt, count, dt


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
    if rank != 0:
        return
    per_step = CPU_SAMPLE_REF.get(args.workload, 8)
    rates = []
    for i in range(args.warmup + args.steps):
        r, n, dt = cpu_oracle_rate(args.workload, per_step)
        if i >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_step / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "parallelism": "host cores, 1 process"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {per_step} chains of the workload per step, NumPy FP64, 1 thread"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_mixed(args, world, rank, local):
    """The uneven mixed batch: chains of three impurities evaluated on one
    stream (one ctq_eval_traces per impurity), lazy bounds on.  The coin of
    each chain sets its threshold to +inf (every bound falls below it: level-0
    reject) or -inf (never rejected: full trace, accepted), which reproduces
    the intended 50 % early rejects without an oracle pass."""
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    batch, coin = w.batch_mixed()
    if args.chains:
        keep = np.arange(min(args.chains, batch.n_chains))
        batch, coin = batch.subset(keep), coin[keep]
    models = [w.model_t2g(), w.model_d5(), w.model_f7()]
    prec = PRECISIONS[args.precision]
    groups, flops = [], 0.0
    for mi, p in enumerate(models):
        idx = np.nonzero(batch.model == mi)[0]
        if idx.size == 0:
            continue
        sub = batch.subset(idx)
        sub.beta = p.beta  # the mixed batch draws each chain's times in [0, beta) of its own model
        thr = np.where(coin[idx] == 1, np.inf, -np.inf)
        imp = ctq.build_impurity(p, device=local)
        db = ctq.DeviceBatch(sub, device=dev, log_threshold=thr)
        ev = ctq.TraceEvaluator(imp, sub.n_chains, db.max_ops, precision=prec, device=dev)
        f, _ = algorithmic_flops(imp, sub.subset(np.nonzero(coin[idx] == 0)[0]))
        flops += f
        groups.append((p.name, imp, db, ev, sub.n_chains))
    n_chains = sum(g[4] for g in groups)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        for _, _, db, ev, _ in groups:
            ev(db, lazy=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # The whole mixed evaluation (every impurity's plan / trace / combine
    # launches) is captured once as a CUDA graph and replayed per step.
    graph, graph_note = None, "captured"
    try:
        cap_stream = torch.cuda.Stream(device=dev)
        cap_stream.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap_stream):
            step()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        graph = g
    except Exception as exc:  # capture is refused: run the same launches eagerly
        torch.cuda.synchronize()
        graph_note = f"eager ({type(exc).__name__}: {str(exc)[:80]})"
    run = graph.replay if graph is not None else step
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks.stop()
    status = {g[0]: np.bincount(g[3].results(g[4])["status"] + 1, minlength=6)[1:].tolist() for g in groups}
    mean = statistics.mean(ms)
    line = {"metric": METRIC, "value": n_chains / (mean * 1e-3), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["mixed"], "n_chains": n_chains,
                       "groups": {g[0]: g[4] for g in groups}, "precision": args.precision,
                       "cuda_graph": graph_note},
            "tflops": flops / (mean * 1e-3) / 1e12, "algorithmic_flops_per_step": flops,
            "status_counts [ok, zero, rejected_early, accepted, rejected]": status,
            "gpu_launches": args.steps * sum(ctq.launches_per_eval(g[1]) for g in groups),
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="t2g", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "tf32", "tf32x3", "bf16x3", "f32x2"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chains", type=int, default=0, help="evaluate only the first N chains of the workload")
    ap.add_argument("--no-autotune", action="store_true", help="library-default launch configuration")
    ap.add_argument("--estimator", default="trace", choices=["trace", "rho", "hst", "hst-seq"],
                    help="trace: local traces (default); rho: traces plus the reduced-density-matrix estimator; "
                         "hst: the static improved-estimator ratio of every annihilator in one pass; "
                         "hst-seq: the same from traces of the replaced sequences")
    ap.add_argument("--autotune-cache", default=None, help="JSON cache of tuned launch configurations")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    if args.workload == "mixed":
        run_mixed(args, world, rank, local)
        return
    if args.estimator == "rho":
        run_density(args, world, rank, local)
        return
    if args.estimator in ("hst", "hst-seq"):
        run_improved(args, world, rank, local)
        return
    import torch
    from paper_2010_08482_gb300 import ctq
    from paper_2010_08482_gb300 import workloads as w

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mf, bf = w.WORKLOADS[args.workload]
    params = mf()
    batch = bf(rank=rank)  # each rank evaluates its own independent batch (weak scaling)
    if args.chains:
        batch = batch.subset(range(min(args.chains, batch.n_chains)))
    imp = ctq.build_impurity(params, device=local)
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
    traffic = profile_traffic("k_trace", args.workload, source_hash()) if (args.precision == "fp64" and not big) else None
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
        "dtype": {"fp64": "f64", "tf32": "tf32 (fp32 accumulate, f64 log scale)",
                  "tf32x3": "3xtf32 (fp32 accumulate, f64 log scale)",
                  "bf16x3": "3xbf16 (fp32 accumulate, f64 log scale)",
                  "f32x2": "two-float f32 pairs (~48-bit products, f64 propagators and log scale)"}[args.precision],
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_first = min(CPU_SAMPLE.get(args.workload, 64), batch.n_chains)
        r, n, dt = cpu_oracle_rate(args.workload, n_first, min_s=10.0)
        line["cpu_baseline"] = {"value": r, "unit": "evals/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} chain evaluations cycling over the first {n_first} chains of the "
                                          f"same workload ({dt:.1f} s), NumPy FP64, 1 thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# FP32 instructions per two-float multiply-add of the product loop
# (trace_fp64.cu): df_fma is one FMUL, three FFMA and eight FADD / FSUB, and
# the accumulator is renormalised (three FADD / FSUB) every four terms.
F32X2_INSTR_PER_FMA = 12.75


def roofline(precision, achieved_tf, fp64_peak, traffic, big=False, fp32_rate=None):
    """Roofline of the dominant kernel: the FP64 pipe for the FP64 path
    (measured FMA rate), the FP32 pipe for the two-float path (measured FP32
    FMA rate / 12.75 instructions per two-float multiply-add, in
    FP64-equivalent flops), the tensor pipe of the operand type for the mixed paths: measured
    bf16 dense peak for bf16 operands, x 1/2 (the nominal TF32:BF16 ratio)
    for tf32 operands."""
    if precision == "f32x2":
        peak = fp32_rate / F32X2_INSTR_PER_FMA / 1e12
        return {"kernel": "k_trace_big64<f32x2>" if big else "k_trace<f32x2>", "bound": "alu",
                "achieved": achieved_tf, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved_tf / peak,
                "peak_source": "measured FP32 FMA rate (ctq_probe_fma_rate, this run) / 12.75 FP32 "
                               "instructions per two-float multiply-add", "traffic": traffic}
    if precision == "fp64":
        return {"kernel": "k_trace_big64<fp64>" if big else "k_trace<fp64>", "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved_tf / (fp64_peak / 1e12),
                "peak_source": "measured FP64 FMA rate (ctq_probe_fma_rate, this run)", "traffic": traffic}
    peaks, src = load_peaks()
    bf16 = precision == "bf16x3"
    peak = peaks["bf16_tflops"] * (1.0 if bf16 else 0.5)
    passes = 1 if precision == "tf32" else 3
    kernel = f"k_trace_big<{precision}>" if big else f"k_trace_tc<{precision}>"
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved_tf, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved_tf / peak, "hardware_passes": passes,
            "peak_source": (f"{src} bf16 dense, MEASURED_PEAKS.json" if bf16 else
                            f"{src} bf16 dense x 0.5 (nominal TF32:BF16 ratio), MEASURED_PEAKS.json"),
            "traffic": traffic}


def ctypes_void_array(n):
    import ctypes
    return ctypes.c_void_p * n


if __name__ == "__main__":
    main()

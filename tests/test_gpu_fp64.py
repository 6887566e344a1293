"""GPU parity of the FP64 path against the FP64 oracle, through the C ABI.

Bar (FP64 mode): |w_gpu - w_oracle| / |w_oracle| <= 1e-12 with the sign
identical, on the oracle's own eigenbasis (ctq_load_impurity), so that only
the GPU arithmetic is compared.  Chains whose q0 terms cancel by more than
10x are measured against sum_q0 |w_q0|; chains whose trace cancels
internally are held to 8x the oracle's own rounding spread, measured per
chain by multiplying the same string in the opposite association order,
never above 1e-10, and at most 8 % of a test's chains (at least two) may be
held to such a widened bar (parity.Bars prints them).  The
impurity built by the library's own eigensolver (ctq_build_impurity) is compared at the tolerance its
eigenvalue differences allow: |d log w| <= beta * max|dE| (the trace's
sensitivity to energies) plus the 1e-12 arithmetic bar.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu


def run(imp, batch, thr=None, lazy=False, S=8, max_ops=None, n_alloc=None):
    db = ctq.DeviceBatch(batch, log_threshold=thr)
    mo = db.max_ops if max_ops is None else max_ops
    ev = ctq.TraceEvaluator(imp, max(1, n_alloc or batch.n_chains), max(mo, 1), segment=S)
    ev(db, lazy=lazy)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


_BATCHES = {}


def full_batch(name):
    if name not in _BATCHES:
        _BATCHES[name] = w.WORKLOADS[name][1]()
    return _BATCHES[name]


def assert_parity(res, ref, chains, tol=parity.FP64_REL, is_complex=False, label="fp64"):
    """Per chain: error <= max(tol, min(1e-10, 8 x the oracle's own
    association spread)); widened chains are counted (parity.Bars)."""
    worst = 0.0
    bars = parity.Bars(label)
    for i, c in enumerate(chains):
        r = ref[int(c)]
        err, kind = parity.chain_error(res["log_abs"][i], res["phase"][i], r)
        worst = max(worst, err)
        t = bars.fp64(c, r, base=tol)
        assert err <= t, (int(c), err, kind, r.get("noise"))
        if r["log_abs"] == -math.inf:
            assert res["status"][i] == ctq.CHAIN_ZERO
            continue
        assert res["status"][i] == ctq.CHAIN_OK
        if kind == "abs" and not is_complex and r.get("noise", 0.0) <= parity.FP64_REL:
            # well-conditioned chain: the sign must agree exactly
            assert res["phase"][i][0] == np.sign(np.real(r["phase"])) and res["phase"][i][1] == 0.0
    bars.check()
    print(f"{label}: worst error {worst:.3e} over {len(chains)} chains")
    return worst


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_fp64_full_batch_on_oracle_eigenbasis(name, models):
    """Every chain of the workload (64 / 4096 / 1024) in one launch, the
    benchmark shape, compared one by one with the oracle."""
    m = models(name)
    b = full_batch(name)
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, b)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    assert_parity(res, ref, range(b.n_chains), label=f"{name} fp64 full batch")
    assert np.all(np.isin(res["status"], [ctq.CHAIN_OK, ctq.CHAIN_ZERO]))


@pytest.mark.parametrize("name,n", [("hubbard2", 64), ("t2g", 256), ("d5", 24)])
def test_fp64_build_impurity_end_to_end(name, n, models):
    m = models(name)
    imp = ctq.build_impurity(w.WORKLOADS[name][0](), device=0)
    dE = max(np.abs(imp.energies(q) - m.E[q]).max() for q in range(m.n_sec))
    tol = parity.FP64_REL + 2.0 * m.beta * max(dE, 1e-16 * max(abs(e).max() for e in m.E))
    sub = full_batch(name).subset(range(n))
    res = run(imp, sub)
    ref = parity.oracle_chain_results(m, sub, range(n))
    print(f"{name}: library vs oracle eigenvalues differ by {dE:.2e}; bar {tol:.2e}")
    assert_parity(res, ref, range(n), tol=tol, label=f"{name} build_impurity")


@pytest.mark.parametrize("name,n,S", [("hubbard2", 64, 3), ("t2g", 128, 8), ("d5", 16, 16)])
def test_bounds_match_oracle(name, n, S, models):
    m = models(name)
    sub = full_batch(name).subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, sub, S=S)
    bounds = res["bounds"]
    for c in range(n):
        tau, ops = sub.chain(c)
        B, ub = OT.chain_bounds(m, tau, ops, sub.beta, S)
        got = bounds[c]
        if B == -math.inf:
            assert got[0] == -math.inf
            continue
        assert got[0] == pytest.approx(B, abs=1e-9 + 1e-12 * abs(B))
        for s in range(1, len(got)):
            exp = ub[min(s, len(ub) - 1)]
            if exp == -math.inf:
                assert got[s] == -math.inf
            else:
                assert got[s] == pytest.approx(exp, abs=1e-9 + 1e-12 * abs(exp)), (c, s)
        r = OT.trace_chain(m, tau, ops)
        assert np.all(got[np.isfinite(got)] >= r["log_abs"] - 1e-9)


@pytest.mark.parametrize("name,n", [("t2g", 240), ("d5", 36)])
def test_lazy_decisions_equal_exact_decisions(name, n, models):
    """Thresholds: T = log B + log 2 (must reject at level 0), T = log|w| - log 2
    (must accept), T = log|w| + 0.5 (must reject, early or after the full
    trace).  Early rejects never contradict the exact decision."""
    m = models(name)
    sub = full_batch(name).subset(range(n))
    ref = parity.oracle_chain_results(m, sub, range(n))
    thr = np.zeros(n)
    kind = np.arange(n) % 3
    for c in range(n):
        tau, ops = sub.chain(c)
        la = ref[c]["log_abs"]
        if kind[c] == 0:
            B, _ = OT.chain_bounds(m, tau, ops, sub.beta, 8)
            thr[c] = B + math.log(2.0) if B != -math.inf else 0.0
        elif kind[c] == 1:
            thr[c] = la - math.log(2.0) if la != -math.inf else -1e300
        else:
            thr[c] = la + 0.5 if la != -math.inf else 0.0
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, sub, thr=thr, lazy=True)
    st = res["status"]
    n_early_late = 0
    bars = parity.Bars(f"{name} lazy accepts")
    for c in range(n):
        la = ref[c]["log_abs"]
        if la == -math.inf:
            assert st[c] in (ctq.CHAIN_ZERO, ctq.CHAIN_REJECTED_EARLY)
            continue
        exact_accept = OT.decide(la, thr[c])
        if st[c] == ctq.CHAIN_REJECTED_EARLY:
            assert not exact_accept
            n_early_late += kind[c] == 2
        elif st[c] == ctq.CHAIN_ACCEPTED:
            assert exact_accept
            err, _ = parity.chain_error(res["log_abs"][c], res["phase"][c], ref[c])
            assert err <= bars.fp64(c, ref[c])
        else:
            assert st[c] == ctq.CHAIN_REJECTED and not exact_accept
        if kind[c] == 0:
            assert st[c] == ctq.CHAIN_REJECTED_EARLY
    bars.check()
    # without lazy evaluation the same thresholds give the same decisions
    res2 = run(imp, sub, thr=thr, lazy=False)
    for c in range(n):
        la = ref[c]["log_abs"]
        if la == -math.inf:
            continue
        assert (res2["status"][c] == ctq.CHAIN_ACCEPTED) == OT.decide(la, thr[c])


def test_edge_cases(models):
    m = models("t2g")
    imp = parity.load_oracle_model(ctq, m)
    rng = np.random.default_rng(5)
    # empty sequences: w = Z
    empty = w.Batch(beta=m.beta, offsets=np.zeros(4, np.int32), tau=np.zeros(0), op=np.zeros(0, np.int32))
    res = run(imp, empty, max_ops=4)
    z = OT.trace_chain(m, [], [])
    for c in range(3):
        assert abs(res["log_abs"][c] - z["log_abs"]) <= 1e-12 * abs(z["log_abs"])
        assert res["phase"][c][0] == 1.0 and res["status"][c] == ctq.CHAIN_OK
    # unstructured operator strings: most die, odd lengths never survive
    b = w.uniform_random_ops_batch(rng, m.n_flav, m.beta, 200, 0, 9)
    res = run(imp, b)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    assert_parity(res, ref, range(b.n_chains), label="unstructured strings")
    assert np.sum(res["status"] == ctq.CHAIN_ZERO) > 50
    # malformed chains
    tau = np.array([0.5, 0.2, 1.0, 2.0, 3.0, 4.0, 0.1, 50.0, -0.1, 0.3, 1.0, 2.0])
    op = np.array([1, 0, 1, 0, 1, 99, 1, 0, 1, 0, 1, 0], np.int32)
    bad = w.Batch(beta=m.beta, offsets=np.array([0, 2, 4, 6, 8, 10, 12], np.int32), tau=tau, op=op)
    res = run(imp, bad, max_ops=2)
    # chain 0 unsorted, 1 ok, 2 op out of range, 3 tau == beta, 4 tau < 0, 5 ok
    assert list(res["status"][[0, 2, 3, 4]]) == [ctq.CHAIN_ERR_ARG] * 4
    assert np.all(np.isnan(res["log_abs"][[0, 2, 3, 4]]))
    assert res["status"][1] in (ctq.CHAIN_OK, ctq.CHAIN_ZERO)
    # chains longer than the max_ops passed to the C ABI are flagged by the kernel
    sub = full_batch("t2g").subset(range(8))
    lens = np.diff(sub.offsets)
    db = ctq.DeviceBatch(sub)
    ev = ctq.TraceEvaluator(imp, sub.n_chains, int(lens.max()))
    ctq.eval_traces(imp, sub.n_chains, sub.beta, db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None,
                    ev.log_abs.data_ptr(), ev.phase.data_ptr(), ev.status.data_ptr(), None, ev.ws_ptr, ev.ws_bytes,
                    torch.cuda.current_stream().cuda_stream, max_ops=int(lens.max()) - 1)
    torch.cuda.synchronize()
    st = ev.results()["status"]
    assert np.all((st == ctq.CHAIN_ERR_ARG) == (lens > lens.max() - 1))


def test_zero_chains_and_errors(models):
    m = models("hubbard2")
    imp = parity.load_oracle_model(ctq, m)
    ev = ctq.TraceEvaluator(imp, 4, 8)
    empty = w.Batch(beta=m.beta, offsets=np.zeros(1, np.int32), tau=np.zeros(0), op=np.zeros(0, np.int32))
    ev(ctq.DeviceBatch(empty))  # n_chains = 0 is a no-op
    db = ctq.DeviceBatch(full_batch("hubbard2").subset(range(4)))
    with pytest.raises(ctq.CtqError) as e:
        ctq.eval_traces(imp, 4, m.beta, db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None,
                        ev.log_abs.data_ptr(), ev.phase.data_ptr(), ev.status.data_ptr(), None, ev.ws_ptr,
                        16, torch.cuda.current_stream().cuda_stream, max_ops=40)
    assert e.value.code == ctq.CTQ_ERR_WORKSPACE
    with pytest.raises(ctq.CtqError) as e:
        ctq.eval_traces(imp, 4, m.beta, db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None,
                        ev.log_abs.data_ptr(), ev.phase.data_ptr(), ev.status.data_ptr(), None, ev.ws_ptr,
                        ev.ws_bytes, torch.cuda.current_stream().cuda_stream, max_ops=8, lazy=True)
    assert e.value.code == ctq.CTQ_ERR_ARG  # lazy without thresholds


def test_graph_capture_and_determinism(models):
    m = models("t2g")
    imp = parity.load_oracle_model(ctq, m)
    b = full_batch("t2g").subset(range(300))
    db = ctq.DeviceBatch(b)
    ev = ctq.TraceEvaluator(imp, b.n_chains, db.max_ops)
    ev(db)
    torch.cuda.synchronize()
    eager = ev.results()
    ev(db)
    torch.cuda.synchronize()
    again = ev.results()
    for k in eager:
        assert np.array_equal(eager[k], again[k], equal_nan=True)
    ev.log_abs.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        ev(db, stream=s)  # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            ev(db, stream=s)
    ev.log_abs.zero_()
    g.replay()
    torch.cuda.synchronize()
    replay = ev.results()
    for k in eager:
        assert np.array_equal(eager[k], replay[k], equal_nan=True)

"""GPU parity of the two-float path (CTQ_F32X2) against the FP64 oracle,
through the C ABI, on the oracle's own eigenbasis.

CTQ_F32X2 runs the float64 shared-memory trace kernel with its block
products in pairs of float32 words (x = hi + lo, about 48 significant bits,
Dekker / Knuth error-free transformations on the FP32 pipe); propagators,
log scale, exponents and the final diagonal sum stay in float64.  Its unit
roundoff is 2^-48 against float64's 2^-53 (ratio 32), and a two-float
product rounds about three times where a float64 fused multiply-add rounds
once, so the stated bar is the FP64 bar times 100: relative error <= X2_REL
= 1e-10, or 32 x the FP64 allowance (8 x the spread, at most 1e-10) on the
few chains whose own float64 rounding spread exceeds half the FP64 bar; the sign must agree on well-conditioned chains, and lazy
early rejects must never contradict the exact decision.
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

ROUNDOFF_RATIO = 2.0 ** 5  # 2^-48 / 2^-53
X2_REL = 100.0 * parity.FP64_REL

_BATCHES = {}


def full_batch(name):
    if name not in _BATCHES:
        _BATCHES[name] = w.WORKLOADS[name][1]()
    return _BATCHES[name]


def run(imp, batch, thr=None, lazy=False, S=8):
    db = ctq.DeviceBatch(batch, log_threshold=thr)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(db.max_ops, 1), precision=ctq.F32X2, segment=S)
    ev(db, lazy=lazy)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


def assert_x2_parity(res, ref, chains, label="x2"):
    worst = 0.0
    bars = parity.Bars(label)
    for i, c in enumerate(chains):
        r = ref[int(c)]
        err, kind = parity.chain_error(res["log_abs"][i], res["phase"][i], r)
        worst = max(worst, err)
        tol = bars.fp64(c, r, base=X2_REL / ROUNDOFF_RATIO, scale=ROUNDOFF_RATIO)
        assert err <= tol, (int(c), err, kind, r.get("noise"))
        if r["log_abs"] == -math.inf:
            assert res["status"][i] == ctq.CHAIN_ZERO
            continue
        assert res["status"][i] == ctq.CHAIN_OK
        if kind == "abs" and r.get("noise", 0.0) <= parity.FP64_REL:
            assert res["phase"][i][0] == np.sign(np.real(r["phase"])) and res["phase"][i][1] == 0.0
    bars.check()
    return worst


@pytest.mark.parametrize("name,n", [("hubbard2", 64), ("t2g", 512), ("d5", 48)])
def test_x2_parity_on_oracle_eigenbasis(name, n, models):
    m = models(name)
    sub = full_batch(name).subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    assert ctq.trace_kernel(imp, ctq.F32X2) == ctq.KERNEL_FP64_SHARED
    res = run(imp, sub)
    ref = parity.oracle_chain_results(m, sub, range(n))
    worst = assert_x2_parity(res, ref, range(n))
    # the float64 kernel on the same chains, for the record
    db = ctq.DeviceBatch(sub)
    ev = ctq.TraceEvaluator(imp, sub.n_chains, max(db.max_ops, 1))
    ev(db)
    torch.cuda.synchronize()
    r64 = ev.results(sub.n_chains)
    w64 = max(parity.chain_error(r64["log_abs"][c], r64["phase"][c], ref[c])[0] for c in range(n))
    print(f"\n{name}: F32X2 max relative error {worst:.3e} over {n} chains (bar {X2_REL:.1e}); "
          f"FP64 kernel {w64:.3e}")


@pytest.mark.parametrize("name,n_sample", [("t2g", 96), ("d5", 12)])
def test_x2_full_size_batch_sampled(name, n_sample, models):
    """The whole batch in one launch (the benchmark shape); sampled chains
    compared one by one with the oracle."""
    m = models(name)
    b = full_batch(name)
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, b)
    rng = np.random.default_rng(23)
    sample = np.sort(rng.choice(b.n_chains, size=n_sample, replace=False))
    ref = parity.oracle_chain_results(m, b, sample)
    sub = {k: v[sample] for k, v in res.items() if k != "bounds"}
    assert_x2_parity(sub, ref, sample)
    assert np.all(np.isin(res["status"], [ctq.CHAIN_OK, ctq.CHAIN_ZERO]))


def test_x2_agrees_with_fp64_path(models):
    """The same batch through the float64 and two-float kernels: every
    chain's value within the two-float bar of the float64 one."""
    m = models("t2g")
    sub = full_batch("t2g").subset(range(256))
    imp = parity.load_oracle_model(ctq, m)
    r2 = run(imp, sub)
    db = ctq.DeviceBatch(sub)
    ev = ctq.TraceEvaluator(imp, sub.n_chains, db.max_ops)
    ev(db)
    torch.cuda.synchronize()
    r1 = ev.results(sub.n_chains)
    ref = parity.oracle_chain_results(m, sub, range(sub.n_chains))
    for c in range(sub.n_chains):
        if r1["log_abs"][c] == -math.inf:
            assert r2["log_abs"][c] == -math.inf
            continue
        a = complex(*r1["phase"][c])
        b = complex(*r2["phase"][c]) * math.exp(r2["log_abs"][c] - r1["log_abs"][c])
        assert abs(a - b) <= max(X2_REL, ROUNDOFF_RATIO * parity.fp64_tolerance(ref[c])) + parity.fp64_tolerance(ref[c]), c


@pytest.mark.parametrize("name,n", [("t2g", 240), ("d5", 36)])
def test_x2_lazy_decisions_equal_exact_decisions(name, n, models):
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
    for c in range(n):
        la = ref[c]["log_abs"]
        if la == -math.inf:
            assert st[c] in (ctq.CHAIN_ZERO, ctq.CHAIN_REJECTED_EARLY)
            continue
        exact_accept = OT.decide(la, thr[c])
        if st[c] == ctq.CHAIN_REJECTED_EARLY:
            assert not exact_accept
        elif st[c] == ctq.CHAIN_ACCEPTED:
            assert exact_accept
        else:
            assert st[c] == ctq.CHAIN_REJECTED and not exact_accept
        if kind[c] == 0:
            assert st[c] == ctq.CHAIN_REJECTED_EARLY

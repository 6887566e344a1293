"""Float64 large-block engine (k_trace_big64: persistent cooperative kernel,
SIMT float64 tiles, complex blocks in the real embedding): parity with the
FP64 oracle at the FP64 bar on models whose blocks are too large for the
shared-memory FP64 kernel (a complex d shell with SOC and complex crystal
field, N in [1, 3], blocks up to 120; a real d shell with sectors by N, N in
[4, 6], blocks up to 252), bounds that bracket |w|, and the f shell against
the stored oracle values (tests/golden/f7_oracle.json)."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402
from test_gpu_big import complex_d_model, real_d_window_model  # noqa: E402

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run(imp, batch, S=8, thr=None, lazy=False):
    db = ctq.DeviceBatch(batch, log_threshold=thr)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(1, db.max_ops), precision=ctq.FP64, segment=S)
    ev(db, lazy=lazy)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.fixture(scope="module")
def small_models():
    return {"dc": atom.Model(complex_d_model()), "dn": atom.Model(real_d_window_model())}


@pytest.mark.parametrize("name", ["dc", "dn"])
def test_big64_parity_at_fp64_bar(name, small_models):
    m = small_models[name]
    assert max(m.dims) > 112  # the shared-memory FP64 kernel cannot hold these blocks
    rng = np.random.default_rng(51)
    b = w.random_batch(rng, m.n_flav, m.beta, 12, 1, 14, gen="g2")
    imp = parity.load_oracle_model(ctq, m)
    assert ctq.trace_kernel(imp, ctq.FP64) == ctq.KERNEL_FP64_LARGE
    assert ctq.trace_kernel(imp, ctq.BF16X3) == ctq.KERNEL_TC_LARGE
    res = run(imp, b)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    worst, n_ok = 0.0, 0
    bars = parity.Bars(f"{name} FP64 large-block")
    for c in range(b.n_chains):
        r = ref[c]
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        assert err <= bars.fp64(c, r), (c, err, kind, r.get("noise"))
        worst = max(worst, err)
        if r["log_abs"] == -math.inf:
            assert res["status"][c] == ctq.CHAIN_ZERO
        else:
            assert res["status"][c] == ctq.CHAIN_OK
            n_ok += 1
    assert n_ok >= 6
    bars.check()
    print(f"{name} FP64 large-block: worst rel err {worst:.3e} over {n_ok} chains")


def test_big64_bounds_and_lazy_decisions(small_models):
    m = small_models["dn"]
    rng = np.random.default_rng(53)
    b = w.random_batch(rng, m.n_flav, m.beta, 8, 6, 12, gen="g2")
    imp = parity.load_oracle_model(ctq, m)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains), noise=False)
    res = run(imp, b, S=4)
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        B, ub = OT.chain_bounds(m, tau, ops, b.beta, 4)
        got = res["bounds"][c]
        if B == -math.inf:
            continue
        assert got[0] == pytest.approx(B, abs=1e-9 + 1e-12 * abs(B))
        fin = got[np.isfinite(got)]
        if ref[c]["log_abs"] != -math.inf:
            assert np.all(fin >= ref[c]["log_abs"] - 1e-9)
    # thresholds that force a level-0 reject or an accept
    thr = np.array([(ref[c]["log_abs"] - math.log(2.0)) if (c % 2 == 0 and ref[c]["log_abs"] != -math.inf)
                    else 1e300 for c in range(b.n_chains)])
    res = run(imp, b, thr=thr, lazy=True)
    for c in range(b.n_chains):
        if thr[c] == 1e300:
            assert res["status"][c] in (ctq.CHAIN_REJECTED_EARLY, ctq.CHAIN_ZERO)
        else:
            assert res["status"][c] == ctq.CHAIN_ACCEPTED


def f7_bar(imp, g, beta):
    """(max|dE|, 2 beta max|dE|): the part of the bar for the library-built f
    shell that comes from the trace's sensitivity to the energies, with dE
    MEASURED between the library's device eigensolver and the oracle's stored
    sector energies (the arithmetic part is added by the caller)."""
    dE = max(float(np.abs(imp.energies(q) - np.asarray(g["E"][q])).max()) for q in range(len(g["dims"])))
    return dE, 2.0 * beta * dE


def test_f7_fp64_against_stored_oracle():
    """Library-built f shell (device eigensolver) in float64 on the GPU against
    the oracle's stored values, at the FP64 bar plus 2 beta max|dE| for the
    measured difference dE of the two independent eigensolvers' energies."""
    path = os.path.join(HERE, "golden", "f7_oracle.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/f7_oracle.json not generated")
    with open(path) as f:
        g = json.load(f)
    imp = ctq.build_impurity(w.model_f7(), device=0)
    n = 2
    b = w.batch_f7().subset(range(n))
    res = run(imp, b)
    dE, e_bar = f7_bar(imp, g, b.beta)
    bars = parity.Bars("f7 FP64 stored oracle")
    for c in range(n):
        ref = g["chains"][c]
        err = abs(complex(*res["phase"][c]) * math.exp(res["log_abs"][c] - ref["log_abs"]) - complex(*ref["phase"]))
        tol = bars.fp64(c, ref) + e_bar
        print(f"f7 FP64 chain {c}: rel err {err:.3e}, bar {tol:.3e} (max|dE| {dE:.2e})")
        assert err <= tol, (c, err)
        assert res["status"][c] == ctq.CHAIN_OK
    bars.check()


def run_x2(imp, batch, S=8):
    db = ctq.DeviceBatch(batch)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(1, db.max_ops), precision=ctq.F32X2, segment=S)
    ev(db)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.mark.parametrize("name", ["dc", "dn"])
def test_big64_two_float_parity(name, small_models):
    """CTQ_F32X2 on the large-block kernel (two-float tiles on the FP32 pipe):
    the two-float bar of tests/test_gpu_x2.py (1e-10 relative, or 32 x the
    FP64 allowance of a chain that cancels internally)."""
    m = small_models[name]
    rng = np.random.default_rng(51)
    b = w.random_batch(rng, m.n_flav, m.beta, 12, 1, 14, gen="g2")
    imp = parity.load_oracle_model(ctq, m)
    assert ctq.trace_kernel(imp, ctq.F32X2) == ctq.KERNEL_FP64_LARGE
    res = run_x2(imp, b)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    worst = 0.0
    bars = parity.Bars(f"{name} two-float large-block")
    for c in range(b.n_chains):
        r = ref[c]
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        assert err <= bars.fp64(c, r, base=1e-10 / 32.0, scale=32.0), (c, err, kind, r.get("noise"))
        worst = max(worst, err)
        if r["log_abs"] == -math.inf:
            assert res["status"][c] == ctq.CHAIN_ZERO
        else:
            assert res["status"][c] == ctq.CHAIN_OK
    bars.check()
    print(f"{name} two-float large-block: worst rel err {worst:.3e}")


def test_f7_two_float_against_stored_oracle():
    """The library-built f shell in two-float arithmetic against the stored
    oracle values: the measured-eigensolver bar of the FP64 test plus the
    two-float bar."""
    path = os.path.join(HERE, "golden", "f7_oracle.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/f7_oracle.json not generated")
    with open(path) as f:
        g = json.load(f)
    imp = ctq.build_impurity(w.model_f7(), device=0)
    assert ctq.trace_kernel(imp, ctq.F32X2) == ctq.KERNEL_FP64_LARGE
    n = 2
    b = w.batch_f7().subset(range(n))
    res = run_x2(imp, b)
    dE, e_bar = f7_bar(imp, g, b.beta)
    bars = parity.Bars("f7 two-float stored oracle")
    for c in range(n):
        ref = g["chains"][c]
        err = abs(complex(*res["phase"][c]) * math.exp(res["log_abs"][c] - ref["log_abs"]) - complex(*ref["phase"]))
        tol = bars.fp64(c, ref, base=1e-10 / 32.0, scale=32.0) + e_bar
        print(f"f7 two-float chain {c}: rel err {err:.3e}, bar {tol:.3e} (max|dE| {dE:.2e})")
        assert err <= tol, (c, err)
        assert res["status"][c] == ctq.CHAIN_OK
    bars.check()

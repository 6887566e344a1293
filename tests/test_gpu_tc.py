"""Tensor-core (tcgen05) path: operand conventions and parity of the TF32,
three-term split TF32 and three-term split bf16 chain products against the
FP64 oracle.

Mixed-precision bar: the paper gives no number, so the error against the
FP64 oracle is stated per configuration (STATED below, relative error of w
per chain; the measured distributions are printed and recorded in the design
notes).  A chain's error grows with its measured condition number kappa
(its float64 perturbation spread over 2^-53): about unit x kappa, with unit
the precision's effective unit roundoff (parity.UNIT).  So a chain is held to
its stated bar, or to unit x kappa where that is larger (only a counted
few chains may need it; a chain with unit x kappa >= 1 is listed as
unresolved, at most 1 % of a test's chains or 3); the d shell
(n ~ 120, d up to 100) is the worst conditioned.  Signs must agree on
well-conditioned chains."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu

# Stated bars: about 3x the largest error measured on the well-conditioned
# chains; a chain whose unit x kappa exceeds its bar is held to that, and one
# whose unit x kappa reaches 1 is listed as unresolved (parity.Bars).  TF32
# in one pass does not resolve the d shell: its errors there are O(1).
STATED = {
    (ctq.TF32X3, "hubbard2"): 1e-5, (ctq.TF32X3, "t2g"): 2e-5, (ctq.TF32X3, "d5"): 1.5e-3,
    (ctq.TF32, "hubbard2"): 1.5e-2, (ctq.TF32, "t2g"): 2.5e-2, (ctq.TF32, "d5"): 2.0,
    (ctq.BF16X3, "hubbard2"): 7e-5, (ctq.BF16X3, "t2g"): 2e-4, (ctq.BF16X3, "d5"): 1.2e-2,
}


# Operand rounding bound of one product relative to max |A B^T| (TF32: 2^-11
# per operand; 3xTF32: ~2^-21; bf16 hi / lo: ~2^-16), FP32 accumulation.
SINGLE_TOL = {ctq.TF32: 2e-3, ctq.TF32X3: 2e-6, ctq.BF16X3: 5e-5}


@pytest.mark.parametrize("split", [ctq.TF32, ctq.TF32X3, ctq.BF16X3])
@pytest.mark.parametrize("N,K", [(16, 16), (48, 32), (112, 112), (64, 112)])
def test_single_mma_conventions(split, N, K):
    """D = A B^T with A in TMEM (one tf32 or two packed bf16 K elements per
    column) and B as K-major core matrices in shared memory."""
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.normal(size=(128, K)).astype(np.float32)
    Bm = rng.normal(size=(N, K)).astype(np.float32)
    D = ctq.tc_gemm_check(A, Bm, split=split)
    ref = A.astype(np.float64) @ Bm.astype(np.float64).T
    err = np.abs(D - ref).max() / np.abs(ref).max()
    print(f"split={split} N={N} K={K}: {err:.3e}")
    assert err < SINGLE_TOL[split], err


def run(imp, batch, precision, thr=None, lazy=False, S=8):
    db = ctq.DeviceBatch(batch, log_threshold=thr)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(1, db.max_ops), precision=precision, segment=S)
    ev(db, lazy=lazy)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.mark.parametrize("precision", [ctq.TF32X3, ctq.TF32, ctq.BF16X3])
@pytest.mark.parametrize("name,n", [("hubbard2", 64), ("t2g", 128), ("d5", 32)])
def test_mixed_precision_parity(precision, name, n, models):
    m = models(name)
    sub = w.WORKLOADS[name][1]().subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, sub, precision)
    ref = parity.oracle_chain_results(m, sub, range(n))
    errs, well = [], []
    bars = parity.Bars(f"{name} precision={precision}")
    for c in range(n):
        r = ref[c]
        if r["log_abs"] == -math.inf:
            continue
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        n_ops = int(sub.offsets[c + 1] - sub.offsets[c])
        bar = bars.mixed(c, r, STATED[(precision, name)], parity.UNIT[precision], err)
        print(f"  chain {c}: n_ops {n_ops} err {err:.3e} float64 spread {r.get('noise', 0.0):.1e} bar {bar:.1e}")
        assert err <= bar, (c, err, kind, n_ops)
        errs.append(err)
        if r.get("noise", 0.0) <= parity.WIDEN_AT:
            well.append(err)
        if r.get("noise", 0.0) <= parity.WIDEN_AT and kind == "abs":
            assert res["phase"][c][0] == np.sign(np.real(r["phase"]))
    bars.check()
    print(f"{name} precision={precision}: n={len(errs)} max rel err {max(errs):.3e}, "
          f"p90 {np.quantile(errs, 0.9):.3e}, median {np.median(errs):.3e}; well-conditioned chains: "
          f"max {max(well):.3e}, median {np.median(well):.3e}")


@pytest.mark.parametrize("precision", [ctq.BF16X3, ctq.TF32X3])
def test_d5_stated_error_across_the_sample(precision, models):
    """The d shell's stated error on all 1024 chains of its batch (stored
    oracle values): every chain within its stated bar, or within
    unit x kappa (at most 10 x) for the counted few whose measured condition
    number needs it; the distribution is printed by kappa.  A chain with
    unit x kappa >= 1 has no significant digit left in the precision (its
    float64 spread says the product cancels internally by more than the
    precision resolves): such chains are listed and may be at most 1 % of
    the batch (at least 3), with no bar (parity.Bars)."""
    n, ref = parity.gold_d5()
    sub = w.batch_d5().subset(range(n))
    assert all(ref[c]["n_ops"] == int(sub.offsets[c + 1] - sub.offsets[c]) for c in range(n))
    imp = parity.load_oracle_model(ctq, models("d5"))
    res = run(imp, sub, precision)
    stated = STATED[(precision, "d5")]
    bars = parity.Bars(f"d5 sample precision={precision}")
    rows = []
    for c in range(n):
        r = ref[c]
        if r["log_abs"] == -math.inf:
            assert res["log_abs"][c] == -math.inf, c
            continue
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        bar = bars.mixed(c, r, stated, parity.UNIT[precision], err)
        assert err <= bar, (c, err, bar, r["noise"])
        if math.isfinite(bar):
            rows.append((err, r["noise"] / parity.U64))
    bars.check()
    e, kap = np.array(rows).T
    print(f"\nd5 precision={precision}: n={len(e)} median {np.median(e):.2e} p99 {np.quantile(e, 0.99):.2e} "
          f"max {e.max():.2e}")
    for lo, hi in [(0, 1e2), (1e2, 1e3), (1e3, 1e4), (1e4, 1e12)]:
        k = (kap >= lo) & (kap < hi)
        if k.any():
            print(f"  kappa in [{lo:.0e}, {hi:.0e}): {k.sum()} chains, median {np.median(e[k]):.2e}, max {e[k].max():.2e}")


def test_mixed_lazy_decisions_never_contradict_exact(models):
    m = models("d5")
    sub = w.batch_d5().subset(range(30))
    ref = parity.oracle_chain_results(m, sub, range(30), noise=False)
    thr = np.array([ref[c]["log_abs"] + (0.5 if c % 2 else -0.7) if ref[c]["log_abs"] != -math.inf else 0.0
                    for c in range(30)])
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, sub, ctq.TF32X3, thr=thr, lazy=True)
    for c in range(30):
        la = ref[c]["log_abs"]
        if la == -math.inf:
            continue
        if res["status"][c] == ctq.CHAIN_REJECTED_EARLY:
            assert la < thr[c]
        elif res["status"][c] == ctq.CHAIN_ACCEPTED:
            assert la >= thr[c]


@pytest.mark.parametrize("precision", [ctq.TF32X3, ctq.BF16X3])
def test_small_block_bounds_match_oracle(precision, models):
    """Segment bounds of the small-block tensor kernel (taken after the
    string, lanes over segments) against the oracle's refined bounds: equal
    up to the products' rounding (the Frobenius norms come from FP32 sums),
    and never below log|w| by more than the early-reject margin."""
    m = models("d5")
    sub = w.batch_d5().subset(range(24))
    imp = parity.load_oracle_model(ctq, m)
    S = 8
    res = run(imp, sub, precision, S=S)
    margin = 5e-2 if precision == ctq.BF16X3 else 1e-2
    n_cmp = 0
    for c in range(sub.n_chains):
        tau, ops = sub.chain(c)
        B, ub = OT.chain_bounds(m, tau, ops, sub.beta, S)
        got = res["bounds"][c]
        if B == -math.inf:
            continue
        r = OT.trace_chain(m, tau, ops, beta=sub.beta)
        for s in range(1, len(got)):
            exp = ub[min(s, len(ub) - 1)]
            if exp == -math.inf or not np.isfinite(got[s]):
                continue
            assert abs(got[s] - exp) <= margin, (c, s, got[s], exp)
            n_cmp += 1
        fin = got[np.isfinite(got)]
        if r["log_abs"] != -math.inf:
            assert np.all(fin >= r["log_abs"] - margin)
    assert n_cmp > 20

"""The uneven mixed batch (chains of the t2g, d5 and f7 models, orders
10-200, lazy bounds on).  Thresholds as in the workload definition: a fair
coin puts a chain at T = log B + log 2 (B the level-0 bound: it must be
rejected before any product) or at T = log|w| - log 2 (it must be accepted,
and its trace must match the oracle).  f-shell chains, too slow for the
oracle here, get T = +inf / -inf and are checked for their decisions."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu

MODELS = [w.model_t2g, w.model_d5, w.model_f7]
# stated 3xTF32 bars of the mixed batch's chains (orders up to 200, longer
# than the t2g and d5 workloads' own chains); FP64 chains take the FP64 bar
STATED_TF32X3 = {0: 2e-4, 1: 4e-3}


def run_lazy(imp, batch, thr, precision):
    db = ctq.DeviceBatch(batch, log_threshold=thr)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(1, db.max_ops), precision=precision)
    ev(db, lazy=True)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.mark.parametrize("precision", [ctq.FP64, ctq.TF32X3])
@pytest.mark.parametrize("mi,n", [(0, 24), (1, 10)])
def test_mixed_batch_decisions(mi, n, precision, models):
    batch, coin = w.batch_mixed()
    p = MODELS[mi]()
    idx = np.nonzero(batch.model == mi)[0][:n]
    sub = batch.subset(idx)
    sub.beta = p.beta
    m = models(p.name)
    thr = np.zeros(n)
    ref = parity.oracle_chain_results(m, sub, range(n))
    for c in range(n):
        tau, ops = sub.chain(c)
        if coin[idx[c]] == 1:
            B = OT.chain_bounds(m, tau, ops, sub.beta, 8)[0]
            thr[c] = B + math.log(2.0) if B != -math.inf else 0.0
        else:
            thr[c] = ref[c]["log_abs"] - math.log(2.0) if ref[c]["log_abs"] != -math.inf else -1e300
    imp = parity.load_oracle_model(ctq, m)
    res = run_lazy(imp, sub, thr, precision)
    bars = parity.Bars(f"mixed {p.name} precision={precision}")
    for c in range(n):
        if ref[c]["log_abs"] == -math.inf:
            continue
        if coin[idx[c]] == 1:
            assert res["status"][c] == ctq.CHAIN_REJECTED_EARLY, c
        else:
            assert res["status"][c] == ctq.CHAIN_ACCEPTED, c
            err, _ = parity.chain_error(res["log_abs"][c], res["phase"][c], ref[c])
            bar = (bars.fp64(c, ref[c]) if precision == ctq.FP64
                   else bars.mixed(c, ref[c], STATED_TF32X3[mi], parity.UNIT[precision], err))
            print(f"  chain {int(idx[c])}: n_ops {len(sub.chain(c)[1])} err {err:.3e} bar {bar:.1e}")
            assert err <= bar, (c, err)
    bars.check()


def test_mixed_batch_f_shell_decisions():
    batch, coin = w.batch_mixed()
    idx = np.nonzero(batch.model == 2)[0][:6]
    sub = batch.subset(idx)
    sub.beta = w.model_f7().beta
    thr = np.where(coin[idx] == 1, np.inf, -np.inf)
    imp = ctq.build_impurity(w.model_f7(), device=0)
    res = run_lazy(imp, sub, thr, ctq.TF32X3)
    for c in range(len(idx)):
        if coin[idx[c]] == 1:
            assert res["status"][c] == ctq.CHAIN_REJECTED_EARLY
        else:
            assert res["status"][c] in (ctq.CHAIN_ACCEPTED, ctq.CHAIN_ZERO)
            if res["status"][c] == ctq.CHAIN_ACCEPTED:
                assert np.isfinite(res["log_abs"][c]) and abs(np.hypot(*res["phase"][c]) - 1.0) < 1e-12

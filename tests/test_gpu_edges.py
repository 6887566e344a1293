"""Edge cases on every trace kernel (the shared-memory FP64 kernel has its
own in test_gpu_fp64.py): empty sequences (w = Z), one-operator strings,
unstructured operator strings of length 0-9 (most sector strings die, odd
lengths never survive), malformed chains (unsorted times, operator code out
of range, tau outside [0, beta)), all against the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402
from test_gpu_big import complex_d_model  # noqa: E402

pytestmark = pytest.mark.gpu

# relative error bars for strings of at most 9 operators
TOL = {ctq.FP64: None, ctq.TF32X3: 1e-4, ctq.BF16X3: 2e-3, ctq.TF32: 2e-2}

CASES = [("t2g", ctq.TF32X3, ctq.KERNEL_TC_SMALL), ("t2g", ctq.BF16X3, ctq.KERNEL_TC_SMALL),
         ("t2g", ctq.TF32, ctq.KERNEL_TC_SMALL), ("dc", ctq.TF32X3, ctq.KERNEL_TC_LARGE),
         ("dc", ctq.BF16X3, ctq.KERNEL_TC_LARGE), ("dc", ctq.FP64, ctq.KERNEL_FP64_LARGE)]


@pytest.fixture(scope="module")
def oracle_models():
    return {"t2g": atom.Model(w.model_t2g()), "dc": atom.Model(complex_d_model())}


def run(imp, batch, precision, max_ops=None):
    db = ctq.DeviceBatch(batch)
    mo = max(1, db.max_ops) if max_ops is None else max_ops
    ev = ctq.TraceEvaluator(imp, batch.n_chains, mo, precision=precision)
    ev(db)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.mark.parametrize("name,precision,kernel", CASES)
def test_edges(name, precision, kernel, oracle_models):
    m = oracle_models[name]
    imp = parity.load_oracle_model(ctq, m)
    assert ctq.trace_kernel(imp, precision) == kernel
    # empty sequences: w = Z, computed in float64 by every kernel
    empty = w.Batch(beta=m.beta, offsets=np.zeros(4, np.int32), tau=np.zeros(0), op=np.zeros(0, np.int32))
    res = run(imp, empty, precision, max_ops=4)
    z = OT.trace_chain(m, [], [])
    for c in range(3):
        assert abs(res["log_abs"][c] - z["log_abs"]) <= 1e-12 * abs(z["log_abs"])
        assert res["phase"][c][0] == 1.0 and res["status"][c] == ctq.CHAIN_OK
    # unstructured strings of 0-9 operators
    rng = np.random.default_rng(17)
    b = w.uniform_random_ops_batch(rng, m.n_flav, m.beta, 160, 0, 9)
    res = run(imp, b, precision)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    n_live = 0
    bars = parity.Bars(f"{name} precision={precision} unstructured strings")
    for c in range(b.n_chains):
        r = ref[c]
        if r["log_abs"] == -math.inf:
            assert res["status"][c] == ctq.CHAIN_ZERO, c
            continue
        n_live += 1
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        tol = (bars.fp64(c, r) if TOL[precision] is None
               else bars.mixed(c, r, TOL[precision], parity.UNIT[precision], err))
        assert err <= tol, (c, err, kind)
        assert res["status"][c] == ctq.CHAIN_OK
    bars.check()
    assert n_live >= 5 and np.sum(res["status"] == ctq.CHAIN_ZERO) > 40
    # malformed chains: unsorted, operator out of range, tau == beta, tau < 0
    tau = np.array([0.5, 0.2, 1.0, 2.0, 3.0, 4.0, 0.1, m.beta, -0.1, 0.3, 1.0, 2.0])
    op = np.array([1, 0, 1, 0, 1, 999, 1, 0, 1, 0, 1, 0], np.int32)
    bad = w.Batch(beta=m.beta, offsets=np.array([0, 2, 4, 6, 8, 10, 12], np.int32), tau=tau, op=op)
    res = run(imp, bad, precision, max_ops=2)
    assert list(res["status"][[0, 2, 3, 4]]) == [ctq.CHAIN_ERR_ARG] * 4
    assert np.all(np.isnan(res["log_abs"][[0, 2, 3, 4]]))
    assert res["status"][1] in (ctq.CHAIN_OK, ctq.CHAIN_ZERO) and res["status"][5] in (ctq.CHAIN_OK, ctq.CHAIN_ZERO)

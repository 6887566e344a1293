"""Failure detection without a GPU fault: the tensor-core kernels and the
float64 / two-float large-block kernel bound every wait by the caller's
timeout.  With CTQ_DEBUG_STALL_WAIT a kernel first waits
on an event that nothing triggers; the wait expires after timeout_ns, the
kernel records the error, frees its tensor memory and returns, every chain
reports CTQ_CHAIN_ERR_TIMEOUT, and the next evaluation on the same context
is correct."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu


def _eval(imp, batch, precision, **kw):
    db = ctq.DeviceBatch(batch)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, db.max_ops, precision=precision)
    ev(db, **kw)
    torch.cuda.synchronize()
    return ev.results()


@pytest.mark.parametrize("which,precision", [("small", ctq.TF32X3), ("large", ctq.TF32X3), ("large", ctq.FP64),
                                             ("large", ctq.F32X2)])
def test_expired_wait_reports_timeout_and_context_survives(which, precision):
    """small: the small-block tensor-core kernel; large: the large-block
    kernels (tensor cores for TF32X3, the float64 and two-float persistent
    kernel for FP64 and F32X2, whose grid barriers are bounded the same way)."""
    if which == "small":
        imp = ctq.build_impurity(w.model_t2g(), device=0)
        batch = w.batch_t2g(64)
    else:
        cf = w.crystal_field_complex(10, 0.1, 99)
        p = w.ModelParams("dc", n_orb=5, l=2, interaction="slater", U=3.0, J=0.6, beta=10.0, mu=None, n0=2,
                          soc_xi=0.3, cf=cf, sector_mode="n", n_min=1, n_max=3)
        imp = ctq.build_impurity(p, device=0)
        batch = w.random_batch(np.random.default_rng(1), 10, p.beta, 8, 2, 8, gen="g2")
    if which == "large":
        expect = ctq.KERNEL_TC_LARGE if precision == ctq.TF32X3 else ctq.KERNEL_FP64_LARGE
        assert ctq.trace_kernel(imp, precision) == expect
    ref = _eval(imp, batch, precision)
    assert np.all(ref["status"] != ctq.CHAIN_ERR_TIMEOUT)
    bad = _eval(imp, batch, precision, timeout_ns=20_000_000, debug_flags=ctq.DEBUG_STALL_WAIT)
    assert np.all(bad["status"] == ctq.CHAIN_ERR_TIMEOUT)
    assert np.all(np.isnan(bad["log_abs"]))
    again = _eval(imp, batch, precision)
    assert np.array_equal(again["status"], ref["status"])
    fin = np.isfinite(ref["log_abs"])
    assert np.allclose(again["log_abs"][fin], ref["log_abs"][fin], rtol=0, atol=1e-9)

"""The allocation-free entry point ctq_eval_traces_static (for callers that
cannot give the library a device workspace: its scratch is a fixed array
inside the library).  Checked through the C ABI against ctq_eval_traces on the
same inputs, on two calls in a row (the array keeps the previous call's
contents, so the second call also checks that everything it reads is
re-initialised).  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu


def _results(log_abs, phase, status, bounds):
    torch.cuda.synchronize()
    return (log_abs.cpu().numpy().copy(), phase.cpu().numpy().copy(), status.cpu().numpy().copy(),
            bounds.cpu().numpy().copy())


@pytest.mark.parametrize("name,n_chains,precision", [("t2g", 4096, ctq.FP64), ("d5", 256, ctq.FP64),
                                                     ("t2g", 1024, ctq.TF32X3)])
def test_static_scratch_matches_workspace_path(name, n_chains, precision):
    imp = ctq.build_impurity(w.WORKLOADS[name][0](), device=0)
    batch = w.WORKLOADS[name][1]().subset(range(n_chains))
    db = ctq.DeviceBatch(batch)
    stream = torch.cuda.current_stream().cuda_stream
    ev = ctq.TraceEvaluator(imp, batch.n_chains, db.max_ops, precision=precision)
    assert ev.ws_bytes <= ctq.STATIC_SCRATCH_BYTES
    ev(db)
    ref = _results(ev.log_abs, ev.phase, ev.status, ev.bounds)
    la = torch.full_like(ev.log_abs, 7.0)
    ph = torch.full_like(ev.phase, 7.0)
    st = torch.full_like(ev.status, 77)
    bd = torch.full_like(ev.bounds, 7.0)
    for _ in range(2):  # two calls in a row share the library's scratch
        ctq.eval_traces_static(imp, batch.n_chains, batch.beta, db.offsets.data_ptr(), db.tau.data_ptr(),
                               db.op.data_ptr(), None, la.data_ptr(), ph.data_ptr(), st.data_ptr(), bd.data_ptr(),
                               stream, precision=precision, max_ops=db.max_ops)
        got = _results(la, ph, st, bd)
        # same kernels on the same inputs: the results agree to rounding of the
        # order in which work items were claimed (bitwise in practice)
        assert np.array_equal(got[2], ref[2])
        fin = np.isfinite(ref[0])
        assert np.array_equal(np.isfinite(got[0]), fin)
        assert np.allclose(got[0][fin], ref[0][fin], rtol=0, atol=1e-12 * np.abs(ref[0][fin]).max())
        assert np.allclose(got[1], ref[1], rtol=0, atol=1e-12)
        bf = np.isfinite(ref[3])
        assert np.allclose(got[3][bf], ref[3][bf], rtol=0, atol=1e-9)
        la.fill_(7.0)
        st.fill_(77)


def test_static_scratch_rejects_oversized_batches():
    imp = ctq.build_impurity(w.model_t2g(), device=0)
    big = w.batch_t2g(4096)
    db = ctq.DeviceBatch(big)
    n = 40000  # far beyond what the fixed scratch holds
    assert ctq.workspace_size(imp, n, max_ops=db.max_ops) > ctq.STATIC_SCRATCH_BYTES
    out = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    stt = torch.empty(n, dtype=torch.int32, device="cuda")
    offs = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ctq.CtqError) as e:
        ctq.eval_traces_static(imp, n, big.beta, offs.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None,
                               out.data_ptr(), out.data_ptr(), stt.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream, max_ops=db.max_ops)
    assert e.value.code == ctq.CTQ_ERR_WORKSPACE
    assert "static scratch" in str(e.value)

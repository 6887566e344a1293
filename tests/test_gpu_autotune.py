"""Autotuner on the GPU: every launch configuration it may pick computes the
same traces as the library default (FP64: to rounding of the reduction
order; tensor paths: identical products, so identical values), and tune()
returns one of its candidates and caches it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from paper_2010_08482_gb300 import autotune, ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu


def _run(imp, db, precision, tune):
    ev = ctq.TraceEvaluator(imp, db.n_chains, max(1, db.max_ops), precision=precision, tune=tune)
    ev(db)
    torch.cuda.synchronize()
    return ev.results(db.n_chains)


def _same(a, b, rtol):
    fin = np.isfinite(a["log_abs"])
    assert np.array_equal(fin, np.isfinite(b["log_abs"]))
    assert np.array_equal(a["status"], b["status"])
    assert np.allclose(a["log_abs"][fin], b["log_abs"][fin], rtol=0, atol=rtol)
    assert np.array_equal(np.sign(a["phase"][fin, 0]), np.sign(b["phase"][fin, 0]))


@pytest.mark.parametrize("name,precision,n,tol", [("t2g", ctq.FP64, 256, 1e-12), ("d5", ctq.FP64, 16, 1e-12),
                                                  ("t2g", ctq.BF16X3, 256, 0.0), ("d5", ctq.TF32, 32, 0.0)])
def test_every_candidate_agrees_with_default(name, precision, n, tol):
    p, mk = w.WORKLOADS[name]
    imp = ctq.build_impurity(p(), device=0)
    assert ctq.trace_kernel(imp, precision) == (ctq.KERNEL_FP64_SHARED if precision == ctq.FP64 else ctq.KERNEL_TC_SMALL)
    db = ctq.DeviceBatch(mk().subset(range(n)))
    ref = _run(imp, db, precision, {})
    cands = autotune.candidates(imp, precision)
    assert len(cands) >= 2
    for cand in cands[1:]:
        _same(_run(imp, db, precision, cand), ref, tol)


def test_big_engine_candidates_agree_with_default():
    cf = w.crystal_field_complex(10, 0.1, 99)
    p = w.ModelParams("dc", n_orb=5, l=2, interaction="slater", U=3.0, J=0.6, beta=10.0, mu=None, n0=2,
                      soc_xi=0.3, cf=cf, sector_mode="n", n_min=1, n_max=3)
    imp = ctq.build_impurity(p, device=0)
    db = ctq.DeviceBatch(w.random_batch(np.random.default_rng(5), 10, p.beta, 6, 6, 12, gen="g2"))
    for prec in (ctq.TF32X3, ctq.BF16X3):
        ref = _run(imp, db, prec, {})
        ran = 0
        for cand in autotune.candidates(imp, prec)[1:]:
            try:
                res = _run(imp, db, prec, cand)
            except ctq.CtqError as exc:  # more stages than fit in shared memory: refused, as the tuner expects
                assert "unsupported" in str(exc)
                continue
            _same(res, ref, 0.0)
            ran += 1
        assert ran >= 2


def test_tune_picks_a_candidate_and_caches_it(tmp_path):
    imp = ctq.build_impurity(w.model_t2g(), device=0)
    db = ctq.DeviceBatch(w.batch_t2g(512))
    path = str(tmp_path / "tune.json")
    best = autotune.tune(imp, db, ctq.FP64, cache_path=path, reps=2)
    assert best in autotune.candidates(imp, ctq.FP64)
    cache = autotune.load_cache(path)
    assert len(cache) == 1
    entry = next(iter(cache.values()))
    assert entry["best"] == best and entry["ms"] == min(t["ms"] for t in entry["timings"])
    assert autotune.tune(imp, db, ctq.FP64, cache_path=path, cands=[{"threads_per_cta": 256}]) == best

"""Large-block tensor-core engine (k_trace_big: persistent cooperative kernel,
complex blocks in the real embedding, tiled operands): parity against the
FP64 oracle on models where the oracle is fast (a complex d shell with SOC
and complex crystal field, N in [1, 3], blocks up to 120; a real d shell
with sectors by N, N in [4, 6], blocks up to 252), and on the f shell against
stored oracle values (tests/golden/f7_oracle.json, written by
tests/golden/make_f7_oracle.py).

Mixed-precision errors are stated per model (STATED); the distributions are
printed."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def complex_d_model(beta=10.0):
    cf = w.crystal_field_complex(10, 0.1, 99)
    return w.ModelParams("dc", n_orb=5, l=2, interaction="slater", U=3.0, J=0.6, beta=beta, mu=None, n0=2,
                         soc_xi=0.3, cf=cf, sector_mode="n", n_min=1, n_max=3)


def real_d_window_model(beta=10.0):
    return w.ModelParams("dn", n_orb=5, l=2, interaction="slater", U=8.0, J=1.0, beta=beta, mu=None, n0=5,
                         sector_mode="n", n_min=4, n_max=6)


STATED = {("dc", ctq.TF32X3): 1e-4, ("dc", ctq.TF32): 5e-2, ("dn", ctq.TF32X3): 1e-4, ("dn", ctq.TF32): 5e-2,
          ("f7", ctq.TF32X3): 1e-3, ("f7", ctq.TF32): 0.1,
          ("dc", ctq.BF16X3): 2e-3, ("dn", ctq.BF16X3): 2e-3, ("f7", ctq.BF16X3): 3e-3}


def run(imp, batch, precision, S=8):
    db = ctq.DeviceBatch(batch)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, max(1, db.max_ops), precision=precision, segment=S)
    ev(db)
    torch.cuda.synchronize()
    return ev.results(batch.n_chains)


@pytest.fixture(scope="module")
def small_models():
    return {"dc": atom.Model(complex_d_model()), "dn": atom.Model(real_d_window_model())}


@pytest.mark.parametrize("precision", [ctq.TF32X3, ctq.TF32, ctq.BF16X3])
@pytest.mark.parametrize("name", ["dc", "dn"])
def test_big_engine_parity(name, precision, small_models):
    m = small_models[name]
    assert max(m.dims) > 112  # the large-block engine is the one that runs
    rng = np.random.default_rng(41)
    b = w.random_batch(rng, m.n_flav, m.beta, 12, 1, 14, gen="g2")
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, b, precision)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains))
    errs = []
    for c in range(b.n_chains):
        r = ref[c]
        if r["log_abs"] == -math.inf:
            continue
        err, kind = parity.chain_error(res["log_abs"][c], res["phase"][c], r)
        assert err <= STATED[(name, precision)], (c, err, kind)
        errs.append(err)
    assert errs
    print(f"{name} precision={precision}: n={len(errs)} max rel err {max(errs):.3e}, median {np.median(errs):.3e}")


# Bound on |D - A B^T| / (|A| |B|^T) elementwise: operand rounding of one
# pass (TF32: 2^-11 per operand), of the dropped lo*lo term and lo rounding
# (3xTF32: ~2^-21; bf16 hi / lo: ~2^-16), plus FP32 accumulation over K.
GEMM_TOL = {ctq.TF32: 3e-3, ctq.TF32X3: 2e-5, ctq.BF16X3: 1e-4}


@pytest.mark.parametrize("precision", [ctq.TF32, ctq.TF32X3, ctq.BF16X3])
@pytest.mark.parametrize("N,K", [(128, 64), (64, 256), (16, 1024), (96, 192)])
def test_big_gemm_conventions(precision, N, K):
    """Operand split, tiled layout, descriptors and MMA kind of the
    large-block engine on one tile: any transposed, shifted or mis-typed
    operand gives O(1) errors, rounding gives GEMM_TOL."""
    rng = np.random.default_rng(N * 7919 + K)
    A = rng.standard_normal((128, K)).astype(np.float32)
    Bm = rng.standard_normal((N, K)).astype(np.float32)
    D = ctq.big_gemm_check(A, Bm, precision)
    A64, B64 = A.astype(np.float64), Bm.astype(np.float64)
    ref = A64 @ B64.T
    scale = np.abs(A64) @ np.abs(B64).T
    err = float(np.max(np.abs(D - ref) / scale))
    print(f"precision={precision} N={N} K={K}: max err {err:.3e}")
    assert err < GEMM_TOL[precision]


def test_big_engine_bounds_bracket(small_models):
    """Segment bounds from the grid-reduced Frobenius norms bracket |w|."""
    m = small_models["dc"]
    rng = np.random.default_rng(43)
    b = w.random_batch(rng, m.n_flav, m.beta, 6, 8, 16, gen="g2")
    imp = parity.load_oracle_model(ctq, m)
    res = run(imp, b, ctq.TF32X3, S=4)
    ref = parity.oracle_chain_results(m, b, range(b.n_chains), noise=False)
    for c in range(b.n_chains):
        if ref[c]["log_abs"] == -math.inf:
            continue
        bd = res["bounds"][c]
        fin = bd[np.isfinite(bd)]
        assert np.all(fin >= ref[c]["log_abs"] - 1e-3)


def _f7_golden():
    path = os.path.join(HERE, "golden", "f7_oracle.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/f7_oracle.json not generated")
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def f7_impurity():
    return ctq.build_impurity(w.model_f7(), device=0)


def test_f7_build_matches_stored_oracle_spectrum(f7_impurity):
    """Library-built f shell (device eigensolver for the 1001 / 2002 / 3003
    sectors): sector sizes, chemical potential and ground-state energy agree
    with the oracle's stored values."""
    g = _f7_golden()
    dims, N, Emin, s = f7_impurity.sectors()
    assert list(dims) == g["dims"]
    assert f7_impurity.mu == pytest.approx(g["mu"], abs=1e-9)
    assert f7_impurity.E_gs == pytest.approx(g["E_gs"], abs=1e-9)
    assert f7_impurity.is_complex


@pytest.mark.parametrize("precision", [ctq.TF32X3, ctq.TF32, ctq.BF16X3])
def test_f7_traces_against_stored_oracle(precision, f7_impurity):
    g = _f7_golden()
    n = len(g["chains"])
    b = w.batch_f7().subset(range(n))
    res = run(f7_impurity, b, precision)
    errs = []
    for c, ref in enumerate(g["chains"]):
        r = {"log_abs": ref["log_abs"], "phase": complex(*ref["phase"]), "per_q0": {}}
        err = abs(complex(*res["phase"][c]) * math.exp(res["log_abs"][c] - r["log_abs"]) - r["phase"])
        errs.append(err)
        assert err <= STATED[("f7", precision)], (c, err)
        assert res["status"][c] == ctq.CHAIN_OK
    print(f"f7 precision={precision}: n={len(errs)} max rel err {max(errs):.3e}, median {np.median(errs):.3e}")

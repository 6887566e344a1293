"""Reduced-density-matrix estimator on the GPU (ctq_eval_density_matrices,
Eq. ImpurityDensityMatrix) against the FP64 oracle (oracle/observables.py)
element by element, on the oracle's eigenbasis; unit trace of every chain's
estimator at the full t2g batch size; a complex impurity; empty sequences
(the thermal density matrix)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from oracle import observables as OB  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu


def complex_two_orbital():
    cf = w.crystal_field_complex(4, 0.3, 123)
    return w.ModelParams("h2c", n_orb=2, l=0, interaction="kanamori", U=4.0, J=0.5, beta=10.0, mu=2.0, n0=2,
                         cf=cf, sector_mode="n")


def run(imp, batch):
    db = ctq.DeviceBatch(batch)
    ev = ctq.DensityEvaluator(imp, batch.n_chains, max(1, db.max_ops))
    ev(db)
    torch.cuda.synchronize()
    return ev


def check_against_oracle(m, batch, chains, ev, rel):
    st = ev.status.cpu().numpy()
    n_live = 0
    for c in chains:
        ref, wv = OB.density_matrix_chain(m, *batch.chain(int(c)), beta=batch.beta)
        got = ev.blocks(int(c))
        if ref is None:
            assert st[c] == ctq.CHAIN_ZERO
            assert all(np.all(got[q] == 0) for q in got)
            continue
        n_live += 1
        scale = max(np.abs(ref[q]).max() for q in ref)
        for q in ref:
            err = np.abs(got[q] - ref[q]).max() / scale
            assert err <= rel, (c, q, err)
    return n_live


@pytest.mark.parametrize("name,n,rel", [("hubbard2", 64, 1e-11), ("t2g", 96, 1e-10), ("d5", 6, 1e-9)])
def test_density_matrix_parity(name, n, rel, models):
    m = models(name)
    sub = w.WORKLOADS[name][1]().subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    ev = run(imp, sub)
    assert check_against_oracle(m, sub, range(n), ev, rel) >= min(n, 5)


def test_density_matrix_complex_impurity():
    m = atom.Model(complex_two_orbital())
    assert m.is_complex
    rng = np.random.default_rng(29)
    b = w.random_batch(rng, m.n_flav, m.beta, 24, 1, 8)
    imp = parity.load_oracle_model(ctq, m)
    ev = run(imp, b)
    assert check_against_oracle(m, b, range(b.n_chains), ev, 1e-10) >= 5


def test_empty_sequences_give_the_thermal_density_matrix(models):
    m = models("t2g")
    imp = parity.load_oracle_model(ctq, m)
    empty = w.Batch(beta=m.beta, offsets=np.zeros(3, np.int32), tau=np.zeros(0), op=np.zeros(0, np.int32))
    db = ctq.DeviceBatch(empty)
    ev = ctq.DensityEvaluator(imp, 2, 4)
    ev(db)
    torch.cuda.synchronize()
    th = OB.thermal_density_matrix(m)
    for c in range(2):
        got = ev.blocks(c)
        for q in th:
            np.testing.assert_allclose(got[q], th[q], rtol=1e-12, atol=1e-15)


def test_unit_trace_full_batch():
    """Every chain of the 4096-chain t2g batch: Tr rho^C = 1 (the intervals
    tile [0, beta)), through the library-built impurity."""
    imp = ctq.build_impurity(w.model_t2g(), device=0)
    b = w.batch_t2g()
    ev = run(imp, b)
    rho = ev.rho.cpu().numpy().reshape(b.n_chains, ev.size)
    dims = imp.sectors()[0]
    diag_idx, o = [], 0
    for d in dims:
        d = int(d)
        diag_idx += [o + u * d + u for u in range(d)]
        o += d * d
    tr = rho[:, diag_idx].sum(axis=1)
    st = ev.status.cpu().numpy()
    live = st == ctq.CHAIN_OK
    assert live.sum() > 4000
    assert np.max(np.abs(tr[live] - 1.0)) < 1e-11
    assert np.all(tr[~live] == 0.0)

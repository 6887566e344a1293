"""The stored d-shell oracle values (tests/golden/d5_oracle.json, written by
make_d5_oracle.py from the oracle only) against a fresh oracle evaluation of
a few of their chains on the CPU, and the mixed-precision bar rule of
tests/parity.py on hand-made cases."""
import math

import pytest

import parity
from oracle import atom
from oracle import trace as OT
from paper_2010_08482_gb300 import workloads as w


def test_stored_values_are_the_oracle():
    n, ref = parity.gold_d5()
    assert n == len(ref) == 1024
    m = atom.Model(w.model_d5())
    b = w.batch_d5()
    for c in (0, 101, 383, 1023):
        tau, ops = b.chain(c)
        r = OT.trace_chain(m, tau, ops, beta=b.beta)
        assert ref[c]["n_ops"] == len(ops)
        assert abs(r["log_abs"] - ref[c]["log_abs"]) <= 1e-12 * abs(r["log_abs"]) + 1e-12
        assert complex(r["phase"]) == pytest.approx(ref[c]["phase"], abs=1e-12)
        assert set(ref[c]["per_q0"]) == set(int(q) for q in r["per_q0"])
    assert all(ref[c]["noise"] >= 0.0 for c in ref)


def test_mixed_bar_rule():
    bars = parity.Bars("rule")
    u = parity.UNIT[2]
    well = {"noise": 0.0}
    assert bars.mixed(0, well, 1e-2, u, err=5e-3) == 1e-2
    kappa = 1e4  # unit x kappa = 0.15: the first-order error on that chain
    ill = {"noise": kappa * parity.U64}
    assert bars.mixed(1, ill, 1e-2, u, err=5e-3) == pytest.approx(u * kappa)
    assert bars.widened == []  # its error did not need the wider bar
    assert bars.mixed(2, ill, 1e-2, u, err=5e-2) == pytest.approx(u * kappa)
    assert [c for c, _, _ in bars.widened] == [2]
    mid = {"noise": 2000 * parity.U64}  # unit x kappa = 0.0305
    assert bars.mixed(3, mid, 1e-2, u) == pytest.approx(u * 2000)
    lost = {"noise": 2.0 ** 17 * parity.U64}  # unit x kappa = 2: no digit left
    assert bars.mixed(4, lost, 1e-2, u, err=3.0) == math.inf
    assert [c for c, _, _ in bars.unresolved] == [4]
    assert math.isclose(parity.UNIT[3], 2.0 ** -19)

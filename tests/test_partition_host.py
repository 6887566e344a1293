"""Host logic of the partition-space sampler (paper_2010_08482_gb300.partition)
on the CPU: the local traces come from the FP64 oracle instead of the GPU
(the sampler's evaluation hook is replaced in this test only).  Checks the
O(k^2) determinant updates against direct inverses, the sign conventions
(every weight of the particle-hole symmetric single-orbital model is
positive), and a short run against exact diagonalisation."""
import math

import numpy as np
import pytest

from oracle import atom
from oracle import ed
from oracle import trace as OT
from paper_2010_08482_gb300 import ctq
from paper_2010_08482_gb300 import partition as P
from paper_2010_08482_gb300 import workloads as w

EPS = [-0.5, 0.0, 0.5]
V = [1.0, 1.0, 1.0]


class _HostImpurity:
    """What the sampler reads from an impurity: n_flav and sectors()."""

    def __init__(self, m):
        self.m = m
        self.n_flav = m.n_flav

    def sectors(self):
        return (np.asarray(self.m.dims), np.asarray(self.m.N), np.asarray(self.m.E_min), self.m.s)


class OracleSampler(P.PartitionSampler):
    """The sampler with every local trace from the oracle: thresholds are
    decided exactly (accept iff log|w| >= T), never early."""

    def __init__(self, m, *a, **k):
        self.m = m
        super().__init__(_HostImpurity(m), *a, **k)

    def _make_evaluator(self):
        return None

    def _evaluate(self, seqs, thresholds):
        st, la, ph = [], [], []
        for i, (t, o) in enumerate(seqs):
            r = OT.trace_chain(self.m, t, o, beta=self.beta)
            la.append(r["log_abs"])
            ph.append((complex(r["phase"]).real, complex(r["phase"]).imag))
            if thresholds is None:
                st.append(ctq.CHAIN_OK if r["log_abs"] != -math.inf else ctq.CHAIN_ZERO)
            else:
                st.append(ctq.CHAIN_ACCEPTED if OT.decide(r["log_abs"], thresholds[i]) else ctq.CHAIN_REJECTED)
        return np.asarray(st), np.asarray(la), np.asarray(ph)


def model(U, beta):
    return atom.Model(w.model_atom1(U=U, mu=U / 2, beta=beta))


def test_fast_updates_and_signs():
    """After every accepted move: M^{-1} equals the inverse of M built from
    the times, the tracked sign of det M is right, and the weight of the
    particle-hole symmetric model is positive."""
    m = model(4.0, 5.0)
    s = OracleSampler(m, EPS, V, 5.0, n_chains=6, seed=3, max_ops=64)
    n_checked = 0
    for _ in range(300):
        s.step(measure=False)
        for ch in s.chains:
            for f in range(s.nf):
                if len(ch.cre[f]) == 0:
                    continue
                M = P.hybridisation(EPS, V, 5.0, ch.cre[f][:, None] - ch.ann[f][None, :])
                assert np.allclose(ch.minv[f], np.linalg.inv(M), rtol=1e-9, atol=1e-9)
                assert ch.det_sign[f] == np.sign(np.linalg.det(M))
                n_checked += 1
            assert ch.perm_sign == ch.sequence()[2]  # the tracked parity is the recomputed one
            assert s.weight_sign(ch) == 1.0
    assert n_checked > 100 and s.n_acc > 50


def test_proposal_ratios_are_reverse_over_forward():
    """Insertion into an empty flavour has ratio beta^2 and its removal
    1/beta^2; with N operators present the insertion ratio is
    [1/(N+2)] / [(1/N) 2/L^2] (N L^2 / (2 (N + 2)))."""
    m = model(4.0, 5.0)
    s = OracleSampler(m, EPS, V, 5.0, n_chains=1, seed=1, max_ops=64)
    ch = s.chains[0]
    seen = {"ins0": False, "rem2": False, "insN": False}
    for _ in range(400):
        pr = s._propose(ch)
        if pr is None:
            continue
        t_f, _ = s._flavour_ops(ch, pr["f"])
        N = len(t_f)
        if pr["kind"] == "ins" and N == 0:
            assert pr["prop"] == pytest.approx(25.0)
            seen["ins0"] = True
        elif pr["kind"] == "rem" and N == 2:
            assert pr["prop"] == pytest.approx(1 / 25.0)
            seen["rem2"] = True
        elif pr["kind"] == "ins":
            # the interval that holds the new pair, between consecutive flavour-f operators
            tt = np.sort(t_f)
            lo = tt[np.searchsorted(tt, pr["tc"]) - 1] if np.searchsorted(tt, pr["tc"]) > 0 else tt[-1] - 5.0
            hi = tt[np.searchsorted(tt, pr["tc"])] if np.searchsorted(tt, pr["tc"]) < N else tt[0] + 5.0
            L = hi - lo
            assert pr["prop"] == pytest.approx(N * L * L / (2.0 * (N + 2)), rel=1e-12)
            seen["insN"] = True
        s._apply(ch, pr)
    assert all(seen.values())


def test_short_run_matches_exact_diagonalisation():
    """Hubbard atom with three bath levels at beta = 2 (low orders): the mean
    expansion order and G(tau) in the middle bin agree with ED within 5
    standard errors of the chain-to-chain spread."""
    beta, U = 2.0, 4.0
    m = model(U, beta)
    x = ed.ImpurityED(w.model_atom1(U=U, mu=U / 2, beta=beta), U / 2, EPS, V, beta)
    s = OracleSampler(m, EPS, V, beta, n_chains=16, seed=11, max_ops=64, n_bins=10)
    s.run(800, n_burn=100)
    est = s.estimates()
    k_mean, k_err = est["order"]
    assert abs(k_mean - x.mean_order()) <= 5 * k_err + 1e-3, (k_mean, k_err, x.mean_order())
    g_mean, g_err = est["green"]
    for b in (2, 5):
        ref = x.green_bin(0, b * beta / 10, (b + 1) * beta / 10)
        got = 0.5 * (g_mean[0][b] + g_mean[1][b])
        err = 0.5 * math.hypot(g_err[0][b], g_err[1][b])
        assert abs(got - ref) <= 5 * err + 1e-3, (b, got, err, ref)
    assert est["sign"][0] == 1.0

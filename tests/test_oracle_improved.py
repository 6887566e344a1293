"""Pins for oracle.improved (the static part of the improved estimator,
Eq. PImprovedEstimatorStatic): a closed form for the Hubbard atom, the
equation of motion of a time-evolved annihilator (a derivative in tau that
no part of the oracle's Bulla construction uses), and the commutator with H
written in the eigenbasis."""
import math

import numpy as np
import pytest

from oracle import atom
from oracle import improved as I
from oracle import trace as T
from paper_2010_08482_gb300 import workloads as w


def value(r, ref_log=0.0):
    """w e^{-ref_log} as a complex number from a trace_chain result."""
    if r["log_abs"] == -math.inf:
        return 0j
    return complex(r["phase"]) * math.exp(r["log_abs"] - ref_log)


@pytest.mark.parametrize("f", [0, 1])
def test_hubbard_atom_closed_form(f):
    """H = eps (n_0 + n_1) + U n_0 n_1 with eps = -mu: [c_f, U n_0 n_1] =
    U c_f n_fbar.  For c+_f at tau1 then c_f at tau2 only the initial state
    |fbar> passes the Bulla operator; for c_f first, only |0 1>."""
    U, mu, beta = 3.0, 1.0, 5.0
    m = I.with_bulla(atom.Model(w.model_atom1(U, mu, beta)))
    eps = -mu
    for t1, t2 in ((0.3, 1.7), (1.1, 4.6), (0.01, 4.99)):
        tau = np.array([t1, t2])
        # creation first
        ops = np.array([2 * f + 1, 2 * f])
        both = math.exp(-(beta - t2) * eps - (t2 - t1) * (2 * eps + U) - t1 * eps)
        w0 = math.exp(-(t2 - t1) * eps) + both
        assert value(T.trace_chain(m, tau, ops)) == pytest.approx(w0, rel=1e-13)
        wu = value(T.trace_chain(m, tau, I.bulla_sequence(m, ops, 1)))
        assert wu == pytest.approx(U * both, rel=1e-13)
        (pos, h), = I.static_ratios(m, tau, ops)
        assert pos == 1 and h == pytest.approx(U * both / w0, rel=1e-12)
        # annihilation first
        ops = np.array([2 * f, 2 * f + 1])
        both = math.exp(-t1 * (2 * eps + U) - (t2 - t1) * eps - (beta - t2) * (2 * eps + U))
        w0 = math.exp(-eps * (beta - t2 + t1)) + both
        assert value(T.trace_chain(m, tau, ops)) == pytest.approx(w0, rel=1e-13)
        (pos, h), = I.static_ratios(m, tau, ops)
        assert pos == 0 and h == pytest.approx(U * both / w0, rel=1e-12)


def small_complex_model():
    cf = w.crystal_field_complex(4, 0.3, 17)
    return w.ModelParams("k2c", n_orb=2, l=0, interaction="kanamori", U=3.0, J=0.6, beta=4.0, mu=1.1,
                         n0=2, cf=cf, sector_mode="n")


def derivative(m, tau, ops, pos, ref_log):
    """d w / d tau_pos by central differences with one Richardson step."""
    lo = tau[pos - 1] if pos > 0 else 0.0
    hi = tau[pos + 1] if pos + 1 < len(tau) else m.beta
    d = min(0.25 * min(tau[pos] - lo, hi - tau[pos]), 1e-2)

    def wt(x):
        t = tau.copy()
        t[pos] = x
        return value(T.trace_chain(m, t, ops), ref_log)

    D1 = (wt(tau[pos] + d) - wt(tau[pos] - d)) / (2 * d)
    D2 = (wt(tau[pos] + d / 2) - wt(tau[pos] - d / 2)) / d
    return (4 * D2 - D1) / 3, d


@pytest.mark.parametrize("which", ["hubbard2", "complex"])
def test_equation_of_motion(which, models):
    """d/dtau of the time-evolved c_f(tau) = e^{tau H} c_f e^{-tau H} is
    [H, c_f] = -[c_f, U] - sum_j h_fj c_j (h = t - mu, the one-body part), so

        w^U_s = - dw/dtau_s - sum_j h_fj w(c_f -> c_j at tau_s).

    The left side uses the Bulla blocks; the right side only ordinary traces
    at shifted times and the one-body matrix."""
    if which == "hubbard2":
        m0 = models("hubbard2")
    else:
        m0 = atom.Model(small_complex_model())
    m = I.with_bulla(m0)
    h = atom.one_body_matrix(m0.params, m0.mu)
    rng = np.random.default_rng(8)
    b = w.random_batch(rng, m0.n_flav, m0.beta, 8, 2, 6)
    n_cmp = 0
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        tau = np.asarray(tau, np.float64)
        base = T.trace_chain(m, tau, ops)
        if base["log_abs"] == -math.inf:
            continue
        L = base["log_abs"]
        for pos in I.annihilators(m, ops):
            f = int(ops[pos]) // 2
            lhs = value(T.trace_chain(m, tau, I.bulla_sequence(m, ops, pos)), L)
            dw, d = derivative(m, tau, ops, pos, L)
            rhs = -dw
            scale = abs(dw) + abs(lhs)
            for j in range(m0.n_flav):
                if h[f, j] == 0:
                    continue
                o2 = np.array(ops).copy()
                o2[pos] = 2 * j
                wj = value(T.trace_chain(m, tau, o2), L)
                rhs -= h[f, j] * wj
                scale += abs(h[f, j] * wj)
            if not m0.is_complex:
                assert isinstance(lhs.real, float)
            assert abs(lhs - rhs) <= 1e-6 * max(scale, 1.0), (c, pos, lhs, rhs, d)
            n_cmp += 1
    assert n_cmp >= 10


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_bulla_blocks_are_the_commutator_with_h_in_the_eigenbasis(name, models):
    """<m|[c_f, H]|n> = F_mn (E_n - E_m) in the eigenbasis of H, and
    [c_f, H - U] = sum_j h_fj c_j, so the Bulla block must equal
    F_f(q) o (E_q,n - E_q',m) - sum_j h_fj F_j(q) (o: elementwise)."""
    m0 = models(name)
    m = I.with_bulla(m0)
    h = atom.one_body_matrix(m0.params, m0.mu)
    nf = m0.n_flav
    worst = 0.0
    for f in range(nf):
        for q in range(m0.n_sec):
            qp = int(m0.s[2 * f, q])
            assert int(m.s[I.bulla_code(nf, f), q]) == qp
            if qp < 0:
                continue
            F = m0.F[(2 * f, q)]
            ref = F * (m0.E[q][None, :] - m0.E[qp][:, None])
            for j in range(nf):
                if h[f, j] != 0 and int(m0.s[2 * j, q]) >= 0:
                    assert int(m0.s[2 * j, q]) == qp
                    ref = ref - h[f, j] * m0.F[(2 * j, q)]
            B = m.F[(I.bulla_code(nf, f), q)]
            err = np.abs(B - ref).max() / max(1.0, np.abs(ref).max())
            worst = max(worst, err)
    assert worst < 1e-11, worst


def test_dead_backward_cases_have_the_stated_property(models):
    """The fixture tests/golden/t2g_dead_backward.json: for some surviving
    starting sector the product of the operators after position j (taken from
    the end of the string) is exactly zero for a j with an annihilator before
    it, the forward products up to the last operator are nonzero, and w != 0
    (another starting sector carries it), so the ratios of those earlier
    annihilators come from the other sectors."""
    import json
    import os
    from oracle import trace as T
    m = models("t2g")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "t2g_dead_backward.json")
    with open(path) as f:
        cases = json.load(f)["chains"]
    assert len(cases) >= 2
    for case in cases:
        tau, ops = np.asarray(case["tau"]), np.asarray(case["op"], np.int64)
        n = len(ops)
        assert T.trace_chain(m, tau, ops)["log_abs"] != -math.inf
        surv = [q0 for q0 in range(m.n_sec) if T.walk(m, ops, q0) is not None]
        hit = False
        for q0 in surv:
            path_q = T.walk(m, ops, q0)
            A = np.eye(m.dims[q0])
            fwd = []
            for i in range(n - 1):
                A = m.F[(int(ops[i]), path_q[i])] @ A
                fwd.append(bool(np.any(A)))
            Y = np.eye(m.dims[q0])
            dead = None
            for i in range(n - 1, -1, -1):
                Y = Y @ m.F[(int(ops[i]), path_q[i])]
                if not np.any(Y):
                    dead = i
                    break
            if all(fwd) and dead is not None and any(ops[j] % 2 == 0 for j in range(dead)):
                hit = True
        assert hit

"""Pins for oracle.trace: closed forms, brute force over the full Fock space,
exact symmetries and bound validity."""
import math

import numpy as np
import pytest

from oracle import atom
from oracle import trace as T
from paper_2010_08482_gb300 import workloads as w


def value(r):
    """w as a complex number from a trace_chain result (0 if log|w| = -inf)."""
    if r["log_abs"] == -math.inf:
        return 0.0
    return complex(r["phase"]) * math.exp(r["log_abs"])


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_log(r, ref):
    """|w - w_ref| / |w_ref| for values held as (log|w|, phase)."""
    if ref["log_abs"] == -math.inf:
        return 0.0 if r["log_abs"] == -math.inf else math.inf
    return abs(complex(r["phase"]) * math.exp(r["log_abs"] - ref["log_abs"]) - complex(ref["phase"]))


# ---------------------------------------------------------------- Z (empty sequence)

def test_partition_function_density_density_closed_form():
    """J = 0: H is diagonal in occupations; Z = sum_n exp(-beta E_n) with
    E_n = -mu N + U sum_a n_a,up n_a,dn + U sum_{a != b} n_a,up n_b,dn
          + U sum_{a<b,s} n_a,s n_b,s   (no eigensolver involved)."""
    n_orb, U, mu, beta = 2, 3.0, 1.2, 7.0
    p = w.ModelParams("dd", n_orb=n_orb, l=0, interaction="kanamori", U=U, J=0.0, beta=beta, mu=mu,
                      n0=2)
    m = atom.Model(p)
    Z = 0.0
    for s in range(1 << (2 * n_orb)):
        n = [(s >> f) & 1 for f in range(2 * n_orb)]
        dn, up = n[:n_orb], n[n_orb:]
        E = -mu * sum(n)
        E += U * sum(dn[a] * up[a] for a in range(n_orb))
        E += U * sum(up[a] * dn[b] for a in range(n_orb) for b in range(n_orb) if a != b)
        E += U * sum(x[a] * x[b] for x in (dn, up) for a in range(n_orb) for b in range(a + 1, n_orb))
        Z += math.exp(-beta * E)
    r = T.trace_chain(m, [], [])
    assert r["phase"] == 1.0
    assert rel(math.exp(r["log_abs"]), Z) < 1e-13


def test_partition_function_matches_expm(models):
    m = models("hubbard2")
    H = atom.full_hamiltonian(m.params, m.mu).real
    Z = T.trace_full_space(H, None, [], [], m.beta)
    r = T.trace_chain(m, [], [])
    assert rel(math.exp(r["log_abs"]), Z) < 1e-12


# ---------------------------------------------------------------- brute force

@pytest.fixture(scope="module")
def brute_hubbard2(models):
    m = models("hubbard2")
    n_f = m.n_flav
    H = atom.full_hamiltonian(m.params, m.mu).real
    mats = {2 * f + d: atom.full_op_matrix(n_f, f, d) for f in range(n_f) for d in (0, 1)}
    return m, H, mats


def test_sector_trace_equals_full_space_expm(brute_hubbard2):
    """Sector-string trace == Tr over the 16-dim Fock space with expm
    propagators and no eigenbasis, on seeded G1 chains and on unstructured
    operator strings (which mostly vanish)."""
    m, H, mats = brute_hubbard2
    rng = np.random.default_rng(7)
    b1 = w.random_batch(rng, m.n_flav, m.beta, 24, 1, 6)
    b2 = w.uniform_random_ops_batch(rng, m.n_flav, m.beta, 24, 0, 6)
    n_nonzero = 0
    for b in (b1, b2):
        for c in range(b.n_chains):
            tau, ops = b.chain(c)
            ref = T.trace_full_space(H, mats, tau, ops, m.beta)
            got = value(T.trace_chain(m, tau, ops))
            scale = max(abs(ref), 1e-12 * math.exp(T.trace_chain(m, [], [])["log_abs"]))
            assert abs(got - ref) <= 1e-11 * scale
            n_nonzero += abs(ref) > 0
    assert n_nonzero >= 24


def test_complex_model_against_full_space():
    """Complex model (d shell with SOC and complex CF, N in [1, 3]): sector trace
    equals the brute-force trace over the truncated space."""
    cf = w.crystal_field_complex(10, 0.1, 99)
    p = w.ModelParams("dc", n_orb=5, l=2, interaction="slater", U=3.0, J=0.6, beta=2.0, mu=None,
                      n0=2, soc_xi=0.3, cf=cf, sector_mode="n", n_min=1, n_max=3)
    m = atom.Model(p)
    assert m.is_complex
    states = np.concatenate(m.states)
    order = np.argsort(states)
    states = states[order]
    H = atom.sector_hamiltonian(states, atom.hamiltonian_terms(p, m.mu))
    mats = {}
    for f in range(10):
        for d in (0, 1):
            ok, sign, new = atom.apply_op(states, f, d)
            cols = np.nonzero(ok)[0]
            idx = np.minimum(np.searchsorted(states, new[cols]), len(states) - 1)
            keep = states[idx] == new[cols]
            M = np.zeros((len(states), len(states)))
            M[idx[keep], cols[keep]] = sign[cols[keep]]
            mats[2 * f + d] = M
    rng = np.random.default_rng(11)
    b = w.random_batch(rng, 10, p.beta, 6, 1, 3, gen="g2")
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        ref = T.trace_full_space(H, mats, tau, ops, p.beta)
        got = value(T.trace_chain(m, tau, ops))
        assert abs(got - ref) <= 1e-10 * abs(ref)


# ---------------------------------------------------------------- Green function

def test_atomic_green_function_closed_form():
    """Hubbard atom: G(tau) = -[e^{-tau eps} + e^{-beta eps} e^{-tau(eps+U)}]/Z,
    Z = 1 + 2 e^{-beta eps} + e^{-beta(2 eps + U)}, eps = -mu."""
    U, mu, beta = 3.0, 1.0, 5.0
    m = atom.Model(w.model_atom1(U, mu, beta))
    eps = -mu
    Z = 1 + 2 * math.exp(-beta * eps) + math.exp(-beta * (2 * eps + U))
    for f in (0, 1):
        for t in (0.1, 1.3, 2.5, 4.9):
            ref = -(math.exp(-t * eps) + math.exp(-beta * eps) * math.exp(-t * (eps + U))) / Z
            assert T.green_atomic(m, f, t) == pytest.approx(ref, rel=1e-13)


def test_green_sum_rule(models):
    """G(0+) + G(beta-) = -1 for every flavour (anticommutator)."""
    m = models("hubbard2")
    for f in range(m.n_flav):
        g0 = T.green_atomic(m, f, 1e-12)
        gb = T.green_atomic(m, f, m.beta - 1e-12)
        assert g0 + gb == pytest.approx(-1.0, abs=1e-9)


# ---------------------------------------------------------------- symmetries

@pytest.mark.parametrize("name", ["hubbard2", "t2g"])
def test_cyclic_invariance(name, models):
    """Rotating all times by delta (mod beta) and re-sorting leaves the matrix
    trace unchanged."""
    m = models(name)
    rng = np.random.default_rng(3)
    b = w.random_batch(rng, m.n_flav, m.beta, 10, 2, 12)
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        delta = rng.uniform(0, m.beta)
        t2 = (tau + delta) % m.beta
        order = np.argsort(t2)
        a = T.trace_chain(m, tau, ops)
        r = T.trace_chain(m, t2[order], ops[order])
        assert rel_log(r, a) < 1e-11


def test_conjugation_symmetry():
    """Reversing the sequence, daggering every operator and mapping
    tau -> beta - tau gives w* (complex model)."""
    cf = w.crystal_field_complex(10, 0.1, 5)
    p = w.ModelParams("dc", n_orb=5, l=2, interaction="slater", U=3.0, J=0.6, beta=4.0, mu=None,
                      n0=2, soc_xi=0.3, cf=cf, sector_mode="n", n_min=1, n_max=3)
    m = atom.Model(p)
    rng = np.random.default_rng(5)
    b = w.random_batch(rng, 10, p.beta, 8, 2, 4, gen="g2")
    n_complex = 0
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        if tau[0] == 0.0:
            continue
        a = value(T.trace_chain(m, tau, ops))
        t2 = (p.beta - tau)[::-1]
        o2 = (ops ^ 1)[::-1]
        bconj = value(T.trace_chain(m, t2, o2))
        assert abs(bconj - np.conj(a)) <= 1e-11 * abs(a)
        n_complex += abs(np.imag(a)) > 1e-6 * abs(a)
    assert n_complex >= 4  # the check is not vacuous


def test_charge_violating_sequences_vanish(models):
    m = models("t2g")
    r = T.trace_chain(m, [0.5, 1.0, 2.0], [1, 3, 0])
    assert r["log_abs"] == -math.inf and not r["per_q0"]
    r = T.trace_chain(m, [0.5, 1.0], [1, 3])
    assert r["log_abs"] == -math.inf


def test_pauli_violation_vanishes_density_density():
    """J = 0 (no flavour mixing): c+_f c+_f on the same flavour is zero even
    though the charge returns."""
    p = w.ModelParams("dd", n_orb=2, l=0, interaction="kanamori", U=3.0, J=0.0, beta=5.0, mu=1.0, n0=2)
    m = atom.Model(p)
    r = T.trace_chain(m, [0.1, 0.2, 0.3, 0.4], [1, 1, 0, 0])
    assert r["log_abs"] == -math.inf


# ---------------------------------------------------------------- bounds

@pytest.mark.parametrize("name", ["hubbard2", "t2g"])
def test_bounds_bracket_and_decrease(name, models):
    m = models(name)
    b = (w.batch_hubbard2() if name == "hubbard2" else w.batch_t2g(64))
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        r = T.trace_chain(m, tau, ops)
        B, ub = T.chain_bounds(m, tau, ops, b.beta, 8)
        assert B >= r["log_abs"] - 1e-12
        assert all(u >= r["log_abs"] - 1e-12 for u in ub)
        assert all(ub[i + 1] <= ub[i] + 1e-12 for i in range(len(ub) - 1))
        # the last refined bound is the sum of |w_q0|, which brackets |w|
        logs = [v[0] for v in r["per_q0"].values() if v[0] != -math.inf]
        if logs:
            mx = max(logs)
            ls = mx + math.log(sum(math.exp(x - mx) for x in logs))
            assert ub[-1] == pytest.approx(ls, abs=1e-12)


def test_level0_bound_is_tight_for_single_state():
    """One state per sector (U only, 1 orbital): ||F||_2 = 1, r = 1 and the
    propagators are scalars, so the level-0 bound equals |w|."""
    m = atom.Model(w.model_atom1(3.0, 1.0, 5.0))
    tau, ops = [0.3, 2.0, 3.5, 4.0], [1, 3, 0, 2]
    r = T.trace_chain(m, tau, ops)
    B, ub = T.chain_bounds(m, tau, ops, m.beta, 2)
    assert B == pytest.approx(r["log_abs"], abs=1e-12)


def test_refined_bounds_are_tight_for_single_state():
    """One state per sector: every block is 1 x 1 with |F| = ||F||_2 = 1,
    r = 1 and each propagator is the scalar e^{-dtau E_min}, so every refined
    bound sqrt(r) ||Y_j||_F prod_{i>j} ||F_i||_2 e^{-dtau E_min} equals |w_q0|
    (a doubled or misplaced tail factor would break the equality)."""
    m = atom.Model(w.model_atom1(3.0, 1.0, 5.0))
    tau, ops = [0.3, 2.0, 3.5, 4.0, 4.2, 4.9], [1, 3, 0, 2, 1, 0]
    r = T.trace_chain(m, tau, ops)
    for S in (1, 2, 4):
        for q0, (lw, _) in r["per_q0"].items():
            ub = T.refined_bounds_q0(m, np.asarray(tau), np.asarray(ops), q0, m.beta, S)
            assert len(ub) == -(-len(ops) // S) + 1
            for u in ub:
                assert u == pytest.approx(lw, abs=1e-12), (S, q0, ub, lw)


class _TwoSectorModel:
    """Hand-built model: sectors q0 and q1 of dimension 2, operator 0 maps
    q0 -> q1 with block A, operator 1 maps q1 -> q0 with block B."""

    def __init__(self, A, B, E0, E1):
        self.n_sec = 2
        self.dims = [2, 2]
        self.s = np.array([[1, -1], [-1, 0]])
        self.F = {(0, 0): np.asarray(A, float), (1, 1): np.asarray(B, float)}
        self.E = [np.asarray(E0, float), np.asarray(E1, float)]
        self.E_min = [min(E0), min(E1)]
        self.E_gs = min(self.E_min)
        self.is_complex = False

    def opnorm(self, alpha, q):
        return float(np.linalg.norm(self.F[(alpha, q)], 2))


def test_refined_bounds_hand_built_two_by_two():
    """Values worked out by hand.  A = [[1, 1], [1, 1]] / 2 (a projector:
    ||A||_2 = ||A||_F = 1), B = I, energies 0 in q0 and 0.5 (twice) in q1,
    tau = (1, 3), beta = 10, one operator per segment (S = 1), r = 2:
      s = 0: sqrt(2) ||I||_F ||A||_2 e^{-2 * 0.5} ||B||_2 = 2 e^{-1}
      s = 1: sqrt(2) ||e^{-1} A||_F ||B||_2 = sqrt(2) e^{-1}
      s = 2: |Tr(B e^{-1} A)| = e^{-1}
    and the level-0 bound r ||A||_2 ||B||_2 e^{-1} = 2 e^{-1}."""
    m = _TwoSectorModel([[0.5, 0.5], [0.5, 0.5]], np.eye(2), [0.0, 0.0], [0.5, 0.5])
    tau, ops = np.array([1.0, 3.0]), np.array([0, 1])
    ub = T.refined_bounds_q0(m, tau, ops, 0, 10.0, 1)
    exp = [math.log(2.0) - 1.0, 0.5 * math.log(2.0) - 1.0, -1.0]
    assert ub == pytest.approx(exp, abs=1e-14)
    assert T.level0_bound(m, tau, ops, 0, 10.0) == pytest.approx(math.log(2.0) - 1.0, abs=1e-14)
    # the string starting in q1 dies at once (operator 0 annihilates q1)
    assert T.refined_bounds_q0(m, tau, ops, 1, 10.0, 1) is None
    r = T.trace_chain(m, tau, ops, beta=10.0)
    assert r["log_abs"] == pytest.approx(-1.0, abs=1e-14)


def test_decide_matches_threshold():
    assert T.decide(-1.0, -1.5) and not T.decide(-2.0, -1.5)


def test_left_and_right_association_agree(models):
    """Multiplying the string from the left or from the right gives the same
    trace to float64 rounding (well-conditioned chains)."""
    m = models("t2g")
    b = w.batch_t2g(40)
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        r = T.trace_chain(m, tau, ops)
        l = T.trace_chain_left(m, tau, ops)
        if r["log_abs"] == -math.inf:
            assert l["log_abs"] == -math.inf
            continue
        assert rel_log(l, r) < 1e-12


# ---------------------------------------------------------------- signed log-space sum

def la_or0(la):
    return 0.0 if la == -math.inf else la


def test_logsumexp_signed_exact():
    """The combine over starting sectors (Sec. 3.3.1: w is the sum of the
    per-sector traces, each held as a value and a log scale) against exact
    rational arithmetic: scales are whole multiples of log 2, so every term
    is a dyadic rational and the sum is exact.  Covers cancellation down to
    a few ulps of the largest term, zero values, -inf scales, an exactly
    cancelling sum and complex phases."""
    from fractions import Fraction
    LN2 = math.log(2.0)
    rng = np.random.default_rng(11)
    n_rel = 0
    for case in range(300):
        k = int(rng.integers(1, 7))
        cplx = case % 3 == 2
        terms, exact_re, exact_im = [], Fraction(0), Fraction(0)
        for _ in range(k):
            e = int(rng.integers(-900, 900)) if case % 5 else int(rng.integers(-3, 3))
            re = float(rng.integers(-2 ** 20, 2 ** 20)) / 2 ** 10
            im = float(rng.integers(-2 ** 20, 2 ** 20)) / 2 ** 10 if cplx else 0.0
            if rng.random() < 0.1:
                re, im = 0.0, 0.0
            v = complex(re, im) if cplx else re
            terms.append((v, e * LN2))
            exact_re += Fraction(re) * Fraction(2) ** e
            exact_im += Fraction(im) * Fraction(2) ** e
        if case % 7 == 0 and terms:  # an opposite copy of the first term: partial cancellation
            v0, l0 = terms[0]
            terms.append((-v0, l0))
            exact_re -= Fraction(v0.real if cplx else v0) * Fraction(2) ** round(l0 / LN2)
            exact_im -= Fraction(v0.imag if cplx else 0.0) * Fraction(2) ** round(l0 / LN2)
        terms.append((1.5, -math.inf))  # a dead sector contributes nothing
        la, ph = T.logsumexp_signed(terms)
        if exact_re == 0 and exact_im == 0:
            assert la == -math.inf and ph == 0.0
            continue
        live = [(v, l) for v, l in terms if v != 0 and l != -math.inf]
        # the largest term as a power of two 2^E (E = its scale in units of
        # log 2 plus the binary exponent of its value)
        E = max(round(l / LN2) + math.frexp(abs(v))[1] for v, l in live)
        # absolute pin: |w - w_exact| <= a few ulps of the largest term per term
        r_ex = complex(float(exact_re / Fraction(2) ** E), float(exact_im / Fraction(2) ** E))
        r = 0.0 if la == -math.inf else complex(ph) * math.exp(la - E * LN2)
        # (the second term: rounding of log|w| and of E log 2 in this check)
        tol_abs = 4 * len(live) * 2.0 ** -52 + 4 * abs(r_ex) * math.ulp(max(abs(la_or0(la)), abs(E * LN2)))
        assert abs(r - r_ex) <= tol_abs, (case, r, r_ex)
        # relative pin where the sum keeps most of its bits
        big = max(abs(exact_re), abs(exact_im))
        sh = big.numerator.bit_length() - big.denominator.bit_length()
        sre, sim = float(exact_re / Fraction(2) ** sh), float(exact_im / Fraction(2) ** sh)
        la_ex = sh * LN2 + math.log(abs(complex(sre, sim)))
        if E * LN2 - la_ex < 20.0:  # the sum keeps all but ~29 of its bits
            rel_tol = 4 * len(live) * 2.0 ** -52 * math.exp(E * LN2 - la_ex)
            assert abs(la - la_ex) <= rel_tol + 8 * math.ulp(abs(la_ex)), (case, la, la_ex)
            ph_ex = complex(sre, sim) / abs(complex(sre, sim))
            assert abs(complex(ph) - ph_ex) <= 2 * rel_tol + 1e-15, (case, ph, ph_ex)
            n_rel += 1
    assert n_rel > 200
    assert T.logsumexp_signed([]) == (-math.inf, 0.0)
    assert T.logsumexp_signed([(0.0, 3.0), (2.0, -math.inf)]) == (-math.inf, 0.0)


@pytest.mark.parametrize("name", ["hubbard2", "t2g"])
def test_split_association_agrees(name, models):
    """The split association (first half right to left, second half left
    to right, then the trace of their product) gives the same trace as the
    plain right-to-left product to float64 rounding."""
    m = models(name)
    b = (w.batch_hubbard2() if name == "hubbard2" else w.batch_t2g(64))
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        r = T.trace_chain(m, tau, ops)
        s = T.trace_chain_split(m, tau, ops)
        if r["log_abs"] == -math.inf:
            assert s["log_abs"] == -math.inf
            continue
        assert rel_log(s, r) < 1e-12, c

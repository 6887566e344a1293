"""CPU checks of libctq: the library loads, exports every declared symbol, and
its host-side model construction (Fock space, H_loc, sectors, Jacobi
eigensolver, eigenbasis blocks) agrees with the oracle on basis-invariant
quantities.  No GPU call is made here (device = -1)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import atom
from oracle import improved as OI
from oracle import trace as OT
from paper_2010_08482_gb300 import ctq
from paper_2010_08482_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ctq_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ctq.lib_path())
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_names_codes():
    assert ctq.strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6, -7):
        assert ctq.strerror(code) not in ("", "unknown error")


@pytest.fixture(scope="module")
def host_models():
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = ctq.build_impurity(w.WORKLOADS[name][0](), device=-1)
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_sectors_and_spectra_match_oracle(name, host_models, models):
    imp = host_models(name)
    m = models(name)
    dims, N, Emin, s = imp.sectors()
    assert imp.n_sec == m.n_sec and list(dims) == m.dims and list(N) == m.N
    assert imp.mu == pytest.approx(m.mu, abs=1e-12 * max(1, abs(m.mu)))
    scale = max(1.0, max(abs(e).max() for e in m.E))
    for q in range(m.n_sec):
        assert np.allclose(imp.energies(q), m.E[q], atol=1e-12 * scale, rtol=0)
    assert np.array_equal(s, m.s)
    assert imp.is_complex == m.is_complex


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_blocks_basis_invariants_match_oracle(name, host_models, models):
    """Tr(F^H D' F D) with D = diag(e^{-x (E - E_min)}) is invariant under any
    unitary change of eigenbasis inside degenerate levels."""
    imp = host_models(name)
    m = models(name)
    x = 0.37
    for (alpha, q), Fo in m.F.items():
        Fl = imp.block(alpha, q)
        qp = m.s[alpha, q]
        D = np.exp(-x * (m.E[q] - m.E[q][0]))
        Dp = np.exp(-x * (m.E[qp] - m.E[qp][0]))
        a = np.trace(Fo.conj().T @ (Dp[:, None] * Fo) * D[None, :])
        b = np.trace(Fl.conj().T @ (Dp[:, None] * Fl) * D[None, :])
        assert abs(a - b) <= 1e-11 * max(1.0, abs(a))
        sv = np.linalg.svd(Fl, compute_uv=False)
        assert np.all((np.abs(sv - 1) < 1e-12) | (sv < 1e-12))


class _LibModel:
    """The library's host model in the attribute layout the oracle's trace
    routine reads (test glue only)."""

    def __init__(self, imp, beta):
        dims, N, Emin, s = imp.sectors()
        self.n_sec = imp.n_sec
        self.dims = [int(d) for d in dims]
        self.E = [imp.energies(q) for q in range(self.n_sec)]
        self.E_min = np.asarray([e[0] for e in self.E])
        self.E_gs = float(self.E_min.min())
        nf = imp.n_flav
        # Bulla operators 2 n_flav + f (when present) map sectors as c_f
        rows = [a if a < 2 * nf else 2 * (a - 2 * nf) for a in range(imp.n_alpha)]
        self.s = s.astype(np.int64)[rows]
        self.n_flav = nf
        self.is_complex = imp.is_complex
        self.beta = beta
        self.F = {(a, q): imp.block(a, q) for a in range(imp.n_alpha) for q in range(self.n_sec)
                  if self.s[a, q] >= 0}

    def opnorm(self, a, q):
        return float(np.linalg.norm(self.F[(a, q)], 2))


@pytest.mark.parametrize("name", ["hubbard2", "t2g"])
def test_library_blocks_reproduce_oracle_traces(name, host_models, models):
    """Full sector-string traces evaluated on the library's eigenbasis equal
    the oracle's on its own eigenbasis (checks relative block signs)."""
    imp = host_models(name)
    m = models(name)
    lm = _LibModel(imp, m.beta)
    b = w.batch_hubbard2() if name == "hubbard2" else w.batch_t2g(48)
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        r1 = OT.trace_chain(m, tau, ops)
        r2 = OT.trace_chain(lm, tau, ops)
        if r1["log_abs"] == -math.inf:
            assert r2["log_abs"] == -math.inf
            continue
        err = abs(complex(r2["phase"]) * math.exp(r2["log_abs"] - r1["log_abs"]) - complex(r1["phase"]))
        tol = 1e-12 * math.exp(r1["log_cond"] - r1["log_abs"]) + 50 * m.beta * 1e-15 * 10
        assert err <= tol, (c, err, tol)


def test_build_rejects_bad_parameters():
    p = w.model_t2g()
    p.n_orb = 0
    with pytest.raises(ctq.CtqError):
        ctq.build_impurity(p, device=-1)
    p = w.model_t2g()
    p.soc_xi = 0.3  # SOC needs a Slater shell
    with pytest.raises(ctq.CtqError):
        ctq.build_impurity(p, device=-1)


def test_load_impurity_roundtrip(models):
    m = models("hubbard2")
    imp = ctq.load_impurity(m.n_flav, m.dims, m.N, m.E, m.s, m.F, mu=m.mu, device=-1)
    dims, N, Emin, s = imp.sectors()
    assert list(dims) == m.dims and np.array_equal(s, m.s)
    for (a, q), F in m.F.items():
        assert np.array_equal(imp.block(a, q), F)


# ---------------------------------------------------------------- Bulla operators

def small_complex_model():
    cf = w.crystal_field_complex(4, 0.3, 17)
    return w.ModelParams("k2c", n_orb=2, l=0, interaction="kanamori", U=3.0, J=0.6, beta=4.0, mu=1.1,
                         n0=2, cf=cf, sector_mode="n")


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_bulla_blocks_on_the_oracle_eigenbasis(name, models):
    """ctq_add_bulla_operators on the oracle's eigenbasis and one-body matrix
    against the oracle's Bulla blocks (formed from the interaction terms in
    the occupation basis): element by element."""
    import parity
    m = models(name)
    mb = OI.with_bulla(m)
    imp = parity.load_oracle_model(ctq, m, device=-1)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    nf = m.n_flav
    assert imp.n_alpha == 3 * nf
    n = 0
    for f in range(nf):
        for q in range(m.n_sec):
            code = OI.bulla_code(nf, f)
            if mb.s[code, q] < 0:
                with pytest.raises(ctq.CtqError):
                    imp.block(code, q)
                continue
            ref = mb.F[(code, q)]
            got = imp.block(code, q)
            assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (f, q)
            n += 1
    assert n > 0


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "complex"])
def test_library_bulla_traces_match_oracle(name, models):
    """Library-built impurity (its own eigenbasis and one-body matrix t - mu):
    traces with one annihilator replaced by its Bulla operator, evaluated by
    the oracle's trace routine on the library's blocks, equal the oracle's
    (basis-invariant)."""
    m = atom.Model(small_complex_model()) if name == "complex" else models(name)
    imp = ctq.build_impurity(m.params, device=-1)
    imp.add_bulla_operators()
    lm = _LibModel(imp, m.beta)
    mb = OI.with_bulla(m)
    rng = np.random.default_rng(12)
    b = w.random_batch(rng, m.n_flav, m.beta, 12, 2, 8)
    n_cmp = 0
    for c in range(b.n_chains):
        tau, ops = b.chain(c)
        base = OT.trace_chain(mb, tau, ops)
        for pos in OI.annihilators(mb, ops)[:3]:
            seq = OI.bulla_sequence(mb, ops, pos)
            r1 = OT.trace_chain(mb, tau, seq)
            r2 = OT.trace_chain(lm, tau, seq)
            if r1["log_abs"] == -math.inf:
                # exactly zero in the oracle's eigenbasis (a hidden symmetry):
                # rounding noise only on the library's
                assert r2["log_abs"] == -math.inf or r2["log_abs"] < base["log_cond"] - 20
                continue
            err = abs(complex(r2["phase"]) * math.exp(r2["log_abs"] - r1["log_abs"]) - complex(r1["phase"]))
            tol = 1e-11 * math.exp(r1["log_cond"] - r1["log_abs"]) + 1e-12
            assert err <= tol, (c, pos, err, tol)
            n_cmp += 1
    assert n_cmp >= 10


def test_bulla_argument_errors(models):
    import parity
    m = models("hubbard2")
    imp = parity.load_oracle_model(ctq, m, device=-1)
    with pytest.raises(ctq.CtqError):  # a loaded impurity has no one-body matrix of its own
        imp.add_bulla_operators()
    h = atom.one_body_matrix(m.params, m.mu)
    imp.add_bulla_operators(h)
    with pytest.raises(ctq.CtqError):  # once per impurity
        imp.add_bulla_operators(h)
    with pytest.raises(ctq.CtqError):  # complex one-body term on a real impurity
        imp2 = parity.load_oracle_model(ctq, m, device=-1)
        imp2.add_bulla_operators(h + 0.1j * np.eye(m.n_flav))

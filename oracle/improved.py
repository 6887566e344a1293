"""Oracle, part 4: the static part of the improved estimator for the
self-energy (TEST INFRASTRUCTURE ONLY; see oracle/__init__).

Definition followed (Sec. 2.4, improved estimators; Eq.
PImprovedEstimatorStatic): for a configuration C and its s-th annihilator
c_{i'_s}(tau'_s),

    h^st_s = w^U_s(C) / w_loc(C),

where w^U_s is the local weight with that annihilator replaced by the Bulla
operator [c_{i'_s}, U] at the same time, and U is the interaction part of
H_loc (the two-body terms of Eq. ImpurityHamiltonian; the one-body part
t - mu is not in U).

Written out plainly: in each sector q, [c_f, U] is the matrix
C_f(q) U(q) - U(q') C_f(q) in the occupation basis, with C_f the signed
partial permutation of c_f (Jordan-Wigner signs) and U(q) the interaction
terms alone restricted to the sector; U conserves every sector label, so the
commutator maps q to the same q' = s_{c_f}(q) as c_f.  In the eigenbasis
its block is V_{q'}^H [C_f U - U C_f] V_q.  These blocks are added to the
oracle model under the operator codes 2 n_f + f, and w^U_s is then the
ordinary sector-string trace of oracle.trace with the s-th annihilator's
code replaced.  The time-ordering sign of C is unchanged by the replacement
and cancels in the ratio.
"""
from __future__ import annotations

import copy
import math

import numpy as np

from . import atom
from . import trace as T


def bulla_code(n_flav: int, f: int) -> int:
    """Operator code of B_f = [c_f, U]: 2 n_f + f (after the 2 n_f codes
    2 f + dag of the creation and annihilation operators)."""
    return 2 * n_flav + f


def with_bulla(model):
    """A shallow copy of an oracle model whose operator table also holds
    B_f = [c_f, U] for every flavour f (codes 2 n_f + f)."""
    p = model.params
    inter = atom.interaction_terms(p)
    nf, ns = model.n_flav, model.n_sec
    m = copy.copy(model)
    m.s = np.full((3 * nf, ns), -1, dtype=np.int64)
    m.s[: 2 * nf] = model.s
    m.F = dict(model.F)
    U = [atom.sector_hamiltonian(st, inter) for st in model.states]
    for f in range(nf):
        for q in range(ns):
            got = model.occupation_op(2 * f, q)
            if got is None:
                continue
            qp, C = got
            B = C @ U[q] - U[qp] @ C
            Bq = model.V[qp].conj().T @ (B @ model.V[q])
            if not model.is_complex:
                if np.abs(Bq.imag).max(initial=0.0) > 0.0:
                    raise RuntimeError("complex Bulla block in a real model")
                Bq = Bq.real
            m.s[bulla_code(nf, f), q] = qp
            m.F[(bulla_code(nf, f), q)] = Bq
    m.has_bulla = True
    return m


def annihilators(model, ops):
    """Positions s of the annihilation operators (codes 2 f) in a sequence."""
    return [i for i, a in enumerate(ops) if int(a) < 2 * model.n_flav and int(a) % 2 == 0]


def bulla_sequence(model, ops, pos: int):
    """The sequence with the annihilator at position pos replaced by its
    Bulla operator."""
    out = np.array(ops, dtype=np.int64).copy()
    a = int(out[pos])
    if a >= 2 * model.n_flav or a % 2:
        raise ValueError("not an annihilation operator")
    out[pos] = bulla_code(model.n_flav, a // 2)
    return out


def static_ratios(model_b, tau, ops, beta: float | None = None):
    """h^st_s for every annihilator of one configuration: a list of
    (position, complex ratio); the ratio is NaN when w_loc(C) = 0.
    model_b comes from with_bulla."""
    r = T.trace_chain(model_b, tau, ops, beta=beta)
    out = []
    for pos in annihilators(model_b, ops):
        ru = T.trace_chain(model_b, tau, bulla_sequence(model_b, ops, pos), beta=beta)
        if r["log_abs"] == -math.inf:
            out.append((pos, complex(math.nan, math.nan)))
        elif ru["log_abs"] == -math.inf:
            out.append((pos, 0j))
        else:
            out.append((pos, complex(ru["phase"]) / complex(r["phase"]) * math.exp(ru["log_abs"] - r["log_abs"])))
    return out

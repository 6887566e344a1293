"""Helpers shared by the GPU parity tests (comparison rules and glue between
the oracle and the library binding).  Test infrastructure only."""
from __future__ import annotations

import math

import numpy as np

from oracle import trace as OT

# FP64 parity bar: relative error of w (|w_gpu - w_ref| / |w_ref|).
FP64_REL = 1e-12
# Chains whose per-q0 terms cancel (sum |w_q0| > CANCEL * |w|) are compared
# against sum |w_q0| instead of |w|.
CANCEL = 10.0


def oracle_chain_results(model, batch, chains):
    return {int(c): OT.trace_chain(model, *batch.chain(int(c)), beta=batch.beta) for c in chains}


def log_sum_abs_q0(r) -> float:
    logs = [v[0] for v in r["per_q0"].values() if v[0] != -math.inf]
    if not logs:
        return -math.inf
    m = max(logs)
    return m + math.log(sum(math.exp(x - m) for x in logs))


def chain_error(log_abs, phase, ref):
    """(error, scale_kind): error of the GPU value relative to |w_ref| (or to
    sum |w_q0| when the q0 terms cancel)."""
    if ref["log_abs"] == -math.inf:
        return (0.0 if log_abs == -math.inf else math.inf), "zero"
    if not np.isfinite(log_abs):
        return math.inf, "missing"
    la_ref = ref["log_abs"]
    denom = la_ref
    kind = "abs"
    lsum = log_sum_abs_q0(ref)
    if lsum - la_ref > math.log(CANCEL):
        denom = lsum
        kind = "sum_q0"
    g = complex(phase[0], phase[1]) * math.exp(log_abs - denom)
    o = complex(ref["phase"]) * math.exp(la_ref - denom)
    return abs(g - o), kind


def model_opnorms(m):
    return {k: m.opnorm(*k) for k in m.F}


def load_oracle_model(ctq, m, device=0, with_norms=True):
    """The oracle's eigenbasis handed to the library (ctq_load_impurity), so
    the GPU arithmetic is compared on identical blocks and energies."""
    return ctq.load_impurity(m.n_flav, m.dims, m.N, m.E, m.s, m.F, mu=m.mu,
                             opnorm=model_opnorms(m) if with_norms else None, device=device)

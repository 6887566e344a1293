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
# Multiple of the oracle's own association-order spread allowed on the GPU.
NOISE_FACTOR = 8.0


def oracle_chain_results(model, batch, chains, noise=True):
    """Oracle trace per chain; with noise=True each result also carries
    'noise': the relative spread between multiplying the strings right-to-left
    and left-to-right (the chain's own float64 rounding spread)."""
    out = {}
    for c in chains:
        tau, ops = batch.chain(int(c))
        r = OT.trace_chain(model, tau, ops, beta=batch.beta)
        if noise:
            l = OT.trace_chain_left(model, tau, ops, beta=batch.beta)
            r["noise"] = rel_spread(l, r)
        out[int(c)] = r
    return out


def rel_spread(a, ref) -> float:
    if ref["log_abs"] == -math.inf:
        return 0.0 if a["log_abs"] == -math.inf else math.inf
    if a["log_abs"] == -math.inf:
        return 1.0
    return abs(complex(a["phase"]) * math.exp(a["log_abs"] - ref["log_abs"]) - complex(ref["phase"]))


def fp64_tolerance(ref) -> float:
    """Parity bar for one chain in FP64 mode: 1e-12, or 8x the chain's own
    float64 rounding spread when cancellation inside the trace makes that
    larger (the spread is measured, not assumed)."""
    return max(FP64_REL, NOISE_FACTOR * ref.get("noise", 0.0))


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

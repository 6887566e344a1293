"""Helpers shared by the GPU parity tests (comparison rules and glue between
the oracle and the library binding).  Test infrastructure only."""
from __future__ import annotations

import json
import math
import os

import numpy as np

from oracle import trace as OT

# FP64 parity bar: relative error of w (|w_gpu - w_ref| / |w_ref|).
FP64_REL = 1e-12
# Chains whose per-q0 terms cancel (sum |w_q0| > CANCEL * |w|) are compared
# against sum |w_q0| instead of |w|.
CANCEL = 10.0
# Multiple of the oracle's own association-order spread allowed on the GPU.
NOISE_FACTOR = 8.0
# No chain's FP64 bar exceeds this, whatever its measured spread.
FP64_CAP = 1e-10
# A chain is ill-conditioned when the oracle's own float64 spread exceeds
# the FP64 bar itself: only then is its bar widened.
WIDEN_AT = FP64_REL
# A mixed-precision chain is held to its stated bar, or, when its measured
# condition number kappa = spread / 2^-53 (the chain's float64 perturbation
# spread in units of float64's unit roundoff) times the precision's
# effective unit exceeds the stated bar, to unit x kappa (the first-order
# error of that precision on that chain).  A chain with unit x kappa above 1
# (and above the stated bar) has no significant digit in the precision: it
# gets no bar, is listed, and at most UNRESOLVED_FRAC of a test's chains
# (at least UNRESOLVED_MIN) may be so.
UNRESOLVED_FRAC = 0.01
UNRESOLVED_MIN = 3
U64 = 2.0 ** -53
# Effective unit roundoff of one block product per precision code (ctq.TF32 = 1,
# BF16X3 = 2, TF32X3 = 3, F32X2 = 4): TF32 operands keep 11 bits; bf16 hi / lo
# about 16; the three-term TF32 split keeps 22 but its FP32 accumulation over
# ~100 terms loses about 3 more (fitted on the d shell's chains); two-float
# about 45.
UNIT = {1: 2.0 ** -11, 2: 2.0 ** -16, 3: 2.0 ** -19, 4: 2.0 ** -45}
# At most this fraction of a test's chains (and at least three chains) may
# be held to a widened bar; every widened chain is printed.  (The d shell at
# beta = 40 has 4.9 % of its 1024 chains above the FP64 bar in float64
# spread; hubbard2 and t2g have none.)
WIDEN_FRAC = 0.10
WIDEN_MIN = 3
# The result is carried as log|w| in float64, which resolves relative changes
# of w only down to the spacing of log|w| (4.5e-13 at |log w| ~ 3600, the d
# shell at beta = 40): the library's and the oracle's final roundings of
# log|w| each contribute up to half a spacing, and the relative parts they
# add to the large -beta E_gs (up to |log w| ~ 900, accumulated over ~100
# operators with a few roundings each at that magnitude) about as much
# again.  Every FP64-class bar adds LOG_ULPS spacings of the oracle's log|w|.
LOG_ULPS = 4.0


def log_carrier(ref) -> float:
    """LOG_ULPS spacings of float64 at the oracle's |log w| (0 for w = 0)."""
    la = ref["log_abs"]
    return LOG_ULPS * float(np.spacing(abs(la))) if np.isfinite(la) else 0.0


class Bars:
    """Per-chain parity bars of one test, with a record of every chain whose
    bar was widened beyond the base bar because the oracle's own float64
    rounding spread (the two association orders of the product) is larger.

    fp64(c, ref):     base x scale, or, when spread > WIDEN_AT,
                      max(base, min(FP64_CAP, 8 x spread)) x scale;
                      plus log_carrier(ref)
    mixed(c, ref, b, unit, err):
                      max(b, unit x spread / 2^-53), or no bar (inf) when
                      that estimate exceeds max(1, b) (an unresolved chain); a chain
                      counts as widened only if its error needed it (err > b;
                      every chain above b when err is not given)
    check():          prints the widened and unresolved chains and asserts
                      that there are at most max(WIDEN_MIN, WIDEN_FRAC x
                      chains seen) widened and max(UNRESOLVED_MIN,
                      UNRESOLVED_FRAC x chains seen) unresolved ones."""

    def __init__(self, label: str, max_frac: float = WIDEN_FRAC):
        self.label = label
        self.max_frac = max_frac
        self.n = 0
        self.widened = []
        self.unresolved = []

    def fp64(self, c, ref, base: float = FP64_REL, scale: float = 1.0, err=None) -> float:
        self.n += 1
        noise = ref.get("noise", 0.0)
        bar = max(base, min(FP64_CAP, NOISE_FACTOR * noise)) if noise > WIDEN_AT else base
        if bar > base:
            self.widened.append((int(c), noise, bar * scale))
        return bar * scale + log_carrier(ref)

    def mixed(self, c, ref, stated: float, unit: float, err=None) -> float:
        self.n += 1
        noise = ref.get("noise", 0.0)
        est = unit * (noise / U64)
        if est > max(1.0, stated):
            self.unresolved.append((int(c), noise, err))
            return math.inf
        bar = max(stated, est)
        if bar > stated and (err is None or err > stated):
            self.widened.append((int(c), noise, bar))
        return bar

    def check(self):
        allowed = max(WIDEN_MIN, int(self.max_frac * self.n))
        for c, noise, bar in self.widened:
            print(f"{self.label}: chain {c} bar widened to {bar:.2e} (float64 spread {noise:.2e})")
        print(f"{self.label}: {len(self.widened)} of {self.n} chains on a widened bar (allowed {allowed})")
        assert len(self.widened) <= allowed, (self.label, self.widened)
        n_unres = max(UNRESOLVED_MIN, int(UNRESOLVED_FRAC * self.n))
        for c, noise, err in self.unresolved:
            print(f"{self.label}: chain {c} not resolved in this precision (float64 spread {noise:.2e}, "
                  f"error {err})")
        assert len(self.unresolved) <= n_unres, (self.label, self.unresolved)


_PERTURBED = {}


def perturbed_model(model, seed: int = 20100848):
    """A copy of an oracle model whose every block entry is multiplied by
    (1 + r 2^-52), r = +-1 seeded: the blocks as another float64 eigensolver
    could have rounded them.  Evaluating a chain on it measures the chain's
    sensitivity to the float64 rounding of its inputs (the perturbation is
    of the inputs only; the oracle's arithmetic is unchanged)."""
    key = id(model)
    if key not in _PERTURBED:
        import copy
        rng = np.random.default_rng(seed)
        m = copy.copy(model)
        m.F = {k: v * (1.0 + rng.choice([-1.0, 1.0], size=v.shape) * 2.0 ** -52) for k, v in model.F.items()}
        _PERTURBED[key] = (model, m)  # keep the original alive so that its id stays unique
    return _PERTURBED[key][1]


def oracle_chain_results(model, batch, chains, noise=True):
    """Oracle trace per chain; with noise=True each result also carries
    'noise': the largest relative spread between the right-to-left product
    and (a) the left-to-right product, (b) the product split in the middle,
    (c) the right-to-left product on blocks perturbed by one unit in the
    last place (perturbed_model): the chain's own float64 rounding spread,
    measured three ways so that one accidental agreement does not hide it."""
    out = {}
    for c in chains:
        tau, ops = batch.chain(int(c))
        r = OT.trace_chain(model, tau, ops, beta=batch.beta)
        if noise:
            l = OT.trace_chain_left(model, tau, ops, beta=batch.beta)
            sp = OT.trace_chain_split(model, tau, ops, beta=batch.beta)
            pt = OT.trace_chain(perturbed_model(model), tau, ops, beta=batch.beta)
            r["noise"] = max(rel_spread(l, r), rel_spread(sp, r), rel_spread(pt, r))
        out[int(c)] = r
    return out


def rel_spread(a, ref) -> float:
    """Relative difference of two oracle evaluations of one chain, taken on
    log|w| + beta E_gs (log_rel) so that it resolves differences below the
    float64 spacing of log|w| itself."""
    if ref["log_abs"] == -math.inf:
        return 0.0 if a["log_abs"] == -math.inf else math.inf
    if a["log_abs"] == -math.inf:
        return 1.0
    return abs(complex(a["phase"]) * math.exp(a["log_rel"] - ref["log_rel"]) - complex(ref["phase"]))


def fp64_tolerance(ref) -> float:
    """Parity bar for one chain in FP64 mode: 1e-12, or 8x the chain's own
    float64 rounding spread when that spread exceeds WIDEN_AT (the spread is
    measured, not assumed), never above FP64_CAP; plus log_carrier(ref).
    Tests that widen bars this way count the widened chains with Bars."""
    noise = ref.get("noise", 0.0)
    bar = max(FP64_REL, min(FP64_CAP, NOISE_FACTOR * noise)) if noise > WIDEN_AT else FP64_REL
    return bar + log_carrier(ref)


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


GOLD_D5 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "d5_oracle.json")


def gold_d5():
    """Stored oracle results of the first chains of the d-shell batch
    (tests/golden/make_d5_oracle.py), in the form chain_error reads."""
    with open(GOLD_D5) as f:
        g = json.load(f)
    refs = {}
    for e in g["chains"]:
        refs[e["chain"]] = {"log_abs": e["log_abs"], "phase": complex(*e["phase"]), "noise": e["noise"],
                            "n_ops": e["n_ops"],
                            "per_q0": {int(q): (v[0], complex(v[1], v[2])) for q, v in e["per_q0"].items()}}
    return g["n_chains"], refs

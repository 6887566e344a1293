"""Partition-space CT-HYB sampling around the batched local trace.

Many independent Markov chains sample the hybridisation expansion of an
impurity coupled to a fermionic bath (Sec. 2.2).  A configuration C holds,
per flavour f, the times of its creation operators tau_r and annihilation
operators tau'_s; its weight is the product of the local weight (Eq.
pweight1, evaluated on the GPU by ctq_eval_traces) and the hybridisation
determinant (Eq. pweight2),

    w(C) = Tr[T e^{-beta H_loc} prod_r c_f(tau'_r) c^+_f(tau_r)]
           x prod_f det M_f,     (M_f)_{rs} = Delta_f(tau_r - tau'_s),

for a diagonal hybridisation function Delta_f(tau) = sum_l V_l^2 g_l(tau),
g_l(tau) = -e^{-eps_l tau} / (1 + e^{-beta eps_l}) on (0, beta),
antiperiodic (the transform of Eq. hybridization for bath levels eps_l).
The operators inside the trace are written pair by pair, r = 0, 1, ... in
the labels of M's rows and columns; time ordering them gives the sign of
the permutation, and the library returns the trace of the time-ordered
product.

Moves (App. B, Pauli-aware pair insertion and removal): a flavour is drawn,
then insertion or removal with probability 1/2 each.
  insertion: with N operators of flavour f already present, one of them is
    picked (probability 1/N) and two times are drawn uniformly between it
    and the next operator of the flavour on the circle of length beta (an
    interval of length L; density 2/L^2 for the ordered pair); their types
    follow the picked operator's (after a c^+ the flavour is occupied, so
    the earlier new operator is a c).  With N = 0 the creator and the
    annihilator times are drawn uniformly on [0, beta) (density 1/beta^2).
  removal: one of the N' operators of flavour f is picked (1/N') and
    removed with the next operator of the flavour; for N' = 2 both picks
    give the same empty configuration (probability 1).
The proposal ratio of each move is the reverse move's probability over the
forward one's, so detailed balance holds for these draws (the paper's
configuration weights belong to its own way of drawing the times).

Decision (Eqs. MHratio and decide): the random number r is drawn first and
folded into a threshold on the local weight,
    T = log r + log|w_loc(C_old)| - log|proposal ratio x det ratio|,
and the move is accepted iff log|w_loc(C_new)| >= T; ctq_eval_traces
receives T with lazy evaluation on, so that the GPU stops a proposal as soon
as its trace bound falls below T (early reject) and evaluates only the
proposals that may be accepted.

Determinants: M_f^{-1} is kept per chain and flavour and updated in
O(k^2) per move (the bordered-matrix inverse for an insertion, the
Schur-complement formula for a removal).

Estimators: the mean expansion order, the sign, the Green function of Eq.
PGreenEstimator in imaginary time (binned; (M^{-1})_{sr} at the time
difference tau'_s - tau_r, antiperiodic), and, through
ctq_eval_density_matrices, the reduced density matrix (Eq.
ImpurityDensityMatrix) and from it the sector occupations.

Host logic only: numpy on the CPU; every local trace and density matrix is
evaluated by the library's kernels.
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np

from . import ctq


def hybridisation(eps, V, beta: float, tau: np.ndarray) -> np.ndarray:
    """Delta(tau) on (-beta, beta): sum_l V_l^2 g_l(tau), g_l(tau) =
    -e^{-eps_l tau} / (1 + e^{-beta eps_l}) for tau in (0, beta) and
    g_l(tau) = -g_l(tau + beta) for tau in (-beta, 0)."""
    tau = np.asarray(tau, dtype=np.float64)
    neg = tau < 0.0
    t = np.where(neg, tau + beta, tau)
    out = np.zeros_like(t)
    for e, v in zip(eps, V):
        if e >= 0.0:
            out -= v * v * np.exp(-e * t) / (1.0 + math.exp(-beta * e))
        else:
            out -= v * v * np.exp(e * (beta - t)) / (1.0 + math.exp(beta * e))
    return np.where(neg, -out, out)


def perm_parity(times_written: np.ndarray) -> int:
    """+1 / -1: parity of the permutation that orders operators written left
    to right with these times into T_tau order (latest time leftmost)."""
    t = np.asarray(times_written)
    n = len(t)
    if n < 2:
        return 1
    inv = int(np.sum(np.triu(t[:, None] < t[None, :], 1)))  # pairs i < j with t_i < t_j
    return -1 if inv % 2 else 1


class _Chain:
    """One Markov chain: per flavour the creation times (row labels of M),
    the annihilation times (column labels), M^{-1} and the sign of det M;
    the local weight as log|w_loc| and its phase."""

    def __init__(self, n_flav: int):
        self.cre: List[np.ndarray] = [np.zeros(0) for _ in range(n_flav)]
        self.ann: List[np.ndarray] = [np.zeros(0) for _ in range(n_flav)]
        self.minv: List[np.ndarray] = [np.zeros((0, 0)) for _ in range(n_flav)]
        self.det_sign = [1.0] * n_flav
        self.perm_sign = 1  # parity of time ordering the pairs as written
        self.log_wloc = 0.0
        self.phase_loc = 1.0 + 0j

    def order(self) -> int:
        return int(sum(len(c) for c in self.cre))

    def sequence(self):
        """(times ascending, operator codes) of the configuration, and the
        parity of time ordering the pairs as written."""
        times, codes = [], []
        for f in range(len(self.cre)):
            for r in range(len(self.cre[f])):
                times += [self.ann[f][r], self.cre[f][r]]  # c_f(tau'_r) c^+_f(tau_r), left to right
                codes += [2 * f, 2 * f + 1]
        times = np.asarray(times, dtype=np.float64)
        codes = np.asarray(codes, dtype=np.int32)
        sgn = perm_parity(times)
        o = np.argsort(times, kind="stable")
        return times[o], codes[o], sgn


class PartitionSampler:
    """Batched partition-space CT-HYB: n_chains independent chains, one
    proposal per chain and step, every proposal's local trace in one
    ctq_eval_traces call (lazy thresholds)."""

    def __init__(self, imp, eps, V, beta: float, n_chains: int, seed: int = 0,
                 max_ops: int = 256, precision: int = ctq.FP64, lazy: bool = True, segment: int = 8,
                 n_bins: int = 50, device="cuda"):
        """imp: a ctq.Impurity (its n_flav flavours each hybridise with the
        bath levels eps [n_b] through V [n_b]); max_ops bounds 2k."""
        try:
            import torch
        except ImportError:  # only the host logic is used (tests that replace _evaluate)
            torch = None
        self.imp = imp
        self.nf = imp.n_flav
        self.eps = np.asarray(eps, dtype=np.float64)
        self.V = np.asarray(V, dtype=np.float64)
        self.beta = float(beta)
        self.n_chains = n_chains
        self.rng = np.random.default_rng(seed)
        self.max_ops = max_ops
        self.sectors = imp.sectors()
        self.precision = precision
        self.lazy = lazy
        self.device = device
        self.segment = segment
        self.chains = [_Chain(self.nf) for _ in range(n_chains)]
        self.n_bins = n_bins
        self._torch = torch
        self.ev = self._make_evaluator()
        self.reset_stats()
        # initial local weights: the empty configuration (w_loc = Z_loc)
        st, la, ph = self._evaluate([(np.zeros(0), np.zeros(0, np.int32))] * n_chains, None)
        for c, ch in enumerate(self.chains):
            if st[c] != ctq.CHAIN_OK:
                raise RuntimeError(f"empty configuration not evaluated (status {st[c]})")
            ch.log_wloc, ch.phase_loc = float(la[c]), complex(ph[c][0], ph[c][1])

    # ------------------------------------------------------------------ GPU
    def _make_evaluator(self):
        return ctq.TraceEvaluator(self.imp, self.n_chains, self.max_ops, precision=self.precision,
                                  segment=self.segment, with_bounds=False, device=self.device)

    def _evaluate(self, seqs, thresholds: Optional[np.ndarray]):
        """Local traces of the sequences [(times, codes)] on the GPU, with
        lazy thresholds when given; returns (status, log|w|, phase)."""
        from . import workloads as w
        n = len(seqs)
        offs = np.zeros(n + 1, np.int32)
        offs[1:] = np.cumsum([len(t) for t, _ in seqs])
        if offs[-1] and int(np.max(np.diff(offs))) > self.max_ops:
            raise ValueError("configuration longer than max_ops")
        tau = np.concatenate([t for t, _ in seqs]) if offs[-1] else np.zeros(0)
        op = np.concatenate([o for _, o in seqs]).astype(np.int32) if offs[-1] else np.zeros(0, np.int32)
        batch = w.Batch(beta=self.beta, offsets=offs, tau=tau, op=op)
        db = ctq.DeviceBatch(batch, device=self.device, log_threshold=thresholds)
        self.ev(db, lazy=thresholds is not None and self.lazy)
        self._torch.cuda.synchronize()
        r = self.ev.results(n)
        return r["status"], r["log_abs"], r["phase"]

    # ------------------------------------------------------------- moves
    def _flavour_ops(self, ch: _Chain, f: int):
        """Times and types (1 = creator) of flavour f, sorted by time."""
        t = np.concatenate([ch.cre[f], ch.ann[f]])
        ty = np.concatenate([np.ones(len(ch.cre[f]), np.int8), np.zeros(len(ch.ann[f]), np.int8)])
        o = np.argsort(t)
        return t[o], ty[o]

    def _delta(self, x):
        return hybridisation(self.eps, self.V, self.beta, x)

    def _propose(self, ch: _Chain):
        """A proposal for one chain: dict(kind, f, ...) with the proposal
        ratio and the determinant ratio, or None (nothing to remove)."""
        f = int(self.rng.integers(0, self.nf))
        t_f, ty_f = self._flavour_ops(ch, f)
        N = len(t_f)
        beta = self.beta
        if self.rng.random() < 0.5:  # insertion
            if N == 0:
                tc, ta = self.rng.uniform(0.0, beta, size=2)
                prop = beta * beta
            else:
                i = int(self.rng.integers(0, N))
                j = (i + 1) % N
                L = (t_f[j] - t_f[i]) % beta if N > 1 else beta
                if L <= 0.0:
                    L = beta
                s1, s2 = np.sort(self.rng.uniform(0.0, L, size=2))
                t1, t2 = (t_f[i] + s1) % beta, (t_f[i] + s2) % beta
                if ty_f[i] == 1:  # occupied after a creator: annihilate first
                    ta, tc = t1, t2
                else:
                    tc, ta = t1, t2
                prop = (1.0 / (N + 2)) / ((1.0 / N) * 2.0 / (L * L))
            if tc == ta or np.any(t_f == tc) or np.any(t_f == ta):
                return None
            # bordered determinant: new row (creator tc), new column (annihilator ta)
            cre, ann, mi = ch.cre[f], ch.ann[f], ch.minv[f]
            row = self._delta(tc - ann)  # M[new, s] = Delta(tc - tau'_s)
            col = self._delta(cre - ta)  # M[r, new] = Delta(tau_r - ta)
            d = float(self._delta(np.array([tc - ta]))[0])
            mu = mi @ col
            rho = d - float(row @ mu)
            return {"kind": "ins", "f": f, "tc": tc, "ta": ta, "prop": prop, "det": rho, "row": row, "mu": mu}
        # removal
        if N == 0:
            return None
        i = int(self.rng.integers(0, N))
        j = (i + 1) % N
        if N == 2:
            prop = (1.0 / (beta * beta)) / 1.0
        else:
            a = (i - 1) % N
            b = (j + 1) % N
            L = (t_f[b] - t_f[a]) % beta
            if L <= 0.0:
                L = beta
            prop = ((1.0 / (N - 2)) * 2.0 / (L * L)) / (1.0 / N)
        ti, tj = t_f[i], t_f[j]
        tc, ta = (ti, tj) if ty_f[i] == 1 else (tj, ti)
        r = int(np.nonzero(ch.cre[f] == tc)[0][0])
        s = int(np.nonzero(ch.ann[f] == ta)[0][0])
        rho = float(ch.minv[f][s, r]) * (-1.0 if (r + s) % 2 else 1.0)
        return {"kind": "rem", "f": f, "r": r, "s": s, "prop": prop, "det": rho}

    def _apply(self, ch: _Chain, pr):
        f = pr["f"]
        if pr["kind"] == "ins":
            mi, row, mu, rho = ch.minv[f], pr["row"], pr["mu"], pr["det"]
            k = mi.shape[0]
            nu = row @ mi  # (v M^-1)
            new = np.empty((k + 1, k + 1))
            new[:k, :k] = mi + np.outer(mu, nu) / rho
            new[:k, k] = -mu / rho
            new[k, :k] = -nu / rho
            new[k, k] = 1.0 / rho
            ch.minv[f] = new
            ch.cre[f] = np.append(ch.cre[f], pr["tc"])
            ch.ann[f] = np.append(ch.ann[f], pr["ta"])
        else:
            r, s = pr["r"], pr["s"]
            mi = ch.minv[f]
            keep_s = np.arange(mi.shape[0]) != s
            keep_r = np.arange(mi.shape[1]) != r
            ch.minv[f] = (mi[np.ix_(keep_s, keep_r)]
                          - np.outer(mi[keep_s, r], mi[s, keep_r]) / mi[s, r])
            ch.cre[f] = ch.cre[f][keep_r]
            ch.ann[f] = ch.ann[f][keep_s]
        ch.det_sign[f] *= 1.0 if pr["det"] > 0 else -1.0

    def _proposed_sequence(self, ch: _Chain, pr):
        """(times, codes, permutation parity) of the proposed configuration."""
        f = pr["f"]
        old = (ch.cre[f], ch.ann[f])
        if pr["kind"] == "ins":
            ch.cre[f] = np.append(old[0], pr["tc"])
            ch.ann[f] = np.append(old[1], pr["ta"])
        else:
            ch.cre[f] = np.delete(old[0], pr["r"])
            ch.ann[f] = np.delete(old[1], pr["s"])
        out = ch.sequence()
        ch.cre[f], ch.ann[f] = old
        return out

    # ------------------------------------------------------------------ run
    def step(self, measure: bool = True):
        """One proposal per chain, all local traces in one batched call."""
        props, seqs, thr, idx = [], [], [], []
        for c, ch in enumerate(self.chains):
            pr = self._propose(ch)
            self.n_prop += 1
            if pr is None or pr["det"] == 0.0:
                continue
            times, codes, sgn = self._proposed_sequence(ch, pr)
            if len(times) > self.max_ops:
                continue
            r = 1.0 - self.rng.random()  # in (0, 1]
            thr.append(math.log(r) + ch.log_wloc - math.log(abs(pr["prop"] * pr["det"])))
            props.append((pr, sgn))
            seqs.append((times, codes))
            idx.append(c)
        if idx:
            st, la, ph = self._evaluate(seqs, np.asarray(thr))
            for k, c in enumerate(idx):
                s = int(st[k])
                if s == ctq.CHAIN_REJECTED_EARLY:
                    self.n_early += 1
                elif s == ctq.CHAIN_ACCEPTED:
                    ch = self.chains[c]
                    self._apply(ch, props[k][0])
                    ch.log_wloc, ch.phase_loc = float(la[k]), complex(ph[k][0], ph[k][1])
                    ch.perm_sign = props[k][1]
                    self.n_acc += 1
                elif s < 0:
                    raise RuntimeError(f"trace evaluation failed (chain status {s})")
        if measure:
            self._measure()

    def weight_sign(self, ch: _Chain) -> float:
        """Sign of w(C) (real models): permutation parity x det signs x sign of
        the local trace."""
        return float(ch.perm_sign * np.prod(ch.det_sign) * np.sign(ch.phase_loc.real))

    def reset_stats(self):
        self.n_prop = self.n_acc = self.n_early = 0
        self.n_meas = 0
        self.sum_sign = np.zeros(self.n_chains)
        self.sum_k = np.zeros(self.n_chains)
        self.g_bins = np.zeros((self.n_chains, self.nf, self.n_bins))
        self.n_chain_meas = np.zeros(self.n_chains)

    def _measure(self):
        dt = self.beta / self.n_bins
        for c, ch in enumerate(self.chains):
            sg = self.weight_sign(ch)
            self.sum_sign[c] += sg
            self.sum_k[c] += sg * ch.order()
            for f in range(self.nf):
                mi = ch.minv[f]
                if mi.size == 0:
                    continue
                x = ch.ann[f][:, None] - ch.cre[f][None, :]  # tau'_s - tau_r, indexed [s, r]
                val = -mi / self.beta
                neg = x < 0
                x = np.where(neg, x + self.beta, x)
                val = np.where(neg, -val, val)
                b = np.minimum((x / dt).astype(np.int64), self.n_bins - 1)
                np.add.at(self.g_bins[c, f], b.ravel(), sg * val.ravel() / dt)
            self.n_chain_meas[c] += 1
        self.n_meas += 1

    def run(self, n_steps: int, n_burn: int = 0):
        for _ in range(n_burn):
            self.step(measure=False)
        self.reset_stats()
        for _ in range(n_steps):
            self.step(measure=True)

    def estimates(self):
        """Per-chain averages (sign-weighted) and their mean and standard
        error across chains: mean order, sign, and G_f(tau) per bin."""
        n = np.maximum(self.n_chain_meas, 1)
        sign = self.sum_sign / n
        k = self.sum_k / n / sign
        g = self.g_bins / n[:, None, None] / sign[:, None, None]

        def ms(a):
            return a.mean(axis=0), a.std(axis=0, ddof=1) / math.sqrt(a.shape[0])
        return {"order": ms(k), "sign": ms(sign), "green": ms(g),
                "acceptance": self.n_acc / max(self.n_prop, 1), "early_rejects": self.n_early / max(self.n_prop, 1)}

    def density_matrices(self):
        """The reduced density matrix estimator of every chain's current
        configuration (ctq_eval_density_matrices): list of {q: d_q x d_q}."""
        from . import workloads as w
        seqs = [ch.sequence()[:2] for ch in self.chains]
        offs = np.zeros(self.n_chains + 1, np.int32)
        offs[1:] = np.cumsum([len(t) for t, _ in seqs])
        tau = np.concatenate([t for t, _ in seqs]) if offs[-1] else np.zeros(0)
        op = np.concatenate([o for _, o in seqs]).astype(np.int32) if offs[-1] else np.zeros(0, np.int32)
        db = ctq.DeviceBatch(w.Batch(beta=self.beta, offsets=offs, tau=tau, op=op), device=self.device)
        if not hasattr(self, "_dens"):
            self._dens = ctq.DensityEvaluator(self.imp, self.n_chains, self.max_ops, device=self.device)
        self._dens(db)
        self._torch.cuda.synchronize()
        return [self._dens.blocks(c) for c in range(self.n_chains)]

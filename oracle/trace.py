"""Oracle, part 2: local traces, bounds and decisions (TEST INFRASTRUCTURE ONLY;
see oracle/__init__).

Definitions followed, all in float64:

* Sector-string trace (Sec. 3.3.1, the sum over initial sectors q0):
      w = sum_{q0} Tr P_{beta - tau_n}(q0) F_{alpha_n}(q_{n-1}) P_{tau_n - tau_{n-1}}(q_{n-1})
                 ... F_{alpha_1}(q0) P_{tau_1}(q0),
  with q_i = s_{alpha_i}(q_{i-1}); a string that reaches the zero sector, or
  does not return to q0, contributes nothing.  P_tau(q) = diag(e^{-tau E_q,j})
  in the eigenbasis (the time-evolution operator).  The operators are
  already time ordered (the caller owns the T_tau permutation sign).
  To keep e^{-tau E} representable, each propagator is applied as
  e^{-tau E_min(q)} * diag(e^{-tau (E_q,j - E_min(q))}) with the scalar factor
  kept as a float64 logarithm, and the running product is rescaled by an exact
  power of two after every factor (the logarithm absorbs it).  Because the
  propagation times sum to beta, the scalar factors are accumulated relative
  to the ground-state energy, sum dtau (E_min(q) - E_gs), with an exactly
  rounded sum, and -beta E_gs is added once at the end.  These steps are exact
  identities; nothing else is reordered.
* Full-space brute force (Eq. pweight1 with Sec. 3.3.1's naive form):
  Tr[e^{-(beta - tau_n) H} O_n ... O_1 e^{-tau_1 H}] over the whole Fock space,
  with scipy.linalg.expm.
* Lazy-trace bounds (Sec. 3.3.1, lazy-trace paragraph: submultiplicative norms,
  the spectral norm for the propagators).  Reading used here:
    level 0:  b(q0) = r * prod_i ||F_i||_2 * prod_segments e^{-dtau E_min(q)},
              r = min_i d_{q_i} (the rank of the product), and
              B = sum_{q0} b(q0);
    refined after j operators (product so far Y_j, including the propagator
    that follows operator j and, at the start, the wrap-around propagator of
    q0 for beta - tau_n + tau_1):
              ub(q0, j) = sqrt(r) * ||Y_j||_F * prod_{i > j} ||F_i||_2
                          * prod_{segments after j} e^{-dtau E_min(q)},
    using |Tr X| <= sqrt(rank X) ||X||_F and ||A B||_F <= ||A||_2 ||B||_F;
    ub(q0, n) = |w_q0| (exact).  Segment s covers operators up to s*S.
* Metropolis decision (Eqs. MHratio, decide): the random number is drawn
  first and folded into a log threshold T; accept iff log|w| >= T.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

LN2 = math.log(2.0)


def _rescale(M: np.ndarray):
    """Scale M by 2^-e with e = floor(log2 max|M|); return (M', e*ln2) or
    (None, 0) if M == 0."""
    s = float(np.max(np.abs(M))) if M.size else 0.0
    if s == 0.0:
        return None, 0.0
    e = math.floor(math.log2(s))
    return M * (2.0 ** -e), e * LN2


def walk(model, ops, q0: int):
    """The sector string q0 -> q1 -> ... ; None if it dies or does not close."""
    path = [q0]
    q = q0
    for a in ops:
        q = int(model.s[int(a), q])
        if q < 0:
            return None
        path.append(q)
    if q != q0:
        return None
    return path


def trace_q0(model, tau, ops, q0: int, beta: float):
    """One initial sector: returns (value, log_rel, log_abs_product) with
    w_q0 = value * e^{log_rel} * e^{-beta E_gs}.

    The scalar factors e^{-dtau E_min(q)} are written as
    e^{-dtau E_gs} e^{-dtau (E_min(q) - E_gs)}; the propagation times tile
    [0, beta) (they sum to beta), so the first factors multiply to
    e^{-beta E_gs} and only the second ones are accumulated, with math.fsum
    (exactly rounded).  log_abs_product is the same product taken with |F|
    entrywise (the scale of float rounding errors), in the same relative
    convention."""
    path = walk(model, ops, q0)
    if path is None:
        return None
    n = len(ops)
    E, Emin, Egs = model.E, model.E_min, model.E_gs

    def prop(q, dt):
        return np.exp(-dt * (E[q] - Emin[q])), -dt * (Emin[q] - Egs)

    p, l0 = prop(q0, tau[0] if n else beta)
    M = np.diag(p).astype(model_dtype(model))
    A = np.diag(p)
    logs = [l0]
    e_sum, ea_sum = 0, 0
    for i in range(n):
        qa, qb = path[i], path[i + 1]
        Fb = model.F[(int(ops[i]), qa)]
        M = Fb @ M
        A = np.abs(Fb) @ A
        dt = (tau[i + 1] - tau[i]) if i + 1 < n else (beta - tau[n - 1])
        p, l = prop(qb, dt)
        M = p[:, None] * M
        A = p[:, None] * A
        logs.append(l)
        M, e = _rescale_exp(M)
        A, ea = _rescale_exp(A)
        if M is None:
            return 0.0, -math.inf, _finish_abs(A, math.fsum(logs) + ea_sum * LN2)
        e_sum += e
        ea_sum += ea
    L = math.fsum(logs)
    val = np.trace(M)
    return val, L + e_sum * LN2, _finish_abs(A, L + ea_sum * LN2)


def _rescale_exp(M: np.ndarray):
    """Scale M by 2^-e with e = floor(log2 max|M|); return (M', e) or (None, 0)."""
    s = float(np.max(np.abs(M))) if M.size else 0.0
    if s == 0.0:
        return None, 0
    e = math.floor(math.log2(s))
    return M * (2.0 ** -e), e


def _finish_abs(A, LA):
    if A is None or LA == -math.inf:
        return -math.inf
    t = float(np.trace(A))
    return math.log(t) + LA if t > 0 else -math.inf


def model_dtype(model):
    return np.complex128 if model.is_complex else np.float64


def logsumexp_signed(terms):
    """Sum of values given as (value, logscale); returns (log|sum|, phase)."""
    terms = [(v, l) for v, l in terms if v != 0 and l != -math.inf]
    if not terms:
        return -math.inf, 0.0
    lmax = max(l + math.log(abs(v)) for v, l in terms)
    s = sum(v * math.exp(l - lmax) for v, l in terms)
    if s == 0:
        return -math.inf, 0.0
    return lmax + math.log(abs(s)), s / abs(s)


def trace_chain(model, tau, ops, beta: float | None = None):
    """w for one chain.  Returns dict(log_abs, phase, per_q0, log_cond, log_rel)
    where per_q0 = {q0: (log|w_q0|, phase_q0)} over surviving q0, log_cond is
    the log of sum_q0 of the |F|-product traces and log_rel is log|w| + beta
    E_gs (the same value before the large shift is added, so that two
    evaluations can be compared below the float64 resolution of log|w|).  The sum over q0 is taken in the
    E_gs-relative log convention of trace_q0; -beta E_gs is added last."""
    beta = model.beta if beta is None else beta
    tau = np.asarray(tau, dtype=np.float64)
    ops = np.asarray(ops, dtype=np.int64)
    shift = -beta * model.E_gs
    terms, per_q0, conds = [], {}, []
    for q0 in range(model.n_sec):
        r = trace_q0(model, tau, ops, q0, beta)
        if r is None:
            continue
        val, L, lc = r
        terms.append((val, L))
        per_q0[q0] = ((math.log(abs(val)) + L + shift) if val != 0 else -math.inf,
                      (val / abs(val)) if val != 0 else 0.0)
        conds.append(lc)
    la, ph = logsumexp_signed(terms)
    finite = [c for c in conds if c != -math.inf]
    if finite:
        m = max(finite)
        lcond = m + math.log(sum(math.exp(c - m) for c in finite)) + shift
    else:
        lcond = -math.inf
    return {"log_abs": la + shift, "phase": ph, "per_q0": per_q0, "log_cond": lcond, "log_rel": la}


def trace_q0_left(model, tau, ops, q0: int, beta: float):
    """The same trace as trace_q0 multiplied in the opposite association order:
    starting from the leftmost factor P_{beta - tau_n}(q0) and moving right.
    Returns (value, log_rel).  Comparing the two orders measures the float64
    rounding spread of a chain (used to set parity tolerances)."""
    path = walk(model, ops, q0)
    if path is None:
        return None
    n = len(ops)
    E, Emin, Egs = model.E, model.E_min, model.E_gs
    if n == 0:
        return trace_q0(model, tau, ops, q0, beta)[:2]

    def prop(q, dt):
        return np.exp(-dt * (E[q] - Emin[q])), -dt * (Emin[q] - Egs)

    p, l0 = prop(q0, beta - tau[n - 1])
    M = np.diag(p).astype(model_dtype(model))
    logs = [l0]
    e_sum = 0
    for i in range(n - 1, -1, -1):
        M = M @ model.F[(int(ops[i]), path[i])]
        dt = (tau[i] - tau[i - 1]) if i > 0 else tau[0]
        p, l = prop(path[i], dt)
        M = M * p[None, :]
        logs.append(l)
        M, e = _rescale_exp(M)
        if M is None:
            return 0.0, -math.inf
        e_sum += e
    return np.trace(M), math.fsum(logs) + e_sum * LN2


def trace_chain_left(model, tau, ops, beta: float | None = None):
    """trace_chain with every q0 product multiplied left to right (see
    trace_q0_left); returns dict(log_abs, phase, log_rel)."""
    beta = model.beta if beta is None else beta
    tau = np.asarray(tau, dtype=np.float64)
    ops = np.asarray(ops, dtype=np.int64)
    terms = []
    for q0 in range(model.n_sec):
        r = trace_q0_left(model, tau, ops, q0, beta)
        if r is not None:
            terms.append(r)
    la, ph = logsumexp_signed(terms)
    return {"log_abs": la - beta * model.E_gs, "phase": ph, "log_rel": la}


def trace_q0_split(model, tau, ops, q0: int, beta: float):
    """The same trace as trace_q0 in a third association order: the first
    half of the string multiplied right to left into A (the propagator
    after operator m included), the second half left to right into B
    (starting from the wrap-around propagator P_{beta - tau_n}), then
    Tr(B A).  Returns (value, log_rel).  With the left-to-right order it
    gives a second measure of the chain's float64 rounding spread."""
    path = walk(model, ops, q0)
    if path is None:
        return None
    n = len(ops)
    if n < 2:
        return trace_q0(model, tau, ops, q0, beta)[:2]
    E, Emin, Egs = model.E, model.E_min, model.E_gs
    m = n // 2

    def prop(q, dt):
        return np.exp(-dt * (E[q] - Emin[q])), -dt * (Emin[q] - Egs)

    # A = P_{tau_{m+1} - tau_m}(q_m) F_m ... F_1 P_{tau_1}(q0)   (operators 0 .. m-1)
    p, l0 = prop(q0, tau[0])
    A = np.diag(p).astype(model_dtype(model))
    logs = [l0]
    e_sum = 0
    for i in range(m):
        A = model.F[(int(ops[i]), path[i])] @ A
        p, l = prop(path[i + 1], tau[i + 1] - tau[i])
        A = p[:, None] * A
        logs.append(l)
        A, e = _rescale_exp(A)
        if A is None:
            return 0.0, -math.inf
        e_sum += e
    # B = P_{beta - tau_n}(q0) F_n P ... P F_{m+1}   (operators n-1 .. m)
    p, l = prop(q0, beta - tau[n - 1])
    Bm = np.diag(p).astype(model_dtype(model))
    logs.append(l)
    for i in range(n - 1, m - 1, -1):
        Bm = Bm @ model.F[(int(ops[i]), path[i])]
        if i > m:
            p, l = prop(path[i], tau[i] - tau[i - 1])
            Bm = Bm * p[None, :]
            logs.append(l)
        Bm, e = _rescale_exp(Bm)
        if Bm is None:
            return 0.0, -math.inf
        e_sum += e
    return np.trace(Bm @ A), math.fsum(logs) + e_sum * LN2


def trace_chain_split(model, tau, ops, beta: float | None = None):
    """trace_chain with every q0 product in the split association of
    trace_q0_split; returns dict(log_abs, phase, log_rel)."""
    beta = model.beta if beta is None else beta
    tau = np.asarray(tau, dtype=np.float64)
    ops = np.asarray(ops, dtype=np.int64)
    terms = []
    for q0 in range(model.n_sec):
        r = trace_q0_split(model, tau, ops, q0, beta)
        if r is not None:
            terms.append(r)
    la, ph = logsumexp_signed(terms)
    return {"log_abs": la - beta * model.E_gs, "phase": ph, "log_rel": la}


def trace_batch(model, batch, chains=None):
    """trace_chain over a workloads.Batch (optionally a subset of chain ids)."""
    idx = range(batch.n_chains) if chains is None else chains
    return [trace_chain(model, *batch.chain(int(c)), beta=batch.beta) for c in idx]


# ---------------------------------------------------------------------------
# brute force over the full Fock space (no sectors, no eigenbasis)
# ---------------------------------------------------------------------------


def trace_full_space(H: np.ndarray, op_mats, tau, ops, beta: float):
    """Tr[e^{-(beta-tau_n)H} O_n e^{-(tau_n - tau_{n-1})H} ... O_1 e^{-tau_1 H}]
    with dense matrices and scipy.linalg.expm; op_mats[alpha] is the full-space
    matrix of operator code alpha."""
    n = len(ops)
    if n == 0:
        return np.trace(scipy.linalg.expm(-beta * H))
    M = scipy.linalg.expm(-tau[0] * H)
    for i in range(n):
        M = op_mats[int(ops[i])] @ M
        dt = (tau[i + 1] - tau[i]) if i + 1 < n else (beta - tau[n - 1])
        M = scipy.linalg.expm(-dt * H) @ M
    return np.trace(M)


# ---------------------------------------------------------------------------
# lazy-trace bounds
# ---------------------------------------------------------------------------


def _segments(tau, n, beta):
    """Propagation times after each operator (the last one is the wrap-around
    part beta - tau_n, which joins tau_1 on q0)."""
    return [((tau[i + 1] - tau[i]) if i + 1 < n else None) for i in range(n)]


def level0_bound(model, tau, ops, q0: int, beta: float):
    """log b(q0) (see module docstring), or -inf if the string dies."""
    path = walk(model, ops, q0)
    if path is None:
        return -math.inf
    n = len(ops)
    Emin = model.E_min
    r = min(model.dims[q] for q in path)
    if n == 0:
        return math.log(model.dims[q0]) - beta * Emin[q0]
    lb = math.log(r) - (beta - tau[n - 1] + tau[0]) * Emin[q0]
    for i in range(n):
        nrm = model.opnorm(int(ops[i]), path[i])
        if nrm == 0.0:
            return -math.inf
        lb += math.log(nrm)
        if i + 1 < n:
            lb -= (tau[i + 1] - tau[i]) * Emin[path[i + 1]]
    return lb


def refined_bounds_q0(model, tau, ops, q0: int, beta: float, S: int):
    """[log ub(q0, min(s*S, n)) for s = 0 .. ceil(n/S)] (see module docstring);
    the last entry is log|w_q0|.  None if the string dies."""
    path = walk(model, ops, q0)
    if path is None:
        return None
    n = len(ops)
    E, Emin = model.E, model.E_min
    r = min(model.dims[q] for q in path)
    if n == 0:
        v = float(np.sum(np.exp(-beta * (E[q0] - Emin[q0]))))
        return [math.log(v) - beta * Emin[q0]]
    t_wrap = beta - tau[n - 1] + tau[0]
    # log of prod_{i > j} ||F_i||_2 e^{-dtau_i E_min(q_i)} for each j (suffix sums)
    tail = [0.0] * (n + 1)
    for i in range(n - 1, -1, -1):
        term = math.log(model.opnorm(int(ops[i]), path[i]))
        if i + 1 < n:
            term -= (tau[i + 1] - tau[i]) * Emin[path[i + 1]]
        tail[i] = tail[i + 1] + term
    # tail[j] covers operators j..n-1 (0-based), i.e. those after the first j
    out = []
    Y = np.diag(np.exp(-t_wrap * (E[q0] - Emin[q0]))).astype(model_dtype(model))
    L = -t_wrap * Emin[q0]
    n_seg = -(-n // S)
    j = 0
    for s in range(n_seg + 1):
        target = min(s * S, n)
        while j < target:
            Fb = model.F[(int(ops[j]), path[j])]
            Y = Fb @ Y
            if j + 1 < n:
                dt = tau[j + 1] - tau[j]
                Y = np.exp(-dt * (E[path[j + 1]] - Emin[path[j + 1]]))[:, None] * Y
                L -= dt * Emin[path[j + 1]]
            Y, e = _rescale(Y)
            j += 1
            if Y is None:
                break
            L += e
        if Y is None:
            out.extend([-math.inf] * (n_seg + 1 - s))
            return out
        if target == n:
            v = np.trace(Y)
            out.append(math.log(abs(v)) + L if v != 0 else -math.inf)
        else:
            fro = float(np.linalg.norm(Y))
            out.append(0.5 * math.log(r) + math.log(fro) + L + tail[j])
    return out


def chain_bounds(model, tau, ops, beta: float, S: int):
    """Per chain: (log B level 0, [log ub(s) for s = 0..ceil(n/S)]) with
    ub(s) = sum over surviving q0 of ub(q0, s); entry 0 is the refined bound
    before any operator (not the level-0 B)."""
    tau = np.asarray(tau, dtype=np.float64)
    ops = np.asarray(ops, dtype=np.int64)
    l0, rows = [], []
    for q0 in range(model.n_sec):
        b = level0_bound(model, tau, ops, q0, beta)
        if b == -math.inf:
            continue
        l0.append(b)
        rows.append(refined_bounds_q0(model, tau, ops, q0, beta, S))
    if not l0:
        return -math.inf, []
    m = max(l0)
    B = m + math.log(sum(math.exp(x - m) for x in l0))
    n_s = len(rows[0])
    ub = []
    for s in range(n_s):
        vals = [row[s] for row in rows if row[s] != -math.inf]
        if not vals:
            ub.append(-math.inf)
            continue
        mm = max(vals)
        ub.append(mm + math.log(sum(math.exp(x - mm) for x in vals)))
    return B, ub


def decide(log_abs_w: float, log_threshold: float) -> bool:
    """Metropolis-Hastings with the random number drawn first (Eq. decide):
    accept iff log|w| >= T, T = log r + log|w_old| - log(other ratios)."""
    return log_abs_w >= log_threshold


# ---------------------------------------------------------------------------
# atomic Green function
# ---------------------------------------------------------------------------


def green_atomic(model, flavour: int, tau: float) -> float:
    """G(tau) = -<c_f(tau) c_f^+(0)>_loc = -Tr[e^{-(beta-tau)H} c e^{-tau H} c^+]/Z
    (Sec. 2.1, G_loc), from two sector-string traces: c^+ at time 0, c at tau."""
    beta = model.beta
    z = trace_chain(model, [], [])
    w = trace_chain(model, [0.0, tau], [2 * flavour + 1, 2 * flavour])
    if w["log_abs"] == -math.inf:
        return 0.0
    return -float(np.real(w["phase"])) * math.exp(w["log_abs"] - z["log_abs"])

"""Oracle, part 3: the reduced-density-matrix estimator (TEST INFRASTRUCTURE
ONLY; see oracle/__init__).

Definition followed (Sec. 2.3, "Estimators", Eq. ImpurityDensityMatrix): for
one configuration C with time-ordered operators at 0 <= tau_1 < ... < tau_n < beta,

    rho^C_{uv} = beta^{-1} int_0^beta  w_loc(C, P_vu(tau)) / w_loc(C)  dtau,

where P_vu = |v><u| (u, v eigenstates of H_loc) is inserted at time tau into
the time-ordered product, and the integral is taken analytically.  Only
u, v in the same sector contribute (the projector must commute with the
abelian quantum numbers).

Written out with the sector strings of Sec. 3.3.1: for tau in the interval
(tau_i, tau_{i+1}) of a string through sector q_i,

    w_loc(C, P_vu(tau)) = sum_{q0} e^{-(tau - tau_i) E_u} (G_i)_{uv} e^{-(tau_{i+1} - tau) E_v},
    G_i = [F_i P_{tau_i - tau_{i-1}} ... F_1 P_{tau_1}] [P_{beta - tau_n} F_n ... P_{tau_{i+2} - tau_{i+1}} F_{i+1}],

with interval 0 = (0, tau_1) (G_0 = P_{beta - tau_n} F_n ... F_1) and interval
n = (tau_n, beta) (G_n = F_n ... F_1 P_{tau_1}), both in q0.  The tau
integral over an interval of length D is

    K(a, b, D) = int_0^D e^{-s a} e^{-(D - s) b} ds
               = (e^{-D b} - e^{-D a}) / (a - b)   (a != b),   D e^{-D a}   (a == b),

so rho^C = beta^{-1} sum_{q0} sum_i G_i o K_i / w_loc(C) (o: elementwise).

All energies are taken relative to the ground-state energy E_gs, which
multiplies numerator and denominator by the same e^{beta E_gs} (the
propagation times sum to beta); the products are plain float64 matrix
products in that convention (no rescaling: e^{-beta (E - E_gs)} stays far
above the float64 underflow for the models used here).
"""
from __future__ import annotations

import math

import numpy as np

from .trace import walk


def kernel_matrix(Ea: np.ndarray, Eb: np.ndarray, D: float) -> np.ndarray:
    """K(Ea[u], Eb[v], D) for all u, v (energies relative to E_gs), written
    as e^{-D min(a, b)} (1 - e^{-D |a - b|}) / |a - b| (the same closed form,
    without the cancellation of the difference quotient for nearly equal
    energies), D e^{-D a} for a == b."""
    a = np.asarray(Ea, dtype=np.float64)[:, None]
    b = np.asarray(Eb, dtype=np.float64)[None, :]
    lo = np.minimum(a, b)
    gap = np.abs(a - b)
    with np.errstate(divide="ignore", invalid="ignore"):
        frac = np.where(gap > 0.0, -np.expm1(-D * gap) / gap, D)
    return np.exp(-D * lo) * frac


def rho_layout(model):
    """Offsets of the sector blocks of rho in the flat layout: block q is
    d_q x d_q, row-major, blocks in sector order."""
    off = [0]
    for d in model.dims:
        off.append(off[-1] + d * d)
    return off


def density_matrix_chain(model, tau, ops, beta: float | None = None):
    """rho^C for one configuration: dict q -> (d_q x d_q) matrix, plus w
    (relative to e^{-beta E_gs}).  Returns (rho, w); rho is None when w == 0."""
    beta = model.beta if beta is None else beta
    tau = np.asarray(tau, dtype=np.float64)
    ops = np.asarray(ops, dtype=np.int64)
    n = len(ops)
    E = [np.asarray(e) - model.E_gs for e in model.E]
    dt = np.complex128 if model.is_complex else np.float64

    def P(q, D):
        return np.diag(np.exp(-D * E[q]))

    num = {q: np.zeros((d, d), dtype=dt) for q, d in enumerate(model.dims)}
    w = 0.0
    for q0 in range(model.n_sec):
        path = walk(model, ops, q0)
        if path is None:
            continue
        F = [model.F[(int(ops[i]), path[i])] for i in range(n)]  # F[i] acts on sector path[i]
        if n == 0:
            w += np.trace(P(q0, beta))
            num[q0] += np.eye(model.dims[q0]) * kernel_matrix(E[q0], E[q0], beta)  # G = identity
            continue
        # A_i = F_i P ... F_1 P_{tau_1}  (i = 1..n, in sector path[i]); A_0 = I
        A = [np.eye(model.dims[q0], dtype=dt)]
        X = P(q0, tau[0]).astype(dt)
        for i in range(1, n + 1):
            X = F[i - 1] @ X
            A.append(X)
            if i < n:
                X = P(path[i], tau[i] - tau[i - 1]) @ X
        # B_i = P_{beta - tau_n} F_n ... P_{tau_{i+2} - tau_{i+1}} F_{i+1}  (i = 0..n-1); B_n = I
        B = [None] * (n + 1)
        B[n] = np.eye(model.dims[q0], dtype=dt)
        Y = P(q0, beta - tau[n - 1]).astype(dt)
        for i in range(n - 1, -1, -1):
            Y = Y @ F[i]
            B[i] = Y
            if i > 0:
                Y = Y @ P(path[i], tau[i] - tau[i - 1])
        w += np.trace(B[0] @ P(q0, tau[0]))  # w_q0 = Tr[P_{beta - tau_n} F_n ... F_1 P_{tau_1}]
        # interval i in sector path[i] (path[n] = q0), length D_i
        for i in range(n + 1):
            q = path[i] if i < n else q0
            if i == 0:
                D = tau[0]
            elif i == n:
                D = beta - tau[n - 1]
            else:
                D = tau[i] - tau[i - 1]
            G = A[i] @ B[i]
            num[q] += G * kernel_matrix(E[q], E[q], D)
    if w == 0:
        return None, 0.0
    rho = {q: num[q] / (beta * w) for q in num}
    return rho, w


def density_matrix_batch(model, batch, chains=None):
    """density_matrix_chain over a workloads.Batch; returns a list of
    (rho, w) per chain."""
    idx = range(batch.n_chains) if chains is None else chains
    return [density_matrix_chain(model, *batch.chain(int(c)), beta=batch.beta) for c in idx]


def thermal_density_matrix(model, beta: float | None = None):
    """e^{-beta H_loc} / Z in the eigenbasis (the n = 0 estimator)."""
    beta = model.beta if beta is None else beta
    Z = sum(float(np.sum(np.exp(-beta * (np.asarray(e) - model.E_gs)))) for e in model.E)
    return {q: np.diag(np.exp(-beta * (np.asarray(e) - model.E_gs))) / Z for q, e in enumerate(model.E)}


def density_matrix_full_space(H: np.ndarray, op_mats, tau, ops, beta: float, U_sec, n_quad: int = 24):
    """Brute force: rho^C_{uv} by Gauss-Legendre quadrature of
    Tr[T(..., P_vu(tau), ...)] / w over every interval, in the full Fock
    space with dense matrix exponentials.  U_sec[q] maps the eigenbasis of
    sector q to Fock-space columns (u, v are eigenstates).  For tiny models."""
    import scipy.linalg
    Hs = H - np.min(np.linalg.eigvalsh(H)) * np.eye(H.shape[0])
    tau = np.asarray(tau, dtype=np.float64)
    n = len(ops)

    def ev(t):
        return scipy.linalg.expm(-t * Hs)

    O = [op_mats[int(a)] for a in ops]
    bounds = [0.0] + list(tau) + [beta]
    # w = Tr[e^{-(beta - tau_n)H} O_n ... O_1 e^{-tau_1 H}]
    M = ev(bounds[1] - bounds[0])
    for i in range(n):
        M = ev(bounds[i + 2] - bounds[i + 1]) @ O[i] @ M
    w = np.trace(M)
    x, wq = np.polynomial.legendre.leggauss(n_quad)
    rho = {q: np.zeros((U.shape[1], U.shape[1]), dtype=np.complex128) for q, U in enumerate(U_sec)}
    for k in range(n + 1):
        a, b = bounds[k], bounds[k + 1]
        if b <= a:
            continue
        # after = evolution and operators from the insertion time to beta; before = from 0 to the insertion time
        for xi, wi in zip(x, wq):
            t = 0.5 * (b - a) * xi + 0.5 * (a + b)
            before = ev(t - a)
            Mb = ev(bounds[1] - bounds[0]) if k > 0 else np.eye(H.shape[0])
            if k > 0:
                for i in range(k - 1):
                    Mb = ev(bounds[i + 2] - bounds[i + 1]) @ O[i] @ Mb
                Mb = O[k - 1] @ Mb
            before = before @ Mb
            after = ev(b - t)
            for i in range(k, n):
                after = ev(bounds[i + 2] - bounds[i + 1]) @ O[i] @ after
            # Tr[after |v><u| before] = <u| before after |v>
            X = before @ after
            for q, U in enumerate(U_sec):
                rho[q] += 0.5 * (b - a) * wi * (U.conj().T @ X @ U)
    return {q: r / (beta * w) for q, r in rho.items()}, w

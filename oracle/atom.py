"""Oracle, part 1: the atomic problem (TEST INFRASTRUCTURE ONLY; see oracle/__init__).

Plain float64 construction of

* fermion operators on occupation-number states (Sec. 3.3.1: the operator
  matrices (F_i)_{nm} in the many-body Hilbert space); Jordan-Wigner sign
  c_i |n> = (-1)^{sum_{j<i} n_j} |n - e_i>;
* the local Hamiltonian, Eq. ImpurityHamiltonian:
  H = sum_ij c^+_i (t_ij - mu delta_ij) c_j + 1/2 sum_ijkl U_ijkl c^+_i c^+_j c_k c_l;
* the Kanamori interaction (named in App. A) written directly in operator form,
  and the Slater-Condon interaction (App. A) from Gaunt coefficients in complex
  harmonics, rotated to the paper's real-harmonic product basis (App. A, real
  spherical harmonics and Eq. enumProduct ordering);
* spin-orbit coupling xi l.s and a crystal field as extra one-body terms;
* the sector decomposition H = (+)_q H(q) by abelian quantum numbers
  (Sec. 3.3.1), an optional window on N (basis truncation), numpy.linalg.eigh
  per sector (per connected component of the sector's nonzero pattern, so
  that exact zeros stay exact), the sector map s_alpha(q) and the operator blocks
  [F_alpha(q)]_{mn} = <m(q')| c_alpha |n(q)> in the eigenbasis.

Matrix-element reading: the paper prints (F_i)_{nm} = <m|c_i|n>; the oracle
uses F_{mn} = <m|c|n> (row = target), so products act right to left.  The
trace is the same either way.
"""
from __future__ import annotations

import functools
import math
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Fock space
# ---------------------------------------------------------------------------


_POP16 = np.asarray([bin(x).count("1") for x in range(1 << 16)], dtype=np.int64)


def _bits_below(states: np.ndarray, i: int) -> np.ndarray:
    """Number of occupied modes j < i in each state (n_f <= 16)."""
    return _POP16[states & ((1 << i) - 1)]


def apply_op(states: np.ndarray, i: int, dag: int):
    """Apply c_i (dag=0) or c_i^+ (dag=1) to each occupation state.

    Returns (ok, sign, new_states): ok is False where the result is the zero
    vector (Pauli), sign = (-1)^{sum_{j<i} n_j} (Jordan-Wigner)."""
    states = np.asarray(states, dtype=np.int64)
    occ = (states >> i) & 1
    ok = occ == (0 if dag else 1)
    sign = np.where(_bits_below(states, i) % 2 == 0, 1.0, -1.0)
    new = states ^ (1 << i)
    return ok, sign, new


def apply_string(states: np.ndarray, ops):
    """Apply a product of operators, written left to right as in the formula
    (e.g. [(i,1),(j,1),(l,0),(k,0)] for c^+_i c^+_j c_l c_k), to each state;
    the rightmost factor acts first."""
    st = np.asarray(states, dtype=np.int64).copy()
    ok = np.ones(st.shape, dtype=bool)
    sign = np.ones(st.shape, dtype=np.float64)
    for (i, dag) in reversed(list(ops)):
        o, s, n = apply_op(st, i, dag)
        ok &= o
        sign *= s
        st = np.where(o, n, st)
    return ok, sign, st


def full_op_matrix(n_f: int, i: int, dag: int) -> np.ndarray:
    """Dense 2^n_f x 2^n_f matrix of c_i or c_i^+, M[m, n] = <m|c|n>."""
    dim = 1 << n_f
    states = np.arange(dim, dtype=np.int64)
    ok, sign, new = apply_op(states, i, dag)
    m = np.zeros((dim, dim))
    m[new[ok], states[ok]] = sign[ok]
    return m


# ---------------------------------------------------------------------------
# Hamiltonian terms: list of (coefficient, operator string)
# ---------------------------------------------------------------------------


def one_body_terms(t: np.ndarray):
    """sum_ij c^+_i t_ij c_j."""
    terms = []
    n = t.shape[0]
    for i in range(n):
        for j in range(n):
            if t[i, j] != 0:
                terms.append((complex(t[i, j]), ((i, 1), (j, 0))))
    return terms


def kanamori_terms(n_orb: int, U: float, J: float):
    """Rotationally invariant Kanamori interaction in operator form, flavour
    f = sigma * n_orb + a (sigma = 0 down, 1 up):

      U sum_a n_a,up n_a,dn + (U-2J) sum_{a != b} n_a,up n_b,dn
      + (U-3J) sum_{a<b, sigma} n_a,sigma n_b,sigma
      - J sum_{a != b} c^+_a,up c_a,dn c^+_b,dn c_b,up
      + J sum_{a != b} c^+_a,up c^+_a,dn c_b,dn c_b,up
    """
    def f(a, s):
        return s * n_orb + a

    def n_(a, s):
        return ((f(a, s), 1), (f(a, s), 0))

    Up = U - 2.0 * J
    terms = []
    for a in range(n_orb):
        terms.append((U, n_(a, 1) + n_(a, 0)))
    for a in range(n_orb):
        for b in range(n_orb):
            if a == b:
                continue
            terms.append((Up, n_(a, 1) + n_(b, 0)))
            if J != 0.0:
                terms.append((-J, ((f(a, 1), 1), (f(a, 0), 0), (f(b, 0), 1), (f(b, 1), 0))))
                terms.append((J, ((f(a, 1), 1), (f(a, 0), 1), (f(b, 0), 0), (f(b, 1), 0))))
    for a in range(n_orb):
        for b in range(a + 1, n_orb):
            for s in (0, 1):
                terms.append((Up - J, n_(a, s) + n_(b, s)))
    return terms


@functools.lru_cache(maxsize=None)
def wigner_3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """Wigner 3j symbol for integer arguments, Racah's closed formula."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    fa = math.factorial
    tri = Fraction(fa(j1 + j2 - j3) * fa(j1 - j2 + j3) * fa(-j1 + j2 + j3), fa(j1 + j2 + j3 + 1))
    pre = tri * fa(j1 + m1) * fa(j1 - m1) * fa(j2 + m2) * fa(j2 - m2) * fa(j3 + m3) * fa(j3 - m3)
    s = Fraction(0)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    for k in range(kmin, kmax + 1):
        den = (fa(k) * fa(j3 - j2 + k + m1) * fa(j3 - j1 + k - m2) * fa(j1 + j2 - j3 - k)
               * fa(j1 - k - m1) * fa(j2 - k + m2))
        s += Fraction((-1) ** k, den)
    sign = (-1) ** (j1 - j2 - m3)
    return float(sign * s * math.sqrt(pre))


def gaunt_ck(l: int, k: int, m: int, mp: int) -> float:
    """c^k(l m, l m') = sqrt(4 pi/(2k+1)) int Y*_{lm} Y_{k,m-m'} Y_{lm'}
    = (-1)^m (2l+1) (l k l; 0 0 0) (l k l; -m, m-m', m')."""
    return ((-1) ** m) * (2 * l + 1) * wigner_3j(l, k, l, 0, 0, 0) * wigner_3j(l, k, l, -m, m - mp, mp)


def slater_F(l: int, U: float, J: float):
    """Slater integrals {k: F^k} from (U, J): F0 = U;
    d: J = (F2 + F4)/14, F4/F2 = 0.625;
    f: J = (286 F2 + 195 F4 + 250 F6)/6435, F4/F2 = 0.668, F6/F2 = 0.494."""
    if l == 2:
        F2 = 14.0 * J / (1.0 + 0.625)
        return {0: U, 2: F2, 4: 0.625 * F2}
    if l == 3:
        F2 = 6435.0 * J / (286.0 + 195.0 * 0.668 + 250.0 * 0.494)
        return {0: U, 2: F2, 4: 0.668 * F2, 6: 0.494 * F2}
    raise ValueError("slater needs l = 2 or 3")


def slater_orbital_tensor(l: int, F: dict) -> np.ndarray:
    """<m1 m2|V|m3 m4> = sum_k F^k c^k(m1,m3) c^k(m4,m2) delta_{m1+m2, m3+m4}
    in complex harmonics, index m + l."""
    n = 2 * l + 1
    V = np.zeros((n, n, n, n))
    for m1 in range(-l, l + 1):
        for m2 in range(-l, l + 1):
            for m3 in range(-l, l + 1):
                m4 = m1 + m2 - m3
                if abs(m4) > l:
                    continue
                v = 0.0
                for k, Fk in F.items():
                    v += Fk * gaunt_ck(l, k, m1, m3) * gaunt_ck(l, k, m4, m2)
                V[m1 + l, m2 + l, m3 + l, m4 + l] = v
    return V


def real_harmonics_T(l: int) -> np.ndarray:
    """Rows: real harmonics Y_{l,m} (m = -l..l) as combinations of complex Y_l^m
    (App. A): m<0: (i/sqrt2)(Y^m - (-1)^m Y^{-m}); m=0: Y^0;
    m>0: (1/sqrt2)(Y^{-m} + (-1)^m Y^m).  |r> = sum_m T[r, m] |m>."""
    n = 2 * l + 1
    T = np.zeros((n, n), dtype=np.complex128)
    r2 = 1.0 / math.sqrt(2.0)
    for m in range(-l, l + 1):
        r = m + l
        if m < 0:
            T[r, m + l] += 1j * r2
            T[r, -m + l] += -1j * r2 * (-1) ** m
        elif m == 0:
            T[r, l] = 1.0
        else:
            T[r, -m + l] += r2
            T[r, m + l] += r2 * (-1) ** m
    return T


def to_real_basis_tensor(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    """V'_{abcd} = sum T*_{a m1} T*_{b m2} V_{m1 m2 m3 m4} T_{c m3} T_{d m4}."""
    return np.einsum("ai,bj,ijkl,ck,dl->abcd", T.conj(), T.conj(), V, T, T)


def to_real_basis_one_body(h: np.ndarray, T: np.ndarray) -> np.ndarray:
    """<r|h|r'> = (T* h T^T)[r, r']."""
    return T.conj() @ h @ T.T


def orbital_tensor_terms(n_orb: int, Vorb: np.ndarray, tol: float = 1e-14):
    """1/2 sum V_{ijkl} c^+_i c^+_j c_l c_k over spin-orbitals i=(a,s), with
    V_{ijkl} = delta_{s_i s_k} delta_{s_j s_l} Vorb_{a_i a_j a_k a_l}."""
    terms = []
    for a in range(n_orb):
        for b in range(n_orb):
            for c in range(n_orb):
                for d in range(n_orb):
                    v = Vorb[a, b, c, d]
                    if abs(v) < tol:
                        continue
                    for s1 in (0, 1):
                        for s2 in (0, 1):
                            i, j = s1 * n_orb + a, s2 * n_orb + b
                            k, l = s1 * n_orb + c, s2 * n_orb + d
                            if i == j or k == l:
                                continue
                            terms.append((0.5 * complex(v), ((i, 1), (j, 1), (l, 0), (k, 0))))
    return terms


def soc_complex(l: int, xi: float) -> np.ndarray:
    """xi l.s in the complex product basis, flavour (sigma, m): index
    sigma*(2l+1) + m + l, sigma = 0 down (s_z=-1/2), 1 up."""
    n = 2 * l + 1
    h = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    for s in (0, 1):
        sz = -0.5 if s == 0 else 0.5
        for m in range(-l, l + 1):
            h[s * n + m + l, s * n + m + l] += xi * m * sz
    # 1/2 (l+ s- + l- s+):  <m+1, dn| l.s |m, up> = 1/2 sqrt(l(l+1) - m(m+1))
    for m in range(-l, l):
        v = 0.5 * xi * math.sqrt(l * (l + 1) - m * (m + 1))
        h[0 * n + (m + 1) + l, 1 * n + m + l] += v
        h[1 * n + m + l, 0 * n + (m + 1) + l] += v
    return h


# ---------------------------------------------------------------------------
# model assembly
# ---------------------------------------------------------------------------


def one_body_matrix(p, mu: float) -> np.ndarray:
    """The one-body part t_ij - mu delta_ij of H_loc (Eq. ImpurityHamiltonian)
    as an n_f x n_f complex matrix in the flavour basis: spin-orbit coupling
    (slater shells) and the crystal field, with -mu on the diagonal."""
    n_orb = p.n_orb
    n_f = 2 * n_orb
    t = np.zeros((n_f, n_f), dtype=np.complex128)
    t -= mu * np.eye(n_f)
    if p.interaction == "slater" and p.soc_xi != 0.0:
        T = real_harmonics_T(p.l)
        TT = np.zeros((n_f, n_f), dtype=np.complex128)
        TT[:n_orb, :n_orb] = T
        TT[n_orb:, n_orb:] = T
        t += to_real_basis_one_body(soc_complex(p.l, p.soc_xi), TT)
    if p.cf is not None:
        t += np.asarray(p.cf, dtype=np.complex128)
    return t


def interaction_terms(p):
    """The interaction part U of H_loc (the two-body terms of Eq.
    ImpurityHamiltonian) for a parameter set."""
    if p.interaction == "kanamori":
        if p.soc_xi != 0.0:
            raise ValueError("SOC needs a slater shell")
        return kanamori_terms(p.n_orb, p.U, p.J)
    if p.interaction == "slater":
        F = slater_F(p.l, p.U, p.J)
        T = real_harmonics_T(p.l)
        Vr = to_real_basis_tensor(slater_orbital_tensor(p.l, F), T)
        return orbital_tensor_terms(p.n_orb, Vr)
    raise ValueError(p.interaction)


def hamiltonian_terms(p, mu: float):
    """All terms of H_loc for a parameter set (see paper_2010_08482_gb300
    workloads.ModelParams for the fields), at chemical potential mu."""
    inter = interaction_terms(p)
    return one_body_terms(one_body_matrix(p, mu)) + inter


def sector_states(p):
    """Sector labels and their occupation states (ascending integers).
    n_sz: label (N_dn, N_up); n: label (N,).  States outside the N window are
    dropped."""
    n_orb, n_f = p.n_orb, 2 * p.n_orb
    groups = {}
    for s in range(1 << n_f):
        nd = bin(s & ((1 << n_orb) - 1)).count("1")
        nu = bin(s >> n_orb).count("1")
        N = nd + nu
        if p.n_min >= 0 and N < p.n_min:
            continue
        if p.n_max >= 0 and N > p.n_max:
            continue
        key = (nd, nu) if p.sector_mode == "n_sz" else (N,)
        groups.setdefault(key, []).append(s)
    labels = sorted(groups.keys(), key=lambda k: (sum(k), k))
    return labels, [np.asarray(groups[k], dtype=np.int64) for k in labels]


def sector_hamiltonian(states: np.ndarray, terms) -> np.ndarray:
    """Dense H restricted to one sector, H[m, n] = <m|H|n>."""
    d = len(states)
    H = np.zeros((d, d), dtype=np.complex128)
    for coef, ops in terms:
        ok, sign, new = apply_string(states, ops)
        cols = np.nonzero(ok)[0]
        if cols.size == 0:
            continue
        rows = np.searchsorted(states, new[cols])
        rows_c = np.minimum(rows, d - 1)
        if np.any(states[rows_c] != new[cols]):
            raise RuntimeError("term leaves its sector")
        np.add.at(H, (rows_c, cols), coef * sign[cols])
    return H


def eigh_by_components(h: np.ndarray):
    """Eigen-decomposition of a Hermitian sector Hamiltonian.

    H restricted to a sector is still block-diagonal over the connected
    components of its nonzero pattern (states that no chain of nonzero matrix
    elements links are never mixed by H).  numpy.linalg.eigh is applied to each
    component on its own, so eigenvectors have exact zeros outside their
    component and strings that such a hidden symmetry forbids give exactly 0
    instead of rounding noise.  Returns (E ascending, V columns)."""
    d = h.shape[0]
    adj = h != 0
    comp = -np.ones(d, dtype=np.int64)
    n_comp = 0
    for start in range(d):
        if comp[start] >= 0:
            continue
        stack = [start]
        comp[start] = n_comp
        while stack:
            i = stack.pop()
            for j in np.nonzero(adj[i])[0]:
                if comp[j] < 0:
                    comp[j] = n_comp
                    stack.append(j)
        n_comp += 1
    E = np.zeros(d)
    V = np.zeros((d, d), dtype=h.dtype)
    col = 0
    for k in range(n_comp):
        idx = np.nonzero(comp == k)[0]
        e, v = np.linalg.eigh(h[np.ix_(idx, idx)])
        E[col:col + len(idx)] = e
        V[idx, col:col + len(idx)] = v
        col += len(idx)
    order = np.argsort(E, kind="stable")
    return E[order], V[:, order]


class Model:
    """Sector-decomposed impurity in its eigenbasis.

    labels[q], N[q], dims[q], E[q] (ascending, mu included), V[q] (columns =
    eigenvectors in the occupation basis of states[q]), s[alpha][q] (target
    sector or -1), F[(alpha, q)] (d_{s(q)} x d_q), is_complex, mu, beta."""

    def __init__(self, p, terms_override=None):
        self.params = p
        self.n_flav = 2 * p.n_orb
        self.beta = p.beta
        self.labels, self.states = sector_states(p)
        self.n_sec = len(self.labels)
        self.N = [sum(k) for k in self.labels]
        self.dims = [len(s) for s in self.states]
        terms0 = terms_override if terms_override is not None else hamiltonian_terms(p, 0.0)
        H0 = [sector_hamiltonian(st, terms0) for st in self.states]
        self.is_complex = any(np.abs(h.imag).max() > 0.0 for h in H0)
        E0, self.V = [], []
        for h in H0:
            e, v = eigh_by_components(h if self.is_complex else h.real)
            E0.append(e)
            self.V.append(v)
        if p.mu is None:
            egs = {}
            for q in range(self.n_sec):
                egs[self.N[q]] = min(egs.get(self.N[q], np.inf), E0[q][0])
            self.mu = 0.5 * (egs[p.n0 + 1] - egs[p.n0 - 1])
        else:
            self.mu = float(p.mu)
        self.E = [E0[q] - self.mu * self.N[q] for q in range(self.n_sec)]
        self.E_min = np.asarray([e[0] for e in self.E])
        self.E_gs = float(self.E_min.min())
        self._build_blocks()

    def _build_blocks(self):
        all_states = np.concatenate(self.states)
        order = np.argsort(all_states)
        self._sorted_states = all_states[order]
        self._sec_of = np.concatenate([np.full(d, q) for q, d in enumerate(self.dims)])[order]
        self._pos_of = np.concatenate([np.arange(d) for d in self.dims])[order]
        n_alpha = 2 * self.n_flav
        self.s = np.full((n_alpha, self.n_sec), -1, dtype=np.int64)
        self.F = {}
        for alpha in range(n_alpha):
            for q in range(self.n_sec):
                got = self.occupation_op(alpha, q)
                if got is None:
                    continue
                qp, C = got
                Fb = self.V[qp].conj().T @ (C @ self.V[q])
                self.s[alpha, q] = qp
                self.F[(alpha, q)] = Fb if self.is_complex else Fb.real

    def occupation_op(self, alpha: int, q: int):
        """Operator alpha = 2 f + dag restricted to sector q in the occupation
        basis: (target sector q', C) with C[m, n] = <m(q')|c_f or c+_f|n(q)>
        (Jordan-Wigner signs), or None if it maps q to zero (or out of the N
        window)."""
        f, dag = alpha // 2, alpha % 2
        st = self.states[q]
        ok, sign, new = apply_op(st, f, dag)
        cols = np.nonzero(ok)[0]
        idx = np.minimum(np.searchsorted(self._sorted_states, new[cols]), len(self._sorted_states) - 1)
        inside = self._sorted_states[idx] == new[cols]  # else: leaves the N window
        cols, idx = cols[inside], idx[inside]
        if cols.size == 0:
            return None
        targets = np.unique(self._sec_of[idx])
        if targets.size != 1:
            raise RuntimeError("operator does not map a sector onto a unique sector")
        qp = int(targets[0])
        C = np.zeros((self.dims[qp], self.dims[q]))
        C[self._pos_of[idx], cols] = sign[cols]
        return qp, C

    def opnorm(self, alpha: int, q: int) -> float:
        """Spectral norm ||F_alpha(q)||_2 (numpy SVD)."""
        return float(np.linalg.norm(self.F[(alpha, q)], 2))

    def spectrum(self) -> np.ndarray:
        return np.sort(np.concatenate(self.E))


def full_hamiltonian(p, mu: float) -> np.ndarray:
    """Dense H over the whole 2^n_f Fock space (no sectors), for brute force."""
    n_f = 2 * p.n_orb
    states = np.arange(1 << n_f, dtype=np.int64)
    H = sector_hamiltonian(states, hamiltonian_terms(p, mu))
    return H

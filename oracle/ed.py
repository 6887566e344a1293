"""Oracle, part 5: exact diagonalisation of an impurity coupled to a discrete
bath (TEST INFRASTRUCTURE ONLY; see oracle/__init__).

The model is the impurity model of Sec. 2.1 with a fermionic bath only:

    H = H_loc + sum_{f, l} eps_l b^+_{f l} b_{f l}
              + sum_{f, l} V_l (c^+_f b_{f l} + b^+_{f l} c_f),

H_loc from oracle.atom (Eq. ImpurityHamiltonian), n_b bath levels eps_l per
flavour f, each hybridised with its own flavour only (a diagonal
hybridisation function).  The benchmark of Sec. 4.1 is the single-orbital
case with three bath levels at -D/2, 0 and D/2, V = D = 1, U = 4 D,
eps_f = -U/2 (mu = U/2) and beta = 10.

Modes: the impurity flavours keep oracle.atom's enumeration (0 .. n_f - 1);
bath level l of flavour f is mode n_f + f n_b + l.  The full Fock space is
split by total particle number (H conserves it) and each block is
diagonalised with numpy.linalg.eigh.

Quantities, all plain sums over the eigenstates |m> (energies E_m):

* Z = sum_m e^{-beta E_m} and thermal averages <O> = Z^-1 sum_m e^{-beta E_m} <m|O|m>;
* the hybridisation energy <H_hyb> and, from it, the mean expansion order
  of the hybridisation expansion (Sec. 2.2): weighting every hybridisation
  pair by lambda^2 (V -> lambda V) gives lambda d ln Z / d lambda = 2 <k> and
  = -beta <H_hyb> (Hellmann-Feynman), so <k> = -beta <H_hyb> / 2;
* the impurity Green function G_f(tau) = -<c_f(tau) c^+_f>
  = -Z^-1 sum_{m,n} e^{-(beta - tau) E_m} e^{-tau E_n} |<m|c_f|n>|^2, and its
  average over a time bin (integrated analytically);
* the hybridisation function of the bath, Delta_f(tau) = sum_l V_l^2 g_l(tau),
  g_l(tau) = -e^{-eps_l tau} / (1 + e^{-beta eps_l}) on (0, beta) (the
  Fourier transform of sum_l V_l^2 / (i nu - eps_l), Eq. hybridization).
"""
from __future__ import annotations

import math

import numpy as np

from . import atom


class ImpurityED:
    """Exact eigenstates of impurity + bath for an oracle.atom parameter set
    p (impurity), bath levels eps [n_b] and hybridisations V [n_b]."""

    def __init__(self, p, mu: float, eps, V, beta: float):
        self.p = p
        self.beta = float(beta)
        self.eps = np.asarray(eps, dtype=np.float64)
        self.V = np.asarray(V, dtype=np.float64)
        self.n_f = 2 * p.n_orb
        self.n_b = len(self.eps)
        self.n_modes = self.n_f * (1 + self.n_b)
        if self.n_modes > 16:
            raise ValueError("at most 16 modes")
        terms = atom.hamiltonian_terms(p, mu)
        self.hyb_terms = []
        for f in range(self.n_f):
            for l_ in range(self.n_b):
                b = self.bath_mode(f, l_)
                terms.append((complex(self.eps[l_]), ((b, 1), (b, 0))))
                self.hyb_terms.append((complex(self.V[l_]), ((f, 1), (b, 0))))
                self.hyb_terms.append((complex(self.V[l_]), ((b, 1), (f, 0))))
        self.terms = terms + self.hyb_terms
        # blocks by total particle number
        states = np.arange(1 << self.n_modes, dtype=np.int64)
        N = np.asarray([bin(int(s)).count("1") for s in states])
        self.blocks = []
        for n in range(self.n_modes + 1):
            st = states[N == n]
            H = atom.sector_hamiltonian(st, self.terms)
            if np.abs(H.imag).max(initial=0.0) > 0.0:
                raise ValueError("complex impurity models are not handled here")
            e, v = np.linalg.eigh(H.real)
            self.blocks.append((st, e, v))
        self.E0 = min(float(e[0]) for _, e, _ in self.blocks)
        self.Z = sum(float(np.sum(np.exp(-self.beta * (e - self.E0)))) for _, e, _ in self.blocks)

    def bath_mode(self, f: int, l_: int) -> int:
        return self.n_f + f * self.n_b + l_

    def thermal(self, terms) -> float:
        """<O> for O given as oracle.atom terms (coefficient, operator string)."""
        tot = 0.0
        for st, e, v in self.blocks:
            O = atom.sector_hamiltonian(st, terms).real
            w = np.exp(-self.beta * (e - self.E0))
            tot += float(np.sum(w * np.einsum("im,ij,jm->m", v, O, v)))
        return tot / self.Z

    def occupation(self, f: int) -> float:
        return self.thermal([(1.0, ((f, 1), (f, 0)))])

    def double_occupancy(self) -> float:
        """sum_a <n_{a,up} n_{a,dn}> over the impurity orbitals."""
        n = self.p.n_orb
        return self.thermal([(1.0, ((a + n, 1), (a + n, 0), (a, 1), (a, 0))) for a in range(n)])

    def hybridisation_energy(self) -> float:
        return self.thermal(self.hyb_terms)

    def mean_order(self) -> float:
        """<k> = -beta <H_hyb> / 2: mean number of hybridisation pairs."""
        return -0.5 * self.beta * self.hybridisation_energy()

    def _c_blocks(self, f: int):
        """(E_m, E_n, |<m|c_f|n>|^2) over block pairs N -> N - 1."""
        out = []
        for n in range(1, len(self.blocks)):
            st_n, e_n, v_n = self.blocks[n]
            st_m, e_m, v_m = self.blocks[n - 1]
            ok, sign, new = atom.apply_op(st_n, f, 0)
            C = np.zeros((len(st_m), len(st_n)))
            pos = np.searchsorted(st_m, new[ok])
            C[pos, np.nonzero(ok)[0]] = sign[ok]
            A = v_m.T @ C @ v_n
            out.append((e_m, e_n, A * A))
        return out

    def green(self, f: int, tau) -> np.ndarray:
        """G_f(tau) for tau in (0, beta) (array)."""
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        g = np.zeros_like(tau)
        for e_m, e_n, A2 in self._c_blocks(f):
            em = (e_m - self.E0)[:, None]
            en = (e_n - self.E0)[None, :]
            for i, t in enumerate(tau):
                g[i] -= float(np.sum(A2 * np.exp(-(self.beta - t) * em - t * en)))
        return g / self.Z

    def green_bin(self, f: int, a: float, b: float) -> float:
        """(b - a)^-1 int_a^b G_f(tau) dtau, integrated analytically."""
        tot = 0.0
        for e_m, e_n, A2 in self._c_blocks(f):
            em = (e_m - self.E0)[:, None]
            en = (e_n - self.E0)[None, :]
            d = em - en  # integrand e^{-beta em} e^{tau d}
            with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
                big = np.abs(d) * (b - a) > 1e-8
                val = np.where(big, (np.exp(-self.beta * em + b * d) - np.exp(-self.beta * em + a * d))
                               / np.where(big, d, 1.0),
                               (b - a) * np.exp(-self.beta * em + 0.5 * (a + b) * d))
            tot -= float(np.sum(A2 * val))
        return tot / self.Z / (b - a)


def hybridisation_function(eps, V, beta: float, tau) -> np.ndarray:
    """Delta(tau) = sum_l V_l^2 g_l(tau) on (-beta, beta), antiperiodic:
    g_l(tau) = -e^{-eps_l tau} / (1 + e^{-beta eps_l}) for 0 < tau < beta and
    g_l(tau) = -g_l(tau + beta) for -beta < tau < 0."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros_like(tau)
    neg = tau < 0
    t = np.where(neg, tau + beta, tau)
    for e, v in zip(eps, V):
        # -e^{-e t} / (1 + e^{-beta e}), written without overflow for either sign of e
        if e >= 0:
            g = -np.exp(-e * t) / (1.0 + math.exp(-beta * e))
        else:
            g = -np.exp(e * (beta - t)) / (1.0 + math.exp(beta * e))
        out += v * v * g
    return np.where(neg, -out, out)

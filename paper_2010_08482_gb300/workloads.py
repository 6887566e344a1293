"""Seeded synthetic inputs for the CT-HYB local-trace path.

This module produces *inputs only*: model parameter sets (the local-Hamiltonian
parameters of Eq. ImpurityHamiltonian, Sec. 2.1, with crystal-field matrices
drawn from a seeded generator) and batches of time-ordered operator sequences
that stand in for Markov-chain configurations (Sec. 3.3.1: configurations are
strings of c / c^dagger operators at imaginary times in [0, beta)).

It holds none of the trace arithmetic: no Fock space, no Hamiltonian, no
sectors, no products.  Both the FP64 oracle (in tests) and the GPU path consume
what it returns; neither is imported here.

Operator code convention (shared by every consumer): alpha = 2*f + dag, where
f is the flavour (spin-orbital) index in the paper's enumeration order
(all spin-down orbitals first, then all spin-up, App. A "Basis functions") and
dag = 1 for c^dagger, 0 for c.

The paper's own workloads (delta-Pu Markov chains, Sec. 4.2; Hubbard chains,
Sec. 4.1) are not available; the five workloads below stand in for them with
the paper's shell sizes (d: 10, f: 14 spin-orbitals), crystal-field / SOC
symmetry breaking and beta range.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 2010084820


@dataclasses.dataclass
class ModelParams:
    """Local-impurity parameters (Eq. ImpurityHamiltonian).

    interaction: "kanamori" (rotationally invariant Kanamori U, U' = U - 2J, J)
                 or "slater" (Slater-Condon with F0 = U and J fixing F2, F4[, F6]).
    l:           angular momentum of the shell for "slater" (2: d, 3: f); for
                 "kanamori" the orbital basis is generic (l = 0 here).
    mu:          chemical potential; None selects the particle-hole symmetric
                 point around n0: E_gs(n0 - 1) = E_gs(n0 + 1).
    soc_xi:      spin-orbit strength xi of xi * l.s (slater shells only).
    cf:          extra one-body term t_ij (complex n_f x n_f Hermitian in the
                 flavour basis), or None.
    sector_mode: "n_sz" (sectors labelled by (N_down, N_up)) or "n" (by N).
    n_min/n_max: Hilbert-space truncation window on N (-1: none).
    """

    name: str
    n_orb: int
    l: int
    interaction: str
    U: float
    J: float
    beta: float
    mu: Optional[float]
    n0: int
    soc_xi: float = 0.0
    cf: Optional[np.ndarray] = None
    sector_mode: str = "n_sz"
    n_min: int = -1
    n_max: int = -1

    @property
    def n_flav(self) -> int:
        return 2 * self.n_orb


@dataclasses.dataclass
class Batch:
    """A batch of time-ordered operator sequences (host arrays).

    offsets: int32 [C+1]; chain c owns entries offsets[c]:offsets[c+1].
    tau:     float64 [sum 2k_c], strictly increasing per chain, in [0, beta).
    op:      int32 [sum 2k_c], alpha = 2*f + dag.
    model:   int32 [C], index of the model of each chain (mixed batches).
    """

    beta: float
    offsets: np.ndarray
    tau: np.ndarray
    op: np.ndarray
    model: Optional[np.ndarray] = None

    @property
    def n_chains(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def chain(self, c: int):
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        return self.tau[a:b], self.op[a:b]

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        taus, ops, offs = [], [], [0]
        for c in idx:
            t, o = self.chain(int(c))
            taus.append(t)
            ops.append(o)
            offs.append(offs[-1] + len(o))
        return Batch(
            beta=self.beta,
            offsets=np.asarray(offs, dtype=np.int32),
            tau=np.concatenate(taus) if taus else np.zeros(0),
            op=np.concatenate(ops).astype(np.int32) if ops else np.zeros(0, np.int32),
            model=None if self.model is None else self.model[idx].copy(),
        )


# ---------------------------------------------------------------------------
# crystal fields (seeded, independent stream: seed + 100)
# ---------------------------------------------------------------------------

def crystal_field_real_orbital(n_orb: int, sigma: float, seed: int) -> np.ndarray:
    """Spin-diagonal real symmetric CF: orbital block (A + A^T)/2, A_ij ~ N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, sigma, size=(n_orb, n_orb))
    h = 0.5 * (a + a.T)
    cf = np.zeros((2 * n_orb, 2 * n_orb), dtype=np.complex128)
    cf[:n_orb, :n_orb] = h
    cf[n_orb:, n_orb:] = h
    return cf


def crystal_field_complex(n_flav: int, sigma: float, seed: int) -> np.ndarray:
    """Complex Hermitian CF over all flavours: (A + A^H)/2, Re, Im ~ N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, sigma, size=(n_flav, n_flav)) + 1j * rng.normal(0.0, sigma, size=(n_flav, n_flav))
    return 0.5 * (a + a.conj().T)


# ---------------------------------------------------------------------------
# model parameter sets
# ---------------------------------------------------------------------------

def model_hubbard2() -> ModelParams:
    """2-orbital Kanamori, U=4, J=0.5, mu=U/2, beta=10, sectors (N_dn, N_up)."""
    return ModelParams("hubbard2", n_orb=2, l=0, interaction="kanamori", U=4.0, J=0.5,
                       beta=10.0, mu=2.0, n0=2)


def model_t2g() -> ModelParams:
    """3-orbital t2g Kanamori, U=5, J=0.7, beta=50, half filling N0=3."""
    return ModelParams("t2g", n_orb=3, l=0, interaction="kanamori", U=5.0, J=0.7,
                       beta=50.0, mu=None, n0=3)


def model_d5() -> ModelParams:
    """5-orbital d shell, Slater-Condon U=8, J=1, real CF sigma=0.1, beta=40."""
    cf = crystal_field_real_orbital(5, 0.1, SEED_BASE + 3 + 100)
    return ModelParams("d5", n_orb=5, l=2, interaction="slater", U=8.0, J=1.0,
                       beta=40.0, mu=None, n0=5, cf=cf)


def model_f7() -> ModelParams:
    """7-orbital f shell, Slater U=4.5, J=0.5, SOC 0.3, complex CF sigma=0.05,
    beta=40, truncated to N in {4, 5, 6}, sectors by N."""
    cf = crystal_field_complex(14, 0.05, SEED_BASE + 4 + 100)
    return ModelParams("f7", n_orb=7, l=3, interaction="slater", U=4.5, J=0.5,
                       beta=40.0, mu=None, n0=5, soc_xi=0.3, cf=cf,
                       sector_mode="n", n_min=4, n_max=6)


def model_f45(mu: float) -> ModelParams:
    """The f shell of model_f7 restricted to N in {4, 5} (blocks 1001 / 2002),
    a smaller large-block case for profiler captures; mu is given (the
    caller takes the particle-hole point of the full N in {4, 5, 6} window)."""
    p = model_f7()
    p.name, p.n_min, p.n_max, p.mu = "f45", 4, 5, float(mu)
    return p


def batch_f45(n_chains: int = 2, k: int = 40) -> Batch:
    """Chains of 2k operators for model_f45: a width-1 particle-number walk
    (alternating between N = 4 and 5), G2."""
    rng = np.random.default_rng(7)
    m = model_f7()
    return _pack([g2_chain(rng, m.n_flav, k, m.beta, width=1) for _ in range(n_chains)], m.beta)


def model_atom1(U: float = 3.0, mu: float = 1.0, beta: float = 5.0) -> ModelParams:
    """Single-orbital Hubbard atom (used for the atomic-limit G(tau) check)."""
    return ModelParams("atom1", n_orb=1, l=0, interaction="kanamori", U=U, J=0.0,
                       beta=beta, mu=mu, n0=1)


# ---------------------------------------------------------------------------
# operator-sequence generators
# ---------------------------------------------------------------------------

def _sorted_taus(rng, n: int, beta: float) -> np.ndarray:
    while True:
        t = np.sort(rng.uniform(0.0, beta, size=n))
        if n < 2 or np.all(np.diff(t) > 0.0):
            return t


def g1_chain(rng, n_flav: int, k: int, beta: float):
    """Literal reading of 'tau uniform, flavours uniform, c/c^dagger alternating
    per flavour': k pairs each pick a flavour uniformly; flavour f with m_f pairs
    gets 2 m_f uniform times; its types alternate starting with c^dagger or c
    (fair coin); all flavours are merged by time."""
    flav = rng.integers(0, n_flav, size=k)
    taus, ops = [], []
    for f in range(n_flav):
        m = int(np.sum(flav == f))
        if m == 0:
            continue
        t = rng.uniform(0.0, beta, size=2 * m)
        t.sort()
        first = int(rng.integers(0, 2))  # 1: starts with c^dagger
        types = [first if j % 2 == 0 else 1 - first for j in range(2 * m)]
        taus.append(t)
        ops.append(np.asarray([2 * f + ty for ty in types], dtype=np.int32))
    if not taus:
        return np.zeros(0), np.zeros(0, np.int32)
    tau = np.concatenate(taus)
    op = np.concatenate(ops)
    order = np.argsort(tau, kind="stable")
    tau, op = tau[order], op[order]
    if len(tau) > 1 and not np.all(np.diff(tau) > 0.0):
        return g1_chain(rng, n_flav, k, beta)
    return tau, op


def g2_chain(rng, n_flav: int, k: int, beta: float, width: int = 2):
    """Step-by-step sequence that keeps per-flavour alternation, keeps the
    walk of the total particle number within `width` of its extremes, and can
    always close every open flavour in the remaining steps.  Then 2k uniform
    times are drawn and sorted.  (Needed for N-truncated models: the literal G1
    reading leaves a width-2 N window almost surely.)"""
    n_ops = 2 * k
    while True:
        last = [-1] * n_flav
        count = [0] * n_flav
        n_open = 0
        n_rel, lo, hi = 0, 0, 0
        seq = []
        stuck = False
        for t in range(n_ops):
            rem_after = n_ops - t - 1
            cands = []
            for f in range(n_flav):
                types = (0, 1) if last[f] == -1 else (1 - last[f],)
                for ty in types:
                    n2 = n_rel + (1 if ty == 1 else -1)
                    if max(hi, n2) - min(lo, n2) > width:
                        continue
                    was_open = count[f] % 2 == 1
                    open2 = n_open - 1 if was_open else n_open + 1
                    if open2 > rem_after:
                        continue
                    cands.append((f, ty, open2, n2))
            if not cands:
                stuck = True
                break
            f, ty, open2, n2 = cands[int(rng.integers(0, len(cands)))]
            seq.append((f, ty))
            last[f] = ty
            count[f] += 1
            n_open = open2
            n_rel = n2
            lo, hi = min(lo, n2), max(hi, n2)
        if not stuck and n_open == 0:
            break
    tau = _sorted_taus(rng, n_ops, beta)
    op = np.asarray([2 * f + ty for f, ty in seq], dtype=np.int32)
    return tau, op


def bulla_sequences(batch: Batch, n_flav: int):
    """Input of the static improved estimator (Eq. PImprovedEstimatorStatic):
    for every chain and each of its annihilators c_f (codes 2 f), the chain
    with that one operator replaced by the Bulla operator [c_f, U] (code
    2 n_flav + f), times unchanged.  Returns (Batch of the replaced sequences,
    int32 chain index of each, int32 position of the replaced operator within
    its chain), sequences ordered by chain, then position."""
    op = np.asarray(batch.op, np.int64)
    offs = np.asarray(batch.offsets, np.int64)
    lens = np.diff(offs)
    chain_of = np.repeat(np.arange(batch.n_chains), lens)
    ann = np.nonzero((op < 2 * n_flav) & (op % 2 == 0))[0]
    c_new = chain_of[ann]
    pos = ann - offs[c_new]
    ln = lens[c_new]
    new_offs = np.zeros(len(ann) + 1, np.int64)
    np.cumsum(ln, out=new_offs[1:])
    # gather index of every entry of the replaced sequences
    start = np.repeat(offs[c_new] - new_offs[:-1], ln)
    gather = np.arange(int(new_offs[-1]), dtype=np.int64) + start
    op_new = op[gather].astype(np.int32)
    op_new[new_offs[:-1] + pos] = (2 * n_flav + op[ann] // 2).astype(np.int32)
    out = Batch(beta=batch.beta, offsets=new_offs.astype(np.int32),
                tau=np.asarray(batch.tau, np.float64)[gather], op=op_new)
    return out, c_new.astype(np.int32), pos.astype(np.int32)


def pair_move(rng, tau: np.ndarray, op: np.ndarray, n_flav: int, beta: float):
    """A random local move of a configuration that respects per-flavour
    alternation (the Pauli-aware pair moves of App. B): a flavour is drawn;
    with probability 1/2 (if it has operators) ("rem", times) removes one of
    its operators and the next one of the flavour; otherwise ("ins", times,
    codes) puts two new operators between consecutive operators of the
    flavour on the circle [0, beta) (anywhere if it has none), the earlier
    one of the type that the preceding operator's type requires next."""
    f = int(rng.integers(0, n_flav))
    mine = np.nonzero(np.asarray(op) // 2 == f)[0]
    if len(mine) >= 2 and rng.random() < 0.5:
        i = int(rng.integers(0, len(mine)))
        j = (i + 1) % len(mine)
        return "rem", np.array([tau[mine[i]], tau[mine[j]]])
    if len(mine) == 0:
        return "ins", rng.uniform(0.0, beta, size=2), np.array([2 * f + 1, 2 * f], np.int32)
    i = int(rng.integers(0, len(mine)))
    j = (i + 1) % len(mine)
    L = (tau[mine[j]] - tau[mine[i]]) % beta or beta
    s1, s2 = np.sort(rng.uniform(0.0, L, size=2))
    t1, t2 = (tau[mine[i]] + s1) % beta, (tau[mine[i]] + s2) % beta
    dag_i = int(op[mine[i]]) % 2  # after a creator the flavour is occupied: annihilate first
    return "ins", np.array([t1, t2]), np.array([2 * f + (0 if dag_i else 1), 2 * f + (1 if dag_i else 0)], np.int32)


def apply_pair_move(move, tau: np.ndarray, op: np.ndarray):
    """The configuration (times ascending, codes) after a pair_move."""
    if move[0] == "rem":
        keep = ~np.isin(tau, move[1])
        return tau[keep], op[keep]
    t = np.concatenate([tau, move[1]])
    o = np.concatenate([op, move[2]]).astype(np.int32)
    order = np.argsort(t)
    return t[order], o[order]


def _pack(chains, beta, model=None) -> Batch:
    offs = [0]
    for t, _ in chains:
        offs.append(offs[-1] + len(t))
    tau = np.concatenate([t for t, _ in chains]) if chains else np.zeros(0)
    op = np.concatenate([o for _, o in chains]).astype(np.int32) if chains else np.zeros(0, np.int32)
    return Batch(beta=beta, offsets=np.asarray(offs, dtype=np.int32), tau=tau.astype(np.float64),
                 op=op, model=None if model is None else np.asarray(model, dtype=np.int32))


def batch_hubbard2(n_chains: int = 64, rank: int = 0) -> Batch:
    """64 chains, k ~ U{8..20}, G1.  rank > 0 draws an independent batch of the
    same shape (one per process in multi-GPU runs)."""
    rng = np.random.default_rng(SEED_BASE + 1 + 1000 * rank)
    m = model_hubbard2()
    chains = [g1_chain(rng, m.n_flav, int(rng.integers(8, 21)), m.beta) for _ in range(n_chains)]
    return _pack(chains, m.beta)


def batch_t2g(n_chains: int = 4096, rank: int = 0) -> Batch:
    """4096 chains, k ~ Poisson(40), G1 (rank: see batch_hubbard2)."""
    rng = np.random.default_rng(SEED_BASE + 2 + 1000 * rank)
    m = model_t2g()
    chains = [g1_chain(rng, m.n_flav, int(rng.poisson(40)), m.beta) for _ in range(n_chains)]
    return _pack(chains, m.beta)


def batch_d5(n_chains: int = 1024, rank: int = 0) -> Batch:
    """1024 chains, k ~ Poisson(60), G1 (rank: see batch_hubbard2)."""
    rng = np.random.default_rng(SEED_BASE + 3 + 1000 * rank)
    m = model_d5()
    chains = [g1_chain(rng, m.n_flav, int(rng.poisson(60)), m.beta) for _ in range(n_chains)]
    return _pack(chains, m.beta)


def batch_f7(n_chains: int = 256, rank: int = 0) -> Batch:
    """256 chains, k ~ Poisson(80), G2 (width-2 N walk; rank: see batch_hubbard2)."""
    rng = np.random.default_rng(SEED_BASE + 4 + 1000 * rank)
    m = model_f7()
    chains = [g2_chain(rng, m.n_flav, int(rng.poisson(80)), m.beta) for _ in range(n_chains)]
    return _pack(chains, m.beta)


def batch_mixed(n_chains: int = 2048, rank: int = 0):
    """2048 chains; model uniform over {t2g, d5, f7}; k ~ U{10..200}; G1 for the
    3- and 5-orbital chains, G2 for the f-shell chains.  Also returns a fair
    coin per chain (1: the threshold is set to force an early reject).
    rank: see batch_hubbard2."""
    rng = np.random.default_rng(SEED_BASE + 5 + 1000 * rank)
    models = [model_t2g(), model_d5(), model_f7()]
    which = rng.integers(0, 3, size=n_chains)
    chains = []
    for c in range(n_chains):
        m = models[int(which[c])]
        k = int(rng.integers(10, 201))
        if m.name == "f7":
            chains.append(g2_chain(rng, m.n_flav, k, m.beta))
        else:
            chains.append(g1_chain(rng, m.n_flav, k, m.beta))
    coin = rng.integers(0, 2, size=n_chains).astype(np.int32)
    betas = {m.beta for m in models}
    assert len(betas) <= 2
    return _pack(chains, models[1].beta, model=which), coin


WORKLOADS = {
    "hubbard2": (model_hubbard2, batch_hubbard2),
    "t2g": (model_t2g, batch_t2g),
    "d5": (model_d5, batch_d5),
    "f7": (model_f7, batch_f7),
}


def random_batch(rng, n_flav: int, beta: float, n_chains: int, k_lo: int, k_hi: int,
                 gen: str = "g1") -> Batch:
    """Small seeded batches for parity tests (orders uniform in [k_lo, k_hi])."""
    chains = []
    for _ in range(n_chains):
        k = int(rng.integers(k_lo, k_hi + 1))
        if gen == "g2":
            chains.append(g2_chain(rng, n_flav, k, beta))
        else:
            chains.append(g1_chain(rng, n_flav, k, beta))
    return _pack(chains, beta)


def uniform_random_ops_batch(rng, n_flav: int, beta: float, n_chains: int, n_ops_lo: int,
                             n_ops_hi: int) -> Batch:
    """Operator codes drawn uniformly with no structure (many strings do not
    survive; used for zero-sector and odd-length edge cases)."""
    chains = []
    for _ in range(n_chains):
        n = int(rng.integers(n_ops_lo, n_ops_hi + 1))
        chains.append((_sorted_taus(rng, n, beta),
                       rng.integers(0, 2 * n_flav, size=n).astype(np.int32)))
    return _pack(chains, beta)

"""The pair-move input generator (workloads.pair_move): every move keeps the
operators of each flavour alternating between creation and annihilation
(so the configuration stays Pauli-allowed), times stay sorted, distinct and
in [0, beta), and insertions and removals both occur."""
import numpy as np

from paper_2010_08482_gb300 import workloads as w


def alternating(tau, op, n_flav):
    for f in range(n_flav):
        ty = op[op // 2 == f] % 2
        if len(ty) % 2 or np.any(ty[1:] == ty[:-1]):
            return False
    return True


def test_pair_moves_keep_alternation():
    rng = np.random.default_rng(4)
    b = w.batch_t2g(4)
    tau, op = (np.asarray(x) for x in b.chain(0))
    assert alternating(tau, op, 6)
    kinds = set()
    for _ in range(300):
        mv = w.pair_move(rng, tau, op, 6, b.beta)
        kinds.add(mv[0])
        tau, op = w.apply_pair_move(mv, tau, op)
        assert np.all(np.diff(tau) > 0) and tau.min() >= 0 and tau.max() < b.beta
        assert alternating(tau, op, 6)
    assert kinds == {"ins", "rem"}

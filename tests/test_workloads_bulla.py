"""CPU checks of the input construction for the static improved estimator
(workloads.bulla_sequences): one sequence per annihilator, that operator
replaced by its Bulla code and nothing else changed; empty chains and chains
without annihilators produce no sequence."""
import numpy as np

from paper_2010_08482_gb300 import workloads as w


def brute(batch, n_flav):
    seqs, chain, pos = [], [], []
    for c in range(batch.n_chains):
        tau, ops = batch.chain(c)
        for p, a in enumerate(ops):
            if a < 2 * n_flav and a % 2 == 0:
                o = np.array(ops).copy()
                o[p] = 2 * n_flav + a // 2
                seqs.append((np.array(tau), o))
                chain.append(c)
                pos.append(p)
    return seqs, chain, pos


def test_bulla_sequences_match_brute_force():
    rng = np.random.default_rng(4)
    b = w.random_batch(rng, 6, 50.0, 40, 0, 9)
    bu, chain, pos = w.bulla_sequences(b, 6)
    seqs, c_ref, p_ref = brute(b, 6)
    assert bu.n_chains == len(seqs) and bu.beta == b.beta
    assert list(chain) == c_ref and list(pos) == p_ref
    assert chain.dtype == np.int32 and pos.dtype == np.int32 and bu.op.dtype == np.int32
    for i, (t, o) in enumerate(seqs):
        t2, o2 = bu.chain(i)
        assert np.array_equal(t2, t) and np.array_equal(o2, o)


def test_bulla_sequences_edge_cases():
    # an empty chain, a chain of creators only, a chain with one annihilator
    b = w.Batch(beta=1.0, offsets=np.array([0, 0, 2, 4], np.int32),
                tau=np.array([0.1, 0.2, 0.3, 0.4]), op=np.array([1, 3, 1, 0], np.int32))
    bu, chain, pos = w.bulla_sequences(b, 2)
    assert bu.n_chains == 1 and list(chain) == [2] and list(pos) == [1]
    t, o = bu.chain(0)
    assert list(o) == [1, 4] and np.array_equal(t, [0.3, 0.4])
    empty = w.Batch(beta=1.0, offsets=np.array([0], np.int32), tau=np.zeros(0), op=np.zeros(0, np.int32))
    bu, chain, pos = w.bulla_sequences(empty, 2)
    assert bu.n_chains == 0 and len(chain) == 0 and len(bu.op) == 0

"""Writes tests/golden/d5_oracle.json: FP64 oracle traces of the chains of the
seeded d-shell workload (by default all 1024; 5 orbitals, Slater-Condon
U = 8, J = 1, real crystal field, beta = 40), with, per chain, the per-sector terms (for the
cancellation rule of the comparison) and the chain's float64 perturbation
spread: the largest relative change of w between the right-to-left product
and the left-to-right product, the product split in the middle, and the
product on blocks perturbed by one unit in the last place.  That spread
over 2^-53 is the chain's measured condition number, which sets how far a
reduced-precision evaluation may stray.  Calls only the oracle (the
perturbed blocks come from the oracle model, through tests/parity.py) and
the seeded input generator; the GPU tests compare against these stored
values because the oracle takes minutes for a thousand d-shell chains.

    python tests/golden/make_d5_oracle.py [n_chains] [processes]
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))


def part(args):
    lo, hi = args
    import parity
    from oracle import atom
    from paper_2010_08482_gb300 import workloads as w
    m = atom.Model(w.model_d5())
    b = w.batch_d5()
    res = parity.oracle_chain_results(m, b, range(lo, hi))
    out = []
    for c in range(lo, hi):
        r = res[c]
        ph = complex(r["phase"]) if r["log_abs"] != -math.inf else 0j
        out.append({"chain": c, "n_ops": int(b.offsets[c + 1] - b.offsets[c]), "log_abs": r["log_abs"],
                    "phase": [ph.real, ph.imag],
                    "per_q0": {str(q): [v[0], complex(v[1]).real, complex(v[1]).imag] for q, v in r["per_q0"].items()},
                    "noise": r.get("noise", 0.0)})
    return out


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count()
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(part, [(lo, min(n, lo + 8)) for lo in range(0, n, 8)])
    chains = [c for p in parts for c in p]
    with open(os.path.join(HERE, "d5_oracle.json"), "w") as f:
        json.dump({"model": "d5", "n_chains": n, "chains": chains}, f, indent=0)
    print(f"{n} chains in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()

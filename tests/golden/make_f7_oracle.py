"""Writes tests/golden/f7_oracle.json: FP64 oracle traces of the first chains
of the seeded f-shell workload (7 orbitals, SOC 0.3, complex CF, N in {4,5,6},
sectors 1001 / 2002 / 3003), the oracle's sector energies (so that a test
can measure how far another eigensolver's energies lie from them) and, per
chain, the relative spread between the two association orders of the
product (the chain's own float64 rounding spread).  Calls only the oracle
(and the seeded input generator); the GPU tests compare against these stored
values because one f-shell chain takes the oracle one to two minutes.

    python tests/golden/make_f7_oracle.py [n_chains]
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import atom  # noqa: E402
from oracle import trace as OT  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    t0 = time.time()
    m = atom.Model(w.model_f7())
    b = w.batch_f7()
    out = {"model": "f7", "mu": m.mu, "E_gs": m.E_gs, "dims": [int(d) for d in m.dims],
           "E": [[float(x) for x in e] for e in m.E], "chains": []}
    for c in range(n):
        tau, ops = b.chain(c)
        r = OT.trace_chain(m, tau, ops, beta=b.beta)
        left = OT.trace_chain_left(m, tau, ops, beta=b.beta)
        spread = abs(complex(left["phase"]) * math.exp(left["log_rel"] - r["log_rel"]) - complex(r["phase"]))
        out["chains"].append({"chain": c, "n_ops": len(ops), "log_abs": r["log_abs"],
                              "phase": [float(complex(r["phase"]).real), float(complex(r["phase"]).imag)],
                              "q0": sorted(int(q) for q in r["per_q0"]), "noise": spread})
        print(c, len(ops), r["log_abs"], time.time() - t0, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "f7_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

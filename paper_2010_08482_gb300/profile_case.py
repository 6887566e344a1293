"""A small large-block case for profilers.

The f-shell benchmark impurity (N in {4, 5, 6}, blocks up to 3003) keeps
about 11 GB of operands on the device, too much for multi-pass profiler
captures that save and restore device memory.  This case uses the same
shell with the window N in {4, 5} (blocks 1001 / 2002, 4.7 GB on the device)
and the full window's particle-hole chemical potential, with two chains of
80 operators whose particle number alternates between 4 and 5, and
evaluates them a few times:

    python -m paper_2010_08482_gb300.profile_case bf16x3     # or tf32x3, tf32, fp64, f32x2
"""
import sys

import numpy as np

from . import ctq
from . import workloads as w

# particle-hole symmetric chemical potential of the N in {4, 5, 6} f shell
# (E_gs(4) = E_gs(6)), as the library computes it for that window
MU_F7 = 18.37060157531069


def main(argv=None):
    import torch
    argv = sys.argv[1:] if argv is None else argv
    prec = {"bf16x3": ctq.BF16X3, "tf32x3": ctq.TF32X3, "tf32": ctq.TF32, "fp64": ctq.FP64,
            "f32x2": ctq.F32X2}[argv[0] if argv else "bf16x3"]
    reps = int(argv[1]) if len(argv) > 1 else 4
    p = w.model_f7()
    p.n_min, p.n_max, p.mu = 4, 5, MU_F7
    imp = ctq.build_impurity(p, device=0)
    rng = np.random.default_rng(7)
    batch = w._pack([w.g2_chain(rng, p.n_flav, 40, p.beta, width=1) for _ in range(2)], p.beta)
    db = ctq.DeviceBatch(batch)
    ev = ctq.TraceEvaluator(imp, batch.n_chains, db.max_ops, precision=prec)
    for _ in range(reps):
        ev(db)
    torch.cuda.synchronize()
    r = ev.results()
    free, total = torch.cuda.mem_get_info()
    print("dims", imp.sectors()[0].tolist(), "status", r["status"].tolist(), "log_abs", r["log_abs"].tolist(),
          "device GB in use", round((total - free) / 1e9, 2))


if __name__ == "__main__":
    main()

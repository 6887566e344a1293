"""Partition-space CT-HYB sampling with the GPU local trace
(paper_2010_08482_gb300.partition) against exact diagonalisation of the
single-band Hubbard impurity with three bath levels of Sec. 4.1 (eps = -D/2,
0, D/2; V = D = 1; U = 4; eps_f = -U/2; beta = 10): mean expansion order,
the Green function from Eq. PGreenEstimator in imaginary-time bins, the
double occupancy from the reduced density matrix (Eq.
ImpurityDensityMatrix), the sign, and lazy early rejects on the GPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ed  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import partition as P  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu

BETA, U = 10.0, 4.0
EPS, V = [-0.5, 0.0, 0.5], [1.0, 1.0, 1.0]


@pytest.fixture(scope="module")
def run():
    p = w.model_atom1(U=U, mu=U / 2, beta=BETA)
    imp = ctq.build_impurity(p, device=0)
    s = P.PartitionSampler(imp, EPS, V, BETA, n_chains=256, seed=2010, max_ops=256, n_bins=20)
    s.run(1500, n_burn=400)
    rho = s.density_matrices()
    x = ed.ImpurityED(p, U / 2, EPS, V, BETA)
    return s, s.estimates(), rho, x


def test_mean_order_and_sign(run):
    s, est, _, x = run
    k, ke = est["order"]
    print(f"<k> = {k:.4f} +- {ke:.4f} (ED {x.mean_order():.4f}); acceptance {est['acceptance']:.3f}, "
          f"early rejects {est['early_rejects']:.3f}")
    assert abs(k - x.mean_order()) <= 5 * ke
    assert est["sign"][0] == 1.0
    assert est["early_rejects"] > 0.01  # the GPU rejected proposals on their bounds


def test_green_function_bins(run):
    s, est, _, x = run
    g, ge = est["green"]
    nb = s.n_bins
    worst = 0.0
    for b in range(nb):
        ref = x.green_bin(0, b * BETA / nb, (b + 1) * BETA / nb)
        got = 0.5 * (g[0][b] + g[1][b])
        err = 0.5 * math.hypot(ge[0][b], ge[1][b])
        worst = max(worst, abs(got - ref) / err)
        assert abs(got - ref) <= 5 * err + 2e-4, (b, got, err, ref)
    print(f"G(tau) in {nb} bins: worst deviation {worst:.2f} standard errors")


def test_density_matrix_double_occupancy(run):
    """Sector occupations of the reduced density matrix of the last
    configurations (one sample per chain): <N> and the doubly occupied
    sector's weight against ED, within 5 standard errors across chains."""
    s, _, rho, x = run
    dims, N, _, _ = s.sectors
    tot = np.array([sum(float(np.trace(r[q]).real) for q in r) for r in rho])
    assert np.allclose(tot, 1.0, atol=1e-10)
    n_avg = np.array([sum(N[q] * float(np.trace(r[q]).real) for q in r) for r in rho])
    d_avg = np.array([sum(float(np.trace(r[q]).real) for q in r if N[q] == 2) for r in rho])
    se = d_avg.std(ddof=1) / math.sqrt(len(d_avg))
    print(f"<N> = {n_avg.mean():.4f}, D = {d_avg.mean():.4f} +- {se:.4f} (ED {x.double_occupancy():.4f})")
    assert abs(n_avg.mean() - 1.0) <= 5 * n_avg.std(ddof=1) / math.sqrt(len(n_avg)) + 1e-3
    assert abs(d_avg.mean() - x.double_occupancy()) <= 5 * se + 1e-3

"""Pins of the oracle's density-matrix estimator (oracle/observables.py,
Eq. ImpurityDensityMatrix) against facts fixed independently of it:

* no operators: the estimator is the thermal atomic density matrix
  e^{-beta H_loc} / Z (closed form);
* every configuration: Tr rho^C = 1 (the propagation intervals tile [0, beta));
* the particle number: Tr rho^C N = (1/beta) sum_q0 (w_q0 / w) sum_i D_i N(q_i),
  the time average of N along each sector string (N is a quantum number);
* brute force: Gauss-Legendre quadrature of Tr[T ... |v><u|(tau) ...] / w over
  the full Fock space with dense matrix exponentials (no sectors, no
  eigenbasis blocks, no closed-form integral), for the 2- and 3-orbital models.
"""
import math

import numpy as np
import pytest

from oracle import atom
from oracle import observables as OB
from oracle import trace as OT
from paper_2010_08482_gb300 import workloads as w


@pytest.fixture(scope="module")
def m2():
    return atom.Model(w.model_hubbard2())


@pytest.fixture(scope="module")
def m3():
    return atom.Model(w.model_t2g())


def live_chains(m, rng, n, k_lo, k_hi):
    out = []
    while len(out) < n:
        b = w.random_batch(rng, m.n_flav, m.beta, 1, k_lo, k_hi)
        tau, ops = b.chain(0)
        if OT.trace_chain(m, tau, ops)["log_abs"] != -math.inf:
            out.append((tau, ops))
    return out


@pytest.mark.parametrize("which", ["m2", "m3"])
def test_empty_configuration_is_thermal(which, request):
    m = request.getfixturevalue(which)
    rho, _ = OB.density_matrix_chain(m, [], [])
    th = OB.thermal_density_matrix(m)
    for q in range(m.n_sec):
        np.testing.assert_allclose(rho[q], th[q], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("which", ["m2", "m3"])
def test_trace_is_one(which, request):
    m = request.getfixturevalue(which)
    for tau, ops in live_chains(m, np.random.default_rng(3), 12, 1, 8):
        rho, wv = OB.density_matrix_chain(m, tau, ops)
        assert wv != 0
        tr = sum(np.trace(rho[q]) for q in range(m.n_sec))
        assert abs(tr - 1.0) < 1e-10


@pytest.mark.parametrize("which", ["m2", "m3"])
def test_particle_number_is_time_average(which, request):
    m = request.getfixturevalue(which)
    for tau, ops in live_chains(m, np.random.default_rng(5), 10, 1, 8):
        rho, _ = OB.density_matrix_chain(m, tau, ops)
        got = sum(m.N[q] * np.trace(rho[q]) for q in range(m.n_sec))
        r = OT.trace_chain(m, tau, ops)
        n = len(ops)
        bounds = [0.0] + list(tau) + [m.beta]
        expect, wsum = 0.0, 0.0
        for q0, (lw, ph) in r["per_q0"].items():
            if lw == -math.inf:
                continue
            path = OT.walk(m, ops, q0)
            wq = ph * math.exp(lw - r["log_abs"])  # w_q0 / |w|
            tavg = sum((bounds[i + 1] - bounds[i]) * m.N[path[i] if i < n else q0] for i in range(n + 1)) / m.beta
            expect += wq * tavg
            wsum += wq
        expect /= wsum
        assert abs(got - expect) < 1e-10 * max(1.0, abs(expect))


def _fock_setup(m):
    p = m.params
    H = atom.full_hamiltonian(p, m.mu)
    n_f = m.n_flav
    mats = {2 * f + dag: atom.full_op_matrix(n_f, f, dag) for f in range(n_f) for dag in (0, 1)}
    U = []
    for q in range(m.n_sec):
        Uq = np.zeros((1 << n_f, m.dims[q]), dtype=np.complex128)
        Uq[m.states[q], :] = m.V[q]
        U.append(Uq)
    return H, mats, U


@pytest.mark.parametrize("which,n_chains", [("m2", 5), ("m3", 2)])
def test_against_full_space_quadrature(which, n_chains, request):
    m = request.getfixturevalue(which)
    H, mats, U = _fock_setup(m)
    for tau, ops in live_chains(m, np.random.default_rng(11), n_chains, 1, 3):
        rho, _ = OB.density_matrix_chain(m, tau, ops)
        ref, _ = OB.density_matrix_full_space(H, mats, tau, ops, m.beta, U, n_quad=32)
        scale = max(np.abs(ref[q]).max() for q in range(m.n_sec))
        for q in range(m.n_sec):
            np.testing.assert_allclose(rho[q], ref[q], rtol=0, atol=1e-9 * scale)


def test_kernel_matrix_closed_form():
    """K(a, b, D) against direct quadrature, including a == b."""
    Ea = np.array([0.0, 0.3, 1.7])
    K = OB.kernel_matrix(Ea, Ea, 2.5)
    x, wq = np.polynomial.legendre.leggauss(40)
    s = 0.5 * 2.5 * (x + 1)
    for u in range(3):
        for v in range(3):
            ref = 0.5 * 2.5 * np.sum(wq * np.exp(-s * Ea[u] - (2.5 - s) * Ea[v]))
            assert abs(K[u, v] - ref) < 1e-13


def test_kernel_matrix_nearly_degenerate_levels():
    """Levels that differ by rounding (1e-15) give the degenerate limit
    D e^{-D a} to full precision (no cancellation in the difference quotient)."""
    a = 0.7
    K = OB.kernel_matrix(np.array([a, a + 3.5e-15]), np.array([a, a + 3.5e-15]), 3.0)
    ref = 3.0 * math.exp(-3.0 * a)
    assert np.all(np.abs(K - ref) <= 1e-13 * ref)

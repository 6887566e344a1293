"""Pins for oracle.ed (exact diagonalisation of impurity + discrete bath):
the non-interacting limit against the single-particle problem, the atomic
limit against its closed form, the Green-function sum rule, the bin average,
and the hybridisation function against its Matsubara sum."""
import math

import numpy as np
import pytest

from oracle import ed
from paper_2010_08482_gb300 import workloads as w

BETA = 10.0
EPS = [-0.5, 0.0, 0.5]
V = [1.0, 1.0, 1.0]


def single_particle(eps_d, eps, V):
    """Eigenvalues and impurity weights |phi_j(imp)|^2 of the one-particle
    hopping matrix [[eps_d, V], [V, diag(eps)]]."""
    n = len(eps)
    h = np.zeros((n + 1, n + 1))
    h[0, 0] = eps_d
    h[0, 1:] = V
    h[1:, 0] = V
    h[1:, 1:] = np.diag(eps)
    e, v = np.linalg.eigh(h)
    return e, v[0] ** 2, v


def test_noninteracting_limit_matches_single_particle():
    """U = 0: G(tau) = sum_j |phi_j(imp)|^2 (-e^{-e_j tau} / (1 + e^{-beta e_j})),
    <n> = sum_j |phi_j(imp)|^2 n_F(e_j), <H_hyb> = 2 sum_l V_l <c^+ b_l>."""
    mu = 0.3
    p = w.model_atom1(U=0.0, mu=mu, beta=BETA)
    x = ed.ImpurityED(p, mu, EPS, V, BETA)
    e, wts, vec = single_particle(-mu, EPS, V)
    nF = 1.0 / (np.exp(BETA * e) + 1.0)
    for f in (0, 1):
        assert x.occupation(f) == pytest.approx(float(np.sum(wts * nF)), abs=1e-12)
    taus = np.array([0.1, 1.3, 5.0, 9.7])
    g_ref = np.array([float(np.sum(wts * (-np.exp(-e * t) / (1.0 + np.exp(-BETA * e))))) for t in taus])
    for f in (0, 1):
        assert np.allclose(x.green(f, taus), g_ref, atol=1e-12)
    # one-particle density matrix: <c^+_i c_j> = sum_k v_ik v_jk n_F(e_k)
    rho = (vec * nF) @ vec.T
    e_hyb = 2 * 2 * sum(V[l] * rho[0, l + 1] for l in range(len(EPS)))  # two flavours, c^+b + b^+c
    assert x.hybridisation_energy() == pytest.approx(e_hyb, abs=1e-12)
    assert x.mean_order() == pytest.approx(-0.5 * BETA * e_hyb, abs=1e-12)


def test_atomic_limit_matches_closed_form():
    """V = 0: the impurity decouples; G(tau) = -[e^{-tau e} + e^{-beta e}
    e^{-tau (e + U)}] / Z_atom, Z_atom = 1 + 2 e^{-beta e} + e^{-beta (2 e + U)},
    e = -mu (the Hubbard atom)."""
    U, mu = 3.0, 1.2
    p = w.model_atom1(U=U, mu=mu, beta=BETA)
    x = ed.ImpurityED(p, mu, EPS, [0.0, 0.0, 0.0], BETA)
    e = -mu
    Z = 1 + 2 * math.exp(-BETA * e) + math.exp(-BETA * (2 * e + U))
    for t in (0.2, 2.5, 7.0):
        ref = -(math.exp(-t * e) + math.exp(-BETA * e) * math.exp(-t * (e + U))) / Z
        assert x.green(0, [t])[0] == pytest.approx(ref, rel=1e-12)
    assert x.double_occupancy() == pytest.approx(math.exp(-BETA * (2 * e + U)) / Z, rel=1e-12)
    assert x.hybridisation_energy() == 0.0 and x.mean_order() == 0.0


def test_green_sum_rule_and_bin_average():
    """G(0+) + G(beta-) = -<c c^+> - <c^+ c> = -1; the analytic bin average
    equals the numerical average of G over the bin."""
    U = 4.0
    p = w.model_atom1(U=U, mu=U / 2, beta=BETA)
    x = ed.ImpurityED(p, U / 2, EPS, V, BETA)
    g = x.green(0, [1e-12, BETA - 1e-12])
    assert g[0] + g[1] == pytest.approx(-1.0, abs=1e-9)
    a, b = 2.0, 2.5
    t = np.linspace(a, b, 2001)
    num = np.trapezoid(x.green(0, t), t) / (b - a)
    assert x.green_bin(0, a, b) == pytest.approx(num, rel=1e-7)
    # particle-hole symmetric point: <n> = 1/2 per flavour, G(tau) = G(beta - tau)
    assert x.occupation(0) == pytest.approx(0.5, abs=1e-12)
    assert x.green(0, [1.7])[0] == pytest.approx(x.green(0, [BETA - 1.7])[0], rel=1e-10)


def test_hybridisation_function_matches_matsubara_sum():
    """Delta(tau) = T sum_n e^{-i nu_n tau} sum_l V_l^2 / (i nu_n - eps_l)
    (Eq. hybridization), summed numerically with the 1 / (i nu) tail taken
    out (its transform is -1/2 on (0, beta))."""
    eps, Vl = [-0.7, 0.4], [0.8, 1.3]
    n = np.arange(-400000, 400000)
    nu = (2 * n + 1) * math.pi / BETA
    for t in (0.3, 4.1, 9.2):
        s = sum(v * v * (1.0 / (1j * nu - e) - 1.0 / (1j * nu)) for e, v in zip(eps, Vl))
        val = float(np.real(np.sum(np.exp(-1j * nu * t) * s))) / BETA - 0.5 * sum(v * v for v in Vl)
        assert ed.hybridisation_function(eps, Vl, BETA, np.array([t]))[0] == pytest.approx(val, abs=2e-5)
    # antiperiodic: Delta(tau - beta) = -Delta(tau)
    t = np.array([0.5, 3.0])
    assert np.allclose(ed.hybridisation_function(eps, Vl, BETA, t - BETA),
                       -ed.hybridisation_function(eps, Vl, BETA, t))

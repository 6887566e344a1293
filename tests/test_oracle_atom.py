"""Pins for oracle.atom: each check is fixed by mathematics or a textbook table,
not by re-running the oracle's own formula."""
import math

import numpy as np
import pytest

from oracle import atom
from paper_2010_08482_gb300 import workloads as w


def same_levels(got, exp, tol=1e-9):
    """Multiplet lists [(energy, degeneracy)] agree level by level."""
    exp = sorted(exp)
    return (len(got) == len(exp) and all(g[1] == e[1] for g, e in zip(got, exp))
            and all(abs(g[0] - e[0]) <= tol * max(1.0, abs(e[0])) for g, e in zip(got, exp)))


def multiplets(E, tol=1e-8):
    E = np.sort(np.asarray(E))
    out, i = [], 0
    while i < len(E):
        j = i
        while j < len(E) and E[j] - E[i] < tol:
            j += 1
        out.append((float(E[i]), j - i))
        i = j
    return out


# ---------------------------------------------------------------- Fock space

@pytest.mark.parametrize("n_f", [1, 2, 3, 4, 5, 6])
def test_canonical_anticommutators(n_f):
    """{c_i, c_j^+} = delta_ij, {c_i, c_j} = 0, exhaustively (Jordan-Wigner signs)."""
    dim = 1 << n_f
    c = [atom.full_op_matrix(n_f, i, 0) for i in range(n_f)]
    cd = [atom.full_op_matrix(n_f, i, 1) for i in range(n_f)]
    eye = np.eye(dim)
    for i in range(n_f):
        assert np.array_equal(cd[i], c[i].T)
        for j in range(n_f):
            assert np.array_equal(c[i] @ cd[j] + cd[j] @ c[i], eye if i == j else 0 * eye)
            assert not np.any(c[i] @ c[j] + c[j] @ c[i])


def test_apply_string_matches_matrix_products():
    n_f = 4
    c = [atom.full_op_matrix(n_f, i, 0) for i in range(n_f)]
    cd = [atom.full_op_matrix(n_f, i, 1) for i in range(n_f)]
    ops = ((3, 1), (0, 1), (2, 0), (1, 0))
    M = cd[3] @ cd[0] @ c[2] @ c[1]
    states = np.arange(1 << n_f)
    ok, sign, new = atom.apply_string(states, ops)
    R = np.zeros_like(M)
    R[new[ok], states[ok]] = sign[ok]
    assert np.array_equal(R, M)


# ---------------------------------------------------------------- Kanamori

def _kanamori_params(n_orb, U, J, mu=0.0):
    return w.ModelParams("k", n_orb=n_orb, l=0, interaction="kanamori", U=U, J=J, beta=1.0,
                         mu=mu, n0=n_orb)


def _spectrum_by_N(p, N):
    labels, states = atom.sector_states(p)
    E = []
    for lab, st in zip(labels, states):
        if sum(lab) == N:
            E.append(np.linalg.eigvalsh(atom.sector_hamiltonian(st, atom.hamiltonian_terms(p, 0.0))))
    return np.concatenate(E)


def test_kanamori_two_orbital_multiplets():
    """2 orbitals, N=2: U-3J (x3), U-J (x2), U+J (x1) (atomic Kanamori, textbook)."""
    U, J = 4.0, 0.5
    got = multiplets(_spectrum_by_N(_kanamori_params(2, U, J), 2))
    assert same_levels(got, [(U - 3 * J, 3), (U - J, 2), (U + J, 1)])


def test_kanamori_three_orbital_multiplets():
    """3 orbitals: N=2: U-3J (x9), U-J (x5), U+2J (x1);
    N=3: 3U-9J (x4), 3U-6J (x10), 3U-4J (x6)."""
    U, J = 5.0, 0.7
    p = _kanamori_params(3, U, J)
    assert same_levels(multiplets(_spectrum_by_N(p, 2)), [(U - 3 * J, 9), (U - J, 5), (U + 2 * J, 1)])
    assert same_levels(multiplets(_spectrum_by_N(p, 3)),
                       [(3 * U - 9 * J, 4), (3 * U - 6 * J, 10), (3 * U - 4 * J, 6)])


def test_kanamori_equals_orbital_tensor_form():
    """The operator-form Kanamori equals 1/2 sum V_ijkl c+_i c+_j c_l c_k with
    V_aaaa = U, V_abab = U-2J, V_abba = J, V_aabb = J (fixes the U_ijkl index
    order, Eq. ImpurityHamiltonian: U_ijkl = <ij|V|lk>)."""
    n_orb, U, J = 3, 5.0, 0.7
    V = np.zeros((n_orb,) * 4)
    for a in range(n_orb):
        V[a, a, a, a] = U
        for b in range(n_orb):
            if a != b:
                V[a, b, a, b] = U - 2 * J
                V[a, b, b, a] = J
                V[a, a, b, b] = J
    p = _kanamori_params(n_orb, U, J)
    labels, states = atom.sector_states(p)
    for st in states:
        H1 = atom.sector_hamiltonian(st, atom.kanamori_terms(n_orb, U, J))
        H2 = atom.sector_hamiltonian(st, atom.orbital_tensor_terms(n_orb, V))
        assert np.allclose(H1, H2, atol=1e-13)


# ---------------------------------------------------------------- Slater-Condon

def test_wigner_3j_matches_sympy():
    sym = pytest.importorskip("sympy.physics.wigner")
    for l in (1, 2, 3):
        for k in range(0, 2 * l + 1):
            for m in range(-l, l + 1):
                for mp in range(-l, l + 1):
                    ref = float(sym.wigner_3j(l, k, l, -m, m - mp, mp))
                    assert atom.wigner_3j(l, k, l, -m, m - mp, mp) == pytest.approx(ref, abs=1e-14)


def _two_electron_levels(l, F):
    T = atom.real_harmonics_T(l)
    Vr = atom.to_real_basis_tensor(atom.slater_orbital_tensor(l, F), T)
    assert np.abs(Vr.imag).max() < 1e-12, "real-harmonic interaction must be real"
    p = w.ModelParams("x", n_orb=2 * l + 1, l=l, interaction="slater", U=F[0], J=0.0, beta=1.0,
                      mu=0.0, n0=2, sector_mode="n", n_min=2, n_max=2)
    _, states = atom.sector_states(p)
    H = atom.sector_hamiltonian(states[0], atom.orbital_tensor_terms(2 * l + 1, Vr))
    return multiplets(np.linalg.eigvalsh(H))


def test_slater_d2_terms_condon_shortley():
    """d^2 term energies (Condon-Shortley F_2 = F^2/49, F_4 = F^4/441):
    1S F0+14F2+126F4, 3P F0+7F2-84F4, 1D F0-3F2+36F4, 3F F0-8F2-9F4, 1G F0+4F2+F4."""
    F0, F2, F4 = 0.3, 1.3, 0.7
    got = _two_electron_levels(2, {0: F0, 2: 49 * F2, 4: 441 * F4})
    exp = sorted([(F0 + 14 * F2 + 126 * F4, 1), (F0 + 7 * F2 - 84 * F4, 9), (F0 - 3 * F2 + 36 * F4, 5),
                  (F0 - 8 * F2 - 9 * F4, 21), (F0 + 4 * F2 + F4, 9)])
    assert same_levels(got, exp)


def test_slater_f2_terms_condon_shortley():
    """f^2 term energies (F_2 = F^2/225, F_4 = F^4/1089, F_6 = 25 F^6/184041):
    3P, 3F, 3H, 1S, 1D, 1G, 1I."""
    F0, F2, F4, F6 = 0.0, 1.1, 0.37, 0.013
    got = _two_electron_levels(3, {0: F0, 2: 225 * F2, 4: 1089 * F4, 6: 184041 / 25 * F6})
    exp = sorted([
        (F0 + 45 * F2 + 33 * F4 - 1287 * F6, 9), (F0 - 10 * F2 - 33 * F4 - 286 * F6, 21),
        (F0 - 25 * F2 - 51 * F4 - 13 * F6, 33), (F0 + 60 * F2 + 198 * F4 + 1716 * F6, 1),
        (F0 + 19 * F2 - 99 * F4 + 715 * F6, 5), (F0 - 30 * F2 + 97 * F4 + 78 * F6, 9),
        (F0 + 25 * F2 + 9 * F4 + F6, 13)])
    assert same_levels(got, exp)


def test_real_harmonics_unitary():
    for l in (1, 2, 3):
        T = atom.real_harmonics_T(l)
        assert np.allclose(T @ T.conj().T, np.eye(2 * l + 1), atol=1e-15)


def _ground_degeneracy(p, N, tol=1e-8):
    labels, states = atom.sector_states(p)
    terms = atom.hamiltonian_terms(p, 0.0)
    E = np.concatenate([np.linalg.eigvalsh(atom.sector_hamiltonian(st, terms))
                        for lab, st in zip(labels, states) if sum(lab) == N])
    return int(np.sum(E < E.min() + tol))


def test_hund_ground_states_d_shell():
    """Slater d shell, no CF: N=5 ground 6S (x6), N=4 ground 5D (x25)."""
    p = w.ModelParams("d", n_orb=5, l=2, interaction="slater", U=8.0, J=1.0, beta=1.0, mu=0.0, n0=5,
                      sector_mode="n", n_min=4, n_max=5)
    assert _ground_degeneracy(p, 5) == 6
    assert _ground_degeneracy(p, 4) == 25


@pytest.mark.slow
def test_hund_ground_states_f_shell_with_soc():
    """f shell with SOC, no CF: ground multiplets 2J+1 = 9 (N=4, 5I4),
    6 (N=5, 6H5/2), 1 (N=6, 7F0)."""
    p = w.ModelParams("f", n_orb=7, l=3, interaction="slater", U=4.5, J=0.5, beta=1.0, mu=0.0,
                      n0=5, soc_xi=0.3, sector_mode="n", n_min=4, n_max=6)
    assert _ground_degeneracy(p, 4) == 9
    assert _ground_degeneracy(p, 5) == 6
    assert _ground_degeneracy(p, 6) == 1


def test_soc_one_body_spectrum():
    """xi l.s: j = l+1/2 at xi l/2 (2l+2 states), j = l-1/2 at -xi (l+1)/2 (2l states)."""
    for l in (1, 2, 3):
        xi = 0.3
        e = np.linalg.eigvalsh(atom.soc_complex(l, xi))
        assert same_levels(multiplets(e), [(-xi * (l + 1) / 2, 2 * l), (xi * l / 2, 2 * l + 2)])


# ---------------------------------------------------------------- sectors and eigenbasis

@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_sector_spectra_union_is_full_spectrum(name, models):
    m = models(name)
    p = m.params
    H = atom.full_hamiltonian(p, m.mu)
    full = np.linalg.eigvalsh(H if m.is_complex else H.real)
    assert np.allclose(np.sort(full), m.spectrum(), atol=1e-10)


@pytest.mark.parametrize("name", ["hubbard2", "t2g", "d5"])
def test_eigenbasis_residual_and_orthonormality(name, models):
    m = models(name)
    terms = atom.hamiltonian_terms(m.params, m.mu)
    for q in range(m.n_sec):
        H = atom.sector_hamiltonian(m.states[q], terms)
        V = m.V[q]
        assert np.allclose(V.conj().T @ V, np.eye(m.dims[q]), atol=1e-12)
        assert np.abs(H @ V - V * m.E[q][None, :]).max() < 1e-11


@pytest.mark.parametrize("name,n0", [("t2g", 3), ("d5", 5)])
def test_particle_hole_symmetric_mu(name, n0, models):
    m = models(name)
    egs = {}
    for q in range(m.n_sec):
        egs[m.N[q]] = min(egs.get(m.N[q], np.inf), m.E[q][0])
    assert egs[n0 - 1] == pytest.approx(egs[n0 + 1], abs=1e-10)


def test_sector_counts(models):
    """(N_dn, N_up) sectors: 9 / 16 / 36 with largest blocks 4 / 9 / 100."""
    for name, ns, dmax in [("hubbard2", 9, 4), ("t2g", 16, 9), ("d5", 36, 100)]:
        m = models(name)
        assert m.n_sec == ns and max(m.dims) == dmax


def test_blocks_are_partial_isometries(models):
    """F_alpha(q) restricts c_alpha, whose nonzero singular values are 1."""
    m = models("t2g")
    for (alpha, q), Fb in m.F.items():
        sv = np.linalg.svd(Fb, compute_uv=False)
        assert np.all((np.abs(sv - 1) < 1e-12) | (np.abs(sv) < 1e-12))


def test_sector_map_unique_and_charge_conserving(models):
    m = models("t2g")
    for alpha in range(2 * m.n_flav):
        dag = alpha % 2
        for q in range(m.n_sec):
            qp = m.s[alpha, q]
            if qp >= 0:
                assert m.N[qp] == m.N[q] + (1 if dag else -1)


def test_eigh_by_components_is_an_eigendecomposition():
    """Block-diagonal input (hidden components permuted together): the result
    diagonalises H, is orthonormal, and keeps exact zeros across components."""
    rng = np.random.default_rng(3)
    a = rng.normal(size=(3, 3))
    b = rng.normal(size=(4, 4))
    H = np.zeros((7, 7))
    H[:3, :3] = a + a.T
    H[3:, 3:] = b + b.T
    perm = rng.permutation(7)
    H = H[np.ix_(perm, perm)]
    E, V = atom.eigh_by_components(H)
    assert np.allclose(V.T @ V, np.eye(7), atol=1e-14)
    assert np.allclose(H @ V, V * E[None, :], atol=1e-13)
    assert np.allclose(E, np.linalg.eigvalsh(H), atol=1e-13)
    for j in range(7):
        orig = perm[np.nonzero(V[:, j])[0]]  # row i of the permuted H is original index perm[i]
        assert np.all(orig < 3) or np.all(orig >= 3)


def test_symmetry_forbidden_string_is_exactly_zero(models):
    """t2g Kanamori conserves every orbital's occupation parity; moving one
    electron between orbitals (c_2 ... c+_0) must give exactly 0."""
    from oracle import trace as OT
    m = models("t2g")
    tau = [0.5, 1.0, 2.0, 3.0, 4.0, 5.0]
    r = OT.trace_chain(m, tau, [11, 10, 8, 4, 1, 9])
    assert r["log_abs"] == -math.inf


@pytest.mark.parametrize("l,U,J", [(2, 8.0, 1.0), (2, 3.0, 0.4), (3, 4.5, 0.5), (3, 6.0, 0.9)])
def test_slater_F_reproduces_average_U_and_J(l, U, J):
    """slater_F pinned through the standard orbital averages of the Slater
    interaction (App. A: F0 = U and J fix the Slater integrals), which any
    reading of (U, J) -> F^k must satisfy:
        U     = (2l+1)^-2        sum_{m,m'} U_{mm'},
        U - J = [2l(2l+1)]^-1    sum_{m,m'} (U_{mm'} - J_{mm'}),
    with U_{mm'} = <m m'|V|m m'> and J_{mm'} = <m m'|V|m' m>.  Averages over
    all orbital pairs are invariant under a unitary change of orbital basis,
    so the complex- and real-harmonic tensors must give the same U and J."""
    V = atom.slater_orbital_tensor(l, atom.slater_F(l, U, J))
    T = atom.real_harmonics_T(l)
    n = 2 * l + 1
    for tensor in (V, atom.to_real_basis_tensor(V, T)):
        Umm = np.array([[tensor[a, b, a, b] for b in range(n)] for a in range(n)])
        Jmm = np.array([[tensor[a, b, b, a] for b in range(n)] for a in range(n)])
        U_avg = Umm.sum() / n ** 2
        UJ_avg = (Umm - Jmm).sum() / (n * (n - 1))
        assert abs(U_avg - U) < 1e-12
        assert abs((U_avg - UJ_avg) - J) < 1e-12

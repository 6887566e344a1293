// Host-side construction of the sector-decomposed impurity.
//
// Follows Sec. 3.2 (phase (1): decompose the Hilbert space into invariant
// spaces, diagonalise them, build the operator matrices in the eigenbasis) and
// Sec. 3.3.1 (sectors by abelian quantum numbers, the unique map
// s_alpha(q) -> q', blocks [F_alpha(q)]_{mn} = <m(q')|c_alpha|n(q)>; the
// paper prints the transposed index order, the trace is unchanged).
//
// H_loc is Eq. ImpurityHamiltonian,
//   H = sum_ij c+_i (t_ij - mu delta_ij) c_j + 1/2 sum_ijkl U_ijkl c+_i c+_j c_k c_l,
// with U_ijkl = <ij|V|lk> (physics-notation matrix elements <ij|V|kl> of the
// interaction, spin-diagonal), from either
//   - Kanamori (named in App. A): <aa|V|aa> = U, <ab|V|ab> = U - 2J,
//     <ab|V|ba> = J, <aa|V|bb> = J (a != b), or
//   - Slater-Condon (App. A): <m1 m2|V|m3 m4> = sum_k F^k c^k(m1,m3) c^k(m4,m2)
//     in complex harmonics, rotated to the real-harmonic product basis of
//     App. A, with F0 = U and J = (F2+F4)/14, F4/F2 = 0.625 (d) or
//     J = (286 F2 + 195 F4 + 250 F6)/6435, F4/F2 = 0.668, F6/F2 = 0.494 (f).
// Spin-orbit coupling xi l.s is added in the same basis; a crystal field is a
// caller-supplied one-body matrix in the flavour basis.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "ctq_internal.h"

namespace ctq {
namespace {

// ------------------------------------------------------------------ Fock space

inline int popc(uint32_t x) { return __builtin_popcount(x); }

// c_i (dag = 0) or c_i^+ (dag = 1) on occupation state st; Jordan-Wigner sign
// (-1)^(number of occupied modes below i).  False if the result is zero.
inline bool apply_op(uint32_t& st, int i, int dag, double& sign) {
  const uint32_t bit = 1u << i;
  const bool occ = (st & bit) != 0;
  if (dag ? occ : !occ) return false;
  if (popc(st & (bit - 1u)) & 1) sign = -sign;
  st ^= bit;
  return true;
}

// A product of up to four operators, written left to right; the rightmost acts first.
struct Term {
  cplx coef;
  int n;
  int f[4];
  int dag[4];
};

inline bool apply_term(const Term& t, uint32_t& st, double& sign) {
  for (int j = t.n - 1; j >= 0; --j)
    if (!apply_op(st, t.f[j], t.dag[j], sign)) return false;
  return true;
}

// ------------------------------------------------------------------ angular algebra

double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;  // exact in double for n <= 18
}

// Wigner 3j symbol (integer arguments) by Racah's formula.
double three_j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  const double delta = factorial(j1 + j2 - j3) * factorial(j1 - j2 + j3) * factorial(-j1 + j2 + j3) /
                       factorial(j1 + j2 + j3 + 1);
  const double norm = std::sqrt(delta * factorial(j1 + m1) * factorial(j1 - m1) * factorial(j2 + m2) *
                                factorial(j2 - m2) * factorial(j3 + m3) * factorial(j3 - m3));
  const int tmin = std::max({0, j2 - j3 - m1, j1 - j3 + m2});
  const int tmax = std::min({j1 + j2 - j3, j1 - m1, j2 + m2});
  double sum = 0.0;
  for (int t = tmin; t <= tmax; ++t) {
    const double den = factorial(t) * factorial(j3 - j2 + t + m1) * factorial(j3 - j1 + t - m2) *
                       factorial(j1 + j2 - j3 - t) * factorial(j1 - t - m1) * factorial(j2 - t + m2);
    sum += ((t & 1) ? -1.0 : 1.0) / den;
  }
  const int ph = j1 - j2 - m3;
  return ((ph % 2 == 0) ? 1.0 : -1.0) * norm * sum;
}

// Gaunt coefficient c^k(l m, l m') = (-1)^m (2l+1) (l k l; 0 0 0) (l k l; -m, m-m', m').
double gaunt(int l, int k, int m, int mp) {
  const double s = (std::abs(m) % 2 == 0) ? 1.0 : -1.0;
  return s * (2 * l + 1) * three_j(l, k, l, 0, 0, 0) * three_j(l, k, l, -m, m - mp, mp);
}

// Real-harmonic rotation (App. A): |r> = sum_m T[r][m] |m>, r and m indexed m + l.
std::vector<cplx> real_harmonics(int l) {
  const int n = 2 * l + 1;
  std::vector<cplx> T(n * n, 0.0);
  const double h = 1.0 / std::sqrt(2.0);
  for (int m = -l; m <= l; ++m) {
    const int r = m + l;
    const double sgn = (std::abs(m) % 2 == 0) ? 1.0 : -1.0;  // (-1)^m
    if (m < 0) {
      T[r * n + (m + l)] += cplx(0.0, h);
      T[r * n + (-m + l)] += cplx(0.0, -h * sgn);
    } else if (m == 0) {
      T[r * n + l] = 1.0;
    } else {
      T[r * n + (-m + l)] += h;
      T[r * n + (m + l)] += h * sgn;
    }
  }
  return T;
}

// Orbital interaction tensor <ab|V|cd> (n^4, index ((a*n+b)*n+c)*n+d).
std::vector<cplx> kanamori_tensor(int n, double U, double J) {
  std::vector<cplx> V(n * n * n * n, 0.0);
  auto at = [&](int a, int b, int c, int d) -> cplx& { return V[((a * n + b) * n + c) * n + d]; };
  for (int a = 0; a < n; ++a) {
    at(a, a, a, a) = U;
    for (int b = 0; b < n; ++b) {
      if (a == b) continue;
      at(a, b, a, b) = U - 2.0 * J;
      at(a, b, b, a) = J;
      at(a, a, b, b) = J;
    }
  }
  return V;
}

std::vector<cplx> slater_tensor(int l, double U, double J) {
  const int n = 2 * l + 1;
  double F[7] = {0, 0, 0, 0, 0, 0, 0};
  F[0] = U;
  if (l == 2) {
    F[2] = 14.0 * J / 1.625;
    F[4] = 0.625 * F[2];
  } else {
    F[2] = 6435.0 * J / (286.0 + 195.0 * 0.668 + 250.0 * 0.494);
    F[4] = 0.668 * F[2];
    F[6] = 0.494 * F[2];
  }
  // complex harmonics
  std::vector<cplx> Vc(n * n * n * n, 0.0);
  for (int m1 = -l; m1 <= l; ++m1)
    for (int m2 = -l; m2 <= l; ++m2)
      for (int m3 = -l; m3 <= l; ++m3) {
        const int m4 = m1 + m2 - m3;
        if (std::abs(m4) > l) continue;
        double v = 0.0;
        for (int k = 0; k <= 2 * l; k += 2) v += F[k] * gaunt(l, k, m1, m3) * gaunt(l, k, m4, m2);
        Vc[(((m1 + l) * n + (m2 + l)) * n + (m3 + l)) * n + (m4 + l)] = v;
      }
  // rotate every index: V'_{abcd} = sum T*_{a i} T*_{b j} V_{ijkl} T_{c k} T_{d l}
  const std::vector<cplx> T = real_harmonics(l);
  std::vector<cplx> A(Vc), B(n * n * n * n);
  for (int pass = 0; pass < 4; ++pass) {
    std::fill(B.begin(), B.end(), 0.0);
    for (int i0 = 0; i0 < n; ++i0)
      for (int i1 = 0; i1 < n; ++i1)
        for (int i2 = 0; i2 < n; ++i2)
          for (int i3 = 0; i3 < n; ++i3) {
            const cplx v = A[((i0 * n + i1) * n + i2) * n + i3];
            if (v == 0.0) continue;
            int idx[4] = {i0, i1, i2, i3};
            const int old = idx[pass];
            for (int r = 0; r < n; ++r) {
              const cplx t = (pass < 2) ? std::conj(T[r * n + old]) : T[r * n + old];
              idx[pass] = r;
              B[((idx[0] * n + idx[1]) * n + idx[2]) * n + idx[3]] += t * v;
            }
          }
    std::swap(A, B);
  }
  return A;
}

// xi l.s in the real-harmonic product basis, flavour s*(2l+1) + (m+l).
std::vector<cplx> soc_matrix(int l, double xi) {
  const int n = 2 * l + 1, nf = 2 * n;
  std::vector<cplx> h(nf * nf, 0.0);
  for (int s = 0; s < 2; ++s) {
    const double sz = s ? 0.5 : -0.5;
    for (int m = -l; m <= l; ++m) h[(s * n + m + l) * nf + (s * n + m + l)] += xi * m * sz;
  }
  for (int m = -l; m < l; ++m) {
    const double v = 0.5 * xi * std::sqrt(double(l * (l + 1) - m * (m + 1)));
    h[(0 * n + (m + 1) + l) * nf + (1 * n + m + l)] += v;  // <m+1, dn| l.s |m, up>
    h[(1 * n + m + l) * nf + (0 * n + (m + 1) + l)] += v;
  }
  const std::vector<cplx> T = real_harmonics(l);
  // h_real[r][r'] = sum T*[r][m] h[m][m'] T[r'][m'] per spin block pair
  std::vector<cplx> out(nf * nf, 0.0);
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < 2; ++s2)
      for (int r1 = 0; r1 < n; ++r1)
        for (int r2 = 0; r2 < n; ++r2) {
          cplx acc = 0.0;
          for (int m1 = 0; m1 < n; ++m1)
            for (int m2 = 0; m2 < n; ++m2)
              acc += std::conj(T[r1 * n + m1]) * h[(s1 * n + m1) * nf + (s2 * n + m2)] * T[r2 * n + m2];
          out[(s1 * n + r1) * nf + (s2 * n + r2)] = acc;
        }
  return out;
}

// ------------------------------------------------------------------ terms

void add_one_body(const std::vector<cplx>& t, int nf, std::vector<Term>& terms) {
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nf; ++j) {
      const cplx c = t[i * nf + j];
      if (c == 0.0) continue;
      Term x;
      x.coef = c;
      x.n = 2;
      x.f[0] = i; x.dag[0] = 1;
      x.f[1] = j; x.dag[1] = 0;
      terms.push_back(x);
    }
}

// 1/2 sum V_ijkl c+_i c+_j c_l c_k over spin-orbitals, V spin-diagonal from <ab|V|cd>.
void add_two_body(const std::vector<cplx>& V, int n, std::vector<Term>& terms) {
  const double tol = 1e-14;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c)
        for (int d = 0; d < n; ++d) {
          const cplx v = V[((a * n + b) * n + c) * n + d];
          if (std::abs(v) < tol) continue;
          for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
              const int i = s1 * n + a, j = s2 * n + b, k = s1 * n + c, l = s2 * n + d;
              if (i == j || k == l) continue;
              Term x;
              x.coef = 0.5 * v;
              x.n = 4;
              x.f[0] = i; x.dag[0] = 1;
              x.f[1] = j; x.dag[1] = 1;
              x.f[2] = l; x.dag[2] = 0;
              x.f[3] = k; x.dag[3] = 0;
              terms.push_back(x);
            }
        }
}

}  // namespace

// ------------------------------------------------------------------ build

int build_host_model(const ctq_model_params* p, HostModel& m, std::string& err) {
  if (!p) { err = "null params"; return CTQ_ERR_ARG; }
  const int n = p->n_orb, nf = 2 * n;
  if (n < 1 || nf > 16) { err = "n_orb must be in [1, 8]"; return CTQ_ERR_ARG; }
  if (p->interaction != CTQ_KANAMORI && p->interaction != CTQ_SLATER) { err = "interaction"; return CTQ_ERR_ARG; }
  if (p->interaction == CTQ_SLATER && !((p->l == 2 && n == 5) || (p->l == 3 && n == 7))) {
    err = "slater needs (l, n_orb) = (2, 5) or (3, 7)";
    return CTQ_ERR_ARG;
  }
  if (p->soc_xi != 0.0 && p->interaction != CTQ_SLATER) { err = "SOC needs a slater shell"; return CTQ_ERR_ARG; }
  if (p->sector_mode != CTQ_SECTORS_N_SZ && p->sector_mode != CTQ_SECTORS_N) { err = "sector_mode"; return CTQ_ERR_ARG; }
  if (p->sector_mode == CTQ_SECTORS_N_SZ && (p->soc_xi != 0.0)) { err = "SOC breaks S_z: use CTQ_SECTORS_N"; return CTQ_ERR_ARG; }

  // one-body part at mu = 0 (mu enters per sector as -mu N afterwards)
  std::vector<cplx> t(nf * nf, 0.0);
  if (p->soc_xi != 0.0) t = soc_matrix(p->l, p->soc_xi);
  if (p->cf_re || p->cf_im)
    for (int i = 0; i < nf * nf; ++i)
      t[i] += cplx(p->cf_re ? p->cf_re[i] : 0.0, p->cf_im ? p->cf_im[i] : 0.0);
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nf; ++j)
      if (std::abs(t[i * nf + j] - std::conj(t[j * nf + i])) > 1e-12) { err = "one-body term not Hermitian"; return CTQ_ERR_ARG; }

  std::vector<Term> terms;
  add_one_body(t, nf, terms);
  add_two_body(p->interaction == CTQ_KANAMORI ? kanamori_tensor(n, p->U, p->J) : slater_tensor(p->l, p->U, p->J),
               n, terms);

  // sectors
  const uint32_t n_states = 1u << nf;
  std::map<std::pair<int, int>, std::vector<uint32_t>> groups;  // key (N, sub-label)
  for (uint32_t st = 0; st < n_states; ++st) {
    const int nd = popc(st & ((1u << n) - 1u)), nu = popc(st >> n), N = nd + nu;
    if (p->n_min >= 0 && N < p->n_min) continue;
    if (p->n_max >= 0 && N > p->n_max) continue;
    const int sub = (p->sector_mode == CTQ_SECTORS_N_SZ) ? nd : 0;
    groups[{N, sub}].push_back(st);
  }
  m.n_flav = nf;
  m.n_sec = int(groups.size());
  std::vector<std::vector<uint32_t>> states;
  for (auto& g : groups) {
    m.N.push_back(g.first.first);
    m.dims.push_back(int(g.second.size()));
    states.push_back(g.second);
  }
  m.max_dim = *std::max_element(m.dims.begin(), m.dims.end());
  std::vector<int> sec_of(n_states, -1), pos_of(n_states, -1);
  for (int q = 0; q < m.n_sec; ++q)
    for (int i = 0; i < m.dims[q]; ++i) {
      sec_of[states[q][i]] = q;
      pos_of[states[q][i]] = i;
    }

  // sector Hamiltonians at mu = 0
  std::vector<std::vector<cplx>> H(m.n_sec);
  double max_abs = 0.0, max_im = 0.0;
  for (int q = 0; q < m.n_sec; ++q) {
    const int d = m.dims[q];
    H[q].assign(size_t(d) * d, 0.0);
    for (const Term& x : terms)
      for (int col = 0; col < d; ++col) {
        uint32_t st = states[q][col];
        double sign = 1.0;
        if (!apply_term(x, st, sign)) continue;
        if (sec_of[st] != q) { err = "term leaves its sector"; return CTQ_ERR_ARG; }
        H[q][size_t(pos_of[st]) * d + col] += sign * x.coef;
      }
    for (const cplx& v : H[q]) {
      max_abs = std::max(max_abs, std::abs(v));
      max_im = std::max(max_im, std::abs(v.imag()));
    }
  }
  // Real-harmonic rotations leave ~1e-16 imaginary residue in a real problem.
  m.is_complex = (max_im > 1e-13 * std::max(1.0, max_abs)) ? 1 : 0;

  // eigenbasis: host Jacobi, or the device solver when any sector is large
  std::vector<std::vector<double>> Vr(m.n_sec);
  std::vector<std::vector<cplx>> Vc(m.n_sec);
  std::vector<std::vector<double>> E0(m.n_sec);
  const bool on_device = m.max_dim > kJacobiMaxDim;
  DeviceSectorLA dla;
  if (on_device) {
    const int st = dla.init(p->device, m.is_complex != 0, m.n_sec, err);
    if (st != CTQ_OK) return st;
  }
  for (int q = 0; q < m.n_sec; ++q) {
    const int d = m.dims[q];
    int st;
    if (on_device) {
      if (m.is_complex) Vc[q].resize(size_t(d) * d);
      else Vr[q].resize(size_t(d) * d);
      st = dla.eigh(q, d, H[q], E0[q], &Vc[q], &Vr[q], err);
    } else if (m.is_complex) {
      st = jacobi_eigh_cplx(d, H[q], E0[q], Vc[q]);
    } else {
      std::vector<double> A(size_t(d) * d);
      for (size_t i = 0; i < A.size(); ++i) A[i] = H[q][i].real();
      st = jacobi_eigh_real(d, A, E0[q], Vr[q]);
    }
    if (st != CTQ_OK) {
      if (err.empty()) err = "eigensolver did not converge";
      return st;
    }
    std::vector<cplx>().swap(H[q]);
  }

  // chemical potential
  if (p->mu_mode == CTQ_MU_PH_SYMMETRIC) {
    double lo = INFINITY, hi = INFINITY;
    for (int q = 0; q < m.n_sec; ++q) {
      if (m.N[q] == p->n0 - 1) lo = std::min(lo, E0[q][0]);
      if (m.N[q] == p->n0 + 1) hi = std::min(hi, E0[q][0]);
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) { err = "n0 +- 1 sectors missing"; return CTQ_ERR_ARG; }
    m.mu = 0.5 * (hi - lo);
  } else if (p->mu_mode == CTQ_MU_GIVEN) {
    m.mu = p->mu;
  } else {
    err = "mu_mode";
    return CTQ_ERR_ARG;
  }
  m.E_off.assign(m.n_sec + 1, 0);
  m.E_min.resize(m.n_sec);
  m.E_gs = INFINITY;
  for (int q = 0; q < m.n_sec; ++q) {
    m.E_off[q + 1] = m.E_off[q] + m.dims[q];
    for (double e : E0[q]) m.E.push_back(e - m.mu * m.N[q]);
    m.E_min[q] = m.E[m.E_off[q]];
    m.E_gs = std::min(m.E_gs, m.E_min[q]);
  }
  m.h1 = t;  // one-body matrix t - mu (for the Bulla operators [c_f, U])
  for (int i = 0; i < nf; ++i) m.h1[size_t(i) * nf + i] -= m.mu;

  // blocks F_alpha(q) = V_{q'}^H C_alpha V_q  (C: signed partial permutation)
  const int na = 2 * nf;
  m.s.assign(size_t(na) * m.n_sec, -1);
  m.blk_off.assign(size_t(na) * m.n_sec, -1);
  m.opnorm.assign(size_t(na) * m.n_sec, 0.0);
  int64_t total = 0;
  for (int a = 0; a < na; ++a) {
    const int f = a / 2, dag = a % 2;
    for (int q = 0; q < m.n_sec; ++q) {
      int qp = -1;
      std::vector<std::pair<int, std::pair<int, double>>> pairs;  // (col j, (row k, sign))
      for (int j = 0; j < m.dims[q]; ++j) {
        uint32_t st = states[q][j];
        double sign = 1.0;
        if (!apply_op(st, f, dag, sign)) continue;
        if (sec_of[st] < 0) continue;  // leaves the N window
        if (qp >= 0 && sec_of[st] != qp) { err = "operator target sector not unique"; return CTQ_ERR_ARG; }
        qp = sec_of[st];
        pairs.push_back({j, {pos_of[st], sign}});
      }
      if (qp < 0) continue;
      const int dq = m.dims[q], dp = m.dims[qp];
      m.s[size_t(a) * m.n_sec + q] = qp;
      m.blk_off[size_t(a) * m.n_sec + q] = total;
      // A nonzero restriction of c or c+ is a signed partial permutation in the
      // occupation basis, rotated by unitaries: its singular values are 0 or 1.
      m.opnorm[size_t(a) * m.n_sec + q] = 1.0;
      const size_t base = size_t(total);
      total += int64_t(dp) * dq;
      m.blk_re.resize(size_t(total), 0.0);
      if (m.is_complex) m.blk_im.resize(size_t(total), 0.0);
      if (on_device) {
        std::vector<int> src, dst;
        std::vector<double> sg;
        for (const auto& pr : pairs) {
          src.push_back(pr.first);
          dst.push_back(pr.second.first);
          sg.push_back(pr.second.second);
        }
        const int st = dla.block(q, qp, src, dst, sg, &m.blk_re[base], m.is_complex ? &m.blk_im[base] : nullptr, err);
        if (st != CTQ_OK) return st;
        continue;
      }
      for (const auto& pr : pairs) {
        const int j = pr.first, k = pr.second.first;
        const double sg = pr.second.second;
        // F[mm][nn] += sg * conj(V'[k][mm]) * V[j][nn]
        if (m.is_complex) {
          for (int mm = 0; mm < dp; ++mm) {
            const cplx left = sg * std::conj(Vc[qp][size_t(k) * dp + mm]);
            if (left == 0.0) continue;
            double* re = &m.blk_re[base + size_t(mm) * dq];
            double* im = &m.blk_im[base + size_t(mm) * dq];
            const cplx* vr = &Vc[q][size_t(j) * dq];
            for (int nn = 0; nn < dq; ++nn) {
              const cplx v = left * vr[nn];
              re[nn] += v.real();
              im[nn] += v.imag();
            }
          }
        } else {
          for (int mm = 0; mm < dp; ++mm) {
            const double left = sg * Vr[qp][size_t(k) * dp + mm];
            if (left == 0.0) continue;
            double* re = &m.blk_re[base + size_t(mm) * dq];
            const double* vr = &Vr[q][size_t(j) * dq];
            for (int nn = 0; nn < dq; ++nn) re[nn] += left * vr[nn];
          }
        }
      }
    }
  }
  return CTQ_OK;
}

// ------------------------------------------------------------------ Jacobi eigensolvers

namespace {

template <typename T>
double sq_abs(const T& v) { return std::norm(cplx(v)); }

template <typename T>
void sort_eigen(int n, std::vector<double>& E, std::vector<T>& V) {
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return E[a] < E[b]; });
  std::vector<double> E2(n);
  std::vector<T> V2(size_t(n) * n);
  for (int c = 0; c < n; ++c) {
    E2[c] = E[idx[c]];
    for (int r = 0; r < n; ++r) V2[size_t(r) * n + c] = V[size_t(r) * n + idx[c]];
  }
  E.swap(E2);
  V.swap(V2);
}

inline double conj_(double v) { return v; }
inline cplx conj_(cplx v) { return std::conj(v); }
inline double abs_(double v) { return std::fabs(v); }
inline double abs_(cplx v) { return std::abs(v); }
inline double phase_of(double v, double /*abs*/) { return v < 0 ? -1.0 : 1.0; }
inline cplx phase_of(cplx v, double a) { return v / a; }

// Cyclic Jacobi for a Hermitian matrix (A row-major).  For the pair (p, q)
// with off-diagonal b = |b| e^{i phi}: tau = (a_qq - a_pp) / (2|b|),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c, and
// the unitary G (G_pp = G_qq = c, G_pq = s e^{i phi}, G_qp = -s e^{-i phi})
// gives (G^H A G)_pq = 0.  Converges quadratically.
template <typename T>
int jacobi(int n, std::vector<T>& A, std::vector<double>& E, std::vector<T>& V) {
  V.assign(size_t(n) * n, T(0));
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = T(1);
  auto a = [&](int r, int c) -> T& { return A[size_t(r) * n + c]; };
  double fro = 0.0;
  for (const T& v : A) fro += sq_abs(v);
  fro = std::sqrt(fro);
  const double tol = 1e-17 * std::max(fro, 1e-300);
  int sweep = 0;
  for (; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += sq_abs(a(p, q));
    if (std::sqrt(2.0 * off) <= tol * std::max(1, n)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const T b = a(p, q);
        const double ab = abs_(b);
        if (ab == 0.0) continue;
        const double app = std::real(cplx(a(p, p))), aqq = std::real(cplx(a(q, q)));
        // skip entries negligible against both diagonals (classical threshold)
        if (sweep > 3 && ab < 1e-18 * (std::fabs(app) + std::fabs(aqq))) {
          a(p, q) = T(0);
          a(q, p) = T(0);
          continue;
        }
        const T ph = phase_of(b, ab);
        const double tau = (aqq - app) / (2.0 * ab);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        const T gpq = s * ph, gqp = -s * conj_(ph);
        // A <- A G (columns p, q)
        for (int k = 0; k < n; ++k) {
          const T akp = a(k, p), akq = a(k, q);
          a(k, p) = akp * c + akq * gqp;
          a(k, q) = akp * gpq + akq * c;
        }
        // A <- G^H A (rows p, q)
        for (int k = 0; k < n; ++k) {
          const T apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk + conj_(gqp) * aqk;
          a(q, k) = conj_(gpq) * apk + c * aqk;
        }
        a(p, q) = T(0);
        a(q, p) = T(0);
        a(p, p) = T(std::real(cplx(a(p, p))));
        a(q, q) = T(std::real(cplx(a(q, q))));
        for (int k = 0; k < n; ++k) {
          const T vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
          V[size_t(k) * n + p] = vkp * c + vkq * gqp;
          V[size_t(k) * n + q] = vkp * gpq + vkq * c;
        }
      }
  }
  if (sweep >= 100) return CTQ_ERR_NUMERIC;
  E.resize(n);
  for (int i = 0; i < n; ++i) E[i] = std::real(cplx(a(i, i)));
  sort_eigen(n, E, V);
  return CTQ_OK;
}

}  // namespace

int jacobi_eigh_real(int n, std::vector<double>& A, std::vector<double>& E, std::vector<double>& V) {
  return jacobi<double>(n, A, E, V);
}

int jacobi_eigh_cplx(int n, std::vector<cplx>& A, std::vector<double>& E, std::vector<cplx>& V) {
  return jacobi<cplx>(n, A, E, V);
}

}  // namespace ctq

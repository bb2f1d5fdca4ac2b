// Series coefficients of Philcox & Slepian (arXiv:2102.08384), host FP64.
//
// The complex-basis coefficients follow the paper's boxed definitions term by
// term (Appendix A building blocks; phi: Appendix B eq. shift-coeff-def;
// f: Appendix E eq. f-alpha-def; B: Appendix F eq. B-def).  The kernels work
// with real spherical harmonics, so each coupling is then rotated into the
// real basis with the unitary map U (Y_R = U Y) and emitted as a sparse list.
#include "coeff.h"

#include <cmath>
#include <complex>
#include <cstdlib>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>

namespace bym {
namespace {

constexpr double kFourPi = 4.0 * M_PI;

long double factorial(int n) {
  static long double table[171];
  static std::once_flag once;
  std::call_once(once, [] {
    table[0] = 1.0L;
    for (int i = 1; i <= 170; ++i) table[i] = table[i - 1] * (long double)i;
  });
  if (n < 0 || n > 170) throw std::out_of_range("factorial argument");
  return table[n];
}

long double double_factorial(int n) {
  long double r = 1.0L;
  for (int i = n; i > 1; i -= 2) r *= (long double)i;
  return r;
}

double binomial(int n, int k) {
  if (n < 0 || k < 0 || k > n) return 0.0;
  return (double)(factorial(n) / (factorial(k) * factorial(n - k)));
}

inline double parity(int n) { return (n % 2 == 0) ? 1.0 : -1.0; }

}  // namespace

static double wigner3j_racah(int j1, int j2, int j3, int m1, int m2, int m3);

// Wigner 3-j symbol, memoised (the tables call it many times with few distinct arguments).
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, double> cache;
  const auto key = std::make_tuple(j1, j2, j3, m1, m2);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const double v = wigner3j_racah(j1, j2, j3, m1, m2, m3);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = v;
  return v;
}

// Racah's closed form of the Wigner 3-j symbol, in long double.
static double wigner3j_racah(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  const long double pre =
      factorial(j1 + j2 - j3) * factorial(j1 - j2 + j3) * factorial(-j1 + j2 + j3) /
      factorial(j1 + j2 + j3 + 1) * factorial(j1 + m1) * factorial(j1 - m1) * factorial(j2 + m2) *
      factorial(j2 - m2) * factorial(j3 + m3) * factorial(j3 - m3);
  const int kmin = std::max(0, std::max(j2 - j3 - m1, j1 - j3 + m2));
  const int kmax = std::min(j1 + j2 - j3, std::min(j1 - m1, j2 + m2));
  long double sum = 0.0L;
  for (int k = kmin; k <= kmax; ++k) {
    const long double den = factorial(k) * factorial(j3 - j2 + k + m1) * factorial(j3 - j1 + k - m2) *
                            factorial(j1 + j2 - j3 - k) * factorial(j1 - k - m1) * factorial(j2 - k + m2);
    sum += ((k % 2) ? -1.0L : 1.0L) / den;
  }
  const int sgn = j1 - j2 - m3;
  return (double)(parity(sgn) * sqrtl(pre) * sum);
}

double gaunt(int l1, int l2, int l3, int m1, int m2, int m3) {
  if (l1 < 0 || l2 < 0 || l3 < 0) return 0.0;
  const double t0 = wigner3j(l1, l2, l3, 0, 0, 0);
  if (t0 == 0.0) return 0.0;
  const double t = wigner3j(l1, l2, l3, m1, m2, m3);
  if (t == 0.0) return 0.0;
  return std::sqrt((2.0 * l1 + 1) * (2.0 * l2 + 1) * (2.0 * l3 + 1) / kFourPi) * t * t0;
}

double solid_coupling(int ell, int m, int lam, int mu) {
  if (lam < 0 || lam > ell || std::abs(mu) > lam || std::abs(m - mu) > ell - lam) return 0.0;
  const double b = binomial(ell + m, lam + mu) * binomial(ell - m, lam - mu);
  if (b == 0.0) return 0.0;
  return std::sqrt(kFourPi * (2.0 * ell + 1) / ((2.0 * lam + 1) * (2.0 * ell - 2.0 * lam + 1))) * std::sqrt(b);
}

double legendre_inverse(int L, int n) {
  if (L < 0 || L > n || (n - L) % 2) return 0.0;
  return (double)((2.0L * L + 1) * factorial(n) * double_factorial(L + n + 2) /
                  (factorial(L + n + 2) * double_factorial(n - L)));
}

double gegenbauer_term(int two_a, int N, int k) {
  if (k < 0 || 2 * k > N) return 0.0;
  if (two_a == 0) return (N == 0) ? 1.0 : 0.0;
  const long double a = 0.5L * two_a;
  long double poch = 1.0L;                     // (a)_{N-k}
  for (int i = 0; i < N - k; ++i) poch *= (a + i);
  return (double)(parity(k) * poch / (factorial(k) * factorial(N - 2 * k)));
}

double shift_phi(int alpha, int ell, int m, int J1, int J2, int M) {
  return shift_sum(alpha, ell, m, J1, J2, M, ell);
}

double shift_omega(int beta, int ell, int m, int alpha, int J1, int J2, int M) {
  return shift_sum(beta, ell, m, J1, J2, M, ell + alpha);
}

double shift_sum(int alpha, int ell, int m, int J1, int J2, int M, int two_gamma) {
  if (std::abs(m) > ell || std::abs(M) > J1 || std::abs(m - M) > J2 || J1 < 0 || J2 < 0) return 0.0;
  double total = 0.0;
  for (int lam = 0; lam <= ell; ++lam) {
    const int N = alpha - lam;
    if (N < 0) continue;
    for (int mu = -lam; mu <= lam; ++mu) {
      const double A = solid_coupling(ell, m, lam, mu);
      if (A == 0.0) continue;
      for (int k = 0; 2 * k <= N; ++k) {
        const double C = gegenbauer_term(two_gamma, N, k);
        if (C == 0.0) continue;
        const int pw = N - 2 * k;
        const double m2pow = std::pow(-2.0, pw);
        for (int Lp = pw; Lp >= 0; Lp -= 2) {
          const double ct = legendre_inverse(Lp, pw);
          if (ct == 0.0) continue;
          const double g1 = gaunt(lam, Lp, J1, mu, M - mu, -M);
          if (g1 == 0.0) continue;
          const double g2 = gaunt(ell - lam, Lp, J2, m - mu, mu - M, M - m);
          if (g2 == 0.0) continue;
          total += A * C * m2pow * ct * kFourPi / (2 * Lp + 1) * g1 * g2 * parity(m + M - mu);
        }
      }
    }
  }
  return total;
}

double legendre_shift_f(int alpha, int ell, int J) { return legendre_shift_sum(alpha, ell, J, ell); }

double legendre_shift_h(int beta, int alpha, int ell, int J) { return legendre_shift_sum(beta, ell, J, ell + alpha); }

double legendre_shift_sum(int alpha, int ell, int J, int two_gamma) {
  if (J < 0) return 0.0;
  double total = 0.0;
  for (int lam = 0; lam <= std::min(alpha, ell); ++lam) {
    const double t0 = wigner3j(ell, lam, ell - lam, 0, 0, 0);
    if (t0 == 0.0) continue;
    const double pre = std::sqrt(binomial(2 * ell, 2 * lam)) * t0;
    const int N = alpha - lam;
    for (int k = 0; 2 * k <= N; ++k) {
      const double C = gegenbauer_term(two_gamma, N, k);
      if (C == 0.0) continue;
      const int pw = N - 2 * k;
      for (int Lp = pw; Lp >= 0; Lp -= 2) {
        const double ct = legendre_inverse(Lp, pw);
        if (ct == 0.0) continue;
        const double t = wigner3j(ell - lam, Lp, J, 0, 0, 0);
        total += pre * C * std::pow(-2.0, pw) * ct * t * t;
      }
    }
  }
  return parity(ell) * std::pow(2.0 * ell + 1, 1.5) * total;
}

double bisector_B(int beta, int ell, int m, int J1, int J2, int M) {
  if (std::abs(m) > ell || std::abs(M) > J1 || std::abs(m - M) > J2 || J1 < 0 || J2 < 0) return 0.0;
  // generalised binomial (-ell/2 choose beta) = prod_{i<beta} (-ell/2 - i) / beta!
  long double gb = 1.0L;
  for (int i = 0; i < beta; ++i) gb *= (-0.5L * ell - i);
  gb /= factorial(beta);
  if (gb == 0.0L) return 0.0;
  double total = 0.0;
  for (int lam = 0; lam <= ell; ++lam) {
    for (int mu = -lam; mu <= lam; ++mu) {
      const double A = solid_coupling(ell, m, lam, mu);
      if (A == 0.0) continue;
      for (int n = 0; n <= beta; ++n) {
        const double bn = binomial(beta, n) * parity(beta - n);
        for (int L = n; L >= 0; L -= 2) {
          const double ct = legendre_inverse(L, n);
          if (ct == 0.0) continue;
          const double g1 = gaunt(lam, L, J1, mu, M - mu, -M);
          if (g1 == 0.0) continue;
          const double g2 = gaunt(ell - lam, L, J2, m - mu, mu - M, M - m);
          if (g2 == 0.0) continue;
          total += A * (double)gb * std::ldexp(1.0, -beta) * bn * ct * kFourPi / (2 * L + 1) *
                   parity(M - mu - m) * g1 * g2;
        }
      }
    }
  }
  return std::ldexp(total, -ell);
}

// Appendix C, eq. generalized-shift-theorem:
// Omega^{beta, alpha J1 J2 m M}_{S1 S2 T} = sum_{J'} omega^{beta, J2 (m-M) alpha}_{J' S2 (T-M)} G_{J1 J' S1}^{M (T-M) (-T)} (-1)^T
double shift_Omega(int beta, int alpha, int J1, int J2, int m, int M, int S1, int S2, int T) {
  double total = 0.0;
  for (int Jp = 0; Jp <= beta; ++Jp) {
    const double w = shift_omega(beta, J2, m - M, alpha, Jp, S2, T - M);
    if (w == 0.0) continue;
    const double g = gaunt(J1, Jp, S1, M, T - M, -T);
    if (g == 0.0) continue;
    total += w * g * parity(T);
  }
  return total;
}

// Appendix D: Phi^0 = phi^0, Phi^2 = -phi^2,
// Phi^4 = -phi^4 + sum_{J1' J2' M'} phi^2_{J1' J2' M'} Omega^{2, 2 J1' J2' m M'}_{J1 J2 M}.
double parity_even_Phi(int alpha, int ell, int m, int J1, int J2, int M) {
  if (alpha == 0) return shift_phi(0, ell, m, J1, J2, M);
  if (alpha == 2) return -shift_phi(2, ell, m, J1, J2, M);
  if (alpha != 4) throw std::runtime_error("parity-even coefficients are written out to alpha = 4");
  double total = -shift_phi(4, ell, m, J1, J2, M);
  for (int J1p = 0; J1p <= 2; J1p += 2)
    for (int J2p = std::max(0, ell - 2); J2p <= ell + 2; ++J2p)
      for (int Mp = -J1p; Mp <= J1p; ++Mp) {
        const double c = shift_phi(2, ell, m, J1p, J2p, Mp);
        if (std::fabs(c) < 1e-14) continue;
        total += c * shift_Omega(2, 2, J1p, J2p, m, Mp, J1, J2, M);
      }
  return total;
}

// Appendix E.2: F^0 = f^0, F^2 = -f^2, F^4 = -f^4 + sum_S f^{2,ell}_S h^{2,2S}_J.
double parity_even_F(int alpha, int ell, int J) {
  if (alpha == 0) return legendre_shift_f(0, ell, J);
  if (alpha == 2) return -legendre_shift_f(2, ell, J);
  if (alpha != 4) throw std::runtime_error("parity-even coefficients are written out to alpha = 4");
  double total = -legendre_shift_f(4, ell, J);
  for (int S = std::max(0, ell - 2); S <= ell + 2; ++S) {
    const double c = legendre_shift_f(2, ell, S);
    if (std::fabs(c) < 1e-14) continue;
    total += c * legendre_shift_h(2, 2, S, J);
  }
  return total;
}

// ---------------------------------------------------------------------------
// real basis
// ---------------------------------------------------------------------------
namespace {

using cplx = std::complex<double>;

// U^l_{mu m}: Y_{l,mu} (real) = sum_m U_{mu m} Y_l^m (complex).
cplx Ucoef(int mu, int m) {
  const double s = 1.0 / std::sqrt(2.0);
  if (mu > 0) {
    if (m == mu) return cplx(parity(mu) * s, 0.0);
    if (m == -mu) return cplx(s, 0.0);
    return 0.0;
  }
  if (mu == 0) return (m == 0) ? cplx(1.0, 0.0) : cplx(0.0, 0.0);
  const int a = -mu;
  if (m == a) return cplx(0.0, -parity(a) * s);
  if (m == -a) return cplx(0.0, s);
  return 0.0;
}

// Rotate a complex coupling C(m, M) (coefficient of Y_J1^M Y_J2^{m-M} in
// Y_l^m) into the real coupling R(mu, nu1, nu2) and call emit for each
// non-zero entry.  The result is real by construction; any imaginary
// residue beyond rounding means a broken table and throws.
template <class Coef, class Emit>
void real_coupling(int l, int J1, int J2, Coef coef, Emit emit) {
  std::map<std::pair<int, int>, double> C;  // (m, M) -> value
  double scale = 0.0;
  for (int m = -l; m <= l; ++m)
    for (int M = -J1; M <= J1; ++M) {
      if (std::abs(m - M) > J2) continue;
      const double v = coef(m, M);
      if (std::fabs(v) > 1e-13) {     // below this the sum is rounding residue of an exact zero
        C[{m, M}] = v;
        scale = std::max(scale, std::fabs(v));
      }
    }
  if (C.empty()) return;
  for (int mu = -l; mu <= l; ++mu)
    for (int nu1 = -J1; nu1 <= J1; ++nu1)
      for (int nu2 = -J2; nu2 <= J2; ++nu2) {
        cplx acc = 0.0;
        for (int sm : {1, -1}) {
          const int m = sm * std::abs(mu);
          if (sm == -1 && mu == 0) continue;
          const cplx um = Ucoef(mu, m);
          if (um == cplx(0.0)) continue;
          for (int sM : {1, -1}) {
            const int M = sM * std::abs(nu1);
            if (sM == -1 && nu1 == 0) continue;
            const cplx uM = std::conj(Ucoef(nu1, M));
            if (uM == cplx(0.0)) continue;
            const auto it = C.find({m, M});
            if (it == C.end()) continue;
            const cplx uN = std::conj(Ucoef(nu2, m - M));
            if (uN == cplx(0.0)) continue;
            acc += um * it->second * uM * uN;
          }
        }
        if (std::fabs(acc.imag()) > 1e-11 * scale)
          throw std::runtime_error("real-basis coupling has an imaginary part");
        if (std::fabs(acc.real()) > 1e-14 * scale) emit(mu, nu1, nu2, acc.real());
      }
}

}  // namespace

std::vector<GField> midpoint_gfields(int ell_max, int K, bool even) {
  std::vector<GField> out;
  for (int a = 0; a <= K; a += even ? 2 : 1)
    for (int J = a % 2; J <= ell_max + a; J += 2)
      for (int nu = -J; nu <= J; ++nu) out.push_back({a, J, nu});
  return out;
}

int midpoint_gfield_index(int ell_max, int alpha, int J, int nu, bool even) {
  int idx = 0;
  for (int a = 0; a <= alpha; a += even ? 2 : 1)
    for (int j = a % 2; j <= ell_max + a; j += 2) {
      if (a == alpha && j == J) return idx + nu + J;
      idx += 2 * j + 1;
    }
  return -1;
}

static std::vector<BisTerm> bisector_terms_parity(int ell_max, int K, int par) {
  const int bmax = K / 2;
  const int Jmax = ell_max + bmax;
  std::map<std::tuple<int, int, int>, double> acc;  // (lm, i, j), i <= j
  for (int l = par; l <= ell_max; l += 2)
    for (int J1 = 0; J1 <= Jmax; ++J1)
      for (int J2 = 0; J2 <= Jmax; ++J2) {
        if ((l + J1 + J2) % 2) continue;
        real_coupling(
            l, J1, J2,
            [&](int m, int M) {
              double s = 0.0;
              for (int b = 0; b <= bmax; ++b) s += bisector_B(b, l, m, J1, J2, M);
              return s;
            },
            [&](int mu, int nu1, int nu2, double v) {
              int i = ylm_index(J1, nu1), j = ylm_index(J2, nu2);
              if (i > j) std::swap(i, j);
              acc[{par ? odd_lm_index(l, mu) : even_lm_index(l, mu), i, j}] += v;
            });
      }
  std::vector<BisTerm> out;
  double scale = 0.0;
  for (auto &kv : acc) scale = std::max(scale, std::fabs(kv.second));
  for (auto &kv : acc)
    if (std::fabs(kv.second) > 1e-14 * scale)
      out.push_back({std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), kv.second});
  return out;
}

std::vector<GField> midpoint_gfields_odd(int ell_max, int K) {
  std::vector<GField> out;
  for (int a = 0; a <= K; ++a)
    for (int J = (a + 1) % 2; J <= ell_max + a; J += 2)
      for (int nu = -J; nu <= J; ++nu) out.push_back({a, J, nu});
  return out;
}

int midpoint_gfield_index_odd(int ell_max, int alpha, int J, int nu) {
  int idx = 0;
  for (int a = 0; a <= alpha; ++a)
    for (int j = (a + 1) % 2; j <= ell_max + a; j += 2) {
      if (a == alpha && j == J) return idx + nu + J;
      idx += 2 * j + 1;
    }
  return -1;
}

std::vector<MidTerm> midpoint_terms_odd(int ell_max, int K) {
  std::vector<MidTerm> out;
  for (int l = 1; l <= ell_max; l += 2)
    for (int a = 0; a <= K; ++a)
      for (int J1 = a % 2; J1 <= a; J1 += 2)
        for (int J2 = std::max(0, l - a); J2 <= l + a; ++J2) {
          if ((l + a + J2) % 2) continue;
          real_coupling(
              l, J1, J2, [&](int m, int M) { return shift_phi(a, l, m, J1, J2, M); },
              [&](int mu, int nu1, int nu2, double v) {
                out.push_back({odd_lm_index(l, mu), a, ylm_index(J1, nu1),
                               midpoint_gfield_index_odd(ell_max, a, J2, nu2), v});
              });
        }
  return out;
}

std::vector<XiTerm> midpoint_xi_terms_odd(int ell_max, int K) {
  std::vector<XiTerm> out;
  for (int l = 1; l <= ell_max; l += 2)
    for (int a = 0; a <= K; ++a)
      for (int J = std::max(0, l - a); J <= l + a; ++J) {
        if ((a + l + J) % 2) continue;
        const double f = legendre_shift_f(a, l, J);
        if (std::fabs(f) > 1e-13) out.push_back({l, a, J, f});
      }
  return out;
}

std::vector<BisTerm> bisector_terms(int ell_max, int K) { return bisector_terms_parity(ell_max, K, 0); }

std::vector<BisTerm> bisector_terms_odd(int ell_max, int K) { return bisector_terms_parity(ell_max, K, 1); }

std::vector<MidTerm> midpoint_terms(int ell_max, int K, bool even) {
  std::vector<MidTerm> out;
  for (int l = 0; l <= ell_max; l += 2)
    for (int a = 0; a <= K; a += even ? 2 : 1)
      for (int J1 = a % 2; J1 <= a; J1 += 2)
        for (int J2 = std::max(0, l - a); J2 <= l + a; ++J2) {
          if ((l + a + J2) % 2) continue;
          real_coupling(
              l, J1, J2,
              [&](int m, int M) {
                return even ? parity_even_Phi(a, l, m, J1, J2, M) : shift_phi(a, l, m, J1, J2, M);
              },
              [&](int mu, int nu1, int nu2, double v) {
                out.push_back({even_lm_index(l, mu), a, ylm_index(J1, nu1),
                               midpoint_gfield_index(ell_max, a, J2, nu2, even), v});
              });
        }
  return out;
}

std::vector<XiTerm> midpoint_xi_terms(int ell_max, int K, bool even) {
  std::vector<XiTerm> out;
  for (int l = 0; l <= ell_max; l += 2)
    for (int a = 0; a <= K; a += even ? 2 : 1)
      for (int J = std::max(0, l - a); J <= l + a; ++J) {
        if ((a + l + J) % 2) continue;
        const double f = even ? parity_even_F(a, l, J) : legendre_shift_f(a, l, J);
        if (std::fabs(f) > 1e-13) out.push_back({l, a, J, f});
      }
  return out;
}

}  // namespace bym

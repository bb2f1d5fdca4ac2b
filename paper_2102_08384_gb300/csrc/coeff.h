// Host-side (FP64) series coefficients of arXiv:2102.08384 and their
// real-spherical-harmonic form, as sparse term lists for the kernel generator.
#pragma once
#include <vector>

namespace bym {

// ---- complex-basis coefficients, taken term by term from the paper --------
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);
double gaunt(int l1, int l2, int l3, int m1, int m2, int m3);      // eq. Gaunt-3j-def
double solid_coupling(int ell, int m, int lam, int mu);              // A_{ell m}^{lam mu}, eq. solid-harm-application
double legendre_inverse(int L, int n);                               // c~^L_n, eq. Leg-polynomial-inv-def
double gegenbauer_term(int two_a, int N, int k);                     // C_{Nk}^{a}, a = two_a / 2, eq. gegenbauer-explicit
double shift_phi(int alpha, int ell, int m, int J1, int J2, int M);  // eq. shift-coeff-def
// the sum of eq. shift-coeff-def with Gegenbauer parameter two_gamma / 2 (phi: two_gamma = ell)
double shift_sum(int alpha, int ell, int m, int J1, int J2, int M, int two_gamma);
// omega^{beta, ell m alpha}_{J1 J2 M}: phi with C^{ell/2} -> C^{(ell+alpha)/2} (Appendix C)
double shift_omega(int beta, int ell, int m, int alpha, int J1, int J2, int M);
// Omega^{beta, alpha J1 J2 m M}_{S1 S2 T}, eq. generalized-shift-theorem
double shift_Omega(int beta, int alpha, int J1, int J2, int m, int M, int S1, int S2, int T);
double legendre_shift_f(int alpha, int ell, int J);                  // eq. f-alpha-def
double legendre_shift_sum(int alpha, int ell, int J, int two_gamma);
double legendre_shift_h(int beta, int alpha, int ell, int J);        // h^{beta, alpha ell}_J (Appendix E.2)
double parity_even_Phi(int alpha, int ell, int m, int J1, int J2, int M);  // Appendix D, alpha <= 4
double parity_even_F(int alpha, int ell, int J);                     // Appendix E.2, alpha <= 4
double bisector_B(int beta, int ell, int m, int J1, int J2, int M);  // eq. B-def

// ---- real-basis indexing ---------------------------------------------------
// Real spherical harmonics (orthonormal, no Condon-Shortley phase):
//   Y_{l,0} = Y_l^0;  Y_{l,+m} = sqrt2 (-1)^m Re Y_l^m;  Y_{l,-m} = sqrt2 (-1)^m Im Y_l^m.
inline int ylm_index(int l, int nu) { return l * l + l + nu; }          // all l
inline int even_lm_index(int l, int mu) { return l * (l + 1) / 2 + mu; } // even l only
inline int n_even_lm(int ell_max) { return (ell_max + 1) * (ell_max + 2) / 2; }
// odd l only (l = 2q + 1): the (2l + 1) entries of l follow those of 1, 3, .., l - 2
inline int odd_lm_index(int l, int mu) { const int q = (l - 1) / 2; return 2 * q * q + q + mu + l; }
inline int n_odd_lm(int ell_max) { const int q = (ell_max + 1) / 2; return 2 * q * q + q; }

// Midpoint convolution fields g^alpha_{J nu}: alpha = 0..K (even alpha only for the
// parity-even form), J = alpha mod 2, alpha mod 2 + 2, .., <= ell_max + alpha, nu = -J..J.
struct GField { int alpha, J, nu; };
std::vector<GField> midpoint_gfields(int ell_max, int K, bool even = false);
int midpoint_gfield_index(int ell_max, int alpha, int J, int nu, bool even = false);
// The g fields of the odd l <= ell_max (ell_max odd): J = alpha + 1, alpha - 1, .. >= 0,
// J <= ell_max + alpha (J1 = alpha mod 2 and J1 + J2 = l mod 2).
std::vector<GField> midpoint_gfields_odd(int ell_max, int K);
int midpoint_gfield_index_odd(int ell_max, int alpha, int J, int nu);

// Bisector P / X: X_{lm}(k) = sum c * Re(conj F_i(k) F_j(k)), i <= j (field i = ylm_index),
// summed over beta <= floor(K/2); c already symmetrised over (i, j) <-> (j, i).
struct BisTerm { int lm, i, j; double c; };
std::vector<BisTerm> bisector_terms(int ell_max, int K);
// The same for the odd l <= ell_max (lm = odd_lm_index), fields J <= ell_max + floor(K/2).
std::vector<BisTerm> bisector_terms_odd(int ell_max, int K);

// Midpoint P: H_{lm}(Delta) = sum c t^alpha Y_{y}(hat Delta) g_{g}(Delta)
// (t = |Delta| / r0, fields carry (2r/r0)^-alpha), y = ylm_index(J1, nu1).
struct MidTerm { int lm, alpha, y, g; double c; };
std::vector<MidTerm> midpoint_terms(int ell_max, int K, bool even = false);   // even: Phi instead of phi
// odd l <= ell_max: lm = odd_lm_index, g = midpoint_gfield_index_odd
std::vector<MidTerm> midpoint_terms_odd(int ell_max, int K);

// Midpoint xi: T_l(Delta) = sum f t^alpha sum_nu Y_{J nu}(hat Delta) g^alpha_{J nu}(Delta).
struct XiTerm { int l, alpha, J; double f; };
std::vector<XiTerm> midpoint_xi_terms(int ell_max, int K, bool even = false);  // even: F instead of f
std::vector<XiTerm> midpoint_xi_terms_odd(int ell_max, int K);                  // odd l <= ell_max

}  // namespace bym

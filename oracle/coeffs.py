"""Series coefficients of the pairwise-LOS expansions, complex basis.

Test infrastructure only (see ``oracle/__init__``).

* ``phi(alpha, ell, m, J1, J2, M)`` -- spherical-harmonic shift theorem,
  Appendix B, eq. shift-coeff-def (boxed), used by eq. Ylm-shift-theorem:
      Y_ell^m(hat(a+A)) = sum phi^{alpha,ell m}_{J1 J2 M} (a/A)^alpha Y_J1^M(hat a) Y_J2^{m-M}(hat A).
* ``f_leg(alpha, ell, J)`` -- Legendre shift theorem, Appendix E, eq.
  f-alpha-def (boxed), used by eq. Legendre-shift-theorem-all-parity.
* ``B(beta, ell, m, J1, J2, M)`` -- bisector expansion, Appendix F, eq. B-def
  (boxed), used by eq. bisector-ylm-expan.

Each coefficient is the paper's sum taken term by term in its own order and
notation (A, C_{Nk}, c~, Gaunt), in FP64 with exact rational prefactors.

Parity pins (tests/test_oracle_coeffs.py):
  * the printed Y_2^1 midpoint example to alpha=2 (eq. Y21-all), every term;
  * the printed L_2 example to alpha=4 (eq. L2-all), every term;
  * the printed bisector Y_2^1 example at beta=0,1 (Sec. 5.1), every term;
  * closed forms phi^0, phi^{alpha,00} (Appendix B), f^0, f^{alpha,0}
    (Appendix E), B^0, B^{beta,00} (Appendix F);
  * selection rules (parities, J ranges) and the sum rule of Appendix E;
  * truncation error of each series against the exact function at random
    geometry, falling as eps^(K+1) (midpoint) or theta^(2 beta+2) (bisector);
  * f by an independent route: a direct Taylor expansion (sympy) of
    L_ell(hat a . hat(a+A)) in a/A (the alternative the paper names in Sec. 4.1).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

from .special import (FOUR_PI, binom, gaunt, gegenbauer_coeff, gen_binom,
                      legendre_inv_coeff, solid_A, w3j, ylm, legendre_L)


# --------------------------------------------------------------------------
# phi: spherical harmonic shift theorem (Appendix B)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def phi(alpha: int, ell: int, m: int, J1: int, J2: int, M: int) -> float:
    """phi^{alpha, ell m}_{J1 J2 M}, eq. shift-coeff-def.

    sum_{lam, mu} A_{ell m}^{lam mu} [N = alpha - lam >= 0]
      sum_k C_{Nk}^{ell/2} (-2)^(N-2k) sum_{L' = N-2k, N-2k-2, ..} c~^{L'}_{N-2k} 4pi/(2L'+1)
      G_{lam L' J1}^{mu (M-mu) (-M)} G_{(ell-lam) L' J2}^{(m-mu) (mu-M) (M-m)} (-1)^(m+M-mu)
    """
    return _shift_sum(alpha, ell, m, J1, J2, M, ell)


@lru_cache(maxsize=None)
def omega(beta: int, ell: int, m: int, alpha: int, J1: int, J2: int, M: int) -> float:
    """omega^{beta, ell m alpha}_{J1 J2 M} of Appendix C (eq. generalized-Ylm-tmp): phi with the
    Gegenbauer coefficient C^{ell/2}_{Nk} replaced by C^{(ell+alpha)/2}_{Nk}."""
    return _shift_sum(beta, ell, m, J1, J2, M, ell + alpha)


def _shift_sum(alpha: int, ell: int, m: int, J1: int, J2: int, M: int, two_gamma: int) -> float:
    """The sum of eq. shift-coeff-def with Gegenbauer parameter two_gamma / 2."""
    if abs(m) > ell or abs(M) > J1 or abs(m - M) > J2 or J1 < 0 or J2 < 0:
        return 0.0
    total = 0.0
    for lam in range(0, ell + 1):
        N = alpha - lam
        if N < 0:
            continue
        for mu in range(-lam, lam + 1):
            A = solid_A(ell, m, lam, mu)
            if A == 0.0:
                continue
            for k in range(0, N // 2 + 1):
                C = gegenbauer_coeff(Fraction(two_gamma, 2), N, k)
                if C == 0:
                    continue
                pw = N - 2 * k
                for Lp in range(pw, -1, -2):
                    ct = legendre_inv_coeff(Lp, pw)
                    if ct == 0:
                        continue
                    g1 = gaunt(lam, Lp, J1, mu, M - mu, -M)
                    if g1 == 0.0:
                        continue
                    g2 = gaunt(ell - lam, Lp, J2, m - mu, mu - M, M - m)
                    if g2 == 0.0:
                        continue
                    sign = -1.0 if (m + M - mu) % 2 else 1.0
                    total += (A * float(C) * float((-2) ** pw) * float(ct)
                              * FOUR_PI / (2 * Lp + 1) * g1 * g2 * sign)
    return total


def phi_table(alpha: int, ell: int, m: int, tol: float = 1e-13) -> dict:
    """All non-zero phi^{alpha, ell m}_{J1 J2 M} with the summation ranges of
    eq. Ylm-shift-theorem: 0 <= J1 <= alpha, max(0, ell-alpha) <= J2 <= ell+alpha, |M| <= J1."""
    out = {}
    for J1 in range(0, alpha + 1):
        for J2 in range(max(0, ell - alpha), ell + alpha + 1):
            for M in range(-J1, J1 + 1):
                v = phi(alpha, ell, m, J1, J2, M)
                if abs(v) > tol:
                    out[(J1, J2, M)] = v
    return out


def shift_series_ylm(ell: int, m: int, a, A, K: int) -> np.ndarray:
    """Truncated eq. Ylm-shift-theorem: sum_{alpha<=K} phi (a/A)^alpha Y_J1^M(hat a) Y_J2^{m-M}(hat A)."""
    a = np.asarray(a, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    eps = np.linalg.norm(a, axis=-1) / np.linalg.norm(A, axis=-1)
    out = np.zeros(eps.shape, dtype=np.complex128)
    for alpha in range(K + 1):
        for (J1, J2, M), c in phi_table(alpha, ell, m).items():
            out = out + c * eps ** alpha * ylm(J1, M, a) * ylm(J2, m - M, A)
    return out


# --------------------------------------------------------------------------
# f: Legendre shift theorem (Appendix E)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def f_leg(alpha: int, ell: int, J: int) -> float:
    """f^{alpha, ell}_J, eq. f-alpha-def.

    (-1)^ell (2ell+1)^(3/2) sum_{lam <= min(alpha, ell)} binom(2ell, 2lam)^(1/2) (ell lam ell-lam; 000)
      sum_k C^{ell/2}_{(alpha-lam) k} (-2)^(alpha-lam-2k)
      sum_{L' = alpha-lam-2k, .., step -2} c~^{L'}_{alpha-lam-2k} (ell-lam L' J; 000)^2
    """
    return _f_sum(alpha, ell, J, ell)


@lru_cache(maxsize=None)
def h_leg(beta: int, alpha: int, ell: int, J: int) -> float:
    """h^{beta, alpha ell}_J of Appendix E.2: f^{beta, ell}_J with C^{ell/2} replaced by C^{(ell+alpha)/2}."""
    return _f_sum(beta, ell, J, ell + alpha)


def _f_sum(alpha: int, ell: int, J: int, two_gamma: int) -> float:
    """The sum of eq. f-alpha-def with Gegenbauer parameter two_gamma / 2."""
    if J < 0:
        return 0.0
    total = 0.0
    for lam in range(0, min(alpha, ell) + 1):
        t0 = w3j(ell, lam, ell - lam, 0, 0, 0)
        if t0 == 0.0:
            continue
        pre = math.sqrt(binom(2 * ell, 2 * lam)) * t0
        N = alpha - lam
        for k in range(0, N // 2 + 1):
            C = gegenbauer_coeff(Fraction(two_gamma, 2), N, k)
            if C == 0:
                continue
            pw = N - 2 * k
            for Lp in range(pw, -1, -2):
                ct = legendre_inv_coeff(Lp, pw)
                if ct == 0:
                    continue
                t = w3j(ell - lam, Lp, J, 0, 0, 0)
                total += pre * float(C) * float((-2) ** pw) * float(ct) * t * t
    return (-1) ** ell * (2 * ell + 1) ** 1.5 * total


def f_table(alpha: int, ell: int, tol: float = 1e-13) -> dict:
    """Non-zero f^{alpha,ell}_J over max(ell-alpha, 0) <= J <= ell+alpha (eq. Legendre-shift-theorem-all-parity)."""
    out = {}
    for J in range(max(ell - alpha, 0), ell + alpha + 1):
        v = f_leg(alpha, ell, J)
        if abs(v) > tol:
            out[J] = v
    return out


def shift_series_legendre(ell: int, a, A, K: int) -> np.ndarray:
    """Truncated eq. Legendre-shift-theorem-all-parity:
    sum_{alpha<=K} sum_J (2J+1)/(2ell+1) f^{alpha,ell}_J (a/A)^alpha L_J(hat a . hat A)."""
    a = np.asarray(a, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    na = np.linalg.norm(a, axis=-1)
    nA = np.linalg.norm(A, axis=-1)
    mu = np.sum(a * A, axis=-1) / (na * nA)
    eps = na / nA
    out = np.zeros(eps.shape)
    for alpha in range(K + 1):
        for J, c in f_table(alpha, ell).items():
            out = out + (2 * J + 1) / (2 * ell + 1) * c * eps ** alpha * legendre_L(J, mu)
    return out


# --------------------------------------------------------------------------
# parity-even midpoint coefficients (Appendix C, D, E.2)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def Omega(beta: int, alpha: int, J1: int, J2: int, m: int, M: int, S1: int, S2: int, T: int) -> float:
    """Omega^{beta, alpha J1 J2 m M}_{S1 S2 T}, eq. generalized-shift-theorem:
    sum_{J'} omega^{beta, J2 (m-M) alpha}_{J' S2 (T-M)} G_{J1 J' S1}^{M (T-M) (-T)} (-1)^T."""
    total = 0.0
    for Jp in range(0, beta + 1):
        w = omega(beta, J2, m - M, alpha, Jp, S2, T - M)
        if w == 0.0:
            continue
        g = gaunt(J1, Jp, S1, M, T - M, -T)
        if g == 0.0:
            continue
        total += w * g * (-1.0 if T % 2 else 1.0)
    return total


@lru_cache(maxsize=None)
def Phi_even(alpha: int, ell: int, m: int, J1: int, J2: int, M: int) -> float:
    """Phi^{alpha, ell m}_{J1 J2 M} of the parity-even expansion (Appendix D, boxed 2 Y = sum over
    even alpha), written out to alpha = 4 as the paper does:
      Phi^0 = sqrt(4pi) delta delta delta, Phi^2 = -phi^2,
      Phi^4 = -phi^4 + sum_{J1' J2' M'} phi^2_{J1' J2' M'} Omega^{2, 2 J1' J2' m M'}_{J1 J2 M}."""
    if alpha == 0:
        return phi(0, ell, m, J1, J2, M)
    if alpha == 2:
        return -phi(2, ell, m, J1, J2, M)
    if alpha == 4:
        total = -phi(4, ell, m, J1, J2, M)
        for (J1p, J2p, Mp), c in phi_table(2, ell, m).items():
            total += c * Omega(2, 2, J1p, J2p, m, Mp, J1, J2, M)
        return total
    if alpha % 2:
        return 0.0
    raise NotImplementedError("the parity-even coefficients are written out to alpha = 4")


def Phi_table(alpha: int, ell: int, m: int, tol: float = 1e-13) -> dict:
    out = {}
    for J1 in range(0, alpha + 1):
        for J2 in range(max(0, ell - alpha), ell + alpha + 1):
            for M in range(-J1, J1 + 1):
                v = Phi_even(alpha, ell, m, J1, J2, M)
                if abs(v) > tol:
                    out[(J1, J2, M)] = v
    return out


@lru_cache(maxsize=None)
def F_even(alpha: int, ell: int, J: int) -> float:
    """F^{alpha, ell}_J of the parity-even Legendre expansion (Appendix E.2, eq. F-coeff-def and the
    explicit forms after it): F^0 = delta_{ell J}, F^2 = -f^2, F^4 = -f^4 + sum_S f^{2,ell}_S h^{2,2S}_J.
    They enter as L_ell = 1/2 sum (2J+1)/(2ell+1) F [...] (the form of the boxed Appendix E.2 equation)."""
    if alpha == 0:
        return f_leg(0, ell, J)
    if alpha == 2:
        return -f_leg(2, ell, J)
    if alpha == 4:
        total = -f_leg(4, ell, J)
        for S, c in f_table(2, ell).items():
            total += c * h_leg(2, 2, S, J)
        return total
    if alpha % 2:
        return 0.0
    raise NotImplementedError("the parity-even coefficients are written out to alpha = 4")


def F_table(alpha: int, ell: int, tol: float = 1e-13) -> dict:
    out = {}
    for J in range(max(ell - alpha, 0), ell + alpha + 1):
        v = F_even(alpha, ell, J)
        if abs(v) > tol:
            out[J] = v
    return out


def even_series_ylm(ell: int, m: int, r1, r2, K: int) -> np.ndarray:
    """Symmetric parity-even expansion of Y_ell^m(hat(r1 + r2)) to even alpha <= K (Appendix D boxed):
    Y = 1/2 sum Phi Y_J1^M(hat Delta) [eps1^alpha Y_J2^{m-M}(hat r1) + eps2^alpha Y_J2^{m-M}(hat r2)]."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    D = r2 - r1
    e1 = np.linalg.norm(D, axis=-1) / (2 * np.linalg.norm(r1, axis=-1))
    e2 = np.linalg.norm(D, axis=-1) / (2 * np.linalg.norm(r2, axis=-1))
    out = np.zeros(e1.shape, dtype=np.complex128)
    for alpha in range(0, K + 1, 2):
        for (J1, J2, M), c in Phi_table(alpha, ell, m).items():
            out += 0.5 * c * ylm(J1, M, D) * (e1 ** alpha * ylm(J2, m - M, r1) + e2 ** alpha * ylm(J2, m - M, r2))
    return out


def even_series_legendre(ell: int, r1, r2, K: int) -> np.ndarray:
    """Symmetric parity-even expansion of L_ell(hat Delta . hat(r1 + r2)) to even alpha <= K:
    1/2 sum (2J+1)/(2ell+1) F [eps1^alpha L_J(mu1) + (-1)^(ell+J) eps2^alpha L_J(mu2)]."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    D = r2 - r1
    nD = np.linalg.norm(D, axis=-1)
    n1, n2 = np.linalg.norm(r1, axis=-1), np.linalg.norm(r2, axis=-1)
    mu1 = np.sum(D * r1, axis=-1) / (nD * n1)
    mu2 = np.sum(D * r2, axis=-1) / (nD * n2)
    e1, e2 = nD / (2 * n1), nD / (2 * n2)
    out = np.zeros(e1.shape)
    for alpha in range(0, K + 1, 2):
        for J, c in F_table(alpha, ell).items():
            w = 0.5 * (2 * J + 1) / (2 * ell + 1) * c
            out += w * (e1 ** alpha * legendre_L(J, mu1) + (-1) ** (ell + J) * e2 ** alpha * legendre_L(J, mu2))
    return out


# --------------------------------------------------------------------------
# B: bisector expansion (Appendix F)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def B(beta: int, ell: int, m: int, J1: int, J2: int, M: int) -> float:
    """B^{beta, ell m}_{J1 J2 M}, eq. B-def.

    2^-ell sum_{lam, mu} A_{ell m}^{lam mu} binom(-ell/2, beta) 2^-beta sum_n binom(beta, n)(-1)^(beta-n)
      sum_{L = n, n-2, ..} c~^L_n 4pi/(2L+1) (-1)^(M-mu-m)
      G^{mu (M-mu) (-M)}_{lam L J1} G^{(m-mu) (mu-M) (M-m)}_{(ell-lam) L J2}
    """
    if abs(m) > ell or abs(M) > J1 or abs(m - M) > J2 or J1 < 0 or J2 < 0:
        return 0.0
    gb = float(gen_binom(Fraction(-ell, 2), beta))
    if gb == 0.0:
        return 0.0
    total = 0.0
    for lam in range(0, ell + 1):
        for mu in range(-lam, lam + 1):
            A = solid_A(ell, m, lam, mu)
            if A == 0.0:
                continue
            for n in range(0, beta + 1):
                bn = binom(beta, n) * (-1) ** (beta - n)
                for L in range(n, -1, -2):
                    ct = float(legendre_inv_coeff(L, n))
                    if ct == 0.0:
                        continue
                    g1 = gaunt(lam, L, J1, mu, M - mu, -M)
                    if g1 == 0.0:
                        continue
                    g2 = gaunt(ell - lam, L, J2, m - mu, mu - M, M - m)
                    if g2 == 0.0:
                        continue
                    sign = -1.0 if (M - mu - m) % 2 else 1.0
                    total += (A * gb * 2.0 ** (-beta) * bn * ct * FOUR_PI / (2 * L + 1)
                              * sign * g1 * g2)
    return total * 2.0 ** (-ell)


def B_table(beta: int, ell: int, m: int, tol: float = 1e-13) -> dict:
    """Non-zero B^{beta, ell m}_{J1 J2 M} with 0 <= J1, J2 <= ell+beta, |M| <= J1 (eq. bisector-ylm-expan)."""
    out = {}
    for J1 in range(0, ell + beta + 1):
        for J2 in range(0, ell + beta + 1):
            for M in range(-J1, J1 + 1):
                v = B(beta, ell, m, J1, J2, M)
                if abs(v) > tol:
                    out[(J1, J2, M)] = v
    return out


def bisector_series_ylm(ell: int, m: int, r1, r2, beta_max: int) -> np.ndarray:
    """Truncated eq. bisector-ylm-expan: sum_{beta<=beta_max} B Y_J1^M(hat r1) Y_J2^{m-M}(hat r2)."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    out = np.zeros(r1.shape[:-1], dtype=np.complex128)
    for beta in range(beta_max + 1):
        for (J1, J2, M), c in B_table(beta, ell, m).items():
            out = out + c * ylm(J1, M, r1) * ylm(J2, m - M, r2)
    return out

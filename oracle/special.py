"""Special functions and coupling symbols (Appendix A of arXiv:2102.08384).

Test infrastructure only (see ``oracle/__init__``).

Parity pins (tests/test_oracle_special.py):
  * legendre_coeff / legendre_inv_coeff: forward-inverse identity
    (eq. leg-forward-reverse-relation) and numpy's Legendre module.
  * gegenbauer_coeff: the generating function (eq. gegenbauer-generator),
    summed numerically.
  * ylm: orthonormality by quadrature, addition theorem (eq. addition-theorem),
    the symmetries stated after it.
  * gaunt: product-to-sum rule (eq. spherical-harmonic-prod-to-sum) at random
    points.
  * solid_A: the solid-harmonic addition theorem (eq. solid-harmonic-addition)
    in the form of eq. solid-harm-application, at random points.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
from scipy.special import sph_harm_y
from sympy.physics.wigner import wigner_3j as _sympy_w3j

FOUR_PI = 4.0 * math.pi


# --------------------------------------------------------------------------
# integer helpers
# --------------------------------------------------------------------------
def binom(n: int, k: int) -> int:
    """Ordinary binomial coefficient, zero outside 0 <= k <= n."""
    if k < 0 or n < 0 or k > n:
        return 0
    return math.comb(n, k)


def gen_binom(a: Fraction, k: int) -> Fraction:
    """Generalised binomial coefficient (a choose k) = (a)_k / k! with the
    falling factorial, as used for binom(-ell/2, beta) in Appendix F."""
    out = Fraction(1)
    for i in range(k):
        out *= (a - i)
    return out / math.factorial(k)


def double_factorial(n: int) -> int:
    """n!! for n >= -1 (with 0!! = (-1)!! = 1)."""
    if n <= 0:
        return 1
    out = 1
    while n > 0:
        out *= n
        n -= 2
    return out


def pochhammer_rising(a: Fraction, j: int) -> Fraction:
    """Rising factorial (a)_j = Gamma(a+j)/Gamma(a)."""
    out = Fraction(1)
    for i in range(j):
        out *= (a + i)
    return out


# --------------------------------------------------------------------------
# Legendre polynomial coefficients (eqs. Leg-polynomial-def, -inv-def)
# --------------------------------------------------------------------------
def legendre_coeff(ell: int, n: int) -> Fraction:
    """c_ell^n of eq. Leg-polynomial-def: L_ell(mu) = sum_n c_ell^n mu^(ell-2n)."""
    if n < 0 or 2 * n > ell:
        return Fraction(0)
    return Fraction((-1) ** n * math.factorial(2 * ell - 2 * n),
                    2 ** ell * math.factorial(n) * math.factorial(ell - n)
                    * math.factorial(ell - 2 * n))


def legendre_inv_coeff(ell: int, n: int) -> Fraction:
    """c~_n^ell of eq. Leg-polynomial-inv-def: mu^n = sum_{ell=n,n-2,..} c~_n^ell L_ell(mu).

    Uses the integer (double-factorial) right-hand form of that equation;
    zero unless 0 <= ell <= n and n - ell even."""
    if ell < 0 or ell > n or (n - ell) % 2:
        return Fraction(0)
    return Fraction((2 * ell + 1) * math.factorial(n) * double_factorial(ell + n + 2),
                    math.factorial(ell + n + 2) * double_factorial(n - ell))


def gegenbauer_coeff(alpha: Fraction, N: int, k: int) -> Fraction:
    """C_{Nk}^alpha of eq. gegenbauer-explicit:
    C_N^(alpha)(s) = sum_k C_{Nk}^alpha (2s)^(N-2k),
    C_{Nk}^alpha = (-1)^k Gamma(alpha+N-k) / (Gamma(alpha) k! (N-2k)!),
    with C_{Nk}^0 = delta_{N0} (the stated special case)."""
    if k < 0 or 2 * k > N:
        return Fraction(0)
    alpha = Fraction(alpha)
    if alpha == 0:
        return Fraction(1) if N == 0 else Fraction(0)
    return ((-1) ** k * pochhammer_rising(alpha, N - k)
            / (math.factorial(k) * math.factorial(N - 2 * k)))


def legendre_L(ell: int, mu):
    """L_ell(mu) summed from the explicit coefficients c_ell^n."""
    mu = np.asarray(mu, dtype=np.float64)
    out = np.zeros_like(mu)
    for n in range(ell // 2 + 1):
        out = out + float(legendre_coeff(ell, n)) * mu ** (ell - 2 * n)
    return out


# --------------------------------------------------------------------------
# Wigner 3-j, Gaunt, solid-harmonic coupling
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def w3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """Wigner 3-j symbol (sympy's exact value, as a float)."""
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3 or m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    return float(_sympy_w3j(j1, j2, j3, m1, m2, m3))


@lru_cache(maxsize=None)
def gaunt(l1: int, l2: int, l3: int, m1: int, m2: int, m3: int) -> float:
    """Gaunt integral of eq. Gaunt-3j-def:
    G^{l1 l2 l3}_{m1 m2 m3} = sqrt((2l1+1)(2l2+1)(2l3+1)/4pi)
                              (l1 l2 l3; m1 m2 m3)(l1 l2 l3; 0 0 0)."""
    if min(l1, l2, l3) < 0:
        return 0.0
    t0 = w3j(l1, l2, l3, 0, 0, 0)
    if t0 == 0.0:
        return 0.0
    t = w3j(l1, l2, l3, m1, m2, m3)
    if t == 0.0:
        return 0.0
    return math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / FOUR_PI) * t * t0


@lru_cache(maxsize=None)
def solid_A(ell: int, m: int, lam: int, mu: int) -> float:
    """A_{ell m}^{lam mu} of eq. solid-harm-application:
    sqrt(4pi(2ell+1)/((2lam+1)(2ell-2lam+1))) * binom(ell+m, lam+mu)^1/2 binom(ell-m, lam-mu)^1/2."""
    if lam < 0 or lam > ell or abs(mu) > lam or abs(m - mu) > ell - lam:
        return 0.0
    b = binom(ell + m, lam + mu) * binom(ell - m, lam - mu)
    if b == 0:
        return 0.0
    return math.sqrt(FOUR_PI * (2 * ell + 1) / ((2 * lam + 1) * (2 * ell - 2 * lam + 1))) * math.sqrt(b)


# --------------------------------------------------------------------------
# complex spherical harmonics (DLMF 14.30 with Condon-Shortley phase)
# --------------------------------------------------------------------------
def direction_angles(v):
    """(theta, phi, zero) of the vectors v[..., 3]: polar and azimuthal angles, and a flag
    for the zero vector (which has no direction; its angles are set to 0)."""
    v = np.asarray(v, dtype=np.float64)
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    theta = np.arccos(np.clip(z / rs, -1.0, 1.0))
    phi = np.arctan2(y, x)
    return theta, phi, zero


def ylm_angles(ell: int, m: int, theta, phi, zero) -> np.ndarray:
    """Complex Y_ell^m at polar angles (theta, phi), scipy.special.sph_harm_y (DLMF
    convention, Condon-Shortley phase).  Where ``zero`` is set (the zero vector) the value is
    Y_ell^m(0) = delta_{ell0}/sqrt(4pi), the only choice under which the series below stay
    exact at zero separation."""
    if abs(m) > ell:
        return np.zeros(np.shape(theta), dtype=np.complex128)
    out = sph_harm_y(ell, m, theta, phi).astype(np.complex128)
    if np.any(zero):
        out = np.where(zero, (1.0 / math.sqrt(FOUR_PI)) if ell == 0 else 0.0, out)
    return out


def ylm(ell: int, m: int, v) -> np.ndarray:
    """Complex Y_ell^m of the direction of the vectors v[..., 3] (``ylm_angles`` of
    ``direction_angles``)."""
    return ylm_angles(ell, m, *direction_angles(v))

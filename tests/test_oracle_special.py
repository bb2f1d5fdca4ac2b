"""Pins of oracle.special against identities of Appendix A and textbook routines."""
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.special import eval_gegenbauer

from oracle.special import (gaunt, gegenbauer_coeff, legendre_L, legendre_coeff,
                            legendre_inv_coeff, solid_A, ylm)


def test_legendre_forward_inverse_identity():
    # eq. leg-forward-reverse-relation: sum_n c_ell^n c~^L_{ell-2n} = delta_{ell L}
    for ell in range(0, 13):
        for L in range(0, 13):
            s = sum(legendre_coeff(ell, n) * legendre_inv_coeff(L, ell - 2 * n)
                    for n in range(ell // 2 + 1))
            assert s == (1 if ell == L else 0)


def test_legendre_against_numpy():
    mu = np.linspace(-1, 1, 41)
    for ell in range(0, 13):
        c = np.zeros(ell + 1)
        c[ell] = 1
        np.testing.assert_allclose(legendre_L(ell, mu), npleg.legval(mu, c), atol=1e-12)


def test_power_to_legendre():
    # eq. Leg-polynomial-inv-def: mu^n = sum_ell c~_n^ell L_ell(mu)
    mu = np.linspace(-1, 1, 37)
    for n in range(0, 12):
        s = sum(float(legendre_inv_coeff(ell, n)) * legendre_L(ell, mu) for ell in range(n, -1, -2))
        np.testing.assert_allclose(s, mu ** n, atol=1e-12)


@pytest.mark.parametrize("alpha", [Fraction(1, 2), Fraction(1), Fraction(3, 2), Fraction(2), Fraction(5, 2)])
def test_gegenbauer_explicit(alpha):
    # eq. gegenbauer-explicit against scipy's Gegenbauer polynomials
    s = np.linspace(-1, 1, 23)
    for N in range(0, 10):
        v = sum(float(gegenbauer_coeff(alpha, N, k)) * (2 * s) ** (N - 2 * k) for k in range(N // 2 + 1))
        np.testing.assert_allclose(v, eval_gegenbauer(N, float(alpha), s), rtol=1e-11, atol=1e-11)


def test_gegenbauer_generating_function():
    # eq. gegenbauer-generator: (1 - 2 s t + t^2)^-alpha = sum_N C_N^(alpha)(s) t^N
    for alpha in (Fraction(1, 2), Fraction(2), Fraction(3, 2)):
        for s in (-0.7, 0.1, 0.9):
            t = 0.05
            series = sum(sum(float(gegenbauer_coeff(alpha, N, k)) * (2 * s) ** (N - 2 * k)
                             for k in range(N // 2 + 1)) * t ** N for N in range(0, 30))
            assert abs(series - (1 - 2 * s * t + t * t) ** (-float(alpha))) < 1e-13
    assert gegenbauer_coeff(0, 0, 0) == 1 and gegenbauer_coeff(0, 3, 1) == 0


def _sphere_quadrature(n=24):
    x, w = np.polynomial.legendre.leggauss(n)
    ph = np.arange(2 * n) * (2 * np.pi / (2 * n))
    T, P = np.meshgrid(np.arccos(x), ph, indexing="ij")
    W = np.repeat(w[:, None], 2 * n, axis=1) * (2 * np.pi / (2 * n))
    v = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    return v.reshape(-1, 3), W.ravel()


def test_ylm_orthonormal():
    # eq. spherical-harmonic-orthog by Gauss-Legendre x uniform quadrature (exact to degree 47)
    v, w = _sphere_quadrature()
    lms = [(l, m) for l in range(0, 7) for m in range(-l, l + 1)]
    Y = np.array([ylm(l, m, v) for l, m in lms])
    G = (Y * w) @ np.conj(Y).T
    np.testing.assert_allclose(G, np.eye(len(lms)), atol=1e-12)


def test_ylm_addition_theorem_and_symmetries():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(50, 3))
    b = rng.normal(size=(50, 3))
    mu = np.sum(a * b, axis=1) / np.linalg.norm(a, axis=1) / np.linalg.norm(b, axis=1)
    for ell in range(0, 9):
        s = sum(ylm(ell, m, a) * np.conj(ylm(ell, m, b)) for m in range(-ell, ell + 1))
        np.testing.assert_allclose(4 * np.pi / (2 * ell + 1) * s, legendre_L(ell, mu), atol=1e-12)
        for m in range(-ell, ell + 1):
            np.testing.assert_allclose(ylm(ell, m, -a), (-1) ** ell * ylm(ell, m, a), atol=1e-13)
            np.testing.assert_allclose(np.conj(ylm(ell, m, a)), (-1) ** m * ylm(ell, -m, a), atol=1e-13)
    np.testing.assert_allclose(ylm(0, 0, a), 1 / math.sqrt(4 * math.pi))
    # zero vector reading
    z = np.zeros((1, 3))
    assert ylm(0, 0, z)[0] == pytest.approx(1 / math.sqrt(4 * math.pi))
    assert ylm(2, 1, z)[0] == 0


def test_gaunt_product_to_sum():
    # eq. spherical-harmonic-prod-to-sum at random points
    rng = np.random.default_rng(4)
    v = rng.normal(size=(30, 3))
    for (L1, M1, L2, M2) in [(1, 1, 1, 0), (2, -1, 3, 2), (2, 2, 2, -2), (4, 3, 3, -1), (0, 0, 5, 4)]:
        lhs = ylm(L1, M1, v) * ylm(L2, M2, v)
        rhs = np.zeros(len(v), dtype=complex)
        for L3 in range(abs(L1 - L2), L1 + L2 + 1):
            for M3 in range(-L3, L3 + 1):
                c = gaunt(L1, L2, L3, M1, M2, -M3)
                if c:
                    rhs += c * (-1) ** M3 * ylm(L3, M3, v)
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_solid_harmonic_addition():
    # eq. solid-harm-application (finite series) at random points
    rng = np.random.default_rng(5)
    a = rng.normal(size=(40, 3))
    A = rng.normal(size=(40, 3)) * 3
    eps = np.linalg.norm(a, axis=1) / np.linalg.norm(A, axis=1)
    Ahat = A / np.linalg.norm(A, axis=1)[:, None]
    ahat = a / np.linalg.norm(a, axis=1)[:, None]
    den = np.linalg.norm(Ahat + eps[:, None] * ahat, axis=1)
    for ell in range(0, 6):
        for m in range(-ell, ell + 1):
            rhs = np.zeros(len(a), dtype=complex)
            for lam in range(ell + 1):
                for mu in range(-lam, lam + 1):
                    c = solid_A(ell, m, lam, mu)
                    if c:
                        rhs += c * eps ** lam / den ** ell * ylm(lam, mu, a) * ylm(ell - lam, m - mu, A)
            np.testing.assert_allclose(rhs, ylm(ell, m, a + A), atol=1e-12)

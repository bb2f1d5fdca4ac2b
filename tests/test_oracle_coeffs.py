"""Pins of the oracle's series coefficients (phi, f, B) against what the paper fixes."""
import math

import numpy as np
import pytest
import sympy as sp

from conftest import load_golden
from oracle.coeffs import (B, B_table, bisector_series_ylm, f_leg, f_table, phi, phi_table,
                           shift_series_legendre, shift_series_ylm)
from oracle.special import legendre_L, solid_A, ylm

S4PI = math.sqrt(4 * math.pi)


# ---------------------------------------------------------------- printed examples
def test_phi_matches_printed_Y21_example():
    gold = {k: v for k, v in load_golden("phi_Y21_midpoint.txt")}
    for alpha in range(3):
        tab = phi_table(alpha, 2, 1)
        keys = {(J1, J2, M) for (a, J1, J2, M) in gold if a == alpha}
        assert set(tab) == keys, (alpha, sorted(set(tab) ^ keys))
        for (J1, J2, M) in keys:
            assert tab[(J1, J2, M)] == pytest.approx(gold[(alpha, J1, J2, M)], rel=1e-12)


def test_f_matches_printed_L2_example():
    gold = {k: v for k, v in load_golden("f_L2_midpoint.txt")}
    for alpha in range(5):
        tab = f_table(alpha, 2)
        keys = {J for (a, J) in gold if a == alpha}
        assert set(tab) == keys
        for J in keys:
            assert (2 * J + 1) / 5 * tab[J] == pytest.approx(gold[(alpha, J)], rel=1e-12)


def test_B_matches_printed_Y21_example():
    gold = {k: v for k, v in load_golden("B_Y21_bisector.txt")}
    for beta in range(2):
        tab = B_table(beta, 2, 1)
        keys = {(J1, J2, M) for (b, J1, J2, M) in gold if b == beta}
        assert set(tab) == keys, (beta, sorted(set(tab) ^ keys))
        for k in keys:
            assert tab[k] == pytest.approx(gold[(beta,) + k], rel=1e-12)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("ell", [0, 1, 2, 3, 4])
def test_phi_closed_forms(ell):
    # eq. shift-coeff-alpha-zero and the ell = m = 0 case of Appendix B
    for m in range(-ell, ell + 1):
        assert phi_table(0, ell, m) == pytest.approx({(0, ell, 0): S4PI})
    for alpha in range(0, 5):
        t = phi_table(alpha, 0, 0)
        assert t == (pytest.approx({(0, 0, 0): S4PI}) if alpha == 0 else {})


def test_f_closed_forms():
    # Appendix E: f^{0,ell}_J = delta_{ell J}; f^{alpha,0}_J = delta_{alpha 0} delta_{J 0}
    for ell in range(0, 7):
        for J in range(0, 9):
            assert f_leg(0, ell, J) == pytest.approx(1.0 if J == ell else 0.0, abs=1e-13)
    for alpha in range(0, 6):
        for J in range(0, 7):
            assert f_leg(alpha, 0, J) == pytest.approx(1.0 if (alpha == 0 and J == 0) else 0.0, abs=1e-13)


def test_B_closed_forms():
    # eq. B-coeff-k=0 and eq. B-coeff-ell=0
    for ell in range(0, 5):
        for m in range(-ell, ell + 1):
            for J1 in range(0, ell + 1):
                for J2 in range(0, ell + 1):
                    for M in range(-J1, J1 + 1):
                        want = 2.0 ** (-ell) * solid_A(ell, m, J1, M) if J2 == ell - J1 else 0.0
                        assert B(0, ell, m, J1, J2, M) == pytest.approx(want, abs=1e-13)
    # eq. B-coeff-ell=0 prints sqrt(4pi) delta delta delta without the delta_{beta 0} that its
    # own step binom(0, beta) = delta_{beta 0} gives; with it Y_0^0(hat d) = 1/sqrt(4pi) exactly.
    for beta in range(0, 4):
        t = B_table(beta, 0, 0)
        assert t == (pytest.approx({(0, 0, 0): S4PI}) if beta == 0 else {})


# ---------------------------------------------------------------- selection rules
def test_selection_rules():
    # phi vanishes unless alpha+J1 and ell+alpha+J2 are even (eq. varphi-relations-main-text)
    for alpha in range(0, 5):
        for ell in range(0, 5):
            for m in range(0, ell + 1):
                for (J1, J2, M) in phi_table(alpha, ell, m):
                    assert (alpha + J1) % 2 == 0 and (ell + alpha + J2) % 2 == 0
                    assert J1 <= alpha and max(0, ell - alpha) <= J2 <= ell + alpha
    # f vanishes unless alpha+ell+J even (Appendix E)
    for alpha in range(0, 6):
        for ell in range(0, 7):
            for J in f_table(alpha, ell):
                assert (alpha + ell + J) % 2 == 0
    # B vanishes if ell+J1+J2 odd (eq. Bk-properties)
    for beta in range(0, 3):
        for ell in range(0, 5):
            for m in range(0, ell + 1):
                for (J1, J2, M) in B_table(beta, ell, m):
                    assert (ell + J1 + J2) % 2 == 0


def test_f_sum_rule():
    # Appendix E: putting A parallel to a gives 1 = sum_alpha sum_J (2J+1)/(2ell+1) f k^-alpha,
    # so the weighted sum vanishes for every alpha > 0 (the printed eq. L2-all, L24-even
    # coefficients show the same); the (2J+1) weight is the reading of the garbled statement.
    for ell in range(0, 7):
        for alpha in range(1, 7):
            s = sum((2 * J + 1) * v for J, v in f_table(alpha, ell).items())
            assert abs(s) < 1e-10


# ---------------------------------------------------------------- truncation error rates
def _rand_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("ell,m", [(2, 1), (2, -2), (4, 0), (4, 3)])
def test_phi_series_convergence_rate(ell, m):
    # truncating eq. Ylm-shift-theorem at alpha = K leaves O(eps^(K+1))
    rng = np.random.default_rng(10 + ell + m)
    ah, Ah = _rand_unit(rng, 6), _rand_unit(rng, 6) * 2.0
    e0 = 0.02
    for K in range(0, 5):
        err = []
        for e in (e0, e0 / 2):
            a = ah * e * 2.0
            exact = ylm(ell, m, a + Ah)
            err.append(np.abs(exact - shift_series_ylm(ell, m, a, Ah, K)))
        ratio = np.median(err[0] / err[1])
        assert 0.8 * 2 ** (K + 1) < ratio < 1.25 * 2 ** (K + 1), (K, ratio)


@pytest.mark.parametrize("ell", [2, 4])
def test_f_series_convergence_rate(ell):
    rng = np.random.default_rng(20 + ell)
    ah, Ah = _rand_unit(rng, 6), _rand_unit(rng, 6)
    for K in range(0, 5):
        err = []
        for e in (0.02, 0.01):
            a = ah * e
            mu = np.sum(ah * (a + Ah), axis=1) / np.linalg.norm(a + Ah, axis=1)
            err.append(np.abs(legendre_L(ell, mu) - shift_series_legendre(ell, a, Ah, K)))
        ratio = np.median(err[0] / err[1])
        assert 0.8 * 2 ** (K + 1) < ratio < 1.25 * 2 ** (K + 1), (K, ratio)


@pytest.mark.parametrize("ell,m", [(2, 1), (4, 2), (4, -4)])
def test_B_series_convergence_rate(ell, m):
    # truncating eq. bisector-ylm-expan at beta leaves O((1 - cos phi)^(beta+1)) = O(theta^(2beta+2))
    rng = np.random.default_rng(30 + ell + m)
    p = _rand_unit(rng, 6)
    u = _rand_unit(rng, 6)
    u = u - np.sum(u * p, axis=1)[:, None] * p
    u /= np.linalg.norm(u, axis=1)[:, None]
    for beta in range(0, 3):
        err = []
        for t in (0.08, 0.04):
            r1 = (p + t * u) * 900.0
            r2 = (p - t * u) * 1300.0
            d = r1 / np.linalg.norm(r1, axis=1)[:, None] + r2 / np.linalg.norm(r2, axis=1)[:, None]
            err.append(np.abs(ylm(ell, m, d) - bisector_series_ylm(ell, m, r1, r2, beta)))
        ratio = np.median(err[0] / err[1])
        assert 0.75 * 4 ** (beta + 1) < ratio < 1.33 * 4 ** (beta + 1), (beta, ratio)


# ---------------------------------------------------------------- f by a second route
@pytest.mark.parametrize("ell", [2, 4])
def test_f_equals_direct_taylor_expansion(ell):
    # Sec. 4.1: the Legendre shift theorem also follows from a Taylor expansion of
    # L_ell(hat a . hat(a + A)) in eps = a/A; with mu = hat a . hat A,
    # hat a . hat(a+A) = (eps + mu)/sqrt(1 + 2 eps mu + eps^2).
    e, mu = sp.symbols("e mu")
    arg = (e + mu) / sp.sqrt(1 + 2 * e * mu + e ** 2)
    expr = sp.legendre(ell, arg)
    ser = sp.series(expr, e, 0, 5).removeO()
    pts = np.linspace(-0.95, 0.95, 13)
    for alpha in range(0, 5):
        coeff = sp.lambdify(mu, sp.expand(ser.coeff(e, alpha)), "numpy")
        want = np.broadcast_to(coeff(pts), pts.shape)
        got = sum((2 * J + 1) / (2 * ell + 1) * v * legendre_L(J, pts)
                  for J, v in f_table(alpha, ell).items())
        np.testing.assert_allclose(got, want, atol=1e-11)


# ---------------------------------------------------------------- parity-even midpoint (Appendices C, D, F.2)
def test_F_matches_printed_L24_even():
    from oracle.coeffs import F_table
    gold = {k: v for k, v in load_golden("F_L24_even.txt")}
    for ell in (2, 4):
        for alpha in (0, 2, 4):
            tab = F_table(alpha, ell)
            keys = {J for (l, a, J) in gold if l == ell and a == alpha}
            assert set(tab) == keys, (ell, alpha, sorted(set(tab) ^ keys))
            for J in keys:
                assert (2 * J + 1) / (2 * ell + 1) * tab[J] == pytest.approx(gold[(ell, alpha, J)], rel=1e-11)


def test_Phi_matches_printed_Y21_even():
    # eq. Y21-even: the second-order terms are those of eq. Y21-all with the opposite sign
    # (Phi^2 = -phi^2, Appendix D); the zeroth-order term is unchanged and alpha = 1 is absent
    from oracle.coeffs import Phi_table
    gold = {k: v for k, v in load_golden("phi_Y21_midpoint.txt")}
    assert Phi_table(0, 2, 1) == pytest.approx({(0, 2, 0): S4PI})
    tab = Phi_table(2, 2, 1)
    keys = {(J1, J2, M) for (a, J1, J2, M) in gold if a == 2}
    assert set(tab) == keys
    for k in keys:
        assert tab[k] == pytest.approx(-gold[(2,) + k], rel=1e-12)
    assert Phi_table(1, 2, 1) == {} and Phi_table(3, 2, 1) == {}


@pytest.mark.parametrize("ell,m", [(2, 1), (4, 2), (4, -3)])
def test_even_Ylm_series_convergence_rate(ell, m):
    # the boxed parity-even expansion truncated at even alpha = K leaves O(theta^(K+2));
    # Phi^4 (built from Omega) must give the theta^6 rate
    from oracle.coeffs import even_series_ylm
    rng = np.random.default_rng(40 + ell + m)
    R = _rand_unit(rng, 6) * 1000.0
    d = _rand_unit(rng, 6)
    for K in (0, 2, 4):
        err = []
        for D in (40.0, 20.0):
            r1, r2 = R - 0.5 * D * d, R + 0.5 * D * d
            err.append(np.abs(ylm(ell, m, r1 + r2) - even_series_ylm(ell, m, r1, r2, K)))
        ratio = np.median(err[0] / err[1])
        assert 0.85 * 4 ** (K // 2 + 1) < ratio < 1.15 * 4 ** (K // 2 + 1), (K, ratio)


@pytest.mark.parametrize("ell", [2, 4])
def test_even_legendre_series_convergence_rate(ell):
    from oracle.coeffs import even_series_legendre
    rng = np.random.default_rng(50 + ell)
    R = _rand_unit(rng, 6) * 1000.0
    d = _rand_unit(rng, 6)
    for K in (0, 2, 4):
        err = []
        for D in (40.0, 20.0):
            r1, r2 = R - 0.5 * D * d, R + 0.5 * D * d
            mu = np.sum(d * (r1 + r2), axis=1) / np.linalg.norm(r1 + r2, axis=1)
            err.append(np.abs(legendre_L(ell, mu) - even_series_legendre(ell, r1, r2, K)))
        ratio = np.median(err[0] / err[1])
        assert 0.85 * 4 ** (K // 2 + 1) < ratio < 1.15 * 4 ** (K // 2 + 1), (K, ratio)

"""Brute-force pair sums: the exact pairwise-LOS estimators (no series).

Test infrastructure only (see ``oracle/__init__``).

* O2, ``mesh_pk`` / ``mesh_xi``: every ordered pair of occupied mesh nodes
  (a, b) with lag Delta = minimal-image(x_b - x_a) and the exact line of sight
  of Sec. 2 (eq. P-ell-midpoint-init, eq. 2pcf-pair):
      yamamoto  n = hat x_b                         (eq. Yamamoto-estimator)
      midpoint  n = hat(x_a + x_b)
      bisector  n = hat(hat x_a + hat x_b)
  P_ell(k) = 4 pi / A mean_shell Re sum_m Y_ell^m*(k) DFT[G_ell^m](k) with
  G_ell^m(Delta) = sum_{pairs at Delta} delta_a delta_b Y_ell^m(n)  (addition
  theorem, eq. addition-theorem); xi_ell(r_b) = (2 ell + 1) / (A V_cell N_b)
  sum_{pairs, |Delta| in b, Delta != 0} delta_a delta_b L_ell(hat Delta . n).
  With ``series=K`` the exact Y_ell^m(n) / L_ell(hat Delta . n) is replaced by
  its truncated expansion taken pair by pair (midpoint: eq. Ylm-shift-theorem
  around A = 2 x_b, a = -Delta, and eq. Legendre-shift-theorem-all-parity;
  bisector: eq. bisector-ylm-expan and eq. bisector-leg-expan).
* Cross spectra (``gal_b``, ``ran_b``, ``ran_nbar_b`` given): the pairs join an
  occupied node a of delta_A to an occupied node b of delta_B, weight
  delta_A(a) delta_B(b), lag Delta = x_b - x_a, normalisation sqrt(A_A A_B).  With
  two densities the anchored forms are not interchangeable, so every pair takes the
  mean of both: Yamamoto the mean of the two endpoint lines of sight, the midpoint
  series the mean of its expansions anchored at x_b and at x_a (Sec. 3.2, the
  bracket before the symmetrisation of eq. P-ell-k-symm); the bisector series is
  symmetric in the pair already.
* O1, ``particle_xi``: the same xi_ell sum over distinct particle pairs
  (weights w and -alpha_r w), no mesh, no periodic wrap; binned with the mesh
  lag-cell counts N_b so that node-snapped catalogs give O2 exactly.

Pins: tests/test_oracle_estimators.py (O1 == O2 on node-snapped CIC
catalogs; O2 with the truncated series == the FFT estimators to rounding).
"""
from __future__ import annotations

import numpy as np

from . import mesh
from .coeffs import B_table, F_table, Phi_table, f_table, phi_table
from .special import FOUR_PI, legendre_L, ylm


def _occupied(delta, N, box_lo, box_len):
    idx = np.argwhere(delta != 0.0)
    h = box_len / N
    x = np.asarray(box_lo, dtype=np.float64)[None, :] + idx * h
    return idx, x, delta[delta != 0.0]


def _pairs(idx, x, d, N, box_len, idx_b=None, d_b=None):
    """Every ordered pair (a, b) of occupied nodes (a of the first density, b of the
    second; one density: both of it)."""
    if idx_b is None:
        idx_b, d_b = idx, d
    ia = np.repeat(np.arange(len(d)), len(d_b))
    ib = np.tile(np.arange(len(d_b)), len(d))
    j = (idx_b[ib] - idx[ia] + N // 2) % N - N // 2       # minimal-image lag labels
    lag = j * (box_len / N)
    flat = np.ravel_multi_index(tuple((j % N).T), (N, N, N))
    return ia, ib, lag, flat, d[ia] * d_b[ib]


def _densities(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len, assign, norm):
    """Occupied nodes of delta_A (and delta_B for a cross spectrum) and the
    normalisation A (cross: sqrt(A_A A_B))."""
    delta, _ = mesh.density_mesh(gal, ran, N, box_lo, box_len, assign)
    A = mesh.norm_factors(gal, ran, ran_nbar)[1] if norm else 1.0
    a = _occupied(delta, N, box_lo, box_len)
    if gal_b is None:
        return a, None, A
    delta_b, _ = mesh.density_mesh(gal_b, ran_b, N, box_lo, box_len, assign)
    if norm:
        A = float(np.sqrt(A * mesh.norm_factors(gal_b, ran_b, ran_nbar_b)[1]))
    return a, _occupied(delta_b, N, box_lo, box_len), A


def _unit(v):
    n = np.linalg.norm(v, axis=-1, keepdims=True)
    return v / np.where(n == 0.0, 1.0, n)


def _los(los, xa, xb):
    if los == "yamamoto":
        return xb
    if los in ("midpoint", "midpoint_even"):
        return xa + xb
    if los == "bisector":
        return _unit(xa) + _unit(xb)
    raise ValueError(los)


def _ylm_pair(los, ell, m, xa, xb, lag, series, both=False):
    """Y_ell^m of the pair's line of sight, exact or its truncated series.  both:
    the mean over the two anchorings (Yamamoto: over the two endpoints; midpoint:
    over the expansions about x_b and about x_a, found by swapping the ends, which
    turns Delta into -Delta)."""
    if both and los in ("yamamoto", "midpoint", "midpoint_even"):
        if los == "yamamoto":
            return 0.5 * (ylm(ell, m, xb) + ylm(ell, m, xa))
        if series is not None:
            return 0.5 * (_ylm_pair(los, ell, m, xa, xb, lag, series)
                          + _ylm_pair(los, ell, m, xb, xa, -lag, series))
    if series is None or los == "yamamoto":
        return ylm(ell, m, _los(los, xa, xb))
    if los == "midpoint":
        # R = x_a + x_b = 2 x_b - Delta: a = -Delta, A = 2 x_b (eq. Ylm-shift-theorem)
        eps = np.linalg.norm(lag, axis=-1) / (2.0 * np.linalg.norm(xb, axis=-1))
        out = np.zeros(len(xb), dtype=np.complex128)
        for alpha in range(series + 1):
            for (J1, J2, M), c in phi_table(alpha, ell, m).items():
                out += c * eps ** alpha * ylm(J1, M, -lag) * ylm(J2, m - M, xb)
        return out
    if los == "midpoint_even":
        # r2-anchored parity-even series (Phi, even alpha): its pair sum equals that of the
        # symmetric boxed form because every J1 is even
        eps = np.linalg.norm(lag, axis=-1) / (2.0 * np.linalg.norm(xb, axis=-1))
        out = np.zeros(len(xb), dtype=np.complex128)
        for alpha in range(0, series + 1, 2):
            for (J1, J2, M), c in Phi_table(alpha, ell, m).items():
                out += c * eps ** alpha * ylm(J1, M, -lag) * ylm(J2, m - M, xb)
        return out
    if los == "bisector":
        out = np.zeros(len(xb), dtype=np.complex128)
        for beta in range(series // 2 + 1):
            for (J1, J2, M), c in B_table(beta, ell, m).items():
                out += c * ylm(J1, M, xa) * ylm(J2, m - M, xb)
        return out
    raise ValueError(los)


def _legendre_pair(los, ell, xa, xb, lag, series, both=False):
    """L_ell(hat Delta . n) of the pair, exact or its truncated series (both: as in
    ``_ylm_pair``; swapping the ends turns Delta into -Delta, so the swapped term takes
    (-1)^ell to stay L_ell of the pair's own Delta)."""
    if both and los in ("yamamoto", "midpoint", "midpoint_even"):
        sgn = (-1) ** ell
        if los == "yamamoto":
            return 0.5 * (_legendre_pair(los, ell, xa, xb, lag, None)
                          + sgn * _legendre_pair(los, ell, xb, xa, -lag, None))
        if series is not None:
            return 0.5 * (_legendre_pair(los, ell, xa, xb, lag, series)
                          + sgn * _legendre_pair(los, ell, xb, xa, -lag, series))
    if series is None or los == "yamamoto":
        n = _unit(_los(los, xa, xb))
        mu = np.sum(_unit(lag) * n, axis=-1)
        return legendre_L(ell, mu)
    if los == "midpoint":
        # L_ell(hat Delta . hat R) = (-1)^ell L_ell(hat a . hat(a + A)), a = -Delta, A = 2 x_b
        eps = np.linalg.norm(lag, axis=-1) / (2.0 * np.linalg.norm(xb, axis=-1))
        mu = np.sum(_unit(-lag) * _unit(xb), axis=-1)
        out = np.zeros(len(xb))
        for alpha in range(series + 1):
            for J, c in f_table(alpha, ell).items():
                out += (2 * J + 1) / (2 * ell + 1) * c * eps ** alpha * legendre_L(J, mu)
        return (-1) ** ell * out
    if los == "midpoint_even":
        if ell % 2:
            raise ValueError("the parity-even midpoint form is defined for even ell")
        eps = np.linalg.norm(lag, axis=-1) / (2.0 * np.linalg.norm(xb, axis=-1))
        mu = np.sum(_unit(-lag) * _unit(xb), axis=-1)
        out = np.zeros(len(xb))
        for alpha in range(0, series + 1, 2):
            for J, c in F_table(alpha, ell).items():
                out += (2 * J + 1) / (2 * ell + 1) * c * eps ** alpha * legendre_L(J, mu)
        return out
    if los == "bisector":
        # eq. bisector-leg-expan
        out = np.zeros(len(xb), dtype=np.complex128)
        for m in range(-ell, ell + 1):
            out += np.conj(ylm(ell, m, lag)) * _ylm_pair(los, ell, m, xa, xb, lag, series)
        return (FOUR_PI / (2 * ell + 1) * out).real
    raise ValueError(los)


def mesh_pk(gal, ran, ran_nbar, *, N, box_lo, box_len, assign, ell_max, los, kedges,
            norm=1, series=None, gal_b=None, ran_b=None, ran_nbar_b=None, odd=False):
    """O2 power-spectrum multipoles from explicit pairs of occupied nodes (cross
    spectrum of two tracers when gal_b is given); with odd, every ell <= ell_max, odd
    ell as the imaginary part of the shell mean (real densities make it imaginary)."""
    (idx, x, d), other, A = _densities(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len,
                                       assign, norm)
    both = other is not None
    idx_b, x_b, d_b = other if both else (idx, x, d)
    ia, ib, lag, flat, w = _pairs(idx, x, d, N, box_len, idx_b, d_b)
    xa, xb = x[ia], x_b[ib]
    kv = mesh.k_vectors(N, box_len)
    kmag = mesh.k_magnitude(N, box_len)
    ells = list(range(0, ell_max + 1, 1 if odd else 2))
    pk, kmean, cnt = [], None, None
    for ell in ells:
        acc = np.zeros((N, N, N), dtype=np.complex128)
        for m in range(-ell, ell + 1):
            G = np.zeros(N * N * N, dtype=np.complex128)
            np.add.at(G, flat, w * _ylm_pair(los, ell, m, xa, xb, lag, series, both))
            acc += np.conj(ylm(ell, m, kv)) * mesh.fftn(G.reshape(N, N, N))
        mean, kmean, cnt = mesh.shell_mean(acc.real if ell % 2 == 0 else acc.imag, kmag, kedges, kmag == 0.0)
        pk.append(FOUR_PI / A * mean)
    return {"ells": ells, "pk": np.array(pk), "k_mean": kmean, "n_modes": cnt}


def mesh_xi(gal, ran, ran_nbar, *, N, box_lo, box_len, assign, ell_max, los, redges,
            norm=1, series=None, gal_b=None, ran_b=None, ran_nbar_b=None, odd=False):
    """O2 correlation-function multipoles from explicit pairs of occupied nodes
    (cross correlation of two tracers when gal_b is given)."""
    (idx, x, d), other, A = _densities(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len,
                                       assign, norm)
    v_cell = (box_len / N) ** 3 if norm else 1.0
    both = other is not None
    idx_b, x_b, d_b = other if both else (idx, x, d)
    ia, ib, lag, flat, w = _pairs(idx, x, d, N, box_len, idx_b, d_b)
    lmag = np.linalg.norm(lag, axis=-1)
    redges = np.asarray(redges, dtype=np.float64)
    b = mesh.shell_index(lmag, redges)
    b[lmag == 0.0] = -1
    sel = b >= 0
    lagmag_grid = mesh.lag_magnitude(N, box_len)
    _, rmean, ncell = mesh.shell_mean(np.zeros_like(lagmag_grid), lagmag_grid, redges,
                                      lagmag_grid == 0.0)
    ells = list(range(0, ell_max + 1, 1 if odd else 2))
    nb = len(redges) - 1
    xi = []
    for ell in ells:
        L = _legendre_pair(los, ell, x[ia][sel], x_b[ib][sel], lag[sel], series, both)
        s = np.bincount(b[sel], weights=w[sel] * L, minlength=nb)
        xi.append(np.where(ncell > 0, (2 * ell + 1) * s / (A * v_cell * np.maximum(ncell, 1)), 0.0))
    return {"ells": ells, "xi": np.array(xi), "r_mean": rmean, "n_cells": ncell}


def particle_xi(gal, ran, ran_nbar, *, N, box_lo, box_len, ell_max, los, redges, norm=1):
    """O1: xi_ell from distinct particle pairs (eq. 2pcf-pair with the bin
    replacement of Sec. 2.2, bin volume v_b = N_b V_cell from the mesh)."""
    alpha, A = mesh.norm_factors(gal, ran, ran_nbar)
    parts = [np.asarray(gal, dtype=np.float64)]
    wts = [parts[0][:, 3]]
    if ran is not None and len(ran):
        r = np.asarray(ran, dtype=np.float64)
        parts.append(r)
        wts.append(-alpha * r[:, 3])
    p = np.concatenate(parts)[:, :3]
    w = np.concatenate(wts)
    if not norm:
        A, v_cell = 1.0, 1.0
    else:
        v_cell = (box_len / N) ** 3
    n = len(w)
    ia = np.repeat(np.arange(n), n)
    ib = np.tile(np.arange(n), n)
    keep = ia != ib
    ia, ib = ia[keep], ib[keep]
    lag = p[ib] - p[ia]
    lmag = np.linalg.norm(lag, axis=-1)
    redges = np.asarray(redges, dtype=np.float64)
    b = mesh.shell_index(lmag, redges)
    b[lmag == 0.0] = -1
    sel = b >= 0
    lagmag_grid = mesh.lag_magnitude(N, box_len)
    _, _, ncell = mesh.shell_mean(np.zeros_like(lagmag_grid), lagmag_grid, redges,
                                  lagmag_grid == 0.0)
    ells = list(range(0, ell_max + 1, 2))
    nb = len(redges) - 1
    xi = []
    for ell in ells:
        L = _legendre_pair(los, ell, p[ia][sel], p[ib][sel], lag[sel], None)
        s = np.bincount(b[sel], weights=(w[ia] * w[ib])[sel] * L, minlength=nb)
        xi.append(np.where(ncell > 0, (2 * ell + 1) * s / (A * v_cell * np.maximum(ncell, 1)), 0.0))
    return {"ells": ells, "xi": np.array(xi), "n_cells": ncell}

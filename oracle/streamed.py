"""The midpoint and bisector estimators in a loop order that holds few full grids (O3, FP64).

Test infrastructure only (see ``oracle/__init__``).

``oracle.estimators`` keeps every series field of a request in memory at once: on a 512^3
mesh in FP64 the 145 midpoint g functions of order 4 alone would take 310 GB.  This module
computes the same sums -- eq. FFT-midpoint with g from eq. g-JM-form, eq.
xi-parity-all-estimator, eq. bisector-pk-fft and the bisector correlation function of Sec. 6
-- from the same coefficient tables, painting, compensation, normalisation and binning, in
another order:

* a series field (2r)^-alpha Y_J^M(r) delta(r) is formed on the non-empty mesh nodes only
  (it is zero wherever delta is);
* midpoint P: the transform is linear, so F[H_ell^m] is the sum, over the terms of H_ell^m, of
  the transforms of the single products Y_J1^M(Delta) Delta^alpha g^alpha_{J2, m-M}(Delta).
  Each distinct product is transformed once and enters every (ell, m) that holds it with its
  coefficient phi and Y_ell^m*(k).  Products are visited in groups of equal (alpha, J1), whose
  2 J1 + 1 factors Y_J1^M(Delta) Delta^alpha are kept for the group; a g function is computed
  once per group that needs it;
* midpoint xi: the sum of f Y_J^M*(Delta) Delta^alpha g^alpha_JM is taken g by g, each g once;
* Yamamoto P and xi (eq. Yamamoto-estimator, eq. 2pcf-yama): one field F[Y_ell^m delta] at a
  time, its product with D*(k) contracted on the binned modes and, inverse-transformed, on the
  binned lags;
* bisector P and xi: the bilinear sum runs pair by pair over the (left, right) fields
  F[Y_J1^M delta](-k) and F[Y_J2^(m-M) delta](k), the left fields held in blocks and the right
  ones made one at a time; xi takes the inverse transform of each pair's product, whose sum
  over the pairs with their coefficients is the inverse transform of X_ell^m (linearity);
* P is evaluated only on the modes with |k| up to the last k edge and xi only on the lags
  with |Delta| up to the last r edge: no other mode or lag enters a bin.  Bins, counts and
  mean magnitudes come from ``mesh.shell_mean`` on those modes and lags, in the same order as
  on the full grid.

Elementwise work on full grids runs slab by slab along the first axis in a thread pool,
which changes no arithmetic.

Parity pin (tests/test_oracle_streamed.py): equal to ``oracle.estimators`` to 1e-12 for the
three lines of sight, orders 2 and 4, ell <= 4, P and xi, CIC and compensated TSC.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft

from . import mesh
from .coeffs import B_table, f_table, phi_table
from .special import FOUR_PI, direction_angles, ylm_angles


def _threads():
    return os.cpu_count() or 1


def _slabs(n, fn, threads):
    """fn(lo, hi) over slabs [lo, hi) of range(n), in a thread pool."""
    step = max(1, n // (4 * threads))
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda lo: fn(lo, min(lo + step, n)), range(0, n, step)))


def _fftn(a):
    return scipy.fft.fftn(a, workers=-1, overwrite_x=True)


def _ifftn(a):
    return scipy.fft.ifftn(a, workers=-1, overwrite_x=True)


class Stop(Exception):
    """Raised by a progress callback to end a run early (timing samples)."""


class _Setup:
    """Painting, transforms of delta, and the index sets of the binned modes and lags."""

    def __init__(self, gal, ran, ran_nbar, N, box_lo, box_len, assign, kedges, redges, compensate, norm,
                 threads):
        self.N, self.threads = int(N), threads
        N = self.N
        self.box_lo = np.asarray(box_lo, dtype=np.float64)
        self.box_len = float(box_len)
        self.h = self.box_len / N
        self.delta, _ = mesh.density_mesh(gal, ran, N, self.box_lo, self.box_len, assign)
        if norm:
            _, A = mesh.norm_factors(gal, ran, ran_nbar)
            if A is None:
                raise ValueError("norm=1 needs randoms with nbar")
            self.A, self.v_cell = A, self.h ** 3
        else:
            self.A, self.v_cell = 1.0, 1.0
        self.inv_w = 1.0 / mesh.compensation(N, assign) if compensate else None

        # non-empty nodes: positions box_lo + i h, their distance and direction
        occ = np.flatnonzero(self.delta)
        self.occ = occ
        i = np.unravel_index(occ, (N, N, N))
        step = np.arange(N, dtype=np.float64) * self.h
        x = np.stack([self.box_lo[a] + step[i[a]] for a in range(3)], axis=-1)
        self.r_occ = np.linalg.norm(x, axis=-1)
        if np.any(self.r_occ == 0.0):
            raise ValueError("a non-empty mesh node sits on the observer")
        self.ang_occ = direction_angles(x)
        self.delta_occ = self.delta.ravel()[occ]

        # D(k) = F[delta] (compensated), and its conjugate
        self.D = self.transform(np.ones(len(occ)))
        self.Dc = np.conj(self.D)

        labels = mesh.fft_labels(N)
        # modes with |k| up to the last k edge (a superset of every bin), in grid order
        self.kf = 2.0 * math.pi / self.box_len
        self.ball = None
        if kedges is not None:
            nmax = int(math.ceil(float(np.max(kedges)) / self.kf)) + 1
            n2 = labels[:, None, None] ** 2 + labels[None, :, None] ** 2 + labels[None, None, :] ** 2
            self.ball = np.flatnonzero(n2 <= nmax * nmax)
            del n2
            nb = np.unravel_index(self.ball, (N, N, N))
            kv = np.stack([labels[nb[a]].astype(np.float64) for a in range(3)], axis=-1) * self.kf
            n2b = (labels[nb[0]] ** 2 + labels[nb[1]] ** 2 + labels[nb[2]] ** 2).astype(np.float64)
            self.k_mag = self.kf * np.sqrt(n2b)
            self.ang_k = direction_angles(kv)
        # lags with every |component| up to the last r edge (a superset of every bin)
        self.cube = None
        if redges is not None:
            jm = int(math.floor(float(np.max(redges)) / self.h)) + 1
            idx = np.arange(N) if 2 * jm + 1 >= N else np.concatenate([np.arange(jm + 1), np.arange(N - jm, N)])
            self.cube = np.ix_(idx, idx, idx)
            j = labels[idx].astype(np.float64)
            J = np.stack(np.meshgrid(j, j, j, indexing="ij"), axis=-1) * self.h
            jj = labels[idx]
            j2 = (jj[:, None, None] ** 2 + jj[None, :, None] ** 2 + jj[None, None, :] ** 2).astype(np.float64)
            self.lag_mag_c = self.h * np.sqrt(j2)
            self.ang_c = direction_angles(J)

    def transform(self, wocc):
        """F[w delta](k) (compensated) for a field w given on the non-empty nodes."""
        N = self.N
        f = np.zeros(N * N * N, dtype=np.complex128)
        f[self.occ] = wocc * self.delta_occ
        F = _fftn(f.reshape(N, N, N))
        if self.inv_w is not None:
            _slabs(N, lambda lo, hi: F[lo:hi].__imul__(self.inv_w[lo:hi]), self.threads)
        return F

    def g_function(self, alpha, J, M):
        """g^alpha_JM(Delta) = (-1)^J IFFT[D*(k) F[(2r)^-alpha Y_J^M delta](k)] (eq. g-JM-form)."""
        w = (2.0 * self.r_occ) ** (-alpha) * ylm_angles(J, M, *self.ang_occ)
        F = self.transform(w)
        _slabs(self.N, lambda lo, hi: F[lo:hi].__imul__(self.Dc[lo:hi]), self.threads)
        g = _ifftn(F)
        if J % 2:
            _slabs(self.N, lambda lo, hi: g[lo:hi].__imul__(-1.0), self.threads)
        return g

    def lag_factor(self, J1, M, alpha, theta, phi, lag_mag):
        """Y_J1^M(Delta) |Delta|^alpha on the full lag grid."""
        N = self.N
        out = np.empty((N, N, N), dtype=np.complex128)

        def work(lo, hi):
            zero = lag_mag[lo:hi] == 0.0
            out[lo:hi] = ylm_angles(J1, M, theta[lo:hi], phi[lo:hi], zero) * lag_mag[lo:hi] ** alpha
        _slabs(N, work, self.threads)
        return out

    def lag_grids(self):
        """Polar angles and magnitude of the minimal-image lag vector on the full grid."""
        N = self.N
        labels = mesh.fft_labels(N)
        theta = np.empty((N, N, N))
        phi = np.empty((N, N, N))
        mag = np.empty((N, N, N))
        j = labels.astype(np.float64)

        def work(lo, hi):
            v = np.stack(np.meshgrid(j[lo:hi], j, j, indexing="ij"), axis=-1) * self.h
            t, p, _ = direction_angles(v)
            theta[lo:hi], phi[lo:hi] = t, p
            jj = labels[lo:hi]
            j2 = jj[:, None, None] ** 2 + labels[None, :, None] ** 2 + labels[None, None, :] ** 2
            mag[lo:hi] = self.h * np.sqrt(j2.astype(np.float64))
        _slabs(N, work, self.threads)
        return theta, phi, mag

    def pk_out(self, ells, T):
        pk, kmean, cnt = [], None, None
        for ell in ells:
            mean, kmean, cnt = mesh.shell_mean(np.real(T[ell]), self.k_mag, self.kedges, self.k_mag == 0.0)
            pk.append(FOUR_PI / self.A * mean)
        return {"pk": np.array(pk), "k_mean": kmean, "n_modes": cnt}

    def xi_out(self, ells, Z):
        xi, rmean, cnt = [], None, None
        for ell in ells:
            mean, rmean, cnt = mesh.shell_mean(np.real(Z[ell]), self.lag_mag_c, self.redges, self.lag_mag_c == 0.0)
            xi.append(FOUR_PI / (self.A * self.v_cell) * mean)
        return {"xi": np.array(xi), "r_mean": rmean, "n_cells": cnt}


def midpoint_products(K, ell_max):
    """The distinct products of eq. FFT-midpoint: {(alpha, J1, M, J2, M2): [(ell, m, phi), ...]}."""
    out = {}
    for alpha in range(K + 1):
        for ell in range(0, ell_max + 1, 2):
            for m in range(-ell, ell + 1):
                for (J1, J2, M), c in phi_table(alpha, ell, m).items():
                    out.setdefault((alpha, J1, M, J2, m - M), []).append((ell, m, c))
    return out


def bisector_pairs(K, ell_max):
    """The field pairs of eq. bisector-pk-fft summed over beta <= K/2:
    {((J1, M), (J2, M2)): [(ell, m, B), ...]}."""
    out = {}
    for beta in range(K // 2 + 1):
        for ell in range(0, ell_max + 1, 2):
            for m in range(-ell, ell + 1):
                for (J1, J2, M), c in B_table(beta, ell, m).items():
                    out.setdefault(((J1, M), (J2, m - M)), []).append((ell, m, c))
    return out


def pk_xi_multipoles(gal, ran, ran_nbar, *, N, box_lo, box_len, assign, ell_max, los, order, kedges=None,
                     redges=None, compensate=False, norm=1, block=8, threads=None, progress=None):
    """P_ell(k) and/or xi_ell(r), ell = 0, 2, .., ell_max, for los 'yamamoto', 'midpoint' or
    'bisector' (order K): the values of ``estimators.pk_multipoles`` / ``xi_multipoles`` (one tracer, no
    interlacing, norm 0 or 1).  ``block``: left bisector fields held at once.  ``progress(kind,
    done, total)`` is called after every product / pair ('unit') and may raise ``Stop`` to end
    the run early (the partial sums are then discarded)."""
    if los not in ("yamamoto", "midpoint", "bisector"):
        raise ValueError("the streamed order covers the Yamamoto, midpoint and bisector lines of sight")
    if ell_max < 0 or ell_max % 2:
        raise ValueError("even ell_max")
    if norm not in (0, 1):
        raise ValueError("norm 0 or 1")
    threads = threads or _threads()
    s = _Setup(gal, ran, ran_nbar, N, box_lo, box_len, assign, kedges, redges, compensate, norm, threads)
    s.kedges, s.redges = kedges, redges
    ells = list(range(0, ell_max + 1, 2))
    want_p, want_x = kedges is not None, redges is not None
    if progress:
        progress("setup", 0, 0)
    if want_p:
        Yk = {(ell, m): np.conj(ylm_angles(ell, m, *s.ang_k)) for ell in ells for m in range(-ell, ell + 1)}
        T = {ell: np.zeros(len(s.ball), dtype=np.complex128) for ell in ells}
    if want_x:
        Z = {ell: np.zeros(s.lag_mag_c.shape, dtype=np.complex128) for ell in ells}

    if los == "yamamoto":
        _yamamoto(s, ells, want_p, want_x, T if want_p else None, Z if want_x else None, Yk if want_p else None,
                  progress)
    elif los == "midpoint":
        _midpoint(s, order, ell_max, ells, want_p, want_x, T if want_p else None, Z if want_x else None,
                  Yk if want_p else None, progress)
    else:
        _bisector(s, order, ell_max, ells, want_p, want_x, T if want_p else None, Z if want_x else None,
                  Yk if want_p else None, block, progress)
    out = {"ells": ells}
    if want_p:
        out.update(s.pk_out(ells, T))
    if want_x:
        out.update(s.xi_out(ells, Z))
    return out


def _yamamoto(s, ells, want_p, want_x, T, Z, Yk, progress):
    """Sum over m of Y_ell^m*(k) D*(k) F[Y_ell^m delta](k) (P) and of Y_ell^m*(Delta) times the
    inverse transform of D* F[Y_ell^m delta] (xi), one field at a time."""
    total = sum(2 * ell + 1 for ell in ells)
    done = 0
    for ell in ells:
        for m in range(-ell, ell + 1):
            prod = s.transform(ylm_angles(ell, m, *s.ang_occ))
            _slabs(s.N, lambda lo, hi: prod[lo:hi].__imul__(s.Dc[lo:hi]), s.threads)
            if want_p:
                T[ell] += Yk[(ell, m)] * prod.ravel()[s.ball]
            if want_x:
                Z[ell] += np.conj(ylm_angles(ell, m, *s.ang_c)) * _ifftn(prod)[s.cube]
            del prod
            done += 1
            if progress:
                progress("unit", done, total)


def _midpoint(s, K, ell_max, ells, want_p, want_x, T, Z, Yk, progress):
    prods = midpoint_products(K, ell_max) if want_p else {}
    xi_terms = {}          # (alpha, J, M) -> [(ell, f)]
    if want_x:
        for alpha in range(K + 1):
            for ell in ells:
                for J, c in f_table(alpha, ell).items():
                    for M in range(-J, J + 1):
                        xi_terms.setdefault((alpha, J, M), []).append((ell, c))
    xi_done = set()

    def add_xi(key, g):
        if not want_x or key in xi_done or key not in xi_terms:
            return
        alpha, J, M = key
        gc = g[s.cube]
        yc = np.conj(ylm_angles(J, M, *s.ang_c)) * s.lag_mag_c ** alpha
        for ell, c in xi_terms[key]:
            Z[ell] += c * yc * gc
        xi_done.add(key)

    total = len(prods)
    done = 0
    if prods:
        theta, phi, mag = s.lag_grids()
        groups = {}
        for key in prods:
            groups.setdefault(key[:2], []).append(key)
        for (alpha, J1), keys in sorted(groups.items()):
            lf = {M: s.lag_factor(J1, M, alpha, theta, phi, mag) for M in sorted({k[2] for k in keys})}
            by_g = {}
            for k in keys:
                by_g.setdefault((k[3], k[4]), []).append(k)
            for (J2, M2), gkeys in sorted(by_g.items()):
                g = s.g_function(alpha, J2, M2)
                add_xi((alpha, J2, M2), g)
                for k in sorted(gkeys):
                    prod = np.empty_like(g)
                    lfm = lf[k[2]]
                    _slabs(s.N, lambda lo, hi: np.multiply(lfm[lo:hi], g[lo:hi], out=prod[lo:hi]), s.threads)
                    Q = _fftn(prod).ravel()[s.ball]
                    for ell, m, c in prods[k]:
                        T[ell] += c * Yk[(ell, m)] * Q
                    del prod
                    done += 1
                    if progress:
                        progress("unit", done, total)
                del g
            del lf
        del theta, phi, mag
    for key in sorted(xi_terms):             # g functions that no P product needed
        if key not in xi_done:
            add_xi(key, s.g_function(*key))
            if progress:
                progress("xi_g", len(xi_done), len(xi_terms))


def _bisector(s, K, ell_max, ells, want_p, want_x, T, Z, Yk, block, progress):
    pairs = bisector_pairs(K, ell_max)
    Yc = ({(ell, m): np.conj(ylm_angles(ell, m, *s.ang_c)) for ell in ells for m in range(-ell, ell + 1)}
          if want_x else None)
    lefts = sorted({p[0] for p in pairs})
    total, done = len(pairs), 0

    def field(JM):
        return s.transform(ylm_angles(JM[0], JM[1], *s.ang_occ))

    def flip(F):
        """F(-k): the value at index (-n mod N) along every axis."""
        return np.roll(F[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))

    for b0 in range(0, len(lefts), block):
        blk = lefts[b0:b0 + block]
        L = {JM: flip(field(JM)) for JM in blk}
        rights = sorted({p[1] for p in pairs if p[0] in L})
        for JM2 in rights:
            R = field(JM2)
            for JM1 in blk:
                terms = pairs.get((JM1, JM2))
                if not terms:
                    continue
                prod = np.empty_like(R)
                Lf = L[JM1]
                _slabs(s.N, lambda lo, hi: np.multiply(Lf[lo:hi], R[lo:hi], out=prod[lo:hi]), s.threads)
                if want_p:
                    pb = prod.ravel()[s.ball]
                    for ell, m, c in terms:
                        T[ell] += c * Yk[(ell, m)] * pb
                if want_x:
                    zc = _ifftn(prod)[s.cube]
                    for ell, m, c in terms:
                        Z[ell] += c * Yc[(ell, m)] * zc
                del prod
                done += 1
                if progress:
                    progress("unit", done, total)
            del R
        del L


def work_units(los, K, ell_max):
    """Number of products (midpoint), field pairs (bisector) or fields (Yamamoto) a request visits."""
    if los == "yamamoto":
        return sum(2 * ell + 1 for ell in range(0, ell_max + 1, 2))
    return len(midpoint_products(K, ell_max)) if los == "midpoint" else len(bisector_pairs(K, ell_max))


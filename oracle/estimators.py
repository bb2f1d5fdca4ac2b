"""FFT series estimators of P_ell(k) and xi_ell(r) (O3), FP64, complex basis.

Test infrastructure only (see ``oracle/__init__``).

Every estimator follows the paper's boxed equation literally, with full complex
``fftn`` transforms and complex spherical harmonics:

  yamamoto  P: eq. Yamamoto-estimator      xi: eq. 2pcf-yama
  midpoint  P: eq. FFT-midpoint, g from eq. g-JM-form
            xi: eq. xi-parity-all-estimator (same g functions)
  midpoint_even  the parity-even forms (Sec. 3.3 / Sec. 4.3 boxed): Phi and F
            coefficients (Appendices D, E.2), even alpha only, same g functions
  bisector  P: eq. bisector-pk-fft (boxed form)
            xi: Sec. 6 boxed estimator, h summed over the B coefficients
                before the inverse transform as Sec. 6 suggests
  fixed     P: eq. after Sec. 2.1 (|delta(k)|^2 L_ell(k.n)); xi: eq.
            2pcf-plane-parallel -- used only for the distant-observer pins.

Discrete normalisation (the reading of Sec. 2 used throughout):
  P_ell(k_b)  = 4 pi / A * mean_{k in b} Re[ sum_m Y_ell^m*(k) X_ell^m(k) ]
  xi_ell(r_b) = 4 pi / (A V_cell) * mean_{Delta in b} Re[ sum_m Y_ell^m*(Delta) Z_ell^m(Delta) ]
with A the FKP normalisation (``norm=1``) or 1 and V_cell = 1 (``norm=0``).
``norm=2`` keeps the FKP A for P and divides xi_ell by the random-random count
RR_0(r_b) of the same mesh estimator applied to alpha_r n_r (ell = 0, where the
line of sight drops out): xi_ell = [DD - 2 DR + RR]_ell / RR_0, the
Landy-Szalay form Sec. 2.2 names for catalogs (the pair counts of eq.
general-2pcf-form with delta = n_g - alpha_r n_r).

``interlace=True`` averages every forward transform of a painted field over the
mesh and the mesh shifted by half a cell along each axis (``_Transforms``), which
cancels the aliased images of odd index sum; the paper paints without it.

Cross spectra of two tracers (``gal_b``, ``ran_b``, ``ran_nbar_b``): delta_A from
(gal, ran), delta_B from the second pair, normalisation A = sqrt(A_A A_B) (V_cell
unchanged).  With two densities the two anchored terms of the midpoint series are
no longer equal, so the estimator keeps both (Sec. 3.2, the bracket before eq.
P-ell-k-symm): for even ell they give g = [g^AB + g^BA] / 2, with
g^XY = (-1)^J IFFT[delta_X*(k) F[(2r)^-alpha Y_J^M delta_Y](k)] (eq. g-JM-form with
the two densities in place of one).  Yamamoto takes the mean of its two endpoint
lines of sight in the same way; the bisector sum of eq. bisector-pk-fft takes
F[Y delta_A](-k) F[Y delta_B](k).  norm=2 is not defined for cross correlations.

``shot_noise`` is the FKP shot-noise level (sum_g w^2 + alpha_r^2 sum_r w^2) / A
that eq. Pk-def includes in P_0 (Sec. 2.1); the estimators do not subtract it.
The order K is the highest power of theta kept: midpoint alpha <= K, bisector
beta <= floor(K/2).

Parity pins (tests/test_oracle_estimators.py): each estimator equals the pair
by pair evaluation of its truncated series (``oracle.pairs``) to rounding;
midpoint K=0 equals Yamamoto; ell=0 equals across LOS; the exact pair sums are
approached as K rises; distant-observer limit; particle pair sum (O1) equals
the mesh pair sum (O2) on node-snapped catalogs.
"""
from __future__ import annotations

import math

import numpy as np

from . import mesh
from .coeffs import B_table, F_table, Phi_table, f_table, phi_table
from .special import FOUR_PI, legendre_L, ylm


class Grid:
    """Node, lag and Fourier grids of one mesh."""

    def __init__(self, N, box_lo, box_len):
        self.N = int(N)
        self.box_lo = np.asarray(box_lo, dtype=np.float64)
        self.box_len = float(box_len)
        self.h = self.box_len / self.N
        self.v_cell = self.h ** 3
        self.x = mesh.node_positions(self.N, self.box_lo, self.box_len)
        self.r = np.linalg.norm(self.x, axis=-1)
        self.lag = mesh.lag_vectors(self.N, self.box_len)
        self.lag_mag = mesh.lag_magnitude(self.N, self.box_len)
        self.k = mesh.k_vectors(self.N, self.box_len)
        self.k_mag = mesh.k_magnitude(self.N, self.box_len)


def _flip_k(a: np.ndarray) -> np.ndarray:
    """a(-k): the value at index (-n mod N) along every axis."""
    return np.roll(a[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))


class _Transforms:
    """Forward transforms of painted fields f(x) = w(x) delta(x), with the optional
    compensation 1/W(k) (Sec. 2.1 footnote) and, with interlacing, the average of
    the transforms on the mesh and on the mesh shifted by s = (h/2)(1, 1, 1):
    F = [F_1(k) + P(k) F_2(k)] / 2, P(k) = prod_d p(n_d), p(n) = exp(-i pi n / N)
    (the shift's phase in the mesh's frame) and p(-N/2) = 0, the mean of the phases
    of the two labels of the Nyquist index, so that F stays Hermitian."""

    def __init__(self, g, delta, delta2, inv_w):
        self.g, self.delta, self.delta2, self.inv_w = g, delta, delta2, inv_w
        if delta2 is not None:
            self.x2 = g.x + 0.5 * g.h
            if np.any((np.linalg.norm(self.x2, axis=-1) == 0.0) & (delta2 != 0.0)):
                raise ValueError("a non-empty shifted mesh node sits on the observer")
            n = mesh.fft_labels(g.N)
            p = np.where(n == -g.N // 2, 0.0, np.exp(-1j * np.pi * n / g.N))
            self.phase = p[:, None, None] * p[None, :, None] * p[None, None, :]

    def fwd(self, wfun=None):
        """F[w delta](k); wfun(x) gives w at positions x (None: w = 1)."""
        f = self.delta if wfun is None else wfun(self.g.x) * self.delta
        F = mesh.fftn(f)
        if self.delta2 is not None:
            f2 = self.delta2 if wfun is None else wfun(self.x2) * self.delta2
            F = 0.5 * (F + self.phase * mesh.fftn(f2))
        return F * self.inv_w if self.inv_w is not None else F


def _prepare(gal, ran, ran_nbar, N, box_lo, box_len, assign, norm, compensate, xi=False, interlace=False):
    g = Grid(N, box_lo, box_len)
    delta, _ = mesh.density_mesh(gal, ran, g.N, g.box_lo, g.box_len, assign)
    delta2 = None
    if interlace:   # the same catalog painted on the nodes box_lo + (i + 1/2) h
        delta2, _ = mesh.density_mesh(gal, ran, g.N, g.box_lo + 0.5 * g.h, g.box_len, assign)
    if norm == 2 and xi:
        if ran is None or len(ran) == 0:
            raise ValueError("norm=2 needs randoms")
        A, v_cell = 1.0, 1.0            # raw sums; divided by RR_0 afterwards
    elif norm:
        _, A = mesh.norm_factors(gal, ran, ran_nbar)
        if A is None:
            raise ValueError("norm=1 needs randoms with nbar")
        v_cell = g.v_cell
    else:
        A, v_cell = 1.0, 1.0
    inv_w = 1.0 / mesh.compensation(g.N, assign) if compensate else None
    return g, delta, A, v_cell, inv_w, _Transforms(g, delta, delta2, inv_w)


class _Tracer:
    """One density on the mesh: its painted delta, transforms and spectrum D."""

    def __init__(self, delta, tr):
        self.delta, self.tr = delta, tr
        self.D = tr.fwd()


def _tracers(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len, assign, norm, compensate,
             xi=False, interlace=False):
    """(grid, tracer A, tracer B, A, V_cell); tracer B is tracer A for an auto spectrum."""
    g, delta, A, v_cell, _, tr = _prepare(gal, ran, ran_nbar, N, box_lo, box_len, assign, norm, compensate,
                                          xi, interlace)
    ta = _Tracer(delta, tr)
    if gal_b is None:
        return g, ta, ta, A, v_cell
    if norm == 2 and xi:
        raise ValueError("norm=2 is not defined for a cross correlation")
    _, delta_b, A_b, _, _, tr_b = _prepare(gal_b, ran_b, ran_nbar_b, N, box_lo, box_len, assign, norm, compensate,
                                           xi, interlace)
    return g, ta, _Tracer(delta_b, tr_b), float(np.sqrt(A * A_b)), v_cell


def _cross_g_fields(g, ta, tb, K, ell_max, even=False, parities=(0,)):
    """g fields of the midpoint series, both anchorings: [(-1)^ell g^AB + g^BA] / 2 with
    g^AB (delta_A conjugated, delta_B carrying the weights) from the expansion anchored on
    the second galaxy and g^BA from the one anchored on the first, after the relabelling
    Delta -> -Delta, k -> -k that brings it to the same form (exact in shell means); ell's
    parity is that of J - alpha.  One density: g^AA for even ell, 0 for odd ell."""
    gab = g_fields(g, tb.delta, ta.D, K, ell_max, tb.tr, even, parities)
    if tb is ta:
        return {key: (v if (key[1] - key[0]) % 2 == 0 else np.zeros_like(v)) for key, v in gab.items()}
    gba = g_fields(g, ta.delta, tb.D, K, ell_max, ta.tr, even, parities)
    return {key: 0.5 * ((-1) ** (key[1] - key[0]) * gab[key] + gba[key]) for key in gab}


def _ells(ell_max, odd=False):
    """ell = 0, 2, .., ell_max (the paper's even multipoles), or every ell <= ell_max with odd."""
    if ell_max < 0 or (ell_max % 2 and not odd):
        raise ValueError("odd ell_max needs odd=True (the paper assumes even ell)")
    return list(range(0, ell_max + 1, 1 if odd else 2))


def _pk_out(g, ells, T, A, kedges):
    """Shell means of T_ell(k) = sum_m Y_ell^m*(k) X_ell^m(k): the real part for even ell, the
    imaginary part for odd ell (the shell mean of an odd multipole is imaginary, since
    T_ell(-k) = (-1)^ell conj T_ell(k) for real densities)."""
    pk, kmean, cnt = [], None, None
    for ell in ells:
        t = np.real(T[ell]) if ell % 2 == 0 else np.imag(T[ell])
        mean, kmean, cnt = mesh.shell_mean(t, g.k_mag, kedges, g.k_mag == 0.0)
        pk.append(FOUR_PI / A * mean)
    return {"ells": ells, "pk": np.array(pk), "k_mean": kmean, "n_modes": cnt}


def _xi_out(g, ells, Z, A, v_cell, redges):
    xi, rmean, cnt = [], None, None
    for ell in ells:
        mean, rmean, cnt = mesh.shell_mean(np.real(Z[ell]), g.lag_mag, redges, g.lag_mag == 0.0)
        xi.append(FOUR_PI / (A * v_cell) * mean)
    return {"ells": ells, "xi": np.array(xi), "r_mean": rmean, "n_cells": cnt}


# --------------------------------------------------------------------------
# midpoint convolution fields g^alpha_JM (eq. g-JM-form)
# --------------------------------------------------------------------------
def g_fields(g: Grid, delta, D, K, ell_max, tr, even=False, parities=(0,)):
    """g^alpha_JM(Delta) = (-1)^J IFFT[ delta*(k) F[(2r)^-alpha Y_J^M delta](k) ](Delta)
    for alpha <= K and J <= ell_max + alpha with J - alpha of the given parities: the J
    with non-zero phi / f are J = alpha, alpha - 2, ... for even ell (parity 0) and
    alpha + 1, alpha - 1, ... for odd ell (parity 1), since J1 = alpha mod 2 and
    J1 + J2 = ell mod 2.  Cells with delta = 0 carry no field; a non-empty cell at the
    observer has no expansion and is rejected."""
    if np.any((g.r == 0.0) & (delta != 0.0)):
        raise ValueError("a non-empty mesh node sits on the observer")
    Dc = np.conj(D)

    def radial(x, alpha):   # (2 r)^-alpha, 0 on the observer (where no painted node may sit)
        r = np.linalg.norm(x, axis=-1)
        return np.where(r == 0.0, 0.0, (2.0 * np.where(r == 0.0, 1.0, r)) ** (-alpha))

    out = {}
    for alpha in range(0, K + 1, 2 if even else 1):
        for par in parities:
            for J in range((alpha + par) % 2, ell_max + alpha + 1, 2):
                for M in range(-J, J + 1):
                    F = tr.fwd(lambda x: radial(x, alpha) * ylm(J, M, x))
                    out[(alpha, J, M)] = (-1) ** J * mesh.ifftn(Dc * F)
    return out


# --------------------------------------------------------------------------
# public entry points (mirror the library's pk_multipoles / xi_multipoles)
# --------------------------------------------------------------------------
def pk_multipoles(gal, ran, ran_nbar, *, N, box_lo, box_len, assign, ell_max, los,
                  order, kedges, compensate=False, norm=1, interlace=False,
                  gal_b=None, ran_b=None, ran_nbar_b=None, odd=False):
    """P_ell(k) for ell = 0, 2, .., ell_max (every ell <= ell_max with odd) with LOS in
    {'yamamoto', 'midpoint', 'midpoint_even', 'bisector', 'fixed'}; the cross
    spectrum of (gal, ran) with (gal_b, ran_b) when gal_b is given."""
    g, ta, tb, A, _ = _tracers(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len, assign, norm,
                               compensate, interlace=interlace)
    ells = _ells(ell_max, odd)
    if odd and los == "midpoint_even":
        raise ValueError("the parity-even midpoint form is defined for even ell")
    pars = (0, 1) if odd else (0,)
    shape = ta.D.shape
    T = {}
    if los == "yamamoto":
        # eq. Yamamoto-estimator: sum_m Y*(k) F[Y delta](k) delta*(k); two tracers: the
        # mean of the lines of sight through either galaxy of the pair
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for m in range(-ell, ell + 1):
                acc += np.conj(ylm(ell, m, g.k)) * _yamamoto_product(ta, tb, ell, m)
            T[ell] = acc
    elif los in ("midpoint", "midpoint_even"):
        # eq. FFT-midpoint: sum_m Y*(k) sum phi F[ Y_J1^M(Delta) Delta^alpha g^alpha_{J2 (m-M)}(Delta) ](k);
        # parity-even form (Sec. 3.3 boxed): phi -> Phi, even alpha only
        even = los == "midpoint_even"
        table = Phi_table if even else phi_table
        gf = _cross_g_fields(g, ta, tb, order, ell_max, even, pars)
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for m in range(-ell, ell + 1):
                H = np.zeros(shape, dtype=np.complex128)
                for alpha in range(0, order + 1, 2 if even else 1):
                    dpow = g.lag_mag ** alpha
                    for (J1, J2, M), c in table(alpha, ell, m).items():
                        H += c * ylm(J1, M, g.lag) * dpow * gf[(alpha, J2, m - M)]
                acc += np.conj(ylm(ell, m, g.k)) * mesh.fftn(H)
            T[ell] = acc
    elif los == "bisector":
        # eq. bisector-pk-fft: sum_m Y*(k) sum B F[Y_J1^M delta_A](-k) F[Y_J2^{m-M} delta_B](k)
        FA, FB = _bisector_fields(ta, tb, ell_max + order // 2)
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for m in range(-ell, ell + 1):
                acc += np.conj(ylm(ell, m, g.k)) * _bisector_X(FA, FB, order // 2, ell, m, shape)
            T[ell] = acc
    elif los == "fixed":
        # delta_A*(k) delta_B(k) L_ell(k . n) with n = the direction of the box centre
        n = g.box_lo + 0.5 * g.box_len
        n = n / np.linalg.norm(n)
        mu = np.where(g.k_mag > 0, (g.k @ n) / np.where(g.k_mag > 0, g.k_mag, 1.0), 0.0)
        for ell in ells:
            T[ell] = (2 * ell + 1) / FOUR_PI * legendre_L(ell, mu) * (np.conj(ta.D) * tb.D)
    else:
        raise ValueError(f"unknown los {los!r}")
    return _pk_out(g, ells, T, A, kedges)


def _yamamoto_product(ta, tb, ell, m):
    """[delta_A*(k) F[Y_ell^m delta_B](k) + (-1)^ell delta_B*(k) F[Y_ell^m delta_A](k)] / 2:
    the lines of sight through the second and through the first galaxy (the latter brought
    to this form by k -> -k, exact in shell means).  One density: the first term for even
    ell, 0 for odd ell."""
    p = np.conj(ta.D) * tb.tr.fwd(lambda x: ylm(ell, m, x))
    if tb is ta:
        return p if ell % 2 == 0 else np.zeros_like(p)
    return 0.5 * (p + (-1) ** ell * np.conj(tb.D) * ta.tr.fwd(lambda x: ylm(ell, m, x)))


def _bisector_fields(ta, tb, Jmax):
    """F[Y_J^M delta](k) for J <= Jmax, of tracer A and of tracer B."""
    FA = {(J, M): ta.tr.fwd(lambda x, J=J, M=M: ylm(J, M, x)) for J in range(Jmax + 1) for M in range(-J, J + 1)}
    FB = FA if tb is ta else {(J, M): tb.tr.fwd(lambda x, J=J, M=M: ylm(J, M, x))
                              for J in range(Jmax + 1) for M in range(-J, J + 1)}
    return FA, FB


def _bisector_X(FA, FB, bmax, ell, m, shape):
    """X_ell^m(k) = sum_beta sum B^{beta, ell m}_{J1 J2 M} F_A[Y_J1^M](-k) F_B[Y_J2^{m-M}](k)."""
    X = np.zeros(shape, dtype=np.complex128)
    for beta in range(bmax + 1):
        for (J1, J2, M), c in B_table(beta, ell, m).items():
            X += c * _flip_k(FA[(J1, M)]) * FB[(J2, m - M)]
    return X


def xi_multipoles(gal, ran, ran_nbar, *, N, box_lo, box_len, assign, ell_max, los,
                  order, redges, compensate=False, norm=1, interlace=False,
                  gal_b=None, ran_b=None, ran_nbar_b=None, odd=False):
    """xi_ell(r) for ell = 0, 2, .., ell_max (every ell <= ell_max with odd) with LOS in
    {'yamamoto', 'midpoint', 'midpoint_even', 'bisector', 'fixed'}; the cross
    correlation of (gal, ran) with (gal_b, ran_b) when gal_b is given."""
    g, ta, tb, A, v_cell = _tracers(gal, ran, ran_nbar, gal_b, ran_b, ran_nbar_b, N, box_lo, box_len, assign,
                                    norm, compensate, xi=True, interlace=interlace)
    ells = _ells(ell_max, odd)
    if odd and los == "midpoint_even":
        raise ValueError("the parity-even midpoint form is defined for even ell")
    pars = (0, 1) if odd else (0,)
    shape = ta.D.shape
    Z = {}
    if los == "yamamoto":
        # eq. 2pcf-yama: sum_m Y*(Delta) IFFT[delta*(k) F[Y delta](k)](Delta); two tracers as for P
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for m in range(-ell, ell + 1):
                acc += np.conj(ylm(ell, m, g.lag)) * mesh.ifftn(_yamamoto_product(ta, tb, ell, m))
            Z[ell] = acc.real
    elif los in ("midpoint", "midpoint_even"):
        # eq. xi-parity-all-estimator: sum f Y_J^M*(Delta) Delta^alpha g^alpha_JM(Delta);
        # parity-even form (Sec. 4.3 boxed): f -> F, even alpha only
        even = los == "midpoint_even"
        table = F_table if even else f_table
        gf = _cross_g_fields(g, ta, tb, order, ell_max, even, pars)
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for alpha in range(0, order + 1, 2 if even else 1):
                dpow = g.lag_mag ** alpha
                for J, c in table(alpha, ell).items():
                    for M in range(-J, J + 1):
                        acc += c * np.conj(ylm(J, M, g.lag)) * dpow * gf[(alpha, J, M)]
            Z[ell] = acc.real
    elif los == "bisector":
        # Sec. 6: sum_m Y*(Delta) IFFT[ sum B F[Y_J1^M delta_A](-k) F[Y_J2^{m-M} delta_B](k) ](Delta)
        FA, FB = _bisector_fields(ta, tb, ell_max + order // 2)
        for ell in ells:
            acc = np.zeros(shape, dtype=np.complex128)
            for m in range(-ell, ell + 1):
                acc += np.conj(ylm(ell, m, g.lag)) * mesh.ifftn(_bisector_X(FA, FB, order // 2, ell, m, shape))
            Z[ell] = acc.real
    elif los == "fixed":
        n = g.box_lo + 0.5 * g.box_len
        n = n / np.linalg.norm(n)
        mu = np.where(g.lag_mag > 0, (g.lag @ n) / np.where(g.lag_mag > 0, g.lag_mag, 1.0), 0.0)
        c = mesh.ifftn(np.conj(ta.D) * tb.D).real
        for ell in ells:
            Z[ell] = (2 * ell + 1) / FOUR_PI * legendre_L(ell, mu) * c
    else:
        raise ValueError(f"unknown los {los!r}")
    out = _xi_out(g, ells, Z, A, v_cell, redges)
    if norm == 2:
        out["xi"] = out["xi"] / _rr0(gal, ran, N, box_lo, box_len, assign, redges, compensate, interlace)[None, :]
    return out


def _rr0(gal, ran, N, box_lo, box_len, assign, redges, compensate, interlace=False):
    """RR_0(r_b): the raw ell = 0 sum of the mesh estimator for alpha_r n_r (any
    line of sight gives the same ell = 0 sum; Yamamoto is used), bins without
    random pairs set to infinity so that their ratio is 0."""
    alpha, _ = mesh.norm_factors(gal, ran, None)
    rr = xi_multipoles(ran, None, None, N=N, box_lo=box_lo, box_len=box_len, assign=assign, ell_max=0,
                       los="yamamoto", order=0, redges=redges, compensate=compensate, norm=0,
                       interlace=interlace)["xi"][0]
    rr = alpha * alpha * rr
    return np.where(rr != 0.0, rr, np.inf)


def shot_noise(gal, ran, ran_nbar, norm=1):
    """FKP shot-noise level of P_0: (sum_g w^2 + alpha_r^2 sum_r w^2) / A, with A
    the FKP normalisation (norm 1 or 2) or 1 (norm 0)."""
    w_g = np.asarray(gal, dtype=np.float64)[:, 3]
    alpha, A = mesh.norm_factors(gal, ran, ran_nbar)
    s = float(np.sum(w_g * w_g))
    if ran is not None and len(ran):
        w_r = np.asarray(ran, dtype=np.float64)[:, 3]
        s += alpha * alpha * float(np.sum(w_r * w_r))
    if norm == 0:
        return s
    if A is None:
        raise ValueError("norm 1 or 2 needs randoms with nbar")
    return s / A

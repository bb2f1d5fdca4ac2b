"""Mesh front-end of the estimators: painting, grids, normalisation, binning.

Test infrastructure only (see ``oracle/__init__``).

Conventions (the readings of Sec. 2 that the whole package uses):
  * mesh node i (per axis) sits at box_lo + i*h, h = box_len/N; the observer
    is at the origin, so the line-of-sight quantities use the node position;
  * delta(x) = w [n_g - alpha_r n_r] painted with CIC (2 nodes per axis) or TSC
    (3 nodes per axis), periodic (Sec. 2.1, eq. after eq. Pk-def); alpha_r is
    sum w_g / sum w_r; the 1/I^(1/2) factor becomes the FKP normalisation
    A = alpha_r sum_r nbar_r w_r^2 applied to the final multipoles;
  * Fourier conventions of Sec. 2 (eq. 2.1): forward transforms use e^{-ik.x};
    on the mesh the forward transform is the plain DFT over node indices
    (numpy/scipy ``fftn``) -- phase factors from box_lo cancel in every
    product the estimators form;
  * integer frequency labels follow fftfreq: index i >= N/2 maps to i - N;
    lags use the same minimal-image labelling;
  * |k| = k_f sqrt(n.n) with k_f = 2 pi / box_len, |Delta| = h sqrt(j.j);
    shell b collects |k| (or |Delta|) in [edge_b, edge_{b+1}); k = 0 and
    Delta = 0 never enter a bin.

Parity pins (tests/test_oracle_mesh.py): painting by hand at 4^3 for CIC and
TSC (weights sum to one, node-snapped particles deposit on one node), the
norm reduction on a hand-made catalog, bin assignment on hand-made edges.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft


def fftn(a):
    return scipy.fft.fftn(a, workers=-1)


def ifftn(a):
    return scipy.fft.ifftn(a, workers=-1)


def fft_labels(N: int) -> np.ndarray:
    """Integer frequency / lag labels: 0..N/2-1, -N/2..-1."""
    return np.fft.fftfreq(N, d=1.0 / N).astype(np.int64)


def node_positions(N: int, box_lo, box_len: float) -> np.ndarray:
    """(N, N, N, 3) array of node positions box_lo + i h."""
    h = box_len / N
    i = np.arange(N, dtype=np.float64) * h
    X, Y, Z = np.meshgrid(box_lo[0] + i, box_lo[1] + i, box_lo[2] + i, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def lag_vectors(N: int, box_len: float) -> np.ndarray:
    """(N, N, N, 3) array of minimal-image lag vectors Delta = h j."""
    h = box_len / N
    j = fft_labels(N).astype(np.float64)
    X, Y, Z = np.meshgrid(j, j, j, indexing="ij")
    return np.stack([X, Y, Z], axis=-1) * h


def k_vectors(N: int, box_len: float) -> np.ndarray:
    """(N, N, N, 3) array of wave vectors k = k_f n."""
    kf = 2.0 * math.pi / box_len
    n = fft_labels(N).astype(np.float64)
    X, Y, Z = np.meshgrid(n, n, n, indexing="ij")
    return np.stack([X, Y, Z], axis=-1) * kf


def k_magnitude(N: int, box_len: float) -> np.ndarray:
    """|k| = k_f sqrt(n.n) on the full grid."""
    kf = 2.0 * math.pi / box_len
    n = fft_labels(N)
    n2 = n[:, None, None] ** 2 + n[None, :, None] ** 2 + n[None, None, :] ** 2
    return kf * np.sqrt(n2.astype(np.float64))


def lag_magnitude(N: int, box_len: float) -> np.ndarray:
    """|Delta| = h sqrt(j.j) on the full lag grid."""
    h = box_len / N
    j = fft_labels(N)
    j2 = j[:, None, None] ** 2 + j[None, :, None] ** 2 + j[None, None, :] ** 2
    return h * np.sqrt(j2.astype(np.float64))


# --------------------------------------------------------------------------
# painting
# --------------------------------------------------------------------------
def paint(xyzw: np.ndarray, weight_scale: float, N: int, box_lo, box_len: float,
          assign: int, out: np.ndarray | None = None) -> np.ndarray:
    """Add weight_scale * w of every particle to the N^3 mesh with CIC (assign=2)
    or TSC (assign=3) kernels, periodic.  xyzw is (n, 4) = x, y, z, w."""
    if out is None:
        out = np.zeros((N, N, N), dtype=np.float64)
    p = np.asarray(xyzw, dtype=np.float64)
    if p.shape[0] == 0:
        return out
    h = box_len / N
    u = (p[:, :3] - np.asarray(box_lo, dtype=np.float64)) / h
    w = p[:, 3] * weight_scale
    if assign == 2:
        base = np.floor(u)
        d = u - base
        base = base.astype(np.int64)
        for ox in (0, 1):
            wx = d[:, 0] if ox else 1.0 - d[:, 0]
            for oy in (0, 1):
                wy = d[:, 1] if oy else 1.0 - d[:, 1]
                for oz in (0, 1):
                    wz = d[:, 2] if oz else 1.0 - d[:, 2]
                    ix = (base[:, 0] + ox) % N
                    iy = (base[:, 1] + oy) % N
                    iz = (base[:, 2] + oz) % N
                    np.add.at(out, (ix, iy, iz), w * wx * wy * wz)
    elif assign == 3:
        base = np.floor(u + 0.5)
        d = u - base                       # in [-1/2, 1/2)
        base = base.astype(np.int64)
        wts = [0.5 * (0.5 - d) ** 2, 0.75 - d ** 2, 0.5 * (0.5 + d) ** 2]
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    ix = (base[:, 0] + ox) % N
                    iy = (base[:, 1] + oy) % N
                    iz = (base[:, 2] + oz) % N
                    ww = w * wts[ox + 1][:, 0] * wts[oy + 1][:, 1] * wts[oz + 1][:, 2]
                    np.add.at(out, (ix, iy, iz), ww)
    else:
        raise ValueError("assign must be 2 (CIC) or 3 (TSC)")
    return out


def norm_factors(gal: np.ndarray, ran: np.ndarray | None, ran_nbar: np.ndarray | None):
    """alpha_r = sum w_g / sum w_r and A = alpha_r sum_r nbar_r w_r^2 (Sec. 2.1,
    FKP normalisation of I).  Without randoms alpha_r = 0 and A is undefined (None)."""
    sw_g = float(np.sum(np.asarray(gal, dtype=np.float64)[:, 3]))
    if ran is None or len(ran) == 0:
        return 0.0, None
    r = np.asarray(ran, dtype=np.float64)
    sw_r = float(np.sum(r[:, 3]))
    alpha = sw_g / sw_r
    A = None
    if ran_nbar is not None:
        A = alpha * float(np.sum(np.asarray(ran_nbar, dtype=np.float64) * r[:, 3] ** 2))
    return alpha, A


def density_mesh(gal, ran, N, box_lo, box_len, assign):
    """delta = paint(gal, w) - alpha_r paint(ran, w) and alpha_r."""
    alpha, _ = norm_factors(gal, ran, None)
    d = paint(gal, 1.0, N, box_lo, box_len, assign)
    if ran is not None and len(ran):
        paint(ran, -alpha, N, box_lo, box_len, assign, out=d)
    return d, alpha


def compensation(N: int, assign: int) -> np.ndarray:
    """Mass-assignment window W(k) = prod_i sinc(pi n_i / N)^p, p = 2 (CIC) or 3
    (TSC) (Sec. 2.1 footnote on the compensation function M(k) = 1/W)."""
    n = fft_labels(N).astype(np.float64)
    x = math.pi * n / N
    s = np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
    s = s ** assign
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


# --------------------------------------------------------------------------
# shell binning
# --------------------------------------------------------------------------
def shell_index(mag: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Bin index of each magnitude for half-open [e_b, e_{b+1}); -1 outside."""
    b = np.searchsorted(np.asarray(edges, dtype=np.float64), mag, side="right") - 1
    b[(b < 0) | (b >= len(edges) - 1)] = -1
    return b


def shell_mean(values: np.ndarray, mag: np.ndarray, edges, exclude_zero: np.ndarray):
    """Per-bin sum / count of values (flattened), mean magnitude and counts.
    Cells flagged by exclude_zero never enter a bin.  Empty bins give 0."""
    edges = np.asarray(edges, dtype=np.float64)
    nb = len(edges) - 1
    b = shell_index(mag.ravel(), edges)
    b[exclude_zero.ravel()] = -1
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=nb).astype(np.int64)
    s = np.bincount(b[sel], weights=values.ravel()[sel], minlength=nb)
    sm = np.bincount(b[sel], weights=mag.ravel()[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
        mmean = np.where(cnt > 0, sm / np.maximum(cnt, 1), 0.0)
    return mean, mmean, cnt

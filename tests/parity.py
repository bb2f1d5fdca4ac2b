"""Tolerances of the GPU-vs-oracle parity tests.

FP32 builds (fields and FFTs in FP32, FP64 shell sums): 1e-5 relative on the
monopole, 1e-4 relative on ell > 0 where |X_ell| exceeds 1 % of the monopole
scale, and an absolute 1e-4 x monopole scale elsewhere.  The monopole scale is
|X_0| in the same k bin for P, and max_r |xi_0| for xi.  FP64 builds: 1e-10
with the same structure.
"""
import numpy as np


def check_multipoles(got, want, kind, rtol0=1e-5, rtol=1e-4, label=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (got.shape, want.shape)
    if kind == "pk":
        scale0 = np.abs(want[0])
    else:
        scale0 = np.full(want.shape[1], np.max(np.abs(want[0])))
    err0 = np.abs(got[0] - want[0])
    bad0 = err0 > rtol0 * np.maximum(np.abs(want[0]), 1e-300) + 1e-300
    if kind == "xi":
        bad0 = err0 > rtol0 * scale0 + 1e-300
    msgs = []
    if np.any(bad0):
        i = np.argmax(err0 / np.maximum(scale0, 1e-300))
        msgs.append(f"ell=0 bin {i}: got {got[0, i]!r} want {want[0, i]!r}")
    for l in range(1, want.shape[0]):
        big = np.abs(want[l]) > 0.01 * scale0
        tol = np.where(big, rtol * np.abs(want[l]), rtol * scale0) + 1e-300
        err = np.abs(got[l] - want[l])
        if np.any(err > tol):
            i = np.argmax(err / tol)
            msgs.append(f"ell={2 * l} bin {i}: got {got[l, i]!r} want {want[l, i]!r} tol {tol[i]:.3e}")
    assert not msgs, label + "; ".join(msgs)


def max_rel(got, want, kind):
    """Largest error per multipole relative to the scale used by check_multipoles (for reports)."""
    got = np.asarray(got)
    want = np.asarray(want)
    scale0 = np.abs(want[0]) if kind == "pk" else np.max(np.abs(want[0]))
    out = []
    for l in range(want.shape[0]):
        s = np.maximum(np.abs(want[l]), 0.01 * scale0) if l else (scale0 if kind == "xi" else np.abs(want[0]))
        out.append(float(np.max(np.abs(got[l] - want[l]) / np.maximum(s, 1e-300))))
    return out

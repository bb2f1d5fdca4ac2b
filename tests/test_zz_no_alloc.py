"""The no-allocation Yamamoto contraction against the regular entry point.

Callers that cannot allocate device memory (another framework owns the
allocator, a fixed budget was carved out up front, or allocation is not
allowed where they run) hand bym_pk_yamamoto_from_spectra_noalloc the field
spectra they already hold.  Fed the spectra of the same catalog, it must
reproduce bym_pk_multipoles (Yamamoto, FP32) within the FP32 parity tolerance,
on two calls in a row: its scratch array keeps the previous call's contents,
so the second call checks that everything that must start at zero is cleared.
This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes
import math

import numpy as np
import pytest

from parity import check_multipoles
from synth import snapped_catalog

pytestmark = pytest.mark.gpu


def _real_ylm(l, m, v):
    """Real spherical harmonics in the convention of include/bym.h, from scipy's
    complex Y_l^m (DLMF 14.30)."""
    from scipy.special import sph_harm_y
    r = np.linalg.norm(v, axis=-1)
    theta = np.arccos(np.clip(v[..., 2] / r, -1.0, 1.0))
    phi = np.arctan2(v[..., 1], v[..., 0])
    y = sph_harm_y(l, abs(m), theta, phi)
    if m == 0:
        return y.real
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * y.real
    return math.sqrt(2.0) * (-1) ** m * y.imag


def _noalloc_fn(pkg):
    fn = pkg.lib().bym_pk_yamamoto_from_spectra_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                   ctypes.POINTER(pkg.Bins), ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return fn


def _spectra(torch, cat, N, lo, h, ell_max):
    """F (the transforms of Y_{l mu} delta, even l <= ell_max) and D for a node-snapped CIC catalog,
    where every object deposits its whole weight on one node."""
    idx = np.rint((cat.gal[:, :3].astype(np.float64) - lo) / h).astype(np.int64)
    delta = np.zeros((N, N, N))
    np.add.at(delta, tuple(idx.T), cat.gal[:, 3].astype(np.float64))
    g = lo[0] + np.arange(N) * h
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    fields = [(_real_ylm(l, m, X) * delta) for l in range(0, ell_max + 1, 2) for m in range(-l, l + 1)]
    dev = torch.device("cuda", 0)
    F = torch.fft.rfftn(torch.tensor(np.stack(fields), dtype=torch.float32, device=dev), dim=(1, 2, 3)).contiguous()
    D = torch.fft.rfftn(torch.tensor(delta, dtype=torch.float32, device=dev)).contiguous()
    torch.cuda.synchronize(dev)
    return F, D


@pytest.mark.parametrize("N,ell_max", [(32, 0), (32, 2), (32, 4), (128, 4)])
def test_noalloc_matches_pk_multipoles(N, ell_max):
    torch = pytest.importorskip("torch")
    import paper_2102_08384_gb300 as pkg

    L = 1024.0
    lo = np.array([512.0, 512.0, 512.0])
    h = L / N
    cat = snapped_catalog(seed=21, n_gal=3000 if N == 32 else 40000, N=N, box_lo=lo, box_len=L, fill=0.5)
    kedges = np.linspace(0.0, math.pi / h, 11)

    ctx = pkg.Context(0)
    p = pkg.make_params(box_lo=lo, box_len=L, n_mesh=N, assign=2, ell_max=ell_max, los="yamamoto", precision=32,
                        norm=0)
    ref = ctx.pk_multipoles(cat.gal, None, p, kedges)
    ctx.close()
    F, D = _spectra(torch, cat, N, lo, h, ell_max)

    fn = _noalloc_fn(pkg)
    e = np.ascontiguousarray(kedges)
    bins = pkg.Bins()
    bins.edges, bins.nbins = e.ctypes.data, len(e) - 1
    nl = ell_max // 2 + 1
    for call in range(2):
        pk = np.full((nl, len(e) - 1), np.nan)
        nm = np.full(len(e) - 1, -1, dtype=np.int64)
        rc = fn(F.data_ptr(), D.data_ptr(), N, L, ell_max, ctypes.byref(bins), 1.0,
                pk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                None)
        assert rc == 0, f"call {call}: rc {rc}"
        np.testing.assert_array_equal(nm, ref["n_modes"])
        check_multipoles(pk, ref["pk"], "pk", label=f"N={N} ell_max={ell_max} call {call}: ")


def test_noalloc_refuses_beyond_its_array():
    # requests beyond the static scratch array are refused, not truncated
    torch = pytest.importorskip("torch")
    import paper_2102_08384_gb300 as pkg

    N, L = 16, 1024.0
    dev = torch.device("cuda", 0)
    F = torch.zeros((9, N, N, N // 2 + 1), dtype=torch.complex64, device=dev)
    D = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device=dev)
    fn = _noalloc_fn(pkg)
    e = np.linspace(0.0, 0.1, 5)
    bins = pkg.Bins()
    bins.edges, bins.nbins = e.ctypes.data, len(e) - 1
    big = np.linspace(0.0, 1.0, 1026)
    bb = pkg.Bins()
    bb.edges, bb.nbins = big.ctypes.data, len(big) - 1
    pk = np.zeros((3, 1025))
    nm = np.zeros(1025, dtype=np.int64)
    args = (pk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            None)
    assert fn(F.data_ptr(), D.data_ptr(), N, L, 4, ctypes.byref(bb), 1.0, *args) == -6
    assert fn(F.data_ptr(), D.data_ptr(), 1024, L, 4, ctypes.byref(bins), 1.0, *args) == -6
    assert fn(F.data_ptr(), D.data_ptr(), N, L, 6, ctypes.byref(bins), 1.0, *args) == -6

"""The library's own 512^3 FP32 FFT kernels against cuFFT (through torch.fft), and
whole requests computed with them against the same requests computed with cuFFT,
with 8-CTA (backend mode 1) and 16-CTA (mode 3) clusters in the plane pass, and
with cuFFT's plane transforms around the library's x pass (mode 4)."""
import ctypes
import math

import numpy as np
import pytest

from parity import check_multipoles

pytestmark = pytest.mark.gpu
N = 512


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import paper_2102_08384_gb300 as pkg
    lib = pkg.lib()
    lib.bym_fft3d.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p]
    lib.bym_set_fft_backend.argtypes = [ctypes.c_void_p, ctypes.c_int]
    ctx = pkg.Context(0)
    assert lib.bym_set_fft_backend(ctx._h, 1) == 0     # the library's kernels wherever they apply
    yield torch, pkg, lib, ctx
    ctx.close()


def _slots(torch, x):
    """(count, N, N, N) real -> padded slots (count, N, N, N + 4)."""
    s = torch.zeros(x.shape[0], N, N, N + 4, dtype=torch.float32, device=x.device)
    s[..., :N] = x
    return s


@pytest.mark.parametrize("mode", [1, 3, 4, 6])
def test_forward_and_inverse_match_cufft(env, mode):
    torch, pkg, lib, ctx = env
    assert lib.bym_set_fft_backend(ctx._h, mode) == 0
    gen = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(2, N, N, N, device="cuda", generator=gen)
    buf = _slots(torch, x)
    torch.cuda.synchronize()
    assert lib.bym_fft3d(ctx._h, buf.data_ptr(), N, 2, 0, None) == 0
    got = torch.view_as_complex(buf.view(2, N, N, N // 2 + 2, 2))[..., :N // 2 + 1]
    want = torch.fft.rfftn(x, dim=(1, 2, 3))
    err = (got - want).abs().max().item() / want.abs().max().item()
    rms = ((got - want).abs().pow(2).mean().sqrt() / want.abs().pow(2).mean().sqrt()).item()
    assert err < 2e-6 and rms < 1e-6, (err, rms)
    # inverse (unnormalised), from the native forward output
    assert lib.bym_fft3d(ctx._h, buf.data_ptr(), N, 2, 1, None) == 0
    back = buf[..., :N] / float(N) ** 3
    err = (back - x).abs().max().item() / x.abs().max().item()
    assert err < 2e-6, err
    # inverse of a cuFFT spectrum against cuFFT's inverse
    spec = torch.fft.rfftn(x[:1], dim=(1, 2, 3))
    want_r = torch.fft.irfftn(spec, s=(N, N, N), dim=(1, 2, 3), norm="forward")
    buf2 = torch.zeros(1, N, N, N // 2 + 2, 2, device=spec.device)
    buf2[..., :N // 2 + 1, :] = torch.view_as_real(spec)
    buf2 = buf2.view(1, N, N, N + 4)
    torch.cuda.synchronize()
    assert lib.bym_fft3d(ctx._h, buf2.data_ptr(), N, 1, 1, None) == 0
    err = (buf2[..., :N] - want_r).abs().max().item() / want_r.abs().max().item()
    assert err < 2e-6, err


@pytest.fixture(scope="module")
def cat():
    from synth import lognormal_cap_catalog
    return lognormal_cap_catalog(seed=9, n_gal=200_000, ran_factor=10.0, gen_mesh=128)


@pytest.mark.parametrize("los,K,mode,il", [("yamamoto", 0, 1, 0), ("midpoint", 4, 1, 0), ("bisector", 4, 1, 0),
                                           ("midpoint_even", 2, 1, 0), ("midpoint", 2, 3, 0), ("bisector", 2, 3, 0),
                                           ("midpoint", 4, 4, 0), ("bisector", 4, 4, 0), ("yamamoto", 0, 4, 0),
                                           ("midpoint", 2, 4, 1), ("bisector", 2, 1, 1),
                                           ("yamamoto", 0, 6, 0), ("midpoint", 4, 6, 0), ("bisector", 4, 6, 0),
                                           ("midpoint_even", 2, 6, 0), ("midpoint", 2, 6, 1)])
def test_requests_native_vs_cufft(env, cat, los, K, mode, il):
    torch, pkg, lib, ctx = env
    p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=4, los=los, order=K,
                        compensate=True, precision=32, interlace=bool(il))
    kedges = np.round(np.arange(0.01, 0.2501, 0.01), 10)
    redges = np.arange(10.0, 190.01, 10.0)
    out = {}
    for m in (0, mode):
        assert lib.bym_set_fft_backend(ctx._h, m) == 0
        out[m] = ctx.pk_xi_multipoles(cat.gal, cat.ran, p, kedges, redges, ran_nbar=cat.ran_nbar)
    check_multipoles(out[mode]["pk"], out[0]["pk"], "pk", label=f"{los} P: ")
    check_multipoles(out[mode]["xi"], out[0]["xi"], "xi", label=f"{los} xi: ")


@pytest.mark.parametrize("mode", [1, 4, 6])
def test_streamed_ranges_with_library_kernels(env, cat, mode):
    # midpoint g fields in ranges of 9 (slots 2.. of the request) through the library's kernels
    torch, pkg, lib, ctx = env
    p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=4, los="midpoint",
                        order=2, compensate=True, precision=32)
    kedges = np.round(np.arange(0.01, 0.2501, 0.01), 10)
    redges = np.arange(10.0, 190.01, 10.0)
    assert lib.bym_set_fft_backend(ctx._h, 0) == 0
    ref = ctx.pk_xi_multipoles(cat.gal, cat.ran, p, kedges, redges, ran_nbar=cat.ran_nbar)
    assert lib.bym_set_fft_backend(ctx._h, mode) == 0
    ctx.set_field_chunk(9)
    try:
        got = ctx.pk_xi_multipoles(cat.gal, cat.ran, p, kedges, redges, ran_nbar=cat.ran_nbar)
    finally:
        ctx.set_field_chunk(0)
    check_multipoles(got["pk"], ref["pk"], "pk", label=f"mode {mode} ranges P: ")
    check_multipoles(got["xi"], ref["xi"], "xi", label=f"mode {mode} ranges xi: ")


def test_xi_only_ranges_of_two(env, cat):
    # a small-memory midpoint request (xi only, order 1, g fields two at a time: four meshes on
    # the device) through cuFFT and through the hybrid backend's fused convolution x pass
    torch, pkg, lib, ctx = env
    p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=4, los="midpoint",
                        order=1, compensate=True, precision=32)
    redges = np.arange(10.0, 190.01, 10.0)
    out = {}
    ctx.set_field_chunk(2)
    try:
        for mode in (0, 4, 6):
            assert lib.bym_set_fft_backend(ctx._h, mode) == 0
            out[mode] = ctx.xi_multipoles(cat.gal, cat.ran, p, redges, ran_nbar=cat.ran_nbar)
    finally:
        ctx.set_field_chunk(0)
    for mode in (4, 6):
        check_multipoles(out[mode]["xi"], out[0]["xi"], "xi", label=f"xi-only ranges of two, mode {mode}: ")


def _slab(rng, lo, box, n, x_ranges, y_ranges=None):
    """n points uniform in the x slabs given (cell units) of the 512^3 mesh box, in y in the y slabs
    given (cell units; default the middle half), the middle half in z."""
    h = box / N
    xs = np.concatenate([rng.uniform(a, b, n // len(x_ranges)) for a, b in x_ranges]) * h
    if y_ranges is None:
        ys = rng.uniform(0.25, 0.75, size=len(xs)) * box
    else:
        ys = np.concatenate([rng.uniform(a, b, n // len(y_ranges)) for a, b in y_ranges]) * h
        ys = rng.permutation(ys)
    zs = rng.uniform(0.25, 0.75, size=len(xs)) * box
    pts = np.column_stack([xs, ys, zs]) + lo[None, :]
    return np.column_stack([pts, np.ones(len(pts))]).astype(np.float32)


@pytest.mark.parametrize("geometry", ["wraps", "top", "middle", "y wraps", "y top"])
def test_occupied_plane_range_edges(env, geometry):
    # the library x pass backends transform only the occupied x planes forward (and the library's
    # own plane passes only the occupied rows y of them): catalogs that wrap across the periodic
    # x boundary (every plane range), a thin slab at the top of the mesh (the range shifted down to
    # fit) and one in the middle; then a slab wrapping in y and one at the top in y; against the
    # cuFFT backend
    torch, pkg, lib, ctx = env
    lo, box = np.array([1000.0, 1000.0, 1000.0]), 1024.0
    x_ranges = {"wraps": [(0.2, 2.5), (508.5, 511.8)], "top": [(500.3, 509.7)], "middle": [(200.2, 205.9)],
                "y wraps": [(100.5, 140.5)], "y top": [(300.1, 330.9)]}[geometry]
    y_ranges = {"y wraps": [(0.3, 3.5), (507.5, 511.6)], "y top": [(480.2, 511.4)]}.get(geometry)
    rng = np.random.default_rng(5)
    gal = _slab(rng, lo, box, 20000, x_ranges, y_ranges)
    ran = _slab(rng, lo, box, 200000, x_ranges, y_ranges)
    nbar = np.full(len(ran), len(gal) / (box ** 3 / 4 * 0.01), np.float32)
    h = box / N
    kedges = np.linspace(0.0, 0.8 * math.pi / h, 9)
    redges = np.linspace(0.0, 12 * h, 7)
    for los, K in (("yamamoto", 0), ("midpoint", 2), ("bisector", 2)):
        p = pkg.make_params(box_lo=lo, box_len=box, n_mesh=N, assign=3, ell_max=4, los=los, order=K,
                            compensate=True, precision=32)
        out = {}
        for m in (0, 4, 5, 6):
            assert lib.bym_set_fft_backend(ctx._h, m) == 0
            out[m] = ctx.pk_xi_multipoles(gal, ran, p, kedges, redges, ran_nbar=nbar)
        for m in (4, 5, 6):
            check_multipoles(out[m]["pk"], out[0]["pk"], "pk", label=f"{geometry} {los} mode {m} P: ")
            check_multipoles(out[m]["xi"], out[0]["xi"], "xi", label=f"{geometry} {los} mode {m} xi: ")
    assert lib.bym_set_fft_backend(ctx._h, 1) == 0


@pytest.mark.parametrize("n_mesh,prec", [(96, 64), (256, 32), (160, 32)])
def test_cufft_plane_backend_any_mesh(env, cat, n_mesh, prec):
    # backend 5: cuFFT 2D plane transforms (forward over the occupied planes of the cap) and cuFFT
    # 1D transforms along x, for meshes the library's own kernels do not cover, against cuFFT 3D
    torch, pkg, lib, ctx = env
    kedges = np.linspace(0.0, 0.8 * math.pi / (cat.box_len / n_mesh), 9)
    redges = np.arange(10.0, 190.01, 20.0)
    tol = (1e-10, 1e-10) if prec == 64 else (1e-5, 1e-4)
    for los, K in (("yamamoto", 0), ("midpoint", 2), ("bisector", 2)):
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=n_mesh, assign=3, ell_max=4, los=los,
                            order=K, compensate=True, precision=prec)
        out = {}
        for m in (0, 5):
            assert lib.bym_set_fft_backend(ctx._h, m) == 0
            out[m] = ctx.pk_xi_multipoles(cat.gal, cat.ran, p, kedges, redges, ran_nbar=cat.ran_nbar)
        check_multipoles(out[5]["pk"], out[0]["pk"], "pk", *tol, label=f"N={n_mesh} {los} P: ")
        check_multipoles(out[5]["xi"], out[0]["xi"], "xi", *tol, label=f"N={n_mesh} {los} xi: ")
    assert lib.bym_set_fft_backend(ctx._h, 1) == 0

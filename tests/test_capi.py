"""CPU checks of the C ABI: the library builds, loads, exports every function
declared in include/bym.h, reports its version, sizes requests, rejects bad
parameters, and its kernel generator compiles (NVRTC needs no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2102_08384_gb300 import build
    build.build()
    import paper_2102_08384_gb300 as pkg
    return pkg


def _declared_functions():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if path.endswith(".h"):
            src = open(os.path.join(ROOT, "include", path)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bym_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    names = _declared_functions()
    assert "bym_pk_multipoles" in names and "bym_xi_multipoles" in names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_footprint(pkg):
    assert "sm_103a" in pkg.version()
    p = pkg.make_params(box_lo=(0, 0, 0), box_len=1000.0, n_mesh=512, ell_max=4, los="bisector", order=4)
    b = pkg.footprint(p, 10**6, 10**7, True, True)
    slot = 512 * 512 * 514 * 4
    assert b >= (1 + 49 + 15) * slot
    p.los = 1
    assert pkg.footprint(p, 0, 0, True, False) >= (1 + 145 + 15) * slot
    p.precision = 64
    assert pkg.footprint(p, 0, 0, True, False) >= 2 * (1 + 145 + 15) * slot


def test_rejects_unsupported_parameters(pkg):
    for kw in (dict(ell_max=3), dict(ell_max=10), dict(order=13), dict(n_mesh=6), dict(n_mesh=2048)):
        args = dict(box_lo=(0, 0, 0), box_len=1000.0, n_mesh=64, ell_max=4)
        args.update(kw)
        with pytest.raises(pkg.BymError) as ei:
            pkg.footprint(pkg.make_params(**args), 1, 1)
        assert ei.value.code == -6


@pytest.mark.parametrize("los,order,precision", [("yamamoto", 0, 32), ("midpoint", 4, 32),
                                                 ("bisector", 4, 32), ("midpoint", 2, 64),
                                                 ("midpoint_even", 4, 32)])
def test_generated_kernels_compile(pkg, los, order, precision):
    p = pkg.make_params(box_lo=(0, 0, 0), box_len=1000.0, n_mesh=64, ell_max=4, los=los, order=order,
                        precision=precision)
    pkg.jit_check(p)


def test_create_without_gpu_fails_cleanly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.BymError):
        pkg.Context(0)

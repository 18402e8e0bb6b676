"""The C-ABI library builds, loads and exports every symbol of include/tsbz.h;
its host-side method helpers (Eqs. 8, 10, 15 and the Halton sequence) agree
with the oracle's independent implementations.  No GPU is used."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import dynamics, kpoints

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_00920_gb300 import _lib, build_library
    build_library()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "tsbz.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = sorted(set(re.findall(r"\b(tsbz_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_version(lib):
    assert lib.tsbz_version() >= 10000


@pytest.mark.parametrize("mp,shift", [((2, 2, 2), (0, 0, 0)), ((4, 4, 4), (0.125, 0.375, 0.875)),
                                      ((3, 2, 5), (0.3, 0.7, 0.1)), ((1, 1, 1), (0.5, 0.5, 0.5))])
def test_kpoints_match_oracle(lib, mp, shift):
    from paper_2112_00920_gb300 import shifted_kpoints
    a = (10.26, 9.0, 11.5)
    np.testing.assert_allclose(shifted_kpoints(a, mp, shift), kpoints.kpoints_cartesian(a, mp, shift),
                               rtol=0, atol=4e-16)


def test_halton_matches_oracle(lib):
    from paper_2112_00920_gb300 import halton
    np.testing.assert_array_equal(halton(40), np.array(kpoints.halton_shifts(40)))


def test_pulse_matches_oracle(lib):
    from paper_2112_00920_gb300 import pulse_samples
    p = W.Pulse()
    got = pulse_samples(p.e0, p.omega0, p.t_pulse, p.direction, 0.04, 500)
    ref = dynamics.field_samples(p, 0.04, 500)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-16)


def test_host_helpers_reject_bad_arguments(lib):
    import ctypes
    from paper_2112_00920_gb300._lib import _dptr
    out = np.zeros(3)
    assert lib.tsbz_halton(5, _dptr(out), out.size) == -1
    a = np.array([1.0, 1.0, 0.0])
    mp = (ctypes.c_int * 3)(1, 1, 1)
    assert lib.tsbz_shifted_kpoints(_dptr(a), mp, _dptr(np.zeros(3)), _dptr(out), 3) == -1


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2112_00920_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved

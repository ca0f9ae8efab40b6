"""The C-ABI library builds, loads and exports every declared entry point (no GPU).

Only host-side logic is exercised: status strings, default parameters and the
argument checks that run before any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    with open(os.path.join(ROOT, "include", "purify.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(purify_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_4370_gb300 import binding, build

    build.build_library()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1307_4370_gb300 import binding

    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.declared_symbols()) == names


def test_status_strings(lib):
    assert lib.purify_status_string(0) == b"ok"
    for code in range(-7, 0):
        s = lib.purify_status_string(code)
        assert s and s != b"unknown status"
    assert lib.purify_status_string(-99) == b"unknown status"


def test_default_params(lib):
    from paper_1307_4370_gb300 import binding

    p = binding.default_params()
    assert (p.max_iters, p.cg_iters, p.rounds, p.check_every) == (300, 10, 1, 0)
    assert (p.beta, p.xi, p.tau) == (1e-3, 1e-3, 0.1)


@pytest.mark.parametrize("field,value,code", [
    ("n", 7, -2), ("n", 20, -2), ("n", 4096 * 2, -2), ("J", 5, -2), ("J", 10, -2),
    ("oversample", 3, -2), ("levels", 0, -2), ("levels", 7, -2), ("M", 0, -2),
    ("bases_mask", 0, -1), ("bases_mask", 0x200, -1), ("n", 80, -7),
    ("tile", 12, -2), ("tile", 2, -2), ("tile", 128, -2), ("kernel", 2, -1), ("kernel", -1, -1),
])
def test_create_rejects_bad_descriptions(lib, field, value, code):
    from paper_1307_4370_gb300 import binding

    d = binding.Desc(64, 100, 4, 2, 4, 0x1FF, 0)
    setattr(d, field, value)
    if field == "n" and value == 80:
        d.levels = 4  # 80 = 16 * 5: 2n = 160 has the prime factor 5
    out = ctypes.c_void_p(1)
    uv = (ctypes.c_float * 2)()
    rc = lib.purify_create(ctypes.byref(out), ctypes.byref(d), ctypes.cast(uv, ctypes.c_void_p), None)
    assert rc == code
    assert out.value is None


def test_null_arguments(lib):
    from paper_1307_4370_gb300 import binding

    d = binding.Desc(64, 100, 4, 2, 4, 0x1FF, 0)
    assert lib.purify_create(None, ctypes.byref(d), None, None) == -1
    out = ctypes.c_void_p()
    assert lib.purify_create(ctypes.byref(out), None, None, None) == -1
    assert lib.purify_phi(None, None, None, None) == -1
    assert lib.purify_sdmm_step(None, None, None) == -1
    assert lib.purify_set_beam(None, None, None) == -1
    assert lib.purify_sdmm_set_blocks(None, None, 0, None, None, None) == -1
    assert lib.purify_sdmm_set_prior(None, None, 1, 20) == -1
    assert lib.purify_prox_tv(None, None, None, ctypes.c_float(1.0), 20, None, None) == -1
    lib.purify_destroy(None)
    lib.purify_sdmm_state_destroy(None)

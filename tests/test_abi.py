"""The C-ABI library builds, loads and exports every declared entry point (CPU only).

No compute call is made here (there is no GPU): only argument validation
paths that return before touching the device, and pure host queries.
"""
import os
import re

import pytest

import __graft_entry__
from paper_2001_04109_gb300 import ffsyrk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ffsyrk.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ffsyrk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:ffsyrk|ffherk)\w*)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "ffsyrk" in names and "ffsyrk_batched" in names and "ffsyrk_plan" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ffsyrk.EXPORTS)


def test_status_strings_and_version(lib):
    for code in range(9):
        s = ffsyrk.status_string(code)
        assert s.startswith("FFSYRK_")
    assert lib.ffsyrk_version() >= 100


@pytest.mark.parametrize("p,code", [(4, ffsyrk.ERR_NOT_PRIME), (65535, ffsyrk.ERR_NOT_PRIME),
                                    (2, ffsyrk.ERR_UNSUPPORTED_P), (1 << 24, ffsyrk.ERR_UNSUPPORTED_P),
                                    (16777259, ffsyrk.ERR_UNSUPPORTED_P), (0, ffsyrk.ERR_UNSUPPORTED_P)])
def test_bad_primes_rejected_before_any_device_work(lib, p, code):
    import ctypes
    h = ctypes.c_void_p(123)
    assert lib.ffsyrk_plan(ctypes.byref(h), p, 10, 10, None) == code
    assert h.value is None
    assert lib.ffsyrk(0, 4, 4, p, None, 4, None, 4, None) == code


def test_bad_arguments_rejected(lib):
    import ctypes
    assert lib.ffsyrk(0, -1, 4, 65521, None, 4, None, 4, None) == ffsyrk.ERR_INVALID_ARG
    assert lib.ffsyrk_with_plan(None, 0, 4, 4, 65521, None, 4, None, 4, None) == ffsyrk.ERR_INVALID_ARG
    assert lib.ffsyrk_plan(None, 65521, 4, 4, None) == ffsyrk.ERR_INVALID_ARG
    o = ffsyrk.Options()
    lib.ffsyrk_options_default(ctypes.byref(o))
    assert o.leaf == ffsyrk.LEAF_AUTO and o.levels == ffsyrk.LEVELS_AUTO and o.winograd == -1
    o.levels = 99
    h = ctypes.c_void_p()
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.levels = 1
    o.reserved = 5
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.reserved = 0
    o.epilogue_warps = 12
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.epilogue_warps = 0
    o.digit_products = 3
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.digit_products = 0
    o.unit_bounds = 2
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.unit_bounds = 0
    assert lib.ffsyrk_plan_units(None, None, None, None) == ffsyrk.ERR_INVALID_ARG
    o.winograd = -2
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    # batched argument checks happen before any device call
    I64 = ctypes.c_int64 * 1
    VP = ctypes.c_void_p * 1
    assert lib.ffsyrk_batched(0, 1, I64(-3), I64(4), 65521, VP(), I64(4), VP(), I64(4), None) == \
        ffsyrk.ERR_INVALID_ARG
    assert lib.ffsyrk_batched(0, 0, None, None, 65521, None, None, None, None, None) == ffsyrk.SUCCESS
    assert lib.ffsyrk_batched(0, 1, I64(4), I64(4), 65521, VP(None), I64(4), VP(None), I64(4), None) == \
        ffsyrk.ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(ffsyrk, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ffsyrk, "_lib", None)
    with pytest.raises(FileNotFoundError):
        ffsyrk.lib()


def test_autotune_option_validated(lib):
    import ctypes
    o = ffsyrk.Options()
    lib.ffsyrk_options_default(ctypes.byref(o))
    assert o.autotune == 0 and o.tile_ctas == 0
    o.autotune = 2
    h = ctypes.c_void_p()
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG
    o.autotune = 0
    o.tile_ctas = 3
    assert lib.ffsyrk_plan(ctypes.byref(h), 65521, 4, 4, ctypes.byref(o)) == ffsyrk.ERR_INVALID_ARG


def test_workspace_query_without_gpu(lib):
    # capacity planning on the host: the workspace a plan would allocate
    ws = {n: ffsyrk.workspace_query(65521, n, n)[0] for n in (1024, 4096, 8192)}
    assert 0 < ws[1024] < ws[4096] < ws[8192]
    # Winograd levels add their uint32 operands, pieces and products
    sb = "schoolbook"
    on = ffsyrk.workspace_query(8388593, 32768, 32768, levels=3, digit_products=sb)[0]
    off = ffsyrk.workspace_query(8388593, 32768, 32768, levels=3, winograd=0, digit_products=sb)[0]
    assert on > 2 * off > 0
    # Karatsuba digit products add the digit-sum planes (6 planes per operand instead of 3)
    ks = ffsyrk.workspace_query(8388593, 32768, 32768, levels=3, winograd=0, digit_products="karatsuba")[0]
    assert ks > off
    # the int64 leaf has no shared-tile slots; the tensor leaf scales them with the SMs
    assert ffsyrk.workspace_query(65521, 4096, 4096, leaf="i64")[1] == 0
    s152 = ffsyrk.workspace_query(65521, 4096, 4096)[1]
    assert 0 < ffsyrk.workspace_query(65521, 4096, 4096, sms=76)[1] <= s152
    with pytest.raises(ffsyrk.FfsyrkError):
        ffsyrk.workspace_query(65521, -1, 4)
    with pytest.raises(ffsyrk.FfsyrkError):
        ffsyrk.workspace_query(65520, 4, 4)   # not prime


def test_other_entry_points_check_arguments_first(lib):
    # every check below returns before the device is touched
    import ctypes
    from oracle import field
    E = ffsyrk
    h = ctypes.c_void_p(123)
    # the Hermitian plan wants a prime p and i² = r a non-square mod p
    assert lib.ffherk_plan(None, 65521, 17, 8, 8, None) == E.ERR_INVALID_ARG
    assert lib.ffherk_plan(ctypes.byref(h), 65535, 3, 8, 8, None) == E.ERR_NOT_PRIME
    assert h.value is None
    for p in (13, 65521):                       # p ≡ 1 mod 4: −1 is a square there
        square = (5 * 5) % p
        assert field.legendre(p - 1, p) == 1
        for r in (0, p, p - 1, square):
            assert lib.ffherk_plan(ctypes.byref(h), p, r, 8, 8, None) == E.ERR_INVALID_ARG, (p, r)
    assert lib.ffherk_plan(ctypes.byref(h), 65521, 17, -1, 8, None) == E.ERR_INVALID_ARG
    assert lib.ffherk_plan_destroy(None) == E.SUCCESS
    assert lib.ffherk_with_plan(None, 0, 4, 4, None, 8, None, None, 4, None) == E.ERR_INVALID_ARG
    assert lib.ffherk_sync_status(None, None) == E.ERR_INVALID_ARG
    assert lib.ffherk(0, 4, 4, 4, 3, None, 8, None, None, 4, None) == E.ERR_NOT_PRIME
    assert lib.ffherk(0, -1, 4, 65521, 17, None, 8, None, None, 4, None) == E.ERR_INVALID_ARG
    # host-buffer product and the scaled products
    assert lib.ffsyrk_host(None, 0, 4, 4, 65521, None, 4, None, 4, None) == E.ERR_INVALID_ARG
    assert lib.ffsyrkbd_with_plan_update(None, 0, 4, 4, 65521, 1, None, 4, None, None, 0, None, 4,
                                         None) == E.ERR_INVALID_ARG
    assert lib.ffsyrkbd_update(0, 4, 4, 65535, 1, None, 4, None, None, 0, None, 4, None) == \
        E.ERR_NOT_PRIME
    assert lib.ffsyrkbd_update(0, 4, -1, 65521, 1, None, 4, None, None, 0, None, 4, None) == \
        E.ERR_INVALID_ARG
    assert lib.ffsyrk_update(0, 4, 4, 2, 1, None, 4, 0, None, 4, None) == E.ERR_UNSUPPORTED_P


def test_rebuild_tracks_every_included_header():
    """The library is rebuilt when any file it is compiled from changes: every
    header a source includes by a quoted name must be among the build's
    dependencies, .cuh device helpers included."""
    from paper_2001_04109_gb300 import build as b
    deps = {os.path.abspath(d) for d in b.dependencies()}
    for src in b.sources():
        for m in re.finditer(r'#include\s+"([^"]+)"', open(src).read()):
            path = os.path.abspath(os.path.join(os.path.dirname(src), m.group(1)))
            assert path in deps, f"{os.path.basename(src)} includes {m.group(1)}, not a build dependency"

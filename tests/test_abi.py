"""The C ABI: every symbol declared in include/dic.h is exported by the
library, the Python binding covers it, and host-side argument checking works
without a GPU (no compute call is made here)."""
import os
import re

import pytest

import paper_1905_06228_gb300 as dic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dic_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    dic.build()
    return dic.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_declarations():
    assert _declared() <= set(dic.SIGNATURES)


def test_version(lib):
    assert dic.dic_version() >= 10000


@pytest.mark.parametrize("args", [
    (4, 5, 10), (1, 5, 10), (65, 5, 10), (21, 0, 10), (21, 5, -1),
])
def test_create_rejects_bad_arguments(args):
    with pytest.raises(dic.DICError) as e:
        dic.dic_create(*args)
    assert e.value.code == dic.DIC_ERR_ARG


def test_create_rejects_bad_tolerance_and_iterations():
    for tol, it in ((0.0, 50), (-1.0, 50), (1e-3, 0)):
        with pytest.raises(dic.DICError):
            dic.dic_create(21, 5, 10, 1, tol, it)


def test_shape_orders():
    """Orders 1 and 2 are built; each refines through its own call (the
    other returns DIC_ERR_STATE before any device work); others are refused."""
    for order in (0, 3):
        with pytest.raises(dic.DICError) as e:
            dic.dic_create(21, 5, 10, order)
        assert e.value.code == dic.DIC_ERR_UNSUPPORTED
    lib = dic.lib()
    h1 = dic.dic_create(21, 5, 10, 1)
    h2 = dic.dic_create(21, 5, 10, 2)
    try:
        assert lib.dic_subpixel2(h1, 0, *[16] * 7) == dic.DIC_ERR_STATE
        assert lib.dic_subpixel(h2, 0, *[16] * 12) == dic.DIC_ERR_STATE
        assert lib.dic_subpixel2(h2, 1, *[16] * 7) == dic.DIC_ERR_UNSUPPORTED
        assert lib.dic_subpixel2(h2, 0, *[16] * 7) == dic.DIC_ERR_STATE  # no pair
    finally:
        dic.dic_destroy(h1)
        dic.dic_destroy(h2)


def test_state_errors_before_set_pair():
    h = dic.dic_create(21, 5, 10)
    try:
        with pytest.raises(dic.DICError) as e:
            dic.dic_num_pois(h)
        assert e.value.code == dic.DIC_ERR_STATE
        assert "no image pair" in dic.dic_last_error(h)
        with pytest.raises(dic.DICError) as e:
            dic.dic_integer_search(h, 0, 0, 0, 0)
        assert e.value.code == dic.DIC_ERR_STATE
        with pytest.raises(dic.DICError) as e:
            dic.dic_set_solve_precision(h, 16)
        assert e.value.code == dic.DIC_ERR_ARG
        dic.dic_set_solve_precision(h, 64)
    finally:
        dic.dic_destroy(h)


def test_set_pair_rejects_null_and_bad_sizes():
    lib = dic.lib()
    h = dic.dic_create(21, 5, 10)
    try:
        assert lib.dic_set_pair(h, None, None, 64, 64, 64) == dic.DIC_ERR_ARG
        assert lib.dic_set_pair(h, 16, 16, 2, 64, 64) == dic.DIC_ERR_ARG
        assert lib.dic_set_pair(h, 16, 16, 64, 64, 32) == dic.DIC_ERR_ARG
    finally:
        dic.dic_destroy(h)


def test_destroy_null_is_harmless():
    dic.lib().dic_destroy(None)


def test_batch_calls_without_a_batch():
    """Batch entry points check their state on the host: no batch bound ->
    DIC_ERR_STATE, null handle -> DIC_ERR_ARG (no device work is issued)."""
    lib = dic.lib()
    assert lib.dic_set_batch_shape(None, 4, 1) == dic.DIC_ERR_ARG
    assert lib.dic_run_batch(None, 0, None) == dic.DIC_ERR_ARG
    assert lib.dic_autotune(None, 0, None, None) == dic.DIC_ERR_ARG
    h = dic.dic_create(21, 5, 10)
    try:
        assert lib.dic_set_batch_shape(h, 4, 1) == dic.DIC_ERR_STATE
        assert lib.dic_run_batch(h, 0, None) == dic.DIC_ERR_STATE
        assert lib.dic_autotune(h, 0, None, None) == dic.DIC_ERR_STATE
        assert lib.dic_batch_pois(h, None, None) == dic.DIC_ERR_STATE
        assert lib.dic_set_pairs(h, 0, None) == dic.DIC_ERR_ARG
    finally:
        dic.dic_destroy(h)


def test_form_and_noalloc_argument_checks():
    lib = dic.lib()
    h = dic.dic_create(21, 5, 10)
    try:
        assert lib.dic_set_form(h, 7) == dic.DIC_ERR_ARG
        assert lib.dic_set_form(h, dic.DIC_FORM_BF16TC) == dic.DIC_OK
    finally:
        dic.dic_destroy(h)
    # images beyond the static array's limit are refused before any device work
    args = [16, 16, 1024, 1024, 1024, 21, 5, 10, 0, 1e-3, 50, 32] + [None] * 13
    assert lib.dic_subpixel_noalloc(*args) == dic.DIC_ERR_ARG
    # a search radius beyond dic_create's bound is refused on the host (the
    # margin M + R + 2 would overflow for radii near INT_MAX)
    for radius in (1001, 2**31 - 1):
        args = [16, 16, 256, 256, 256, 21, 5, radius, 0, 1e-3, 50, 32] + [None] * 13
        assert lib.dic_subpixel_noalloc(*args) == dic.DIC_ERR_ARG


def test_check_before_any_launch():
    """dic_check on a fresh handle has no flag to read: DIC_OK without any
    device work; a null handle is DIC_ERR_ARG."""
    lib = dic.lib()
    assert lib.dic_check(None) == dic.DIC_ERR_ARG
    h = dic.dic_create(21, 5, 10)
    try:
        assert lib.dic_check(h) == dic.DIC_OK
    finally:
        dic.dic_destroy(h)


def test_measure_peak_argument_checks():
    """Unknown kinds and a null output are refused on the host, before any
    device work."""
    lib = dic.lib()
    import ctypes
    r = ctypes.c_double()
    assert lib.dic_measure_peak(7, None, ctypes.byref(r)) == dic.DIC_ERR_ARG
    assert lib.dic_measure_peak(-1, None, ctypes.byref(r)) == dic.DIC_ERR_ARG
    assert lib.dic_measure_peak(dic.DIC_PEAK_FP32_FMA, None, None) == dic.DIC_ERR_ARG


def test_stream_calls_host_side_checks():
    """Frame-stream entry points refuse null handles and frames and bad sizes
    before any device work."""
    lib = dic.lib()
    assert lib.dic_stream_flush(None) == dic.DIC_ERR_ARG
    assert lib.dic_stream_reset(None) == dic.DIC_ERR_ARG
    assert lib.dic_stream_push(None, 16, 64, 64, 64, 0, None) == dic.DIC_ERR_ARG
    h = dic.dic_create(21, 5, 10)
    try:
        assert lib.dic_stream_flush(h) == dic.DIC_OK   # nothing pushed yet
        assert lib.dic_stream_reset(h) == dic.DIC_OK
        assert lib.dic_stream_push(h, None, 64, 64, 64, 0, None) == dic.DIC_ERR_ARG
        assert lib.dic_stream_push(h, 16, 2, 64, 64, 0, None) == dic.DIC_ERR_ARG
        assert lib.dic_stream_push(h, 16, 64, 64, 32, 0, None) == dic.DIC_ERR_ARG
        assert lib.dic_stream_push(h, 16, 64, 64, 64, 5, None) == dic.DIC_ERR_ARG
    finally:
        dic.dic_destroy(h)

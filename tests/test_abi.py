"""The C-ABI library loads on a machine without a GPU, exports every entry point that
include/ssg.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1907_06146_gb300 import build_ext, ssg, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_ext.build()
    return ssg.lib()


def _declared():
    with open(os.path.join(ROOT, "include", "ssg.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    # and the binding declares argument types for each of them
    assert set(names) <= set(ssg.SYMBOLS)


def test_nav_ids_match_generator(L):
    for n, s, seed in [(1000, 10, 1), (17, 17, 2), (10_000_000, 10, 190706145)]:
        np.testing.assert_array_equal(ssg.nav_ids(n, s, seed), synth.nav_ids(n, s, seed))


def test_nav_ids_rejects(L):
    out = np.empty(4, np.int32)
    assert L.ssg_nav_ids(3, 4, 0, out.ctypes.data_as(ctypes.c_void_p)) == 1
    assert b"s <= n" in L.ssg_last_error()


def test_strerror(L):
    assert L.ssg_strerror(0) == b"ok"
    assert L.ssg_strerror(1) == b"invalid argument"
    assert L.ssg_strerror(99) == b"unknown status"


def test_invalid_arguments_rejected_without_device(L):
    P = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    s = ctypes.c_void_p(0)
    # K > n - 1
    assert L.ssg_knn(P, 10, 4, 10, 0, P, P, s) == 1
    # K too large for the selection buffers
    assert L.ssg_knn(P, 10_000, 4, 701, 0, P, P, s) == 1
    # null output
    assert L.ssg_knn(P, 10, 4, 3, 0, None, P, s) == 1
    # L + K too large
    assert L.ssg_pool(P, 5000, 8, P, 600, 500, P, P, P, s) == 1
    # alpha outside (0, 180)
    assert L.ssg_prune(P, 100, 8, P, P, 10, 8, 0.0, P, P, s) == 1
    assert L.ssg_prune(P, 100, 8, P, P, 10, 8, 180.0, P, P, s) == 1
    # R or d out of range
    assert L.ssg_prune(P, 100, 8, P, P, 10, 0, 60.0, P, P, s) == 1
    assert L.ssg_prune(P, 100, 8, P, P, 10, 129, 60.0, P, P, s) == 1
    assert L.ssg_prune(P, 100, 9000, P, P, 10, 70, 60.0, P, P, s) == 1
    # k > L_search
    assert L.ssg_search_adj(P, 100, 8, P, P, 8, P, 1, P, 5, 20, 10, P, P, s) == 1
    # build: n_nav > n
    opts = ssg.BuildOpts()
    L.ssg_default_opts(ctypes.byref(opts))
    opts.n_nav = 50
    h = ctypes.c_void_p()
    assert L.ssg_build(P, 20, 4, 5, 10, 8, 60.0, ctypes.byref(opts), s, ctypes.byref(h), None) == 1
    assert h.value is None
    # batched build: no streams, a host nav list, negative count; count 0 does nothing
    one = (ctypes.c_int64 * 1)(100)
    i1 = (ctypes.c_int32 * 1)(8)
    a1 = (ctypes.c_double * 1)(60.0)
    bases = (ctypes.c_void_p * 1)(16)
    graphs = (ctypes.c_void_p * 1)()
    L.ssg_default_opts(ctypes.byref(opts))
    assert L.ssg_build_batched(1, bases, one, i1, i1, i1, i1, a1, ctypes.byref(opts), 0, graphs,
                               None) == 1
    nav_one = (ctypes.c_int32 * 1)(0)
    opts.nav_ids_host = ctypes.addressof(nav_one)
    assert L.ssg_build_batched(1, bases, one, i1, i1, i1, i1, a1, ctypes.byref(opts), 2, graphs,
                               None) == 1
    assert L.ssg_build_batched(-1, None, None, None, None, None, None, None, None, 2, None,
                               None) == 1
    assert L.ssg_build_batched(0, None, None, None, None, None, None, None, None, 2, None,
                               None) == 0
    # the invariant check: outputs required, R within [1, 128]
    row, code = ctypes.c_int64(), ctypes.c_int32()
    assert L.ssg_check_graph(P, P, 10, 8, None, ctypes.byref(code), s) == 1
    assert L.ssg_check_graph(P, P, 10, 0, ctypes.byref(row), ctypes.byref(code), s) == 1
    assert L.ssg_check_graph(P, P, 10, 129, ctypes.byref(row), ctypes.byref(code), s) == 1
    # the bounded-wait self-test: only modes 0..2, outputs required
    ok, ms = ctypes.c_int32(), ctypes.c_int32()
    assert L.ssg_selftest_wait(3, ctypes.byref(ok), ctypes.byref(ms)) == 1
    assert L.ssg_selftest_wait(-1, ctypes.byref(ok), ctypes.byref(ms)) == 1
    assert L.ssg_selftest_wait(0, None, ctypes.byref(ms)) == 1


def test_precision_margin_and_tune_table_rejected_without_device(L, tmp_path):
    """FP8 is declared but not built; the reporting band and the launch-parameter file are
    validated before anything reaches the device."""
    P = ctypes.c_void_p(16)
    s = ctypes.c_void_p(0)
    assert L.ssg_knn(P, 100, 8, 5, ssg.PREC["fp8"], P, P, s) == 1
    assert b"FP8" in L.ssg_last_error()
    assert L.ssg_knn(P, 100, 8, 5, 7, P, P, s) == 1
    assert L.ssg_knn_query(P, 100, 8, P, 10, 5, ssg.PREC["fp8"], P, P, s) == 1
    h = ctypes.c_void_p()

    def build_with(**fields):
        o = ssg.BuildOpts()
        L.ssg_default_opts(ctypes.byref(o))
        for k, v in fields.items():
            setattr(o, k, v)
        return L.ssg_build(P, 200, 8, 5, 10, 8, 60.0, ctypes.byref(o), s, ctypes.byref(h), None)

    assert build_with(gemm_prec=ssg.PREC["fp8"]) == 1
    assert build_with(gram_prec=ssg.PREC["fp8"]) == 1 and b"gram_prec" in L.ssg_last_error()
    assert build_with(cos_margin_fp64=-1e-3) == 1
    assert build_with(cos_margin_fp64=0.9) == 1
    missing = str(tmp_path / "absent.txt").encode()
    assert build_with(tune_table=missing) == 1 and b"cannot open" in L.ssg_last_error()
    for text, msg in [("knn_sample_rows = 9000\n", b"knn_sample_rows"),
                      ("knn_slack_quantile = 0.2\n", b"knn_slack_quantile"),
                      ("no_such_knob = 1\n", b"unknown name"),
                      ("knn_sample_rows 12\n", b"name = value")]:
        f = tmp_path / "t.txt"
        f.write_text("# launch parameters\n" + text)
        assert build_with(tune_table=str(f).encode()) == 1, text
        assert msg in L.ssg_last_error(), (text, L.ssg_last_error())
    assert h.value is None


def test_last_device_status_starts_clear(L):
    assert L.ssg_last_device_status() == 0
    assert ssg.last_device_status() == 0


def test_default_opts(L):
    o = ssg.BuildOpts()
    L.ssg_default_opts(ctypes.byref(o))
    assert o.gemm_prec == ssg.PREC["auto"] and o.n_nav == 10 and o.nav_ids_host is None
    assert o.gram_prec == ssg.PREC["auto"] and o.cos_margin_fp64 == 1e-5
    assert o.tune_table is None

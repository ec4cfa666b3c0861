"""The C ABI library without a GPU: it loads, exports every declared symbol, and
its host-side validation rejects malformed inputs (no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

from workloads import EAGLE, heavy_hex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import _abi
    _abi.load()
    return _abi


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gpeps.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(gpeps_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(abi):
    lib = abi.load()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
        assert s in abi.SIGNATURES, s
    assert set(abi.SIGNATURES) == set(syms)


def _create(abi, graphs, D=4, dtype=0, colours=None):
    lib = abi.load()
    keep = []
    arr = (abi.GraphC * len(graphs))()
    for k, (n, e) in enumerate(graphs):
        e = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 2))
        keep.append(e)
        arr[k].n_qubits = n
        arr[k].n_edges = e.shape[0]
        arr[k].edges = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if colours is not None:
            c = np.ascontiguousarray(np.asarray(colours[k], dtype=np.int8))
            keep.append(c)
            arr[k].colour = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    h = ctypes.c_void_p()
    st = lib.gpeps_create(ctypes.cast(arr, ctypes.c_void_p), len(graphs), D, dtype, None, ctypes.byref(h))
    return st, h


def test_valid_heavy_hex(abi):
    lib = abi.load()
    n, e = heavy_hex(*EAGLE)
    for dtype, elt in ((0, 16), (1, 8)):
        st, h = _create(abi, [(n, e)], D=4, dtype=dtype)
        assert st == 0
        nc = ctypes.c_int32()
        assert lib.gpeps_n_colours(h, ctypes.byref(nc)) == 0 and nc.value == 3
        q, ed = ctypes.c_int64(), ctypes.c_int64()
        assert lib.gpeps_sizes(h, ctypes.byref(q), ctypes.byref(ed)) == 0
        assert (q.value, ed.value) == (127, 144)
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.gpeps_query_workspace(h, ctypes.byref(sb), ctypes.byref(wb)) == 0
        deg = np.bincount(e.ravel(), minlength=n)
        assert sb.value >= sum(2 * 4 ** int(d) for d in deg) * elt + 144 * 4 * 8
        assert lib.gpeps_destroy(h) == 0


@pytest.mark.parametrize("graph,D,dtype", [
    ((3, [[0, 1], [1, 2]]), 0, 0),               # D < 1
    ((3, [[0, 1], [1, 2]]), 129, 0),             # D beyond the complex128 limit (128)
    ((3, [[0, 1], [1, 2]]), 65, 1),              # D beyond the mixed path's limit (64)
    ((3, [[0, 1], [1, 2]]), 4, 7),               # unknown dtype
    ((3, [[0, 1], [1, 1]]), 4, 0),               # self loop
    ((3, [[0, 1], [1, 3]]), 4, 0),               # label out of range
    ((3, [[0, 1], [1, 0]]), 4, 0),               # duplicate coupler
    ((5, [[0, 1], [0, 2], [0, 3], [0, 4]]), 4, 0),   # degree 4
    ((8, [[0, 1], [0, 2], [0, 3], [1, 4], [1, 5]]), 4, 0),  # two degree-3 ends joined
    ((0, []), 4, 0),                              # no qubits
])
def test_rejects_malformed(abi, graph, D, dtype):
    st, h = _create(abi, [graph], D=D, dtype=dtype)
    assert st == abi.GPEPS_EINVAL and not h.value


def test_rejects_colouring_that_is_not_a_matching(abi):
    st, _ = _create(abi, [(3, [[0, 1], [1, 2]])], colours=[[0, 0]])
    assert st == abi.GPEPS_EINVAL
    st, h = _create(abi, [(3, [[0, 1], [1, 2]])], colours=[[0, 1]])
    assert st == 0
    abi.load().gpeps_destroy(h)


def test_calls_before_bind_are_rejected(abi):
    lib = abi.load()
    st, h = _create(abi, [(3, [[0, 1], [1, 2]])])
    assert st == 0
    assert lib.gpeps_reset(h) == abi.GPEPS_EINVAL
    assert lib.gpeps_zz_layer(h, 0) == abi.GPEPS_EINVAL
    assert lib.gpeps_expect_z(h, None, None) == abi.GPEPS_EINVAL
    assert lib.gpeps_bind(h, ctypes.c_void_p(8), ctypes.c_void_p(256)) == abi.GPEPS_EINVAL   # misaligned
    assert lib.gpeps_destroy(h) == 0


def test_error_strings(abi):
    lib = abi.load()
    for s in range(6):
        assert lib.gpeps_error_string(s)
    assert lib.gpeps_error_string(99) == b"unknown status"


def test_product_path_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2309_15642_gb300 import GPEPS
    with pytest.raises(RuntimeError):
        GPEPS([(3, [[0, 1], [1, 2]])], 2)


def test_state_layout_host_only(abi):
    """Site and lambda offsets tile the state buffer without overlap (no GPU needed)."""
    lib = abi.load()
    n, e = heavy_hex(*EAGLE)
    D = 3
    for dtype, elt in ((0, 16), (1, 8)):
        st, h = _create(abi, [(n, e), (n, e)], D=D, dtype=dtype)
        assert st == 0
        spans = []
        for inst in range(2):
            for v in range(n):
                off, deg = ctypes.c_int64(), ctypes.c_int32()
                nb = (ctypes.c_int32 * 3)()
                assert lib.gpeps_site_layout(h, inst, v, ctypes.byref(off), ctypes.byref(deg), nb) == 0
                d = int(np.count_nonzero(e == v))
                assert deg.value == d
                assert list(nb[:d]) == sorted(int(b if a == v else a) for a, b in e if v in (a, b))
                spans.append((off.value, off.value + 2 * D ** d * elt))
            for k in range(len(e)):
                off = ctypes.c_int64()
                assert lib.gpeps_lambda_layout(h, inst, k, ctypes.byref(off)) == 0
                spans.append((off.value, off.value + D * 8))
        spans.sort()
        assert all(a[1] <= b[0] for a, b in zip(spans[:-1], spans[1:]))
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        lib.gpeps_query_workspace(h, ctypes.byref(sb), ctypes.byref(wb))
        assert spans[-1][1] <= sb.value
        off = ctypes.c_int64()
        assert lib.gpeps_lambda_layout(h, 2, 0, ctypes.byref(off)) == abi.GPEPS_EINVAL
        lib.gpeps_destroy(h)


def test_tensor_core_switch_host_checks(abi):
    """gpeps_set_tensor_cores (host-only): accepted for the complex64 path at D = 32 and 64,
    rejected for complex128, for other bond dimensions and for a NULL handle; off is always
    accepted."""
    lib = abi.load()
    n, e = heavy_hex(*EAGLE)
    assert lib.gpeps_set_tensor_cores(None, 1) == abi.GPEPS_EINVAL
    for dtype, D, ok in ((1, 32, True), (1, 64, True), (1, 16, False), (1, 8, False), (0, 32, False),
                         (0, 64, False)):
        st, h = _create(abi, [(n, e)], D=D, dtype=dtype)
        assert st == 0
        assert lib.gpeps_set_tensor_cores(h, 1) == (0 if ok else abi.GPEPS_EINVAL), (dtype, D)
        assert lib.gpeps_set_tensor_cores(h, 0) == 0
        assert lib.gpeps_destroy(h) == 0


def test_schedule_host_checks(abi):
    """gpeps_set_schedule (host-only): 0 and 1 need nothing bound; 2 to 6 need the work buffer
    and are rejected on an unbound handle; values outside 0..6 and a NULL handle are rejected."""
    lib = abi.load()
    n, e = heavy_hex(*EAGLE)
    assert lib.gpeps_set_schedule(None, 0) == abi.GPEPS_EINVAL
    for dtype in (0, 1):
        st, h = _create(abi, [(n, e)], D=32, dtype=dtype)
        assert st == 0
        for s in (0, 1):
            assert lib.gpeps_set_schedule(h, s) == 0, (dtype, s)
        for s in (2, 3, 4, 5, 6, 7, -1):
            assert lib.gpeps_set_schedule(h, s) == abi.GPEPS_EINVAL, (dtype, s)
        assert lib.gpeps_destroy(h) == 0

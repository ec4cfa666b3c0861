"""gpeps_bond_update_noalloc: the bond update for callers that cannot allocate device memory.

It is called through the C ABI on copies of two site tensors taken from a
handle, and must give what gpeps_zz_layer gives on the same bond, on two calls
in a row (the second without kicks), within the parity tolerances of the other
GPU tests (1e-10 complex128, 1e-4 mixed).  This file is collected last so that
a run stopping at the first failure has run every other test first; it also
passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "mixed": 1e-4}
# a degree-3 site (0) bonded to a degree-2 site (1): edge 0 = (0, 1) is the only edge of colour 0
EDGES = [[0, 1], [0, 2], [0, 3], [1, 4]]


def _lib_and_cls():
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import GPEPS, _abi
    return _abi.load(), _abi, GPEPS


@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_noalloc_matches_zz_layer_on_two_calls(dtype):
    import torch
    lib, abi, GPEPS = _lib_and_cls()
    D, th = 8, 0.8
    g = GPEPS([(5, EDGES)], D, dtype=dtype)
    g.reset()
    theta = torch.tensor([th], dtype=torch.float64, device="cuda")
    g.step(2, theta)                         # a state with full bonds
    g.synchronize()
    ga, nba = g.site_tensor(0, 0)
    gb, nbb = g.site_tensor(0, 1)
    assert nba == [1, 2, 3] and nbb == [0, 4]
    A = ga.clone()
    B = gb.clone()
    lam = torch.zeros((5, D), dtype=torch.float64, device="cuda")
    lam[0] = g.lambda_tensor(0, 0)           # the bond (0, 1)
    lam[1] = g.lambda_tensor(0, 1)           # site 0, legs to 2 and 3
    lam[2] = g.lambda_tensor(0, 2)
    lam[3] = g.lambda_tensor(0, 3)           # site 1, leg to 4
    dt = abi.GPEPS_C128 if dtype == "c128" else abi.GPEPS_MIXED_C64
    torch.cuda.synchronize()
    for call, angle in enumerate((th, 0.0)):
        # existing entry point: a kick (first call only) then colour class 0
        if angle:
            g.kick(theta)
        g.zz_layer(0)
        g.synchronize()
        ang = (ctypes.c_double * 2)(angle, angle)
        flags = ctypes.c_int32(-1)
        st = lib.gpeps_bond_update_noalloc(D, dt, ctypes.c_void_p(A.data_ptr()), 3, 0,
                                           ctypes.c_void_p(B.data_ptr()), 2, 0,
                                           ctypes.c_void_p(lam.data_ptr()), ang, None, ctypes.byref(flags))
        assert st == 0 and flags.value == 0, (call, st, flags.value)
        torch.cuda.synchronize()
        ref_a, _ = g.site_tensor(0, 0)
        ref_b, _ = g.site_tensor(0, 1)
        assert (A - ref_a).abs().max().item() < TOL[dtype], call
        assert (B - ref_b).abs().max().item() < TOL[dtype], call
        assert (lam[0] - g.lambda_tensor(0, 0)).abs().max().item() < TOL[dtype], call
    g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib, abi, _ = _lib_and_cls()
    import torch
    x = torch.zeros(64, dtype=torch.complex128, device="cuda")
    y = torch.zeros(64, dtype=torch.complex128, device="cuda")
    lam = torch.zeros(5 * 64, dtype=torch.float64, device="cuda")
    args = (ctypes.c_void_p(x.data_ptr()),)
    for D, da, db in ((33, 2, 2), (0, 2, 2), (4, 3, 3), (4, 4, 2)):
        st = lib.gpeps_bond_update_noalloc(D, abi.GPEPS_C128, args[0], da, 0, ctypes.c_void_p(y.data_ptr()), db, 0,
                                           ctypes.c_void_p(lam.data_ptr()), None, None, None)
        assert st == abi.GPEPS_EINVAL

"""gpeps_bond_update_noalloc: the bond update for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc once they run: a host framework that owns
every device allocation through its own pool, or a latency-critical loop that
must not pay for (and synchronise on) an allocation.  For them the library
offers one bond update that works only on the tensors they pass and on a
fixed scratch array inside the library.

It is called through the C ABI on copies of two site tensors taken from a
handle, and must give what gpeps_zz_layer gives on the same bond, on two calls
in a row (the second without kicks), within the parity tolerances of the other
GPU tests (1e-10 complex128, 1e-4 mixed).  Cases: a degree-3 end at D = 8 and
at D = 32 (1024 rows in 16 tiles, the largest layout of the scratch), the same
bond with the ends passed in the other order (degree of a below that of b), a
bond between two degree-2 sites, a degree-2 site bonded to a degree-1 site, and
calls without kick angles (theta = NULL).  Repeated calls after the first leave
the device's free memory unchanged.  This file is collected last so that a run
stopping at the first failure has run every other test first; it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "mixed": 1e-4}
# STAR: a degree-3 site (0) bonded to a degree-2 site (1); greedy colours: (0,1) -> 0,
# (0,2) -> 1, (0,3) -> 2, (1,4) -> 1 (site 4 has degree 1).  PATH: 0-1-2-3, (1,2) alone in colour 1.
STAR = [[0, 1], [0, 2], [0, 3], [1, 4]]
PATH = [[0, 1], [1, 2], [2, 3]]
CASES = {  # name: (graph, D, site passed as a, site passed as b, colour of the bond)
    "deg3_first_d8": (STAR, 8, 0, 1, 0),
    "deg3_first_d32": (STAR, 32, 0, 1, 0),
    "deg3_second_d32": (STAR, 32, 1, 0, 0),
    "deg2_deg2_d16": (PATH, 16, 1, 2, 1),
    "deg2_deg1_d8": (STAR, 8, 1, 4, 1),
    "deg1_deg2_d8": (STAR, 8, 4, 1, 1),
}


def _lib_and_cls():
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import GPEPS, _abi
    return _abi.load(), _abi, GPEPS


def _edge(edges, u, v):
    return next(k for k, (x, y) in enumerate(edges) if {x, y} == {u, v})


@pytest.mark.parametrize("kick", [True, False], ids=["kick", "no_theta"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", ["c128", "mixed"])
def test_noalloc_matches_zz_layer_on_two_calls(dtype, case, kick):
    import torch
    lib, abi, GPEPS = _lib_and_cls()
    edges, D, a, b, colour = CASES[case]
    n = max(max(e) for e in edges) + 1
    th = 0.8
    g = GPEPS([(n, edges)], D, dtype=dtype)
    g.reset()
    theta = torch.tensor([th], dtype=torch.float64, device="cuda")
    g.step(3, theta)                         # a state with non-trivial bonds
    g.synchronize()
    ga, nba = g.site_tensor(0, a)
    gb, nbb = g.site_tensor(0, b)
    A, B = ga.clone(), gb.clone()
    lam = torch.zeros((5, D), dtype=torch.float64, device="cuda")
    e_ab = _edge(edges, a, b)
    lam[0] = g.lambda_tensor(0, e_ab)
    for row0, site, nbs, other in ((1, a, nba, b), (3, b, nbb, a)):
        for r, v in enumerate(x for x in nbs if x != other):
            lam[row0 + r] = g.lambda_tensor(0, _edge(edges, site, v))
    dt = abi.GPEPS_C128 if dtype == "c128" else abi.GPEPS_MIXED_C64
    torch.cuda.synchronize()
    for call in range(2):
        angle = th if (kick and call == 0) else 0.0
        if angle:
            g.kick(theta)                    # existing entry point: the kick, then the colour class
        g.zz_layer(colour)
        g.synchronize()
        ang = (ctypes.c_double * 2)(angle, angle) if kick else None
        flags = ctypes.c_int32(-1)
        st = lib.gpeps_bond_update_noalloc(D, dt, ctypes.c_void_p(A.data_ptr()), len(nba), nba.index(b),
                                           ctypes.c_void_p(B.data_ptr()), len(nbb), nbb.index(a),
                                           ctypes.c_void_p(lam.data_ptr()), ang, None, ctypes.byref(flags))
        assert st == 0 and flags.value == 0, (call, st, flags.value)
        torch.cuda.synchronize()
        ref_a, _ = g.site_tensor(0, a)
        ref_b, _ = g.site_tensor(0, b)
        assert (A - ref_a).abs().max().item() < TOL[dtype], call
        assert (B - ref_b).abs().max().item() < TOL[dtype], call
        assert (lam[0] - g.lambda_tensor(0, e_ab)).abs().max().item() < TOL[dtype], call
    g.close()


def test_noalloc_repeated_calls_leave_free_memory_unchanged():
    import torch
    lib, abi, GPEPS = _lib_and_cls()
    D = 32
    g = GPEPS([(5, STAR)], D, dtype="c128")
    g.reset()
    g.step(3, torch.tensor([0.8], dtype=torch.float64, device="cuda"))
    g.synchronize()
    A = g.site_tensor(0, 0)[0].clone()
    B = g.site_tensor(0, 1)[0].clone()
    lam = torch.zeros((5, D), dtype=torch.float64, device="cuda")
    for r, k in enumerate((0, 1, 2, 3)):
        lam[r] = g.lambda_tensor(0, k)
    g.close()
    torch.cuda.synchronize()

    def call():
        return lib.gpeps_bond_update_noalloc(D, abi.GPEPS_C128, ctypes.c_void_p(A.data_ptr()), 3, 0,
                                             ctypes.c_void_p(B.data_ptr()), 2, 0, ctypes.c_void_p(lam.data_ptr()),
                                             None, None, None)

    assert call() == 0                       # the first call on the device looks the scratch up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


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

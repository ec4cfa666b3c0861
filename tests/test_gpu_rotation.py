"""The FP64 Jacobi rotation helpers against CUDA's own FP64 functions (gpeps_selftest_rotation).

Both helpers avoid FP64 divides and square roots: 1/|g| and c = 1/sqrt(1 + t^2)
start from FP32 rsqrtf and take two Newton-Raphson steps of the reciprocal
square root (relative error 1e-7 -> 1e-14 -> rounding), and the tangent t
starts from the FP32 formula and takes one Newton-Raphson step on
t^2 + 2 zeta t - 1 = 0 with an FP32 reciprocal of the derivative (relative
error about (3e-7)^2).  Bounds held here, against the textbook formulas in
CUDA's hypot, sqrt and rsqrt: |e| and c^2 + s^2 equal 1 within 4 ulp, e within
4 ulp of conj(g)/|g|, c within 5e-13 and s within 5e-13 relative of the
reference, and the rotated 2 x 2 matrix has an off-diagonal below 5e-13 of
|g| (the rotation zeroes it up to the angle's error).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _inputs(rng, n, lo, hi, two_sided):
    a = 10.0 ** rng.uniform(lo, hi, n)
    b = 10.0 ** rng.uniform(lo, hi, n)
    # |g| up to sqrt(a b) (a positive semi-definite pair, as in a Gram matrix), random phase
    mag = np.sqrt(a * b) * 10.0 ** rng.uniform(-12 if two_sided else -14, 0, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    x = np.stack([a, b, mag * np.cos(ph), mag * np.sin(ph)], axis=1)
    # special cases: equal diagonals (zeta = 0), real and imaginary g, a >> b and a << b
    x[0] = [1.0, 1.0, 0.3, 0.0]
    x[1] = [0.5, 0.5, 0.0, -0.2]
    x[2] = [1.0, 1e-10, 1e-9, 2e-9]
    x[3] = [1e-10, 1.0, -1e-9, 1e-9]
    if two_sided:   # |g|^2 must stay above FP32's smallest normal: the squared form's range
        x = x[x[:, 2] ** 2 + x[:, 3] ** 2 > 1e-30]
    return x


def _run(which, x):
    import torch
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import _abi
    lib = _abi.load()
    xin = torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
    out = torch.empty((len(x), 8), dtype=torch.float64, device="cuda")
    st = lib.gpeps_selftest_rotation(which, len(x), ctypes.c_void_p(xin.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     None)
    assert st == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("which,lo,hi", [(0, -12, 0), (1, -12, 0), (1, -120, -100), (1, 100, 120)],
                         ids=["two_sided", "one_sided", "one_sided_tiny", "one_sided_huge"])
def test_rotation_helpers_against_cuda_functions(which, lo, hi):
    rng = np.random.default_rng(103 + which)
    x = _inputs(rng, 4096, lo, hi, which == 0)
    o = _run(which, x)
    c, s, e = o[:, 0], o[:, 1], o[:, 2] + 1j * o[:, 3]
    cr, sr, er = o[:, 4], o[:, 5], o[:, 6] + 1j * o[:, 7]
    assert np.abs(np.abs(e) ** 2 - 1).max() <= 4 * EPS
    assert np.abs(c * c + s * s - 1).max() <= 4 * EPS
    assert np.abs(e - er).max() <= 4 * EPS
    assert np.abs(c - cr).max() <= 5e-13
    assert (np.abs(s - sr) <= 5e-13 * np.abs(sr) + 4 * EPS * np.abs(c)).all()
    # the rotation J = [[c, s], [-s e, c e]] (columns p, q) applied to [[a, g], [conj g, b]]
    a, b, g = x[:, 0], x[:, 1], x[:, 2] + 1j * x[:, 3]
    off = c * s * (a - b) + c * c * e * g - s * s * np.conj(e * g)
    assert (np.abs(off) <= 5e-13 * np.abs(g) + 8 * EPS * np.sqrt(a * b)).all()


def test_rotation_selftest_rejects_bad_arguments():
    from paper_2309_15642_gb300 import _build
    _build.build()
    from paper_2309_15642_gb300 import _abi
    lib = _abi.load()
    assert lib.gpeps_selftest_rotation(2, 1, None, None, None) == _abi.GPEPS_EINVAL
    assert lib.gpeps_selftest_rotation(0, -1, None, None, None) == _abi.GPEPS_EINVAL
    assert lib.gpeps_selftest_rotation(1, 4, None, None, None) == _abi.GPEPS_EINVAL
    assert lib.gpeps_selftest_rotation(1, 0, None, None, None) == 0

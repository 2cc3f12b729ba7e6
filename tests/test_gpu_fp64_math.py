"""The library's FP64 reciprocal and reciprocal square root (Newton-Raphson
from the FP32 hardware approximations; used in the FP64 force and backward
passes) against CUDA's correctly rounded division 1.0 / x and its rsqrt, and
against the exact values computed on the host in extended precision.

Bounds, from the iterations' error analysis:
  * reciprocal: the seed's relative error e0 < 2^-21 (FP32 approximation plus
    the rounding of x to FP32) falls to ~e0^2 after one step and to ~e0^4
    (~2^-84) after the residual-form step, so only the final rounding is
    left: at most 1 ulp from the exact value, i.e. equal to 1.0 / x or one
    ulp away;
  * reciprocal square root: two steps take e0 to ~1.5^3 e0^4, below 2^-80,
    leaving the roundings of the last step (y*y, the fused multiply-add, the
    product): at most 2 ulp from the exact value, and at most 3 ulp from
    CUDA's rsqrt (itself within 1 ulp).
The inputs span the squared distances the force passes see (LJ r^2 from ~0.5
to (rc + skin)^2, EAM r^2 up to ~30 A^2) and well beyond, on both sides of
powers of two.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(91)
    x = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 200000))
    r2 = rng.uniform(0.3, 32.0, 200000)  # the range of the force passes
    p2 = 2.0 ** np.arange(-60, 61)
    near = np.concatenate([np.nextafter(p2, 0), p2, np.nextafter(p2, np.inf)])
    return np.concatenate([x, r2, near, [1.0, 3.0, 7.84, 6.25, 2.0 ** (1 / 3)]])


def _ulps(a, ref):
    """|a - ref| in units of the last place of ref (float64)."""
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_rcp_within_one_ulp():
    import torch
    from paper_1009_4330_gb300 import fp64_math
    x = _inputs()
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = fp64_math("rcp", xt).cpu().numpy()
    cuda_div = (1.0 / xt).cpu().numpy()  # IEEE division, correctly rounded
    assert _ulps(y, cuda_div).max() <= 1.0
    # against the exact value (extended precision on the host), where available
    if np.finfo(np.longdouble).nmant >= 63:
        exact = (np.longdouble(1) / x.astype(np.longdouble))
        err = np.abs(y.astype(np.longdouble) - exact) / np.spacing(np.abs(exact.astype(np.float64))).astype(np.longdouble)
        assert float(err.max()) <= 1.0


def test_rsqrt_within_two_ulp():
    import torch
    from paper_1009_4330_gb300 import fp64_math
    x = _inputs()
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = fp64_math("rsqrt", xt).cpu().numpy()
    cuda_rsqrt = torch.rsqrt(xt).cpu().numpy()
    assert _ulps(y, cuda_rsqrt).max() <= 3.0
    if np.finfo(np.longdouble).nmant >= 63:
        exact = np.longdouble(1) / np.sqrt(x.astype(np.longdouble))
        err = np.abs(y.astype(np.longdouble) - exact) / np.spacing(np.abs(exact.astype(np.float64))).astype(np.longdouble)
        assert float(err.max()) <= 2.0


def test_bad_op_rejected():
    import torch
    from paper_1009_4330_gb300 import MDError, _lib
    import ctypes
    lib = _lib.load()
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    st = lib.md_probe_fp64_math(2, 4, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert st == _lib.MD_ERR_INVALID
    assert MDError  # the binding's error type exists for the Python wrapper

"""The FP64 cut-off band of the mixed LJ pass is wide enough.

The mixed force pass computes a pair's squared distance in FP32 from
cell-relative records (each position relative to the centre of its bin, as
FP32), the FP32 bin edge times the pair's stencil offset, one fused
multiply-add per component and a fused sum of squares; pairs whose FP32 r^2
lies within a band of rc^2 get the FP64 decision instead.  The band is four
times the bound u rc (2 sqrt(3) (3 h + 2 skin + rc) + 4 rc), u = 2^-24, h the
bin edge.  Here those FP32 operations are emulated with NumPy (a fused
multiply-add is the exact FP64 value rounded once to FP32) for random pairs
at rc in several geometries, and the FP32 error of r^2 (plus rc^2's own
rounding) must stay below the bound, so that no pair outside the band can be
decided differently from FP64."""
import numpy as np
import pytest

U = 2.0 ** -24


def bound(rc, skin, h):
    return U * rc * (2.0 * np.sqrt(3.0) * (3.0 * h + 2.0 * skin + rc) + 4.0 * rc)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma32(a, b, c):
    return f32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def fp32_r2(xi, xj, code, h):
    """FP32 r^2 of the kernel's operations: records rounded to FP32, then per
    component fma(-code, h32, xi32 - xj32), then fma(dz, dz, fma(dy, dy, dx*dx))."""
    ri, rj, h32 = f32(xi), f32(xj), f32(h)
    d = fma32(-code.astype(np.float32), h32, f32(ri - rj))
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    return fma32(dz, dz, fma32(dy, dy, f32(dx * dx)))


@pytest.mark.parametrize("rc,skin,h", [(2.5, 0.3, 2.8794), (2.5, 0.3, 5.7), (1.7, 1.2, 3.36), (5.0, 0.3, 5.3),
                                       (4.95, 0.5, 5.5), (1.2, 0.1, 1.3)])
def test_fp32_r2_error_stays_inside_the_band(rc, skin, h):
    rng = np.random.default_rng(12345)
    m = 200000
    lim = 0.5 * h + 0.5 * skin  # |xr| after up to skin/2 of drift since the build
    xi = rng.uniform(-lim, lim, size=(m, 3))
    # a partner at distance rc (1 + tiny) in a random direction, expressed in
    # its own bin's frame: x_j = x_i - d - code h, code the stencil offset
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    d = u * (rc * (1.0 + rng.uniform(-1e-6, 1e-6, size=(m, 1))))
    xj_abs = xi - d
    code = np.round(xj_abs / h)
    xj = xj_abs - code * h  # partner's cell-relative position
    keep = np.all(np.abs(xj) <= lim, axis=1)
    xi, xj, code, d = xi[keep], xj[keep], code[keep], d[keep]
    assert xi.shape[0] > m // 4
    r2_64 = np.sum((xi - xj - code * h) ** 2, axis=1)  # the FP64 value the decision is defined on
    r2_32 = fp32_r2(xi, xj, code, h).astype(np.float64)
    err = np.abs(r2_32 - r2_64) + abs(float(f32(rc * rc)) - rc * rc)
    b = bound(rc, skin, h)
    assert err.max() < b, f"max FP32 error {err.max():.3e} vs bound {b:.3e}"
    # the band (4x the bound) is also far below the spacing of real pairs
    assert 4.0 * b < 1e-4 * rc * rc

"""Pins of the oracle renderer (paper Section 3.6): exact reproduction of a
view at an integer camera position, constants, exact reproduction of a light
field affine in (u, v, s, t), and bilinear resampling checked against
scipy.ndimage.map_coordinates."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def test_integer_camera_reproduces_the_view():
    rng = np.random.default_rng(0)
    U, V, W, H = 4, 3, 10, 7
    lf = rng.integers(0, 256, size=(U * V, H, W, 3), dtype=np.uint8)
    for j in range(V):
        for i in range(U):
            for d in (0.0, 1.7):
                out = oracle.render_view(lf, U, V, float(i), float(j), d, W, H)
                assert np.array_equal(out, lf[j * U + i] / 255.0)


def test_constant_field_renders_constant():
    lf = np.full((9, 6, 5, 3), 77, dtype=np.uint8)
    out = oracle.render_view(lf, 3, 3, 1.3, 0.4, -2.5, 11, 9)
    assert np.allclose(out, 77 / 255.0, atol=1e-12)


@pytest.mark.parametrize("u,v,d", [(0.3, 1.6, 0.0), (2.25, 0.75, 1.5), (1.9, 2.0, -0.8), (3.0, 0.1, 2.0)])
def test_affine_light_field_is_reproduced(u, v, d):
    U, V, W, H = 4, 3, 40, 30
    a0, a1, a2, a3, a4 = 20, 7, 11, 2, 3   # f = a0 + a1 i + a2 j + a3 x + a4 y
    j, i, y, x = np.meshgrid(np.arange(V), np.arange(U), np.arange(H), np.arange(W), indexing="ij")
    f = a0 + a1 * i + a2 * j + a3 * x + a4 * y
    assert f.max() <= 255
    lf = np.repeat(f.reshape(U * V, H, W, 1), 3, axis=-1).astype(np.uint8)
    out = oracle.render_view(lf, U, V, u, v, d, W, H)
    checked = 0
    for yy in range(H):
        for xx in range(W):
            s, t = float(xx), float(yy)
            lo = min(s + d * (k - u) for k in (np.floor(u), np.floor(u) + 1))
            hi = max(s + d * (k - u) for k in (np.floor(u), np.floor(u) + 1))
            lo_t = min(t + d * (k - v) for k in (np.floor(v), np.floor(v) + 1))
            hi_t = max(t + d * (k - v) for k in (np.floor(v), np.floor(v) + 1))
            if lo < 0 or hi > W - 1 or lo_t < 0 or hi_t > H - 1:
                continue   # clamped at the image edge
            expect = (a0 + a1 * u + a2 * v + a3 * s + a4 * t) / 255.0
            assert abs(out[yy, xx, 0] - expect) < 1e-12
            checked += 1
    assert checked > W * H // 3


@pytest.mark.parametrize("out_w,out_h", [(17, 13), (5, 4), (32, 9)])
def test_resampling_matches_scipy_bilinear(out_w, out_h):
    rng = np.random.default_rng(1)
    U, V, W, H = 3, 3, 12, 10
    lf = rng.integers(0, 256, size=(U * V, H, W, 3), dtype=np.uint8)
    out = oracle.render_view(lf, U, V, 2.0, 1.0, 0.9, out_w, out_h)
    s = (np.arange(out_w) + 0.5) * W / out_w - 0.5
    t = (np.arange(out_h) + 0.5) * H / out_h - 0.5
    tt, ss = np.meshgrid(t, s, indexing="ij")
    img = lf[1 * U + 2].astype(np.float64)
    for ch in range(3):
        ref = ndimage.map_coordinates(img[..., ch], [tt, ss], order=1, mode="nearest")
        assert np.allclose(out[..., ch], ref / 255.0, atol=1e-12)

"""Seeded synthetic two-plane light fields.

Input generation only: this module holds none of the compression method's
arithmetic.  Both the CPU oracle and the CUDA library are fed from here.

A scene is a stack of fronto-parallel textured planes.  Plane k has disparity
d_k pixels per unit of camera motion; a scene point X of plane k appears in
view (i, j) at x = X + d_k (i - c_u), y = Y + d_k (j - c_v), with (c_u, c_v)
the grid centre, so a renderer focused at disparity d_k (sampling view i at
s + d (i - u)) brings that plane into focus.  Textures are multi-octave value
noise (a random lattice per octave, bilinear, amplitude halved per octave);
every plane but the farthest carries a value-noise opacity mask (> 0.5 is
opaque) and nearer planes (larger disparity) cover farther ones.  Gaussian
noise of standard deviation sigma is added per pixel and channel, then values
are rounded and clipped to uint8.

The presets follow the light fields of the paper's evaluation (grids of 5x5
to 17x17 views of 64^2 to 1024^2 pixels) and are seeded with
1805_06019 + preset id.  The real captures (Stanford archive) are not used.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

SEED_BASE = 1805_06019

PRESETS = {
    # 5x5 views of 64x64, 3 planes, sigma 1; 2-level tree, tau 2.
    "tiny": dict(id=0, U=5, V=5, W=64, H=64, disparities=[0.0, 0.5, 1.5], sigma=1.0,
                 L=2, c=[0, 5], B=4, taus=[2], n_render=16, render_size=(64, 64)),
    # 9x9 views of 512x512, 5 planes at -2..2, sigma 1; 3-level (3, 3), taus 1/4/8.
    "plain": dict(id=1, U=9, V=9, W=512, H=512, disparities=[-2.0, -1.0, 0.0, 1.0, 2.0],
                  sigma=1.0, L=3, c=[0, 3, 3], B=4, taus=[1, 4, 8], n_render=1000,
                  render_size=(512, 512)),
    # 17x17 views of 1024x1024, 8 planes at -3..3, contrast modulated; 3-level (5, 4).
    "batching": dict(id=2, U=17, V=17, W=1024, H=1024,
                     disparities=list(np.linspace(-3.0, 3.0, 8)), sigma=1.0,
                     L=3, c=[0, 5, 4], B=4, taus=[4], n_requests=1_000_000,
                     contrast=True),
    # 15x15 views of 625x434, lenslet-like disparities within +-1, sigma 2; 3-level (3, 5);
    # threshold 3 leaves about 1.5 M level-0 blocks for the learned aid's training data.
    "learned": dict(id=3, U=15, V=15, W=625, H=434, disparities=[-1.0, -0.4, 0.3, 1.0],
                    sigma=2.0, L=3, c=[0, 3, 5], B=4, taus=[3]),
    # serving light fields: 5x5x256^2, 9x9x512^2, 17x17x1024^2, 3-level each.
    "serving_small": dict(id=4, U=5, V=5, W=256, H=256, disparities=[-1.0, 0.0, 1.0],
                          sigma=1.0, L=3, c=[0, 2, 3], B=4, taus=[4]),
    "serving_medium": dict(id=5, U=9, V=9, W=512, H=512, disparities=[-2.0, -1.0, 0.0, 1.0, 2.0],
                           sigma=1.0, L=3, c=[0, 3, 3], B=4, taus=[4]),
    "serving_large": dict(id=6, U=17, V=17, W=1024, H=1024,
                          disparities=list(np.linspace(-3.0, 3.0, 8)), sigma=1.0,
                          L=3, c=[0, 5, 4], B=4, taus=[4], contrast=True),
}


def rng_for(preset_id: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + preset_id, stream]))


def _shift_bilinear(img: np.ndarray, sx: float, sy: float) -> np.ndarray:
    """out[y, x] = img sampled at (x - sx, y - sy), bilinear, wrapping."""
    kx = int(np.floor(-sx))
    fx = np.float32(-sx - kx)
    ky = int(np.floor(-sy))
    fy = np.float32(-sy - ky)
    a = np.roll(img, -kx, axis=1)
    if fx != 0:
        a = (1 - fx) * a + fx * np.roll(a, -1, axis=1)
    b = np.roll(a, -ky, axis=0)
    if fy != 0:
        b = (1 - fy) * b + fy * np.roll(b, -1, axis=0)
    return b


def value_noise(rng: np.random.Generator, H: int, W: int, cell: float,
                octaves: int = 4, channels: int = 1) -> np.ndarray:
    """[H, W, channels] float32 in [0, 1]: bilinear random lattices, octave o
    at cell size cell / 2^o with amplitude 2^-o."""
    out = np.zeros((H, W, channels), dtype=np.float32)
    total = 0.0
    for o in range(octaves):
        cs = max(cell / (2 ** o), 1.0)
        gh, gw = int(np.ceil(H / cs)) + 1, int(np.ceil(W / cs)) + 1
        lat = rng.random((gh, gw, channels), dtype=np.float32)
        ys = np.arange(H, dtype=np.float32) / cs
        xs = np.arange(W, dtype=np.float32) / cs
        y0 = np.floor(ys).astype(np.int64)
        x0 = np.floor(xs).astype(np.int64)
        fy = (ys - y0)[:, None, None]
        fx = (xs - x0)[None, :, None]
        y1 = np.minimum(y0 + 1, gh - 1)
        x1 = np.minimum(x0 + 1, gw - 1)
        top = lat[y0][:, x0] * (1 - fx) + lat[y0][:, x1] * fx
        bot = lat[y1][:, x0] * (1 - fx) + lat[y1][:, x1] * fx
        amp = 0.5 ** o
        out += amp * (top * (1 - fy) + bot * fy)
        total += amp
    return out / np.float32(total)


def _planes(U: int, V: int, W: int, H: int, disparities, preset_id: int, contrast: bool):
    """The scene's planes, farthest first: (disparity, texture [H, W, 3]
    float32 in [0, 255], opacity mask [H, W, 1] or None for the farthest)."""
    rng = rng_for(preset_id, 0)
    order = np.argsort(np.asarray(disparities, dtype=np.float64), kind="stable")
    planes = []
    for rank, k in enumerate(order):
        cell = float(rng.uniform(12.0, 40.0)) * max(W, H) / 512.0
        lum = value_noise(rng, H, W, cell, 4, 1)
        chroma = value_noise(rng, H, W, cell * 1.5, 3, 3)
        tex = 0.75 * lum + 0.25 * chroma
        if contrast:
            # regional contrast: some areas nearly flat, some at full contrast,
            # so that residual blocks range from very sparse to dense
            m = value_noise(rng, H, W, max(W, H) / 6.0, 2, 1)
            m = np.clip((m - 0.3) * 2.5, 0.0, 1.0) ** 2 * 0.95 + 0.05
            tex = 0.5 + (tex - 0.5) * m * 1.6
        tex = np.clip(tex, 0.0, 1.0) * np.float32(255.0)
        mask = None
        if rank > 0:
            mask = value_noise(rng, H, W, cell * 2.0, 3, 1)
        planes.append((float(disparities[k]), tex.astype(np.float32), mask))
    return planes


def make_lightfield(U: int, V: int, W: int, H: int, disparities, sigma: float,
                    preset_id: int, contrast: bool = False) -> np.ndarray:
    """Views [V*U, H, W, 3] uint8, view index j*U + i (i along u / x)."""
    cu, cv = (U - 1) / 2.0, (V - 1) / 2.0
    planes = _planes(U, V, W, H, disparities, preset_id, contrast)
    noise_rng = rng_for(preset_id, 1)
    out = np.empty((V * U, H, W, 3), dtype=np.uint8)
    for j in range(V):
        for i in range(U):
            acc = None
            for d, tex, mask in planes:
                sx, sy = d * (i - cu), d * (j - cv)
                layer = _shift_bilinear(tex, sx, sy)
                if acc is None:
                    acc = layer
                else:
                    opaque = _shift_bilinear(mask, sx, sy) > 0.5
                    acc = np.where(opaque, layer, acc)
            if sigma > 0:
                acc = acc + noise_rng.normal(0.0, sigma, size=acc.shape).astype(np.float32)
            out[j * U + i] = np.clip(np.rint(acc), 0, 255).astype(np.uint8)
    return out


def _shift_bilinear_torch(img, sx: float, sy: float):
    """_shift_bilinear on a torch tensor: the same float32 operations in the
    same order, so the result is the same bits."""
    import torch
    kx = int(np.floor(-sx))
    fx = np.float32(-sx - kx)
    ky = int(np.floor(-sy))
    fy = np.float32(-sy - ky)
    a = torch.roll(img, -kx, dims=1)
    if fx != 0:
        a = float(np.float32(1) - fx) * a + float(fx) * torch.roll(a, -1, dims=1)
    b = torch.roll(a, -ky, dims=0)
    if fy != 0:
        b = float(np.float32(1) - fy) * b + float(fy) * torch.roll(b, -1, dims=0)
    return b


def make_lightfield_torch(U: int, V: int, W: int, H: int, disparities, sigma: float,
                          preset_id: int, contrast: bool = False, device="cuda"):
    """make_lightfield with the per-view compositing done by torch on
    `device` (the textures, masks and noise still come from the same numpy
    generators): the same views, bit for bit, as a [V*U, H, W, 3] uint8
    tensor on the device, in a fraction of the time for large presets."""
    import torch
    cu, cv = (U - 1) / 2.0, (V - 1) / 2.0
    planes = [(d, torch.from_numpy(tex).to(device), None if mask is None else torch.from_numpy(mask).to(device))
              for d, tex, mask in _planes(U, V, W, H, disparities, preset_id, contrast)]
    noise_rng = rng_for(preset_id, 1)
    out = torch.empty((V * U, H, W, 3), dtype=torch.uint8, device=device)
    for j in range(V):
        for i in range(U):
            acc = None
            for d, tex, mask in planes:
                sx, sy = d * (i - cu), d * (j - cv)
                layer = _shift_bilinear_torch(tex, sx, sy)
                if acc is None:
                    acc = layer
                else:
                    opaque = _shift_bilinear_torch(mask, sx, sy) > 0.5
                    acc = torch.where(opaque, layer, acc)
            if sigma > 0:
                noise = noise_rng.normal(0.0, sigma, size=tuple(acc.shape)).astype(np.float32)
                acc = acc + torch.from_numpy(noise).to(device)
            out[j * U + i] = torch.clamp(torch.round(acc), 0, 255).to(torch.uint8)
    return out


def preset_lightfield_torch(name: str, device="cuda"):
    """preset_lightfield's views as a uint8 tensor on `device`
    (make_lightfield_torch: the same bits)."""
    p = PRESETS[name]
    return make_lightfield_torch(p["U"], p["V"], p["W"], p["H"], p["disparities"], p["sigma"],
                                 p["id"], p.get("contrast", False), device)


def preset_lightfield(name: str) -> np.ndarray:
    """The preset's views.  When RLFC_SYNTH_CACHE names a directory, the
    views are kept there as .npy, keyed by preset and by this module's source,
    so that several processes of one session synthesise a large preset once."""
    p = PRESETS[name]
    cache = os.environ.get("RLFC_SYNTH_CACHE")
    path = None
    if cache:
        with open(__file__, "rb") as f:
            key = hashlib.sha1(f.read()).hexdigest()[:12]
        path = os.path.join(cache, f"{name}_{key}.npy")
        if os.path.exists(path):
            return np.load(path)
    lf = make_lightfield(p["U"], p["V"], p["W"], p["H"], p["disparities"], p["sigma"],
                         p["id"], p.get("contrast", False))
    if path:
        os.makedirs(cache, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp.npy"
        np.save(tmp, lf)
        os.replace(tmp, path)
    return lf


def random_views(n: int, U: int, V: int, preset_id: int, d_choices=(0.0,)) -> np.ndarray:
    """[n, 3] float32 rows (u, v, d): camera positions uniform on the grid and a
    focus disparity drawn from d_choices."""
    rng = rng_for(preset_id, 2)
    uv = rng.random((n, 2)) * np.array([U - 1, V - 1], dtype=np.float64)
    d = rng.choice(np.asarray(d_choices, dtype=np.float64), size=n)
    return np.concatenate([uv, d[:, None]], axis=1).astype(np.float32)


def random_requests(n: int, n_views: int, n_loc: int, preset_id: int):
    """n uniform random (view, location) block requests as two uint32 arrays."""
    rng = rng_for(preset_id, 3)
    views = rng.integers(0, n_views, size=n, dtype=np.uint32)
    locs = rng.integers(0, n_loc, size=n, dtype=np.uint32)
    return views, locs


def poisson_arrivals(rate: float, n: int, preset_id: int, stream: int = 4) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson process of `rate`
    requests per second: cumulative sums of exponential gaps."""
    rng = rng_for(preset_id, stream)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


SERVING_FLEET = [
    # (preset, residual threshold): three 5x5x256^2, three 9x9x512^2 and two
    # 17x17x1024^2 light fields, each size class encoded at different
    # thresholds so that every resident stream differs
    ("serving_small", 2), ("serving_small", 4), ("serving_small", 8),
    ("serving_medium", 2), ("serving_medium", 4), ("serving_medium", 8),
    ("serving_large", 4), ("serving_large", 8),
]


def serving_requests(n: int, n_lf: int, preset_id: int, stream: int = 5):
    """n requests as (light-field index, u01, v01, plane choice u01): uniform
    over the resident light fields, camera position and focus plane drawn as
    fractions that the caller maps to each light field's grid and planes."""
    rng = rng_for(preset_id, stream)
    return (rng.integers(0, n_lf, size=n), rng.random(n), rng.random(n), rng.random(n))

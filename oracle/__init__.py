"""RLFC CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement in C of the RLFC method (Pratapa & Manocha, I3D
2019), wrapped with ctypes.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product library never does, and
the two share no code.  Each wrapped function names the passage of the paper
that its C implementation follows (see the C sources for the readings taken
where the paper is silent).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRCS = ["colour.c", "bise.c", "tree.c", "encode.c", "decode.c", "render.c", "ks.c", "mlp.c"]
_MAXL = 8
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= lib_m for d in deps):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Tree(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int),
        ("Gu", ctypes.c_int * _MAXL),
        ("Gv", ctypes.c_int * _MAXL),
        ("parent", ctypes.POINTER(ctypes.c_int) * _MAXL),
        ("n_top", ctypes.c_int),
        ("S", ctypes.c_int),
        ("bfs_level", ctypes.POINTER(ctypes.c_int)),
        ("bfs_node", ctypes.POINTER(ctypes.c_int)),
        ("pos_of", ctypes.POINTER(ctypes.c_int) * _MAXL),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("U", ctypes.c_int), ("V", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int),
        ("B", ctypes.c_int), ("L", ctypes.c_int), ("c", ctypes.c_int * _MAXL),
        ("tau_p", ctypes.c_int), ("tau_b", ctypes.c_int), ("q", ctypes.c_int),
        ("mode_space", ctypes.c_int), ("tau_err", ctypes.c_int), ("lam_q8", ctypes.c_int),
        ("leaf_modes", ctypes.c_void_p), ("leaf_resid", ctypes.c_void_p), ("leaf_label", ctypes.c_void_p),
    ]


class _Stream(ctypes.Structure):
    _fields_ = [
        ("bytes", ctypes.c_void_p), ("nbytes", ctypes.c_size_t),
        ("U", ctypes.c_int), ("V", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int),
        ("B", ctypes.c_int), ("L", ctypes.c_int), ("q", ctypes.c_int),
        ("n_top", ctypes.c_int), ("S", ctypes.c_int),
        ("Wp", ctypes.c_int), ("Hp", ctypes.c_int), ("nlx", ctypes.c_int),
        ("nly", ctypes.c_int), ("nloc", ctypes.c_int),
        ("off_top", ctypes.c_long), ("off_offsets", ctypes.c_long),
        ("off_records", ctypes.c_long), ("record_words", ctypes.c_long),
        ("tree", _Tree),
    ]


def _P(t):
    return ctypes.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            i, l, v, sz = ctypes.c_int, ctypes.c_long, ctypes.c_void_p, ctypes.c_size_t
            L.or_mode_N.argtypes = [i]
            L.or_mode_kind.argtypes = [i]
            L.or_mode_b.argtypes = [i]
            L.or_bise_bits.argtypes = [i, i]
            L.or_bise_bits.restype = l
            L.or_choose_mode_search.argtypes = [i, i]
            L.or_put_bits.argtypes = [v, l, i, ctypes.c_uint32]
            L.or_get_bits.argtypes = [v, l, i]
            L.or_get_bits.restype = ctypes.c_uint32
            L.or_bise_pack.argtypes = [v, l, i, i, v]
            L.or_bise_unpack.argtypes = [v, l, i, i, v]
            L.or_bise_exhaustive.argtypes = [i, i, l]
            L.or_bise_exhaustive.restype = l
            L.or_ycocg_fwd_array.argtypes = [v, l, v]
            L.or_ycocg_inv_array.argtypes = [v, l, v]
            L.or_tile_count.argtypes = [i, i]
            L.or_tile_lo.argtypes = [i, i, i]
            L.or_tree_from_clusters.argtypes = [_P(_Tree), i, i, i, v]
            L.or_tree_free.argtypes = [_P(_Tree)]
            L.or_filter_level.argtypes = [v, i, i, i, i, v]
            L.or_encode.argtypes = [v, _P(_Params), _P(ctypes.POINTER(ctypes.c_uint8)), _P(sz)]
            L.or_free.argtypes = [v]
            L.or_stream_open.argtypes = [_P(_Stream), v, sz]
            L.or_stream_close.argtypes = [_P(_Stream)]
            L.or_decode_block.argtypes = [_P(_Stream), i, i, v]
            L.or_decode_block_ycc.argtypes = [_P(_Stream), i, i, i, v]
            L.or_decode_all.argtypes = [_P(_Stream), v, i]
            d = ctypes.c_double
            L.or_render_pixel.argtypes = [v, i, i, i, i, d, d, d, i, i, i, i, v]
            L.or_render_view.argtypes = [v, i, i, i, i, d, d, d, i, i, v]
            L.or_ks_quantise.argtypes = [v, i, i, i, v]
            L.or_ks_cost.argtypes = [v, i, i, i, i, i, i, _P(ctypes.c_longlong)]
            L.or_ks_search.argtypes = [v, i, i, i, i, _P(i), _P(i)]
            L.or_ks_features.argtypes = [v, v]
            L.or_mlp_nparams.argtypes = []
            L.or_mlp_forward.argtypes = [v, v, i, v]
            L.or_mlp_loss_grad.argtypes = [v, v, v, i, v, _P(d)]
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- Section 4: YCoCg-R -------------------------------------------------------

def ycocg_fwd(rgb: np.ndarray) -> np.ndarray:
    """Forward YCoCg-R of uint8 RGB triples (last axis 3) -> int32 (Y, Co, Cg)."""
    a = np.ascontiguousarray(rgb, dtype=np.uint8)
    out = np.empty(a.shape, dtype=np.int32)
    lib().or_ycocg_fwd_array(_ptr(a), a.size // 3, _ptr(out))
    return out


def ycocg_inv(ycc: np.ndarray) -> np.ndarray:
    """Inverse YCoCg-R of int (Y, Co, Cg) triples -> int32 RGB, not clamped."""
    a = np.ascontiguousarray(ycc, dtype=np.int32)
    out = np.empty(a.shape, dtype=np.int32)
    lib().or_ycocg_inv_array(_ptr(a), a.size // 3, _ptr(out))
    return out


# ---- Section 3.3: BISE --------------------------------------------------------

NMODES = 28


def mode_table():
    """[(N, kind, b)] for the 28 modes, kind 0 bits / 1 trits / 2 quints."""
    L = lib()
    return [(L.or_mode_N(k), L.or_mode_kind(k), L.or_mode_b(k)) for k in range(NMODES)]


def bise_bits(n: int, k: int) -> int:
    return int(lib().or_bise_bits(n, k))


def choose_mode(n: int, span: int) -> int:
    """Exhaustive search: cheapest mode with N >= span + 1 (ties: smaller k)."""
    return int(lib().or_choose_mode_search(n, span))


def bise_pack(u, k: int, pos: int = 0) -> bytes:
    """Pack the values u (each < N_k) from bit `pos` of a zeroed buffer."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    nbits = pos + bise_bits(len(u), k)
    buf = np.zeros((nbits + 7) // 8 + 8, dtype=np.uint8)
    lib().or_bise_pack(_ptr(buf), pos, len(u), k, _ptr(u))
    return bytes(buf[: (nbits + 7) // 8])


def bise_unpack(buf: bytes, n: int, k: int, pos: int = 0) -> np.ndarray:
    b = np.frombuffer(bytes(buf) + b"\0" * 8, dtype=np.uint8).copy()
    u = np.zeros(n, dtype=np.int32)
    lib().or_bise_unpack(_ptr(b), pos, n, k, _ptr(u))
    return u


def bise_exhaustive(n: int, k: int, max_count: int) -> int:
    """Failures of an exhaustive pack/unpack round trip over [0, N_k)^n
    (-1 if there are more than max_count sequences)."""
    return int(lib().or_bise_exhaustive(n, k, max_count))


def get_bits(buf: bytes, pos: int, width: int) -> int:
    b = np.frombuffer(bytes(buf) + b"\0" * 8, dtype=np.uint8).copy()
    return int(lib().or_get_bits(_ptr(b), pos, width))


# ---- Eq. 1 / Section 3.4: tree and BFS ---------------------------------------

def tree_from_clusters(U: int, V: int, L: int, c) -> dict:
    """Cluster tiling per level (Eq. 1 reading) and the BFS numbering."""
    t = _Tree()
    carr = (ctypes.c_int * _MAXL)(*([0] + list(c[1:L]) + [0] * (_MAXL - L)))
    rc = lib().or_tree_from_clusters(ctypes.byref(t), U, V, L, carr)
    try:
        if rc != 0:
            raise ValueError("invalid tree parameters")
        out = {"L": L, "Gu": [t.Gu[l] for l in range(L)], "Gv": [t.Gv[l] for l in range(L)],
               "n_top": t.n_top, "S": t.S}
        out["parent"] = [[t.parent[l][i] for i in range(t.Gu[l] * t.Gv[l])] for l in range(L - 1)]
        out["bfs_level"] = [t.bfs_level[p] for p in range(t.S)]
        out["bfs_node"] = [t.bfs_node[p] for p in range(t.S)]
        out["pos_of"] = [[t.pos_of[l][i] for i in range(t.Gu[l] * t.Gv[l])] for l in range(L - 1)]
        return out
    finally:
        lib().or_tree_free(ctypes.byref(t))


def tile_count(G: int, c: int) -> int:
    return int(lib().or_tile_count(G, c))


def filter_level(child: np.ndarray, Gu: int, Gv: int, c: int) -> np.ndarray:
    """Eq. 2 for one level: child is [Gu*Gv, npix] int32 -> [ku*kv, npix]."""
    a = np.ascontiguousarray(child, dtype=np.int32)
    ku, kv = tile_count(Gu, c), tile_count(Gv, c)
    out = np.empty((ku * kv, a.shape[1]), dtype=np.int32)
    rc = lib().or_filter_level(_ptr(a), Gu, Gv, c, a.shape[1], _ptr(out))
    if rc != 0:
        raise ValueError("filter failed")
    return out


# ---- Algorithm 1: encoder ----------------------------------------------------

def encode(lf: np.ndarray, U: int, V: int, B: int = 4, L: int = 2, c=(0, 5),
           tau_p: int = 0, tau_b: int = 0, q: int = 0, mode_space: int = 0, tau_err: int = 0,
           lam_q8: int = 0, leaf_modes: np.ndarray | None = None, leaf_out: dict | None = None) -> bytes:
    """Compress views lf[V*U, H, W, 3] (uint8) into an RLFC stream (format v1).

    c[l] is the cluster side used to build level l from level l-1 (c[0] unused).
    mode_space 1 picks each block's (mode, shift) with ks_search (tau_err,
    lam_q8), or takes the level-0 ones from leaf_modes [U*V, 3, nloc] uint8
    (k | s << 5, 0xFF = search).  leaf_out, when given, receives "resid"
    [U*V, 3, nloc, B*B] int16 and "label" [U*V, 3, nloc] uint8 of the level-0
    blocks.
    """
    a = np.ascontiguousarray(lf, dtype=np.uint8)
    H, W = a.shape[-3], a.shape[-2]
    assert a.size == U * V * H * W * 3
    p = _Params()
    p.U, p.V, p.W, p.H, p.B, p.L = U, V, W, H, B, L
    for l in range(1, L):
        p.c[l] = int(c[l])
    p.tau_p, p.tau_b, p.q = int(tau_p), int(tau_b), int(q)
    p.mode_space, p.tau_err, p.lam_q8 = int(mode_space), int(tau_err), int(lam_q8)
    nloc = ((W + B - 1) // B) * ((H + B - 1) // B)
    keep = []
    if leaf_modes is not None:
        lm = np.ascontiguousarray(leaf_modes, dtype=np.uint8)
        assert lm.size == U * V * 3 * nloc
        keep.append(lm)
        p.leaf_modes = lm.ctypes.data
    if leaf_out is not None:
        leaf_out["resid"] = np.zeros((U * V, 3, nloc, B * B), dtype=np.int16)
        leaf_out["label"] = np.zeros((U * V, 3, nloc), dtype=np.uint8)
        p.leaf_resid = leaf_out["resid"].ctypes.data
        p.leaf_label = leaf_out["label"].ctypes.data
    out = ctypes.POINTER(ctypes.c_uint8)()
    n = ctypes.c_size_t()
    rc = lib().or_encode(_ptr(a), ctypes.byref(p), ctypes.byref(out), ctypes.byref(n))
    if rc != 0:
        raise ValueError("oracle encoder rejected the parameters or the data")
    try:
        return ctypes.string_at(out, n.value)
    finally:
        lib().or_free(out)


# ---- Algorithm 2: decoder ----------------------------------------------------

class Stream:
    """An opened RLFC stream (Algorithm 2 initialisation)."""

    def __init__(self, data: bytes):
        self._buf = np.frombuffer(bytes(data), dtype=np.uint8).copy()
        self._s = _Stream()
        rc = lib().or_stream_open(ctypes.byref(self._s), _ptr(self._buf), self._buf.size)
        if rc != 0:
            lib().or_stream_close(ctypes.byref(self._s))
            raise ValueError("corrupt or unsupported RLFC stream")
        s = self._s
        self.U, self.V, self.W, self.H, self.B = s.U, s.V, s.W, s.H, s.B
        self.L, self.q, self.n_top, self.S = s.L, s.q, s.n_top, s.S
        self.Wp, self.Hp, self.nlx, self.nly, self.nloc = s.Wp, s.Hp, s.nlx, s.nly, s.nloc
        self.nbytes = self._buf.size
        self.top_bytes = s.off_offsets - s.off_top

    def __del__(self):
        try:
            lib().or_stream_close(ctypes.byref(self._s))
        except Exception:
            pass

    def decode_block(self, view: int, loc: int) -> np.ndarray:
        """DecompressLFIBlock(view, loc) -> [B, B, 3] uint8 RGB."""
        out = np.zeros((self.B, self.B, 3), dtype=np.uint8)
        if lib().or_decode_block(ctypes.byref(self._s), view, loc, _ptr(out)) != 0:
            raise ValueError(f"cannot decode view {view} block {loc}")
        return out

    def decode_block_ycc(self, view: int, loc: int, stop_level: int = 0) -> np.ndarray:
        """[3, B, B] int32 YCoCg-R before the colour inverse; stop_level > 0 is
        the progressive (filtered) value of that level."""
        out = np.zeros((3, self.B, self.B), dtype=np.int32)
        if lib().or_decode_block_ycc(ctypes.byref(self._s), view, loc, stop_level, _ptr(out)) != 0:
            raise ValueError(f"cannot decode view {view} block {loc}")
        return out

    def decode_all(self, nthreads: int = 1) -> np.ndarray:
        """Every view, cropped: [V*U, H, W, 3] uint8."""
        out = np.zeros((self.U * self.V, self.H, self.W, 3), dtype=np.uint8)
        if lib().or_decode_all(ctypes.byref(self._s), _ptr(out), nthreads) != 0:
            raise ValueError("corrupt record")
        return out


# ---- Section 3.6: renderer ---------------------------------------------------

def render_pixel(lf: np.ndarray, U: int, V: int, u: float, v: float, d: float,
                 out_w: int, out_h: int, x: int, y: int) -> np.ndarray:
    a = np.ascontiguousarray(lf, dtype=np.uint8)
    H, W = a.shape[-3], a.shape[-2]
    out = np.zeros(3, dtype=np.float64)
    lib().or_render_pixel(_ptr(a), U, V, W, H, float(u), float(v), float(d),
                          out_w, out_h, x, y, _ptr(out))
    return out


def render_view(lf: np.ndarray, U: int, V: int, u: float, v: float, d: float,
                out_w: int, out_h: int) -> np.ndarray:
    """[out_h, out_w, 3] float64 in [0, 1]."""
    a = np.ascontiguousarray(lf, dtype=np.uint8)
    H, W = a.shape[-3], a.shape[-2]
    out = np.zeros((out_h, out_w, 3), dtype=np.float64)
    lib().or_render_view(_ptr(a), U, V, W, H, float(u), float(v), float(d),
                         out_w, out_h, _ptr(out))
    return out


def to_u8(x: np.ndarray) -> np.ndarray:
    """Rendered [0, 1] values to 8 bits: floor(clamp(v, 0, 1) * 255 + 0.5)."""
    return np.floor(np.clip(x, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)


# ---- Section 4: metrics ------------------------------------------------------

def mse_ycocg(orig: np.ndarray, dec: np.ndarray) -> np.ndarray:
    """Per-image, per-channel MSE in YCoCg-R: [nviews, 3] float64."""
    a = ycocg_fwd(orig).reshape(orig.shape[0], -1, 3).astype(np.float64)
    b = ycocg_fwd(dec).reshape(dec.shape[0], -1, 3).astype(np.float64)
    return ((a - b) ** 2).mean(axis=1)


def psnr_ycocg(orig: np.ndarray, dec: np.ndarray, cap: float = 99.0) -> float:
    """Eq. 4-5: (6 PSNR_Y + PSNR_Co + PSNR_Cg) / 8 with peak 255, averaged
    over the images; a lossless channel is capped at `cap` dB."""
    mse = mse_ycocg(orig, dec)
    with np.errstate(divide="ignore"):
        p = np.where(mse > 0, 10.0 * np.log10(255.0 ** 2 / np.maximum(mse, 1e-300)), cap)
    p = np.minimum(p, cap)
    per_img = (6.0 * p[:, 0] + p[:, 1] + p[:, 2]) / 8.0
    return float(per_img.mean())


def bpp(stream: bytes, n_pixels: int) -> float:
    """Bits per (24-bit RGB) pixel of the whole stream."""
    return 8.0 * len(stream) / n_pixels


# ---- the learned encoder aid: (mode, shift) search, statistics, network ------

NCLASSES = 4 * NMODES   # class s * 28 + k


def ks_search(r, q: int = 0, tau_err: int = 0, lam_q8: int = 0):
    """(k, s) of the exhaustive search over the 112 (shift, mode) pairs for
    the residual block r (16 ints), or None when no pair fits."""
    a = np.ascontiguousarray(r, dtype=np.int32)
    k, s_ = ctypes.c_int(), ctypes.c_int()
    if lib().or_ks_search(_ptr(a), a.size, q, tau_err, lam_q8, ctypes.byref(k), ctypes.byref(s_)) != 0:
        return None
    return k.value, s_.value


def ks_cost(r, q: int, s: int, k: int, tau_err: int, lam_q8: int):
    """256 * bits + lam_q8 * SSE of (s, k) for block r, or None when (s, k)
    is not a candidate."""
    a = np.ascontiguousarray(r, dtype=np.int32)
    c = ctypes.c_longlong()
    if lib().or_ks_cost(_ptr(a), a.size, q, s, k, tau_err, lam_q8, ctypes.byref(c)) != 0:
        return None
    return c.value


def ks_quantise(r, q: int, s: int) -> np.ndarray:
    a = np.ascontiguousarray(r, dtype=np.int32)
    out = np.empty_like(a)
    lib().or_ks_quantise(_ptr(a), a.size, q, s, _ptr(out))
    return out


def ks_features(r) -> np.ndarray:
    """The 48 block statistics (float64) of a 16-value residual block."""
    a = np.ascontiguousarray(r, dtype=np.int32)
    assert a.size == 16
    f = np.empty(48, dtype=np.float64)
    lib().or_ks_features(_ptr(a), _ptr(f))
    return f


def mlp_nparams() -> int:
    return lib().or_mlp_nparams()


def mlp_forward(w: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Logits [n, 112] (float64) of the aid's network for inputs x [n, 48]."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    out = np.empty((n, NCLASSES), dtype=np.float64)
    lib().or_mlp_forward(_ptr(w), _ptr(x), n, _ptr(out))
    return out


def mlp_loss_grad(w: np.ndarray, x: np.ndarray, y: np.ndarray):
    """(summed cross-entropy, summed gradient [P]) in float64."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.int32)
    g = np.empty(mlp_nparams(), dtype=np.float64)
    loss = ctypes.c_double()
    if lib().or_mlp_loss_grad(_ptr(w), _ptr(x), _ptr(y), x.shape[0], _ptr(g), ctypes.byref(loss)) != 0:
        raise ValueError("label out of range")
    return loss.value, g

"""Python binding of librlfc.so (include/rlfc.h).

Argument marshalling only: torch tensors provide device memory and the CUDA
stream; every step of decoding and rendering runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or the device is
not a CUDA GPU, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from .buildlib import LIB, LIB_DEBUG

RLFC_OK = 0
RLFC_E_RANGE = 6   # a size beyond what the call supports (include/rlfc.h)
REQ_OK, REQ_BAD_VIEW, REQ_BAD_LOCATION = 0, 1, 2


class RLFCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in
                ("U", "V", "W", "H", "B", "L", "q", "n_top", "S", "Wp", "Hp", "nloc_x", "nloc_y")] + \
               [(k, ctypes.c_uint64) for k in ("stream_bytes", "record_bytes", "top_bytes", "device_bytes")]


class EncParams(ctypes.Structure):
    _fields_ = [("U", ctypes.c_uint32), ("V", ctypes.c_uint32), ("W", ctypes.c_uint32),
                ("H", ctypes.c_uint32), ("B", ctypes.c_uint32), ("L", ctypes.c_uint32),
                ("c", ctypes.c_uint32 * 8), ("tau_p", ctypes.c_int32), ("tau_b", ctypes.c_int32),
                ("q", ctypes.c_uint32), ("mode_space", ctypes.c_uint32), ("tau_err", ctypes.c_int32),
                ("lam_q8", ctypes.c_uint32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_uint32), ("locs_per_pop", ctypes.c_uint32),
                ("stage", ctypes.c_uint32), ("graph", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("memory_budget", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("lf", ctypes.c_uint32),
                ("batch", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 56), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


EXPORTS = ["rlfc_load_stream", "rlfc_stream_info", "rlfc_free_stream", "rlfc_decode_all",
           "rlfc_decode_blocks", "rlfc_render_views", "rlfc_render_views_u8", "rlfc_encode", "rlfc_encode_ex", "rlfc_encode_no_alloc",
           "rlfc_free_host", "rlfc_strerror", "rlfc_last_error", "rlfc_trace_enable", "rlfc_trace_read",
           "rlfc_batch_create", "rlfc_batch_set_config", "rlfc_batch_get_config", "rlfc_batch_decode",
           "rlfc_batch_autotune", "rlfc_batch_free", "rlfc_server_create", "rlfc_server_add",
           "rlfc_server_submit", "rlfc_server_submit_u8", "rlfc_server_poll", "rlfc_server_now", "rlfc_server_free",
           "rlfc_ks_search", "rlfc_ks_compact", "rlfc_ks_features", "rlfc_mlp_loss_grad", "rlfc_mlp_adam",
           "rlfc_mlp_predict", "rlfc_debug_flags"]

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process binds: the release build, or the debug build
    (device bounds checks, rlfc_debug_flags) when RLFC_DEBUG_LIBRARY=1 is set
    before the first call."""
    return LIB_DEBUG if os.environ.get("RLFC_DEBUG_LIBRARY") == "1" else LIB


def lib():
    """The loaded librlfc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"librlfc.so not built ({path}); run paper_1805_06019_gb300.build()")
            L = ctypes.CDLL(path)
            vp, sz, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32
            L.rlfc_load_stream.argtypes = [vp, sz, vp, ctypes.POINTER(vp)]
            L.rlfc_stream_info.argtypes = [vp, ctypes.POINTER(Info)]
            L.rlfc_free_stream.argtypes = [vp]
            L.rlfc_free_stream.restype = None
            L.rlfc_decode_all.argtypes = [vp, vp, vp]
            L.rlfc_decode_blocks.argtypes = [vp, vp, vp, sz, vp, vp, vp]
            L.rlfc_render_views.argtypes = [vp, vp, vp, u32, u32, sz, vp, vp]
            L.rlfc_render_views_u8.argtypes = [vp, vp, vp, u32, u32, sz, vp, vp]
            L.rlfc_encode.argtypes = [ctypes.POINTER(EncParams), vp, vp, ctypes.POINTER(vp), ctypes.POINTER(sz)]
            L.rlfc_encode_ex.argtypes = [ctypes.POINTER(EncParams), vp, vp, vp, vp, vp, ctypes.POINTER(vp),
                                         ctypes.POINTER(sz)]
            L.rlfc_encode_no_alloc.argtypes = [ctypes.POINTER(EncParams), vp, vp, vp, sz, ctypes.POINTER(sz)]
            L.rlfc_free_host.argtypes = [vp]
            L.rlfc_free_host.restype = None
            L.rlfc_strerror.argtypes = [ctypes.c_int]
            L.rlfc_strerror.restype = ctypes.c_char_p
            L.rlfc_last_error.argtypes = []
            L.rlfc_last_error.restype = ctypes.c_char_p
            L.rlfc_batch_create.argtypes = [vp, sz, ctypes.POINTER(vp)]
            L.rlfc_batch_set_config.argtypes = [vp, ctypes.POINTER(BatchConfig)]
            L.rlfc_batch_get_config.argtypes = [vp, ctypes.POINTER(BatchConfig)]
            L.rlfc_batch_decode.argtypes = [vp, vp, vp, sz, u32, vp, vp, vp]
            L.rlfc_batch_autotune.argtypes = [vp, vp, vp, sz, vp, vp, vp, ctypes.POINTER(BatchConfig)]
            L.rlfc_batch_free.argtypes = [vp]
            L.rlfc_batch_free.restype = None
            L.rlfc_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
            L.rlfc_server_add.argtypes = [vp, vp, ctypes.POINTER(u32)]
            L.rlfc_server_submit.argtypes = [vp, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float, u32, u32, vp,
                                             ctypes.POINTER(ctypes.c_uint64)]
            L.rlfc_server_submit_u8.argtypes = L.rlfc_server_submit.argtypes
            L.rlfc_server_poll.argtypes = [vp, ctypes.POINTER(Completion), sz, ctypes.POINTER(sz), ctypes.c_int]
            L.rlfc_server_now.argtypes = []
            L.rlfc_server_now.restype = ctypes.c_double
            L.rlfc_server_free.argtypes = [vp]
            L.rlfc_server_free.restype = None
            i32, f32 = ctypes.c_int32, ctypes.c_float
            L.rlfc_ks_search.argtypes = [vp, sz, u32, i32, u32, vp, vp]
            L.rlfc_ks_compact.argtypes = [vp, sz, vp, vp, vp]
            L.rlfc_ks_features.argtypes = [vp, vp, vp, sz, vp, vp, vp]
            L.rlfc_mlp_loss_grad.argtypes = [vp, vp, vp, vp, sz, vp, vp, vp]
            L.rlfc_mlp_adam.argtypes = [vp, vp, vp, vp, vp, f32, f32, f32, f32, f32, u32, vp]
            L.rlfc_mlp_predict.argtypes = [vp, vp, sz, vp, vp, vp]
            L.rlfc_trace_enable.argtypes = [ctypes.c_int]
            L.rlfc_trace_read.argtypes = [ctypes.POINTER(TraceEntry), sz, ctypes.POINTER(sz), ctypes.c_int]
            L.rlfc_debug_flags.argtypes = [vp, ctypes.POINTER(u32), ctypes.c_int]
            _lib = L
        return _lib


def _check(code: int):
    if code != RLFC_OK:
        L = lib()
        raise RLFCError(code, f"{L.rlfc_strerror(code).decode()}: {L.rlfc_last_error().decode()}")


def trace_enable(on: bool = True):
    """Bracket every library kernel launch with CUDA events (rlfc_trace_enable)."""
    _check(lib().rlfc_trace_enable(1 if on else 0))


def trace_read(reset: bool = True) -> dict:
    """{kernel name: (launches, total ms)} since the last reset, after waiting
    for the traced work (rlfc_trace_read)."""
    L = lib()
    n = ctypes.c_size_t()
    _check(L.rlfc_trace_read(None, 0, ctypes.byref(n), 0))
    cap = max(n.value, 1)
    arr = (TraceEntry * cap)()
    _check(L.rlfc_trace_read(arr, cap, ctypes.byref(n), 1 if reset else 0))
    return {arr[k].kernel.decode(): (int(arr[k].launches), float(arr[k].total_ms)) for k in range(min(n.value, cap))}


def _stream_handle(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dev(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return t.data_ptr()


class Stream:
    """A compressed light field resident on the current CUDA device
    (rlfc_load_stream)."""

    def __init__(self, data: bytes, stream=None):
        L = lib()
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        h = ctypes.c_void_p()
        _check(L.rlfc_load_stream(buf, len(data), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.info = Info()
        _check(L.rlfc_stream_info(self._h, ctypes.byref(self.info)))
        i = self.info
        self.U, self.V, self.W, self.H, self.B, self.L = i.U, i.V, i.W, i.H, i.B, i.L
        self.nloc_x, self.nloc_y = i.nloc_x, i.nloc_y
        self.nloc = i.nloc_x * i.nloc_y
        self.n_views = i.U * i.V

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rlfc_free_stream(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def debug_flags(self, reset: bool = True) -> int:
        """The flags the device bounds checks raised for this stream
        (rlfc_debug_flags; debug builds only, raises RLFCError otherwise)."""
        f = ctypes.c_uint32(0)
        _check(lib().rlfc_debug_flags(self._h, ctypes.byref(f), 1 if reset else 0))
        return int(f.value)

    def decode_all(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Every view: [U*V, H, W, 3] uint8 (rlfc_decode_all)."""
        if out is None:
            out = torch.empty((self.n_views, self.H, self.W, 3), dtype=torch.uint8, device="cuda")
        assert out.numel() == self.n_views * self.H * self.W * 3
        _check(lib().rlfc_decode_all(self._h, ctypes.c_void_p(_dev(out, torch.uint8, "out")),
                                     _stream_handle(stream)))
        return out

    def decode_blocks(self, views: torch.Tensor, locs: torch.Tensor, out: torch.Tensor | None = None,
                      status: torch.Tensor | None = None, stream=None):
        """Random blocks: (out [n, 4, 4, 3] uint8, status [n] uint8) (rlfc_decode_blocks)."""
        n = views.numel()
        if locs.numel() != n:
            raise ValueError("views and locs differ in length")
        if out is None:
            out = torch.empty((n, self.B, self.B, 3), dtype=torch.uint8, device="cuda")
        if status is None:
            status = torch.empty((n,), dtype=torch.uint8, device="cuda")
        if n == 0:
            return out, status
        _check(lib().rlfc_decode_blocks(
            self._h, ctypes.c_void_p(_dev(views, torch.int32, "views") if views.dtype == torch.int32
                                     else _dev(views, torch.uint32, "views")),
            ctypes.c_void_p(_dev(locs, torch.int32, "locs") if locs.dtype == torch.int32
                            else _dev(locs, torch.uint32, "locs")),
            n, ctypes.c_void_p(_dev(out, torch.uint8, "out")),
            ctypes.c_void_p(_dev(status, torch.uint8, "status")), _stream_handle(stream)))
        return out, status

    def render(self, uv: torch.Tensor, disp: torch.Tensor, out_w: int, out_h: int,
               out: torch.Tensor | None = None, stream=None, u8: bool = False) -> torch.Tensor:
        """New views: [n, out_h, out_w, 3] float32 in [0, 1] (rlfc_render_views),
        or uint8 with u8=True or a uint8 `out` (rlfc_render_views_u8)."""
        n = disp.numel()
        if uv.numel() != 2 * n:
            raise ValueError("uv must hold two floats per view")
        if out is None:
            out = torch.empty((n, out_h, out_w, 3), dtype=torch.uint8 if u8 else torch.float32, device="cuda")
        if n == 0:
            return out
        if out.dtype == torch.uint8:
            _check(lib().rlfc_render_views_u8(
                self._h, ctypes.c_void_p(_dev(uv, torch.float32, "uv")),
                ctypes.c_void_p(_dev(disp, torch.float32, "disp")), out_w, out_h, n,
                ctypes.c_void_p(_dev(out, torch.uint8, "out")), _stream_handle(stream)))
            return out
        _check(lib().rlfc_render_views(
            self._h, ctypes.c_void_p(_dev(uv, torch.float32, "uv")),
            ctypes.c_void_p(_dev(disp, torch.float32, "disp")), out_w, out_h, n,
            ctypes.c_void_p(_dev(out, torch.float32, "out")), _stream_handle(stream)))
        return out


def _u32_ptr(t: torch.Tensor, name: str) -> int:
    return _dev(t, torch.int32, name) if t.dtype == torch.int32 else _dev(t, torch.uint32, name)


class Batch:
    """Batched random-access decode of one loaded stream (rlfc_batch_*):
    requests grouped by location, one persistent kernel, optionally replayed
    as a captured CUDA graph.  Calls on one object must not overlap."""

    def __init__(self, stream: Stream, max_requests: int):
        self.stream = stream          # keeps the stream alive
        h = ctypes.c_void_p()
        _check(lib().rlfc_batch_create(stream._h, int(max_requests), ctypes.byref(h)))
        self._h = h
        self.max_requests = int(max_requests)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rlfc_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def config(self) -> dict:
        c = BatchConfig()
        _check(lib().rlfc_batch_get_config(self._h, ctypes.byref(c)))
        return c.as_dict()

    @config.setter
    def config(self, cfg: dict):
        c = BatchConfig()
        cur = self.config
        cur.update(cfg)
        for k, v in cur.items():
            setattr(c, k, int(v))
        _check(lib().rlfc_batch_set_config(self._h, ctypes.byref(c)))

    def decode(self, views: torch.Tensor, locs: torch.Tensor, out: torch.Tensor | None = None,
               status: torch.Tensor | None = None, level: int = 0, stream=None):
        """(out [n, 4, 4, 3] uint8, status [n] uint8 or None) at tree level
        `level` (rlfc_batch_decode)."""
        n = views.numel()
        if locs.numel() != n:
            raise ValueError("views and locs differ in length")
        s = self.stream
        if out is None:
            out = torch.empty((n, s.B, s.B, 3), dtype=torch.uint8, device="cuda")
        if n == 0:
            return out, status
        st_ptr = ctypes.c_void_p(_dev(status, torch.uint8, "status")) if status is not None else None
        _check(lib().rlfc_batch_decode(self._h, ctypes.c_void_p(_u32_ptr(views, "views")),
                                       ctypes.c_void_p(_u32_ptr(locs, "locs")), n, int(level),
                                       ctypes.c_void_p(_dev(out, torch.uint8, "out")), st_ptr,
                                       _stream_handle(stream)))
        return out, status

    def autotune(self, views: torch.Tensor, locs: torch.Tensor, out: torch.Tensor,
                 status: torch.Tensor | None = None, stream=None) -> dict:
        """Time the candidate configurations on these requests and keep the
        fastest (rlfc_batch_autotune); returns it."""
        c = BatchConfig()
        st_ptr = ctypes.c_void_p(_dev(status, torch.uint8, "status")) if status is not None else None
        _check(lib().rlfc_batch_autotune(self._h, ctypes.c_void_p(_u32_ptr(views, "views")),
                                         ctypes.c_void_p(_u32_ptr(locs, "locs")), views.numel(),
                                         ctypes.c_void_p(_dev(out, torch.uint8, "out")), st_ptr,
                                         _stream_handle(stream), ctypes.byref(c)))
        return c.as_dict()


class Server:
    """Serving runtime (rlfc_server_*): resident streams, a worker thread that
    batches view requests continuously over several CUDA streams, admission
    by device memory.  Results land in host tensors given at submit."""

    def __init__(self, n_streams: int = 4, max_batch: int = 64, memory_budget: int = 1 << 30,
                 max_inflight: int = 1):
        cfg = ServerConfig(n_streams, max_batch, memory_budget, max_inflight, 0)
        h = ctypes.c_void_p()
        _check(lib().rlfc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._streams = []
        self._outs = {}

    def add(self, stream: Stream) -> int:
        lf = ctypes.c_uint32()
        _check(lib().rlfc_server_add(self._h, stream._h, ctypes.byref(lf)))
        self._streams.append(stream)
        return lf.value

    def submit(self, lf: int, u: float, v: float, disp: float, out: torch.Tensor) -> int:
        """Queue a view of out.shape [H, W, 3] (float32 host tensor, or uint8
        for 8-bit RGB; ideally pinned); returns its ticket."""
        if out.is_cuda or out.dtype not in (torch.float32, torch.uint8) or not out.is_contiguous() \
                or out.dim() != 3:
            raise TypeError("out must be a contiguous float32 or uint8 host tensor [H, W, 3]")
        t = ctypes.c_uint64()
        fn = lib().rlfc_server_submit_u8 if out.dtype == torch.uint8 else lib().rlfc_server_submit
        _check(fn(self._h, int(lf), float(u), float(v), float(disp), out.shape[1], out.shape[0],
                  ctypes.c_void_p(out.data_ptr()), ctypes.byref(t)))
        self._outs[t.value] = out          # keep the destination alive until completion
        return t.value

    def poll(self, wait: bool = False, cap: int = 4096) -> list:
        """Completed requests as dicts (ticket, status, lf, batch, t_submit,
        t_start, t_done); wait=True first waits for every submitted one."""
        arr = (Completion * cap)()
        n = ctypes.c_size_t()
        res = []
        first = True
        while True:
            _check(lib().rlfc_server_poll(self._h, arr, cap, ctypes.byref(n), 1 if (wait and first) else 0))
            first = False
            for k in range(n.value):
                c = arr[k]
                res.append({"ticket": int(c.ticket), "status": int(c.status), "lf": int(c.lf),
                            "batch": int(c.batch), "t_submit": c.t_submit, "t_start": c.t_start,
                            "t_done": c.t_done})
                self._outs.pop(int(c.ticket), None)
            if n.value < cap:
                return res

    @staticmethod
    def now() -> float:
        return lib().rlfc_server_now()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rlfc_server_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode(rgb: torch.Tensor, U: int, V: int, L: int, c, tau_p: int = 0, tau_b: int = 0,
           q: int = 0, B: int = 4, stream=None, mode_space: int = 0, tau_err: int = 0, lam_q8: int = 0,
           leaf_modes: torch.Tensor | None = None, leaf_resid: torch.Tensor | None = None,
           leaf_label: torch.Tensor | None = None) -> bytes:
    """Algorithm 1 on the GPU (rlfc_encode / rlfc_encode_ex): views rgb
    [U*V, H, W, 3] uint8 on the device -> stream bytes.  c[l] is the cluster
    side building level l.  mode_space 1 selects per-block (mode, shift); the
    leaf_* device tensors ([U*V*3*nloc] uint8, [U*V*3*nloc, 16] int16) give
    level-0 modes or receive the level-0 residuals and search labels."""
    if rgb.dim() != 4 or rgb.shape[0] != U * V or rgb.shape[-1] != 3:
        raise ValueError("rgb must be [U*V, H, W, 3]")
    p = EncParams()
    p.U, p.V, p.W, p.H, p.B, p.L = U, V, rgb.shape[2], rgb.shape[1], B, L
    for l in range(1, L):
        p.c[l] = int(c[l])
    p.tau_p, p.tau_b, p.q = int(tau_p), int(tau_b), int(q)
    p.mode_space, p.tau_err, p.lam_q8 = int(mode_space), int(tau_err), int(lam_q8)
    nblk = U * V * 3 * ((rgb.shape[2] + 3) // 4) * ((rgb.shape[1] + 3) // 4)
    ptrs = []
    for t, dt, shape in ((leaf_modes, torch.uint8, nblk), (leaf_resid, torch.int16, nblk * 16),
                         (leaf_label, torch.uint8, nblk)):
        if t is None:
            ptrs.append(None)
        else:
            if t.numel() != shape:
                raise ValueError("leaf tensors must hold one entry (16 for residuals) per level-0 block")
            ptrs.append(ctypes.c_void_p(_dev(t, dt, "leaf tensor")))
    out = ctypes.c_void_p()
    n = ctypes.c_size_t()
    _check(lib().rlfc_encode_ex(ctypes.byref(p), ctypes.c_void_p(_dev(rgb, torch.uint8, "rgb")), *ptrs,
                                _stream_handle(stream), ctypes.byref(out), ctypes.byref(n)))
    try:
        return ctypes.string_at(out, n.value)
    finally:
        lib().rlfc_free_host(out)


def encode_no_alloc(rgb: torch.Tensor, U: int, V: int, L: int, c, tau_p: int = 0, tau_b: int = 0,
                    q: int = 0, B: int = 4, capacity: int | None = None, stream=None) -> bytes:
    """rlfc_encode_no_alloc: the GPU encoder with its device scratch taken from
    the library's fixed 32 MiB array (no device allocation); small light fields
    only.  `capacity` sizes the host output buffer (default: the raw views)."""
    if rgb.dim() != 4 or rgb.shape[0] != U * V or rgb.shape[-1] != 3:
        raise ValueError("rgb must be [U*V, H, W, 3]")
    p = EncParams()
    p.U, p.V, p.W, p.H, p.B, p.L = U, V, rgb.shape[2], rgb.shape[1], B, L
    for l in range(1, L):
        p.c[l] = int(c[l])
    p.tau_p, p.tau_b, p.q = int(tau_p), int(tau_b), int(q)
    cap = int(capacity) if capacity is not None else 4 * rgb.numel() + (1 << 16)
    for _ in range(2):
        buf = ctypes.create_string_buffer(max(cap, 1))
        n = ctypes.c_size_t()
        rc = lib().rlfc_encode_no_alloc(ctypes.byref(p), ctypes.c_void_p(_dev(rgb, torch.uint8, "rgb")),
                                        _stream_handle(stream), buf, cap, ctypes.byref(n))
        if rc == RLFC_E_RANGE and n.value > cap:
            cap = n.value   # the stream did not fit the host buffer: its size is known now
            continue
        _check(rc)
        return buf.raw[: n.value]
    _check(rc)

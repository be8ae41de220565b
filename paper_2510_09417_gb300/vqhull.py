"""Python binding of libvqhull (include/vqhull.h): argument marshalling only.

Every function here forwards to the C ABI of the CUDA library with the
same name; PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library cannot be loaded, or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import libbuild as _build

_lock = threading.Lock()
_lib = None

VQ_OK = 0
VQ_PENDING = 1


class VQError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Config(ctypes.Structure):
    _fields_ = [
        ("points_per_thread", ctypes.c_int32),
        ("small_max", ctypes.c_int32),
        ("k1_blocks_per_sm", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("timeout_ns", ctypes.c_int64),
        ("debug_drop_tile", ctypes.c_int32),
        ("ordered", ctypes.c_int32),
        ("host_loop", ctypes.c_int32),
        ("prefilter", ctypes.c_int32),
        ("k1_shape", ctypes.c_int32),
        ("worklist_points", ctypes.c_int64),
    ]


class Profile(ctypes.Structure):
    _fields_ = [
        ("calls", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("k1_launches", ctypes.c_int64),
        ("levels", ctypes.c_int64),
        ("k1_points_read", ctypes.c_int64),
        ("k1_points_kept", ctypes.c_int64),
        ("k0_ms", ctypes.c_double),
        ("k1_ms", ctypes.c_double),
        ("k2_ms", ctypes.c_double),
        ("k3_ms", ctypes.c_double),
        ("k4_ms", ctypes.c_double),
        ("other_ms", ctypes.c_double),
        ("graph_launches", ctypes.c_int64),
        ("sample_ms", ctypes.c_double),
        ("k5_ms", ctypes.c_double),
        ("worklist_reruns", ctypes.c_int64),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("mem_budget_bytes", ctypes.c_size_t),
        ("max_inflight", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("lanes", ctypes.c_int32),
        ("pinned_bytes", ctypes.c_size_t),
    ]


class ServerInfo(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("max_busy_lanes", ctypes.c_int64),
        ("admitted_while_busy", ctypes.c_int64),
        ("peak_bytes", ctypes.c_int64),
        ("budget_bytes", ctypes.c_int64),
    ]


SYMBOLS = (
    "vq_status_string", "vq_version", "vq_hull2d", "vq_hull2d_aos", "vq_hull2d_batched", "vq_hull2d_host", "vq_hull2d_noalloc",
    "vq_get_config", "vq_set_config", "vq_last_stats", "vq_profile_read", "vq_autotune", "vq_debug_orient_f32",
    "vq_debug_round_f32",
    "vq_server_create", "vq_server_submit",
    "vq_server_poll", "vq_server_wait", "vq_server_wait_any", "vq_server_stats", "vq_server_info_read", "vq_server_destroy",
)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvqhull.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("VQHULL_LIB") or _build.LIB  # override: an alternative build
        if build_if_missing and path == _build.LIB:
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libvqhull.so not found at {path}; run build()")
        lib = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.vq_status_string.argtypes = [ctypes.c_int]
        lib.vq_status_string.restype = ctypes.c_char_p
        lib.vq_version.restype = ctypes.c_int
        lib.vq_hull2d.argtypes = [vp, vp, i64, vp, i64p, vp]
        lib.vq_hull2d.restype = ctypes.c_int
        lib.vq_hull2d_aos.argtypes = [vp, i64, vp, i64p, vp]
        lib.vq_hull2d_aos.restype = ctypes.c_int
        lib.vq_hull2d_batched.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        lib.vq_hull2d_batched.restype = ctypes.c_int
        lib.vq_hull2d_host.argtypes = [vp, vp, i64, vp, i64p, vp]
        lib.vq_hull2d_host.restype = ctypes.c_int
        lib.vq_hull2d_noalloc.argtypes = [vp, vp, i64, vp, i64p, vp]
        lib.vq_hull2d_noalloc.restype = ctypes.c_int
        lib.vq_get_config.argtypes = [ctypes.POINTER(Config)]
        lib.vq_get_config.restype = ctypes.c_int
        lib.vq_set_config.argtypes = [ctypes.POINTER(Config)]
        lib.vq_set_config.restype = ctypes.c_int
        lib.vq_last_stats.argtypes = [i64p, i64p, i64p, i64p, i32]
        lib.vq_last_stats.restype = ctypes.c_int
        lib.vq_profile_read.argtypes = [ctypes.POINTER(Profile), i32]
        lib.vq_profile_read.restype = ctypes.c_int
        lib.vq_autotune.argtypes = [vp, vp, i64, i32, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_double), vp]
        lib.vq_autotune.restype = ctypes.c_int
        lib.vq_debug_orient_f32.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.vq_debug_orient_f32.restype = ctypes.c_int
        lib.vq_debug_round_f32.argtypes = [vp, i64, vp, vp]
        lib.vq_debug_round_f32.restype = ctypes.c_int
        lib.vq_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        lib.vq_server_create.restype = ctypes.c_int
        lib.vq_server_submit.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
        lib.vq_server_submit.restype = ctypes.c_int
        lib.vq_server_poll.argtypes = [vp, ctypes.c_uint64, vp, i64, i64p]
        lib.vq_server_poll.restype = ctypes.c_int
        lib.vq_server_wait.argtypes = [vp, ctypes.c_uint64, vp, i64, i64p, i32]
        lib.vq_server_wait.restype = ctypes.c_int
        lib.vq_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.vq_server_stats.restype = ctypes.c_int
        lib.vq_server_wait_any.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), vp, i64, i64p, i32,
                                           ctypes.POINTER(ctypes.c_double)]
        lib.vq_server_wait_any.restype = ctypes.c_int
        lib.vq_server_info_read.argtypes = [vp, ctypes.POINTER(ServerInfo)]
        lib.vq_server_info_read.restype = ctypes.c_int
        lib.vq_server_destroy.argtypes = [vp]
        lib.vq_server_destroy.restype = None
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().vq_status_string(int(status)).decode()


def vq_status_string(status: int) -> str:
    return status_string(status)


def vq_version() -> int:
    return int(load().vq_version())


def _check(st: int, where: str, ok=(VQ_OK,)) -> int:
    if st not in ok:
        raise VQError(st, where)
    return st


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 1:
        raise TypeError(f"{name} must be a 1-D float64 CUDA tensor")
    return t.contiguous()


def vq_hull2d(x: torch.Tensor, y: torch.Tensor, hull_idx: torch.Tensor | None = None, stream=None):
    """Hull of one point set: returns hull_idx[:h] (int32, device), clockwise
    from the lexicographic minimum.  hull_idx, if given, needs n entries."""
    lib = load()
    x, y = _dev_f64(x, "x"), _dev_f64(y, "y")
    n = x.shape[0]
    if y.shape[0] != n:
        raise ValueError("x and y differ in length")
    if hull_idx is None:
        hull_idx = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
    elif hull_idx.dtype != torch.int32 or hull_idx.numel() < n or not hull_idx.is_cuda:
        raise ValueError("hull_idx must be an int32 CUDA tensor with room for n indices")
    h = ctypes.c_int64(0)
    st = lib.vq_hull2d(x.data_ptr(), y.data_ptr(), n, hull_idx.data_ptr(), ctypes.byref(h), _stream_ptr(stream))
    _check(st, "vq_hull2d")
    return hull_idx[: h.value]


def vq_hull2d_aos(xy: torch.Tensor, hull_idx: torch.Tensor | None = None, stream=None):
    """Hull of one point set given interleaved: xy is an (n, 2) (or 2n-long)
    float64 CUDA tensor of (x, y) pairs.  Returns hull_idx[:h] as vq_hull2d."""
    lib = load()
    if not isinstance(xy, torch.Tensor) or not xy.is_cuda or xy.dtype != torch.float64:
        raise TypeError("xy must be a float64 CUDA tensor")
    xy = xy.contiguous().reshape(-1)
    if xy.numel() % 2:
        raise ValueError("xy holds an odd number of values")
    n = xy.numel() // 2
    if hull_idx is None:
        hull_idx = torch.empty(max(n, 1), dtype=torch.int32, device=xy.device)
    elif hull_idx.dtype != torch.int32 or hull_idx.numel() < n or not hull_idx.is_cuda:
        raise ValueError("hull_idx must be an int32 CUDA tensor with room for n indices")
    h = ctypes.c_int64(0)
    _check(lib.vq_hull2d_aos(xy.data_ptr(), n, hull_idx.data_ptr(), ctypes.byref(h), _stream_ptr(stream)),
           "vq_hull2d_aos")
    return hull_idx[: h.value]


def vq_hull2d_batched(x: torch.Tensor, y: torch.Tensor, offsets: torch.Tensor,
                      hull_idx: torch.Tensor | None = None, hull_offsets: torch.Tensor | None = None,
                      stream=None, allow_nonfinite: bool = False):
    """Hulls of the sets x[offsets[s]:offsets[s+1]]: returns (hull_idx,
    hull_offsets); hull s is hull_idx[hull_offsets[s]:hull_offsets[s+1]]
    with set-local indices."""
    lib = load()
    x, y = _dev_f64(x, "x"), _dev_f64(y, "y")
    if not offsets.is_cuda or offsets.dtype != torch.int64:
        raise TypeError("offsets must be an int64 CUDA tensor")
    offsets = offsets.contiguous()
    nsets = offsets.shape[0] - 1
    n = x.shape[0]
    if hull_idx is None:
        hull_idx = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
    if hull_offsets is None:
        hull_offsets = torch.empty(nsets + 1, dtype=torch.int64, device=x.device)
    st = lib.vq_hull2d_batched(x.data_ptr(), y.data_ptr(), offsets.data_ptr(), nsets, hull_idx.data_ptr(),
                               hull_offsets.data_ptr(), _stream_ptr(stream))
    _check(st, "vq_hull2d_batched", ok=(VQ_OK, -2) if allow_nonfinite else (VQ_OK,))
    return hull_idx, hull_offsets


def vq_hull2d_host(x, y, hull_idx=None, stream=None):
    """Hull of host points (numpy or CPU tensors, float64); copies in and out.
    Returns the int32 indices as a numpy array."""
    lib = load()
    xa = x.numpy() if isinstance(x, torch.Tensor) else np.asarray(x)
    ya = y.numpy() if isinstance(y, torch.Tensor) else np.asarray(y)
    xa = np.ascontiguousarray(xa, dtype=np.float64)
    ya = np.ascontiguousarray(ya, dtype=np.float64)
    n = xa.shape[0]
    out = hull_idx if hull_idx is not None else np.empty(max(n, 1), dtype=np.int32)
    out_ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
    h = ctypes.c_int64(0)
    st = lib.vq_hull2d_host(xa.ctypes.data, ya.ctypes.data, n, out_ptr, ctypes.byref(h), _stream_ptr(stream))
    _check(st, "vq_hull2d_host")
    return out[: h.value]


def vq_hull2d_noalloc(x: torch.Tensor, y: torch.Tensor, hull_idx: torch.Tensor, stream=None):
    """vq_hull2d without any allocation inside the library (fixed scratch;
    n <= 1,048,576).  The caller provides hull_idx (int32, room for n)."""
    lib = load()
    x, y = _dev_f64(x, "x"), _dev_f64(y, "y")
    n = x.shape[0]
    if y.shape[0] != n:
        raise ValueError("x and y differ in length")
    if hull_idx.dtype != torch.int32 or hull_idx.numel() < n or not hull_idx.is_cuda:
        raise ValueError("hull_idx must be an int32 CUDA tensor with room for n indices")
    h = ctypes.c_int64(0)
    st = lib.vq_hull2d_noalloc(x.data_ptr(), y.data_ptr(), n, hull_idx.data_ptr(), ctypes.byref(h),
                               _stream_ptr(stream))
    _check(st, "vq_hull2d_noalloc")
    return hull_idx[: h.value]


def vq_get_config() -> Config:
    cfg = Config()
    _check(load().vq_get_config(ctypes.byref(cfg)), "vq_get_config")
    return cfg


def vq_set_config(cfg: Config | None = None, **kw) -> Config:
    """Set tuning knobs; keyword arguments update the current config."""
    c = cfg if cfg is not None else vq_get_config()
    for k, v in kw.items():
        setattr(c, k, v)
    _check(load().vq_set_config(ctypes.byref(c)), "vq_set_config")
    return c


def vq_debug_round_f32(v: torch.Tensor, stream=None) -> torch.Tensor:
    """The FP32 tiers' FP64 -> FP32 rounding (round to nearest, ties to even)
    of device FP64 values: returns the FP32 results on the device."""
    lib = load()
    if not isinstance(v, torch.Tensor) or v.device.type != "cuda" or v.dtype != torch.float64:
        raise TypeError("v must be a CUDA float64 tensor")
    t = v.contiguous().reshape(-1)
    out = torch.empty(t.shape[0], dtype=torch.float32, device=t.device)
    _check(lib.vq_debug_round_f32(t.data_ptr(), t.shape[0], out.data_ptr(), _stream_ptr(stream)), "vq_debug_round_f32")
    return out


def vq_debug_orient_f32(tri: torch.Tensor, tier: int = 0, stream=None):
    """An FP32 tier's value and bound of orient(a, b, u) for device FP64
    triples tri[k] = (ax, ay, bx, by, ux, uy) (tier 0: absolute
    coordinates, 1: relative to a): returns (d, e) on the device."""
    lib = load()
    if not isinstance(tri, torch.Tensor) or tri.device.type != "cuda" or tri.dtype != torch.float64:
        raise TypeError("tri must be a CUDA float64 tensor")
    t = tri.contiguous().reshape(-1, 6)
    m = t.shape[0]
    d = torch.empty(m, dtype=torch.float32, device=t.device)
    e = torch.empty(m, dtype=torch.float32, device=t.device)
    _check(lib.vq_debug_orient_f32(t.data_ptr(), m, int(tier), d.data_ptr(), e.data_ptr(), _stream_ptr(stream)),
           "vq_debug_orient_f32")
    return d, e


def vq_autotune(x: torch.Tensor, y: torch.Tensor, reps: int = 3, stream=None):
    """Times the hull of (x, y) under each candidate configuration, makes
    the fastest the process-wide one and returns (config, median ms)."""
    lib = load()
    x, y = _dev_f64(x, "x"), _dev_f64(y, "y")
    if y.shape[0] != x.shape[0]:
        raise ValueError("x and y differ in length")
    cfg = Config()
    ms = ctypes.c_double(0.0)
    _check(lib.vq_autotune(x.data_ptr(), y.data_ptr(), x.shape[0], reps, ctypes.byref(cfg), ctypes.byref(ms),
                           _stream_ptr(stream)), "vq_autotune")
    return cfg, float(ms.value)


def vq_last_stats() -> dict:
    """Per-level partition counters of the last call on the current device."""
    cap = 512
    levels = ctypes.c_int64(0)
    rd = (ctypes.c_int64 * cap)()
    kp = (ctypes.c_int64 * cap)()
    sg = (ctypes.c_int64 * cap)()
    _check(load().vq_last_stats(ctypes.byref(levels), rd, kp, sg, cap), "vq_last_stats")
    L = min(int(levels.value), cap)
    return {"levels": L, "read": list(rd[:L]), "written": list(kp[:L]), "segments": list(sg[:L])}


def vq_profile_read(reset: bool = False) -> dict:
    """Counters and per-kernel device times accumulated since the last reset."""
    p = Profile()
    _check(load().vq_profile_read(ctypes.byref(p), 1 if reset else 0), "vq_profile_read")
    return {name: getattr(p, name) for name, _ in Profile._fields_}


class Server:
    """vq_server_*: hull requests admitted against a device-memory budget."""

    def __init__(self, mem_budget_bytes: int, max_inflight: int = 64, device: int = 0, lanes: int = 0,
                 pinned_bytes: int = 0):
        self._lib = load()
        cfg = ServerConfig(mem_budget_bytes, max_inflight, device, lanes, pinned_bytes)
        h = ctypes.c_void_p()
        _check(self._lib.vq_server_create(ctypes.byref(cfg), ctypes.byref(h)), "vq_server_create")
        self._h = h

    def submit(self, x, y) -> int:
        xa = np.ascontiguousarray(x, dtype=np.float64)
        ya = np.ascontiguousarray(y, dtype=np.float64)
        t = ctypes.c_uint64(0)
        _check(self._lib.vq_server_submit(self._h, xa.ctypes.data, ya.ctypes.data, xa.shape[0], ctypes.byref(t)),
               "vq_server_submit")
        return int(t.value)

    def poll(self, ticket: int, cap: int):
        out = np.empty(max(cap, 1), dtype=np.int32)
        h = ctypes.c_int64(0)
        st = self._lib.vq_server_poll(self._h, ticket, out.ctypes.data, cap, ctypes.byref(h))
        if st == VQ_PENDING:
            return None
        _check(st, "vq_server_poll")
        return out[: h.value]

    def wait(self, ticket: int, cap: int, timeout_ms: int = -1):
        out = np.empty(max(cap, 1), dtype=np.int32)
        h = ctypes.c_int64(0)
        st = self._lib.vq_server_wait(self._h, ticket, out.ctypes.data, cap, ctypes.byref(h), timeout_ms)
        if st == VQ_PENDING:
            return None
        _check(st, "vq_server_wait")
        return out[: h.value]

    def wait_any(self, cap: int, timeout_ms: int = -1):
        """The first finished request not yet taken: (ticket, hull, latency
        in ms from submission to completion), or None on timeout."""
        out = np.empty(max(cap, 1), dtype=np.int32)
        t = ctypes.c_uint64(0)
        h = ctypes.c_int64(0)
        lat = ctypes.c_double(0.0)
        st = self._lib.vq_server_wait_any(self._h, ctypes.byref(t), out.ctypes.data, cap, ctypes.byref(h),
                                          timeout_ms, ctypes.byref(lat))
        if st == VQ_PENDING:
            return None
        _check(st, "vq_server_wait_any")
        return int(t.value), out[: h.value], float(lat.value)

    def stats(self):
        p50, p99, hps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.vq_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(hps)),
               "vq_server_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "hulls_per_s": hps.value}

    def info(self) -> dict:
        p = ServerInfo()
        _check(self._lib.vq_server_info_read(self._h, ctypes.byref(p)), "vq_server_info_read")
        return {name: getattr(p, name) for name, _ in ServerInfo._fields_}

    def close(self):
        if self._h:
            self._lib.vq_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

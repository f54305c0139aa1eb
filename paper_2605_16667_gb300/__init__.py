"""DialSort hot path on GB300 (sm_103a): tensor-level Python binding.

Thin wrappers over the C ABI of ``libdialsort.so`` (``include/dialsort.h``).
PyTorch supplies device memory and streams only; every step runs in the
library's CUDA kernels, and a missing library or a non-CUDA tensor is an
error (there is no CPU fallback).

Keys are 32-bit (torch.int32 / torch.uint32 storage, read as uint32) or
16-bit (torch.int16 / torch.uint16, read as uint16).  Histograms are uint32
values held in torch.int32 tensors.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import native

__all__ = [
    "DialSortError", "histogram", "reconstruct", "sort", "offsets", "plan_histogram", "stream_status",
    "sort_workspace_size", "reconstruct_workspace_size", "REGIMES", "lib", "Batch", "batched", "Server",
    "replay", "device_view", "pageable_host_access", "histogram_accumulate", "frequency", "presence",
    "range_count", "radix_sort", "sort_mapped", "probe_skew", "tune_table_load", "tune_table_size",
    "SKEW_CLASSES", "histogram_chunked", "sort_chunked",
]

OK, ERR_INVALID_ARG, ERR_KEY_RANGE, ERR_CUDA, ERR_BUDGET, ERR_TIMEOUT, ERR_BUSY, ERR_OVERFLOW, ERR_WORKSPACE = range(9)

REGIMES = {"auto": 0, "smem32": 1, "smem16": 2, "cluster": 3, "global_crn": 4, "global": 5, "two_level": 6}
REGIME_NAMES = {v: k for k, v in REGIMES.items()}
# skew classes (dialsort_skew_class_t): what the skew probe reports and the tuning table is keyed by
SKEW_CLASSES = {"unknown": 0, "low": 1, "hot": 2, "runs": 3}
SKEW_NAMES = {v: k for k, v in SKEW_CLASSES.items()}

_W4 = (torch.int32, torch.uint32)
_W2 = (torch.int16, torch.uint16)


class DialSortError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = native.load().dialsort_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def lib():
    """The loaded ctypes library (raises if it is not built)."""
    return native.load()


def _check(status: int, what: str) -> None:
    if status != OK:
        raise DialSortError(status, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _width(t: torch.Tensor) -> int:
    if t.dtype in _W4:
        return 4
    if t.dtype in _W2:
        return 2
    raise TypeError(f"keys must be 32- or 16-bit integers, got {t.dtype}")


def _cuda(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (DialSort has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _reachable(t: torch.Tensor, name: str) -> torch.Tensor:
    """A CUDA tensor, or a page-locked host tensor that the kernels read or write over the host link."""
    if not (t.is_cuda or t.is_pinned() or t.numel() == 0):  # (an empty tensor holds no pages to pin)
        raise ValueError(f"{name} must be a CUDA tensor or pinned host memory (DialSort has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _device(t: torch.Tensor) -> torch.device:
    return t.device if t.is_cuda else torch.device("cuda", torch.cuda.current_device())


def _like(t: torch.Tensor) -> torch.Tensor:
    return torch.empty_like(t) if t.is_cuda else torch.empty(t.shape, dtype=t.dtype, pin_memory=True)


def _config(config) -> ctypes.c_void_p | None:
    if config is None:
        return None
    c = native.dialsort_hist_config_t()
    for k, v in config.items():
        if k == "regime" and isinstance(v, str):
            v = REGIMES[v]
        if k == "crn" and isinstance(v, bool):
            v = 1 if v else 2
        if k == "crn" and v == "adaptive":
            v = 3
        if k == "skew" and isinstance(v, str):
            v = SKEW_CLASSES[v]
        setattr(c, k, int(v))
    return c


def probe_skew(keys: torch.Tensor, U: int, stream=None) -> dict:
    """The device skew probe (4096 sampled keys, equality tests only): counts and the skew class."""
    _reachable(keys, "keys")
    r = native.dialsort_skew_t()
    _check(native.load().dialsort_probe_skew(keys.data_ptr(), _width(keys), keys.numel(), U, ctypes.byref(r),
                                             _stream(stream)), "dialsort_probe_skew")
    d = {f: getattr(r, f) for f, _ in r._fields_ if f != "reserved"}
    d["skew_name"] = SKEW_NAMES[d["skew_class"]]
    return d


# the table the library loads when DIALSORT_TUNE_CACHE is not set (written by python -m paper_2605_16667_gb300.tune)
TUNE_TABLE = os.path.join(os.path.dirname(native.LIB_PATH), "tune_table.txt")


def tune_table_load(path: str | None) -> None:
    """Replace the autotuner's measured table by the file at path (None: no table, the cost model alone)."""
    _check(native.load().dialsort_tune_table_load(path.encode() if path is not None else None), "tune_table_load")


def tune_table_size() -> int:
    return int(native.load().dialsort_tune_table_size())


def _with_skew(config, skew, keys, U, stream):
    """config with the skew class set: an int or name, or "probe" to run the skew probe first."""
    if skew is None:
        return config
    if skew == "probe":
        skew = probe_skew(keys, U, stream)["skew_class"]
    c = dict(config or {})
    c["skew"] = SKEW_CLASSES[skew] if isinstance(skew, str) else int(skew)
    return c


def histogram_workspace_size(n: int, U: int, width: int = 4) -> int:
    return native.load().dialsort_histogram_workspace_size(n, U, width)


def histogram(keys: torch.Tensor, U: int, H: torch.Tensor | None = None, *, config: dict | None = None,
              ws: torch.Tensor | None = None, use_workspace: bool = True, stream=None, skew=None) -> torch.Tensor:
    """Eq. (1): H[k] = number of keys equal to k, for k in [0, U).  Returns H (int32 storage of uint32).

    With use_workspace (default) a workspace is passed, so large universes can use the two-level regime.
    keys may be pinned host memory: the kernels then read it over the host link.  skew: the keys' skew
    class for the autotuner (a SKEW_CLASSES name or number, or "probe" to measure it first).
    """
    _reachable(keys, "keys")
    w = _width(keys)
    if H is None:
        H = torch.empty(U, dtype=torch.int32, device=_device(keys))
    _reachable(H, "H")
    cfg = _config(_with_skew(config, skew, keys, U, stream))
    L = native.load()
    need = histogram_workspace_size(keys.numel(), U, w) if use_workspace else 0
    if need:
        ws = _workspace(need, _device(keys), ws)
        st = L.dialsort_histogram_ws(keys.data_ptr(), w, keys.numel(), U, H.data_ptr(),
                                     ctypes.byref(cfg) if cfg is not None else None, ws.data_ptr(), ws.numel(),
                                     _stream(stream))
    else:
        st = L.dialsort_histogram_ex(keys.data_ptr(), w, keys.numel(), U, H.data_ptr(),
                                     ctypes.byref(cfg) if cfg is not None else None, _stream(stream))
    _check(st, "dialsort_histogram")
    return H


def reconstruct_workspace_size(U: int, n: int) -> int:
    return native.load().dialsort_reconstruct_workspace_size(U, n)


def sort_workspace_size(n: int, U: int) -> int:
    return native.load().dialsort_sort_workspace_size(n, U)


def _workspace(nbytes: int, device, ws: torch.Tensor | None) -> torch.Tensor:
    if ws is not None and ws.numel() * ws.element_size() >= nbytes:
        return ws
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def reconstruct(H: torch.Tensor, U: int, n: int, out: torch.Tensor | None = None, *, width: int = 4,
                ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Eq. (2): out[0..sum H) = k repeated H[k] times, k ascending.  n is out's capacity.

    out may be pinned host memory: the kernels then write it over the host link.
    """
    _reachable(H, "H")
    if out is None:
        out = torch.empty(n, dtype=torch.int32 if width == 4 else torch.int16, device=_device(H))
    _reachable(out, "out")
    width = _width(out)
    ws = _workspace(reconstruct_workspace_size(U, n), _device(H), ws)
    fn = native.load().dialsort_reconstruct if width == 4 else native.load().dialsort_reconstruct_u16
    _check(fn(H.data_ptr(), U, out.data_ptr(), n, ws.data_ptr(), ws.numel(), _stream(stream)), "dialsort_reconstruct")
    return out


def offsets(H: torch.Tensor, U: int, n: int, *, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The offset scan alone: start of every 1024-bin chunk's run (int64[ceil(U/1024)+1], last = sum H)."""
    _cuda(H, "H")
    ws = _workspace(reconstruct_workspace_size(U, n), H.device, ws)
    L = native.load()
    _check(L.dialsort_offsets(H.data_ptr(), U, n, ws.data_ptr(), ws.numel(), _stream(stream)), "dialsort_offsets")
    chunks = (U + 1023) // 1024
    O = torch.empty(chunks + 1, dtype=torch.int64, device=H.device)
    _check(L.dialsort_read_chunk_offsets(ws.data_ptr(), U, n, O.data_ptr(), _stream(stream)), "read_chunk_offsets")
    return O


def sort(keys: torch.Tensor, U: int, out: torch.Tensor | None = None, *, ws: torch.Tensor | None = None,
         stream=None, return_histogram: bool = False, config: dict | None = None, skew=None):
    """Eq. (1) then Eq. (2).  out may be keys itself (in place).

    keys and out may be pinned host memory: the kernels then read the keys and write the output over
    the host link (no staging copies); the workspace is device memory either way.  config / skew: step 1's
    launch choices and the keys' skew class, as for histogram().
    """
    _reachable(keys, "keys")
    w = _width(keys)
    n = keys.numel()
    if out is None:
        out = _like(keys)
    _reachable(out, "out")
    if _width(out) != w:
        raise TypeError("out must have the key width of keys")
    nbytes = sort_workspace_size(n, U)
    ws = _workspace(nbytes, _device(keys), ws)
    L = native.load()
    cfg = _config(_with_skew(config, skew, keys, U, stream))
    if cfg is not None:
        _check(L.dialsort_sort_ex(keys.data_ptr(), w, n, U, out.data_ptr(), ctypes.byref(cfg), ws.data_ptr(),
                                  ws.numel(), _stream(stream)), "dialsort_sort_ex")
    else:
        fn = L.dialsort_sort if w == 4 else L.dialsort_sort_u16
        _check(fn(keys.data_ptr(), n, U, out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "dialsort_sort")
    if return_histogram:
        return out, ws[: 4 * U].view(torch.int32)
    return out


def sort_stage_times(keys: torch.Tensor, U: int, out: torch.Tensor, ws: torch.Tensor, stream=None) -> list:
    """One dialsort_sort with CUDA events between its stages (synchronous): the stage durations in ms --
    [pass 1, split + schedule, counting fused with the projection, long runs] for the two-level form,
    else [whole sort]."""
    ms = (ctypes.c_float * 4)()
    stages = ctypes.c_uint32()
    _check(native.load().dialsort_sort_stage_times(keys.data_ptr(), _width(keys), keys.numel(), U, out.data_ptr(),
                                                   ws.data_ptr(), ws.numel(), _stream(stream), ms,
                                                   ctypes.byref(stages)), "dialsort_sort_stage_times")
    return [float(ms[i]) for i in range(stages.value)]


def histogram_accumulate(keys: torch.Tensor, U: int, H: torch.Tensor, *, ws: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """Eq. (1) without zeroing: H[x] += 1 for every key x (H already holds counts).  Returns H."""
    _reachable(keys, "keys")
    _reachable(H, "H")
    w = _width(keys)
    need = histogram_workspace_size(keys.numel(), U, w)
    ws = _workspace(need, _device(keys), ws) if need else None
    _check(native.load().dialsort_histogram_accumulate(
        keys.data_ptr(), w, keys.numel(), U, H.data_ptr(), ws.data_ptr() if ws is not None else None,
        ws.numel() if ws is not None else 0, _stream(stream)), "dialsort_histogram_accumulate")
    return H


def _host_keys(keys: torch.Tensor):
    if keys.is_cuda:
        raise TypeError("keys must be host memory (page-locked for the copies to overlap)")
    if not keys.is_contiguous():
        raise TypeError("keys must be contiguous")
    return _width(keys)


def histogram_chunked(keys: torch.Tensor, U: int, H: torch.Tensor, *, chunk_keys: int = 1 << 24,
                      ws: torch.Tensor | None = None, stream=None, copy_stream=None) -> torch.Tensor:
    """Eq. (1) streamed from host memory: H += histogram of keys, chunk by chunk, each chunk's copy to the
    device overlapping the ingestion of the one before (copy_stream: a second CUDA stream)."""
    w = _host_keys(keys)
    _cuda(H, "H")
    L = native.load()
    need = L.dialsort_chunked_workspace_size(keys.numel(), U, w, chunk_keys, 0)
    ws = _workspace(need, H.device, ws)
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=H.device)
    _check(L.dialsort_histogram_chunked(keys.data_ptr(), w, keys.numel(), U, chunk_keys, H.data_ptr(),
                                        ws.data_ptr(), ws.numel(), _stream(stream), _stream(cs)),
           "dialsort_histogram_chunked")
    return H


def sort_chunked(keys: torch.Tensor, U: int, out: torch.Tensor | None = None, *, chunk_keys: int = 1 << 24,
                 ws: torch.Tensor | None = None, stream=None, copy_stream=None, device=None) -> torch.Tensor:
    """Sort host-resident keys: the chunked, copy-overlapped ingestion, then Eq. (2) into out (device by
    default, or page-locked host memory)."""
    w = _host_keys(keys)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty(keys.numel(), dtype=keys.dtype, device=dev)
    _reachable(out, "out")
    L = native.load()
    need = L.dialsort_chunked_workspace_size(keys.numel(), U, w, chunk_keys, 1)
    ws = _workspace(need, dev, ws)
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=dev)
    _check(L.dialsort_sort_chunked(keys.data_ptr(), w, keys.numel(), U, chunk_keys, out.data_ptr(), ws.data_ptr(),
                                   ws.numel(), _stream(stream), _stream(cs)), "dialsort_sort_chunked")
    return out


_W1 = (torch.uint8, torch.int8)


def sort_mapped(keys: torch.Tensor, U: int, phi: torch.Tensor | None = None, phi_inv: torch.Tensor | None = None,
                out: torch.Tensor | None = None, *, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sort through an order-preserving map onto [0, U) (Prop. "General Self-Indexing Principle").

    keys: 8-, 16- or 32-bit raw keys.  phi: int32/uint32 tensor of M indices (0xffffffff = outside the
    domain) or None (a key is its own index).  phi_inv: U raw values of the keys' width or None.
    """
    _reachable(keys, "keys")
    w = 1 if keys.dtype in _W1 else _width(keys)
    n = keys.numel()
    if out is None:
        out = _like(keys)
    _reachable(out, "out")
    if out.element_size() != w or out.numel() < n:
        raise ValueError("out must hold n keys of the keys' width")
    M = 0
    if phi is not None:
        _reachable(phi, "phi")
        if phi.dtype not in _W4:
            raise TypeError("phi must hold 32-bit indices")
        M = phi.numel()
    if phi_inv is not None:
        _reachable(phi_inv, "phi_inv")
        if phi_inv.element_size() != w or phi_inv.numel() < U:
            raise ValueError("phi_inv must hold U values of the keys' width")
    L = native.load()
    ws = _workspace(L.dialsort_sort_mapped_workspace_size(n, U), _device(keys), ws)
    _check(L.dialsort_sort_mapped(keys.data_ptr(), w, n, phi.data_ptr() if phi is not None else None, M,
                                  phi_inv.data_ptr() if phi_inv is not None else None, U, out.data_ptr(),
                                  ws.data_ptr(), ws.numel(), _stream(stream)), "dialsort_sort_mapped")
    return out


def radix_sort(keys: torch.Tensor, out: torch.Tensor | None = None, *, signed: bool | None = None,
               ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """DialSort-Radix: full-range 32-bit sort by four base-256 DialSort passes.

    torch.int32 keys sort as signed, torch.uint32 as unsigned (``signed`` overrides).  out may be keys.
    """
    _reachable(keys, "keys")
    if keys.dtype not in _W4:
        raise TypeError("radix_sort takes 32-bit keys")
    if signed is None:
        signed = keys.dtype == torch.int32
    n = keys.numel()
    if out is None:
        out = _like(keys)
    _reachable(out, "out")
    if out.dtype not in _W4 or out.numel() < n:
        raise ValueError("out must hold n 32-bit keys")
    L = native.load()
    ws = _workspace(L.dialsort_radix_workspace_size(n), _device(keys), ws)
    fn = L.dialsort_radix_sort_i32 if signed else L.dialsort_radix_sort_u32
    _check(fn(keys.data_ptr(), n, out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "dialsort_radix_sort")
    return out


def _queries(q: torch.Tensor, name: str) -> torch.Tensor:
    _reachable(q, name)
    if q.dtype not in _W4:
        raise TypeError(f"{name} must hold 32-bit keys")
    return q


def frequency(H: torch.Tensor, U: int, q: torch.Tensor, out: torch.Tensor | None = None, *,
              stream=None) -> torch.Tensor:
    """frequency(k) = H[k] for every query key k (0 outside [0, U)), as int32 storage of uint32."""
    _reachable(H, "H")
    _queries(q, "q")
    out = torch.empty(q.numel(), dtype=torch.int32, device=_device(q)) if out is None else _reachable(out, "out")
    _check(native.load().dialsort_frequency(H.data_ptr(), U, q.data_ptr(), q.numel(), out.data_ptr(),
                                            _stream(stream)), "dialsort_frequency")
    return out


def presence(H: torch.Tensor, U: int, q: torch.Tensor, out: torch.Tensor | None = None, *,
             stream=None) -> torch.Tensor:
    """presence(k) = 1 if H[k] > 0 else 0, as uint8."""
    _reachable(H, "H")
    _queries(q, "q")
    out = torch.empty(q.numel(), dtype=torch.uint8, device=_device(q)) if out is None else _reachable(out, "out")
    _check(native.load().dialsort_presence(H.data_ptr(), U, q.data_ptr(), q.numel(), out.data_ptr(),
                                           _stream(stream)), "dialsort_presence")
    return out


def range_count(H: torch.Tensor, U: int, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None, *,
                stream=None) -> torch.Tensor:
    """range-count(a, b) = sum of H[k] for a <= k <= b (inclusive, clipped to [0, U)); uint32 in int32."""
    _reachable(H, "H")
    _queries(a, "a")
    _queries(b, "b")
    if a.numel() != b.numel():
        raise ValueError("a and b must have the same length")
    out = torch.empty(a.numel(), dtype=torch.int32, device=_device(a)) if out is None else _reachable(out, "out")
    _check(native.load().dialsort_range_count(H.data_ptr(), U, a.data_ptr(), b.data_ptr(), a.numel(),
                                              out.data_ptr(), _stream(stream)), "dialsort_range_count")
    return out


def pageable_host_access() -> bool:
    """True if the kernels may read and write plain (pageable) host memory on the current device."""
    return native.load().dialsort_pageable_host_access() == 1


def stream_status(stream=None, sync: bool = True) -> int:
    """Read and clear the device error word (OK, ERR_KEY_RANGE, ERR_TIMEOUT, ERR_OVERFLOW)."""
    return native.load().dialsort_stream_status(_stream(stream), 1 if sync else 0)


def plan_histogram(n: int, U: int, width: int = 4, skew_hint: int = 0, **forced) -> dict:
    """The autotuner's launch choices for step 1, as a dict."""
    c = _config(forced) or native.dialsort_hist_config_t()
    _check(native.load().dialsort_plan_histogram(n, U, width, skew_hint, ctypes.byref(c)), "plan_histogram")
    d = {f: getattr(c, f) for f, _ in c._fields_}
    d["regime_name"] = REGIME_NAMES[d["regime"]]
    return d


class Batch:
    """A planned batch of independent instances (dialsort_batch_*), run by one persistent launch.

    keys: list of CUDA tensors (32- or 16-bit keys); U: list of universe sizes; H: list of int32
    tensors (allocated when None); out: list of output tensors (allocated when sort and None).
    """

    def __init__(self, keys, U, H=None, out=None, *, sort: bool = True, skew=None, regime=None):
        L = native.load()
        n = len(keys)
        self.keys = list(keys)
        self.U = [int(u) for u in U]
        self.sort = bool(sort)
        dev = keys[0].device if n else torch.device("cuda")
        self.H = list(H) if H is not None else [torch.empty(u, dtype=torch.int32, device=dev) for u in self.U]
        if self.sort:
            self.out = list(out) if out is not None else [torch.empty_like(k) for k in self.keys]
        else:
            self.out = [None] * n
        arr = (native.dialsort_instance_t * max(n, 1))()
        for i in range(n):
            _cuda(self.keys[i], "keys")
            _cuda(self.H[i], "H")
            arr[i].keys = self.keys[i].data_ptr()
            arr[i].H = self.H[i].data_ptr()
            arr[i].out = self.out[i].data_ptr() if self.out[i] is not None else None
            arr[i].n = self.keys[i].numel()
            arr[i].U = self.U[i]
            arr[i].key_bytes = _width(self.keys[i])
            if regime is not None:  # one name / number for all, or one per instance
                r = regime if isinstance(regime, (str, int)) else regime[i]
                arr[i].regime = REGIMES[r] if isinstance(r, str) else int(r)
            if skew is not None and skew != "probe":
                arr[i].skew = SKEW_CLASSES[skew[i]] if isinstance(skew[i], str) else int(skew[i])
        if skew == "probe" and n:  # one probe launch for every instance
            _check(L.dialsort_probe_skew_batched(arr, n, _stream(None)), "probe_skew_batched")
        self.skew = [arr[i].skew for i in range(n)]
        self._handle = ctypes.c_void_p()
        _check(L.dialsort_batch_create(arr, n, 1 if self.sort else 0, ctypes.byref(self._handle)), "batch_create")
        self.ws = torch.empty(max(L.dialsort_batch_workspace_size(self._handle), 256), dtype=torch.uint8,
                              device=dev)

    def launch(self, stream=None):
        _check(native.load().dialsort_batch_launch(self._handle, self.ws.data_ptr(), self.ws.numel(), _stream(stream)),
               "batch_launch")
        return self

    def describe(self, i: int) -> dict:
        c = native.dialsort_hist_config_t()
        items = (ctypes.c_uint32 * 4)()
        _check(native.load().dialsort_batch_describe(self._handle, i, ctypes.byref(c), items), "batch_describe")
        return {"regime_name": REGIME_NAMES[c.regime], "replicas": c.replicas, "items": list(items),
                "crn": {1: "on", 2: "off", 3: "adaptive"}[c.crn], "skew": SKEW_NAMES[self.skew[i]]}

    def close(self):
        if self._handle:
            torch.cuda.synchronize()
            native.load().dialsort_batch_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched(keys, U, *, sort: bool = True, stream=None):
    """One-shot batched run; returns (H list, out list)."""
    b = Batch(keys, U, sort=sort)
    b.launch(stream)
    torch.cuda.current_stream().synchronize()
    b.close()
    return b.H, b.out


class _CudaArray:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, n: int, dtype: torch.dtype) -> torch.Tensor:
    """A zero-copy tensor over n elements of device memory at ptr (memory owned elsewhere)."""
    typestr = {torch.int32: "<i4", torch.int16: "<i2", torch.uint8: "|u1"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")


class Server:
    """The served form (dialsort_server_*): continuous batching under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int = 1 << 30, max_slots: int = 64, idle_timeout_ns: int = 0):
        cfg = native.dialsort_server_cfg_t(hbm_budget_bytes, max_slots, 0, idle_timeout_ns)
        self._h = ctypes.c_void_p()
        _check(native.load().dialsort_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "server_create")
        self._keep = {}

    def submit(self, keys: torch.Tensor, U: int, kind: str = "sort", skew=0) -> int:
        _cuda(keys, "keys")
        sk = SKEW_CLASSES[skew] if isinstance(skew, str) else int(skew)
        r = native.dialsort_request_t(keys.data_ptr(), keys.numel(), U, _width(keys), 1 if kind == "sort" else 0, sk)
        t = ctypes.c_uint64()
        _check(native.load().dialsort_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "server_submit")
        self._keep[t.value] = (keys, U, kind)  # keys must stay alive until the request finishes
        return t.value

    def _result(self, ticket, res):
        keys, U, kind = self._keep[ticket]
        w = _width(keys)
        H = device_view(res.H, U, torch.int32)
        out = device_view(res.out, keys.numel(), torch.int32 if w == 4 else torch.int16) if kind == "sort" else None
        return {"H": H, "out": out, "status": res.status, "submit_ns": res.submit_ns, "admit_ns": res.admit_ns,
                "done_ns": res.done_ns}

    def poll(self, ticket: int):
        res = native.dialsort_result_t()
        st = native.load().dialsort_server_poll(self._h, ticket, ctypes.byref(res))
        if st == ERR_BUSY:
            return None
        _check(st, "server_poll")
        return self._result(ticket, res)

    def wait(self, ticket: int, timeout_s: float = 30.0):
        res = native.dialsort_result_t()
        _check(native.load().dialsort_server_wait(self._h, ticket, int(timeout_s * 1e9), ctypes.byref(res)),
               "server_wait")
        return self._result(ticket, res)

    def release(self, ticket: int):
        _check(native.load().dialsort_server_release(self._h, ticket), "server_release")
        self._keep.pop(ticket, None)

    def close(self):
        if self._h:
            native.load().dialsort_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay(entries, *, use_server: bool, hbm_budget_bytes: int = 64 << 30, max_slots: int = 64,
           idle_timeout_ns: int = 0):
    """Replay a timed request trace (list of (keys tensor, U, kind, arrival_ns)); returns (results, wall_ns)."""
    import numpy as np

    n = len(entries)
    arr = (native.dialsort_trace_entry_t * max(n, 1))()
    for i, (keys, U, kind, t) in enumerate(entries):
        arr[i].keys = keys.data_ptr()
        arr[i].n = keys.numel()
        arr[i].U = U
        arr[i].key_bytes = _width(keys)
        arr[i].kind = 1 if kind == "sort" else 0
        arr[i].arrival_ns = int(t)
    res = (native.dialsort_trace_result_t * max(n, 1))()
    cfg = native.dialsort_server_cfg_t(hbm_budget_bytes, max_slots, 0, idle_timeout_ns)
    wall = ctypes.c_uint64()
    _check(native.load().dialsort_replay(arr, n, 1 if use_server else 0, ctypes.byref(cfg), res, ctypes.byref(wall)),
           "replay")
    out = np.zeros(n, dtype=[("arrival_ns", "u8"), ("done_ns", "u8"), ("status", "u4")])
    for i in range(n):
        out[i] = (res[i].arrival_ns, res[i].done_ns, res[i].status)
    return out, wall.value

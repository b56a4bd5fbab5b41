"""Python binding for libmegopolis.so (Megopolis / Metropolis resampling on
GB300).  Argument marshalling only: every step runs in the library's CUDA
kernels.  torch supplies device memory and the current CUDA stream.

The functions carry the C ABI's names (``mego_resample``,
``mego_resample_gather``, ``mego_compute_B``, ``mego_compute_B_noalloc``,
``mego_likelihood_B``,
``mego_resample_host``, ``mego_sync_status``, ``mego_probe_read``); they take
torch tensors instead of raw pointers and raise ``MegoError`` on a non-OK
status.  ``resample`` is a convenience wrapper that allocates the output.

If the shared library has not been built (``__graft_entry__.build()`` or
``python -m paper_2109_13504_gb300.build``) every call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmegopolis.so")

MEGO_OK = 0
MEGO_EINVAL = 1
MEGO_ENOMEM = 2
MEGO_ECUDA = 3
MEGO_ETIMEOUT = 4
MEGO_EWEIGHTS = 5

MEGOPOLIS = 0
METROPOLIS = 1
METROPOLIS_C1 = 2
METROPOLIS_C2 = 3

LAYOUT_SOA = 0
LAYOUT_AOS4 = 1

PATH_AUTO = 0
PATH_GLOBAL = 1
PATH_SMEM = 2
PATH_TMA = 3

N_MAX = 1 << 30
B_MAX = 1 << 24


class MegoError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


class LaunchCfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ppt", ctypes.c_int32),
                ("path", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class Filter(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("anc", ctypes.c_void_p), ("x_in", ctypes.c_void_p),
                ("x_out", ctypes.c_void_p), ("ld", ctypes.c_int64), ("n", ctypes.c_int32),
                ("B", ctypes.c_int32), ("stream_id", ctypes.c_uint32), ("dim", ctypes.c_int32),
                ("w_host", ctypes.c_void_p)]


class BatchHandle(ctypes.Structure):
    _fields_ = [("d_plan", ctypes.c_void_p), ("plan_bytes", ctypes.c_size_t),
                ("count", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("total_items", ctypes.c_uint64),
                ("total_chunks", ctypes.c_uint64), ("d_B", ctypes.c_void_p),
                ("d_status", ctypes.c_void_p), ("d_q", ctypes.c_void_p),
                ("cfg", LaunchCfg), ("grid", ctypes.c_int32), ("graph_exec", ctypes.c_void_p),
                ("graph_kernels", ctypes.c_int32), ("smem_max_n", ctypes.c_int32),
                ("smem_filters", ctypes.c_int32), ("smem_bytes", ctypes.c_size_t),
                ("h_filters", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("h_w", ctypes.c_void_p), ("h_x", ctypes.c_void_p),
                ("h_anc", ctypes.c_void_p), ("h_x_out", ctypes.c_void_p), ("n", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("n", ctypes.c_int32),
                ("latency_ns", ctypes.c_int64), ("B", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("d_arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("seed", ctypes.c_uint64), ("eps", ctypes.c_double), ("variant", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ppt", ctypes.c_int32), ("poll_us", ctypes.c_int32),
                ("with_state", ctypes.c_int32), ("host_copies", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("max_batch", ctypes.c_uint64),
                ("peak_arena_bytes", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("inflight", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libmegopolis.so is not built (%s); run __graft_entry__.build() -- "
            "there is no CPU fallback" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t)
    ci = ctypes.c_int
    sigs = {
        "mego_abi_version": ([], ci),
        "mego_status_string": ([ci], ctypes.c_char_p),
        "mego_launch_count": ([], u64),
        "mego_workspace_bytes": ([i32], sz),
        "mego_resample": ([vp, i32, i32, u64, u32, ci, vp, vp], ci),
        "mego_resample_gather": ([vp, i32, i32, vp, u64, u32, ci, u32, vp, vp, i32,
                                  ctypes.c_int64, ci, vp, ctypes.POINTER(LaunchCfg), vp],
                                 ci),
        "mego_compute_B": ([vp, i32, f64, i32, vp, vp, vp, vp, sz, vp], ci),
        "mego_compute_B_noalloc": ([vp, i32, f64, i32, vp, vp, vp, vp], ci),
        "mego_likelihood_B": ([vp, i32, ctypes.c_float, f64, i32, vp, vp, vp, vp, vp,
                               sz, vp], ci),
        "mego_resample_host": ([vp, i32, i32, f64, u64, u32, ci, vp, vp, vp, vp, vp, vp,
                                sz, vp], ci),
        "mego_sync_status": ([vp, vp, f64, vp], ci),
        "mego_probe_read": ([vp, sz, i32, vp, vp], ci),
        "mego_device_fault": ([vp], ci),
        "mego_set_stage_poll_budget": ([ctypes.c_int64], ci),
        "mego_batch_plan_bytes": ([ctypes.POINTER(Filter), i32], sz),
        "mego_batch_plan": ([ctypes.POINTER(Filter), i32, ci, ci, u64, vp, sz,
                             ctypes.POINTER(BatchHandle), vp], ci),
        "mego_batch_bound": ([ctypes.POINTER(BatchHandle), f64, i32, vp], ci),
        "mego_batch_resample": ([ctypes.POINTER(BatchHandle), vp], ci),
        "mego_batch_set_shape": ([ctypes.POINTER(BatchHandle), i32, i32], ci),
        "mego_batch_set_smem": ([ctypes.POINTER(BatchHandle), i32, vp], ci),
        "mego_batch_autotune": ([ctypes.POINTER(BatchHandle), i32,
                                 ctypes.POINTER(ctypes.c_float), vp], ci),
        "mego_batch_graph": ([ctypes.POINTER(BatchHandle), f64, i32, vp], ci),
        "mego_batch_launch_graph": ([ctypes.POINTER(BatchHandle), vp], ci),
        "mego_batch_destroy": ([ctypes.POINTER(BatchHandle)], ci),
        "mego_server_create": ([ctypes.POINTER(ServerCfg), ctypes.POINTER(ctypes.c_void_p)], ci),
        "mego_server_submit": ([vp, ctypes.POINTER(Request)], ci),
        "mego_server_poll": ([vp, ctypes.POINTER(Completion), i32], i32),
        "mego_server_drain": ([vp, f64], ci),
        "mego_server_stats": ([vp, ctypes.POINTER(ServerStats)], ci),
        "mego_server_destroy": ([vp], ci),
        "mego_server_replay": ([vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double),
                                i32, f64], ci),
        "mego_sir_predict_update": ([vp, vp, i32, ctypes.c_float, ctypes.c_float, vp, vp, vp],
                                    ci),
        "mego_mean_workspace_bytes": ([], sz),
        "mego_mean": ([vp, i32, vp, vp, sz, vp], ci),
        "mego_autotune": ([vp, i32, i32, ci, u32, vp, vp, i32, ctypes.c_int64, ci, vp, i32,
                           ctypes.POINTER(LaunchCfg), ctypes.POINTER(ctypes.c_float), vp], ci),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def loaded_library_path() -> str:
    _load()
    return LIB_PATH


def status_string(status: int) -> str:
    try:
        return _load().mego_status_string(int(status)).decode()
    except Exception:
        return "status"


def abi_version() -> int:
    return int(_load().mego_abi_version())


def launch_count() -> int:
    return int(_load().mego_launch_count())


def workspace_bytes(n: int) -> int:
    return int(_load().mego_workspace_bytes(int(n)))


def _check(status: int, what: str) -> None:
    if status != MEGO_OK:
        raise MegoError(status, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str, numel: Optional[int] = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), numel))
    return t.data_ptr()


def _anc_ptr(t: torch.Tensor, numel: int) -> int:
    """Ancestor output of a batch filter: a CUDA tensor, or a page-locked host
    tensor that the resample writes directly (over the CPU-GPU link)."""
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned() or t.dtype != torch.int32 or not t.is_contiguous() \
                or t.numel() < numel:
            raise TypeError("a host anc must be a contiguous page-locked int32 tensor of n "
                            "elements")
        return t.data_ptr()
    return _dev(t, torch.int32, "anc", numel)


def _cfg(cfg) -> Optional[LaunchCfg]:
    if cfg is None:
        return None
    if isinstance(cfg, dict):
        cfg = LaunchCfg(**{k: int(v) for k, v in cfg.items()})
    return cfg


# --------------------------------------------------------------------------
# C-ABI wrappers


def mego_resample(w: torch.Tensor, B: int, seed: int, stream_id: int = 0,
                  variant: int = MEGOPOLIS, anc: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    n = w.numel()
    if anc is None:
        anc = torch.empty(n, dtype=torch.int32, device=w.device)
    st = _load().mego_resample(_dev(w, torch.float32, "w"), n, int(B), int(seed),
                               int(stream_id), int(variant),
                               _dev(anc, torch.int32, "anc", n), _stream(stream))
    _check(st, "mego_resample")
    return anc


def mego_resample_gather(w: torch.Tensor, B: int = 0, B_dev: Optional[torch.Tensor] = None,
                         seed: int = 0, stream_id: int = 0, variant: int = MEGOPOLIS,
                         psize_bytes: int = 0, x_in: Optional[torch.Tensor] = None,
                         x_out: Optional[torch.Tensor] = None, layout: int = LAYOUT_SOA,
                         anc: Optional[torch.Tensor] = None, cfg=None, stream=None):
    """Resample and (optionally) gather state.  SoA state is [dim, n] (row
    stride = its second dimension); AoS4 state is [n, 4]."""
    n = w.numel()
    dim, ld = 0, 0
    px_in = px_out = None
    if x_in is not None or x_out is not None:
        if x_in is None or x_out is None:
            raise ValueError("x_in and x_out go together")
        if layout == LAYOUT_SOA:
            if x_in.dim() != 2 or x_in.shape[1] < n or x_out.shape != x_in.shape:
                raise ValueError("SoA state must be [dim, >= n] and x_out the same shape")
            dim, ld = x_in.shape[0], x_in.shape[1]
        else:
            if x_in.shape != (n, 4) or x_out.shape != (n, 4):
                raise ValueError("AoS4 state must be [n, 4]")
            dim, ld = 4, 4
        px_in = _dev(x_in, torch.float32, "x_in")
        px_out = _dev(x_out, torch.float32, "x_out")
    panc = _dev(anc, torch.int32, "anc", n) if anc is not None else None
    pB = _dev(B_dev, torch.int32, "B_dev", 1) if B_dev is not None else None
    c = _cfg(cfg)
    st = _load().mego_resample_gather(
        _dev(w, torch.float32, "w"), n, int(B), pB, int(seed), int(stream_id), int(variant),
        int(psize_bytes), px_in, px_out, int(dim), int(ld), int(layout), panc,
        ctypes.byref(c) if c is not None else None, _stream(stream))
    _check(st, "mego_resample_gather")
    return anc, x_out


def _scalars(device, B_dev, status, q):
    if B_dev is None:
        B_dev = torch.empty(1, dtype=torch.int32, device=device)
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=device)
    if q is None:
        q = torch.empty(1, dtype=torch.float64, device=device)
    return B_dev, status, q


def _workspace(n, device, ws):
    need = workspace_bytes(n)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=device)
    return ws, need


def mego_compute_B(w: torch.Tensor, eps: float = 0.01, b_max: int = B_MAX,
                   B_dev=None, status=None, q=None, ws=None, stream=None):
    """Eq. 3 on the device.  Returns (B_dev, status, q) device tensors."""
    n = w.numel()
    B_dev, status, q = _scalars(w.device, B_dev, status, q)
    ws, _ = _workspace(n, w.device, ws)
    st = _load().mego_compute_B(_dev(w, torch.float32, "w"), n, float(eps), int(b_max),
                                _dev(B_dev, torch.int32, "B_dev", 1),
                                _dev(status, torch.int32, "status", 1),
                                _dev(q, torch.float64, "q", 1),
                                _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(st, "mego_compute_B")
    return B_dev, status, q


def mego_compute_B_noalloc(w: torch.Tensor, eps: float, B_dev: torch.Tensor,
                           status: torch.Tensor, q: Optional[torch.Tensor] = None,
                           b_max: int = B_MAX, stream=None):
    """Eq. 3 on the device without a workspace: for callers that cannot
    allocate device memory.  The output tensors are the caller's (nothing is
    allocated here); the library keeps the reduction's partials in a fixed
    array of its own.  Calls that overlap on the GPU share that array and
    race, so issue them on one stream.  Returns (B_dev, status, q)."""
    n = w.numel()
    pq = _dev(q, torch.float64, "q", 1) if q is not None else None
    st = _load().mego_compute_B_noalloc(_dev(w, torch.float32, "w"), n, float(eps),
                                        int(b_max), _dev(B_dev, torch.int32, "B_dev", 1),
                                        _dev(status, torch.int32, "status", 1), pq,
                                        _stream(stream))
    _check(st, "mego_compute_B_noalloc")
    return B_dev, status, q


def mego_likelihood_B(x0: torch.Tensor, y: float, eps: float = 0.01, b_max: int = B_MAX,
                      w: Optional[torch.Tensor] = None, B_dev=None, status=None, q=None,
                      ws=None, stream=None):
    """w = exp(-(x0 - y)^2/2) and Eq. 3.  Returns (w, B_dev, status, q)."""
    n = x0.numel()
    if w is None:
        w = torch.empty(n, dtype=torch.float32, device=x0.device)
    B_dev, status, q = _scalars(x0.device, B_dev, status, q)
    ws, _ = _workspace(n, x0.device, ws)
    st = _load().mego_likelihood_B(_dev(x0, torch.float32, "x0"), n, ctypes.c_float(y),
                                   float(eps), int(b_max), _dev(w, torch.float32, "w", n),
                                   _dev(B_dev, torch.int32, "B_dev", 1),
                                   _dev(status, torch.int32, "status", 1),
                                   _dev(q, torch.float64, "q", 1),
                                   _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(st, "mego_likelihood_B")
    return w, B_dev, status, q


def mego_resample_host(h_w: torch.Tensor, B: int, eps: float, seed: int, stream_id: int,
                       variant: int, h_anc: torch.Tensor, d_w: torch.Tensor,
                       d_anc: torch.Tensor, d_scalars: torch.Tensor, ws: torch.Tensor,
                       stream=None) -> int:
    """End-to-end call on host tensors (pinned for full speed).  Returns B."""
    n = h_w.numel()
    if h_w.is_cuda or h_anc.is_cuda:
        raise TypeError("h_w and h_anc must be host tensors")
    if h_w.dtype != torch.float32 or h_anc.dtype != torch.int32:
        raise TypeError("h_w float32, h_anc int32")
    if not (h_w.is_contiguous() and h_anc.is_contiguous()) or h_anc.numel() < n:
        raise ValueError("host tensors must be contiguous and large enough")
    hB = ctypes.c_int32(-1)
    st = _load().mego_resample_host(
        h_w.data_ptr(), n, int(B), float(eps), int(seed), int(stream_id), int(variant),
        h_anc.data_ptr(), ctypes.addressof(hB), _dev(d_w, torch.float32, "d_w", n),
        _dev(d_anc, torch.int32, "d_anc", n), _dev(d_scalars, torch.uint8, "d_scalars", 32),
        _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(st, "mego_resample_host")
    return int(hB.value)


def mego_sync_status(status: torch.Tensor, timeout_s: float = 10.0, stream=None) -> int:
    h = ctypes.c_int32(-1)
    st = _load().mego_sync_status(_dev(status, torch.int32, "status", 1), _stream(stream),
                                  float(timeout_s), ctypes.addressof(h))
    _check(st, "mego_sync_status")
    return int(h.value)


def mego_autotune(w: torch.Tensor, B: int, variant: int = MEGOPOLIS, psize_bytes: int = 0,
                  x_in: Optional[torch.Tensor] = None, x_out: Optional[torch.Tensor] = None,
                  layout: int = LAYOUT_SOA, anc: Optional[torch.Tensor] = None, reps: int = 3,
                  stream=None):
    """Time every launch shape and cache the fastest for this size/B bucket.
    Returns (shape dict, milliseconds)."""
    n = w.numel()
    dim, ld = 0, 0
    px_in = px_out = None
    if x_in is not None:
        if layout == LAYOUT_SOA:
            dim, ld = x_in.shape[0], x_in.shape[1]
        else:
            dim, ld = 4, 4
        px_in = _dev(x_in, torch.float32, "x_in")
        px_out = _dev(x_out, torch.float32, "x_out")
    if anc is None and x_in is None:
        anc = torch.empty(n, dtype=torch.int32, device=w.device)
    panc = _dev(anc, torch.int32, "anc", n) if anc is not None else None
    best = LaunchCfg()
    ms = ctypes.c_float()
    st = _load().mego_autotune(_dev(w, torch.float32, "w"), n, int(B), int(variant),
                               int(psize_bytes), px_in, px_out, int(dim), int(ld), int(layout),
                               panc, int(reps), ctypes.byref(best), ctypes.byref(ms),
                               _stream(stream))
    _check(st, "mego_autotune")
    return ({"threads": best.threads, "ppt": best.ppt, "path": best.path,
             "ctas_per_sm": best.ctas_per_sm}, float(ms.value))


def mego_device_fault() -> int:
    """OR of the faults recorded by the resample kernels since the last call."""
    h = ctypes.c_int32(-1)
    _check(_load().mego_device_fault(ctypes.addressof(h)), "mego_device_fault")
    return int(h.value)


def mego_set_stage_poll_budget(polls: int) -> None:
    """Polls of the shared-memory staging wait before it reports a fault
    (diagnostics; polls < 0 restores the default)."""
    _check(_load().mego_set_stage_poll_budget(int(polls)), "mego_set_stage_poll_budget")


def mego_probe_read(buf: torch.Tensor, reps: int, sink: torch.Tensor, stream=None) -> None:
    if not buf.is_cuda or not buf.is_contiguous():
        raise TypeError("buf must be a contiguous CUDA tensor")
    st = _load().mego_probe_read(buf.data_ptr(), buf.numel() * buf.element_size(), int(reps),
                                 _dev(sink, torch.float32, "sink"), _stream(stream))
    _check(st, "mego_probe_read")


# --------------------------------------------------------------------------
# Convenience


def resample(w: torch.Tensor, B: Optional[int] = None, eps: float = 0.01, seed: int = 0,
             stream_id: int = 0, variant: int = MEGOPOLIS, psize_bytes: int = 0,
             cfg=None, stream=None) -> torch.Tensor:
    """Ancestors as an int32 CUDA tensor.  B=None computes B from eps on the
    device (Eq. 3) without a host synchronisation."""
    n = w.numel()
    anc = torch.empty(n, dtype=torch.int32, device=w.device)
    if B is None:
        B_dev, _, _ = mego_compute_B(w, eps, stream=stream)
        mego_resample_gather(w, 0, B_dev, seed, stream_id, variant, psize_bytes, anc=anc,
                             cfg=cfg, stream=stream)
    else:
        mego_resample_gather(w, int(B), None, seed, stream_id, variant, psize_bytes, anc=anc,
                             cfg=cfg, stream=stream)
    return anc


# --------------------------------------------------------------------------
# Batched resampling


class Batch:
    """Many independent filters resampled by one persistent launch.

    filters: list of dicts with keys w (CUDA float32 [n]), anc (CUDA int32
    [n], optional when gathering), x_in/x_out (optional state), B (int, or
    -1 to use the batch bound), stream_id (int).  The tensors must stay alive
    while the batch is used; the Batch keeps references to them.
    """

    def __init__(self, filters, variant: int = MEGOPOLIS, layout: int = LAYOUT_SOA,
                 seed: int = 0, stream=None):
        lib = _load()
        self._keep = filters
        self.count = len(filters)
        arr = (Filter * self.count)()
        dev = None
        for f, d in enumerate(filters):
            w = d["w"]
            dev = w.device
            n = w.numel()
            x_in, x_out = d.get("x_in"), d.get("x_out")
            dim, ld = 0, 0
            if x_in is not None:
                if layout == LAYOUT_SOA:
                    dim, ld = x_in.shape[0], x_in.shape[1]
                else:
                    dim, ld = 4, 4
            anc = d.get("anc")
            w_host = d.get("w_host")
            if w_host is not None and (w_host.is_cuda or not w_host.is_pinned()
                                       or w_host.dtype != torch.float32
                                       or not w_host.is_contiguous() or w_host.numel() != n):
                raise TypeError("w_host must be a contiguous page-locked float32 host tensor "
                                "of n elements")
            arr[f] = Filter(_dev(w, torch.float32, "w"),
                            _anc_ptr(anc, n) if anc is not None else None,
                            _dev(x_in, torch.float32, "x_in") if x_in is not None else None,
                            _dev(x_out, torch.float32, "x_out") if x_out is not None else None,
                            int(ld), int(n), int(d.get("B", -1)), int(d.get("stream_id", f)),
                            int(dim), w_host.data_ptr() if w_host is not None else None)
        self._filters = arr
        nbytes = int(lib.mego_batch_plan_bytes(arr, self.count))
        if nbytes == 0:
            raise MegoError(MEGO_EINVAL, "mego_batch_plan_bytes")
        self.plan = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.handle = BatchHandle()
        st = lib.mego_batch_plan(arr, self.count, int(variant), int(layout), int(seed),
                                 self.plan.data_ptr(), nbytes, ctypes.byref(self.handle),
                                 _stream(stream))
        _check(st, "mego_batch_plan")

    def _view(self, ptr, dtype, numel):
        off = int(ptr) - self.plan.data_ptr()
        esz = torch.empty(0, dtype=dtype).element_size()
        return self.plan[off:off + esz * numel].view(dtype)

    @property
    def B(self) -> torch.Tensor:
        return self._view(self.handle.d_B, torch.int32, self.count)

    @property
    def status(self) -> torch.Tensor:
        return self._view(self.handle.d_status, torch.int32, self.count)

    @property
    def q(self) -> torch.Tensor:
        return self._view(self.handle.d_q, torch.float64, self.count)

    def bound(self, eps: float = 0.01, b_max: int = B_MAX, stream=None):
        _check(_load().mego_batch_bound(ctypes.byref(self.handle), float(eps), int(b_max),
                                        _stream(stream)), "mego_batch_bound")

    def resample(self, stream=None):
        _check(_load().mego_batch_resample(ctypes.byref(self.handle), _stream(stream)),
               "mego_batch_resample")

    def set_shape(self, threads: int, ppt: int):
        _check(_load().mego_batch_set_shape(ctypes.byref(self.handle), int(threads), int(ppt)),
               "mego_batch_set_shape")

    def set_smem(self, smem_max_n: int, stream=None):
        """Filters of at most smem_max_n weights: one CTA each, from shared
        memory (0: none)."""
        _check(_load().mego_batch_set_smem(ctypes.byref(self.handle), int(smem_max_n),
                                           _stream(stream)), "mego_batch_set_smem")

    def autotune(self, reps: int = 3, stream=None) -> float:
        ms = ctypes.c_float()
        _check(_load().mego_batch_autotune(ctypes.byref(self.handle), int(reps),
                                           ctypes.byref(ms), _stream(stream)),
               "mego_batch_autotune")
        return float(ms.value)

    @property
    def shape(self):
        return {"threads": self.handle.cfg.threads, "ppt": self.handle.cfg.ppt,
                "grid": self.handle.grid, "smem_max_n": self.handle.smem_max_n,
                "smem_filters": self.handle.smem_filters}

    def capture(self, eps: float = 0.01, b_max: int = B_MAX, stream=None):
        """Capture [bound if eps > 0] + resample into a CUDA graph (needs a
        non-default stream)."""
        _check(_load().mego_batch_graph(ctypes.byref(self.handle), float(eps), int(b_max),
                                        _stream(stream)), "mego_batch_graph")

    def replay(self, stream=None):
        _check(_load().mego_batch_launch_graph(ctypes.byref(self.handle), _stream(stream)),
               "mego_batch_launch_graph")

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.mego_batch_destroy(ctypes.byref(self.handle))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Serving


def _host_ptr(t: Optional[torch.Tensor], dtype, name: str):
    if t is None:
        return None
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous host tensor of %s" % (name, dtype))
    return t.data_ptr()


class Server:
    """Continuous-batching resample server over a device arena (the memory
    budget).  Requests carry host tensors: w [n] float32, optionally x
    [n, 4] float32 state, and outputs anc [n] int32 / x_out [n, 4]."""

    def __init__(self, arena_bytes: int, seed: int = 0, eps: float = 0.01,
                 variant: int = MEGOPOLIS, max_batch: int = 256, streams: int = 2,
                 with_state: bool = True, threads: int = 0, ppt: int = 0, poll_us: int = 0,
                 host_copies: int = 0, device=None):
        lib = _load()
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        cfg = ServerCfg(self.arena.data_ptr(), int(arena_bytes), int(seed), float(eps),
                        int(variant), int(max_batch), int(streams), int(threads), int(ppt),
                        int(poll_us), 1 if with_state else 0, int(host_copies))
        self._h = ctypes.c_void_p()
        _check(lib.mego_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
               "mego_server_create")
        self._keep = {}
        self._poll_buf = {}

    def _req(self, rid, w, x=None, anc=None, x_out=None):
        return Request(int(rid), _host_ptr(w, torch.float32, "w"),
                       _host_ptr(x, torch.float32, "x"), _host_ptr(anc, torch.int32, "anc"),
                       _host_ptr(x_out, torch.float32, "x_out"), int(w.numel()))

    def submit(self, rid: int, w, x=None, anc=None, x_out=None):
        r = self._req(rid, w, x, anc, x_out)
        self._keep[int(rid)] = (w, x, anc, x_out)
        _check(_load().mego_server_submit(self._h, ctypes.byref(r)), "mego_server_submit")

    def poll(self, max_out: int = 4096):
        """Completed requests as (id, status, n, latency_ns, B) tuples."""
        buf = self._poll_buf.get(max_out)
        if buf is None:
            buf = self._poll_buf[max_out] = (Completion * max_out)()
        k = _load().mego_server_poll(self._h, buf, int(max_out))
        out = [(c.id, c.status, c.n, c.latency_ns, c.B) for c in buf[:k]]
        for c in out:
            self._keep.pop(int(c[0]), None)
        return out

    def drain(self, timeout_s: float = 60.0):
        _check(_load().mego_server_drain(self._h, float(timeout_s)), "mego_server_drain")

    def replay(self, requests, t_arrival, timeout_s: float = 120.0):
        """requests: list of (id, w, x, anc, x_out) host tensors."""
        arr = (Request * len(requests))(*[self._req(*r) for r in requests])
        t = (ctypes.c_double * len(requests))(*[float(v) for v in t_arrival])
        _check(_load().mego_server_replay(self._h, arr, t, len(requests), float(timeout_s)),
               "mego_server_replay")

    def stats(self):
        st = ServerStats()
        _check(_load().mego_server_stats(self._h, ctypes.byref(st)), "mego_server_stats")
        return {"batches": st.batches, "max_batch": st.max_batch,
                "peak_arena_bytes": st.peak_arena_bytes, "queued": st.queued,
                "inflight": st.inflight}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _load().mego_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# SIR filter stages (Algorithm 6)


def mego_sir_predict_update(x: torch.Tensor, v: torch.Tensor, drift: float, z: float,
                            x_pred: Optional[torch.Tensor] = None,
                            w: Optional[torch.Tensor] = None, stream=None):
    n = x.numel()
    if x_pred is None:
        x_pred = torch.empty_like(x)
    if w is None:
        w = torch.empty_like(x)
    st = _load().mego_sir_predict_update(_dev(x, torch.float32, "x"), _dev(v, torch.float32, "v", n),
                                         n, ctypes.c_float(drift), ctypes.c_float(z),
                                         _dev(x_pred, torch.float32, "x_pred", n),
                                         _dev(w, torch.float32, "w", n), _stream(stream))
    _check(st, "mego_sir_predict_update")
    return x_pred, w


def mego_mean(x: torch.Tensor, out: Optional[torch.Tensor] = None,
              ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    n = x.numel()
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    need = int(_load().mego_mean_workspace_bytes())
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=x.device)
    st = _load().mego_mean(_dev(x, torch.float32, "x"), n, _dev(out, torch.float64, "out", 1),
                           _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream))
    _check(st, "mego_mean")
    return out

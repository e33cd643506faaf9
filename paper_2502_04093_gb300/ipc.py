"""Thin Python binding of libipcomp's C ABI (include/ipc.h).

Argument marshalling only: every step of compression and retrieval runs in
the library's CUDA kernels. Function names are the C names. Device buffers
are torch CUDA tensors (PyTorch provides device memory and streams); the
stream defaults to torch's current stream.

The library must be built (``paper_2502_04093_gb300.build.build()``); this
module raises ImportError-derived errors if it is missing - there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libipcomp.so")
# IPC_BOUNDS_CHECK=1 loads the bounds-checking build instead (device-side
# index checks on the level kernels' global accesses; see ipc_debug_bounds)
BOUNDS_LIB_PATH = os.path.join(HERE, "libipcomp_bounds.so")

IPC_OK, IPC_EINVAL, IPC_EBOUND, IPC_EBUDGET = 0, -1, -2, -3
IPC_ENOMEM, IPC_ECORRUPT, IPC_ECUDA, IPC_ETIMEOUT, IPC_EBUSY = -4, -5, -6, -7, -8
IPC_F32, IPC_F64 = 0, 1
IPC_LINEAR, IPC_CUBIC, IPC_CUBIC_QUAD, IPC_INTERP_AUTO = 0, 1, 2, 3
IPC_EB_ABS, IPC_EB_REL = 0, 1
IPC_BOUND_STRICT, IPC_BOUND_PAPER = 0, 1
IPC_TARGET_EB, IPC_TARGET_BITRATE = 0, 1
IPC_REFINE_CANONICAL, IPC_REFINE_INCREMENTAL, IPC_REFINE_AUTO = 0, 1, 2
IPC_KERNEL_RETRIEVE_LEVEL, IPC_KERNEL_INCREMENT_LEVEL = 2, 6


class ipc_target(C.Structure):
    _fields_ = [("kind", C.c_int), ("value", C.c_double)]


class ipc_batch_item(C.Structure):
    _fields_ = [("d_in", C.c_void_p), ("dtype", C.c_int), ("ndim", C.c_int),
                ("dims", C.c_int64 * 3), ("eb_mode", C.c_int), ("eb", C.c_double),
                ("interp", C.c_int), ("bound", C.c_int)]


class ipc_error_metrics(C.Structure):
    _fields_ = [("max_abs_err", C.c_double), ("mse", C.c_double), ("psnr", C.c_double),
                ("range", C.c_double), ("finite", C.c_uint64), ("nonfinite_mismatch", C.c_uint64)]


class ipc_server_cfg(C.Structure):
    _fields_ = [("mem_budget", C.c_uint64), ("hbm_reserve", C.c_uint64), ("max_batch", C.c_int),
                ("max_inflight", C.c_int), ("nstreams", C.c_int), ("plain", C.c_int),
                ("max_batch_values", C.c_uint64), ("refine_mode", C.c_int)]


class ipc_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("field", C.c_void_p), ("view_id", C.c_uint64),
                ("target", ipc_target), ("user_tag", C.c_uint64)]


class ipc_completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("user_tag", C.c_uint64), ("status", C.c_int),
                ("view_id", C.c_uint64), ("d_out", C.c_void_p), ("bytes", C.c_uint64),
                ("bound", C.c_double), ("latency_us", C.c_double), ("queue_us", C.c_double)]


IPC_REQ_RETRIEVE, IPC_REQ_REFINE, IPC_REQ_RELEASE = 0, 1, 2


class IpcError(RuntimeError):
    def __init__(self, rc: int, what: str, detail: str):
        super().__init__("%s failed with status %d: %s" % (what, rc, detail))
        self.rc = rc


class LibraryMissing(ImportError):
    pass


_lib = None


def lib() -> C.CDLL:
    """Load libipcomp.so from the package directory (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = BOUNDS_LIB_PATH if os.environ.get("IPC_BOUNDS_CHECK") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise LibraryMissing("%s is not built: run paper_2502_04093_gb300.build.build(%s)" %
                             (os.path.basename(path), "bounds=True" if path != LIB_PATH else ""))
    L = C.CDLL(path)
    vp, u64p = C.c_void_p, C.POINTER(C.c_uint64)
    i64p = C.POINTER(C.c_int64)
    L.ipc_compress.argtypes = [vp, C.c_int, C.c_int, i64p, C.c_int, C.c_double, C.c_int,
                               C.c_int, vp, C.POINTER(vp)]
    L.ipc_retrieve.argtypes = [vp, ipc_target, vp, vp, C.POINTER(vp)]
    L.ipc_refine.argtypes = [vp, ipc_target, vp, vp]
    L.ipc_retrieve_ex.argtypes = [vp, ipc_target, vp, vp, C.c_int, C.POINTER(vp)]
    L.ipc_view_set_refine_mode.argtypes = [vp, C.c_int]
    L.ipc_refine_info.argtypes = [vp, C.POINTER(C.c_int), u64p]
    L.ipc_autotune_retrieve.argtypes = [vp, ipc_target, vp, vp, C.c_int, C.POINTER(C.c_int)]
    L.ipc_autotune_entry.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), i64p,
                                     C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.ipc_autotune_set.argtypes = [C.c_int, C.c_int, i64p, C.c_int, C.c_int]
    L.ipc_error_metrics_host.argtypes = [vp, vp, C.c_int, C.c_uint64, C.POINTER(ipc_error_metrics)]
    L.ipc_free.argtypes = [vp]
    L.ipc_selection.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), u64p,
                                C.POINTER(C.c_double)]
    L.ipc_select_container.argtypes = [C.c_char_p, C.c_uint64, ipc_target, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), u64p, C.POINTER(C.c_double)]
    L.ipc_compressed_size.argtypes = [vp, u64p]
    L.ipc_export.argtypes = [vp, vp, u64p]
    L.ipc_import.argtypes = [vp, C.c_uint64, vp, C.POINTER(vp)]
    L.ipc_nvtx_enable.argtypes = [C.c_int]
    L.ipc_debug_bounds.argtypes = [u64p, C.c_int]
    L.ipc_encode_container.argtypes = [C.c_char_p, C.c_uint64, C.c_int, vp, u64p, C.c_int]
    L.ipc_container_ranges.argtypes = [C.c_char_p, C.c_uint64, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.c_int, u64p, C.POINTER(C.c_int)]
    L.ipc_import_partial.argtypes = [C.c_char_p, C.c_uint64, C.POINTER(C.c_int), C.c_int, vp,
                                     C.POINTER(vp)]
    L.ipc_field_load_planes.argtypes = [vp, C.c_char_p, C.c_uint64, C.POINTER(C.c_int), C.c_int,
                                        vp]
    L.ipc_field_resident.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.ipc_decode_container.argtypes = [C.c_char_p, C.c_uint64, vp, u64p, C.c_int]
    L.ipc_field_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), i64p,
                                 C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.ipc_last_error.restype = C.c_char_p
    L.ipc_compress_batch.argtypes = [C.c_int, C.POINTER(ipc_batch_item), vp, C.POINTER(vp)]
    L.ipc_retrieve_batch.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(ipc_target),
                                     C.POINTER(vp), vp, C.POINTER(vp)]
    L.ipc_plan_retrieve_batch.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(ipc_target),
                                          C.POINTER(vp), vp, C.POINTER(vp)]
    L.ipc_plan_launch.argtypes = [vp, vp]
    L.ipc_server_create.argtypes = [C.POINTER(ipc_server_cfg), C.POINTER(vp)]
    L.ipc_server_submit.argtypes = [vp, C.POINTER(ipc_request), C.POINTER(C.c_uint64)]
    L.ipc_server_poll.argtypes = [vp, C.POINTER(ipc_completion), C.c_int, C.POINTER(C.c_int),
                                  C.c_int]
    L.ipc_server_stats.argtypes = [vp, u64p, u64p, u64p]
    L.ipc_server_destroy.argtypes = [vp]
    L.ipc_server_stop.argtypes = [vp]
    L.ipc_profile_enable.argtypes = [C.c_int]
    L.ipc_profile_read.argtypes = [C.c_int, u64p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.ipc_launch_count.restype = C.c_uint64
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != IPC_OK:
        raise IpcError(rc, what, lib().ipc_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return IPC_F32
    if t.dtype == torch.float64:
        return IPC_F64
    raise TypeError("ipc takes float32 or float64 tensors")


def _require_cuda(t, name):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)


def ipc_compress(x, eb: float, eb_mode: int = IPC_EB_ABS, interp: int = IPC_CUBIC,
                 bound: int = IPC_BOUND_STRICT, stream=None, dims=None) -> C.c_void_p:
    """Compress the CUDA tensor x; returns an ipc_field handle."""
    _require_cuda(x, "x")
    shape = tuple(x.shape) if dims is None else tuple(dims)
    arr = (C.c_int64 * max(len(shape), 1))(*[int(s) for s in shape])
    h = C.c_void_p()
    _check(lib().ipc_compress(C.c_void_p(x.data_ptr()), _dtype_code(x), len(shape), arr,
                              int(eb_mode), float(eb), int(interp), int(bound), _stream(stream),
                              C.byref(h)), "ipc_compress")
    return h


def ipc_retrieve(field, kind: int, value: float, out, stream=None, want_view=True):
    """Reconstruct into the CUDA tensor `out`; returns an ipc_view handle
    (or None when want_view is False)."""
    _require_cuda(out, "out")
    v = C.c_void_p()
    _check(lib().ipc_retrieve(field, ipc_target(int(kind), float(value)),
                              C.c_void_p(out.data_ptr()), _stream(stream),
                              C.byref(v) if want_view else None), "ipc_retrieve")
    return v if want_view else None


def ipc_autotune_retrieve(field, kind: int, value: float, out, stream=None, reps: int = 3) -> int:
    """Time the launch shapes of each level of this retrieval and record the
    fastest (process-wide); `out` receives the reconstruction. Returns the
    number of recorded shapes."""
    _require_cuda(out, "out")
    n = C.c_int()
    _check(lib().ipc_autotune_retrieve(field, ipc_target(int(kind), float(value)),
                                       C.c_void_p(out.data_ptr()), _stream(stream), int(reps),
                                       C.byref(n)), "ipc_autotune_retrieve")
    return n.value


def ipc_autotune_clear() -> None:
    _check(lib().ipc_autotune_clear(), "ipc_autotune_clear")


def ipc_autotune_entries():
    """The recorded shapes: [(dtype, w16, (M0, M1, M2), ns, per_sm)]."""
    out, i = [], 0
    while True:
        dt, w, ns, ps = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        M = (C.c_int64 * 3)()
        rc = lib().ipc_autotune_entry(i, C.byref(dt), C.byref(w), M, C.byref(ns), C.byref(ps))
        if rc != IPC_OK:
            return out
        out.append((dt.value, w.value, tuple(M), ns.value, ps.value))
        i += 1


def ipc_error_metrics_host(x, y) -> dict:
    """L-inf error, MSE, value range and PSNR of y against x (host arrays of
    one float type, compared in FP64; Sec. 3.1.1 definitions)."""
    import numpy as np
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    if x.shape != y.shape or x.dtype != y.dtype or x.dtype not in (np.float32, np.float64):
        raise IpcError(IPC_EINVAL, "ipc_error_metrics_host",
                       "x and y must be float32 or float64 arrays of one shape and type")
    m = ipc_error_metrics()
    _check(lib().ipc_error_metrics_host(x.ctypes.data, y.ctypes.data,
                                        IPC_F32 if x.dtype == np.float32 else IPC_F64, x.size,
                                        C.byref(m)), "ipc_error_metrics_host")
    return {"max_abs_err": m.max_abs_err, "mse": m.mse, "psnr": m.psnr, "range": m.range,
            "finite": m.finite, "nonfinite_mismatch": m.nonfinite_mismatch}


def ipc_autotune_set(dtype: int, w16: int, M, ns: int, per_sm: int) -> None:
    """Record one shape in the table (as ipc_autotune_entries lists them)."""
    arr = (C.c_int64 * 3)(*[int(m) for m in M])
    _check(lib().ipc_autotune_set(int(dtype), int(w16), arr, int(ns), int(per_sm)),
           "ipc_autotune_set")


def ipc_autotune_save(path: str) -> int:
    """Write the table to a JSON file; returns the number of entries."""
    import json
    ents = [{"dtype": d, "w16": w, "M": list(M), "ns": ns, "per_sm": ps}
            for d, w, M, ns, ps in ipc_autotune_entries()]
    with open(path, "w") as fh:
        json.dump({"launch_shapes": ents}, fh, indent=1)
    return len(ents)


def ipc_autotune_load(path: str) -> int:
    """Add the entries of a file written by ipc_autotune_save to the table
    (each checked by ipc_autotune_set); returns their number."""
    import json
    with open(path) as fh:
        ents = json.load(fh)["launch_shapes"]
    for e in ents:
        ipc_autotune_set(e["dtype"], e["w16"], e["M"], e["ns"], e["per_sm"])
    return len(ents)


def ipc_retrieve_ex(field, kind: int, value: float, out, refine_mode: int, stream=None):
    """ipc_retrieve whose view refines in `refine_mode` (IPC_REFINE_*)."""
    _require_cuda(out, "out")
    v = C.c_void_p()
    _check(lib().ipc_retrieve_ex(field, ipc_target(int(kind), float(value)),
                                 C.c_void_p(out.data_ptr()), _stream(stream), int(refine_mode),
                                 C.byref(v)), "ipc_retrieve_ex")
    return v


def ipc_view_set_refine_mode(view, refine_mode: int) -> None:
    _check(lib().ipc_view_set_refine_mode(view, int(refine_mode)), "ipc_view_set_refine_mode")


def ipc_refine_info(view):
    """(whether the last refinement added an increment, plane-stream bytes it read)."""
    inc = C.c_int()
    by = C.c_uint64()
    _check(lib().ipc_refine_info(view, C.byref(inc), C.byref(by)), "ipc_refine_info")
    return bool(inc.value), by.value


def ipc_refine(view, kind: int, value: float, out, stream=None) -> None:
    _require_cuda(out, "out")
    _check(lib().ipc_refine(view, ipc_target(int(kind), float(value)),
                            C.c_void_p(out.data_ptr()), _stream(stream)), "ipc_refine")


def ipc_free(handle) -> None:
    if handle is not None:
        _check(lib().ipc_free(handle), "ipc_free")


def ipc_selection(view):
    """(b_per_level list, loaded bytes, guaranteed bound)."""
    b = (C.c_int * 64)()
    nl = C.c_int()
    by = C.c_uint64()
    bd = C.c_double()
    _check(lib().ipc_selection(view, b, C.byref(nl), C.byref(by), C.byref(bd)), "ipc_selection")
    return list(b)[:nl.value], by.value, bd.value


def ipc_select_container(buf: bytes, kind: int, value: float):
    """Selection of a retrieval computed on the host from a container's
    leading bytes (header, stage and plane-size tables): (b_per_level list,
    loaded bytes, guaranteed bound). Needs no GPU."""
    b = (C.c_int * 64)()
    nl = C.c_int()
    by = C.c_uint64()
    bd = C.c_double()
    _check(lib().ipc_select_container(bytes(buf), len(buf), ipc_target(int(kind), float(value)), b,
                                      C.byref(nl), C.byref(by), C.byref(bd)),
           "ipc_select_container")
    return list(b)[:nl.value], by.value, bd.value


def ipc_compressed_size(field) -> int:
    n = C.c_uint64()
    _check(lib().ipc_compressed_size(field, C.byref(n)), "ipc_compressed_size")
    return n.value


def ipc_export_size(field) -> int:
    n = C.c_uint64()
    _check(lib().ipc_export(field, None, C.byref(n)), "ipc_export")
    return n.value


def _ints(v):
    return (C.c_int * max(len(v), 1))(*[int(x) for x in v])


def ipc_container_ranges(head: bytes, b_new, b_old=None):
    """(offset, length) byte ranges of a container holding the planes
    b_new <= k < b_old of each level (b_old None: the leading tables and the
    planes k >= b_new), from the container's leading bytes."""
    head = bytes(head)
    n = C.c_int(0)
    bo = _ints(b_old) if b_old is not None else None
    _check(lib().ipc_container_ranges(head, len(head), _ints(b_new), bo, len(b_new), None,
                                      C.byref(n)), "ipc_container_ranges")
    r = (C.c_uint64 * max(2 * n.value, 1))()
    _check(lib().ipc_container_ranges(head, len(head), _ints(b_new), bo, len(b_new), r,
                                      C.byref(n)), "ipc_container_ranges")
    return [(r[2 * i], r[2 * i + 1]) for i in range(n.value)]


def ipc_import_partial(parts: bytes, b_per_level, stream=None) -> C.c_void_p:
    """A device field holding the planes k >= b_per_level[l-1] of each level,
    from the bytes of ipc_container_ranges(head, b_per_level) in order."""
    parts = bytes(parts)
    h = C.c_void_p()
    _check(lib().ipc_import_partial(parts, len(parts), _ints(b_per_level), len(b_per_level),
                                    _stream(stream), C.byref(h)), "ipc_import_partial")
    return h


def ipc_field_load_planes(field, parts: bytes, b_new, stream=None) -> None:
    """Adds planes b_new <= k < resident of each level (bytes of
    ipc_container_ranges(head, b_new, resident) in order)."""
    parts = bytes(parts)
    h = field.h if hasattr(field, "h") else field
    _check(lib().ipc_field_load_planes(h, parts, len(parts), _ints(b_new), len(b_new),
                                       _stream(stream)), "ipc_field_load_planes")


def ipc_field_resident(field):
    h = field.h if hasattr(field, "h") else field
    b = (C.c_int * 64)()
    n = C.c_int()
    _check(lib().ipc_field_resident(h, b, C.byref(n)), "ipc_field_resident")
    return list(b)[:n.value]


def ipc_debug_bounds(reset: bool = False):
    """Bounds-checking build only: (count, site, index, limit) of the first
    out-of-bounds global access of the level kernels since the last reset."""
    r = (C.c_uint64 * 4)()
    _check(lib().ipc_debug_bounds(r, 1 if reset else 0), "ipc_debug_bounds")
    return tuple(r)


def ipc_nvtx_enable(on: bool = True) -> None:
    """NVTX ranges around the library's calls and level launches."""
    _check(lib().ipc_nvtx_enable(1 if on else 0), "ipc_nvtx_enable")


def ipc_encode_container(raw: bytes, block_log2: int = 0, nthreads: int = 0) -> bytes:
    """The lossless stage (host): `raw` (normally an exported container) as
    an rANS-coded container."""
    raw = bytes(raw)
    n = C.c_uint64()
    _check(lib().ipc_encode_container(raw, len(raw), block_log2, None, C.byref(n), nthreads),
           "ipc_encode_container")
    out = C.create_string_buffer(max(n.value, 1))
    _check(lib().ipc_encode_container(raw, len(raw), block_log2, out, C.byref(n), nthreads),
           "ipc_encode_container")
    return out.raw[:n.value]


def ipc_decode_container(coded: bytes, nthreads: int = 0) -> bytes:
    """Inverse of ipc_encode_container."""
    coded = bytes(coded)
    n = C.c_uint64()
    _check(lib().ipc_decode_container(coded, len(coded), None, C.byref(n), nthreads),
           "ipc_decode_container")
    out = C.create_string_buffer(max(n.value, 1))
    _check(lib().ipc_decode_container(coded, len(coded), out, C.byref(n), nthreads),
           "ipc_decode_container")
    return out.raw[:n.value]


def ipc_export(field, out=None):
    """The container as bytes; or, when `out` is a writable host array (e.g.
    a numpy view of pinned memory) of at least ipc_export_size bytes, the
    container is written into it and a memoryview of its bytes returned."""
    n = C.c_uint64(ipc_export_size(field))
    if out is None:
        buf = (C.c_uint8 * max(n.value, 1))()
        _check(lib().ipc_export(field, buf, C.byref(n)), "ipc_export")
        return bytes(buf)[:n.value]
    mv = memoryview(out).cast("B")
    if mv.readonly or len(mv) < n.value:
        raise ValueError("export buffer must be writable and hold %d bytes" % n.value)
    addr = C.addressof(C.c_uint8.from_buffer(mv))
    n = C.c_uint64(len(mv))
    _check(lib().ipc_export(field, C.c_void_p(addr), C.byref(n)), "ipc_export")
    return mv[:n.value]


def ipc_import(data: bytes, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    arr = (C.c_uint8 * max(len(data), 1)).from_buffer_copy(data if data else b"\0")
    _check(lib().ipc_import(arr, len(data), _stream(stream), C.byref(h)), "ipc_import")
    return h


def ipc_field_info(field) -> dict:
    dt, nd, K, S = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    dims = (C.c_int64 * 3)()
    eb, mn, mx = C.c_double(), C.c_double(), C.c_double()
    _check(lib().ipc_field_info(field, C.byref(dt), C.byref(nd), dims, C.byref(K), C.byref(S),
                                C.byref(eb), C.byref(mn), C.byref(mx)), "ipc_field_info")
    return dict(dtype=dt.value, ndim=nd.value, dims=tuple(dims)[:nd.value], K=K.value,
                S=S.value, eb=eb.value, xmin=mn.value, xmax=mx.value)


def ipc_compress_batch(xs, ebs, eb_mode=IPC_EB_ABS, interp=IPC_CUBIC, bound=IPC_BOUND_STRICT,
                       stream=None):
    """Compress a list of CUDA tensors (any shapes) in one batch; returns the
    list of ipc_field handles."""
    n = len(xs)
    items = (ipc_batch_item * max(n, 1))()
    for i, x in enumerate(xs):
        _require_cuda(x, "x")
        it = items[i]
        it.d_in = x.data_ptr()
        it.dtype = _dtype_code(x)
        it.ndim = x.dim()
        for e, d in enumerate(x.shape):
            it.dims[e] = int(d)
        it.eb_mode = int(eb_mode[i] if isinstance(eb_mode, (list, tuple)) else eb_mode)
        it.eb = float(ebs[i] if isinstance(ebs, (list, tuple)) else ebs)
        it.interp = int(interp[i] if isinstance(interp, (list, tuple)) else interp)
        it.bound = int(bound)
    outs = (C.c_void_p * max(n, 1))()
    _check(lib().ipc_compress_batch(n, items, _stream(stream), outs), "ipc_compress_batch")
    return [C.c_void_p(outs[i]) for i in range(n)]


def _batch_args(fields, targets, outs):
    n = len(fields)
    fa = (C.c_void_p * max(n, 1))(*[f.value if isinstance(f, C.c_void_p) else f for f in fields])
    ta = (ipc_target * max(n, 1))()
    for i, (k, v) in enumerate(targets):
        ta[i].kind = int(k)
        ta[i].value = float(v)
    for o in outs:
        _require_cuda(o, "out")
    oa = (C.c_void_p * max(n, 1))(*[o.data_ptr() for o in outs])
    return n, fa, ta, oa


def ipc_retrieve_batch(fields, targets, outs, stream=None, want_views=False):
    """targets: list of (kind, value); outs: CUDA tensors. Returns the views
    (or None)."""
    n, fa, ta, oa = _batch_args(fields, targets, outs)
    va = (C.c_void_p * max(n, 1))()
    _check(lib().ipc_retrieve_batch(n, fa, ta, oa, _stream(stream), va if want_views else None),
           "ipc_retrieve_batch")
    return [C.c_void_p(va[i]) for i in range(n)] if want_views else None


def ipc_plan_retrieve_batch(fields, targets, outs, stream=None):
    n, fa, ta, oa = _batch_args(fields, targets, outs)
    h = C.c_void_p()
    _check(lib().ipc_plan_retrieve_batch(n, fa, ta, oa, _stream(stream), C.byref(h)),
           "ipc_plan_retrieve_batch")
    return h


def ipc_plan_launch(plan, stream=None):
    _check(lib().ipc_plan_launch(plan, _stream(stream)), "ipc_plan_launch")


def ipc_server_create(mem_budget, max_batch=0, max_inflight=2, nstreams=2, plain=False,
                      hbm_reserve=1 << 30, max_batch_values=0, refine_mode=IPC_REFINE_CANONICAL):
    cfg = ipc_server_cfg(int(mem_budget), int(hbm_reserve), int(max_batch), int(max_inflight),
                         int(nstreams), 1 if plain else 0, int(max_batch_values),
                         int(refine_mode))
    h = C.c_void_p()
    _check(lib().ipc_server_create(C.byref(cfg), C.byref(h)), "ipc_server_create")
    return h


def ipc_server_submit(server, kind, field=None, view_id=0, target=(0, 0.0), user_tag=0):
    r = ipc_request(int(kind), field.value if isinstance(field, C.c_void_p) else field,
                    int(view_id), ipc_target(int(target[0]), float(target[1])), int(user_tag))
    t = C.c_uint64()
    _check(lib().ipc_server_submit(server, C.byref(r), C.byref(t)), "ipc_server_submit")
    return t.value


def ipc_server_poll(server, max_n=256, timeout_us=0):
    """List of completions (dicts); empty when none arrived in time."""
    buf = (ipc_completion * max_n)()
    n = C.c_int()
    rc = lib().ipc_server_poll(server, buf, max_n, C.byref(n), int(timeout_us))
    if rc not in (IPC_OK, IPC_ETIMEOUT):
        _check(rc, "ipc_server_poll")
    return [dict(ticket=c.ticket, user_tag=c.user_tag, status=c.status, view_id=c.view_id,
                 d_out=c.d_out, bytes=c.bytes, bound=c.bound, latency_us=c.latency_us,
                 queue_us=c.queue_us) for c in buf[:n.value]]


def ipc_server_stats(server):
    b, r, m = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(lib().ipc_server_stats(server, C.byref(b), C.byref(r), C.byref(m)), "ipc_server_stats")
    return dict(batches=b.value, requests=r.value, mem_used=m.value)


def ipc_server_stop(server) -> None:
    _check(lib().ipc_server_stop(server), "ipc_server_stop")


def ipc_server_destroy(server):
    _check(lib().ipc_server_destroy(server), "ipc_server_destroy")


def device_view(ptr, shape, dtype):
    """A torch tensor aliasing device memory the library owns (no copy)."""
    import torch

    class _Arr:
        pass

    a = _Arr()
    a.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape),
                                  "typestr": "<f4" if dtype in (torch.float32, "f4") else "<f8",
                                  "data": (int(ptr), False), "version": 2}
    return torch.as_tensor(a, device="cuda")


IPC_KERNEL_NAMES = ["range", "compress_level", "retrieve_level", "anchor", "pack", "unpack",
                    "increment_level", "coarse"]


def ipc_profile_enable(on: bool) -> None:
    _check(lib().ipc_profile_enable(1 if on else 0), "ipc_profile_enable")


def ipc_profile_reset() -> None:
    _check(lib().ipc_profile_reset(), "ipc_profile_reset")


def ipc_profile_read(kind: int):
    """(launches, total device ms, algorithmic bytes) of one kernel kind."""
    n = C.c_uint64()
    ms = C.c_double()
    by = C.c_double()
    _check(lib().ipc_profile_read(int(kind), C.byref(n), C.byref(ms), C.byref(by)),
           "ipc_profile_read")
    return n.value, ms.value, by.value


def ipc_launch_count() -> int:
    return int(lib().ipc_launch_count())


def ipc_last_error() -> str:
    return lib().ipc_last_error().decode(errors="replace")


# -- convenience wrappers (own the handles) ---------------------------------
class Field:
    """An ipc_field handle that frees itself."""

    def __init__(self, handle, shape, dtype):
        self.h = handle
        self.shape = tuple(shape)
        self.dtype = dtype

    @classmethod
    def compress(cls, x, eb, eb_mode=IPC_EB_ABS, interp=IPC_CUBIC, bound=IPC_BOUND_STRICT,
                 stream=None):
        return cls(ipc_compress(x, eb, eb_mode, interp, bound, stream), x.shape, x.dtype)

    @classmethod
    def from_bytes(cls, data, shape, dtype, stream=None):
        return cls(ipc_import(data, stream), shape, dtype)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.ipc_free(self.h)
            self.h = None

    def retrieve(self, kind, value, out=None, stream=None, refine_mode=IPC_REFINE_CANONICAL):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        v = ipc_retrieve_ex(self.h, kind, value, out, refine_mode, stream)
        return out, View(v, self, out)

    def export(self) -> bytes:
        return ipc_export(self.h)

    def size(self) -> int:
        return ipc_compressed_size(self.h)

    def info(self) -> dict:
        return ipc_field_info(self.h)


class View:
    def __init__(self, handle, field: Field, out):
        self.h = handle
        self.field = field
        self.out = out

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.ipc_free(self.h)
            self.h = None

    def refine(self, kind, value, stream=None):
        ipc_refine(self.h, kind, value, self.out, stream)
        return self.out

    def refine_info(self):
        return ipc_refine_info(self.h)

    def selection(self):
        return ipc_selection(self.h)

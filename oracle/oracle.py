"""ctypes binding of the IPComp CPU oracle (test infrastructure only).

The oracle (``ipcomp_oracle.cpp``) is a plain single-threaded C++ restatement
of the IPComp paper (arXiv 2502.04093). Only ``tests/``, the smoke check and
the CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ipcomp_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

OK, EINVAL, EBOUND, EBUDGET, ENOMEM, ECORRUPT = 0, -1, -2, -3, -4, -5
F32, F64 = 0, 1
LINEAR, CUBIC, CUBIC_QUAD, AUTO = 0, 1, 2, 3
ABS, REL = 0, 1
STRICT, PAPER = 0, 1
EB, BITRATE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with plain g++ (no FMA contraction)."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        vp, i64p, u64p = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_uint64)
        L.ipco_compress.argtypes = [vp, C.c_int, C.c_int, i64p, C.c_int, C.c_double,
                                    C.c_int, C.c_int, C.POINTER(vp)]
        L.ipco_auto_interp.argtypes = [vp, C.c_int, C.c_int, i64p, C.c_int, C.c_double, C.c_int,
                                       C.POINTER(C.c_int)]
        L.ipco_export.argtypes = [vp, vp, u64p]
        L.ipco_import.argtypes = [vp, C.c_uint64, C.POINTER(vp)]
        L.ipco_free_field.argtypes = [vp]
        L.ipco_free_view.argtypes = [vp]
        L.ipco_retrieve.argtypes = [vp, C.c_int, C.c_double, vp, C.POINTER(vp)]
        L.ipco_refine.argtypes = [vp, C.c_int, C.c_double, vp]
        L.ipco_refine_delta.argtypes = [vp, C.c_int, C.c_double, vp, C.POINTER(C.c_int)]
        L.ipco_decode_window.argtypes = [C.c_uint32, C.c_uint32, C.c_int, C.c_int]
        L.ipco_decode_window.restype = C.c_uint32
        L.ipco_reconstruct.argtypes = [vp, C.POINTER(C.c_int), vp]
        L.ipco_selection.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), u64p,
                                     C.POINTER(C.c_double)]
        L.ipco_field_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), u64p,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), u64p]
        L.ipco_stage_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      u64p, C.POINTER(C.c_int), C.POINTER(C.c_uint32), u64p]
        L.ipco_stage_codes.argtypes = [vp, C.c_int, vp]
        L.ipco_delta_table.argtypes = [vp, C.c_int, vp]
        L.ipco_set_delta_model.argtypes = [vp, C.c_int]
        L.ipco_stream_size.argtypes = [vp, C.c_int, C.c_int, u64p]
        L.ipco_point_stage.argtypes = [C.c_int, i64p, vp]
        L.ipco_option_tables.argtypes = [vp, C.c_double, vp, vp]
        L.ipco_negabinary.argtypes = [C.c_int32]
        L.ipco_negabinary.restype = C.c_uint32
        L.ipco_negabinary_inv.argtypes = [C.c_uint32]
        L.ipco_negabinary_inv.restype = C.c_int64
        L.ipco_xor_encode.argtypes = [C.c_uint32]
        L.ipco_xor_encode.restype = C.c_uint32
        L.ipco_xor_decode.argtypes = [C.c_uint32]
        L.ipco_xor_decode.restype = C.c_uint32
        L.ipco_xor_check.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        L.ipco_xor_check.restype = C.c_uint64
    return _lib


class OracleError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"{what} failed with status {rc}")
        self.rc = rc


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(rc, what)


def _dims(shape):
    arr = (C.c_int64 * len(shape))(*[int(s) for s in shape])
    return arr


class Field:
    """A field compressed by the oracle."""

    def __init__(self, handle, shape, dtype):
        self.h = C.c_void_p(handle)
        self.shape = tuple(shape)
        self.dtype = np.dtype(dtype)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipco_free_field(self.h)
            self.h = None

    # -- container ---------------------------------------------------------
    def export(self) -> bytes:
        n = C.c_uint64(0)
        _check(lib().ipco_export(self.h, None, C.byref(n)), "ipco_export")
        buf = (C.c_uint8 * n.value)()
        _check(lib().ipco_export(self.h, buf, C.byref(n)), "ipco_export")
        return bytes(buf)

    def info(self) -> dict:
        K, S = C.c_int(), C.c_int()
        n, mand = C.c_uint64(), C.c_uint64()
        eb, mn, mx, ma = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        _check(lib().ipco_field_info(self.h, C.byref(K), C.byref(S), C.byref(n),
                                     C.byref(eb), C.byref(mn), C.byref(mx), C.byref(ma),
                                     C.byref(mand)), "ipco_field_info")
        return dict(K=K.value, S=S.value, n=n.value, eb=eb.value, xmin=mn.value,
                    xmax=mx.value, xmaxabs=ma.value, mandatory=mand.value)

    def stage(self, t: int) -> dict:
        lv, dm, H = C.c_int(), C.c_int(), C.c_int()
        nc, no = C.c_uint64(), C.c_uint64()
        Q = C.c_uint32()
        _check(lib().ipco_stage_info(self.h, t, C.byref(lv), C.byref(dm), C.byref(nc),
                                     C.byref(H), C.byref(Q), C.byref(no)), "ipco_stage_info")
        return dict(level=lv.value, dim=dm.value, ncodes=nc.value, H=H.value, Q=Q.value,
                    noutliers=no.value)

    def codes(self, t: int) -> np.ndarray:
        nc = self.stage(t)["ncodes"]
        q = np.zeros(nc, dtype=np.int32)
        _check(lib().ipco_stage_codes(self.h, t, q.ctypes.data), "ipco_stage_codes")
        return q

    def delta_table(self, t: int) -> np.ndarray:
        """Data maximum of |q - q'_b| over stage t's codes, b = 0..32."""
        m = np.zeros(33, dtype=np.uint64)
        _check(lib().ipco_delta_table(self.h, t, m.ctypes.data), "ipco_delta_table")
        return m

    def set_delta_model(self, model: int) -> None:
        """0: closed-form bound (the container's); 1: data maximum (study)."""
        _check(lib().ipco_set_delta_model(self.h, model), "ipco_set_delta_model")

    def stream_size(self, t: int, k: int) -> int:
        b = C.c_uint64()
        _check(lib().ipco_stream_size(self.h, t, k, C.byref(b)), "ipco_stream_size")
        return b.value

    def option_tables(self, E_abs: float):
        K = self.info()["K"]
        cost = np.zeros((K, 33), dtype=np.uint64)
        byts = np.zeros((K, 33), dtype=np.uint64)
        _check(lib().ipco_option_tables(self.h, float(E_abs), cost.ctypes.data,
                                        byts.ctypes.data), "ipco_option_tables")
        return cost, byts

    # -- retrieval ---------------------------------------------------------
    def retrieve(self, kind: int, value: float):
        out = np.empty(self.shape, dtype=self.dtype)
        v = C.c_void_p()
        _check(lib().ipco_retrieve(self.h, kind, float(value), out.ctypes.data,
                                   C.byref(v)), "ipco_retrieve")
        return out, View(v.value, self, out)

    def reconstruct(self, b) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.dtype)
        arr = (C.c_int * len(b))(*[int(v) for v in b])
        _check(lib().ipco_reconstruct(self.h, arr, out.ctypes.data), "ipco_reconstruct")
        return out


class View:
    def __init__(self, handle, field: Field, out: np.ndarray):
        self.h = C.c_void_p(handle)
        self.field = field  # keeps the field alive
        self.out = out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipco_free_view(self.h)
            self.h = None

    def refine(self, kind: int, value: float) -> np.ndarray:
        _check(lib().ipco_refine(self.h, kind, float(value), self.out.ctypes.data),
               "ipco_refine")
        return self.out

    def refine_delta(self, kind: int, value: float):
        """Algorithm 2 on the view's output array (updated in place); returns
        (output, whether the incremental path ran)."""
        inc = C.c_int()
        _check(lib().ipco_refine_delta(self.h, kind, float(value), self.out.ctypes.data,
                                       C.byref(inc)), "ipco_refine_delta")
        return self.out, bool(inc.value)

    def selection(self):
        K = self.field.info()["K"]
        b = (C.c_int * max(K, 1))()
        nl = C.c_int()
        byts = C.c_uint64()
        bound = C.c_double()
        _check(lib().ipco_selection(self.h, b, C.byref(nl), C.byref(byts), C.byref(bound)),
               "ipco_selection")
        return list(b)[:nl.value], byts.value, bound.value


def compress(x: np.ndarray, eb: float, eb_mode: int = ABS, interp: int = CUBIC,
             bound: int = STRICT) -> Field:
    x = np.ascontiguousarray(x)
    if x.dtype == np.float32:
        dt = F32
    elif x.dtype == np.float64:
        dt = F64
    else:
        raise TypeError("oracle takes float32 or float64")
    h = C.c_void_p()
    _check(lib().ipco_compress(x.ctypes.data, dt, x.ndim, _dims(x.shape), eb_mode,
                               float(eb), interp, bound, C.byref(h)), "ipco_compress")
    return Field(h.value, x.shape, x.dtype)


def auto_interp(x: np.ndarray, eb: float, eb_mode: int = ABS, bound: int = STRICT) -> int:
    """The interpolation mode compress(..., interp=AUTO) takes for x."""
    x = np.ascontiguousarray(x)
    dt = F32 if x.dtype == np.float32 else F64
    m = C.c_int(-1)
    _check(lib().ipco_auto_interp(x.ctypes.data, dt, x.ndim, _dims(x.shape), eb_mode, float(eb),
                                  bound, C.byref(m)), "ipco_auto_interp")
    return m.value


def compress_rc(x: np.ndarray, eb: float, eb_mode: int = ABS, interp: int = CUBIC,
                bound: int = STRICT, dims=None) -> int:
    """Status code only (for argument-validation tests)."""
    x = np.ascontiguousarray(x)
    shape = x.shape if dims is None else dims
    h = C.c_void_p()
    rc = lib().ipco_compress(x.ctypes.data, F32 if x.dtype == np.float32 else F64,
                             len(shape), _dims(shape), eb_mode, float(eb), interp,
                             bound, C.byref(h))
    if rc == 0:
        lib().ipco_free_field(h)
    return rc


def import_bytes(buf: bytes, shape, dtype) -> Field:
    h = C.c_void_p()
    arr = (C.c_uint8 * len(buf)).from_buffer_copy(buf)
    _check(lib().ipco_import(arr, len(buf), C.byref(h)), "ipco_import")
    return Field(h.value, shape, dtype)


def import_rc(buf: bytes) -> int:
    h = C.c_void_p()
    arr = (C.c_uint8 * max(len(buf), 1)).from_buffer_copy(buf if buf else b"\0")
    rc = lib().ipco_import(arr, len(buf), C.byref(h))
    if rc == 0:
        lib().ipco_free_field(h)
    return rc


def point_stage(shape) -> np.ndarray:
    n = int(np.prod(shape))
    sp = np.zeros(n, dtype=np.int32)
    _check(lib().ipco_point_stage(len(shape), _dims(shape), sp.ctypes.data),
           "ipco_point_stage")
    return sp.reshape(shape)


def negabinary(q: int) -> int:
    return lib().ipco_negabinary(q)


def negabinary_inv(n: int) -> int:
    return lib().ipco_negabinary_inv(n)


def xor_encode(n: int) -> int:
    return lib().ipco_xor_encode(n)


def xor_decode(e: int) -> int:
    return lib().ipco_xor_decode(e)


def decode_window(e: int, nold: int, bn: int, bo: int) -> int:
    return int(lib().ipco_decode_window(e & 0xFFFFFFFF, nold & 0xFFFFFFFF, bn, bo))


def xor_check(start: int, count: int, step: int) -> int:
    return lib().ipco_xor_check(start, count, step)

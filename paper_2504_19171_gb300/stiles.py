"""Python binding of the C ABI in ``include/stiles.h`` (argument marshalling
only: every step of the factorization and the selected inversion runs in the
CUDA library).

The low-level functions carry the C names (``stiles_create``,
``stiles_factor`` ...) and take raw pointers; :class:`Stiles` wraps a handle
with torch-allocated device buffers. The library is loaded from the in-tree
build (``_build/libstiles.so``); importing this module raises if it is
missing, and the launch functions raise if no CUDA device is present: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# STILES_CHECKED=1 selects the self-checking build (diagnostics only)
LIB_PATH = os.path.join(_PKG, "_build", "libstiles_checked.so" if os.environ.get("STILES_CHECKED") == "1"
                        else "libstiles.so")

STILES_OK = 0
STILES_ERR_INVALID_ARG = -1
STILES_ERR_NOT_SPD = -2
STILES_ERR_TIMEOUT = -3
STILES_ERR_CUDA = -4
STILES_ERR_OOM = -5
STILES_ERR_UNSUPPORTED = -6
STILES_ERR_PLAN = -7
STILES_ERR_TOO_LARGE = -8
STILES_ERR_BUSY = -9
NOALLOC_SCRATCH_BYTES = 64 << 20
STILES_FP64 = 0
STILES_EMU64 = 1
STILES_FP32X = 2
STILES_OPT_WAIT_BUDGET_NS = 1
STILES_OPT_GRID = 2
STILES_OPT_TRACE = 3

PLAN_FACTOR, PLAN_SELINV, PLAN_FUSED = 0, 1, 2

EXPORTS = [
    "stiles_create", "stiles_layout_doubles", "stiles_workspace_bytes", "stiles_factor", "stiles_selinv",
    "stiles_factor_selinv", "stiles_logdet", "stiles_status", "stiles_set_option", "stiles_plan_stats",
    "stiles_debug_check_corrupted", "stiles_debug_break_plan", "stiles_destroy", "stiles_strerror", "stiles_trace",
    "stiles_factor_selinv_noalloc", "stiles_debug_validate", "stiles_factor_selinv_host",
    "stiles_batch_create", "stiles_batch_offsets", "stiles_batch_workspace_bytes", "stiles_batch_factor_selinv",
    "stiles_batch_status", "stiles_batch_logdet", "stiles_batch_set_option", "stiles_batch_stats",
    "stiles_batch_destroy", "stiles_debug_validate_batch", "stiles_create_tuned",
    "stiles_server_create", "stiles_server_shape_doubles", "stiles_server_set_base", "stiles_server_start",
    "stiles_server_submit", "stiles_server_poll", "stiles_server_result", "stiles_server_sigma",
    "stiles_server_release", "stiles_server_request_bytes", "stiles_server_stop", "stiles_server_destroy",
    "stiles_debug_validate_serve", "stiles_create_selected", "stiles_server_status", "stiles_server_submit_values",
    "stiles_debug_occupancy", "stiles_debug_race_check", "stiles_debug_race_check_serve",
    "stiles_debug_race_check_batch",
]


class StilesError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2504_19171_gb300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "stiles_create": [i32, i32, i32, i32, i32, P(vp)],
        "stiles_layout_doubles": [vp, P(sz)],
        "stiles_workspace_bytes": [vp, P(sz), P(sz), P(sz)],
        "stiles_factor": [vp, vp, vp, vp, vp],
        "stiles_selinv": [vp, vp, vp, vp, vp],
        "stiles_factor_selinv": [vp, vp, vp, vp, vp, vp],
        "stiles_logdet": [vp, P(ctypes.c_double)],
        "stiles_status": [vp, P(i32), P(i64), P(i64)],
        "stiles_set_option": [vp, i32, i64],
        "stiles_plan_stats": [i32, i32, i32, i32, i32, i32, P(i64)],
        "stiles_debug_check_corrupted": [i32, i32, i32, i32, i32, i32],
        "stiles_debug_race_check": [i32, i32, i32, i32, i32, i32],
        "stiles_debug_race_check_serve": [i32, i32, i32, i32, i32, i32, i32],
        "stiles_debug_break_plan": [vp, i32],
        "stiles_destroy": [vp],
        "stiles_strerror": [i32],
        "stiles_debug_occupancy": [ctypes.c_int, P(ctypes.c_int)],
        "stiles_trace": [vp, P(ctypes.c_ulonglong), sz, P(sz)],
        "stiles_factor_selinv_noalloc": [vp, vp, vp, vp, vp],
        "stiles_debug_validate": [i32, i32, i32, i32, i32],
        "stiles_factor_selinv_host": [vp, vp, vp, vp, vp, vp, vp, vp],
        "stiles_batch_create": [i32, P(i32), P(i32), P(i32), P(i32), i32, P(i32), P(vp)],
        "stiles_create_tuned": [i32, i32, i32, i32, i32, i32, P(vp)],
        "stiles_server_create": [i32, P(i32), P(i32), P(i32), P(i32), i32, P(i32), sz, i32, P(vp)],
        "stiles_server_shape_doubles": [vp, i32, P(sz), P(sz)],
        "stiles_server_set_base": [vp, i32, vp, vp, vp],
        "stiles_server_start": [vp, ctypes.c_double],
        "stiles_server_submit": [vp, i32, ctypes.c_double, ctypes.c_double, i64, P(i32)],
        "stiles_server_poll": [vp, i32, P(i32), P(i64), P(i32)],
        "stiles_server_result": [vp, i32, P(i32), P(i64), P(ctypes.c_double)],
        "stiles_server_sigma": [vp, i32, vp, P(vp)],
        "stiles_server_release": [vp, i32],
        "stiles_server_request_bytes": [vp, i32, P(sz)],
        "stiles_server_stop": [vp],
        "stiles_server_destroy": [vp],
        "stiles_debug_validate_serve": [i32, i32, i32, i32, i32, i32],
        "stiles_create_selected": [i32, i32, i32, i32, i32, i32, P(vp)],
        "stiles_server_status": [vp, P(i32), P(i64), P(i64)],
        "stiles_server_submit_values": [vp, i32, vp, i64, P(i32)],
        "stiles_batch_offsets": [vp, P(sz)],
        "stiles_batch_workspace_bytes": [vp, P(sz), P(sz)],
        "stiles_batch_factor_selinv": [vp, vp, vp, vp, vp, vp],
        "stiles_batch_status": [vp, i32, P(i32), P(i64)],
        "stiles_batch_logdet": [vp, P(ctypes.c_double)],
        "stiles_batch_set_option": [vp, i32, i64],
        "stiles_batch_stats": [vp, P(i64)],
        "stiles_batch_destroy": [vp],
        "stiles_debug_validate_batch": [i32, P(i32), P(i32), P(i32), P(i32), i32, P(i32)],
        "stiles_debug_race_check_batch": [i32, P(i32), P(i32), P(i32), P(i32), i32, P(i32), i32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "stiles_strerror" else i32
    return lib


_lib = _load()


def strerror(code: int) -> str:
    return _lib.stiles_strerror(int(code)).decode()


def _check(rc: int, what: str) -> None:
    if rc != STILES_OK:
        raise StilesError(rc, what)


# ----------------------------------------------------------- C names -----
def stiles_create(nt: int, b: int, band: int, arrow: int, precision: int = STILES_FP64, tuning: int = 0,
                  first_column: int = 0) -> int:
    h = ctypes.c_void_p()
    if first_column:
        if tuning:
            raise ValueError("a selected plan takes the default tuning")
        _check(_lib.stiles_create_selected(nt, b, band, arrow, precision, first_column, ctypes.byref(h)),
               "stiles_create_selected")
    elif tuning:
        _check(_lib.stiles_create_tuned(nt, b, band, arrow, precision, tuning, ctypes.byref(h)), "stiles_create_tuned")
    else:
        _check(_lib.stiles_create(nt, b, band, arrow, precision, ctypes.byref(h)), "stiles_create")
    return h.value


def stiles_layout_doubles(h: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib.stiles_layout_doubles(h, ctypes.byref(n)), "stiles_layout_doubles")
    return n.value


def stiles_workspace_bytes(h: int) -> Tuple[int, int, int]:
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.stiles_workspace_bytes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "stiles_workspace_bytes")
    return a.value, b.value, c.value


def stiles_factor(h: int, A_ptr: int, L_ptr: int, scratch_ptr: int, stream: int = 0) -> None:
    _check(_lib.stiles_factor(h, A_ptr, L_ptr, scratch_ptr, stream), "stiles_factor")


def stiles_selinv(h: int, L_ptr: int, S_ptr: int, scratch_ptr: int, stream: int = 0) -> None:
    _check(_lib.stiles_selinv(h, L_ptr, S_ptr, scratch_ptr, stream), "stiles_selinv")


def stiles_factor_selinv(h: int, A_ptr: int, L_ptr: int, S_ptr: int, scratch_ptr: int, stream: int = 0) -> None:
    _check(_lib.stiles_factor_selinv(h, A_ptr, L_ptr, S_ptr, scratch_ptr, stream), "stiles_factor_selinv")


def stiles_factor_selinv_host(h: int, A_host_ptr: int, S_host_ptr: int, A_ptr: int, L_ptr: int, S_ptr: int,
                              scratch_ptr: int, stream: int = 0) -> None:
    """H2D copy of the packed A, fused factor + selected inversion, D2H copy
    of Sigma, all enqueued on `stream` by the library."""
    _check(_lib.stiles_factor_selinv_host(h, A_host_ptr, S_host_ptr, A_ptr, L_ptr, S_ptr, scratch_ptr, stream),
           "stiles_factor_selinv_host")


def stiles_factor_selinv_noalloc(h: int, A_ptr: int, L_ptr: int, S_ptr: int, stream: int = 0) -> None:
    """Factor + selected inversion without any device allocation: the scratch
    is the library's fixed 64 MiB array (shared by all calls; see the C
    header). Raises StilesError(STILES_ERR_TOO_LARGE) for shapes whose scratch
    does not fit."""
    _check(_lib.stiles_factor_selinv_noalloc(h, A_ptr, L_ptr, S_ptr, stream), "stiles_factor_selinv_noalloc")


def stiles_logdet(h: int) -> Tuple[int, float]:
    """(status code, logdet); logdet is NaN unless the code is STILES_OK."""
    v = ctypes.c_double(float("nan"))
    rc = _lib.stiles_logdet(h, ctypes.byref(v))
    return rc, (v.value if rc == STILES_OK else float("nan"))


def stiles_status(h: int) -> Tuple[int, int, int]:
    code, info, done = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.stiles_status(h, ctypes.byref(code), ctypes.byref(info), ctypes.byref(done)), "stiles_status")
    return code.value, info.value, done.value


def stiles_set_option(h: int, option: int, value: int) -> None:
    _check(_lib.stiles_set_option(h, option, int(value)), "stiles_set_option")


def stiles_plan_stats(nt: int, b: int, band: int, arrow: int, which: int, workers: int = 152,
                      precision: int = STILES_FP64) -> Dict[str, int]:
    st = (ctypes.c_longlong * 10)()
    _check(_lib.stiles_plan_stats(nt, b, band, arrow, which + 16 * precision, workers, st), "stiles_plan_stats")
    keys = ["tasks", "segments", "waits", "counters", "flops", "tile_gemms", "critical_path_ns", "makespan_ns",
            "flops_lowered", "edges"]
    return dict(zip(keys, list(st)))


def stiles_debug_validate(nt: int, b: int, band: int, arrow: int, which: int, precision: int = STILES_FP64) -> int:
    return _lib.stiles_debug_validate(nt, b, band, arrow, which + 16 * precision)


def stiles_debug_race_check(nt: int, b: int, band: int, arrow: int, which: int, precision: int = STILES_FP64,
                            plant: int = 0) -> int:
    """Host race check of a plan (0 = race-free; see include/stiles.h)."""
    return _lib.stiles_debug_race_check(nt, b, band, arrow, which + 16 * precision, plant)


def stiles_debug_race_check_serve(nt: int, b: int, band: int, arrow: int, precision: int = STILES_FP64,
                                  tuning: int = 0, plant: int = 0) -> int:
    """Host race check of a request-server template (0 = race-free)."""
    return _lib.stiles_debug_race_check_serve(nt, b, band, arrow, precision, tuning, plant)


def stiles_debug_check_corrupted(nt: int, b: int, band: int, arrow: int, which: int, mode: int) -> int:
    return _lib.stiles_debug_check_corrupted(nt, b, band, arrow, which, mode)


def stiles_debug_break_plan(h: int, which: int) -> None:
    _check(_lib.stiles_debug_break_plan(h, which), "stiles_debug_break_plan")


def stiles_debug_occupancy(tensor_parts: bool) -> int:
    """Resident CTAs of the persistent kernel per SM (FP64 plans, or plans
    with tensor-core parts)."""
    n = ctypes.c_int(0)
    _check(_lib.stiles_debug_occupancy(1 if tensor_parts else 0, ctypes.byref(n)), "stiles_debug_occupancy")
    return n.value


def stiles_trace(h: int) -> np.ndarray:
    """Per-part trace of the last launch as an (n_tasks, 4 parts, 4) uint64
    array: search start, got-part and end times (ns) and the packed
    (sm, cta, precision, last part, urgent, op) word; absent parts are zero."""
    n = ctypes.c_size_t()
    _check(_lib.stiles_trace(h, None, 0, ctypes.byref(n)), "stiles_trace")
    out = np.zeros((n.value, 4, 4), dtype=np.uint64)
    _check(_lib.stiles_trace(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), out.size, ctypes.byref(n)),
           "stiles_trace")
    return out


def stiles_destroy(h: Optional[int]) -> None:
    _check(_lib.stiles_destroy(h), "stiles_destroy")


# ----------------------------------------------------------- batch ----
def _ivec(vals):
    arr = (ctypes.c_int * len(vals))(*[int(v) for v in vals])
    return arr


def stiles_batch_create(shapes, precision: int = STILES_FP64, tuning=None) -> int:
    """shapes: sequence of (nt, b, band, arrow); tuning: per-matrix codes or None."""
    n = len(shapes)
    cols = list(zip(*shapes)) if n else [[], [], [], []]
    h = ctypes.c_void_p()
    tun = _ivec(tuning) if tuning is not None else None
    _check(_lib.stiles_batch_create(n, _ivec(cols[0]), _ivec(cols[1]), _ivec(cols[2]), _ivec(cols[3]), precision,
                                    tun, ctypes.byref(h)), "stiles_batch_create")
    return h.value


def stiles_batch_offsets(h: int, count: int) -> np.ndarray:
    off = (ctypes.c_size_t * (count + 1))()
    _check(_lib.stiles_batch_offsets(h, off), "stiles_batch_offsets")
    return np.array(off[:], dtype=np.int64)


def stiles_batch_workspace_bytes(h: int) -> Tuple[int, int]:
    bb, sb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.stiles_batch_workspace_bytes(h, ctypes.byref(bb), ctypes.byref(sb)), "stiles_batch_workspace_bytes")
    return bb.value, sb.value


def stiles_batch_factor_selinv(h: int, A_ptr: int, L_ptr: int, S_ptr: int, scratch_ptr: int, stream: int = 0) -> None:
    _check(_lib.stiles_batch_factor_selinv(h, A_ptr, L_ptr, S_ptr, scratch_ptr, stream), "stiles_batch_factor_selinv")


def stiles_batch_status(h: int, index: int) -> Tuple[int, int]:
    code, info = ctypes.c_int(), ctypes.c_longlong()
    _check(_lib.stiles_batch_status(h, index, ctypes.byref(code), ctypes.byref(info)), "stiles_batch_status")
    return code.value, info.value


def stiles_batch_logdet(h: int, count: int) -> Tuple[int, np.ndarray]:
    out = (ctypes.c_double * count)()
    rc = _lib.stiles_batch_logdet(h, out)
    return rc, np.array(out[:], dtype=np.float64)


def stiles_batch_set_option(h: int, option: int, value: int) -> None:
    _check(_lib.stiles_batch_set_option(h, option, value), "stiles_batch_set_option")


def stiles_batch_stats(h: int) -> Dict[str, int]:
    st = (ctypes.c_longlong * 9)()
    _check(_lib.stiles_batch_stats(h, st), "stiles_batch_stats")
    keys = ["tasks", "segments", "waits", "counters", "flops", "tile_gemms", "critical_path_ns", "makespan_ns",
            "flops_lowered"]
    return dict(zip(keys, st[:]))


def stiles_batch_destroy(h: Optional[int]) -> None:
    _check(_lib.stiles_batch_destroy(h), "stiles_batch_destroy")


def stiles_debug_validate_batch(shapes, precision: int = STILES_FP64, tuning=None) -> int:
    cols = list(zip(*shapes))
    return _lib.stiles_debug_validate_batch(len(shapes), _ivec(cols[0]), _ivec(cols[1]), _ivec(cols[2]),
                                            _ivec(cols[3]), precision, _ivec(tuning) if tuning is not None else None)


def stiles_debug_race_check_batch(shapes, precision: int = STILES_FP64, tuning=None, plant: int = 0) -> int:
    """Host race check of a batch's merged table (0 = race-free)."""
    cols = list(zip(*shapes))
    return _lib.stiles_debug_race_check_batch(len(shapes), _ivec(cols[0]), _ivec(cols[1]), _ivec(cols[2]),
                                              _ivec(cols[3]), precision,
                                              _ivec(tuning) if tuning is not None else None, plant)


# --------------------------------------------------------- layout -----
class PackedLayout:
    """Offsets of the packed band+arrow layout (column-major tiles; see the
    header for the definition)."""

    def __init__(self, nt: int, b: int, w: int, a: int):
        self.nt, self.b, self.w, self.a = nt, b, min(w, nt - 1), a
        self.colstride = (1 + self.w) * b * b + a * b
        self.doubles = nt * self.colstride + a * a

    def rows(self, i: int) -> int:
        return self.a if i == self.nt else self.b

    def offset(self, i: int, k: int) -> int:
        if k == self.nt:
            return self.nt * self.colstride
        if i == self.nt:
            return k * self.colstride + (1 + self.w) * self.b * self.b
        return k * self.colstride + (i - k) * self.b * self.b

    def pattern(self):
        for k in range(self.nt):
            yield (k, k)
            for i in range(k + 1, min(k + self.w, self.nt - 1) + 1):
                yield (i, k)
            if self.a > 0:
                yield (self.nt, k)
        if self.a > 0:
            yield (self.nt, self.nt)

    def pack(self, tiles, out: np.ndarray) -> np.ndarray:
        """Write a {(i,k): array} tile dict into the flat float64 array."""
        for (i, k) in self.pattern():
            r, c = self.rows(i), self.rows(k)
            off = self.offset(i, k)
            out[off:off + r * c] = np.asarray(tiles[(i, k)], dtype=np.float64).reshape(r, c).ravel(order="F")
        return out

    def unpack(self, flat: np.ndarray) -> Dict[Tuple[int, int], np.ndarray]:
        res = {}
        for (i, k) in self.pattern():
            r, c = self.rows(i), self.rows(k)
            off = self.offset(i, k)
            res[(i, k)] = flat[off:off + r * c].reshape(c, r).T.copy()
        return res

    def tile_view(self, flat, i: int, k: int):
        """(rows x cols) view of one tile of a flat array/tensor (transposed
        strides: column-major storage)."""
        r, c = self.rows(i), self.rows(k)
        off = self.offset(i, k)
        return flat[off:off + r * c].reshape(c, r).T


# ------------------------------------------------------ torch helper -----
class Stiles:
    """One handle plus its device buffers (torch float64 tensors on CUDA)."""

    def __init__(self, nt: int, b: int, band: int, arrow: int, device: str = "cuda", wait_budget_s: float = None,
                 precision: int = STILES_FP64, tuning: int = 0, first_column: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("stiles needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.h = stiles_create(nt, b, band, arrow, precision, tuning, first_column)
        self.layout = PackedLayout(nt, b, band, arrow)
        self.nt, self.b, self.w, self.a = nt, b, self.layout.w, arrow
        Lb, Sb, Wb = stiles_workspace_bytes(self.h)
        self.doubles = Lb // 8
        self.L = torch.empty(self.doubles, dtype=torch.float64, device=self.device)
        self.S = torch.empty(self.doubles, dtype=torch.float64, device=self.device)
        self.scratch = torch.empty(Wb, dtype=torch.uint8, device=self.device)
        self.A = None
        if wait_budget_s is not None:
            stiles_set_option(self.h, STILES_OPT_WAIT_BUDGET_NS, int(wait_budget_s * 1e9))

    def upload(self, M) -> "Stiles":
        """Pack an ArrowheadTiles (host) into a device A buffer."""
        host = self.layout.pack(M.tiles, np.zeros(self.doubles))
        self.A = self.torch.from_numpy(host).to(self.device)
        return self

    def stream_ptr(self, stream=None) -> int:
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return int(s.cuda_stream)

    def factor(self, stream=None, inplace: bool = False) -> None:
        dst = self.A if inplace else self.L
        if inplace:
            self.L = self.A
        stiles_factor(self.h, self.A.data_ptr(), dst.data_ptr(), self.scratch.data_ptr(), self.stream_ptr(stream))

    def selinv(self, stream=None) -> None:
        stiles_selinv(self.h, self.L.data_ptr(), self.S.data_ptr(), self.scratch.data_ptr(), self.stream_ptr(stream))

    def factor_selinv(self, stream=None) -> None:
        stiles_factor_selinv(self.h, self.A.data_ptr(), self.L.data_ptr(), self.S.data_ptr(),
                             self.scratch.data_ptr(), self.stream_ptr(stream))

    def factor_selinv_host(self, A_host, S_host, stream=None) -> float:
        """End-to-end call with host buffers (packed layout, CPU float64):
        factor and invert A_host in one launch, Sigma into S_host, return
        logdet (synchronizes). With two separate pinned tensors the kernel
        reads A and writes Sigma over the host link while it computes;
        otherwise the library copies A in before and Sigma out after."""
        torch = self.torch
        if self.A is None:
            self.A = torch.empty(self.doubles, dtype=torch.float64, device=self.device)
        for t in (A_host, S_host):
            if t.dtype != torch.float64 or t.device.type != "cpu" or not t.is_contiguous() or t.numel() != self.doubles:
                raise ValueError("host buffers must be contiguous CPU float64 tensors of the packed layout size")
        stiles_factor_selinv_host(self.h, A_host.data_ptr(), S_host.data_ptr(), self.A.data_ptr(), self.L.data_ptr(),
                                  self.S.data_ptr(), self.scratch.data_ptr(), self.stream_ptr(stream))
        return self.logdet()

    def status(self) -> Tuple[int, int, int]:
        return stiles_status(self.h)

    def logdet(self) -> float:
        rc, v = stiles_logdet(self.h)
        _check(rc, "stiles_logdet")
        return v

    def sigma_tiles(self) -> Dict[Tuple[int, int], np.ndarray]:
        return self.layout.unpack(self.S.cpu().numpy())

    def L_tiles(self) -> Dict[Tuple[int, int], np.ndarray]:
        return self.layout.unpack(self.L.cpu().numpy())

    def close(self) -> None:
        if getattr(self, "h", None):
            stiles_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StilesBatch:
    """One batch handle plus its device buffers: every matrix of `shapes`
    ((nt, b, band, arrow) each) is factored and inverted by one graph launch."""

    def __init__(self, shapes, device: str = "cuda", wait_budget_s: float = None, precision: int = STILES_FP64,
                 tuning=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("stiles needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device(device)
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.count = len(self.shapes)
        with torch.cuda.device(self.device):
            self.h = stiles_batch_create(self.shapes, precision, tuning)
        self.off = stiles_batch_offsets(self.h, self.count)
        self.layouts = [PackedLayout(*sh) for sh in self.shapes]
        nbytes, sbytes = stiles_batch_workspace_bytes(self.h)
        self.doubles = nbytes // 8
        self.L = torch.empty(self.doubles, dtype=torch.float64, device=self.device)
        self.S = torch.empty(self.doubles, dtype=torch.float64, device=self.device)
        self.scratch = torch.empty(sbytes, dtype=torch.uint8, device=self.device)
        self.A = None
        if wait_budget_s is not None:
            stiles_batch_set_option(self.h, STILES_OPT_WAIT_BUDGET_NS, int(wait_budget_s * 1e9))

    def pack(self, mats, out: np.ndarray = None) -> np.ndarray:
        """Host array of the batch layout holding every ArrowheadTiles of `mats`."""
        out = np.zeros(self.doubles) if out is None else out
        for m, M in enumerate(mats):
            lay = self.layouts[m]
            lay.pack(M.tiles, out[self.off[m]:self.off[m] + lay.doubles])
        return out

    def upload(self, mats) -> "StilesBatch":
        self.A = self.torch.from_numpy(self.pack(mats)).to(self.device)
        return self

    def stream_ptr(self, stream=None) -> int:
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return int(s.cuda_stream)

    def factor_selinv(self, stream=None) -> None:
        stiles_batch_factor_selinv(self.h, self.A.data_ptr(), self.L.data_ptr(), self.S.data_ptr(),
                                   self.scratch.data_ptr(), self.stream_ptr(stream))

    def status(self, index: int) -> Tuple[int, int]:
        return stiles_batch_status(self.h, index)

    def logdet(self) -> np.ndarray:
        rc, v = stiles_batch_logdet(self.h, self.count)
        _check(rc, "stiles_batch_logdet")
        return v

    def _unpack(self, flat: np.ndarray, m: int):
        lay = self.layouts[m]
        return lay.unpack(flat[self.off[m]:self.off[m] + lay.doubles])

    def sigma_tiles(self, m: int, host: np.ndarray = None):
        return self._unpack(self.S.cpu().numpy() if host is None else host, m)

    def L_tiles(self, m: int, host: np.ndarray = None):
        return self._unpack(self.L.cpu().numpy() if host is None else host, m)

    def close(self) -> None:
        if getattr(self, "h", None):
            stiles_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- server -----
def stiles_debug_validate_serve(nt: int, b: int, band: int, arrow: int, precision: int = STILES_FP64,
                                tuning: int = 0) -> int:
    return _lib.stiles_debug_validate_serve(nt, b, band, arrow, precision, tuning)


class StilesServer:
    """Request server with continuous batching (see the C header). Shapes
    (nt, b, band, arrow) form the pool; every shape needs a base matrix
    (set_base) before start(). submit() admits a request (tau, rho) of a pool
    shape or returns None when memory / slots are full; poll() returns the
    completed (request, tag) pairs; result() / sigma() read them; release()
    frees them."""

    def __init__(self, shapes, data_bytes: int, max_requests: int = 64, precision: int = STILES_FP64,
                 tuning=None, device: str = "cuda"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("stiles needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device(device)
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        cols = list(zip(*self.shapes))
        h = ctypes.c_void_p()
        tun = _ivec(tuning) if tuning is not None else None
        with torch.cuda.device(self.device):
            _check(_lib.stiles_server_create(len(self.shapes), _ivec(cols[0]), _ivec(cols[1]), _ivec(cols[2]),
                                             _ivec(cols[3]), precision, tun, int(data_bytes), max_requests,
                                             ctypes.byref(h)), "stiles_server_create")
        self.h = h.value
        self.max_requests = max_requests
        self.layouts = [PackedLayout(*sh) for sh in self.shapes]
        self._req = (ctypes.c_int * max_requests)()
        self._tag = (ctypes.c_longlong * max_requests)()

    def shape_doubles(self, shape: int) -> Tuple[int, int]:
        d, n = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.stiles_server_shape_doubles(self.h, shape, ctypes.byref(d), ctypes.byref(n)), "shape_doubles")
        return d.value, n.value

    def request_bytes(self, shape: int) -> int:
        v = ctypes.c_size_t()
        _check(_lib.stiles_server_request_bytes(self.h, shape, ctypes.byref(v)), "request_bytes")
        return v.value

    def set_base(self, shape: int, base, rb, ra) -> None:
        """base / rb / ra: contiguous float64 torch tensors (host or device)."""
        _check(_lib.stiles_server_set_base(self.h, shape, base.data_ptr(), rb.data_ptr(), ra.data_ptr()),
               "stiles_server_set_base")

    def start(self, window_s: float) -> None:
        _check(_lib.stiles_server_start(self.h, float(window_s)), "stiles_server_start")

    def submit(self, shape: int, tau: float, rho: float, tag: int = 0):
        r = ctypes.c_int()
        rc = _lib.stiles_server_submit(self.h, shape, float(tau), float(rho), int(tag), ctypes.byref(r))
        if rc == STILES_ERR_BUSY:
            return None
        _check(rc, "stiles_server_submit")
        return r.value

    def submit_values(self, shape: int, A_host, tag: int = 0):
        """Admit a request with explicit values: A_host is a contiguous host
        float64 tensor (or array) in the shape's packed layout."""
        import numpy as _np
        if isinstance(A_host, _np.ndarray):
            if A_host.dtype != _np.float64 or not A_host.flags["C_CONTIGUOUS"]:
                raise ValueError("A_host must be a contiguous float64 array")
            ptr, size = A_host.ctypes.data, A_host.size
        else:
            if A_host.dtype != self.torch.float64 or A_host.device.type != "cpu" or not A_host.is_contiguous():
                raise ValueError("A_host must be a contiguous CPU float64 tensor")
            ptr, size = A_host.data_ptr(), A_host.numel()
        if size != self.layouts[shape].doubles:
            raise ValueError("A_host must hold the shape's packed layout")
        r = ctypes.c_int()
        rc = _lib.stiles_server_submit_values(self.h, shape, ptr, int(tag), ctypes.byref(r))
        if rc == STILES_ERR_BUSY:
            return None
        _check(rc, "stiles_server_submit_values")
        return r.value

    def poll(self):
        n = ctypes.c_int()
        _check(_lib.stiles_server_poll(self.h, self.max_requests, self._req, self._tag, ctypes.byref(n)),
               "stiles_server_poll")
        return [(self._req[i], self._tag[i]) for i in range(n.value)]

    def result(self, request: int) -> Tuple[int, int, float]:
        code, info, ld = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_double()
        _check(_lib.stiles_server_result(self.h, request, ctypes.byref(code), ctypes.byref(info), ctypes.byref(ld)),
               "stiles_server_result")
        return code.value, info.value, ld.value

    def sigma(self, request: int, out=None):
        """Sigma of a completed request into `out` (float64 tensor, host or
        device; allocated on the host if None) in its shape's packed layout."""
        if out is None:
            raise ValueError("pass an output tensor of the shape's packed size")
        _check(_lib.stiles_server_sigma(self.h, request, out.data_ptr(), None), "stiles_server_sigma")
        return out

    def release(self, request: int) -> None:
        _check(_lib.stiles_server_release(self.h, request), "stiles_server_release")

    def status(self) -> Tuple[int, int, int]:
        code, info, done = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(_lib.stiles_server_status(self.h, ctypes.byref(code), ctypes.byref(info), ctypes.byref(done)),
               "stiles_server_status")
        return code.value, info.value, done.value

    def stop(self) -> int:
        return _lib.stiles_server_stop(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            _lib.stiles_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def first_column_for(entries, nt: int, b: int) -> int:
    """Symbolic pruning of a selection: the first tile column whose Sigma a
    set of requested entries (r, c) of Sigma needs (entries of the arrow rows /
    columns map to tile nt). Pass the result as ``first_column``."""
    cols = [min(min(int(r), int(c)) // b, nt) for r, c in entries]
    if not cols:
        raise ValueError("empty selection")
    return min(cols)


def widen_band(M, w_full: int = None):
    """The same matrix with its tile band widened (default: every tile, the
    full inverse of Fig. 2 case 6): tiles outside the original band are zero."""
    from .workloads import ArrowheadTiles
    w_full = M.nt - 1 if w_full is None else w_full
    out = ArrowheadTiles(M.nt, M.b, w_full, M.a)
    for i, k in out.pattern():
        out.tiles[(i, k)] = M.tiles[(i, k)].copy() if (i, k) in M.tiles else np.zeros((out.rows(i), out.rows(k)))
    return out

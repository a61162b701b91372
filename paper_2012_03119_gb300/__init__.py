"""GB300 clause x assignment tests (GpuShareSat's data-parallel path, arXiv 2012.03119).

Thin Python binding of the C ABI in ``include/gss.h`` (``libgss.so``, built in-tree
for sm_103a).  Functions keep the C names; ``Context`` wraps a ``gss_ctx*``.  The
binding only marshals arguments: every step of the path (clause ingest, packing,
testing, report compaction) runs in the library's CUDA kernels.  There is no CPU
fallback: importing fails loudly if the library is missing.

Inputs may be numpy arrays (host) or torch tensors (host or CUDA); torch is used
only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["Batch", "Context", "Server", "GssError", "REPORT_DTYPE", "expand_reports", "load", "GSS_MODE_ALLF", "GSS_MODE_TRIGGER"]

GSS_OK, GSS_E_INVAL, GSS_E_NOMEM, GSS_E_CUDA, GSS_E_OVERFLOW, GSS_E_TIMEOUT, GSS_E_BUSY, GSS_E_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
GSS_MODE_ALLF, GSS_MODE_TRIGGER = 0, 1
GSS_LAYOUT_IDENTITY, GSS_LAYOUT_FREQUENCY = 0, 1
GSS_MAX_ASSIGNMENTS = 32768
GSS_MAX_NARROW_ASSIGNMENTS = 4096
GSS_SUBMIT_KEEP = 1
GSS_WATERMARK_ALL = 0xFFFFFFFFFFFFFFFF
GSS_HEAD_WIDTH = 16

REPORT_DTYPE = np.dtype([("clause_id", "<u4"), ("word", "<u4"), ("mask", "<u4")])


class gss_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("report_capacity", ctypes.c_uint64),
                ("max_assignments", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("mem_budget_bytes", ctypes.c_uint64), ("layout", ctypes.c_uint32), ("pipeline", ctypes.c_uint32),
                ("pack_stream", ctypes.c_void_p), ("clauses_per_tile", ctypes.c_uint32)]


class gss_stats(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_uint32), ("n_assign", ctypes.c_uint32), ("n_clauses", ctypes.c_uint64),
                ("n_lits", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64), ("report_capacity", ctypes.c_uint64),
                ("tests_run", ctypes.c_uint64), ("pair_tests", ctypes.c_uint64),
                ("candidate_pairs", ctypes.c_uint64), ("group_pairs", ctypes.c_uint64),
                ("clauses_removed", ctypes.c_uint64), ("next_clause_id", ctypes.c_uint64),
                ("records", ctypes.c_uint64), ("overflows", ctypes.c_uint64), ("super_pairs", ctypes.c_uint64)]


class gss_batch_info(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_uint32), ("n_groups", ctypes.c_uint32),
                ("tiles_per_steal", ctypes.c_uint32 * 3), ("grid", ctypes.c_uint32 * 3),
                ("n_tiles", ctypes.c_uint64 * 3), ("runs", ctypes.c_uint64), ("tuned_test_us", ctypes.c_float),
                ("clauses_per_tile", ctypes.c_uint32 * 3)]


class gss_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mode", ctypes.c_uint32), ("layout", ctypes.c_uint32),
                ("max_clauses", ctypes.c_uint64), ("max_lits", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("lanes", ctypes.c_uint32), ("lane_report_capacity", ctypes.c_uint64),
                ("slot_memory_bytes", ctypes.c_uint64), ("tests_in_flight", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("result_ttl_us", ctypes.c_uint64)]


class gss_request_info(ctypes.Structure):
    _fields_ = [("watermark", ctypes.c_uint64), ("n_assign", ctypes.c_uint32), ("batch_words", ctypes.c_uint32),
                ("latency_us", ctypes.c_double), ("admit_us", ctypes.c_double), ("queue_us", ctypes.c_double),
                ("run_us", ctypes.c_double)]


class gss_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("dropped", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("words_launched", ctypes.c_uint64), ("pair_tests", ctypes.c_uint64),
                ("reports", ctypes.c_uint64), ("committed_clauses", ctypes.c_uint64), ("expired", ctypes.c_uint64),
                ("slots", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("next_clause_id", ctypes.c_uint64),
                ("reductions", ctypes.c_uint64), ("clauses_removed", ctypes.c_uint64)]


class GssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STRERR.get(code, code)}: {msg}")
        self.code = code


_STRERR = {0: "GSS_OK", -1: "GSS_E_INVAL", -2: "GSS_E_NOMEM", -3: "GSS_E_CUDA", -4: "GSS_E_OVERFLOW",
           -5: "GSS_E_TIMEOUT", -6: "GSS_E_BUSY", -7: "GSS_E_STATE"}

_lib = None

# (name, restype, argtypes) of every entry point declared in include/gss.h
P, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
SIGNATURES = {
    "gss_config_init": (i32, [P]),
    "gss_create": (i32, [P, u32, P]),
    "gss_destroy": (i32, [P]),
    "gss_add_clauses": (i32, [P, P, u64, P, P]),
    "gss_set_assignments": (i32, [P, P, u32]),
    "gss_set_assignments_device": (i32, [P, P, u64, u32]),
    "gss_set_assignments_async": (i32, [P, P, u32]),
    "gss_copy_wait": (i32, [P]),
    "gss_test": (i32, [P]),
    "gss_fetch_reports": (i32, [P, P, u64, P]),
    "gss_report_count": (i32, [P, P]),
    "gss_reports_device": (i32, [P, P, P]),
    "gss_set_report_capacity": (i32, [P, u64]),
    "gss_set_mode": (i32, [P, u32]),
    "gss_get_stats": (i32, [P, P]),
    "gss_last_error": (ctypes.c_char_p, [P]),
    "gss_strerror": (ctypes.c_char_p, [i32]),
    "gss_version": (u32, []),
    "gss_batch_create": (i32, [P, P]),
    "gss_batch_destroy": (i32, [P]),
    "gss_batch_add_instance": (i32, [P, u32, u32, u64, P, u64, P, P]),
    "gss_batch_set_assignments": (i32, [P, u32, P, u32]),
    "gss_batch_set_assignments_device": (i32, [P, u32, P, u64, u32]),
    "gss_batch_test": (i32, [P]),
    "gss_batch_report_count": (i32, [P, u32, P]),
    "gss_batch_fetch_reports": (i32, [P, u32, P, u64, P]),
    "gss_batch_get_info": (i32, [P, P]),
    "gss_batch_last_error": (ctypes.c_char_p, [P]),
    "gss_test_noalloc": (i32, [P, u64, P, u32, P, u64, u32, u32, P, u64, P, P, P, ctypes.c_size_t]),
    "gss_set_activity": (i32, [P, ctypes.c_float]),
    "gss_get_activity": (i32, [P, P, u64, P]),
    "gss_get_clause_ids": (i32, [P, P, u64, P]),
    "gss_reduce_db": (i32, [P, ctypes.c_double, P]),
    "gss_export_clauses": (i32, [P, P, u64, P, u64, P, P, P]),
    "gss_debug_bounds": (i32, [P, P, i32]),
    "gss_server_config_init": (i32, [P]),
    "gss_server_create": (i32, [P, u32, P]),
    "gss_server_destroy": (i32, [P]),
    "gss_server_add_clauses": (i32, [P, P, u64, P, P]),
    "gss_server_submit": (i32, [P, P, u32, u64, ctypes.c_int64, u32, P]),
    "gss_server_wait": (i32, [P, u64, ctypes.c_int64, P, u64, P, P]),
    "gss_server_get_stats": (i32, [P, P]),
    "gss_server_last_error": (ctypes.c_char_p, [P]),
    "gss_fetch_reports_async": (i32, [P, P, u64]),
    "gss_fetch_wait": (i32, [P, P]),
    "gss_server_set_activity": (i32, [P, ctypes.c_float]),
    "gss_server_reduce": (i32, [P, ctypes.c_double, P]),
    "gss_server_get_activity": (i32, [P, P, u64, P]),
    "gss_server_get_clause_ids": (i32, [P, P, u64, P]),
}


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libgss.so (in-tree).  Raises ImportError when it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx_ptr, rc: int):
    if rc != GSS_OK:
        msg = load().gss_last_error(ctx_ptr)
        raise GssError(rc, msg.decode() if msg else "")


def _host_or_dev(a, dtype):
    """Return (pointer, keepalive, is_device) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            assert a.is_contiguous(), "tensor must be contiguous"
            return ctypes.c_void_p(a.data_ptr()), a, a.is_cuda
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr, False


# ---------------------------------------------------------------- C-named wrappers
def gss_config_init() -> gss_config:
    cfg = gss_config()
    load().gss_config_init(ctypes.byref(cfg))
    return cfg


def gss_create(n_vars: int, cfg: gss_config | None = None) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    rc = load().gss_create(ctypes.byref(out), n_vars, ctypes.byref(cfg) if cfg is not None else None)
    if rc != GSS_OK:
        raise GssError(rc, "gss_create failed")
    return out


def gss_destroy(ctx) -> None:
    load().gss_destroy(ctx)


def gss_add_clauses(ctx, offsets, lits) -> int:
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    lt = np.ascontiguousarray(lits, dtype=np.uint32)
    first = ctypes.c_uint32()
    n = len(off) - 1
    _check(ctx, load().gss_add_clauses(ctx, ctypes.c_void_p(off.ctypes.data), n, ctypes.c_void_p(lt.ctypes.data),
                                       ctypes.byref(first)))
    return first.value


def gss_set_assignments(ctx, values) -> None:
    ptr, keep, dev = _host_or_dev(values, np.uint8)
    n = keep.shape[0] if keep.ndim == 2 else 0
    if dev:
        pitch = keep.stride(0) * keep.element_size()
        _check(ctx, load().gss_set_assignments_device(ctx, ptr, pitch, n))
    else:
        _check(ctx, load().gss_set_assignments(ctx, ptr, n))


def gss_set_assignments_async(ctx, values) -> object:
    """Queue the copy of host ``values`` and return; the returned keepalive (and ``values``)
    must stay unchanged until gss_copy_wait."""
    ptr, keep, dev = _host_or_dev(values, np.uint8)
    if dev:
        raise ValueError("gss_set_assignments_async takes host values; device values: gss_set_assignments_device")
    n = keep.shape[0] if keep.ndim == 2 else 0
    _check(ctx, load().gss_set_assignments_async(ctx, ptr, n))
    return keep


def gss_copy_wait(ctx) -> None:
    _check(ctx, load().gss_copy_wait(ctx))


def gss_set_assignments_device(ctx, d_ptr: int, pitch: int, n_assign: int) -> None:
    _check(ctx, load().gss_set_assignments_device(ctx, ctypes.c_void_p(d_ptr), pitch, n_assign))


def gss_test(ctx) -> None:
    _check(ctx, load().gss_test(ctx))


def gss_report_count(ctx) -> int:
    n = ctypes.c_uint64()
    _check(ctx, load().gss_report_count(ctx, ctypes.byref(n)))
    return n.value


def gss_fetch_reports(ctx, out: np.ndarray | None = None) -> np.ndarray:
    """Wait for the last test and return its records (numpy REPORT_DTYPE).  ``out`` may be a
    preallocated buffer (e.g. a numpy view of pinned memory) large enough for every record."""
    lib = load()
    n = ctypes.c_uint64()
    if out is None:
        rc = lib.gss_fetch_reports(ctx, None, 0, ctypes.byref(n))  # count only
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            _check(ctx, rc)
        out = np.empty(n.value, dtype=REPORT_DTYPE)
    assert out.dtype == REPORT_DTYPE and out.flags["C_CONTIGUOUS"]
    _check(ctx, lib.gss_fetch_reports(ctx, ctypes.c_void_p(out.ctypes.data), len(out), ctypes.byref(n)))
    return out[: n.value]


def gss_set_report_capacity(ctx, cap: int) -> None:
    _check(ctx, load().gss_set_report_capacity(ctx, cap))


def gss_set_mode(ctx, mode: int) -> None:
    _check(ctx, load().gss_set_mode(ctx, mode))


def gss_get_stats(ctx) -> dict:
    s = gss_stats()
    _check(ctx, load().gss_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


def gss_reports_device(ctx) -> tuple[int, int]:
    p = ctypes.c_void_p()
    cap = ctypes.c_uint64()
    _check(ctx, load().gss_reports_device(ctx, ctypes.byref(p), ctypes.byref(cap)))
    return p.value or 0, cap.value


def gss_test_noalloc(d_offsets: int, n_clauses: int, d_lits: int, n_vars: int, d_values: int, pitch: int,
                     n_assign: int, mode: int, d_out: int, cap: int, d_count: int, stream: int = 0) -> None:
    """The whole test on caller-owned device buffers, allocating nothing (see include/gss.h).
    Arguments are device addresses (ints); raises GssError on failure."""
    buf = ctypes.create_string_buffer(256)
    rc = load().gss_test_noalloc(ctypes.c_void_p(d_offsets), n_clauses, ctypes.c_void_p(d_lits), n_vars,
                                 ctypes.c_void_p(d_values), pitch, n_assign, mode, ctypes.c_void_p(d_out), cap,
                                 ctypes.c_void_p(d_count), ctypes.c_void_p(stream), buf, len(buf))
    if rc != GSS_OK:
        raise GssError(rc, buf.value.decode())


def gss_debug_bounds(reset: bool = False) -> tuple[bool, int]:
    """(bounds-checked build?, index violations counted on the current device)."""
    en, n = ctypes.c_uint32(), ctypes.c_uint64()
    rc = load().gss_debug_bounds(ctypes.byref(en), ctypes.byref(n), 1 if reset else 0)
    if rc != GSS_OK:
        raise GssError(rc, "gss_debug_bounds failed")
    return bool(en.value), n.value


def gss_strerror(code: int) -> str:
    return load().gss_strerror(code).decode()


def gss_version() -> int:
    return load().gss_version()


# ---------------------------------------------------------------- object API
class Context:
    """Owns one ``gss_ctx``: a resident clause database, one assignment set and a report buffer."""

    def __init__(self, n_vars: int, device: int = 0, stream=None, report_capacity: int = 1 << 22,
                 max_assignments: int = 1024, mode: int = GSS_MODE_ALLF, mem_budget_bytes: int = 0,
                 layout: int = GSS_LAYOUT_FREQUENCY, pipeline: int = 1, pack_stream=None,
                 clauses_per_tile: int = 0):
        cfg = gss_config_init()
        cfg.device = device
        cfg.stream = ctypes.c_void_p(_stream_handle(stream)) if stream is not None else None
        cfg.pipeline = pipeline
        cfg.clauses_per_tile = clauses_per_tile
        cfg.pack_stream = ctypes.c_void_p(_stream_handle(pack_stream)) if pack_stream is not None else None
        self._pack_stream = pack_stream
        cfg.report_capacity = report_capacity
        cfg.max_assignments = max_assignments
        cfg.mode = mode
        cfg.mem_budget_bytes = mem_budget_bytes
        cfg.layout = layout
        self.n_vars = n_vars
        self._stream = stream
        self.ptr = gss_create(n_vars, cfg)

    def close(self):
        if getattr(self, "ptr", None):
            gss_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_clauses(self, offsets, lits) -> int:
        return gss_add_clauses(self.ptr, offsets, lits)

    def set_assignments(self, values) -> None:
        gss_set_assignments(self.ptr, values)

    def set_assignments_async(self, values) -> None:
        """As set_assignments, but returns once the copy is queued: ``values`` must stay
        unchanged until copy_wait (pinned memory lets the copy run meanwhile)."""
        keep = gss_set_assignments_async(self.ptr, values)
        self.__dict__.setdefault("_copy_keep", []).append(keep)

    def copy_wait(self) -> None:
        """Wait until every queued host copy has read its values."""
        gss_copy_wait(self.ptr)
        self.__dict__.pop("_copy_keep", None)

    def test(self) -> None:
        gss_test(self.ptr)

    def report_count(self) -> int:
        return gss_report_count(self.ptr)

    def fetch_reports(self, out=None) -> np.ndarray:
        return gss_fetch_reports(self.ptr, out)

    def fetch_reports_async(self, out: np.ndarray) -> None:
        """Queue the copy of the last test's records into ``out`` (REPORT_DTYPE, memory the GPU
        can write, e.g. a numpy view of pinned memory); ``fetch_wait`` finishes it."""
        assert out.dtype == REPORT_DTYPE and out.flags["C_CONTIGUOUS"]
        self._fetch_out = out
        _check(self.ptr, load().gss_fetch_reports_async(self.ptr, ctypes.c_void_p(out.ctypes.data), len(out)))

    def fetch_wait(self) -> np.ndarray:
        """Wait for fetch_reports_async; returns the records (a view of its buffer)."""
        n = ctypes.c_uint64()
        _check(self.ptr, load().gss_fetch_wait(self.ptr, ctypes.byref(n)))
        out, self._fetch_out = self._fetch_out, None
        return out[: n.value]

    def set_report_capacity(self, cap: int) -> None:
        gss_set_report_capacity(self.ptr, cap)

    def set_mode(self, mode: int) -> None:
        gss_set_mode(self.ptr, mode)

    def stats(self) -> dict:
        return gss_get_stats(self.ptr)

    def set_activity(self, decay: float) -> None:
        _check(self.ptr, load().gss_set_activity(self.ptr, decay))

    def activity(self) -> np.ndarray:
        n = ctypes.c_uint64()
        rc = load().gss_get_activity(self.ptr, None, 0, ctypes.byref(n))
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            _check(self.ptr, rc)
        out = np.empty(n.value, np.float32)
        _check(self.ptr, load().gss_get_activity(self.ptr, ctypes.c_void_p(out.ctypes.data), len(out),
                                                 ctypes.byref(n)))
        return out

    def clause_ids(self) -> np.ndarray:
        n = ctypes.c_uint64()
        rc = load().gss_get_clause_ids(self.ptr, None, 0, ctypes.byref(n))
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            _check(self.ptr, rc)
        out = np.empty(n.value, np.uint32)
        _check(self.ptr, load().gss_get_clause_ids(self.ptr, ctypes.c_void_p(out.ctypes.data), len(out),
                                                   ctypes.byref(n)))
        return out

    def export_clauses(self):
        """(offsets, lits, ids) of the resident clauses, in the caller's variable numbering."""
        n, L = ctypes.c_uint64(), ctypes.c_uint64()
        rc = load().gss_export_clauses(self.ptr, None, 0, None, 0, None, ctypes.byref(n), ctypes.byref(L))
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            _check(self.ptr, rc)
        off = np.empty(n.value + 1, np.uint64)
        lits = np.empty(max(1, L.value), np.uint32)
        ids = np.empty(max(1, n.value), np.uint32)
        _check(self.ptr, load().gss_export_clauses(self.ptr, ctypes.c_void_p(off.ctypes.data), n.value,
                                                   ctypes.c_void_p(lits.ctypes.data), L.value,
                                                   ctypes.c_void_p(ids.ctypes.data), ctypes.byref(n), ctypes.byref(L)))
        return off, lits[: L.value], ids[: n.value]

    def reduce_db(self, remove_fraction: float) -> int:
        n = ctypes.c_uint64()
        _check(self.ptr, load().gss_reduce_db(self.ptr, remove_fraction, ctypes.byref(n)))
        return n.value

    def run(self, values) -> np.ndarray:
        """set_assignments + test + fetch_reports."""
        self.set_assignments(values)
        self.test()
        return self.fetch_reports()


def _stream_handle(stream) -> int:
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def expand_reports(rec: np.ndarray) -> np.ndarray:
    """Records -> (clause, assignment) pairs sorted by clause then assignment (uint32 [R, 2])."""
    rec = np.asarray(rec)
    if len(rec) == 0:
        return np.zeros((0, 2), np.uint32)
    bits = np.unpackbits(rec["mask"].astype("<u4").view(np.uint8).reshape(-1, 4), axis=1, bitorder="little")
    r, j = np.nonzero(bits)
    c = rec["clause_id"][r].astype(np.uint64)
    a = rec["word"][r].astype(np.uint64) * 32 + j.astype(np.uint64)
    key = np.sort((c << np.uint64(32)) | a)
    out = np.empty((len(key), 2), np.uint32)
    out[:, 0] = (key >> np.uint64(32)).astype(np.uint32)
    out[:, 1] = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


# ---------------------------------------------------------------- batches
class Batch:
    """Many independent clause databases tested together (gss_batch_*): one CUDA graph per run,
    per-instance packing on parallel branches and one work-stealing test launch."""

    def __init__(self, device: int = 0, stream=None, mode: int = GSS_MODE_ALLF, layout: int = GSS_LAYOUT_FREQUENCY):
        cfg = gss_config_init()
        cfg.device = device
        cfg.stream = ctypes.c_void_p(_stream_handle(stream)) if stream is not None else None
        cfg.mode = mode
        cfg.layout = layout
        self._stream = stream
        self.ptr = ctypes.c_void_p()
        rc = load().gss_batch_create(ctypes.byref(self.ptr), ctypes.byref(cfg))
        if rc != GSS_OK:
            raise GssError(rc, "gss_batch_create failed")
        self._keep = {}

    def _check(self, rc):
        if rc != GSS_OK:
            msg = load().gss_batch_last_error(self.ptr)
            raise GssError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ptr", None):
            load().gss_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_instance(self, n_vars, offsets, lits, max_assignments=1024, report_capacity=0) -> int:
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        lt = np.ascontiguousarray(lits, dtype=np.uint32)
        out = ctypes.c_uint32()
        self._check(load().gss_batch_add_instance(self.ptr, n_vars, max_assignments, report_capacity,
                                                  ctypes.c_void_p(off.ctypes.data), len(off) - 1,
                                                  ctypes.c_void_p(lt.ctypes.data), ctypes.byref(out)))
        return out.value

    def set_assignments(self, i: int, values) -> None:
        ptr, keep, dev = _host_or_dev(values, np.uint8)
        n = keep.shape[0] if keep.ndim == 2 else 0
        if dev:
            self._keep[i] = keep  # the graph reads it on every run
            pitch = keep.stride(0) * keep.element_size()
            self._check(load().gss_batch_set_assignments_device(self.ptr, i, ptr, pitch, n))
        else:
            self._check(load().gss_batch_set_assignments(self.ptr, i, ptr, n))

    def test(self) -> None:
        self._check(load().gss_batch_test(self.ptr))

    def report_count(self, i: int) -> int:
        n = ctypes.c_uint64()
        self._check(load().gss_batch_report_count(self.ptr, i, ctypes.byref(n)))
        return n.value

    def fetch_reports(self, i: int) -> np.ndarray:
        n = ctypes.c_uint64()
        rc = load().gss_batch_fetch_reports(self.ptr, i, None, 0, ctypes.byref(n))
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            self._check(rc)
        out = np.empty(n.value, dtype=REPORT_DTYPE)
        self._check(load().gss_batch_fetch_reports(self.ptr, i, ctypes.c_void_p(out.ctypes.data), len(out),
                                                   ctypes.byref(n)))
        return out[: n.value]

    def info(self) -> dict:
        x = gss_batch_info()
        self._check(load().gss_batch_get_info(self.ptr, ctypes.byref(x)))
        k = x.n_groups
        return {"n_instances": x.n_instances, "n_groups": k, "tiles_per_steal": list(x.tiles_per_steal)[:k],
                "grid": list(x.grid)[:k], "n_tiles": list(x.n_tiles)[:k], "runs": x.runs,
                "tuned_test_us": x.tuned_test_us, "clauses_per_tile": list(x.clauses_per_tile)[:k]}


# ---------------------------------------------------------------- serving
class Server:
    """A resident, growing clause database serving 32-assignment requests (gss_server_*):
    slot admission, a scheduler thread batching the waiting requests into overlapping
    launches, per-request watermarks.  Methods may be called from several threads (the
    library releases the GIL inside each call)."""

    def __init__(self, n_vars: int, device: int = 0, mode: int = GSS_MODE_ALLF, layout: int = GSS_LAYOUT_FREQUENCY,
                 max_clauses: int = 1 << 20, max_lits: int = 1 << 24, slots: int = 64, lanes: int = 3,
                 lane_report_capacity: int = 1 << 20, slot_memory_bytes: int = 0, tests_in_flight: int = 1,
                 result_ttl_us: int = 0):
        cfg = gss_server_config()
        load().gss_server_config_init(ctypes.byref(cfg))
        cfg.device, cfg.mode, cfg.layout = device, mode, layout
        cfg.max_clauses, cfg.max_lits, cfg.slots, cfg.lanes = max_clauses, max_lits, slots, lanes
        cfg.lane_report_capacity, cfg.slot_memory_bytes = lane_report_capacity, slot_memory_bytes
        cfg.tests_in_flight = tests_in_flight
        cfg.result_ttl_us = result_ttl_us
        self.n_vars = n_vars
        self.ptr = ctypes.c_void_p()
        rc = load().gss_server_create(ctypes.byref(self.ptr), n_vars, ctypes.byref(cfg))
        if rc != GSS_OK:
            self.ptr = None
            raise GssError(rc, "gss_server_create failed")

    def _check(self, rc):
        if rc != GSS_OK:
            msg = load().gss_server_last_error(self.ptr)
            raise GssError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ptr", None):
            load().gss_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_clauses(self, offsets, lits) -> int:
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        lt = np.ascontiguousarray(lits, dtype=np.uint32)
        out = ctypes.c_uint32()
        self._check(load().gss_server_add_clauses(self.ptr, ctypes.c_void_p(off.ctypes.data), len(off) - 1,
                                                  ctypes.c_void_p(lt.ctypes.data), ctypes.byref(out)))
        return out.value

    def submit(self, values, watermark: int | None = None, wait_us: int = 0, keep: bool = True) -> int | None:
        """Submit rows of value codes (host, [n <= 32][n_vars] uint8).  Returns the request id,
        or None when no slot freed up within wait_us (GSS_E_BUSY)."""
        ptr, arr, dev = _host_or_dev(values, np.uint8)
        if dev:
            raise ValueError("requests are host memory")
        if arr.ndim != 2 or arr.shape[1] != self.n_vars:
            raise ValueError(f"values must be [n_assign][{self.n_vars}]")
        rid = ctypes.c_uint64()
        wm = GSS_WATERMARK_ALL if watermark is None else watermark
        rc = load().gss_server_submit(self.ptr, ptr, arr.shape[0], wm, wait_us, GSS_SUBMIT_KEEP if keep else 0,
                                      ctypes.byref(rid))
        if rc == GSS_E_BUSY:
            return None
        self._check(rc)
        return rid.value

    def wait(self, request_id: int, wait_us: int = -1):
        """Records (REPORT_DTYPE, word 0) and info of a kept request; None if not finished in wait_us."""
        n = ctypes.c_uint64()
        info = gss_request_info()
        out = np.empty(64, dtype=REPORT_DTYPE)
        while True:
            rc = load().gss_server_wait(self.ptr, request_id, wait_us, ctypes.c_void_p(out.ctypes.data), len(out),
                                        ctypes.byref(n), ctypes.byref(info))
            if rc == GSS_E_TIMEOUT:
                return None
            if rc == GSS_E_OVERFLOW and n.value > len(out):
                out = np.empty(n.value, dtype=REPORT_DTYPE)
                continue
            self._check(rc)
            return out[: n.value].copy(), {k: getattr(info, k) for k, _ in info._fields_}

    def stats(self) -> dict:
        x = gss_server_stats()
        self._check(load().gss_server_get_stats(self.ptr, ctypes.byref(x)))
        return {k: getattr(x, k) for k, _ in x._fields_ if k != "pad"}

    def set_activity(self, decay: float) -> None:
        self._check(load().gss_server_set_activity(self.ptr, decay))

    def reduce(self, remove_fraction: float) -> int:
        n = ctypes.c_uint64()
        self._check(load().gss_server_reduce(self.ptr, remove_fraction, ctypes.byref(n)))
        return n.value

    def _per_clause(self, fn, dtype) -> np.ndarray:
        n = ctypes.c_uint64()
        rc = fn(self.ptr, None, 0, ctypes.byref(n))
        if rc not in (GSS_OK, GSS_E_OVERFLOW):
            self._check(rc)
        out = np.empty(n.value, dtype)
        self._check(fn(self.ptr, ctypes.c_void_p(out.ctypes.data), len(out), ctypes.byref(n)))
        return out

    def activity(self) -> np.ndarray:
        """Activities of the resident clauses, in position order."""
        return self._per_clause(load().gss_server_get_activity, np.float32)

    def clause_ids(self) -> np.ndarray:
        """Ids of the resident clauses, in position order."""
        return self._per_clause(load().gss_server_get_clause_ids, np.uint32)

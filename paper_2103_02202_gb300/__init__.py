"""GB300-native bulk stabilizer-circuit sampler (the bulk-sampling path of
Gidney, "Stim: a fast stabilizer circuit simulator", Quantum 2021).

This module is a thin ctypes binding of the C ABI in ``include/stimgb.h``:
the functions ``stim_compile``, ``stim_info_get``, ``stim_reference_sample``,
``stim_frame_sample``, ``stim_frame_sample_ex``, ``stim_free`` and
``stim_last_error`` take the same arguments as their C counterparts (device
or host pointers as integers, a CUDA stream handle as an integer) and only
marshal arguments; every step of the path runs in the CUDA library. The
``Circuit`` class wraps them with torch tensors for convenience.

The library is built in-tree by ``paper_2103_02202_gb300.build`` (or
``__graft_entry__.build()``). Importing this package does not load it;
the first call does, and raises ``RuntimeError`` if it has not been built --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (seeded input generators)

__all__ = [
    "STIM_OK", "STIM_E_PARSE", "STIM_E_INVALID_ARG", "STIM_E_OOM", "STIM_E_CUDA",
    "STIM_E_TIMEOUT", "STIM_E_BUSY", "STIM_E_UNSUPPORTED", "STIM_E_CAPACITY", "STIM_ASYNC", "STIM_EVENTS_IN_KERNEL",
    "stim_frame_sample_detections",
    "STIM_MEAS_MAJOR", "STIM_SHOT_MAJOR", "STIM_DEVICE", "STIM_HOST", "STIM_RECOMPUTE",
    "StimError", "library", "library_path", "stim_compile", "stim_info_get", "stim_frame_program_info_get",
    "stim_free",
    "stim_last_error", "stim_reference_sample", "stim_reference_many", "stim_reference_cache_set",
    "stim_reference_cache_stats", "stim_prefix_cache_set", "stim_prefix_cache_stats", "stim_debug_fail_allocations", "stim_debug_tableau_barrier", "stim_probe_smem_bandwidth", "stim_frame_sample", "stim_frame_sample_ex",
    "Circuit", "EXPORTED_SYMBOLS", "stim_frame_sample_noalloc", "stim_batch_create", "stim_batch_sample",
    "stim_batch_info", "stim_batch_free", "Batch", "Server", "STIM_OUT_MEAS", "STIM_OUT_DET", "stim_profile", "stim_profile_read", "KERNEL_NAMES",
]

STIM_OK = 0
STIM_E_PARSE = -1
STIM_E_INVALID_ARG = -2
STIM_E_OOM = -3
STIM_E_CUDA = -4
STIM_E_TIMEOUT = -5
STIM_E_BUSY = -6
STIM_E_UNSUPPORTED = -7
STIM_E_CAPACITY = -8

STIM_MEAS_MAJOR = 0x0
STIM_SHOT_MAJOR = 0x1
STIM_DEVICE = 0x0
STIM_HOST = 0x2
STIM_RECOMPUTE = 0x4
STIM_ASYNC = 0x8
STIM_EVENTS_IN_KERNEL = 0x10

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libstimgb.so")
_lock = threading.Lock()
_lib = None


class StimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("stimgb error %d: %s" % (code, msg))
        self.code = code


class StimInfo(ctypes.Structure):
    _fields_ = [("num_qubits", ctypes.c_uint32), ("num_measurements", ctypes.c_uint64),
                ("num_detectors", ctypes.c_uint64), ("num_gate_targets", ctypes.c_uint64),
                ("num_noise_targets", ctypes.c_uint64), ("num_instructions", ctypes.c_uint64),
                ("num_layers", ctypes.c_uint64), ("num_program_layers", ctypes.c_uint64),
                ("num_observables", ctypes.c_uint64), ("reference_key", ctypes.c_uint64),
                ("flip_ring_rows", ctypes.c_uint64)]


class StimFrameProgramInfo(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_uint32), ("qubits_per_cta", ctypes.c_uint32),
                ("merged_layers", ctypes.c_uint64), ("stored_layers", ctypes.c_uint64),
                ("segments", ctypes.c_uint64), ("chains", ctypes.c_uint64), ("ops", ctypes.c_uint64),
                ("max_chain_ops", ctypes.c_uint32), ("max_cta_ops", ctypes.c_uint32),
                ("deferred_ops", ctypes.c_uint64), ("tails_repeating_qubit", ctypes.c_uint64),
                ("feedforward_not_first", ctypes.c_uint64)]


class StimTileHint(ctypes.Structure):
    _fields_ = [("words_per_cta", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("frame_in_global", ctypes.c_uint32), ("cluster_size", ctypes.c_uint32)]


class StimKernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


KERNEL_NAMES = ("frame", "detectors", "transpose", "tableau")

class StimResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("num_shots", ctypes.c_uint64), ("words_per_row", ctypes.c_uint64),
                ("meas", ctypes.c_void_p), ("det", ctypes.c_void_p), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double)]


class StimServerStatistics(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("running", ctypes.c_uint64), ("shots", ctypes.c_uint64), ("gate_shots", ctypes.c_double),
                ("budget_bytes", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes_in_use", ctypes.c_size_t), ("p50_latency_s", ctypes.c_double),
                ("p99_latency_s", ctypes.c_double), ("max_latency_s", ctypes.c_double),
                ("wall_s", ctypes.c_double)]


STIM_OUT_MEAS = 0x1
STIM_OUT_DET = 0x2

STIM_NOALLOC_SCRATCH_BYTES = 32 << 20

STIM_KERNEL_FRAME = 0
STIM_KERNEL_DETECTORS = 1
STIM_KERNEL_TRANSPOSE = 2
STIM_KERNEL_TABLEAU = 3
STIM_KERNEL_COUNT = 4

_VP = ctypes.c_void_p
_U64 = ctypes.c_uint64
# name -> (restype, argtypes); every entry is declared in include/stimgb.h
_SIGNATURES = {
    "stim_compile": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "stim_info_get": (ctypes.c_int, [_VP, ctypes.POINTER(StimInfo)]),
    "stim_frame_program_info_get": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(StimFrameProgramInfo)]),
    "stim_free": (None, [_VP]),
    "stim_last_error": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t]),
    "stim_reference_sample": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "stim_reference_many": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_size_t, ctypes.c_int]),
    "stim_reference_cache_set": (ctypes.c_int, [ctypes.c_size_t]),
    "stim_prefix_cache_set": (ctypes.c_int, [ctypes.c_size_t]),
    "stim_prefix_cache_stats": (ctypes.c_int, [ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                               ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "stim_debug_fail_allocations": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "stim_debug_tableau_barrier": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64]),
    "stim_probe_smem_bandwidth": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "stim_reference_cache_stats": (ctypes.c_int, [ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                                  ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "stim_frame_sample": (ctypes.c_int, [_VP, _U64, _U64, _VP, _VP, ctypes.c_int, _VP]),
    "stim_frame_sample_ex": (ctypes.c_int, [_VP, _U64, _U64, _U64, _VP, _VP, ctypes.c_int,
                                            ctypes.POINTER(StimTileHint), _VP]),
    "stim_frame_sample_noalloc": (ctypes.c_int, [_VP, _U64, _U64, _U64, _VP, _VP]),
    "stim_frame_sample_detections": (ctypes.c_int, [_VP, _U64, _U64, _U64, _VP, _VP, _U64,
                                                    ctypes.POINTER(_U64), ctypes.c_int, _VP]),
    "stim_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_U64), ctypes.c_size_t,
                                         ctypes.POINTER(StimTileHint), _VP, ctypes.POINTER(_VP)]),
    "stim_batch_sample": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                         ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    "stim_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(_U64)]),
    "stim_batch_free": (None, [_VP]),
    "stim_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_VP)]),
    "stim_server_submit": (ctypes.c_int, [_VP, _VP, _U64, _U64, _U64, ctypes.c_int, ctypes.POINTER(_U64)]),
    "stim_server_poll": (ctypes.c_int, [_VP, _U64, ctypes.POINTER(StimResult)]),
    "stim_server_wait": (ctypes.c_int, [_VP, _U64, _U64, ctypes.POINTER(StimResult)]),
    "stim_server_cancel": (ctypes.c_int, [_VP, _U64]),
    "stim_server_release": (ctypes.c_int, [_VP, _U64]),
    "stim_server_copy_result": (ctypes.c_int, [_VP, _U64, _VP, _VP, ctypes.c_int, _VP]),
    "stim_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(StimServerStatistics)]),
    "stim_server_destroy": (None, [_VP]),
    "stim_profile": (ctypes.c_int, [ctypes.c_int]),
    "stim_profile_read": (ctypes.c_int, [ctypes.POINTER(StimKernelStat), ctypes.c_int]),
}
EXPORTED_SYMBOLS = tuple(_SIGNATURES)


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load libstimgb.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError("libstimgb.so is not built (%s); run __graft_entry__.build() "
                                   "or python -m paper_2103_02202_gb300.build" % _LIB_PATH)
            L = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def stim_last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    library().stim_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != STIM_OK:
        raise StimError(rc, stim_last_error())


def stim_compile(text: str) -> int:
    """Compile circuit text; returns an opaque handle (int)."""
    b = text.encode()
    h = _VP()
    _check(library().stim_compile(b, len(b), ctypes.byref(h)))
    return h.value


def stim_info_get(handle: int) -> dict:
    info = StimInfo()
    _check(library().stim_info_get(handle, ctypes.byref(info)))
    return {k: int(getattr(info, k)) for k, _ in StimInfo._fields_}


def stim_frame_program_info_get(handle: int, cluster_size: int) -> dict:
    """Shape of the frame-kernel program for a cluster of cluster_size CTAs (host only)."""
    info = StimFrameProgramInfo()
    _check(library().stim_frame_program_info_get(handle, int(cluster_size), ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in StimFrameProgramInfo._fields_}


def stim_free(handle: int) -> None:
    if handle:
        library().stim_free(handle)


def stim_reference_sample(handle: int, ref_bits: int, det_bits: int = 0, flags: int = 0,
                          stream: int = 0) -> None:
    _check(library().stim_reference_sample(handle, ref_bits or None, det_bits or None, flags,
                                           stream or None))


def stim_reference_many(handles, flags: int = 0) -> None:
    """Reference samples of several circuits at once (small ones side by side)."""
    arr = (_VP * max(len(handles), 1))(*[h for h in handles])
    _check(library().stim_reference_many(arr, len(handles), flags))


def stim_probe_smem_bandwidth() -> tuple:
    """(local, cluster) shared-memory GB/s of the current device (see include/stimgb.h)."""
    lo, cl = ctypes.c_double(), ctypes.c_double()
    _check(library().stim_probe_smem_bandwidth(ctypes.byref(lo), ctypes.byref(cl)))
    return lo.value, cl.value


def stim_debug_tableau_barrier(extra_arrivals: int, timeout_ns: int) -> None:
    """Test knob: bounded tableau grid-barrier waits (see include/stimgb.h)."""
    _check(library().stim_debug_tableau_barrier(int(extra_arrivals), int(timeout_ns)))


def stim_debug_fail_allocations(skip: int, count: int) -> None:
    """Fault injection for tests: after `skip` more device allocations, the
    next `count` fail (STIM_E_OOM); count = 0 turns it off."""
    _check(library().stim_debug_fail_allocations(int(skip), int(count)))


def stim_reference_cache_set(budget_bytes: int) -> None:
    _check(library().stim_reference_cache_set(int(budget_bytes)))


def stim_reference_cache_stats() -> dict:
    v = [_U64() for _ in range(4)]
    _check(library().stim_reference_cache_stats(*[ctypes.byref(x) for x in v]))
    return dict(zip(("hits", "misses", "entries", "bytes"), (int(x.value) for x in v)))


def stim_prefix_cache_set(budget_bytes: int) -> None:
    """Device-byte budget of the stored tableau prefix states (0: off)."""
    _check(library().stim_prefix_cache_set(int(budget_bytes)))


def stim_prefix_cache_stats() -> dict:
    v = [_U64() for _ in range(4)]
    _check(library().stim_prefix_cache_stats(*[ctypes.byref(x) for x in v]))
    return dict(zip(("resumes", "saves", "entries", "bytes"), (int(x.value) for x in v)))


def stim_frame_sample(handle: int, num_shots: int, seed: int, meas_out: int = 0, det_out: int = 0,
                      flags: int = 0, stream: int = 0) -> None:
    _check(library().stim_frame_sample(handle, num_shots, seed & (2**64 - 1), meas_out or None,
                                       det_out or None, flags, stream or None))


def stim_frame_sample_detections(handle: int, num_shots: int, seed: int, shot_offset: int = 0,
                                 shot_begin: int = 0, detectors: int = 0, capacity: int = 0, flags: int = 0,
                                 stream: int = 0) -> int:
    """Per-shot lists of fired detectors; returns the total number of events.
    Raises StimError(STIM_E_CAPACITY) when `capacity` is too small."""
    cnt = _U64(0)
    rc = library().stim_frame_sample_detections(handle, num_shots, seed & (2**64 - 1), shot_offset,
                                                shot_begin or None, detectors or None, capacity,
                                                ctypes.byref(cnt), flags, stream or None)
    _check(rc)
    return int(cnt.value)


def stim_frame_sample_ex(handle: int, num_shots: int, seed: int, shot_offset: int = 0,
                         meas_out: int = 0, det_out: int = 0, flags: int = 0, hint=None,
                         stream: int = 0) -> None:
    h = None
    if hint is not None:
        hint = tuple(hint) + (0,) * (4 - len(hint))
        h = ctypes.byref(StimTileHint(*(int(v) for v in hint[:4])))
    _check(library().stim_frame_sample_ex(handle, num_shots, seed & (2**64 - 1), shot_offset,
                                          meas_out or None, det_out or None, flags, h,
                                          stream or None))


def stim_frame_sample_noalloc(handle: int, num_shots: int, seed: int, shot_offset: int = 0,
                              det_out: int = 0, stream: int = 0) -> None:
    """Detection events into device memory without any device allocation
    (records kept in the library's fixed 32 MiB array; see include/stimgb.h)."""
    _check(library().stim_frame_sample_noalloc(handle, num_shots, seed & (2**64 - 1), shot_offset,
                                               det_out or None, stream or None))


def _hint(hint):
    if hint is None:
        return None
    hint = tuple(hint) + (0,) * (4 - len(hint))
    return ctypes.byref(StimTileHint(*(int(v) for v in hint[:4])))


def stim_batch_create(handles, num_shots, hint=None, stream: int = 0) -> int:
    """Plan one persistent launch over circuits `handles` sampling num_shots[i] each."""
    k = len(handles)
    hs = (_VP * k)(*handles)
    ns = (_U64 * k)(*[int(x) for x in num_shots])
    out = _VP()
    _check(library().stim_batch_create(hs, ns, k, _hint(hint), stream or None, ctypes.byref(out)))
    return out.value


def stim_batch_sample(plan: int, seeds, shot_offsets=None, meas_out=None, det_out=None, stream: int = 0) -> None:
    k = len(seeds)
    sd = (_U64 * k)(*[int(x) & (2**64 - 1) for x in seeds])
    off = (_U64 * k)(*[int(x) for x in shot_offsets]) if shot_offsets is not None else None
    mo = (_VP * k)(*[p or None for p in meas_out]) if meas_out is not None else None
    do = (_VP * k)(*[p or None for p in det_out]) if det_out is not None else None
    _check(library().stim_batch_sample(plan, sd, off, mo, do, stream or None))


def stim_batch_info(plan: int) -> dict:
    w, t, c, ctas = (ctypes.c_uint32() for _ in range(4))
    items = _U64()
    _check(library().stim_batch_info(plan, ctypes.byref(w), ctypes.byref(t), ctypes.byref(c), ctypes.byref(ctas),
                                     ctypes.byref(items)))
    return dict(words_per_tile=w.value, threads=t.value, cluster_size=c.value, ctas=ctas.value,
                work_items=items.value)


def stim_batch_free(plan: int) -> None:
    if plan:
        library().stim_batch_free(plan)


def stim_profile(enable: bool) -> None:
    """Start (clearing statistics) or stop per-kernel event timing."""
    _check(library().stim_profile(1 if enable else 0))


def stim_profile_read() -> dict:
    """{kernel name: (launches, total device ms)} since the last stim_profile(True)."""
    n = len(KERNEL_NAMES)
    arr = (StimKernelStat * n)()
    _check(library().stim_profile_read(arr, n))
    return {KERNEL_NAMES[k]: (int(arr[k].launches), float(arr[k].total_ms)) for k in range(n)}


def _words(bits: int) -> int:
    return (bits + 63) // 64


class Circuit:
    """Compiled circuit with torch-tensor helpers (outputs are int64 tensors
    holding uint64 bit words; use ``.cpu().numpy().view(np.uint64)``)."""

    def __init__(self, text: str):
        self.handle = stim_compile(text)
        self.info = stim_info_get(self.handle)
        self.num_qubits = self.info["num_qubits"]
        self.num_measurements = self.info["num_measurements"]
        self.num_detectors = self.info["num_detectors"]
        self.num_observables = self.info["num_observables"]
        # rows of a detection-event output: the detectors, then the observables
        self.num_detector_rows = self.num_detectors + self.num_observables

    def close(self):
        if getattr(self, "handle", None):
            stim_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reference(self, *, recompute: bool = False, stream=None):
        """(ref_words, deterministic_words) as device int64 tensors."""
        import torch
        w = max(_words(self.num_measurements), 1)
        ref = torch.zeros(w, dtype=torch.int64, device="cuda")
        det = torch.zeros(w, dtype=torch.int64, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        stim_reference_sample(self.handle, ref.data_ptr(), det.data_ptr(),
                              STIM_RECOMPUTE if recompute else 0, s.cuda_stream)
        return ref, det

    def sample(self, num_shots: int, seed: int, *, shot_offset: int = 0, shot_major: bool = False,
               meas: bool = True, dets: bool = True, hint=None, stream=None, events_in_kernel: bool = False):
        """Sample on the device; returns (meas, dets) int64 tensors (None when not asked).
        events_in_kernel: with dets only, ask for STIM_EVENTS_IN_KERNEL."""
        import torch
        M, D = self.num_measurements, self.num_detector_rows
        if shot_major:
            ms = (num_shots, _words(M))
            ds = (num_shots, _words(D))
        else:
            ms = (M, _words(num_shots))
            ds = (D, _words(num_shots))
        mt = torch.empty(ms, dtype=torch.int64, device="cuda") if meas else None
        dt = torch.empty(ds, dtype=torch.int64, device="cuda") if dets else None
        s = stream if stream is not None else torch.cuda.current_stream()
        flags = STIM_SHOT_MAJOR if shot_major else STIM_MEAS_MAJOR
        if events_in_kernel:
            flags |= STIM_EVENTS_IN_KERNEL
        stim_frame_sample_ex(self.handle, num_shots, seed, shot_offset,
                             mt.data_ptr() if mt is not None and mt.numel() else 0,
                             dt.data_ptr() if dt is not None and dt.numel() else 0,
                             flags, hint, s.cuda_stream)
        return mt, dt

    def sample_host(self, num_shots: int, seed: int, *, shot_offset: int = 0, shot_major: bool = False,
                    meas: bool = True, dets: bool = True, hint=None):
        """Sample into host numpy uint64 arrays through the STIM_HOST path."""
        M, D = self.num_measurements, self.num_detector_rows
        if shot_major:
            ms, ds = (num_shots, _words(M)), (num_shots, _words(D))
        else:
            ms, ds = (M, _words(num_shots)), (D, _words(num_shots))
        ma = np.zeros(ms, np.uint64) if meas else None
        da = np.zeros(ds, np.uint64) if dets else None
        flags = STIM_HOST | (STIM_SHOT_MAJOR if shot_major else 0)
        stim_frame_sample_ex(self.handle, num_shots, seed, shot_offset,
                             ma.ctypes.data if ma is not None and ma.size else 0,
                             da.ctypes.data if da is not None and da.size else 0, flags, hint, 0)
        return ma, da


    def sample_detections(self, num_shots: int, seed: int, *, shot_offset: int = 0, capacity: int = 0):
        """Per-shot lists of fired detectors in host memory: returns
        (shot_begin uint64[num_shots + 1], detectors uint32[count]). With
        capacity 0 the count is taken first and the lists fetched second."""
        begin = np.zeros(num_shots + 1, np.uint64)
        if capacity <= 0:
            capacity = stim_frame_sample_detections(self.handle, num_shots, seed, shot_offset, 0, 0, 0, STIM_HOST, 0)
        dets = np.zeros(max(capacity, 1), np.uint32)
        n = stim_frame_sample_detections(self.handle, num_shots, seed, shot_offset, begin.ctypes.data,
                                         dets.ctypes.data, capacity, STIM_HOST, 0)
        return begin, dets[:n]


class Batch:
    """A persistent batched launch over several Circuit objects (device
    MEAS_MAJOR outputs as int64 tensors)."""

    def __init__(self, circuits, num_shots, hint=None, stream=None):
        import torch
        self.circuits = list(circuits)
        self.num_shots = [int(x) for x in num_shots]
        s = stream if stream is not None else torch.cuda.current_stream()
        self.plan = stim_batch_create([c.handle for c in self.circuits], self.num_shots, hint, s.cuda_stream)

    def info(self):
        return stim_batch_info(self.plan)

    def sample(self, seeds, shot_offsets=None, meas=True, dets=True, stream=None, out=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        if out is None:
            out = []
            for c, S in zip(self.circuits, self.num_shots):
                w = _words(S)
                m = torch.empty((c.num_measurements, w), dtype=torch.int64, device="cuda") \
                    if meas and c.num_measurements else None
                d = torch.empty((c.num_detector_rows, w), dtype=torch.int64, device="cuda") \
                    if dets and c.num_detector_rows else None
                out.append((m, d))
        stim_batch_sample(self.plan, seeds, shot_offsets,
                          [m.data_ptr() if m is not None else 0 for m, _ in out],
                          [d.data_ptr() if d is not None else 0 for _, d in out], s.cuda_stream)
        return out

    def close(self):
        if getattr(self, "plan", None):
            stim_batch_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching sampling server (see include/stimgb.h)."""

    def __init__(self, hbm_budget_bytes: int, streams: int = 0):
        out = _VP()
        _check(library().stim_server_create(int(hbm_budget_bytes), int(streams), ctypes.byref(out)))
        self.handle = out.value

    def submit(self, circuit, num_shots: int, seed: int, shot_offset: int = 0,
               outputs: int = STIM_OUT_MEAS | STIM_OUT_DET) -> int:
        rid = _U64()
        _check(library().stim_server_submit(self.handle, circuit.handle, int(num_shots), int(seed) & (2**64 - 1),
                                            int(shot_offset), int(outputs), ctypes.byref(rid)))
        return rid.value

    def poll(self, rid: int):
        r = StimResult()
        rc = library().stim_server_poll(self.handle, rid, ctypes.byref(r))
        return rc, r

    def wait(self, rid: int, timeout_s: float = 60.0):
        r = StimResult()
        rc = library().stim_server_wait(self.handle, rid, int(timeout_s * 1e9), ctypes.byref(r))
        if rc != STIM_OK:
            raise StimError(rc, stim_last_error())
        return r

    def fetch(self, circuit, rid: int, num_shots: int):
        """Copy a finished request's outputs into new device int64 tensors."""
        import torch
        w = _words(num_shots)
        m = torch.empty((circuit.num_measurements, w), dtype=torch.int64, device="cuda")
        d = torch.empty((circuit.num_detector_rows, w), dtype=torch.int64, device="cuda")
        s = torch.cuda.current_stream()
        _check(library().stim_server_copy_result(self.handle, rid, m.data_ptr() if m.numel() else None,
                                                 d.data_ptr() if d.numel() else None, STIM_DEVICE, s.cuda_stream))
        return m, d

    def cancel(self, rid: int) -> int:
        return library().stim_server_cancel(self.handle, rid)

    def release(self, rid: int) -> None:
        _check(library().stim_server_release(self.handle, rid))

    def stats(self) -> dict:
        st = StimServerStatistics()
        _check(library().stim_server_stats(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in StimServerStatistics._fields_}

    def close(self):
        if getattr(self, "handle", None):
            library().stim_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

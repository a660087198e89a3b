"""CPU oracle for bulk stabilizer-circuit sampling -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package. It shares no code with the CUDA
library. ``oracle.c`` holds the tableau reference sampler (Section 4 of the
paper), the per-shot Pauli frame simulator (Section 3), the Philox RNG and the
exact geometric noise tables; ``statevector.py`` is a brute-force check for
circuits of at most ~17 qubits.

Parity status: the gate tables, Pauli multiplication, tableau reference
sample, frame simulator, noise rates, geometric tables and Philox are each
pinned by ``tests/test_oracle_*.py`` against matrices, state vectors, closed
forms or independent library implementations. The exact bit pattern of the
RNG keying is a convention (the paper uses an unseeded Mersenne twister), so
GPU-vs-oracle equality is its only check beyond the Philox known answers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GATES = {"H": 0, "S": 1, "CX": 2, "CZ": 3, "M": 4, "MR": 5, "R": 6,
         "X_ERROR": 7, "Z_ERROR": 8, "DEPOLARIZE1": 9, "DEPOLARIZE2": 10,
         "DETECTOR": 11, "X": 12, "Y": 13, "Z": 14, "S_DAG": 15, "SQRT_X": 16,
         "SQRT_X_DAG": 17, "SQRT_Y": 18, "SQRT_Y_DAG": 19, "Y_ERROR": 20,
         "MX": 21, "MY": 22, "MRX": 23, "MRY": 24, "RX": 25, "RY": 26}
TAG_NOISE, TAG_COLLAPSE, TAG_INIT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC,
                    "-lm", "-lpthread"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_u64p = ctypes.POINTER(ctypes.c_uint64)
            L.orc_parse.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.c_char_p, ctypes.c_size_t]
            L.orc_parse.restype = ctypes.c_int
            L.orc_free.argtypes = [ctypes.c_void_p]
            L.orc_info.argtypes = [ctypes.c_void_p, c_u64p]
            L.orc_reference.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_reference.restype = ctypes.c_int
            L.orc_frame_shots.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            L.orc_frame_shots.restype = ctypes.c_int
            L.orc_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_geo_table.argtypes = [ctypes.c_double, ctypes.c_void_p]
            L.orc_half_mask.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint64]
            L.orc_half_mask.restype = ctypes.c_uint64
            L.orc_noise_word.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_void_p]
            L.orc_conj_local.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.orc_conj_local.restype = ctypes.c_int
            L.orc_string_mul.argtypes = [ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
            L.orc_string_mul.restype = ctypes.c_int
            L.orc_conj_custom.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.orc_conj_custom.restype = ctypes.c_int
            _lib = L
    return _lib


class OracleError(ValueError):
    pass


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Circuit:
    """A parsed (flattened) circuit held by the C oracle."""

    def __init__(self, text: str):
        L = lib()
        h = ctypes.c_void_p()
        err = ctypes.create_string_buffer(512)
        if L.orc_parse(text.encode(), ctypes.byref(h), err, 512) != 0:
            raise OracleError(err.value.decode())
        self._h = h
        info = (ctypes.c_uint64 * 7)()
        L.orc_info(h, info)
        (self.num_qubits, self.num_measurements, self.num_detectors,
         self.num_gate_targets, self.num_noise_targets, self.num_instructions,
         self.num_observables) = map(int, info)
        self._ref = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def reference(self):
        """(ref_bits, deterministic_flags), uint8 arrays of length M."""
        if self._ref is None:
            M = self.num_measurements
            ref = np.zeros(max(M, 1), np.uint8)
            det = np.zeros(max(M, 1), np.uint8)
            if lib().orc_reference(self._h, _ptr(ref), _ptr(det)) != 0:
                raise MemoryError("oracle tableau allocation failed")
            self._ref = (ref[:M].copy(), det[:M].copy())
        return self._ref

    def sample(self, shots, seed: int, shot_offset: int = 0, *, threads: int = 1,
               ref: np.ndarray | None = None):
        """Per-shot frame simulation of the given shot indices (global index =
        shot_offset + shots[i]). Returns (meas [k, M] uint8, dets [k, D + K] uint8):
        the D detectors, then the K observables (OBSERVABLE_INCLUDE)."""
        shots = np.ascontiguousarray(np.asarray(shots, dtype=np.uint64))
        if ref is None:
            ref = self.reference()[0]
        ref = np.ascontiguousarray(ref, dtype=np.uint8)
        k = len(shots)
        M, D = self.num_measurements, self.num_detectors + self.num_observables
        meas = np.zeros((k, max(M, 1)), np.uint8)
        dets = np.zeros((k, max(D, 1)), np.uint8)
        lib().orc_frame_shots(self._h, _ptr(ref if M else np.zeros(1, np.uint8)),
                              ctypes.c_uint64(seed & (2**64 - 1)), ctypes.c_uint64(shot_offset),
                              _ptr(shots), k, _ptr(meas), _ptr(dets), threads)
        return meas[:, :M], dets[:, :D]


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def geo_table(p: float) -> np.ndarray:
    G = np.zeros(64, np.uint64)
    lib().orc_geo_table(float(p), _ptr(G))
    return G


def half_mask(seed: int, tag: int, instr: int, slot: int, word: int) -> int:
    return int(lib().orc_half_mask(seed & (2**64 - 1), tag, instr, slot, word))


def noise_word(seed: int, gate: str, p: float, instr: int, slot: int, word: int):
    out = np.zeros(4, np.uint64)
    lib().orc_noise_word(seed & (2**64 - 1), GATES[gate], float(p), instr, slot, word, _ptr(out))
    return [int(v) for v in out]


def conj_local(gate: str, x: int, z: int):
    ox, oz = ctypes.c_int(), ctypes.c_int()
    ph = lib().orc_conj_local(GATES[gate], x, z, ctypes.byref(ox), ctypes.byref(oz))
    return ox.value, oz.value, ph


def string_mul(dx, dz, sx, sz):
    """In-place dx,dz := (dx,dz)*(sx,sz) over uint64 words; returns power of i."""
    return lib().orc_string_mul(len(dx), _ptr(dx), _ptr(dz), _ptr(sx), _ptr(sz))


def conj_custom(images, x: int, z: int):
    """Conjugate local Pauli bits (x, z) by a gate given as generator images
    [(x bits, z bits, sign), ...] in the order X_a, Z_a[, X_b, Z_b]."""
    k = len(images) // 2
    ix = np.array([im[0] for im in images], np.int32)
    iz = np.array([im[1] for im in images], np.int32)
    isg = np.array([im[2] for im in images], np.int32)
    ox, oz = ctypes.c_int(), ctypes.c_int()
    ph = lib().orc_conj_custom(k, _ptr(ix), _ptr(iz), _ptr(isg), x, z,
                               ctypes.byref(ox), ctypes.byref(oz))
    return ox.value, oz.value, ph

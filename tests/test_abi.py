"""The C-ABI library loads and exports every function include/stimgb.h
declares; the host compiler (no GPU needed) agrees with the oracle's counts
and rejects malformed circuits."""
import ctypes

import numpy as np
import os
import re

import pytest

import oracle
import paper_2103_02202_gb300 as sg
from paper_2103_02202_gb300 import build as sgbuild
from paper_2103_02202_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    sgbuild.build()
    yield


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:int|void)\s+(stim_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(sg.library_path())
    decl = declared_functions()
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(sg.EXPORTED_SYMBOLS) == decl


def test_binding_constants_match_header():
    """Every STIM_* integer #define of the header has the same value in the binding."""
    txt = open(os.path.join(ROOT, "include", "stimgb.h")).read()
    defs = re.findall(r"^#define\s+(STIM_\w+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))u?(?:\s*<<\s*(\d+))?\)?", txt, flags=re.M)
    assert defs
    for name, val, shift in defs:
        v = int(val, 0) << (int(shift) if shift else 0)
        assert hasattr(sg, name), name
        assert getattr(sg, name) == v, name


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(sg, "_lib", None)
    monkeypatch.setattr(sg, "_LIB_PATH", "/nonexistent/libstimgb.so")
    with pytest.raises(RuntimeError):
        sg.library()


CIRCUITS = {
    "surface_d3": W.surface_code_memory(3, 3, 1e-3),
    "surface_d5_noiseless": W.surface_code_memory(5, 4, 0.0),
    "repetition": W.repetition_code(5, 20, 0.01),
    "random_clifford": W.random_clifford(60, 20, 7),
    "random_noisy": W.random_clifford(40, 10, 8, p=0.01),
    "nested": "REPEAT 3 {\n H 0\n REPEAT 2 {\n CX 0 1\n M 1\n }\n DETECTOR rec[-1] rec[-2]\n}\nM 0\n",
    "empty": "",
    "comments": "# only a comment\n\n   \n",
    "wide_gate_set": ("H 0\nSQRT_X 1 2\nSQRT_Y_DAG 3\nMX 0 1\nY_ERROR(0.1) 0 3\nMRY 1\nRX 2\nS_DAG 2\n"
                      "X 2\nY 0\nZ 3\nSQRT_X_DAG 0\nSQRT_Y 1\nRY 3\nMRX 0\nMY 3\nM 2\n"
                      "DETECTOR rec[-1] rec[-2]\n"),
    "feedforward": ("H 0 1\nM 0 1\nCX rec[-1] 2 rec[-2] 3\nCZ 2 rec[-1]\nREPEAT 3 {\n"
                    "CZ rec[-2] 0\nMR 1 2\nDETECTOR rec[-1]\n}\nM 3\n"),
    "observables": ("H 0\nM 0 1\nOBSERVABLE_INCLUDE(3) rec[-1]\nREPEAT 4 {\nMR 1\nDETECTOR rec[-1]\n"
                    "OBSERVABLE_INCLUDE(1) rec[-1] rec[-2]\n}\n"),
    "observable_without_targets": "M 0\nOBSERVABLE_INCLUDE(5)\nDETECTOR rec[-1]\n",
    "pauli_channels": ("PAULI_CHANNEL_1(0.1, 0, 0.2) 0 1 2\nPAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) +
                       ") 0 1 2 3\nDEPOLARIZE1(0.1) 3\nM 0 1 2 3\n"),
}


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_counts_match_oracle(name):
    text = CIRCUITS[name]
    h = sg.stim_compile(text)
    try:
        info = sg.stim_info_get(h)
    finally:
        sg.stim_free(h)
    o = oracle.Circuit(text)
    assert info["num_qubits"] == o.num_qubits
    assert info["num_measurements"] == o.num_measurements
    assert info["num_detectors"] == o.num_detectors
    assert info["num_gate_targets"] == o.num_gate_targets
    assert info["num_noise_targets"] == o.num_noise_targets
    assert info["num_instructions"] == o.num_instructions
    assert info["num_observables"] == o.num_observables


def test_surface_code_layers_are_fused():
    d, r = 5, 5
    h = sg.stim_compile(W.surface_code_memory(d, r, 1e-3))
    info = sg.stim_info_get(h)
    sg.stim_free(h)
    # per round: H, 4 CX steps, H, MR (+ noise folded into neighbouring layers)
    assert info["num_layers"] <= r * 16 + 8
    assert info["num_program_layers"] < info["num_layers"]


BAD = [
    ("FOO 0\n", sg.STIM_E_PARSE),
    ("H -1\n", sg.STIM_E_PARSE),
    ("H 1.5\n", sg.STIM_E_PARSE),
    ("CX 0 1 2\n", sg.STIM_E_PARSE),
    ("CX 3 3\n", sg.STIM_E_PARSE),
    ("CZ 1 1\n", sg.STIM_E_PARSE),
    ("DEPOLARIZE2(0.1) 4 4\n", sg.STIM_E_PARSE),
    ("X_ERROR(1.5) 0\n", sg.STIM_E_PARSE),
    ("X_ERROR(-0.1) 0\n", sg.STIM_E_PARSE),
    ("X_ERROR 0\n", sg.STIM_E_PARSE),
    ("X_ERROR(0.1, 0.2) 0\n", sg.STIM_E_PARSE),
    ("H(0.1) 0\n", sg.STIM_E_PARSE),
    ("M 0\nDETECTOR rec[-2]\n", sg.STIM_E_PARSE),
    ("M 0\nDETECTOR rec[-0]\n", sg.STIM_E_PARSE),
    ("M 0\nDETECTOR rec[1]\n", sg.STIM_E_PARSE),
    ("REPEAT 2 {\nH 0\n", sg.STIM_E_PARSE),
    ("H 0\n}\n", sg.STIM_E_PARSE),
    ("REPEAT 0 {\nH 0\n}\n", sg.STIM_E_PARSE),
    ("REPEAT x {\nH 0\n}\n", sg.STIM_E_PARSE),
    ("H 16777216\n", sg.STIM_E_UNSUPPORTED),
    ("M 0\nCX 1 rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nCX rec[-0] 1\n", sg.STIM_E_PARSE),
    ("M 0 1\nCZ rec[-1] rec[-2]\n", sg.STIM_E_PARSE),
    ("CX rec[-1] 0\n", sg.STIM_E_PARSE),
    ("M 0\nCX rec[-2] 1\n", sg.STIM_E_PARSE),
    ("REPEAT 2 {\nCX rec[-1] 0\nM 0\n}\n", sg.STIM_E_PARSE),
    ("M 0\nDEPOLARIZE2(0.1) rec[-1] 0\n", sg.STIM_E_PARSE),
    ("M 0\nH rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(0.5) rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(-1) rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(0) 0\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(0) rec[-2]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(1, 2) rec[-1]\n", sg.STIM_E_PARSE),
    ("M 0\nOBSERVABLE_INCLUDE(65536) rec[-1]\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_1(0.1, 0.2) 0\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_1(0.5, 0.4, 0.2) 0\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_1(-0.1, 0.2, 0.1) 0\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_2(0.1) 0 1\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) + ") 0\n", sg.STIM_E_PARSE),
    ("PAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) + ") 1 1\n", sg.STIM_E_PARSE),
]


@pytest.mark.parametrize("text,code", BAD)
def test_parse_errors(text, code):
    with pytest.raises(sg.StimError) as ei:
        sg.stim_compile(text)
    assert ei.value.code == code
    assert sg.stim_last_error()


def test_parse_error_reports_line():
    with pytest.raises(sg.StimError) as ei:
        sg.stim_compile("H 0\nCX 0 1\nBOGUS 2\n")
    assert "line 3" in str(ei.value)


def test_aliases_and_detector_coordinates():
    h = sg.stim_compile("CNOT 0 1\nM 0 1\nDETECTOR(1, 2.5, 0) rec[-1] rec[-2]\n")
    info = sg.stim_info_get(h)
    sg.stim_free(h)
    assert info["num_detectors"] == 1 and info["num_gate_targets"] == 3


def test_invalid_arguments_without_gpu():
    lib = sg.library()
    assert lib.stim_reference_sample(None, None, None, 0, None) == sg.STIM_E_INVALID_ARG
    assert lib.stim_frame_sample(None, 10, 0, None, None, 0, None) == sg.STIM_E_INVALID_ARG
    assert lib.stim_reference_many(None, 2, 0) == sg.STIM_E_INVALID_ARG
    h = sg.stim_compile("H 0\nM 0\n")
    try:
        arr = (ctypes.c_void_p * 1)(h)
        assert lib.stim_reference_many(arr, 1, 0x40) == sg.STIM_E_INVALID_ARG     # unknown flag
        rc = lib.stim_frame_sample_ex(h, 10, 0, 3, None, None, 0, None, None)
        assert rc == sg.STIM_E_INVALID_ARG      # shot_offset not a multiple of 64
        rc = lib.stim_frame_sample(h, 10, 0, None, None, 0x40, None)
        assert rc == sg.STIM_E_INVALID_ARG      # unknown flag
    finally:
        sg.stim_free(h)


def _key(text):
    h = sg.stim_compile(text)
    try:
        return sg.stim_info_get(h)["reference_key"]
    finally:
        sg.stim_free(h)


def test_reference_key_ignores_noise_detectors_and_observables():
    base = W.surface_code_memory(5, 4, 0.001)
    same = [W.surface_code_memory(5, 4, 0.01), W.surface_code_memory(5, 4, 0.0),
            W.surface_code_memory(5, 4, 0.001, observable=True),
            "\n".join(l for l in base.splitlines() if not l.strip().startswith("DETECTOR")) + "\n",
            base.replace("DEPOLARIZE1", "PAULI_CHANNEL_1(0.01, 0.02, 0.03) #")]
    for t in same:
        assert _key(t) == _key(base)
    # anything the noiseless state sees changes the key
    different = [W.surface_code_memory(5, 5, 0.001), W.surface_code_memory(7, 4, 0.001),
                 base.replace("MR", "M", 1), base.replace("REPEAT 3", "REPEAT 7"),
                 base + "H 0\n", base.replace("H ", "S ", 1), base + "CX rec[-1] 0\n"]
    keys = {_key(t) for t in different}
    assert _key(base) not in keys and len(keys) == len(different)
    # equal skeletons written differently (rounds 5 = REPEAT 4) share the key
    assert _key(W.surface_code_memory(5, 5, 0.02)) == _key(base.replace("REPEAT 3", "REPEAT 4"))


def test_reference_cache_controls_without_gpu():
    st = sg.stim_reference_cache_stats()
    assert set(st) == {"hits", "misses", "entries", "bytes"}
    sg.stim_reference_cache_set(0)
    assert sg.stim_reference_cache_stats()["entries"] == 0
    sg.stim_reference_cache_set(256 << 20)


def _fp(text, C):
    h = sg.stim_compile(text)
    try:
        return sg.stim_frame_program_info_get(h, C)
    finally:
        sg.stim_free(h)


def _noisy_wide(rng, n, L):
    """Random circuits whose chains end in several noise ops on shared qubits."""
    lines = []
    nmeas = 0
    for _ in range(L):
        k = rng.random()
        if k < 0.25:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        elif k < 0.6:
            ch = str(rng.choice(["X_ERROR", "Y_ERROR", "DEPOLARIZE1"]))
            lines.append(f"{ch}(0.1) " + " ".join(map(str, rng.choice(n, int(rng.integers(1, n + 1)), replace=False))))
        elif k < 0.75:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"DEPOLARIZE2(0.1) {a} {b}")
        elif k < 0.85 and nmeas:
            lines.append(f"CX rec[-{int(rng.integers(1, nmeas + 1))}] {int(rng.integers(n))}")
        else:
            q = int(rng.integers(n))
            lines.append(f"M {q}")
            nmeas += 1
    return "\n".join(lines) + "\nM " + " ".join(map(str, range(n))) + "\n"


def test_frame_program_invariants():
    """Host-only checks of the frame builder: chain structure does not depend
    on the cluster size; chains stay within 12 ops; with a cluster no
    deferred tail names a qubit twice (duplicate addresses in one cluster
    reduction lost updates); classically controlled ops always start their
    chain (they read a record written before the previous barrier)."""
    rng = np.random.default_rng(2600)
    single_repeats = 0
    for _ in range(40):
        n = int(rng.integers(3, 40))
        text = _noisy_wide(rng, n, int(rng.integers(10, 80)))
        infos = {C: _fp(text, C) for C in (1, 2, 4, 8)}
        for C, inf in infos.items():
            assert inf["chains"] == infos[1]["chains"] and inf["ops"] == infos[1]["ops"]
            assert inf["max_chain_ops"] <= 12
            assert inf["feedforward_not_first"] == 0
            assert inf["deferred_ops"] <= infos[1]["deferred_ops"]
            if C > 1:
                assert inf["tails_repeating_qubit"] == 0
        single_repeats += infos[1]["tails_repeating_qubit"]
    assert single_repeats > 0      # single CTAs keep long tails (their local reductions merge duplicates)
    dup = ("H 0 1 2 3\nCZ 2 0\nCZ 1 3\nX_ERROR(0.5) 0\nX_ERROR(0.5) 0\nY_ERROR(0.5) 0\n"
           "DEPOLARIZE1(0.5) 0\nCX 0 1\nM 0 1 2 3\n")
    one, two = _fp(dup, 1), _fp(dup, 2)
    assert one["tails_repeating_qubit"] == 1 and two["tails_repeating_qubit"] == 0
    assert two["deferred_ops"] == one["deferred_ops"] - 3
    with pytest.raises(sg.StimError):
        _fp(dup, 3)


def test_fault_injection_controls_without_gpu():
    lib = sg.library()
    assert lib.stim_debug_fail_allocations(-1, 1) == sg.STIM_E_INVALID_ARG
    assert lib.stim_debug_fail_allocations(0, -1) == sg.STIM_E_INVALID_ARG
    sg.stim_debug_fail_allocations(3, 1)
    sg.stim_debug_fail_allocations(0, 0)          # off again


@pytest.mark.parametrize("d,rounds,qubits,meas,dets", [(3, 3, 17, 33, 24), (25, 25, 1249, 16225, 15600),
                                                       (100, 100, 19999, 1009900, 999901)])
def test_surface_code_workload_sizes(d, rounds, qubits, meas, dets):
    """The seeded surface-code generator produces the sizes the benchmark
    configurations are stated with (gate and noise targets too at d=100)."""
    h = sg.stim_compile(W.surface_code_memory(d, rounds, 1e-3))
    try:
        info = sg.stim_info_get(h)
    finally:
        sg.stim_free(h)
    assert (info["num_qubits"], info["num_measurements"], info["num_detectors"]) == (qubits, meas, dets)
    if d == 100:
        assert info["num_gate_targets"] == 5989699 and info["num_noise_targets"] == 5969700


def test_workload_generators_are_seeded():
    a = W.batch_circuits()
    b = W.batch_circuits()
    assert [e["text"] for e in a] == [e["text"] for e in b] and len(a) == 64
    assert W.random_clifford(50, 10, 3) == W.random_clifford(50, 10, 3)
    assert W.random_clifford(50, 10, 3) != W.random_clifford(50, 10, 4)

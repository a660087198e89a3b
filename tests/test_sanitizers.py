"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer: the
circuit compiler with the frame-program builder, and the C oracle (parse,
tableau reference, frame sampling), each driven over a corpus of valid and
malformed circuits (no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2103_02202_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_02202_gb300", "csrc")
SAN = ["-g", "-O1", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:halt_on_error=1:abort_on_error=0",
           UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")

MALFORMED = ["FOO 0\n", "H -1\n", "CX 0 1 2\n", "CX 3 3\n", "X_ERROR(1.5) 0\n", "M 0\nDETECTOR rec[-2]\n",
             "REPEAT 2 {\nH 0\n", "H 0\n}\n", "M 0\nCX 1 rec[-1]\n", "M 0 1\nCZ rec[-1] rec[-2]\n",
             "M 0\nOBSERVABLE_INCLUDE(0.5) rec[-1]\n", "PAULI_CHANNEL_1(0.5, 0.4, 0.2) 0\n",
             "PAULI_CHANNEL_2(0.1) 0 1\n", "REPEAT 0 {\nH 0\n}\n", "H(0.1) 0\n", "DETECTOR rec[-1]\n",
             "M 0\nX_ERROR(0.1, 0.2) 0\n", "H 16777216\n", "", "# only a comment\n"]


def _random(rng, n, L):
    lines, nmeas = [], 0
    for _ in range(L):
        k = rng.random()
        q = int(rng.integers(n))
        if k < 0.2 and n > 1:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        elif k < 0.35:
            lines.append(f"{str(rng.choice(['H', 'S', 'S_DAG', 'SQRT_X', 'SQRT_Y_DAG', 'X', 'Y']))} {q}")
        elif k < 0.5:
            lines.append(f"{str(rng.choice(['X_ERROR', 'Y_ERROR', 'DEPOLARIZE1']))}(0.2) {q}")
        elif k < 0.55:
            lines.append(f"PAULI_CHANNEL_1(0.1, 0.2, 0.05) {q}")
        elif k < 0.6 and n > 1:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"PAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) + f") {a} {b}")
        elif k < 0.7 and nmeas:
            lines.append(f"CX rec[-{int(rng.integers(1, nmeas + 1))}] {q}")
        elif k < 0.75 and nmeas:
            lines.append(f"OBSERVABLE_INCLUDE({int(rng.integers(3))}) rec[-{int(rng.integers(1, nmeas + 1))}]")
        elif k < 0.8 and nmeas:
            lines.append(f"DETECTOR rec[-{int(rng.integers(1, nmeas + 1))}]")
        else:
            lines.append(f"{str(rng.choice(['M', 'MR', 'MX', 'MY', 'R', 'RX']))} {q}")
            if lines[-1][0] == "M":
                nmeas += 1
    body = "\n".join(lines)
    return f"REPEAT {int(rng.integers(1, 4))} {{\n{body}\n}}\n" if rng.random() < 0.3 else body + "\n"


@pytest.fixture(scope="module")
def corpus(tmp_path_factory):
    rng = np.random.default_rng(2700)
    texts = [W.surface_code_memory(3, 3, 1e-3), W.surface_code_memory(5, 4, 1e-3, observable=True),
             W.repetition_code(5, 20, 0.01), W.random_clifford(60, 10, 1, p=0.01)]
    texts += [_random(rng, int(rng.integers(2, 12)), int(rng.integers(1, 40))) for _ in range(60)]
    texts += MALFORMED
    p = tmp_path_factory.mktemp("san") / "corpus.txt"
    p.write_text("\n%%\n".join(texts))
    return str(p), len(texts)


def _compiler(name):
    exe = shutil.which(name)
    if exe is None:
        pytest.skip(f"{name} not available")
    return exe


def _build_and_run(cmd, exe, corpus_file):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and ("unrecognized" in r.stderr or "cannot find" in r.stderr):
        pytest.skip("sanitizer runtime not available: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe, corpus_file], capture_output=True, text=True, env=ENV, timeout=600)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-6000:])
    return r.stdout


def test_compiler_under_sanitizers(corpus, tmp_path):
    corpus_file, count = corpus
    exe = str(tmp_path / "compiler_driver")
    cmd = [_compiler("g++"), "-std=c++17", *SAN, "-I", CSRC, os.path.join(ROOT, "tests", "sanitize", "compiler_driver.cpp"),
           os.path.join(CSRC, "compiler.cpp"), "-o", exe]
    out = _build_and_run(cmd, exe, corpus_file)
    ok, rejected = (int(v) for v in out.split()[1::2])
    assert ok + rejected == count and rejected >= len(MALFORMED) - 2


def test_oracle_under_sanitizers(corpus, tmp_path):
    corpus_file, count = corpus
    exe = str(tmp_path / "oracle_driver")
    cmd = [_compiler("gcc"), "-std=c11", *SAN, os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"),
           os.path.join(ROOT, "oracle", "oracle.c"), "-o", exe, "-lpthread", "-lm"]
    out = _build_and_run(cmd, exe, corpus_file)
    ok, rejected = (int(v) for v in out.split()[1::2])
    assert ok + rejected == count

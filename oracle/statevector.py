"""Brute-force state-vector simulation -- TEST INFRASTRUCTURE ONLY.

Used to pin the tableau and frame oracles on small circuits (Section 5.5 of
the paper checks gate tableaus against unitaries the same way). Holds its own
tiny parser and the gate unitaries as plain matrices; measurements and resets
in the X, Y and Z bases are projections onto the measured Pauli's eigenspaces;
noise channels are ignored (noiseless semantics only).

* ``reference(text)``: the outcome-0 noiseless sample: each measurement whose
  outcome is random (P(0) = 1/2) is projected onto 0, otherwise onto its
  deterministic outcome; also returns the per-measurement deterministic flag.
* ``branches(text)``: every record the noiseless circuit can produce, by
  enumerating both outcomes of every random measurement.
"""
from __future__ import annotations

import re

import numpy as np

_S2 = 1 / np.sqrt(2)
UNITARY = {
    "H": np.array([[1, 1], [1, -1]], complex) * _S2,
    "S": np.diag([1, 1j]).astype(complex),
    "S_DAG": np.diag([1, -1j]).astype(complex),
    "X": np.array([[0, 1], [1, 0]], complex),
    "Y": np.array([[0, -1j], [1j, 0]], complex),
    "Z": np.diag([1, -1]).astype(complex),
    # square roots: SQRT_X^2 = X, SQRT_Y^2 = Y (the e^{-i pi/4 P} forms up to phase)
    "SQRT_X": np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], complex) / 2,
    "SQRT_X_DAG": np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]], complex) / 2,
    "SQRT_Y": np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], complex) / 2,
    "SQRT_Y_DAG": np.array([[1 - 1j, 1 - 1j], [-1 + 1j, 1 - 1j]], complex) / 2,
    # two-qubit gates in the basis |a b> with a the first target
    "CX": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex),
    "CZ": np.diag([1, 1, 1, -1]).astype(complex),
}
PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], complex),
    "Y": np.array([[0, -1j], [1j, 0]], complex),
    "Z": np.array([[1, 0], [0, -1]], complex),
}
NOISE = {"X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2"}
ONE_QUBIT = {"H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG", "SQRT_Y", "SQRT_Y_DAG"}
# collapsing ops: measured Pauli and whether they record / reset
COLLAPSE = {"M": ("Z", 1, 0), "MR": ("Z", 1, 1), "R": ("Z", 0, 1),
            "MX": ("X", 1, 0), "MRX": ("X", 1, 1), "RX": ("X", 0, 1),
            "MY": ("Y", 1, 0), "MRY": ("Y", 1, 1), "RY": ("Y", 0, 1)}
# a Pauli that anticommutes with the measured one: maps its -1 eigenstate to +1
FLIPPER = {"Z": "X", "X": "Z", "Y": "Z"}


def parse(text: str):
    """Flatten the circuit into (name, targets) pairs. DETECTOR targets are
    absolute measurement indices."""
    stack = [[]]
    reps = []
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        if line == "}":
            body = stack.pop()
            stack[-1].append(("REPEAT", reps.pop(), body))
            continue
        m = re.fullmatch(r"REPEAT\s+(\d+)\s*\{", line)
        if m:
            stack.append([])
            reps.append(int(m.group(1)))
            continue
        m = re.fullmatch(r"([A-Z_0-9]+)(\([^)]*\))?(.*)", line)
        name = m.group(1)
        if name == "CNOT":
            name = "CX"
        toks = m.group(3).split()
        if name in ("DETECTOR", "OBSERVABLE_INCLUDE"):
            tg = [int(re.fullmatch(r"rec\[-(\d+)\]", t).group(1)) for t in toks]
        else:
            # CX/CZ may take a measurement record rec[-k] as control (a
            # classically controlled X or Z): kept as ("rec", k) until flattening
            tg = [("rec", int(t[5:-1])) if t.startswith("rec[-") else int(t) for t in toks]
        stack[-1].append((name, tg))
    assert len(stack) == 1

    flat = []
    count = [0]

    def walk(items):
        for it in items:
            if it[0] == "REPEAT":
                for _ in range(it[1]):
                    walk(it[2])
                continue
            name, tg = it
            if name in ("DETECTOR", "OBSERVABLE_INCLUDE"):
                flat.append((name, [count[0] - k for k in tg]))
            else:
                flat.append((name, [("rec", count[0] - t[1]) if isinstance(t, tuple) else t for t in tg]))
                if name in COLLAPSE and COLLAPSE[name][1]:
                    count[0] += len(tg)

    walk(stack[0])
    return flat


def num_qubits(ops) -> int:
    n = 0
    for name, tg in ops:
        qs = [t for t in tg if not isinstance(t, tuple)]
        if name not in ("DETECTOR", "OBSERVABLE_INCLUDE") and qs:
            n = max(n, max(qs) + 1)
    return n


def _two_qubit(st, name, a, b, rec):
    """CX/CZ on qubits, or the classically controlled X/Z when one side is a
    measurement record (applied when that record is 1)."""
    if isinstance(a, tuple) or isinstance(b, tuple):
        m, q = (a[1], b) if isinstance(a, tuple) else (b[1], a)
        if rec[m]:
            st.apply1(PAULI["X" if name == "CX" else "Z"], q)
    else:
        st.apply2(UNITARY[name], a, b)


class State:
    """n-qubit state vector; qubit q is bit q of the basis index."""

    def __init__(self, n: int):
        self.n = n
        self.psi = np.zeros((2,) * n, complex)
        self.psi[(0,) * n] = 1

    def _ax(self, q):
        return self.n - 1 - q

    def apply1(self, U, q):
        ax = self._ax(q)
        self.psi = np.moveaxis(np.tensordot(U, self.psi, axes=([1], [ax])), 0, ax)

    def apply2(self, U, a, b):
        U4 = U.reshape(2, 2, 2, 2)
        axa, axb = self._ax(a), self._ax(b)
        out = np.tensordot(U4, self.psi, axes=([2, 3], [axa, axb]))
        self.psi = np.moveaxis(out, [0, 1], [axa, axb])

    def _projector(self, pauli, outcome):
        return (np.eye(2) + (1 - 2 * outcome) * PAULI[pauli]) / 2

    def prob0(self, q, pauli="Z"):
        """Probability of the +1 eigenvalue (outcome 0) of `pauli` on qubit q."""
        s2 = self.copy()
        s2.apply1(self._projector(pauli, 0), q)
        return float(np.sum(np.abs(s2.psi) ** 2))

    def project(self, q, outcome, pauli="Z"):
        self.apply1(self._projector(pauli, outcome), q)
        self.psi /= np.linalg.norm(self.psi)

    def copy(self):
        s = State.__new__(State)
        s.n = self.n
        s.psi = self.psi.copy()
        return s


def _measure_kind(p0: float):
    if p0 > 1 - 1e-9:
        return "det", 0
    if p0 < 1e-9:
        return "det", 1
    assert abs(p0 - 0.5) < 1e-6, p0
    return "rand", None


def reference(text: str):
    ops = parse(text)
    st = State(num_qubits(ops))
    ref, det = [], []
    for name, tg in ops:
        if name in ONE_QUBIT:
            for q in tg:
                st.apply1(UNITARY[name], q)
        elif name in ("CX", "CZ"):
            for a, b in zip(tg[::2], tg[1::2]):
                _two_qubit(st, name, a, b, ref)
        elif name in COLLAPSE:
            pauli, records, resets = COLLAPSE[name]
            for q in tg:
                kind, val = _measure_kind(st.prob0(q, pauli))
                r = 0 if kind == "rand" else val
                st.project(q, r, pauli)
                if records:
                    ref.append(r)
                    det.append(1 if kind == "det" else 0)
                if resets and r == 1:
                    st.apply1(PAULI[FLIPPER[pauli]], q)
    return np.array(ref, np.uint8), np.array(det, np.uint8)


def branches(text: str, max_random: int = 14):
    """All record tuples of the noiseless circuit with their probabilities,
    as a dict, by branching on both outcomes of every random measurement."""
    ops = []
    for name, tg in parse(text):
        if name in COLLAPSE:
            ops += [(name, [q]) for q in tg]    # broadcast runs left to right
        else:
            ops.append((name, tg))
    n = num_qubits(ops)
    out = {}

    def run(i, st, rec, prob, nrand):
        while i < len(ops):
            name, tg = ops[i]
            if name in ONE_QUBIT:
                for q in tg:
                    st.apply1(UNITARY[name], q)
            elif name in ("CX", "CZ"):
                for a, b in zip(tg[::2], tg[1::2]):
                    _two_qubit(st, name, a, b, rec)
            elif name in COLLAPSE:
                pauli, records, resets = COLLAPSE[name]
                q = tg[0]
                kind, val = _measure_kind(st.prob0(q, pauli))
                if kind == "rand":
                    assert nrand < max_random, "too many random measurements"
                    for r in (0, 1):
                        s2 = st.copy()
                        s2.project(q, r, pauli)
                        if resets and r == 1:
                            s2.apply1(PAULI[FLIPPER[pauli]], q)
                        run(i + 1, s2, rec + ([r] if records else []), prob / 2, nrand + 1)
                    return
                st.project(q, val, pauli)
                if records:
                    rec = rec + [val]
                if resets and val == 1:
                    st.apply1(PAULI[FLIPPER[pauli]], q)
            i += 1
        key = tuple(rec)
        out[key] = out.get(key, 0.0) + prob

    run(0, State(n), [], 1.0, 0)
    return out

"""Pins for the CPU oracle: each test ties a piece of the oracle to something
other than itself -- matrices, state vectors, closed forms, values printed in
the paper, or independent library implementations of Philox."""
import ctypes
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import statevector as sv
from paper_2103_02202_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P = sv.PAULI
SYM = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}


def pauli_matrix(xbits, zbits, k):
    """Hermitian-form Pauli on k qubits as a matrix; local qubit 0 is the
    first tensor factor (matching the |a b> basis of the 2-qubit unitaries)."""
    m = np.array([[1]], complex)
    for q in range(k):
        m = np.kron(m, P[SYM[((xbits >> q) & 1, (zbits >> q) & 1)]])
    return m


# --------------------------------------------------------------------------
# Section 2.1 / 2.3: encodings, gate tables, Pauli multiplication
# --------------------------------------------------------------------------
def test_xz_encoding_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "xz_encoding.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 4
    for name, x, z in rows:
        # product of encodings = encoding of product up to phase (Section 2.1)
        m = pauli_matrix(int(x), int(z), 1)
        np.testing.assert_allclose(m, P[name])


@pytest.mark.parametrize("gate,k", [("H", 1), ("S", 1), ("X", 1), ("CX", 2), ("CZ", 2), ("Y", 1), ("Z", 1),
                                    ("S_DAG", 1), ("SQRT_X", 1), ("SQRT_X_DAG", 1), ("SQRT_Y", 1),
                                    ("SQRT_Y_DAG", 1)])
def test_gate_conjugation_matches_unitary(gate, k):
    """U^dagger P U == i^ph * image for every local Pauli (the paper's
    unitary-vs-tableau cross-check, Section 5.5)."""
    U = sv.UNITARY[gate]
    for x in range(2 ** k):
        for z in range(2 ** k):
            ox, oz, ph = oracle.conj_local(gate, x, z)
            lhs = U.conj().T @ pauli_matrix(x, z, k) @ U
            rhs = (1j ** ph) * pauli_matrix(ox, oz, k)
            np.testing.assert_allclose(lhs, rhs, atol=1e-12, err_msg=f"{gate} x={x} z={z}")


def _parse_pauli2(s):
    x = z = 0
    for q, ch in enumerate(s):
        xb, zb = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}[ch]
        x |= xb << q
        z |= zb << q
    return x, z


def test_controlled_y_tableau_golden():
    """Section 2.3 prints the C_Y tableau; Section 2.3.1 conjugates X1 Y2
    through it to get X1. Check the printed columns against the C_Y matrix
    and the worked example through the oracle's generic conjugation."""
    cols, example = {}, None
    for line in open(os.path.join(GOLD, "cy_tableau.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "column":
            cols[t[1]] = (0 if t[2] == "+" else 1, t[3])
        else:
            example = (t[1], 0 if t[3] == "+" else 1, t[4])
    CY = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, -1j], [0, 0, 1j, 0]], complex)
    images = []
    for g in ("X1", "Z1", "X2", "Z2"):
        sign, pauli = cols[g]
        x, z = _parse_pauli2(pauli)
        gx, gz = _parse_pauli2(("X" if g[0] == "X" else "Z") + "I" if g[1] == "1" else "I" + g[0])
        lhs = CY.conj().T @ pauli_matrix(gx, gz, 2) @ CY
        np.testing.assert_allclose(lhs, (-1) ** sign * pauli_matrix(x, z, 2), atol=1e-12)
        images.append((x, z, sign))
    inp, sign, out = example
    x, z = _parse_pauli2(inp)
    ox, oz, ph = oracle.conj_custom(images, x, z)
    assert (ox, oz) == _parse_pauli2(out)
    assert ph == 2 * sign


def test_frame_rules_golden():
    """The batched frame updates printed in Section 5.1 (S: z ^= x; CNOT:
    z1 ^= z2, x2 ^= x1) are the oracle's gate images with the phase dropped."""
    lines = [l.split() for l in open(os.path.join(GOLD, "frame_rules.txt")) if l.strip() and l[0] != "#"]
    assert [l[0] for l in lines] == ["S", "CX", "CX"]
    for x in range(2):
        for z in range(2):
            ox, oz, _ = oracle.conj_local("S", x, z)
            assert (ox, oz) == (x, z ^ x)
    for bits in range(16):
        x0, z0, x1, z1 = (bits >> 0) & 1, (bits >> 1) & 1, (bits >> 2) & 1, (bits >> 3) & 1
        ox, oz, _ = oracle.conj_local("CX", x0 | (x1 << 1), z0 | (z1 << 1))
        assert ox == (x0 | ((x1 ^ x0) << 1))
        assert oz == ((z0 ^ z1) | (z1 << 1))


def test_pauli_string_multiplication_phase():
    """(dx,dz)*(sx,sz) == i^ph (result) as matrices, on random 1..5-qubit
    strings, plus the exhaustive single-qubit table."""
    rng = np.random.default_rng(0)
    for a in range(4):
        for b in range(4):
            dx = np.array([a & 1], np.uint64); dz = np.array([a >> 1], np.uint64)
            sx = np.array([b & 1], np.uint64); sz = np.array([b >> 1], np.uint64)
            m1, m2 = pauli_matrix(a & 1, a >> 1, 1), pauli_matrix(b & 1, b >> 1, 1)
            ph = oracle.string_mul(dx, dz, sx, sz)
            np.testing.assert_allclose(m1 @ m2, (1j ** ph) * pauli_matrix(int(dx[0]), int(dz[0]), 1))
    for _ in range(200):
        k = int(rng.integers(1, 6))
        v = rng.integers(0, 2 ** k, 4)
        dx, dz, sx, sz = [np.array([int(t)], np.uint64) for t in v]
        m1 = pauli_matrix(int(v[0]), int(v[1]), k)
        m2 = pauli_matrix(int(v[2]), int(v[3]), k)
        ph = oracle.string_mul(dx, dz, sx, sz)
        np.testing.assert_allclose(m1 @ m2, (1j ** ph) * pauli_matrix(int(dx[0]), int(dz[0]), k), atol=1e-12)


def test_pauli_string_multiplication_multiword():
    """Phase over several 64-bit words equals the sum of per-word phases."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        nw = int(rng.integers(1, 5))
        dx, dz, sx, sz = [rng.integers(0, 2 ** 63, nw, dtype=np.uint64) for _ in range(4)]
        tot = 0
        for w in range(nw):
            a = [np.array([v[w]], np.uint64) for v in (dx, dz, sx, sz)]
            tot += oracle.string_mul(*a)
        ph = oracle.string_mul(dx.copy(), dz.copy(), sx, sz)
        assert ph == tot % 4


# --------------------------------------------------------------------------
# Section 4: inverse-tableau reference sample vs brute-force state vectors
# --------------------------------------------------------------------------
def _rand_circuit(rng, n, L, noise=False):
    lines = []
    for _ in range(L):
        g = str(rng.choice(["H", "S", "CX", "CZ", "M", "MR", "R", "BCAST"]))
        if g == "BCAST":
            g2 = str(rng.choice(["H", "S", "M", "MR", "R"]))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g2} " + " ".join(map(str, rng.choice(n, k, replace=False))))
        elif g in ("CX", "CZ"):
            if n < 2:
                continue
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{g} {a} {b}")
        else:
            lines.append(f"{g} {rng.integers(n)}")
        if noise and rng.random() < 0.3:
            lines.append(f"X_ERROR(0.25) {rng.integers(n)}")
    lines.append("M " + " ".join(map(str, range(n))))
    return "\n".join(lines) + "\n"


def test_reference_matches_statevector_random():
    rng = np.random.default_rng(2021)
    for _ in range(250):
        n = int(rng.integers(1, 8))
        txt = _rand_circuit(rng, n, int(rng.integers(1, 50)))
        ref, det = oracle.Circuit(txt).reference()
        ref2, det2 = sv.reference(txt)
        np.testing.assert_array_equal(ref, ref2, err_msg=txt)
        np.testing.assert_array_equal(det, det2, err_msg=txt)


WIDE_1Q = ["H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG", "SQRT_Y", "SQRT_Y_DAG"]
WIDE_COLLAPSE = ["M", "MR", "R", "MX", "MY", "MRX", "MRY", "RX", "RY"]


def _rand_wide_circuit(rng, n, L, feedforward=False):
    """Random circuits over the wider gate set: all one-qubit Cliffords,
    CX/CZ, measurements/resets in the X, Y and Z bases and (optionally)
    classically controlled X/Z on earlier measurement records."""
    lines = []
    nmeas = 0
    for _ in range(L):
        kind = rng.random()
        if feedforward and nmeas and kind < 0.15:
            k = int(rng.integers(1, nmeas + 1))
            q = int(rng.integers(n))
            lines.append(f"CX rec[-{k}] {q}" if rng.random() < 0.5 else f"CZ {q} rec[-{k}]")
            continue
        if kind < 0.45:
            g = str(rng.choice(WIDE_1Q))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g} " + " ".join(map(str, rng.choice(n, k, replace=False))))
        elif kind < 0.7 and n >= 2:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        else:
            g = str(rng.choice(WIDE_COLLAPSE))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g} " + " ".join(map(str, rng.choice(n, k, replace=False))))
            if g[0] == "M":
                nmeas += k
    lines.append(str(rng.choice(["M", "MX", "MY"])) + " " + " ".join(map(str, range(n))))
    return "\n".join(lines) + "\n"


def test_reference_wide_gate_set_matches_statevector():
    """Reference samples over the wider gate set (one-qubit Cliffords and X/Y
    basis measurements and resets) equal the state-vector outcome-0 samples,
    with measurements as projections onto Pauli eigenspaces."""
    rng = np.random.default_rng(2103)
    for _ in range(300):
        n = int(rng.integers(1, 7))
        txt = _rand_wide_circuit(rng, n, int(rng.integers(1, 40)))
        ref, det = oracle.Circuit(txt).reference()
        ref2, det2 = sv.reference(txt)
        np.testing.assert_array_equal(ref, ref2, err_msg=txt)
        np.testing.assert_array_equal(det, det2, err_msg=txt)


def test_frame_wide_gate_set_support():
    """Noiseless shots over the wider gate set stay inside the state-vector
    branch support, with branch frequencies near their probabilities."""
    rng = np.random.default_rng(2104)
    checked = 0
    while checked < 12:
        n = int(rng.integers(2, 5))
        txt = _rand_wide_circuit(rng, n, int(rng.integers(4, 20)))
        try:
            br = sv.branches(txt)
        except AssertionError:
            continue
        if len(br) > 64:
            continue
        meas, _ = oracle.Circuit(txt).sample(np.arange(2048), seed=int(rng.integers(0, 2**62)))
        counts = {}
        for row in meas:
            k = tuple(int(b) for b in row)
            assert k in br, (txt, k)
            counts[k] = counts.get(k, 0) + 1
        if len(br) > 1:
            chi2 = sum((counts.get(k, 0) - 2048 * p) ** 2 / (2048 * p) for k, p in br.items())
            dof = len(br) - 1
            assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (txt, chi2, dof)
        checked += 1


def test_feedforward_matches_statevector():
    """Classically controlled X/Z (CX rec[-k] q, CZ q rec[-k]): tableau
    references equal the state-vector outcome-0 samples, and frame shots lie
    in the state-vector branch support (the Pauli applied when the record is 1)."""
    rng = np.random.default_rng(2105)
    for _ in range(200):
        n = int(rng.integers(1, 6))
        txt = _rand_wide_circuit(rng, n, int(rng.integers(1, 40)), feedforward=True)
        ref, det = oracle.Circuit(txt).reference()
        ref2, det2 = sv.reference(txt)
        np.testing.assert_array_equal(ref, ref2, err_msg=txt)
        np.testing.assert_array_equal(det, det2, err_msg=txt)
    checked = 0
    while checked < 10:
        n = int(rng.integers(2, 5))
        txt = _rand_wide_circuit(rng, n, int(rng.integers(4, 20)), feedforward=True)
        if "rec[" not in txt:
            continue
        try:
            br = sv.branches(txt)
        except AssertionError:
            continue
        if len(br) > 64:
            continue
        meas, _ = oracle.Circuit(txt).sample(np.arange(1024), seed=int(rng.integers(0, 2**62)))
        for row in meas:
            assert tuple(int(b) for b in row) in br, txt
        checked += 1


@pytest.mark.parametrize("prep,basis,out", [("X 0", "M", 1), ("H 0", "MX", 0), ("H 0\nS 0", "MY", 0),
                                            ("H 0\nZ 0", "MX", 1)])
def test_teleportation_with_feedforward(prep, basis, out):
    """Teleporting a prepared one-qubit state with corrections from the two
    Bell-measurement records gives a deterministic result on every shot."""
    txt = (f"{prep}\nH 1\nCX 1 2\nCX 0 1\nH 0\nM 0 1\nCX rec[-1] 2\nCZ rec[-2] 2\n{basis} 2\n")
    ref, det = oracle.Circuit(txt).reference()
    assert int(ref[2]) == out and int(det[2]) == 1
    meas, _ = oracle.Circuit(txt).sample(np.arange(512), seed=5)
    assert np.all(meas[:, 2] == out)
    assert 0.35 < meas[:, 0].mean() < 0.65 and 0.35 < meas[:, 1].mean() < 0.65


def test_feedforward_parse_errors():
    for bad in ("M 0\nCX 1 rec[-1]\n", "M 0\nCX rec[-0] 1\n", "M 0 1\nCZ rec[-1] rec[-2]\n",
                "CX rec[-1] 0\n"):
        with pytest.raises(ValueError):
            oracle.Circuit(bad)


def test_basis_measurement_special_cases():
    # |+> measured in X is deterministic 0, |-> gives 1; |+i> in Y gives 0
    ref, det = oracle.Circuit("H 0\nMX 0\nX 0\nZ 0\nMX 0\n").reference()
    assert list(ref) == [0, 1] and list(det) == [1, 1]
    ref, det = oracle.Circuit("H 0\nS 0\nMY 0\nS_DAG 0\nS_DAG 0\nMY 0\n").reference()
    assert list(ref) == [0, 1] and list(det) == [1, 1]
    # RX prepares |+>: a following MX is deterministic 0; M after RX is random
    ref, det = oracle.Circuit("X 0\nRX 0\nMX 0\nM 0\n").reference()
    assert list(ref) == [0, 0] and list(det) == [1, 0]
    # SQRT_X twice is X (up to phase): |0> -> |1>
    ref, det = oracle.Circuit("SQRT_X 0\nSQRT_X 0\nM 0\nSQRT_Y 0\nSQRT_Y_DAG 0\nM 0\n").reference()
    assert list(ref) == [1, 1] and list(det) == [1, 1]


def test_reference_matches_statevector_surface_d3():
    txt = W.surface_code_memory(3, 2, 0.0)
    ref, det = oracle.Circuit(txt).reference()
    ref2, det2 = sv.reference(txt)
    np.testing.assert_array_equal(ref, ref2)
    np.testing.assert_array_equal(det, det2)


def test_reference_noise_is_ignored():
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = int(rng.integers(1, 6))
        txt = _rand_circuit(rng, n, 30, noise=True)
        clean = "\n".join(l for l in txt.splitlines() if not l.startswith("X_ERROR")) + "\n"
        np.testing.assert_array_equal(oracle.Circuit(txt).reference()[0],
                                      oracle.Circuit(clean).reference()[0])


def test_reference_special_cases():
    # Bell pair: first Z measurement random (-> 0), second deterministic and equal.
    ref, det = oracle.Circuit("H 0\nCX 0 1\nM 0 1\n").reference()
    assert list(ref) == [0, 0] and list(det) == [0, 1]
    # |1> after H H X-equivalent: H S S H = X
    ref, det = oracle.Circuit("H 0\nS 0\nS 0\nH 0\nM 0\n").reference()
    assert list(ref) == [1] and list(det) == [1]
    # MR resets: a 1 outcome is followed by 0
    ref, _ = oracle.Circuit("H 0\nS 0\nS 0\nH 0\nMR 0\nM 0\n").reference()
    assert list(ref) == [1, 0]
    # empty circuit
    c = oracle.Circuit("")
    assert c.num_qubits == 0 and c.num_measurements == 0
    assert len(c.reference()[0]) == 0


# --------------------------------------------------------------------------
# Section 3: frame simulator
# --------------------------------------------------------------------------
def test_frame_noiseless_support_and_uniformity():
    """Every noiseless shot lies in the support of the state-vector branch
    distribution, and branch frequencies match it (chi-squared)."""
    rng = np.random.default_rng(4)
    checked = 0
    while checked < 12:
        n = int(rng.integers(2, 6))
        txt = _rand_circuit(rng, n, int(rng.integers(5, 30)))
        br = sv.branches(txt)
        if len(br) > 64:
            continue
        c = oracle.Circuit(txt)
        shots = 4096
        meas, _ = c.sample(np.arange(shots), seed=int(rng.integers(0, 2**62)))
        keys = [tuple(int(b) for b in row) for row in meas]
        counts = {}
        for k in keys:
            assert k in br, (txt, k)
            counts[k] = counts.get(k, 0) + 1
        if len(br) > 1:
            chi2 = sum((counts.get(k, 0) - shots * p) ** 2 / (shots * p) for k, p in br.items())
            dof = len(br) - 1
            assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (txt, chi2, dof)
        checked += 1


@pytest.mark.parametrize("d,rounds", [(3, 1), (3, 3), (5, 2), (5, 5)])
def test_frame_noiseless_surface_invariants(d, rounds):
    """Noiseless surface-code detectors are all 0, Z-type stabilizer outcomes
    are all 0, and records of random X-type outcomes vary between shots."""
    c = oracle.Circuit(W.surface_code_memory(d, rounds, 0.0))
    meas, dets = c.sample(np.arange(512), seed=11, threads=4)
    assert dets.sum() == 0
    lay = W.surface_code_layout(d)
    na = len(lay.anc)
    zpos = [k for k, a in enumerate(lay.anc) if a in set(lay.z_anc)]
    xpos = [k for k, a in enumerate(lay.anc) if a in set(lay.x_anc)]
    for r in range(rounds):
        assert meas[:, [r * na + k for k in zpos]].sum() == 0
    x1 = meas[:, xpos]
    assert 0.3 < x1.mean() < 0.7


def test_repetition_code_golden_counts_and_noiseless():
    gold = dict(l.split() for l in open(os.path.join(GOLD, "repetition_code.txt")) if l.strip() and l[0] != "#")
    c = oracle.Circuit(W.repetition_code(5, 20, 0.01))
    assert c.num_qubits == int(gold["qubits"])
    assert c.num_measurements == int(gold["measurements"])
    c0 = oracle.Circuit(W.repetition_code(5, 20, 0.0))
    meas, _ = c0.sample(np.arange(256), seed=3)
    assert meas.sum() == 0


def _zscore(k, n, p):
    return abs(k - n * p) / math.sqrt(n * p * (1 - p))


def _qs(n):
    return " ".join(map(str, range(n)))


@pytest.mark.parametrize("p", [0.001, 0.05, 0.3])
def test_x_error_rate(p):
    n = 1000
    c = oracle.Circuit(f"X_ERROR({p}) {_qs(n)}\nM {_qs(n)}\n")
    meas, _ = c.sample(np.arange(1024), seed=5, threads=4)
    assert _zscore(int(meas.sum()), meas.size, p) < 5


def test_z_error_rate_in_x_basis():
    p, n = 0.02, 1000
    c = oracle.Circuit(f"H {_qs(n)}\nZ_ERROR({p}) {_qs(n)}\nH {_qs(n)}\nM {_qs(n)}\n")
    meas, _ = c.sample(np.arange(1024), seed=6, threads=4)
    assert _zscore(int(meas.sum()), meas.size, p) < 5
    # Z errors are invisible in the Z basis
    c = oracle.Circuit(f"Z_ERROR({p}) {_qs(n)}\nM {_qs(n)}\n")
    meas, _ = c.sample(np.arange(256), seed=6)
    assert meas.sum() == 0


@pytest.mark.parametrize("basis,rate", [("M", 1.0), ("MX", 1.0), ("MY", 0.0)])
def test_y_error_rates(basis, rate):
    """Y_ERROR(p) flips Z- and X-basis measurements with probability p and
    leaves Y-basis measurements alone."""
    p, n = 0.04, 1000
    prep = {"M": "", "MX": f"H {_qs(n)}\n", "MY": f"H {_qs(n)}\nS {_qs(n)}\n"}[basis]
    c = oracle.Circuit(f"{prep}Y_ERROR({p}) {_qs(n)}\n{basis} {_qs(n)}\n")
    meas, _ = c.sample(np.arange(1024), seed=8, threads=4)
    if rate == 0.0:
        assert meas.sum() == 0
    else:
        assert _zscore(int(meas.sum()), meas.size, p * rate) < 5


def test_depolarize1_rates():
    p, n = 0.03, 1000
    cz = oracle.Circuit(f"DEPOLARIZE1({p}) {_qs(n)}\nM {_qs(n)}\n")
    m, _ = cz.sample(np.arange(1024), seed=7, threads=4)
    assert _zscore(int(m.sum()), m.size, 2 * p / 3) < 5
    cx = oracle.Circuit(f"H {_qs(n)}\nDEPOLARIZE1({p}) {_qs(n)}\nH {_qs(n)}\nM {_qs(n)}\n")
    m, _ = cx.sample(np.arange(1024), seed=8, threads=4)
    assert _zscore(int(m.sum()), m.size, 2 * p / 3) < 5


def test_depolarize2_rates():
    p, n = 0.03, 1000
    c = oracle.Circuit(f"DEPOLARIZE2({p}) {_qs(n)}\nM {_qs(n)}\n")
    m, _ = c.sample(np.arange(1024), seed=9, threads=4)
    a, b = m[:, 0::2], m[:, 1::2]
    assert _zscore(int(a.sum()), a.size, 8 * p / 15) < 5
    assert _zscore(int(b.sum()), b.size, 8 * p / 15) < 5
    assert _zscore(int((a & b).sum()), a.size, 4 * p / 15) < 5


def test_repetition_code_first_round_rate():
    """Appendix A circuit: an odd qubit's first MR reads x_{a-1}^x_a^x_{a+1},
    so it flips with probability 3p(1-p)^2 + p^3."""
    p = 0.05
    c = oracle.Circuit(W.repetition_code(50, 1, p))
    m, _ = c.sample(np.arange(8192), seed=10, threads=4)
    q = 3 * p * (1 - p) ** 2 + p ** 3
    assert _zscore(int(m.sum()), m.size, q) < 5


def _inject_after_first_round(text, line):
    i = text.index("REPEAT")
    return text[:i] + line + "\n" + text[i:]


def test_single_data_error_flips_two_detectors():
    """An X error on a data qubit flips the Z plaquettes that contain it at
    the next round and nothing later (Section 5.6): 2 detectors in the bulk,
    1 on a Z-type boundary."""
    d = 5
    lay = W.surface_code_layout(d)
    zsets = {a: set(lay.neighbors[a].values()) for a in lay.z_anc}
    for q in lay.data:
        expect = sum(1 for s in zsets.values() if q in s)
        txt = _inject_after_first_round(W.surface_code_memory(d, 3, 0.0), f"X_ERROR(1) {q}")
        _, dets = oracle.Circuit(txt).sample(np.arange(64), seed=1)
        assert np.all(dets.sum(axis=1) == expect), q


def test_collapse_coins_are_fair():
    n = 2000
    c = oracle.Circuit(f"H {_qs(n)}\nM {_qs(n)}\n")
    m, _ = c.sample(np.arange(512), seed=12, threads=4)
    assert _zscore(int(m.sum()), m.size, 0.5) < 5


def test_shot_offset_is_a_pure_index_shift():
    c = oracle.Circuit(W.surface_code_memory(3, 3, 0.01))
    a, da = c.sample(np.arange(64, 192), seed=99)
    b, db = c.sample(np.arange(0, 128), seed=99, shot_offset=64)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(da, db)


# --------------------------------------------------------------------------
# Section 5.4: exact geometric gap tables
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", [0.0, 1e-4, 1e-3, 0.0123, 0.25, 0.5, 0.9, 1.0])
def test_geometric_table_definition(p):
    G = [int(v) for v in oracle.geo_table(p)]
    two32 = 1 << 32
    t = min(max(round(p * two32), 0), two32)      # Python round is half-even
    S = two32
    for k in range(64):
        S_next = S * (two32 - t) // two32
        assert G[k] == two32 - S_next
        # P(gap = k) = (S_k - S_{k+1}) / 2^32
        prev = 0 if k == 0 else G[k - 1]
        assert G[k] - prev == S - S_next
        S = S_next
    assert G[0] == t


def test_geometric_table_half_even_rounding():
    two32 = 2.0 ** 32
    assert int(oracle.geo_table(0.5 / two32)[0]) == 0
    assert int(oracle.geo_table(1.5 / two32)[0]) == 2
    assert int(oracle.geo_table(2.5 / two32)[0]) == 2


def test_noise_extremes():
    assert oracle.noise_word(1, "X_ERROR", 1.0, 3, 4, 5)[0] == 2**64 - 1
    assert oracle.noise_word(1, "X_ERROR", 0.0, 3, 4, 5) == [0, 0, 0, 0]
    x0, z0, _, _ = oracle.noise_word(1, "DEPOLARIZE1", 1.0, 3, 4, 5)
    assert (x0 | z0) == 2**64 - 1


# --------------------------------------------------------------------------
# Philox4x32-10 against independent implementations
# --------------------------------------------------------------------------
def test_philox_vs_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator (seed = key (seed lo, seed hi),
    offset 0) emits the blocks at counters (0, 0, b, 0), b = 0, 1, 2, ...:
    check the oracle on the first 4096 outputs (1024 blocks) of several seeds."""
    path = None
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10"):
        if os.path.exists(cand):
            path = cand
            break
    if path is None:
        pytest.skip("libcurand not found")
    cur = ctypes.CDLL(path)
    for seed in (0, 1, 0x123456789ABCDEF, 2**64 - 1):
        gen = ctypes.c_void_p()
        assert cur.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
        assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4096, np.uint32)
        assert cur.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4096)) == 0
        cur.curandDestroyGenerator(gen)  # noqa
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for b in range(1024):
            np.testing.assert_array_equal(oracle.philox([0, 0, b, 0], key), out[4 * b:4 * b + 4])


def test_philox_known_answers():
    """The published Philox4x32-10 known-answer vectors (Salmon et al., SC'11;
    tests/golden/philox4x32_10_kat.txt)."""
    rows = 0
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            v = [int(t, 16) for t in line]
            assert len(v) == 10
            np.testing.assert_array_equal(oracle.philox(v[0:4], v[4:6]), np.array(v[6:10], np.uint32))
            rows += 1
    assert rows == 3


def test_philox_vs_triton_interpreter():
    """Triton's tl.philox (run by its CPU interpreter) at arbitrary counters."""
    os.environ.setdefault("TRITON_INTERPRET", "1")
    if os.environ.get("TRITON_INTERPRET") != "1":
        pytest.skip("TRITON_INTERPRET is set to something else")
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def kern(out_ptr, c_ptr, seed):
        c0 = tl.load(c_ptr + 0)
        c1 = tl.load(c_ptr + 1)
        c2 = tl.load(c_ptr + 2)
        c3 = tl.load(c_ptr + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + 0, a)
        tl.store(out_ptr + 1, b)
        tl.store(out_ptr + 2, c)
        tl.store(out_ptr + 3, d)

    rng = np.random.default_rng(13)
    try:
        for _ in range(16):
            seed = int(rng.integers(0, 2**63))
            ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
            out = torch.zeros(4, dtype=torch.uint32)
            kern[(1,)](out, torch.from_numpy(ctr.copy()), seed)
            got = out.numpy().astype(np.uint32)
            exp = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
            np.testing.assert_array_equal(got, exp)
    except Exception as e:  # interpreter unavailable on this platform
        if "interpret" in str(e).lower() and "not" in str(e).lower():
            pytest.skip(str(e))
        raise


def test_noise_mask_structure():
    """The mask of (instr, slot, word) uses counter (j//4, slot, instr, word)
    and takes the first draw as the first gap (p large so bit 0 is set when
    draw 0 < G[0])."""
    seed, instr, slot, word = 77, 5, 9, 3
    p = 0.5
    G = [int(v) for v in oracle.geo_table(p)]
    blk = oracle.philox([0, slot, instr, word], [seed & 0xFFFFFFFF, seed >> 32])
    x0 = oracle.noise_word(seed, "X_ERROR", p, instr, slot, word)[0]
    u0 = int(blk[0])
    gap = next((k for k in range(64) if u0 < G[k]), 64)
    assert (x0 & ((1 << (gap + 1)) - 1)) == (1 << gap)
    hm = oracle.half_mask(seed, oracle.TAG_COLLAPSE, instr, slot, word)
    blk = oracle.philox([0, slot, (1 << 28) | instr, word], [seed & 0xFFFFFFFF, seed >> 32])
    assert hm == int(blk[0]) | (int(blk[1]) << 32)


# ---------------------------------------------------------------------------
# Logical observables (OBSERVABLE_INCLUDE): D detectors, then K observables,
# each the XOR of the flips of every record it includes.
# ---------------------------------------------------------------------------
def _rep_memory(d, rounds, p, final_noise=0.0):
    """Repetition-code memory ending with a data-qubit readout; the logical
    observable is the last data qubit's final measurement."""
    txt = W.repetition_code(d, rounds, p)
    data = " ".join(str(q) for q in range(0, 2 * d + 1, 2))
    if final_noise:
        txt += f"X_ERROR({final_noise}) {2 * d}\n"
    txt += f"M {data}\nOBSERVABLE_INCLUDE(0) rec[-1]\n"
    return txt


def test_observable_of_noiseless_memory_never_flips():
    c = oracle.Circuit(_rep_memory(4, 6, 0.0))
    assert c.num_observables == 1 and c.num_detectors == 0
    _, dets = c.sample(np.arange(400), seed=3)
    assert dets.shape == (400, 1) and not dets.any()


def test_observable_flips_with_certain_error():
    # X_ERROR(1) on the observable's qubit right before its readout: every shot flips
    c = oracle.Circuit(_rep_memory(3, 2, 0.0, final_noise=1.0))
    _, dets = c.sample(np.arange(300), seed=4)
    assert dets[:, 0].all()


def test_observable_flip_rate_matches_p():
    p, n = 0.2, 20000
    c = oracle.Circuit("R 0\nX_ERROR(0.2) 0\nM 0\nOBSERVABLE_INCLUDE(0) rec[-1]\n")
    _, dets = c.sample(np.arange(n), seed=5, threads=8)
    sd = math.sqrt(p * (1 - p) / n)
    assert abs(dets[:, 0].mean() - p) < 5 * sd


def test_observables_accumulate_index_gaps_and_loops():
    txt = ("H 0 1\nM 0 1\nOBSERVABLE_INCLUDE(2) rec[-1]\nOBSERVABLE_INCLUDE(2) rec[-1]\n"
           "REPEAT 3 {\nH 2\nM 2\nOBSERVABLE_INCLUDE(1) rec[-1]\n}\nDETECTOR rec[-4]\n")
    c = oracle.Circuit(txt)
    assert c.num_observables == 3 and c.num_detectors == 1
    meas, dets = c.sample(np.arange(500), seed=6)
    assert dets.shape == (500, 4)
    ref = c.reference()[0]
    flips = meas ^ ref
    np.testing.assert_array_equal(dets[:, 0], flips[:, 1])                      # DETECTOR rec[-4]
    assert not dets[:, 1].any() and not dets[:, 3].any()                          # index 0 unused; 2 cancels
    np.testing.assert_array_equal(dets[:, 2], flips[:, 2] ^ flips[:, 3] ^ flips[:, 4])
    assert 0.4 < dets[:, 2].mean() < 0.6


def test_deterministic_parities_as_observables_never_flip():
    """Any parity of records that the state vector finds deterministic (the
    same in every branch) is an observable that never flips in noiseless
    frame sampling: the collapse coins cancel in it."""
    rng = np.random.default_rng(2200)
    checked = 0
    while checked < 12:
        n = int(rng.integers(2, 5))
        txt = _rand_wide_circuit(rng, n, int(rng.integers(4, 18)))
        txt = "\n".join(l for l in txt.splitlines() if "ERROR" not in l and "DEPOLARIZE" not in l) + "\n"
        try:
            br = sv.branches(txt)
        except AssertionError:
            continue
        if len(br) > 64 or len(br) < 2:
            continue
        outs = np.array(sorted(br), np.uint8)
        M = outs.shape[1]
        found = None
        for mask in range(1, min(1 << M, 1 << 12)):
            sel = [i for i in range(M) if (mask >> i) & 1]
            par = np.bitwise_xor.reduce(outs[:, sel], axis=1)
            if np.all(par == par[0]) and len(sel) >= 2:
                found = sel
                break
        if found is None:
            continue
        obs = "OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{M - i}]" for i in found) + "\n"
        c = oracle.Circuit(txt + obs)
        _, dets = c.sample(np.arange(256), seed=int(rng.integers(2**62)))
        assert not dets[:, -1].any(), txt + obs
        checked += 1


def test_observable_parse_errors():
    for bad in ("M 0\nOBSERVABLE_INCLUDE rec[-1]\n", "M 0\nOBSERVABLE_INCLUDE(0.5) rec[-1]\n",
                "M 0\nOBSERVABLE_INCLUDE(-1) rec[-1]\n", "M 0\nOBSERVABLE_INCLUDE(0) 0\n",
                "M 0\nOBSERVABLE_INCLUDE(0) rec[-2]\n", "M 0\nOBSERVABLE_INCLUDE(1, 2) rec[-1]\n"):
        with pytest.raises(ValueError):
            oracle.Circuit(bad)


@pytest.mark.parametrize("d", [3, 5])
def test_surface_code_logical_observable_is_deterministic(d):
    """The logical Z line chosen by the workload generator commutes with every
    X stabilizer: without noise its parity never flips; with noise it does."""
    c = oracle.Circuit(W.surface_code_memory(d, 3, 0.0, observable=True))
    _, dets = c.sample(np.arange(512), seed=d, threads=8)
    assert c.num_observables == 1 and not dets.any()
    c = oracle.Circuit(W.surface_code_memory(d, 3, 0.02, observable=True))
    _, dets = c.sample(np.arange(512), seed=d, threads=8)
    assert dets[:, -1].any()


# ---------------------------------------------------------------------------
# Pauli channels. Each channel qubit is half of a Bell pair with an ancilla; a
# Bell measurement afterwards reads the Pauli that hit it: (XX flip, ZZ flip)
# = (0, 1) X, (1, 1) Y, (1, 0) Z, so every Pauli's rate is observable.
# ---------------------------------------------------------------------------
_PAULI_OF = {(0, 0): 0, (0, 1): 1, (1, 1): 2, (1, 0): 3}      # I, X, Y, Z


def _bell_probe(channel, nq):
    qs = list(range(nq))
    anc = [q + nq for q in qs]
    pre = "".join(f"H {q}\nCX {q} {a}\n" for q, a in zip(qs, anc))
    post = "".join(f"CX {q} {a}\nH {q}\nM {q} {a}\n" for q, a in zip(qs, anc))
    return pre + channel + "\n" + post


def _pauli_counts(text, nq, shots, seed):
    c = oracle.Circuit(text)
    ref = c.reference()[0]
    assert not ref.any()            # the Bell measurements are deterministic without noise
    meas, _ = c.sample(np.arange(shots), seed, threads=8)
    idx = np.zeros(shots, np.int64)
    for k in range(nq):
        p = np.array([_PAULI_OF[(int(a), int(b))] for a, b in meas[:, 2 * k:2 * k + 2]])
        idx = idx * 4 + p
    return np.bincount(idx, minlength=4 ** nq)


def test_pauli_channel_1_rates():
    probs = [0.1, 0.2, 0.05]
    shots = 60000
    cnt = _pauli_counts(_bell_probe("PAULI_CHANNEL_1(0.1, 0.2, 0.05) 0", 1), 1, shots, 7)
    want = np.array([1 - sum(probs)] + probs)
    sd = np.sqrt(want * (1 - want) / shots)
    assert np.all(np.abs(cnt / shots - want) < 5 * sd + 1e-12), (cnt / shots, want)


def test_pauli_channel_2_rates():
    probs = [0.01, 0.02, 0.03, 0.04, 0.005, 0.0, 0.015, 0.02, 0.01, 0.03, 0.0, 0.025, 0.02, 0.01, 0.05]
    shots = 60000
    args = ", ".join(map(str, probs))
    cnt = _pauli_counts(_bell_probe(f"PAULI_CHANNEL_2({args}) 0 1", 2), 2, shots, 8)
    want = np.array([1 - sum(probs)] + probs)        # index 4a + b, a on qubit 0
    sd = np.sqrt(want * (1 - want) / shots)
    assert np.all(np.abs(cnt / shots - want) < 5 * sd + 1e-12), (cnt / shots, want)
    assert cnt[6] == 0 and cnt[11] == 0               # XY and YZ have probability 0


def test_pauli_channel_special_cases():
    # probability-one Y: every shot reads Y
    cnt = _pauli_counts(_bell_probe("PAULI_CHANNEL_1(0, 1, 0) 0", 1), 1, 500, 9)
    assert cnt[2] == 500
    # a single non-zero pair Pauli: only ZX or nothing
    cnt = _pauli_counts(_bell_probe("PAULI_CHANNEL_2(0,0,0,0,0,0,0,0,0,0,0,0,0.4,0,0) 0 1", 2), 2, 4000, 10)
    assert cnt[0] + cnt[13] == 4000 and 0.35 < cnt[13] / 4000 < 0.45
    # an all-zero channel never hits
    c = oracle.Circuit("PAULI_CHANNEL_1(0, 0, 0) 0\nM 0\n")
    assert not c.sample(np.arange(256), 4)[0].any()


def test_pauli_channel_parse_errors():
    for bad in ("PAULI_CHANNEL_1(0.1, 0.2) 0\n", "PAULI_CHANNEL_1(0.5, 0.4, 0.2) 0\n",
                "PAULI_CHANNEL_1(-0.1, 0.2, 0.1) 0\n", "PAULI_CHANNEL_2(0.1) 0 1\n",
                "PAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) + ") 0\n",
                "PAULI_CHANNEL_2(" + ", ".join(["0.01"] * 15) + ") 1 1\n"):
        with pytest.raises(ValueError):
            oracle.Circuit(bad)


def _teleportation_golden():
    gold = {}
    for line in open(os.path.join(GOLD, "teleportation.txt")):
        if line.strip() and line[0] != "#":
            k, v = line.rstrip("\n").split(" ", 1)
            gold[k] = v
    return gold["circuit"].replace(";", "\n") + "\n", int(gold["final_measurement"])


def test_paper_teleportation_example_golden():
    """The paper's teleportation example: with Bob's corrections applied from
    Alice's two records, the uncomputed qubit always measures False, while
    Alice's bits are random. Checked on the reference, the frame shots and the
    state vector (which also confirms the final bit is deterministic)."""
    txt, final = _teleportation_golden()
    ref, det = oracle.Circuit(txt).reference()
    assert int(ref[-1]) == final and int(det[-1]) == 1
    meas, _ = oracle.Circuit(txt).sample(np.arange(4096), seed=11, threads=4)
    assert np.all(meas[:, -1] == final)
    assert 0.45 < meas[:, 0].mean() < 0.55 and 0.45 < meas[:, 1].mean() < 0.55
    br = sv.branches(txt)
    assert len(br) == 4 and all(k[-1] == final for k in br)
    # without Bob's corrections the final bit is random
    bare = txt.replace("CX rec[-2] 9\n", "").replace("CZ rec[-1] 9\n", "")
    assert {k[-1] for k in sv.branches(bare)} == {0, 1}


# ---------------------------------------------------------------------------
# Section 2.3, "Inverting Tableaus": the terms on qubit b of T(X_a), T(Z_a)
# determine the terms on qubit a of T^-1(X_b), T^-1(Z_b): x(T^-1 X_b)_a =
# z(T Z_a)_b, z(T^-1 X_b)_a = z(T X_a)_b, x(T^-1 Z_b)_a = x(T Z_a)_b,
# z(T^-1 Z_b)_a = x(T X_a)_b (the symplectic transpose).
# ---------------------------------------------------------------------------
_TERM = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
_NAME = {v: k for k, v in _TERM.items()}


def _inverse_terms(tx_a_b, tz_a_b):
    """(term of T(X_a) on b, term of T(Z_a) on b) -> (term of T^-1(X_b) on a, of T^-1(Z_b) on a)."""
    (xx, xz), (zx, zz) = _TERM[tx_a_b], _TERM[tz_a_b]
    return _NAME[(zz, xz)], _NAME[(zx, xx)]


def test_inverse_locality_golden():
    """The paper's worked example of inverting a tableau locally: the rule
    above turns its four given terms of T into the four terms of T^-1 it
    prints."""
    rows = [l.split() for l in open(os.path.join(GOLD, "inverse_locality.txt")) if l.strip() and l[0] != "#"]
    given = {r[1]: r[3] for r in rows if r[0] == "given"}
    derived = {r[1]: r[3] for r in rows if r[0] == "derived"}
    inv_x, inv_z = _inverse_terms(given["X3"], given["Z3"])
    assert (inv_x, inv_z) == (derived["X4"], derived["Z4"])


_DAGGER = {"H": "H", "S": "S_DAG", "S_DAG": "S", "SQRT_X": "SQRT_X_DAG", "SQRT_X_DAG": "SQRT_X",
           "SQRT_Y": "SQRT_Y_DAG", "SQRT_Y_DAG": "SQRT_Y", "X": "X", "Y": "Y", "Z": "Z", "CX": "CX", "CZ": "CZ"}


def _propagate(gates, n, x, z):
    """Pauli terms (no sign) of a generator pushed through the gate list with
    the oracle's per-gate conjugation tables."""
    x, z = list(x), list(z)
    for name, qs in gates:
        lx = sum(x[q] << i for i, q in enumerate(qs))
        lz = sum(z[q] << i for i, q in enumerate(qs))
        ox, oz, _ = oracle.conj_local(name, lx, lz)
        for i, q in enumerate(qs):
            x[q], z[q] = (ox >> i) & 1, (oz >> i) & 1
    return x, z


def test_inverse_tableau_terms_are_the_local_transpose():
    """For random Clifford circuits, the tableau of the reversed, daggered
    circuit (built from the oracle's gate tables) has exactly the Pauli terms
    the paper's local rule derives from the circuit's own tableau. The oracle
    itself never inverts a tableau; what this checks of it is that every
    per-gate term table preserves commutation and undoes its dagger's at the
    term level (a non-symplectic table entry fails). Signs are not compared:
    a dagger pair has the same terms."""
    rng = np.random.default_rng(2800)
    one = [g for g in _DAGGER if g not in ("CX", "CZ")]
    for _ in range(30):
        n = int(rng.integers(2, 7))
        gates = []
        for _ in range(int(rng.integers(5, 40))):
            if rng.random() < 0.4:
                a, b = (int(v) for v in rng.choice(n, 2, replace=False))
                gates.append((str(rng.choice(["CX", "CZ"])), (a, b)))
            else:
                gates.append((str(rng.choice(one)), (int(rng.integers(n)),)))
        inverse = [(_DAGGER[g], qs) for g, qs in reversed(gates)]
        unit = [[int(i == j) for j in range(n)] for i in range(n)]
        zero = [0] * n
        T = {("X", a): _propagate(gates, n, unit[a], zero) for a in range(n)}
        T.update({("Z", a): _propagate(gates, n, zero, unit[a]) for a in range(n)})
        Ti = {("X", b): _propagate(inverse, n, unit[b], zero) for b in range(n)}
        Ti.update({("Z", b): _propagate(inverse, n, zero, unit[b]) for b in range(n)})
        for a in range(n):
            for b in range(n):
                tx = _NAME[(T[("X", a)][0][b], T[("X", a)][1][b])]
                tz = _NAME[(T[("Z", a)][0][b], T[("Z", a)][1][b])]
                want_x, want_z = _inverse_terms(tx, tz)
                assert _NAME[(Ti[("X", b)][0][a], Ti[("X", b)][1][a])] == want_x
                assert _NAME[(Ti[("Z", b)][0][a], Ti[("Z", b)][1][a])] == want_z


def test_stabilizer_facts_from_the_paper():
    """Section 2.2's examples: +Z stabilizes |0> but not |1>, +X stabilizes
    |0> + |1>, -YY stabilizes |00> + |11>, and |000> is the state stabilized
    by ZII, IZI, IIZ. As matrices, and as
    what the oracle's tableau reports for the matching measurements: a fresh
    qubit measures 0 in Z deterministically; on the Bell pair the two Y-basis
    outcomes have odd parity (eigenvalue -1 of YY), the second one fixed by
    the first."""
    P = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
         "Z": np.diag([1, -1])}
    zero, one, plus = np.array([1, 0]), np.array([0, 1]), np.array([1, 1]) / math.sqrt(2)
    np.testing.assert_allclose(P["Z"] @ zero, zero)
    assert not np.allclose(P["Z"] @ one, one)                  # +Z does not stabilize |1>
    np.testing.assert_allclose(P["X"] @ plus, plus)            # +X stabilizes |0> + |1>
    bell = np.array([1, 0, 0, 1]) / math.sqrt(2)
    np.testing.assert_allclose(-np.kron(P["Y"], P["Y"]) @ bell, bell)
    z3 = np.zeros(8)
    z3[0] = 1
    for k in range(3):
        ops = [P["Z"] if i == k else P["I"] for i in range(3)]
        np.testing.assert_allclose(np.kron(np.kron(ops[0], ops[1]), ops[2]) @ z3, z3)
    ref, det = oracle.Circuit("H 0\nMX 0\nX 1\nM 1\n").reference()
    assert list(ref) == [0, 1] and list(det) == [1, 1]         # |0> + |1> reads +1 in X; |1> reads 1 in Z
    ref, det = oracle.Circuit("M 0 1 2\n").reference()
    assert list(ref) == [0, 0, 0] and list(det) == [1, 1, 1]
    ref, det = oracle.Circuit("H 0\nCX 0 1\nMY 0 1\n").reference()
    assert list(det) == [0, 1] and int(ref[0]) ^ int(ref[1]) == 1
    meas, _ = oracle.Circuit("H 0\nCX 0 1\nMY 0 1\n").sample(np.arange(512), seed=2)
    assert np.all(meas[:, 0] ^ meas[:, 1] == 1) and 0.4 < meas[:, 0].mean() < 0.6

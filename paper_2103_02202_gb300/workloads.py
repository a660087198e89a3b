"""Seeded synthetic circuit generators (inputs only).

This module emits circuit *text* in the paper's line format (Section 5.8:
one gate per line, broadcast targets, ``#`` comments, ``REPEAT N {...}``).
It contains none of the simulation arithmetic: both the CUDA library and the
CPU oracle consume the text it produces, so it is the one module they share.

Workload families (the paper prints no circuit files, so the shapes follow
its benchmark descriptions):

* rotated surface-code memory experiments in the Z basis (Fig. 1 / Section 6
  surface-code benchmarks), with the noise model DEPOLARIZE1 after each H
  layer, DEPOLARIZE2 after each CX layer and X_ERROR before every measurement;
* random Clifford circuits (Section 6 random-circuit benchmark, with MR on a
  random 10% of qubits per layer instead of random-basis measurement);
* the repetition code of Appendix A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SurfaceCodeLayout",
    "surface_code_layout",
    "surface_code_memory",
    "random_clifford",
    "repetition_code",
    "batch_circuits",
    "serve_requests",
]


def _fmt_p(p: float) -> str:
    return repr(float(p))


@dataclass
class SurfaceCodeLayout:
    """Qubit numbering of a distance-d rotated surface code patch."""

    d: int
    index: dict            # (x, y) -> qubit index
    data: list             # data qubit indices, in index order
    x_anc: list            # X-type measure qubits, in index order
    z_anc: list            # Z-type measure qubits, in index order
    anc: list              # all measure qubits, in index order
    neighbors: dict        # measure qubit -> {offset: data qubit}

    @property
    def num_qubits(self) -> int:
        return len(self.index)


# CX visiting order of the four diagonal neighbours of a measure qubit.
# X-type measure qubits sweep an "N" and Z-type ones a "Z"; the middle two
# steps are exchanged between the two types so that the X and Z stabilizer
# measurements do not disturb one another.
_X_ORDER = ((1, 1), (1, -1), (-1, 1), (-1, -1))
_Z_ORDER = ((1, 1), (-1, 1), (1, -1), (-1, -1))


def surface_code_layout(d: int) -> SurfaceCodeLayout:
    """Rotated surface code on a (2d+1) x (2d+1) coordinate grid.

    Data qubits sit at odd (x, y); measure qubits at even (x, y). A measure
    qubit at (2i, 2j) is X-type when i + j is even and Z-type otherwise.
    Interior plaquettes are weight 4; on the top and bottom edges only X-type
    weight-2 plaquettes are kept, on the left and right edges only Z-type
    ones; corners are dropped. That yields d^2 data qubits and d^2 - 1
    measure qubits, (d^2 - 1)/2 of each type.
    """
    if d < 2:
        raise ValueError("distance must be >= 2")
    coords = set()
    data_c = [(2 * i + 1, 2 * j + 1) for j in range(d) for i in range(d)]
    coords.update(data_c)
    data_set = set(data_c)
    kind = {}
    for j in range(d + 1):
        for i in range(d + 1):
            x, y = 2 * i, 2 * j
            is_x = (i + j) % 2 == 0
            nb = [(x + dx, y + dy) for dx in (-1, 1) for dy in (-1, 1)
                  if (x + dx, y + dy) in data_set]
            if len(nb) < 2:
                continue
            if len(nb) == 2:
                top_bottom = j == 0 or j == d
                if top_bottom and not is_x:
                    continue
                if not top_bottom and is_x:
                    continue
            kind[(x, y)] = "X" if is_x else "Z"
            coords.add((x, y))
    order = sorted(coords, key=lambda c: (c[1], c[0]))
    index = {c: k for k, c in enumerate(order)}
    data = sorted(index[c] for c in data_c)
    x_anc = sorted(index[c] for c, t in kind.items() if t == "X")
    z_anc = sorted(index[c] for c, t in kind.items() if t == "Z")
    anc = sorted(x_anc + z_anc)
    neighbors = {}
    for c, t in kind.items():
        nbs = {}
        for off in (_X_ORDER if t == "X" else _Z_ORDER):
            dc = (c[0] + off[0], c[1] + off[1])
            if dc in data_set:
                nbs[off] = index[dc]
        neighbors[index[c]] = nbs
    return SurfaceCodeLayout(d, index, data, x_anc, z_anc, anc, neighbors)


def _surface_round(lay: SurfaceCodeLayout, p: float) -> list:
    out = []
    xs = " ".join(map(str, lay.x_anc))
    out.append(f"H {xs}")
    if p > 0:
        out.append(f"DEPOLARIZE1({_fmt_p(p)}) {xs}")
    x_set = set(lay.x_anc)
    for step in range(4):
        pairs = []
        for a in lay.anc:
            if a in x_set:
                off = _X_ORDER[step]
                q = lay.neighbors[a].get(off)
                if q is not None:
                    pairs.append((a, q))
            else:
                off = _Z_ORDER[step]
                q = lay.neighbors[a].get(off)
                if q is not None:
                    pairs.append((q, a))
        flat = " ".join(f"{c} {t}" for c, t in pairs)
        out.append(f"CX {flat}")
        if p > 0:
            out.append(f"DEPOLARIZE2({_fmt_p(p)}) {flat}")
    out.append(f"H {xs}")
    if p > 0:
        out.append(f"DEPOLARIZE1({_fmt_p(p)}) {xs}")
    anc = " ".join(map(str, lay.anc))
    if p > 0:
        out.append(f"X_ERROR({_fmt_p(p)}) {anc}")
    out.append(f"MR {anc}")
    return out


def logical_z_support(lay: SurfaceCodeLayout) -> list:
    """Data qubits of a logical Z: a straight line of data qubits across the
    patch whose overlap with every X plaquette is even (so it commutes with
    all X stabilizers)."""
    coords = {q: c for c, q in lay.index.items()}
    xs = [set(lay.neighbors[a].values()) for a in lay.x_anc]
    for axis in (0, 1):
        lines = {}
        for q in lay.data:
            lines.setdefault(coords[q][axis], []).append(q)
        for key in sorted(lines):
            sup = set(lines[key])
            if len(sup) == lay.d and all(len(sup & x) % 2 == 0 for x in xs):
                return sorted(sup)
    raise RuntimeError("no logical Z line found")


def surface_code_memory(d: int, rounds: int, p: float, observable: bool = False) -> str:
    """Z-basis memory experiment on the distance-d rotated surface code.

    Round 1 carries detectors on Z-type measure qubits only; each later round
    compares every measure qubit with its previous result; the final data
    measurement closes each Z plaquette against its last round. With
    observable=True the final data measurements of a logical Z line are
    logical observable 0 (OBSERVABLE_INCLUDE(0)).
    """
    if rounds < 1:
        raise ValueError("rounds must be >= 1")
    lay = surface_code_layout(d)
    na = len(lay.anc)
    pos_in_round = {a: k for k, a in enumerate(lay.anc)}
    lines = [f"# rotated surface code memory, d={d}, rounds={rounds}, p={p}",
             "R " + " ".join(map(str, range(lay.num_qubits)))]
    lines += _surface_round(lay, p)
    for a in lay.z_anc:
        lines.append(f"DETECTOR rec[-{na - pos_in_round[a]}]")
    if rounds > 1:
        lines.append(f"REPEAT {rounds - 1} {{")
        lines += ["    " + s for s in _surface_round(lay, p)]
        for a in lay.anc:
            k = na - pos_in_round[a]
            lines.append(f"    DETECTOR rec[-{k}] rec[-{k + na}]")
        lines.append("}")
    data = " ".join(map(str, lay.data))
    if p > 0:
        lines.append(f"X_ERROR({_fmt_p(p)}) {data}")
    lines.append(f"M {data}")
    nd = len(lay.data)
    pos_data = {q: k for k, q in enumerate(lay.data)}
    for a in lay.z_anc:
        recs = [f"rec[-{nd - pos_data[q]}]" for q in lay.neighbors[a].values()]
        recs.append(f"rec[-{nd + na - pos_in_round[a]}]")
        lines.append("DETECTOR " + " ".join(recs))
    if observable:
        lines.append("OBSERVABLE_INCLUDE(0) " +
                     " ".join(f"rec[-{nd - pos_data[q]}]" for q in logical_z_support(lay)))
    return "\n".join(lines) + "\n"


def random_clifford(n: int, depth: int, seed: int, *, mr_fraction: float = 0.1,
                    p: float = 0.0) -> str:
    """Random Clifford circuit: per layer, floor(n/4) disjoint random pairs
    each get CX or CZ (random orientation), every other qubit gets H or S,
    then MR on round(mr_fraction * n) random qubits. With p > 0 a
    DEPOLARIZE2 follows the two-qubit gates and a DEPOLARIZE1 the single-qubit
    gates."""
    rng = np.random.default_rng(seed)
    lines = [f"# random clifford n={n} depth={depth} seed={seed}"]
    nm = int(round(mr_fraction * n))
    for _ in range(depth):
        perm = rng.permutation(n)
        npairs = n // 4
        pairs = perm[: 2 * npairs].reshape(npairs, 2)
        rest = perm[2 * npairs:]
        kinds = rng.integers(0, 2, npairs)
        single = rng.integers(0, 2, len(rest))
        cx = pairs[kinds == 0]
        cz = pairs[kinds == 1]
        if len(cx):
            lines.append("CX " + " ".join(f"{a} {b}" for a, b in cx))
        if len(cz):
            lines.append("CZ " + " ".join(f"{a} {b}" for a, b in cz))
        if p > 0 and npairs:
            lines.append(f"DEPOLARIZE2({_fmt_p(p)}) " + " ".join(f"{a} {b}" for a, b in pairs))
        h = rest[single == 0]
        s = rest[single == 1]
        if len(h):
            lines.append("H " + " ".join(map(str, h)))
        if len(s):
            lines.append("S " + " ".join(map(str, s)))
        if p > 0 and len(rest):
            lines.append(f"DEPOLARIZE1({_fmt_p(p)}) " + " ".join(map(str, rest)))
        if nm:
            m = rng.choice(n, size=nm, replace=False)
            lines.append("MR " + " ".join(map(str, m)))
    return "\n".join(lines) + "\n"


def repetition_code(distance: int, rounds: int, p: float) -> str:
    """The noisy repetition code of Appendix A: 2*distance+1 qubits, X_ERROR
    on every qubit, two CNOT chains onto the odd qubits, MR of the odd
    qubits, repeated ``rounds`` times."""
    nq = 2 * distance + 1
    qs = list(range(nq))
    body = [
        f"X_ERROR({_fmt_p(p)}) " + " ".join(map(str, qs)),
        "CNOT " + " ".join(map(str, qs[:-1])),
        "CNOT " + " ".join(map(str, qs[::-1][:-1])),
        "MR " + " ".join(map(str, qs[1::2])),
    ]
    return "REPEAT %d {\n%s\n}\n" % (rounds, "\n".join("    " + b for b in body))


def bacon_shor(d: int, rounds: int, p: float, observable: bool = False) -> str:
    """Memory experiment on the distance-d Bacon-Shor code (the subsystem
    code of the paper's time-to-first-sample benchmarks, Section 6): data
    qubits on a d x d grid, q(r, c) = r * d + c; two-qubit gauge operators
    X(r, c) X(r + 1, c) on vertical pairs and Z(r, c) Z(r, c + 1) on
    horizontal pairs, each measured through an ancilla (X gauges: H, CX
    ancilla -> data twice, H, MR; Z gauges: CX data -> ancilla twice, MR),
    X gauges first each round. The gauges do not commute with each other, so
    most gauge outcomes are random and the inverse-tableau reference sample
    spends its time on random measurements. Noise as in the surface-code
    memory: DEPOLARIZE1 after H layers, DEPOLARIZE2 after CX layers, X_ERROR
    before measurements.

    Detectors compare the stabilizers (products of gauges) between rounds:
    the Z stabilizer of columns (c, c + 1) is the product of the d Z gauges of
    that column pair, the X stabilizer of rows (r, r + 1) that of the d X
    gauges of that row pair; round 1 has Z-stabilizer detectors only, and the
    final Z-basis data measurement closes each Z stabilizer. With
    observable=True the data of column 0 (a logical Z) is observable 0."""
    if d < 2 or rounds < 1:
        raise ValueError("need d >= 2 and rounds >= 1")
    nd = d * d
    xg = [(r, c) for r in range(d - 1) for c in range(d)]        # X(r,c) X(r+1,c)
    zg = [(r, c) for r in range(d) for c in range(d - 1)]        # Z(r,c) Z(r,c+1)
    xa = {g: nd + k for k, g in enumerate(xg)}
    za = {g: nd + len(xg) + k for k, g in enumerate(zg)}
    q = lambda r, c: r * d + c   # noqa: E731
    pp = _fmt_p(p) if p > 0 else None
    xs = " ".join(str(xa[g]) for g in xg)
    zs = " ".join(str(za[g]) for g in zg)
    rnd = [f"H {xs}"]
    if pp:
        rnd.append(f"DEPOLARIZE1({pp}) {xs}")
    for dr in (0, 1):
        pairs = " ".join(f"{xa[(r, c)]} {q(r + dr, c)}" for (r, c) in xg)
        rnd.append(f"CX {pairs}")
        if pp:
            rnd.append(f"DEPOLARIZE2({pp}) {pairs}")
    rnd.append(f"H {xs}")
    if pp:
        rnd.append(f"DEPOLARIZE1({pp}) {xs}")
        rnd.append(f"X_ERROR({pp}) {xs}")
    rnd.append(f"MR {xs}")
    for dc in (0, 1):
        pairs = " ".join(f"{q(r, c + dc)} {za[(r, c)]}" for (r, c) in zg)
        rnd.append(f"CX {pairs}")
        if pp:
            rnd.append(f"DEPOLARIZE2({pp}) {pairs}")
    if pp:
        rnd.append(f"X_ERROR({pp}) {zs}")
    rnd.append(f"MR {zs}")
    nx, nz = len(xg), len(zg)
    per_round = nx + nz
    # record offsets (rec[-k]) of a round's gauges, counted back from the end of the round
    xrec = {g: per_round - k for k, g in enumerate(xg)}
    zrec = {g: nz - k for k, g in enumerate(zg)}

    def zstab(c, back):
        return " ".join(f"rec[-{zrec[(r, c)] + back}]" for r in range(d))

    def xstab(r, back):
        return " ".join(f"rec[-{xrec[(r, c)] + back}]" for c in range(d))

    lines = [f"# Bacon-Shor memory, d={d}, rounds={rounds}, p={p}", "R " + " ".join(map(str, range(nd + nx + nz)))]
    lines += rnd
    for c in range(d - 1):
        lines.append(f"DETECTOR {zstab(c, 0)}")
    if rounds > 1:
        lines.append(f"REPEAT {rounds - 1} {{")
        lines += ["    " + x for x in rnd]
        for c in range(d - 1):
            lines.append(f"    DETECTOR {zstab(c, 0)} {zstab(c, per_round)}")
        for r in range(d - 1):
            lines.append(f"    DETECTOR {xstab(r, 0)} {xstab(r, per_round)}")
        lines.append("}")
    data = " ".join(map(str, range(nd)))
    if pp:
        lines.append(f"X_ERROR({pp}) {data}")
    lines.append(f"M {data}")
    for c in range(d - 1):
        dat = " ".join(f"rec[-{nd - q(r, cc)}]" for r in range(d) for cc in (c, c + 1))
        lines.append(f"DETECTOR {dat} {zstab(c, nd)}")
    if observable:
        lines.append("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{nd - q(r, 0)}]" for r in range(d)))
    return "\n".join(lines) + "\n"


def _log_uniform_int(rng, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_circuits(seed: int = 2021, count: int = 64):
    """Heterogeneous batch: half surface-code memories (d uniform over the odd
    values 3..31, rounds uniform in [d, 2d], p log-uniform in [1e-4, 1e-2]),
    half random Clifford circuits (n uniform in [50, 2000], depth uniform in
    [100, 1000]); shots log-uniform in [1e3, 1e6].

    Returns a list of dicts with keys ``kind``, ``text``, ``shots``, ``seed``
    and the family parameters."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        shots = _log_uniform_int(rng, 1e3, 1e6)
        if k % 2 == 0:
            d = int(rng.choice(np.arange(3, 32, 2)))
            r = int(rng.integers(d, 2 * d + 1))
            p = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-2))))
            p = float("%.4g" % p)
            out.append(dict(kind="surface", d=d, rounds=r, p=p, shots=shots,
                            seed=int(rng.integers(0, 2**63)),
                            text=surface_code_memory(d, r, p)))
        else:
            n = int(rng.integers(50, 2001))
            depth = int(rng.integers(100, 1001))
            cseed = int(rng.integers(0, 2**31))
            out.append(dict(kind="random", n=n, depth=depth, shots=shots,
                            seed=int(rng.integers(0, 2**63)),
                            text=random_clifford(n, depth, cseed)))
    return out


def serve_requests(seed: int = 5, count: int = 10000, rate_hz: float = 1000.0,
                   max_d: int = 51):
    """Poisson request stream for the sampling server: surface codes with odd
    d in [3, max_d] (rounds = d) and p log-uniform in [1e-4, 1e-2], or random
    Clifford circuits; shots log-uniform in [1e3, 1e5]. Circuits repeat from a
    finite catalogue so that compiled circuits can stay resident.

    Returns (catalogue, requests); requests are dicts with ``t`` (arrival
    time, s), ``circuit`` (catalogue index), ``shots`` and ``seed``."""
    rng = np.random.default_rng(seed)
    catalogue = []
    for d in range(3, max_d + 1, 2):
        for p in (1e-4, 1e-3, 1e-2):
            catalogue.append(dict(kind="surface", d=d, rounds=d, p=p,
                                  text=None))
    for k in range(8):
        n = int(rng.integers(50, 2001))
        depth = int(rng.integers(100, 1001))
        catalogue.append(dict(kind="random", n=n, depth=depth, cseed=1000 + k,
                              text=None))
    t = 0.0
    reqs = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        reqs.append(dict(t=t, circuit=int(rng.integers(0, len(catalogue))),
                         shots=_log_uniform_int(rng, 1e3, 1e5),
                         seed=int(rng.integers(0, 2**63))))
    return catalogue, reqs


def catalogue_text(entry: dict) -> str:
    """Circuit text for a ``serve_requests`` catalogue entry."""
    if entry.get("text"):
        return entry["text"]
    if entry["kind"] == "surface":
        return surface_code_memory(entry["d"], entry["rounds"], entry["p"])
    return random_clifford(entry["n"], entry["depth"], entry["cseed"])

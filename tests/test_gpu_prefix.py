"""Tableau prefix states (reuse across slight variations of a circuit, the
paper's Section 7 outlook): the inverse tableau at a top-level REPEAT boundary
depends only on the noiseless skeleton before it, so a memory experiment that
differs from an earlier one only after its REPEAT block resumes its reference
computation there. Every resumed reference must equal the oracle's, bit for
bit, for tails with random measurements, feed-forward on records from before
the cut, a further REPEAT block, and on the single-CTA, multi-CTA and batched
tableau paths."""
import numpy as np
import pytest

import oracle
import paper_2103_02202_gb300 as sg
from paper_2103_02202_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_02202_gb300 import build
    build.build()
    yield
    sg.stim_prefix_cache_set(1 << 30)
    sg.stim_reference_cache_set(256 << 20)


_BASE = {}


def _fresh(prefix_budget=1 << 30):
    """Empty caches; the counters of _stats() start again from zero."""
    sg.stim_reference_cache_set(0)
    sg.stim_reference_cache_set(256 << 20)
    sg.stim_prefix_cache_set(0)
    sg.stim_prefix_cache_set(prefix_budget)
    _BASE.update(sg.stim_prefix_cache_stats())


def _stats():
    """Prefix-state counters since the last _fresh() (entries and bytes as held)."""
    st = sg.stim_prefix_cache_stats()
    return {k: st[k] - _BASE[k] if k in ("resumes", "saves") else st[k] for k in st}


def _split(text):
    """(source through the top-level REPEAT block, data qubits, ancilla qubits)."""
    end = text.index("\n}\n", text.index("REPEAT")) + 3
    lines = text.splitlines()
    data = [ln for ln in lines if ln.startswith("M ")][-1].split()[1:]
    anc = [ln.strip() for ln in lines if ln.strip().startswith("MR ")][0].split()[1:]
    return text[:end], [int(q) for q in data], [int(q) for q in anc]


def _q(v):
    return " ".join(map(str, v))


TAILS = [
    # readout in the X basis: random outcomes after the cut
    lambda d, a: f"H {_q(d)}\nM {_q(d)}\n",
    # gates, then a classically controlled X on the last record before the cut
    lambda d, a: f"CX {d[0]} {d[1]}\nS {d[2]}\nCX rec[-1] {d[3]}\nCZ rec[-2] {d[0]}\nM {_q(d)}\nMR {_q(a[:2])}\n",
    # a further REPEAT block of X-type checks, then the readout
    lambda d, a: f"REPEAT 3 {{\nH {_q(a)}\nCX {a[0]} {d[0]} {a[1]} {d[1]}\nH {_q(a)}\nMR {_q(a)}\n}}\nM {_q(d)}\n",
]


def _bits(t, M):
    w = t.cpu().numpy().view(np.uint64)
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:M]


def _check_against_oracle(text, c):
    ref, det = c.reference()
    torch.cuda.synchronize()
    M = c.num_measurements
    oref, odet = oracle.Circuit(text).reference()
    np.testing.assert_array_equal(_bits(ref, M), oref)
    np.testing.assert_array_equal(_bits(det, M), odet)


@pytest.mark.parametrize("dist", [3, 7, 15])
@pytest.mark.parametrize("k", range(len(TAILS)))
def test_resumed_reference_matches_oracle(dist, k):
    _fresh()
    base = W.surface_code_memory(dist, 6, 1e-3)
    head, data, anc = _split(base)
    a = sg.Circuit(base)
    a.reference()
    torch.cuda.synchronize()
    st = _stats()
    assert st["saves"] == 1 and st["entries"] == 1 and st["resumes"] == 0
    text = head + TAILS[k](data, anc)
    b = sg.Circuit(text)
    _check_against_oracle(text, b)
    st = _stats()
    assert st["resumes"] == 1
    # the tail with a REPEAT block stores the state after that block too
    assert st["saves"] == (2 if k == 2 else 1)
    a.close()
    b.close()


def test_resumed_samples_match_oracle():
    """Frame samples drawn against a resumed reference equal the oracle's."""
    _fresh()
    base = W.surface_code_memory(5, 8, 0.01)
    head, data, anc = _split(base)
    sg.Circuit(base).reference()
    text = head + TAILS[1](data, anc)
    c = sg.Circuit(text)
    S = 500
    m, _ = c.sample(S, 17, dets=False)
    torch.cuda.synchronize()
    assert _stats()["resumes"] == 1
    bits = np.unpackbits(m.cpu().numpy().view(np.uint64).view(np.uint8).reshape(m.shape[0], -1), axis=1,
                         bitorder="little")[:, :S].T
    om, _ = oracle.Circuit(text).sample(np.arange(S), 17, threads=8)
    np.testing.assert_array_equal(bits, om)
    c.close()


def test_different_qubit_count_does_not_resume():
    _fresh()
    base = W.surface_code_memory(5, 4, 1e-3)
    head, data, anc = _split(base)
    sg.Circuit(base).reference()
    extra = max(data + anc) + 1
    text = head + f"CX {data[0]} {extra}\nM {extra}\nM {_q(data)}\n"
    c = sg.Circuit(text)
    _check_against_oracle(text, c)
    assert _stats()["resumes"] == 0
    c.close()


def test_fewer_rounds_do_not_resume():
    """A stored state after four iterations of the round block serves no
    memory that repeats the block three times."""
    _fresh()
    sg.Circuit(W.surface_code_memory(5, 5, 1e-3)).reference()
    text = W.surface_code_memory(5, 4, 1e-3)
    c = sg.Circuit(text)
    _check_against_oracle(text, c)
    st = _stats()
    assert st["resumes"] == 0 and st["saves"] == 2
    c.close()


@pytest.mark.parametrize("dist", [3, 9, 17])
def test_more_rounds_resume_inside_the_loop(dist):
    """A sweep over the number of rounds: each memory resumes inside its
    REPEAT block from the state the previous one stored after its own, and
    stores its state for the next."""
    _fresh()
    rounds = [4, 6, 9, 10]
    for i, r in enumerate(rounds):
        text = W.surface_code_memory(dist, r, 1e-3)
        c = sg.Circuit(text)
        _check_against_oracle(text, c)
        st = _stats()
        assert st["resumes"] == i and st["saves"] == i + 1
        c.close()


def test_other_body_does_not_resume():
    """Same source before the block, another body: no resume."""
    _fresh()
    base = W.surface_code_memory(5, 4, 1e-3)
    sg.Circuit(base).reference()
    text = base.replace("REPEAT 3 {\n", "REPEAT 5 {\n    S 0\n", 1)
    assert text != base
    c = sg.Circuit(text)
    _check_against_oracle(text, c)
    assert _stats()["resumes"] == 0
    c.close()


def test_recompute_neither_stores_nor_resumes():
    _fresh()
    base = W.surface_code_memory(5, 4, 1e-3)
    head, data, anc = _split(base)
    sg.Circuit(base).reference(recompute=True)
    assert _stats()["saves"] == 0
    sg.Circuit(base).reference()
    text = head + TAILS[0](data, anc)
    c = sg.Circuit(text)
    c.reference(recompute=True)
    torch.cuda.synchronize()
    st = _stats()
    assert st["saves"] == 1 and st["resumes"] == 0
    c.close()


def test_budget_off_and_eviction():
    _fresh(prefix_budget=0)
    base = W.surface_code_memory(7, 4, 1e-3)
    head, data, anc = _split(base)
    sg.Circuit(base).reference()
    st = _stats()
    assert st["saves"] == 0 and st["entries"] == 0
    text = head + TAILS[0](data, anc)
    _check_against_oracle(text, sg.Circuit(text))
    # room for one d=7 state: a second prefix evicts the first
    _fresh()
    sg.Circuit(base).reference()
    one = _stats()["bytes"]
    assert one > 0
    _fresh(prefix_budget=one + one // 2)
    sg.Circuit(base).reference()
    sg.Circuit(W.surface_code_memory(7, 5, 1e-3)).reference()      # resumes inside its loop
    torch.cuda.synchronize()
    st = _stats()
    assert st["entries"] == 1 and st["saves"] == 2 and st["bytes"] <= one + one // 2
    c = sg.Circuit(text)
    _check_against_oracle(text, c)
    assert _stats()["resumes"] == st["resumes"]      # base's state was evicted


def test_many_side_by_side_and_batched():
    """stim_reference_many: small circuits on the single-CTA tableau (which
    stores states too) and large ones in a batched launch (which resumes)."""
    _fresh()
    texts, tails = [], []
    for dist in (3, 5, 15, 21):
        base = W.surface_code_memory(dist, 5, 1e-3)
        head, data, anc = _split(base)
        texts.append(base)
        tails.append(head + TAILS[0](data, anc))
    bases = [sg.Circuit(t) for t in texts]
    sg.stim_reference_many([c.handle for c in bases])
    torch.cuda.synchronize()
    # the single-CTA ones stored their states; the batched launch does not split
    assert _stats()["saves"] == 2
    sg.stim_reference_cache_set(0)      # recompute the large ones one by one, storing their states
    sg.stim_reference_cache_set(256 << 20)
    for i in (2, 3):
        sg.Circuit(texts[i]).reference()
    torch.cuda.synchronize()
    assert _stats()["saves"] == 4
    cs = [sg.Circuit(t) for t in tails]
    sg.stim_reference_many([c.handle for c in cs])
    torch.cuda.synchronize()
    assert _stats()["resumes"] == 4
    for t, c in zip(tails, cs):
        _check_against_oracle(t, c)


def _random_block(rng, n, L):
    """L random Clifford, Pauli, measurement and reset lines on n qubits, with
    classically controlled Paulis on recent records (after the first
    measurement)."""
    lines, measured = [], False
    for _ in range(L):
        g = str(rng.choice(["H", "S", "S_DAG", "SQRT_X", "X", "Y", "Z", "CX", "CZ", "M", "MR", "R", "FF"]))
        k = int(rng.integers(1, max(2, n // 3)))
        if g in ("CX", "CZ"):
            q = rng.choice(n, 2 * min(k, n // 2), replace=False)
            lines.append(f"{g} {_q(q)}")
        elif g == "FF":
            if measured:
                lines.append(f"CX rec[-1] {int(rng.integers(n))}")
                lines.append(f"CZ rec[-1] {int(rng.integers(n))}")
        else:
            lines.append(f"{g} {_q(rng.choice(n, k, replace=False))}")
            measured |= g in ("M", "MR")
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_share_a_prefix(seed):
    """Random prefixes (Pauli signs, random and deterministic outcomes, feed-
    forward) ending in a REPEAT block; two different random tails."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.choice([23, 90, 300, 700]) if seed < 4 else rng.integers(30, 400))
    prefix = f"H {n - 1}\nM 0\n" + _random_block(rng, n, 30) + f"REPEAT {int(rng.integers(2, 5))} {{\n" + \
        _random_block(rng, n, 12) + "}\n"
    tails = [_random_block(rng, n, 25) + f"M {_q(range(n))}\n" for _ in range(2)]
    _fresh()
    a = sg.Circuit(prefix + tails[0])
    _check_against_oracle(prefix + tails[0], a)
    assert _stats()["saves"] == 1
    b = sg.Circuit(prefix + tails[1])
    _check_against_oracle(prefix + tails[1], b)
    assert _stats()["resumes"] == 1
    a.close()
    b.close()

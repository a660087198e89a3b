"""GPU vs oracle parity through the C ABI: reference samples, measurement
records and detection events must be bit-identical to the CPU oracle on the
same seeded inputs, for every tile shape, layout and shot split."""
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
    torch.cuda.init()
    yield


def words_to_bits(words: np.ndarray, nbits: int) -> np.ndarray:
    """(R, nwords) uint64 -> (R, nbits) uint8 (LSB-first)."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    b = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], -1), axis=1, bitorder="little")
    return b[:, :nbits]


def to_np(t):
    return t.cpu().numpy().view(np.uint64)


def gpu_sample(text, shots, seed, shot_offset=0, hint=None):
    c = sg.Circuit(text)
    m, d = c.sample(shots, seed, shot_offset=shot_offset, hint=hint)
    torch.cuda.synchronize()
    M, D = c.num_measurements, c.num_detectors
    mb = words_to_bits(to_np(m), shots).T if M else np.zeros((shots, 0), np.uint8)
    db = words_to_bits(to_np(d), shots).T if D else np.zeros((shots, 0), np.uint8)
    c.close()
    return mb, db


def gpu_reference(text):
    c = sg.Circuit(text)
    r, d = c.reference()
    torch.cuda.synchronize()
    M = c.num_measurements
    out = (words_to_bits(to_np(r)[None, :], M)[0], words_to_bits(to_np(d)[None, :], M)[0])
    c.close()
    return out


def _rand_circuit(rng, n, L, noise=True):
    lines = []
    for _ in range(L):
        g = str(rng.choice(["H", "S", "CX", "CZ", "M", "MR", "R", "BCAST", "NOISE"]))
        if g == "BCAST":
            g2 = str(rng.choice(["H", "S", "M", "MR", "R"]))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g2} " + " ".join(map(str, rng.choice(n, k, replace=False))))
        elif g in ("CX", "CZ"):
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{g} {a} {b}")
        elif g == "NOISE":
            if not noise:
                continue
            ch = str(rng.choice(["X_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2"]))
            p = float(rng.choice([0.01, 0.2, 0.5, 1.0]))
            if ch == "DEPOLARIZE2":
                a, b = rng.choice(n, 2, replace=False)
                lines.append(f"{ch}({p}) {a} {b}")
            else:
                lines.append(f"{ch}({p}) {rng.integers(n)}")
        else:
            lines.append(f"{g} {rng.integers(n)}")
    lines.append("M " + " ".join(map(str, range(n))))
    lines.append("DETECTOR rec[-1] rec[-2]")
    return "\n".join(lines) + "\n"


# ---------------------------------------------------------------------------
# reference sample (inverse tableau)
# ---------------------------------------------------------------------------
REF_CIRCUITS = {
    "surface_d3_r3": W.surface_code_memory(3, 3, 1e-3),
    "surface_d5_r5": W.surface_code_memory(5, 5, 1e-3),
    "surface_d25_r25": W.surface_code_memory(25, 25, 1e-3),
    "repetition": W.repetition_code(5, 20, 0.01),
    "random_clifford_200": W.random_clifford(200, 60, 3),
    "random_clifford_700": W.random_clifford(700, 40, 4),
    "bell": "H 0\nCX 0 1\nM 0 1\n",
    "reset_after_one": "H 0\nS 0\nS 0\nH 0\nMR 0\nM 0\nR 0\nM 0\n",
}


@pytest.mark.parametrize("name", sorted(REF_CIRCUITS))
def test_reference_matches_oracle(name):
    text = REF_CIRCUITS[name]
    ref, det = gpu_reference(text)
    oref, odet = oracle.Circuit(text).reference()
    np.testing.assert_array_equal(ref, oref)
    np.testing.assert_array_equal(det, odet)


def test_reference_random_small_circuits():
    rng = np.random.default_rng(7)
    for _ in range(40):
        n = int(rng.integers(2, 70))
        text = _rand_circuit(rng, n, int(rng.integers(5, 120)))
        ref, det = gpu_reference(text)
        oref, odet = oracle.Circuit(text).reference()
        np.testing.assert_array_equal(ref, oref, err_msg=text)
        np.testing.assert_array_equal(det, odet, err_msg=text)


def test_reference_wide_fanout_bursts_match_oracle():
    """An 1800-qubit random Clifford circuit of depth 400: once scrambled, its
    random measurements fan out to more rows of 57 words than one CTA takes in
    a row-major burst, so the burst cluster walks them (the cluster-wide chunk
    sums of the fan-out: several hundred such layers); the reference equals
    the oracle's, recomputed as well as cold."""
    text = W.random_clifford(1800, 400, 11)
    ref, det = gpu_reference(text)
    oref, odet = oracle.Circuit(text).reference()
    np.testing.assert_array_equal(ref, oref)
    np.testing.assert_array_equal(det, odet)
    c = sg.Circuit(text)
    r2, d2 = c.reference(recompute=True)
    torch.cuda.synchronize()
    M = c.num_measurements
    np.testing.assert_array_equal(words_to_bits(to_np(r2)[None, :], M)[0], oref)
    np.testing.assert_array_equal(words_to_bits(to_np(d2)[None, :], M)[0], odet)
    c.close()


def test_reference_recompute_is_stable():
    c = sg.Circuit(W.random_clifford(300, 30, 9))
    r1, d1 = c.reference()
    r2, d2 = c.reference(recompute=True)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2) and torch.equal(d1, d2)
    c.close()


# ---------------------------------------------------------------------------
# frame sampling
# ---------------------------------------------------------------------------
def test_surface_d3_full_parity():
    """The d=3, 3-round, p=1e-3, 1024-shot, seed-0 workload: every shot."""
    text = W.surface_code_memory(3, 3, 1e-3)
    mb, db = gpu_sample(text, 1024, 0)
    om, od = oracle.Circuit(text).sample(np.arange(1024), 0, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


@pytest.mark.parametrize("d", [23, 27, 31, 37])
def test_default_tiles_of_mid_size_circuits(d):
    """Default tile shapes for 1,000-2,700-qubit circuits (the library sizes
    the CTA from the qubits' shared memory; every CTA must be whole warps)."""
    text = W.surface_code_memory(d, 2, 0.01)
    mb, db = gpu_sample(text, 640, 9)
    om, od = oracle.Circuit(text).sample(np.arange(640), 9, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


@pytest.mark.parametrize("shots", [1, 63, 64, 65, 1000, 3 * 64 * 16 + 5])
def test_ragged_shot_counts(shots):
    text = W.surface_code_memory(3, 2, 0.02)
    mb, db = gpu_sample(text, shots, 12345)
    om, od = oracle.Circuit(text).sample(np.arange(shots), 12345, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


def test_random_circuits_with_all_noise_kinds():
    rng = np.random.default_rng(11)
    for _ in range(12):
        n = int(rng.integers(2, 40))
        text = _rand_circuit(rng, n, int(rng.integers(10, 80)))
        shots = int(rng.integers(1, 700))
        seed = int(rng.integers(0, 2**63))
        mb, db = gpu_sample(text, shots, seed)
        om, od = oracle.Circuit(text).sample(np.arange(shots), seed, threads=8)
        np.testing.assert_array_equal(mb, om, err_msg=text)
        np.testing.assert_array_equal(db, od, err_msg=text)


@pytest.mark.parametrize("hint", [(1, 64, 0, 1), (2, 128, 0, 1), (4, 256, 0, 1), (8, 512, 0, 1),
                                  (1, 256, 1, 1), (4, 128, 1, 1), (8, 256, 1, 1),
                                  (1, 128, 0, 2), (2, 256, 0, 4), (4, 512, 0, 8), (8, 512, 0, 8),
                                  (1, 32, 0, 8)])
def test_tile_shapes_are_invisible(hint):
    text = W.surface_code_memory(5, 4, 5e-3)
    base_m, base_d = gpu_sample(text, 2000, 99)
    m, d = gpu_sample(text, 2000, 99, hint=hint)
    np.testing.assert_array_equal(m, base_m)
    np.testing.assert_array_equal(d, base_d)


def test_shot_offset_splits_are_invisible():
    text = W.surface_code_memory(5, 3, 1e-2)
    full_m, full_d = gpu_sample(text, 640, 5)
    a_m, a_d = gpu_sample(text, 192, 5)
    b_m, b_d = gpu_sample(text, 448, 5, shot_offset=192)
    np.testing.assert_array_equal(np.concatenate([a_m, b_m]), full_m)
    np.testing.assert_array_equal(np.concatenate([a_d, b_d]), full_d)
    om, od = oracle.Circuit(text).sample(np.arange(448), 5, shot_offset=192, threads=8)
    np.testing.assert_array_equal(b_m, om)


def test_layouts_and_host_outputs_agree():
    text = W.surface_code_memory(3, 3, 0.05)
    c = sg.Circuit(text)
    S = 777
    mm, dm = c.sample(S, 3)
    ms, ds = c.sample(S, 3, shot_major=True)
    hm, hd = c.sample_host(S, 3)
    hs, hds = c.sample_host(S, 3, shot_major=True)
    torch.cuda.synchronize()
    M, D = c.num_measurements, c.num_detectors
    meas = words_to_bits(to_np(mm), S)
    np.testing.assert_array_equal(words_to_bits(to_np(ms), M), meas.T)
    np.testing.assert_array_equal(words_to_bits(hm, S), meas)
    np.testing.assert_array_equal(words_to_bits(hs, M), meas.T)
    dets = words_to_bits(to_np(dm), S)
    np.testing.assert_array_equal(words_to_bits(to_np(ds), D), dets.T)
    np.testing.assert_array_equal(words_to_bits(hd, S), dets)
    np.testing.assert_array_equal(words_to_bits(hds, D), dets.T)
    # padding bits are zero in both layouts
    assert np.all(to_np(mm)[:, -1] >> np.uint64(S % 64) == 0)
    assert np.all(to_np(ms)[:, -1] >> np.uint64(M % 64) == 0)
    c.close()


def test_async_host_outputs_on_two_streams_agree():
    """STIM_ASYNC host copies from alternating streams (double-buffered staging)
    equal synchronous device outputs, call for call."""
    text = W.surface_code_memory(5, 5, 0.02)
    c = sg.Circuit(text)
    S = 4000
    M, D = c.num_measurements, c.num_detectors
    nw = (S + 63) // 64
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    calls = 6
    host_m = [torch.empty((M, nw), dtype=torch.int64, pin_memory=True) for _ in range(calls)]
    host_d = [torch.empty((D, nw), dtype=torch.int64, pin_memory=True) for _ in range(calls)]
    for i in range(calls):
        st = streams[i % 2]
        sg.stim_frame_sample_ex(c.handle, S, 11 + i, 64 * i, host_m[i].data_ptr(), host_d[i].data_ptr(),
                                sg.STIM_HOST | sg.STIM_ASYNC, None, st.cuda_stream)
    torch.cuda.synchronize()
    for i in range(calls):
        mm, dm = c.sample(S, 11 + i, shot_offset=64 * i)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host_m[i].numpy().view(np.uint64), to_np(mm))
        np.testing.assert_array_equal(host_d[i].numpy().view(np.uint64), to_np(dm))
    c.close()


def test_noiseless_surface_detectors_vanish_at_scale():
    text = W.surface_code_memory(15, 15, 0.0)
    c = sg.Circuit(text)
    _, d = c.sample(65536, 1, meas=False)
    torch.cuda.synchronize()
    assert int(d.count_nonzero()) == 0
    c.close()


def test_surface_d25_bench_size_sampled_parity():
    """d=25, 25 rounds, p=1e-3, 131072 shots in the default launch: compare the
    first shot, the last shot, a word boundary and 200 random shots."""
    text = W.surface_code_memory(25, 25, 1e-3)
    S = 131072
    c = sg.Circuit(text)
    m, d = c.sample(S, 0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([[0, 63, 64, S - 1], rng.choice(S, 200, replace=False)]))
    cols = torch.as_tensor(pick // 64, device="cuda")
    bits = torch.as_tensor(pick % 64, device="cuda")
    gm = ((m[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T
    gd = ((d[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T
    om, od = oracle.Circuit(text).sample(pick, 0, threads=8)
    np.testing.assert_array_equal(gm, om)
    np.testing.assert_array_equal(gd, od)
    c.close()


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_cluster_partitions_random_circuits(cluster):
    """Qubit slices split over a cluster: two-qubit gates and DEPOLARIZE2 that
    cross slices go through distributed shared memory."""
    rng = np.random.default_rng(100 + cluster)
    for _ in range(4):
        n = int(rng.integers(cluster, 60))
        text = _rand_circuit(rng, n, 60)
        shots = int(rng.integers(1, 900))
        mb, db = gpu_sample(text, shots, 3, hint=(int(rng.choice([1, 2, 4])), 128, 0, cluster))
        om, od = oracle.Circuit(text).sample(np.arange(shots), 3, threads=8)
        np.testing.assert_array_equal(mb, om, err_msg=text)
        np.testing.assert_array_equal(db, od, err_msg=text)


def test_random_clifford_parity():
    text = W.random_clifford(500, 40, 21)
    mb, db = gpu_sample(text, 300, 77)
    om, od = oracle.Circuit(text).sample(np.arange(300), 77, threads=8)
    np.testing.assert_array_equal(mb, om)


def test_edge_cases():
    # empty circuit, no measurements, zero shots
    for text in ("", "H 0\nCX 0 1\n", "X_ERROR(0.5) 3\n"):
        c = sg.Circuit(text)
        c.sample(100, 1)
        c.reference()
        c.close()
    c = sg.Circuit("H 0\nM 0\n")
    c.sample(0, 1)
    c.close()
    torch.cuda.synchronize()
    # p = 1 noise flips every shot
    mb, _ = gpu_sample("X_ERROR(1) 0 1 2\nM 0 1 2\n", 200, 1)
    assert mb.all()


@pytest.mark.slow
def test_surface_d100_bench_configuration_sampled_parity():
    """d=100, 100 rounds, p=1e-3, 16384 shots at shot offset 16384 (step 1
    of the benchmark), default launch (thread-block clusters): the first and
    last shots, a word boundary and 256 random shots vs the oracle, and the
    full reference sample vs the oracle's tableau. A second call of 16377
    shots (a partial last word) gives the same bits on every shared shot and
    zero padding, and its last shot matches the oracle too."""
    text = W.surface_code_memory(100, 100, 1e-3)
    S, off = 16384, 16384
    c = sg.Circuit(text)
    ref, det = c.reference()
    _, d = c.sample(S, 2021, shot_offset=off, meas=False)
    Sp = S - 7
    _, dp = c.sample(Sp, 2021, shot_offset=off, meas=False)
    # the same events computed inside the frame kernel (flip ring, no records)
    _, dk = c.sample(S, 2021, shot_offset=off, meas=False, events_in_kernel=True)
    torch.cuda.synchronize()
    assert torch.equal(dk, d)
    o = oracle.Circuit(text)
    oref, odet = o.reference()
    M = c.num_measurements
    np.testing.assert_array_equal(words_to_bits(to_np(ref)[None, :], M)[0], oref)
    np.testing.assert_array_equal(words_to_bits(to_np(det)[None, :], M)[0], odet)
    rnd = np.random.default_rng(3).choice(S, 256, replace=False)
    pick = np.unique(np.concatenate([[0, 1, 63, 64, 8191, Sp - 1, S - 1], rnd]))
    cols = torch.as_tensor(pick // 64, device="cuda")
    bits = torch.as_tensor(pick % 64, device="cuda")
    gd = ((d[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T
    _, od = o.sample(pick, 2021, shot_offset=off, threads=16, ref=oref)
    np.testing.assert_array_equal(gd, od)
    # partial last word: same bits on shared shots, padding bits zero
    nw = (Sp + 63) // 64
    assert torch.equal(dp[:, :nw - 1], d[:, :nw - 1])
    keep = (1 << (Sp % 64)) - 1
    assert torch.equal(dp[:, nw - 1] & ~keep, torch.zeros_like(dp[:, nw - 1]))
    assert torch.equal(dp[:, nw - 1] & keep, d[:, nw - 1] & keep)
    c.close()


def _lists_from_bits(bits):
    """(shots, D) uint8 -> (begin, detectors) per-shot ascending lists."""
    begin = [0]
    dets = []
    for row in bits:
        idx = np.flatnonzero(row)
        dets.extend(idx.tolist())
        begin.append(len(dets))
    return np.array(begin, np.uint64), np.array(dets, np.uint32)


def test_detection_lists_match_oracle():
    """stim_frame_sample_detections (per-shot fired-detector lists, host) equals
    the oracle's detection events of the same shots."""
    text = W.surface_code_memory(5, 6, 0.02)
    S, off = 3001, 128
    c = sg.Circuit(text)
    begin, dets = c.sample_detections(S, 42, shot_offset=off)
    _, od = oracle.Circuit(text).sample(np.arange(S), 42, shot_offset=off, threads=8)
    eb, ed = _lists_from_bits(od)
    np.testing.assert_array_equal(begin, eb)
    np.testing.assert_array_equal(dets, ed)
    # device outputs give the same lists
    dbeg = torch.zeros(S + 1, dtype=torch.int64, device="cuda")
    ddet = torch.zeros(len(ed) + 5, dtype=torch.int32, device="cuda")
    n = sg.stim_frame_sample_detections(c.handle, S, 42, off, dbeg.data_ptr(), ddet.data_ptr(), len(ed) + 5,
                                        sg.STIM_DEVICE, torch.cuda.current_stream().cuda_stream)
    assert n == len(ed)
    np.testing.assert_array_equal(dbeg.cpu().numpy().view(np.uint64), eb)
    np.testing.assert_array_equal(ddet.cpu().numpy()[:n].view(np.uint32), ed)
    c.close()


def test_detection_lists_capacity_and_edges():
    text = W.surface_code_memory(3, 3, 0.05)
    c = sg.Circuit(text)
    total = sg.stim_frame_sample_detections(c.handle, 500, 7, 0, 0, 0, 0, sg.STIM_HOST, 0)
    assert total > 10
    begin = np.zeros(501, np.uint64)
    small = np.zeros(5, np.uint32)
    with pytest.raises(sg.StimError) as ei:
        sg.stim_frame_sample_detections(c.handle, 500, 7, 0, begin.ctypes.data, small.ctypes.data, 5,
                                        sg.STIM_HOST, 0)
    assert ei.value.code == sg.STIM_E_CAPACITY
    fb, fd = c.sample_detections(500, 7)
    assert int(fb[-1]) == total and len(fd) == total
    np.testing.assert_array_equal(begin, fb)          # offsets are written in full
    np.testing.assert_array_equal(small, fd[:5])      # and the first `capacity` entries
    b0, d0 = c.sample_detections(0, 7)
    assert b0.tolist() == [0] and len(d0) == 0
    c.close()
    nodet = sg.Circuit("H 0\nM 0\n")
    b1, d1 = nodet.sample_detections(100, 1)
    assert np.all(b1 == 0) and len(d1) == 0
    nodet.close()


WIDE_1Q = ["H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG", "SQRT_Y", "SQRT_Y_DAG"]
WIDE_COLLAPSE = ["M", "MR", "R", "MX", "MY", "MRX", "MRY", "RX", "RY"]
WIDE_NOISE = ["X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2"]


def _wide_circuit(rng, n, L, feedforward=False):
    lines = []
    nmeas = 0
    for _ in range(L):
        kind = rng.random()
        if feedforward and nmeas and kind < 0.15:
            k = int(rng.integers(1, min(nmeas, 12) + 1))
            q = int(rng.integers(n))
            lines.append(f"CX rec[-{k}] {q}" if rng.random() < 0.5 else f"CZ {q} rec[-{k}]")
            continue
        if kind < 0.4:
            g = str(rng.choice(WIDE_1Q))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g} " + " ".join(map(str, rng.choice(n, k, replace=False))))
        elif kind < 0.6:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        elif kind < 0.8:
            ch = str(rng.choice(WIDE_NOISE))
            p = float(rng.choice([0.02, 0.3, 1.0]))
            if ch == "DEPOLARIZE2":
                a, b = rng.choice(n, 2, replace=False)
                lines.append(f"{ch}({p}) {a} {b}")
            else:
                lines.append(f"{ch}({p}) " + " ".join(map(str, rng.choice(n, int(rng.integers(1, n + 1)), replace=False))))
        else:
            g = str(rng.choice(WIDE_COLLAPSE))
            k = int(rng.integers(1, n + 1))
            lines.append(f"{g} " + " ".join(map(str, rng.choice(n, k, replace=False))))
            if g[0] == "M":
                lines.append("DETECTOR rec[-1]")
                nmeas += k
    lines.append(str(rng.choice(["M", "MX", "MY"])) + " " + " ".join(map(str, range(n))))
    lines.append("DETECTOR rec[-1] rec[-2]")
    return "\n".join(lines) + "\n"


def test_wide_gate_set_reference_and_samples_match_oracle():
    """The wider gate set (one-qubit Cliffords, Paulis, Y_ERROR, X/Y-basis
    measurements and resets): GPU reference and records equal the oracle's."""
    rng = np.random.default_rng(77)
    for it in range(30):
        n = int(rng.integers(2, 40))
        text = _wide_circuit(rng, n, int(rng.integers(5, 60)))
        gr, gd = gpu_reference(text)
        orf, odf = oracle.Circuit(text).reference()
        np.testing.assert_array_equal(gr, orf, err_msg=text)
        np.testing.assert_array_equal(gd, odf, err_msg=text)
        shots = int(rng.integers(1, 700))
        mb, db = gpu_sample(text, shots, 1000 + it)
        om, od = oracle.Circuit(text).sample(np.arange(shots), 1000 + it, threads=8)
        np.testing.assert_array_equal(mb, om, err_msg=text)
        np.testing.assert_array_equal(db, od, err_msg=text)


@pytest.mark.parametrize("hint", [(1, 64, 0, 2), (4, 128, 0, 1), (8, 256, 0, 1), (2, 128, 1, 1)])
def test_wide_gate_set_tile_shapes(hint):
    rng = np.random.default_rng(78)
    text = _wide_circuit(rng, 30, 80)
    mb, db = gpu_sample(text, 1000, 5, hint=hint)
    om, od = oracle.Circuit(text).sample(np.arange(1000), 5, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


def _feedforward_loop_circuit(rng, n, reps):
    """A REPEAT body whose classically controlled ops read records of the
    previous iteration and of the measurements before the loop."""
    body = []
    for _ in range(int(rng.integers(4, 12))):
        kind = rng.random()
        if kind < 0.3:
            k = int(rng.integers(1, n + 1))
            q = int(rng.integers(n))
            body.append(f"CX rec[-{k}] {q}" if rng.random() < 0.5 else f"CZ rec[-{k}] {q}")
        elif kind < 0.55:
            a, b = rng.choice(n, 2, replace=False)
            body.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        elif kind < 0.75:
            body.append(f"{str(rng.choice(WIDE_1Q))} {int(rng.integers(n))}")
        else:
            ch = str(rng.choice(["X_ERROR", "Z_ERROR", "DEPOLARIZE1"]))
            body.append(f"{ch}(0.05) {int(rng.integers(n))}")
    body.append("MR " + " ".join(map(str, range(n))))
    body.append("DETECTOR rec[-1] rec[-2]")
    return ("H " + " ".join(map(str, range(n))) + "\nM " + " ".join(map(str, range(n))) +
            f"\nREPEAT {reps} {{\n" + "\n".join(body) + "\n}\nM 0\nDETECTOR rec[-1]\n")


def test_feedforward_reference_and_samples_match_oracle():
    """Classically controlled X/Z (CX rec[-k] q, CZ q rec[-k]): GPU reference
    and records equal the oracle's, including loops that read records of the
    previous iteration."""
    rng = np.random.default_rng(2105)
    for it in range(30):
        n = int(rng.integers(2, 40))
        if it % 3 == 2:
            text = _feedforward_loop_circuit(rng, min(n, 8), int(rng.integers(2, 30)))
        else:
            text = _wide_circuit(rng, n, int(rng.integers(5, 60)), feedforward=True)
        gr, gd = gpu_reference(text)
        orf, odf = oracle.Circuit(text).reference()
        np.testing.assert_array_equal(gr, orf, err_msg=text)
        np.testing.assert_array_equal(gd, odf, err_msg=text)
        shots = int(rng.integers(1, 700))
        mb, db = gpu_sample(text, shots, 3000 + it)
        om, od = oracle.Circuit(text).sample(np.arange(shots), 3000 + it, threads=8)
        np.testing.assert_array_equal(mb, om, err_msg=text)
        np.testing.assert_array_equal(db, od, err_msg=text)


@pytest.mark.parametrize("hint", [(1, 64, 0, 2), (4, 128, 0, 1), (8, 256, 0, 1), (2, 128, 1, 1), (1, 96, 0, 4)])
def test_feedforward_tile_shapes(hint):
    rng = np.random.default_rng(2106)
    text = _wide_circuit(rng, 30, 120, feedforward=True) + _feedforward_loop_circuit(rng, 6, 9)
    mb, db = gpu_sample(text, 1000, 5, hint=hint)
    om, od = oracle.Circuit(text).sample(np.arange(1000), 5, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


def test_feedforward_detectors_only_and_detection_lists():
    """Detection events alone (no measurement output buffer) still see the
    classically controlled ops: the records are kept in scratch."""
    rng = np.random.default_rng(2107)
    text = _feedforward_loop_circuit(rng, 7, 25)
    shots = 777
    c = sg.Circuit(text)
    _, d = c.sample(shots, 11, meas=False)
    torch.cuda.synchronize()
    db = words_to_bits(to_np(d), shots).T
    _, dh = c.sample_host(shots, 11, meas=False, shot_major=True)
    begin, dets = c.sample_detections(shots, 11)
    c.close()
    _, od = oracle.Circuit(text).sample(np.arange(shots), 11, threads=8)
    np.testing.assert_array_equal(db, od)
    np.testing.assert_array_equal(words_to_bits(dh, od.shape[1]), od)
    lists = [list(np.flatnonzero(row)) for row in od]
    got = [list(dets[begin[s]:begin[s + 1]]) for s in range(shots)]
    assert got == lists


def test_teleportation_is_deterministic_on_the_gpu():
    txt = "H 0\nS 0\nH 1\nCX 1 2\nCX 0 1\nH 0\nM 0 1\nCX rec[-1] 2\nCZ rec[-2] 2\nMY 2\n"
    mb, _ = gpu_sample(txt, 5000, 9)
    assert np.all(mb[:, 2] == 0)
    assert 0.45 < mb[:, 0].mean() < 0.55 and 0.45 < mb[:, 1].mean() < 0.55


OBS_TEXTS = [
    W.surface_code_memory(5, 5, 0.01, observable=True),
    ("H 0 1\nM 0 1\nOBSERVABLE_INCLUDE(2) rec[-1]\nOBSERVABLE_INCLUDE(2) rec[-2]\n"
     "REPEAT 7 {\nH 2\nX_ERROR(0.1) 2\nM 2\nOBSERVABLE_INCLUDE(1) rec[-1]\nDETECTOR rec[-1]\n}\n"
     "CX rec[-1] 3\nM 3\nOBSERVABLE_INCLUDE(0) rec[-1]\n"),
]


@pytest.mark.parametrize("idx", range(len(OBS_TEXTS)))
def test_observables_match_oracle(idx):
    """Logical observables follow the detectors as rows D..D+K-1 of every
    detection-event output: dense device, shot-major host and per-shot lists."""
    text = OBS_TEXTS[idx]
    shots = 1111
    c = sg.Circuit(text)
    assert c.num_observables >= 1
    m, d = c.sample(shots, 21)
    torch.cuda.synchronize()
    R = c.num_detector_rows
    db = words_to_bits(to_np(d), shots).T
    _, dh = c.sample_host(shots, 21, meas=False, shot_major=True)
    begin, dets = c.sample_detections(shots, 21)
    c.close()
    _, od = oracle.Circuit(text).sample(np.arange(shots), 21, threads=8)
    assert od.shape[1] == R
    np.testing.assert_array_equal(db, od)
    np.testing.assert_array_equal(words_to_bits(dh, R), od)
    got = [list(dets[begin[s]:begin[s + 1]]) for s in range(shots)]
    assert got == [list(np.flatnonzero(row)) for row in od]


def _dyadic_probs(rng, m, total):
    """m probabilities k_i / 2^j * total with integer k_i summing to 2^j (so
    the sum is exactly `total`, a power of two), about half of them zero."""
    den = 16 if m == 3 else 32
    k = rng.integers(0, 4, m) * (rng.random(m) < 0.6)
    k[int(rng.integers(m))] += den - int(k.sum()) if k.sum() < den else 0
    while k.sum() > den:
        k[int(np.argmax(k))] -= 1
    return [float(v) / den * total for v in k]


def _channel_circuit(rng, n, L):
    """Random Clifford layers mixed with PAULI_CHANNEL_1/2 (random, sparse and
    probability-one distributions) and the depolarizing channels."""
    lines = ["H " + " ".join(map(str, range(n)))]
    for _ in range(L):
        kind = rng.random()
        if kind < 0.3:
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"{str(rng.choice(['CX', 'CZ']))} {a} {b}")
        elif kind < 0.45:
            lines.append(f"{str(rng.choice(WIDE_1Q))} {int(rng.integers(n))}")
        elif kind < 0.65:
            q = _dyadic_probs(rng, 3, float(rng.choice([0.0625, 0.5, 1.0])))
            tg = " ".join(map(str, rng.choice(n, int(rng.integers(1, n + 1)), replace=False)))
            lines.append("PAULI_CHANNEL_1(" + ", ".join(repr(float(v)) for v in q) + f") {tg}")
        elif kind < 0.8:
            q = _dyadic_probs(rng, 15, float(rng.choice([0.03125, 0.5, 1.0])))
            if rng.random() < 0.3:
                q = [v * 0.3 for v in q]     # a total that is not a power of two
            a, b = rng.choice(n, 2, replace=False)
            lines.append("PAULI_CHANNEL_2(" + ", ".join(repr(float(v)) for v in q) + f") {a} {b}")
        elif kind < 0.9:
            p = float(rng.choice([0.01, 0.3]))
            a, b = rng.choice(n, 2, replace=False)
            lines.append(f"DEPOLARIZE2({p}) {a} {b}" if rng.random() < 0.5 else f"DEPOLARIZE1({p}) {a}")
        else:
            k = int(rng.integers(1, n + 1))
            lines.append("MR " + " ".join(map(str, rng.choice(n, k, replace=False))))
            lines.append("DETECTOR rec[-1]")
    lines.append(str(rng.choice(["M", "MX", "MY"])) + " " + " ".join(map(str, range(n))))
    return "\n".join(lines) + "\n"


def test_pauli_channels_match_oracle():
    rng = np.random.default_rng(2300)
    for it in range(20):
        n = int(rng.integers(2, 30))
        text = _channel_circuit(rng, n, int(rng.integers(5, 60)))
        shots = int(rng.integers(1, 900))
        mb, db = gpu_sample(text, shots, 500 + it)
        om, od = oracle.Circuit(text).sample(np.arange(shots), 500 + it, threads=8)
        np.testing.assert_array_equal(mb, om, err_msg=text)
        np.testing.assert_array_equal(db, od, err_msg=text)


@pytest.mark.parametrize("hint", [(1, 64, 0, 2), (4, 128, 0, 1), (8, 256, 0, 1), (2, 128, 1, 1)])
def test_pauli_channels_tile_shapes(hint):
    rng = np.random.default_rng(2301)
    text = _channel_circuit(rng, 24, 150)
    mb, db = gpu_sample(text, 1000, 6, hint=hint)
    om, od = oracle.Circuit(text).sample(np.arange(1000), 6, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(db, od)


@pytest.mark.parametrize("hint", [(1, 64, 0, 2), (2, 64, 0, 2), (4, 128, 0, 4), (1, 64, 0, 8), (8, 256, 0, 2)])
def test_cluster_deferred_hits_on_one_remote_word(hint):
    """A chain owned by one CTA of a cluster ends in several likely noise ops on
    a qubit of another CTA: their deferred hits reach the same remote word in
    one flush and must all land (XOR-merged per address within the warp)."""
    text = ("H 0 1 2 3\nCZ 2 0\nCZ 1 3\nX_ERROR(0.5) 0\nX_ERROR(0.5) 0\nY_ERROR(0.5) 0\n"
            "DEPOLARIZE1(0.5) 0\nCX 0 1\nM 0 1 2 3\n") * 3
    mb, _ = gpu_sample(text, 3000, 17, hint=hint)
    om, _ = oracle.Circuit(text).sample(np.arange(3000), 17, threads=8)
    np.testing.assert_array_equal(mb, om)


def test_reference_many_matches_oracle_and_one_by_one():
    """stim_reference_many (small circuits side by side, the others one at a
    time) gives the references the oracle gives, and the ones the
    one-at-a-time path gives."""
    rng = np.random.default_rng(2400)
    texts = [W.random_clifford(int(n), int(dp), int(sd)) for n, dp, sd in
             zip(rng.integers(20, 300, 10), rng.integers(10, 80, 10), rng.integers(0, 1000, 10))]
    texts += [W.surface_code_memory(d, 3, 0.001) for d in (3, 5, 9)]
    texts += [_wide_circuit(rng, 12, 40), _wide_circuit(rng, 25, 50, feedforward=True)]
    texts.append(texts[0])
    cs = [sg.Circuit(t) for t in texts]
    sg.stim_reference_many([c.handle for c in cs] + [cs[1].handle])      # a repeated handle is fine
    got = []
    for c in cs:
        r, d = c.reference()            # the cached sample
        torch.cuda.synchronize()
        got.append((words_to_bits(to_np(r)[None, :], c.num_measurements)[0],
                    words_to_bits(to_np(d)[None, :], c.num_measurements)[0]))
    for t, (r, d) in zip(texts, got):
        orf, odf = oracle.Circuit(t).reference()
        np.testing.assert_array_equal(r, orf, err_msg=t[:200])
        np.testing.assert_array_equal(d, odf, err_msg=t[:200])
    # recompute one by one (library's block count) and compare, plus a large circuit
    big = sg.Circuit(W.surface_code_memory(47, 2, 0.001))     # 4417 qubits
    sg.stim_reference_many([big.handle, cs[2].handle], sg.STIM_RECOMPUTE)
    rb, db = big.reference()
    rb2, db2 = big.reference(recompute=True)
    torch.cuda.synchronize()
    assert torch.equal(rb, rb2) and torch.equal(db, db2)
    for c in cs + [big]:
        c.close()


def test_reference_cache_reuses_equal_skeletons():
    """A circuit that differs from an earlier one only in noise, detectors and
    observables takes the cached reference sample; it equals a recomputed one
    and the oracle's, and STIM_RECOMPUTE bypasses the cache."""
    sg.stim_reference_cache_set(256 << 20)
    a = sg.Circuit(W.surface_code_memory(9, 6, 0.001))
    a.reference()
    torch.cuda.synchronize()
    before = sg.stim_reference_cache_stats()
    text_b = W.surface_code_memory(9, 6, 0.02, observable=True)
    b = sg.Circuit(text_b)
    assert b.info["reference_key"] == a.info["reference_key"]
    rb, db = b.reference()
    torch.cuda.synchronize()
    after = sg.stim_reference_cache_stats()
    assert after["hits"] == before["hits"] + 1
    rb2, db2 = b.reference(recompute=True)
    torch.cuda.synchronize()
    assert sg.stim_reference_cache_stats()["hits"] == after["hits"]
    assert torch.equal(rb, rb2) and torch.equal(db, db2)
    orf, odf = oracle.Circuit(text_b).reference()
    np.testing.assert_array_equal(words_to_bits(to_np(rb)[None, :], b.num_measurements)[0], orf)
    # sampling with the cached reference matches the oracle
    mb, dbits = gpu_sample(text_b, 700, 31)
    om, od = oracle.Circuit(text_b).sample(np.arange(700), 31, threads=8)
    np.testing.assert_array_equal(mb, om)
    np.testing.assert_array_equal(dbits, od)
    # with the cache off nothing is looked up
    sg.stim_reference_cache_set(0)
    c = sg.Circuit(W.surface_code_memory(9, 6, 0.005))
    c.reference()
    torch.cuda.synchronize()
    assert sg.stim_reference_cache_stats()["entries"] == 0
    sg.stim_reference_cache_set(256 << 20)
    for h in (a, b, c):
        h.close()


def test_reference_many_batched_launch_with_scaled_ctas():
    """Mid-size circuits whose tableaus together want more CTAs than can be
    co-resident share batched cooperative launches with scaled-down CTA
    counts; their references equal the one-at-a-time ones."""
    rng = np.random.default_rng(2500)
    texts = [W.random_clifford(int(n), 30, int(sd)) for n, sd in
             zip(rng.integers(900, 1600, 14), rng.integers(0, 1000, 14))]
    texts += [W.surface_code_memory(21, 4, 0.001), W.random_clifford(300, 60, 9)]
    cs = [sg.Circuit(t) for t in texts]
    sg.stim_reference_many([c.handle for c in cs], sg.STIM_RECOMPUTE)
    batched = []
    for c in cs:
        r, d = c.reference()
        batched.append((r.clone(), d.clone()))
    for c, (r, d) in zip(cs, batched):
        r2, d2 = c.reference(recompute=True)
        torch.cuda.synchronize()
        assert torch.equal(r, r2) and torch.equal(d, d2)
    for c in cs:
        c.close()


def test_reference_cache_budget_evicts_least_recent():
    """The cache keeps within its byte budget by dropping the least recently
    used samples; dropped skeletons are computed again (a miss)."""
    sg.stim_reference_cache_set(0)                 # empty
    texts = [W.surface_code_memory(d, 4, 0.001) for d in (5, 7, 9)]
    cs = [sg.Circuit(t) for t in texts]
    sg.stim_reference_cache_set(256 << 20)
    for c in cs:
        c.reference()
    torch.cuda.synchronize()
    st = sg.stim_reference_cache_stats()
    assert st["entries"] == 3
    # one byte less than held: exactly the least recently used entry (d=5) goes
    sg.stim_reference_cache_set(st["bytes"] - 1)
    st2 = sg.stim_reference_cache_stats()
    assert st2["entries"] == 2 and st2["bytes"] < st["bytes"]
    # a new handle of the evicted skeleton misses; one of a kept skeleton hits
    before = sg.stim_reference_cache_stats()
    again = sg.Circuit(W.surface_code_memory(5, 4, 0.02))
    again.reference()
    torch.cuda.synchronize()
    mid = sg.stim_reference_cache_stats()
    assert mid["misses"] == before["misses"] + 1 and mid["hits"] == before["hits"]
    kept = sg.Circuit(W.surface_code_memory(9, 4, 0.02))
    kept.reference()
    torch.cuda.synchronize()
    assert sg.stim_reference_cache_stats()["hits"] == mid["hits"] + 1
    sg.stim_reference_cache_set(256 << 20)
    for c in cs + [again, kept]:
        c.close()


def test_paper_teleportation_example_on_the_gpu():
    """The paper's teleportation example (golden fixture): the final bit is
    False in every GPU shot and the records equal the oracle's."""
    import os
    gold = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "teleportation.txt")):
        if line.strip() and line[0] != "#":
            k, v = line.rstrip("\n").split(" ", 1)
            gold[k] = v
    txt = gold["circuit"].replace(";", "\n") + "\n"
    mb, _ = gpu_sample(txt, 10000, 12)
    assert np.all(mb[:, -1] == int(gold["final_measurement"]))
    om, _ = oracle.Circuit(txt).sample(np.arange(10000), 12, threads=8)
    np.testing.assert_array_equal(mb, om)


def test_failed_device_allocations_leave_handles_usable():
    """Fault injection: each device allocation of compile-upload, reference
    and sampling fails in turn (STIM_E_OOM); the same handle then samples
    bit-exactly once injection is off."""
    text = W.surface_code_memory(5, 4, 0.01)
    om, od = oracle.Circuit(text).sample(np.arange(300), 4, threads=8)
    sg.stim_reference_cache_set(0)             # every reference runs the tableau (its scratch is allocated)
    failed_sites = 0
    try:
        for skip in range(14):
            c = sg.Circuit(text)
            sg.stim_debug_fail_allocations(skip, 1)
            try:
                c.sample_host(300, 4, shot_major=False)
            except sg.StimError as e:
                assert e.code == sg.STIM_E_OOM, (skip, e)
                failed_sites += 1
            sg.stim_debug_fail_allocations(0, 0)
            m, d = c.sample_host(300, 4, shot_major=False)
            mb = words_to_bits(m, 300).T
            db = words_to_bits(d, 300).T
            np.testing.assert_array_equal(mb, om, err_msg=f"skip={skip}")
            np.testing.assert_array_equal(db, od, err_msg=f"skip={skip}")
            c.close()
    finally:
        sg.stim_debug_fail_allocations(0, 0)
        sg.stim_reference_cache_set(256 << 20)
    assert failed_sites >= 8


@pytest.mark.parametrize("d", [3, 8, 20, 30])
def test_bacon_shor_reference_matches_oracle(d):
    """Bacon-Shor memory (a random-measurement workload for the tableau):
    reference sample and deterministic flags equal the oracle's, and sampled
    detection events equal the oracle's on a few hundred shots."""
    text = W.bacon_shor(d, d, 1e-3, observable=True)
    ref, det = gpu_reference(text)
    o = oracle.Circuit(text)
    oref, odet = o.reference()
    np.testing.assert_array_equal(ref, oref)
    np.testing.assert_array_equal(det, odet)
    c = sg.Circuit(text)
    _, d_ev = c.sample(300, 17, meas=False)
    torch.cuda.synchronize()
    gd = words_to_bits(to_np(d_ev), 300).T
    _, od = o.sample(np.arange(300), 17, threads=8, ref=oref)
    np.testing.assert_array_equal(gd, od)
    c.close()

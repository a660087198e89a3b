"""Bit-exact parity at the benchmark configurations' own scale.

- The 64-circuit heterogeneous batch (row a9), exactly as the benchmark
  builds it (same generator seed, shots and per-circuit seeds): every
  circuit's reference sample equals the oracle's tableau, and every circuit's
  batched output equals the oracle on its first and last shots, the shots
  around the first word boundary, the last (partial) word and 64 random
  shots.
- A seeded 300-request slice of the serving stream (row a10) through the
  server: every request's reference sample (per circuit) and 8 of its shots
  (first, last, 6 random) equal the oracle.

The oracle runs in a spawn process pool, one item per circuit."""
import numpy as np
import pytest

import oracle_jobs
import paper_2103_02202_gb300 as sg
from paper_2103_02202_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_02202_gb300 import build
    build.build()
    yield


def _bits(t, nbits):
    w = np.ascontiguousarray(t.cpu().numpy().view(np.uint64))
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:nbits]


def _gather(rows, picks):
    """(R, words) int64 device tensor -> (len(picks), R) uint8 bits of the given shots."""
    cols = torch.as_tensor(np.asarray(picks) // 64, device="cuda")
    bits = torch.as_tensor(np.asarray(picks) % 64, device="cuda")
    return ((rows[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T


def _picks(rng, S, k):
    base = [0, S - 1, min(63, S - 1), min(64, S - 1), S - 1 - (S - 1) % 64]
    rnd = rng.choice(S, min(k, S), replace=False) if S > 0 else []
    return np.unique(np.concatenate([base, rnd])).astype(np.int64)


def test_c3_batch_bit_exact_against_oracle():
    spec = W.batch_circuits()
    rng = np.random.default_rng(31)
    picks = [_picks(rng, e["shots"], 64) for e in spec]
    items = [(e["text"], [(e["seed"], 0, p)]) for e, p in zip(spec, picks)]
    want = oracle_jobs.run_pool(items)

    cs = [sg.Circuit(e["text"]) for e in spec]
    sg.stim_reference_many([c.handle for c in cs])
    shots = [e["shots"] for e in spec]
    b = sg.Batch(cs, shots)
    outs = []
    for c, S in zip(cs, shots):
        w = (S + 63) // 64
        if c.num_detector_rows:
            outs.append((None, torch.empty((c.num_detector_rows, w), dtype=torch.int64, device="cuda")))
        else:
            outs.append((torch.empty((c.num_measurements, w), dtype=torch.int64, device="cuda"), None))
    b.sample([e["seed"] for e in spec], out=outs)
    torch.cuda.synchronize()
    for i, (c, e) in enumerate(zip(cs, spec)):
        oref, odet, [(om, od)] = want[i]
        ref, det = c.reference()
        M = c.num_measurements
        msg = "circuit %d (%s)" % (i, e["kind"])
        np.testing.assert_array_equal(_bits(ref, M), oref, err_msg=msg)
        np.testing.assert_array_equal(_bits(det, M), odet, err_msg=msg)
        m, d = outs[i]
        if d is not None:
            np.testing.assert_array_equal(_gather(d, picks[i]), od, err_msg=msg)
        else:
            np.testing.assert_array_equal(_gather(m, picks[i]), om, err_msg=msg)
        outs[i] = None
    b.close()
    for c in cs:
        c.close()


def test_c5_served_slice_bit_exact_against_oracle():
    catalogue, reqs = W.serve_requests(seed=5, count=300)
    rng = np.random.default_rng(55)
    picks = [_picks(rng, r["shots"], 6) for r in reqs]
    by_circuit = {}
    for k, r in enumerate(reqs):
        by_circuit.setdefault(r["circuit"], []).append(k)
    keys = sorted(by_circuit)
    items = [(W.catalogue_text(catalogue[ci]), [(reqs[k]["seed"], 0, picks[k]) for k in by_circuit[ci]])
             for ci in keys]
    got = oracle_jobs.run_pool(items)
    want = {}
    for ci, res in zip(keys, got):
        oref, odet, samples = res
        for k, s in zip(by_circuit[ci], samples):
            want[k] = (oref, odet, s)

    cs = {ci: sg.Circuit(W.catalogue_text(catalogue[ci])) for ci in keys}
    sg.stim_reference_many([cs[ci].handle for ci in keys])
    srv = sg.Server(150 << 30, streams=16)
    ids = [srv.submit(cs[r["circuit"]], r["shots"], r["seed"], 0) for r in reqs]
    for k, (r, rid) in enumerate(zip(reqs, ids)):
        c = cs[r["circuit"]]
        res = srv.wait(rid, 600)
        assert res.status == sg.STIM_OK
        m, d = srv.fetch(c, rid, r["shots"])
        srv.release(rid)
        oref, odet, (om, od) = want[k]
        msg = "request %d (circuit %d)" % (k, r["circuit"])
        if c.num_measurements:
            np.testing.assert_array_equal(_gather(m, picks[k]), om, err_msg=msg)
        if c.num_detector_rows:
            np.testing.assert_array_equal(_gather(d, picks[k]), od, err_msg=msg)
        del m, d
    st = srv.stats()
    assert st["failed"] == 0 and st["completed"] == len(reqs)
    srv.close()
    for ci in keys:
        ref, det = cs[ci].reference()
        M = cs[ci].num_measurements
        k0 = by_circuit[ci][0]
        np.testing.assert_array_equal(_bits(ref, M), want[k0][0])
        np.testing.assert_array_equal(_bits(det, M), want[k0][1])
        cs[ci].close()

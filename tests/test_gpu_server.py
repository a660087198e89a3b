"""Sampling server: continuous batching under an HBM budget. Each request's
result is bit-identical alone and in a busy mix, and equals the plain
entry point's result."""
import threading
import time

import numpy as np
import pytest

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


def _circuits():
    texts = [W.surface_code_memory(3, 3, 1e-3), W.surface_code_memory(5, 5, 5e-3),
             W.random_clifford(150, 30, 4), W.surface_code_memory(9, 9, 1e-3),
             W.random_clifford(400, 20, 5, p=0.005)]
    cs = [sg.Circuit(t) for t in texts]
    for c in cs:
        c.reference()
    torch.cuda.synchronize()
    return cs


def test_result_same_alone_and_in_the_mix():
    cs = _circuits()
    srv = sg.Server(512 << 20, streams=6)
    probe = (cs[1], 3000, 77, 128)
    # alone
    rid = srv.submit(*probe)
    srv.wait(rid)
    alone = srv.fetch(probe[0], rid, probe[1])
    srv.release(rid)
    # in a mix: many concurrent requests submitted from two threads
    rng = np.random.default_rng(1)
    ids = []

    def feeder(seed):
        r = np.random.default_rng(seed)
        for _ in range(40):
            c = cs[int(r.integers(len(cs)))]
            ids.append((c, srv.submit(c, int(r.integers(1, 5000)), int(r.integers(2**62)))))

    th = [threading.Thread(target=feeder, args=(s,)) for s in (2, 3)]
    for t in th:
        t.start()
    time.sleep(0.001)
    rid = srv.submit(*probe)
    for t in th:
        t.join()
    srv.wait(rid)
    mixed = srv.fetch(probe[0], rid, probe[1])
    torch.cuda.synchronize()
    assert torch.equal(alone[0], mixed[0]) and torch.equal(alone[1], mixed[1])
    # and equal to the plain entry point
    pm, pd = probe[0].sample(probe[1], probe[2], shot_offset=probe[3])
    torch.cuda.synchronize()
    assert torch.equal(pm, mixed[0]) and torch.equal(pd, mixed[1])
    srv.release(rid)
    for c, r in ids:
        res = srv.wait(r)
        assert res.status == sg.STIM_OK
        srv.release(r)
    st = srv.stats()
    assert st["completed"] == 2 + len(ids) and st["failed"] == 0
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    assert st["bytes_in_use"] == 0
    srv.close()


def test_admission_respects_the_budget():
    cs = _circuits()
    c = cs[3]                      # d=9 surface code
    shots = 20000
    need = (c.num_measurements + c.num_detectors) * ((shots + 63) // 64) * 8
    srv = sg.Server(int(need * 2.5), streams=8)   # room for two requests at a time
    ids = [srv.submit(c, shots, s) for s in range(10)]
    outs = []
    for i, r in enumerate(ids):
        res = srv.wait(r)
        assert res.status == sg.STIM_OK
        outs.append(srv.fetch(c, r, shots))
        srv.release(r)
    st = srv.stats()
    assert st["peak_bytes_in_use"] <= st["budget_bytes"]
    assert st["completed"] == 10
    for s, (m, d) in enumerate(outs):
        pm, pd = c.sample(shots, s)
        torch.cuda.synchronize()
        assert torch.equal(m, pm) and torch.equal(d, pd)
    # a request larger than the whole budget fails instead of waiting forever
    r = srv.submit(c, shots * 10, 1)
    with pytest.raises(sg.StimError):
        srv.wait(r)
    srv.close()


def test_cancel_and_wait_timeout():
    cs = _circuits()
    srv = sg.Server(64 << 20, streams=1)
    big = [srv.submit(cs[3], 60000, s) for s in range(4)]
    rc = srv.cancel(big[-1])
    assert rc in (sg.STIM_OK, sg.STIM_E_BUSY)
    for r in big[:-1]:
        srv.wait(r)
        srv.release(r)
    srv.close()


def test_feedforward_detectors_only_request():
    """A detectors-only request for a circuit with classically controlled ops
    reserves record scratch and matches the plain entry point."""
    text = ("H 0 1\nM 0 1\nREPEAT 30 {\nCX rec[-1] 2\nCZ 2 rec[-2]\nDEPOLARIZE1(0.05) 2\nMR 2\n"
            "DETECTOR rec[-1]\nH 0\nM 0\n}\n")
    c = sg.Circuit(text)
    srv = sg.Server(64 << 20, streams=2)
    rid = srv.submit(c, 1500, 42, 64, outputs=sg.STIM_OUT_DET)
    srv.wait(rid)
    d = torch.empty((c.num_detectors, (1500 + 63) // 64), dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    sg._check(sg.library().stim_server_copy_result(srv.handle, rid, None, d.data_ptr(), sg.STIM_DEVICE,
                                                   s.cuda_stream))
    _, pd = c.sample(1500, 42, shot_offset=64, meas=False)
    torch.cuda.synchronize()
    assert torch.equal(d, pd)
    srv.release(rid)
    srv.close()
    c.close()


def test_observable_rows_in_server_results():
    c = sg.Circuit(W.surface_code_memory(3, 3, 0.01, observable=True))
    srv = sg.Server(64 << 20, streams=2)
    rid = srv.submit(c, 900, 5)
    srv.wait(rid)
    m, d = srv.fetch(c, rid, 900)
    pm, pd = c.sample(900, 5)
    torch.cuda.synchronize()
    assert d.shape[0] == c.num_detectors + 1
    assert torch.equal(m, pm) and torch.equal(d, pd)
    srv.release(rid)
    srv.close()
    c.close()


def test_release_right_after_device_copy_keeps_the_copy():
    """A device copy out of a request's result buffers is asynchronous; a
    release right after it must not hand the buffers to queued requests
    before the copy has read them. With a small budget every release lets the
    next queued request reuse the same arena bytes at once."""
    cs = _circuits()
    c = cs[3]
    srv = sg.Server(3 << 20, streams=2)      # room for about two of these requests at a time
    reqs = [(5000 + 37 * k, 1000 + k) for k in range(24)]
    ids = [srv.submit(c, shots, seed) for shots, seed in reqs]
    side = torch.cuda.Stream()
    got = []
    with torch.cuda.stream(side):
        for rid, (shots, seed) in zip(ids, reqs):
            srv.wait(rid)
            got.append(srv.fetch(c, rid, shots))
            srv.release(rid)
    torch.cuda.synchronize()
    for (shots, seed), (m, d) in zip(reqs, got):
        pm, pd = c.sample(shots, seed)
        torch.cuda.synchronize()
        assert torch.equal(pm, m) and torch.equal(pd, d)
    srv.close()

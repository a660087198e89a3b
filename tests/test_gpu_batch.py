"""Batched persistent launch: every circuit of a heterogeneous batch returns
exactly what the single-circuit entry point returns for the same shots."""
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


TEXTS = [
    W.surface_code_memory(3, 3, 1e-3),
    W.surface_code_memory(5, 7, 5e-3),
    W.random_clifford(120, 40, 1),
    W.repetition_code(5, 20, 0.02),
    W.random_clifford(300, 25, 2, p=0.01),
    W.surface_code_memory(7, 3, 0.02),
]
SHOTS = [1024, 777, 4096, 65, 2000, 1]


def plain(c, shots, seed, offset=0):
    m, d = c.sample(shots, seed, shot_offset=offset)
    return m, d


@pytest.mark.parametrize("hint", [None, (1, 256, 0, 1), (2, 512, 0, 1), (4, 256, 0, 2), (1, 128, 0, 4)])
def test_batch_equals_plain(hint):
    cs = [sg.Circuit(t) for t in TEXTS]
    b = sg.Batch(cs, SHOTS, hint=hint)
    seeds = [11 * i + 3 for i in range(len(cs))]
    offs = [64 * i for i in range(len(cs))]
    out = b.sample(seeds, offs)
    torch.cuda.synchronize()
    for c, S, sd, off, (m, d) in zip(cs, SHOTS, seeds, offs, out):
        pm, pd = plain(c, S, sd, off)
        torch.cuda.synchronize()
        if m is not None:
            assert torch.equal(m, pm)
        if d is not None:
            assert torch.equal(d, pd)
    info = b.info()
    assert info["work_items"] >= len(cs)
    b.close()


def test_batch_replay_new_seeds_and_outputs():
    cs = [sg.Circuit(t) for t in TEXTS[:4]]
    b = sg.Batch(cs, SHOTS[:4])
    for rep in range(3):
        seeds = [rep * 1000 + i for i in range(4)]
        out = b.sample(seeds, dets=(rep != 1), meas=(rep != 2))
        torch.cuda.synchronize()
        for c, S, sd, (m, d) in zip(cs, SHOTS[:4], seeds, out):
            pm, pd = plain(c, S, sd)
            torch.cuda.synchronize()
            if m is not None:
                assert torch.equal(m, pm)
            if d is not None:
                assert torch.equal(d, pd)
    b.close()


def test_batch_matches_oracle_on_sampled_shots():
    text = W.surface_code_memory(5, 5, 0.01)
    c = sg.Circuit(text)
    b = sg.Batch([c, c], [3000, 3000])
    (m0, d0), (m1, d1) = b.sample([5, 5], [0, 3008])
    torch.cuda.synchronize()
    o = oracle.Circuit(text)
    pick = np.array([0, 1, 63, 64, 2999])
    for m, d, off in ((m0, d0, 0), (m1, d1, 3008)):
        cols = torch.as_tensor(pick // 64, device="cuda")
        bits = torch.as_tensor(pick % 64, device="cuda")
        gm = ((m[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T
        gd = ((d[:, cols] >> bits) & 1).cpu().numpy().astype(np.uint8).T
        om, od = o.sample(pick, 5, shot_offset=off, threads=4)
        np.testing.assert_array_equal(gm, om)
        np.testing.assert_array_equal(gd, od)
    b.close()


def test_batch_feedforward_detectors_only():
    """Circuits with classically controlled X/Z in a batch, detection events
    only: the batch keeps their records in scratch and matches the plain
    entry point and the oracle."""
    texts = ["H 0 1\nM 0 1\nCX rec[-1] 2\nCZ rec[-2] 2\nREPEAT 20 {\nH 3\nCX rec[-1] 3\n"
             "X_ERROR(0.1) 2\nMR 2 3\nDETECTOR rec[-1] rec[-2]\nCZ 2 rec[-2]\nH 2\n}\nM 2\nDETECTOR rec[-1]\n",
             W.surface_code_memory(3, 3, 1e-3)]
    shots = [900, 300]
    cs = [sg.Circuit(t) for t in texts]
    b = sg.Batch(cs, shots)
    out = b.sample([7, 8], meas=False)
    torch.cuda.synchronize()
    for c, t, S, sd, (m, d) in zip(cs, texts, shots, [7, 8], out):
        assert m is None
        _, pd = c.sample(S, sd, meas=False)
        torch.cuda.synchronize()
        assert torch.equal(d, pd)
    o = oracle.Circuit(texts[0])
    _, od = o.sample(np.arange(shots[0]), 7, threads=4)
    dd = out[0][1].cpu().numpy().view(np.uint64)
    got = np.unpackbits(dd.view(np.uint8).reshape(dd.shape[0], -1), axis=1, bitorder="little")[:, :shots[0]].T
    np.testing.assert_array_equal(got, od)
    b.close()


def test_batch_with_observables_equals_plain():
    texts = [W.surface_code_memory(3, 4, 0.01, observable=True),
             "M 0\nOBSERVABLE_INCLUDE(1) rec[-1]\nX_ERROR(0.3) 1\nM 1\nOBSERVABLE_INCLUDE(0) rec[-1]\n"]
    shots = [700, 1300]
    cs = [sg.Circuit(t) for t in texts]
    b = sg.Batch(cs, shots)
    out = b.sample([1, 2])
    torch.cuda.synchronize()
    for c, S, sd, (m, d) in zip(cs, shots, [1, 2], out):
        assert d.shape[0] == c.num_detector_rows
        pm, pd = c.sample(S, sd)
        torch.cuda.synchronize()
        assert torch.equal(m, pm) and torch.equal(d, pd)
    b.close()

"""Detection events computed inside the frame kernel (paper Section 5.6):
when only detection events are asked for with STIM_EVENTS_IN_KERNEL, the
frame kernel keeps each measurement's flip in a ring of recent measurements and evaluates
the DETECTOR / OBSERVABLE_INCLUDE lines of each straight-line stretch between
its layers, so no measurement record is written and the detector kernel does
not run. The events must equal those of the record path (asked for together
with the records) and the oracle, bit for bit."""
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


def _both(text, shots, seed, offset=0, hint=None):
    """(events alone, events with records, detector-kernel launches of the
    events-alone call)."""
    c = sg.Circuit(text)
    c.reference()
    torch.cuda.synchronize()
    sg.stim_profile(True)
    _, alone = c.sample(shots, seed, shot_offset=offset, meas=False, hint=hint, events_in_kernel=True)
    torch.cuda.synchronize()
    prof = sg.stim_profile_read()
    sg.stim_profile(False)
    _, with_rec = c.sample(shots, seed, shot_offset=offset, hint=hint)
    torch.cuda.synchronize()
    c.close()
    return alone, with_rec, prof["detectors"][0]


# The ring holds the last ~3 rounds of measurements (a power of two), so it is
# used once a memory runs long enough to have at least four times as many
# measurements: rounds = 3d + 10 here.
@pytest.mark.parametrize("d,shots", [(3, 1000), (5, 4096), (9, 777), (15, 20000)])
def test_surface_events_in_kernel_equal_record_path(d, shots):
    text = W.surface_code_memory(d, 3 * d + 10, 0.01, observable=True)
    alone, with_rec, det_launches = _both(text, shots, 7, 64)
    assert det_launches == 0, "events were expected from the frame kernel"
    assert torch.equal(alone, with_rec)


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_events_in_kernel_with_clusters(cluster):
    text = W.surface_code_memory(7, 31, 0.02, observable=True)
    alone, with_rec, det_launches = _both(text, 3000, 11, 0, hint=(1, 256, 0, cluster))
    assert det_launches == 0
    assert torch.equal(alone, with_rec)


def test_events_in_kernel_wide_tiles():
    """Eight-word tiles (a single CTA per tile) evaluate detectors too."""
    text = W.surface_code_memory(5, 25, 0.02)
    alone, with_rec, det_launches = _both(text, 9000, 3, 0, hint=(8, 512, 0, 1))
    assert det_launches == 0
    assert torch.equal(alone, with_rec)


def test_events_in_kernel_match_oracle():
    text = W.surface_code_memory(5, 25, 0.03, observable=True)
    S = 2000
    c = sg.Circuit(text)
    _, d = c.sample(S, 21, shot_offset=128, meas=False, events_in_kernel=True)
    torch.cuda.synchronize()
    bits = np.unpackbits(d.cpu().numpy().view(np.uint64).view(np.uint8).reshape(d.shape[0], -1), axis=1,
                         bitorder="little")[:, :S].T
    _, od = oracle.Circuit(text).sample(np.arange(S), 21, shot_offset=128, threads=8)
    np.testing.assert_array_equal(bits, od)
    c.close()


LOOPY = [
    # detectors reaching into earlier loop iterations, nested loops, and a
    # stretch of detectors alone after a loop (two DETS entries in a row)
    "R 0 1 2\nM 1 2\nREPEAT 400 {\nX_ERROR(0.2) 0 1 2\nCX 0 1 1 2\nMR 1 2\nDETECTOR rec[-1] rec[-3]\n}\n"
    "DETECTOR rec[-2]\nDETECTOR rec[-1] rec[-4]\nOBSERVABLE_INCLUDE(0) rec[-1]\n",
    "REPEAT 100 {\nH 0\nREPEAT 4 {\nDEPOLARIZE1(0.1) 0 1\nCX 0 1\nM 1\nDETECTOR rec[-1]\n}\n"
    "MR 0\nDETECTOR rec[-1] rec[-5]\n}\nM 0 1\nDETECTOR rec[-1] rec[-2]\nOBSERVABLE_INCLUDE(2) rec[-2]\n",
    W.repetition_code(5, 30, 0.05) + "M " + " ".join(map(str, range(0, 11, 2))) + "\n"
    "DETECTOR rec[-1] rec[-2]\nOBSERVABLE_INCLUDE(0) rec[-1]\n",
]


@pytest.mark.parametrize("k", range(len(LOOPY)))
def test_events_in_kernel_loops_and_observables(k):
    text = LOOPY[k]
    for shots in (64, 1000, 4097):
        alone, with_rec, det_launches = _both(text, shots, 5 + k, 0)
        assert det_launches == 0
        assert torch.equal(alone, with_rec), (k, shots)
    S = 700
    c = sg.Circuit(text)
    _, d = c.sample(S, 9, meas=False, events_in_kernel=True)
    torch.cuda.synchronize()
    bits = np.unpackbits(d.cpu().numpy().view(np.uint64).view(np.uint8).reshape(d.shape[0], -1), axis=1,
                         bitorder="little")[:, :S].T
    _, od = oracle.Circuit(text).sample(np.arange(S), 9, threads=8)
    np.testing.assert_array_equal(bits, od)
    c.close()


def test_flat_circuit_keeps_record_path():
    """Detectors listed after a long flat circuit look back over all of it: a
    ring would be as large as the records, so the record path is kept (and
    gives the same events)."""
    rng = np.random.default_rng(4)
    lines = []
    for _ in range(60):
        q = rng.choice(30, 30, replace=False)
        lines.append("CX " + " ".join(map(str, q)))
        lines.append("DEPOLARIZE1(0.01) " + " ".join(map(str, range(30))))
        lines.append("MR " + " ".join(map(str, range(0, 30, 3))))
    lines.append("DETECTOR rec[-1] rec[-600]")
    text = "\n".join(lines) + "\n"
    alone, with_rec, det_launches = _both(text, 5000, 2, 0)
    assert det_launches == 1
    assert torch.equal(alone, with_rec)

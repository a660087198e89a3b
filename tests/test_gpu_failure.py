"""Failure detection on the GPU without a GPU fault: the inverse-tableau
kernel's grid barrier waits are bounded. A test knob makes every barrier wait
for one arrival that never comes, with a 50 ms limit; the kernel must give up,
the call must return STIM_E_TIMEOUT, and the same handle must then produce
the oracle's reference sample once the knob is off."""
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
    sg.stim_debug_tableau_barrier(0, 0)


def _bits(t, nbits):
    w = np.ascontiguousarray(t.cpu().numpy().view(np.uint64))
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:nbits]


def test_tableau_barrier_timeout_returns_error_and_handle_recovers():
    # n = 700: 2n columns x 11 words -> about 15 CTAs, so the grid barrier is used
    text = W.random_clifford(700, 30, 8)
    c = sg.Circuit(text)
    sg.stim_debug_tableau_barrier(1, 50_000_000)
    try:
        with pytest.raises(sg.StimError) as ei:
            c.reference(recompute=True)
        assert ei.value.code == sg.STIM_E_TIMEOUT
        assert "timed out" in sg.stim_last_error()
    finally:
        sg.stim_debug_tableau_barrier(0, 0)
    ref, det = c.reference(recompute=True)
    torch.cuda.synchronize()
    oref, odet = oracle.Circuit(text).reference()
    M = c.num_measurements
    np.testing.assert_array_equal(_bits(ref, M), oref)
    np.testing.assert_array_equal(_bits(det, M), odet)
    c.close()


def test_batched_tableau_barrier_timeout_returns_error():
    texts = [W.random_clifford(600, 20, 11), W.random_clifford(650, 20, 12)]
    cs = [sg.Circuit(t) for t in texts]
    sg.stim_debug_tableau_barrier(1, 50_000_000)
    try:
        with pytest.raises(sg.StimError) as ei:
            sg.stim_reference_many([c.handle for c in cs], sg.STIM_RECOMPUTE)
        assert ei.value.code == sg.STIM_E_TIMEOUT
    finally:
        sg.stim_debug_tableau_barrier(0, 0)
    sg.stim_reference_many([c.handle for c in cs], sg.STIM_RECOMPUTE)
    for c, t in zip(cs, texts):
        ref, _ = c.reference()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_bits(ref, c.num_measurements), oracle.Circuit(t).reference()[0])
        c.close()


def test_smem_bandwidth_probe_is_plausible():
    """The shared-memory bandwidth probe (the frame kernel's roofline
    denominator) returns positive figures of the right order: between 1 and
    200 TB/s for local shared memory, and a cluster figure no larger than
    twice the local one."""
    lo, cl = sg.stim_probe_smem_bandwidth()
    assert 1e3 < lo < 2e5
    assert 0 < cl < 2 * lo

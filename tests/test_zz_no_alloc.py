"""stim_frame_sample_noalloc: detection events without device allocation.

Callers that cannot allocate device memory while sampling (all memory owned
by another allocator, or no tolerance for the synchronization that freeing
memory implies) use this entry point; its records live in a fixed array
inside the library. It must return exactly the detection events of
stim_frame_sample_ex for the same shots -- checked here on two calls in a
row, through the C ABI. This file is named to be collected last.
"""
import ctypes

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


def test_noalloc_matches_allocating_entry_point_twice():
    text = W.surface_code_memory(5, 5, 0.01)
    c = sg.Circuit(text)
    lib = sg.library()
    D = c.num_detectors
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.zeros(max((c.num_measurements + 63) // 64, 1), dtype=torch.int64, device="cuda")
    rc = lib.stim_reference_sample(c.handle, ref.data_ptr(), None, 0, stream)
    assert rc == sg.STIM_OK, sg.stim_last_error()
    calls = [(3000, 17, 0), (1000, 17, 3008)]     # ragged shot counts, second call offset
    outs = []
    for shots, seed, off in calls:
        nw = (shots + 63) // 64
        want = torch.full((D, nw), -1, dtype=torch.int64, device="cuda")
        got = torch.full((D, nw), -1, dtype=torch.int64, device="cuda")
        outs.append((want, got))
    torch.cuda.synchronize()
    free = []
    for (shots, seed, off), (want, got) in zip(calls, outs):
        rc = lib.stim_frame_sample_ex(c.handle, shots, seed, off, None, want.data_ptr(), sg.STIM_DEVICE,
                                      None, stream)
        assert rc == sg.STIM_OK, sg.stim_last_error()
        rc = lib.stim_frame_sample_noalloc(c.handle, shots, seed, off, got.data_ptr(), stream)
        assert rc == sg.STIM_OK, sg.stim_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert torch.equal(want, got)
    # the second call took no device memory (the fixed array was already in place)
    assert free[0] == free[1]
    # the two calls saw different shots
    assert not torch.equal(outs[0][1][:, :15], outs[1][1][:, :15])
    c.close()


def test_noalloc_rejects_oversize_and_missing_setup():
    lib = sg.library()
    c = sg.Circuit(W.surface_code_memory(3, 3, 0.01))
    out = torch.zeros(64, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # no reference sample on this handle yet
    assert lib.stim_frame_sample_noalloc(c.handle, 64, 1, 0, out.data_ptr(), stream) == sg.STIM_E_INVALID_ARG
    c.reference()
    torch.cuda.synchronize()
    # M = 33 measurements: 33 * ceil(S/64) * 8 bytes > 32 MiB for S = 2^23 shots
    rc = lib.stim_frame_sample_noalloc(c.handle, 1 << 23, 1, 0, out.data_ptr(), stream)
    assert rc == sg.STIM_E_UNSUPPORTED
    assert "32 MiB" in sg.stim_last_error()
    c.close()


def test_noalloc_with_classically_controlled_ops():
    text = ("H 0 1\nM 0 1\nREPEAT 12 {\nCX rec[-1] 2\nCZ 2 rec[-2]\nX_ERROR(0.05) 2\nMR 2\n"
            "DETECTOR rec[-1]\nH 0\nM 0\n}\n")
    c = sg.Circuit(text)
    lib = sg.library()
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.zeros(max((c.num_measurements + 63) // 64, 1), dtype=torch.int64, device="cuda")
    assert lib.stim_reference_sample(c.handle, ref.data_ptr(), None, 0, stream) == sg.STIM_OK
    shots = 2000
    nw = (shots + 63) // 64
    got = torch.full((c.num_detectors, nw), -1, dtype=torch.int64, device="cuda")
    rc = lib.stim_frame_sample_noalloc(c.handle, shots, 3, 0, got.data_ptr(), stream)
    assert rc == sg.STIM_OK, sg.stim_last_error()
    _, want = c.sample(shots, 3, meas=False)
    torch.cuda.synchronize()
    assert torch.equal(want, got)
    c.close()


@pytest.mark.parametrize("shots", [40000, 80000, 160000])
def test_noalloc_wide_tiles_match(shots):
    """Shot counts large enough that the no-allocation call picks tiles of 2,
    4 and 8 words per CTA (on a 152-SM GB300: at least 2 x 152 x W words);
    the results still equal the allocating entry point's bit for bit."""
    c = sg.Circuit(W.surface_code_memory(3, 3, 0.01))
    lib = sg.library()
    stream = torch.cuda.current_stream().cuda_stream
    c.reference()
    nw = (shots + 63) // 64
    want = torch.full((c.num_detectors, nw), -1, dtype=torch.int64, device="cuda")
    got = torch.full((c.num_detectors, nw), -1, dtype=torch.int64, device="cuda")
    rc = lib.stim_frame_sample_ex(c.handle, shots, 5, 128, None, want.data_ptr(), sg.STIM_DEVICE, None, stream)
    assert rc == sg.STIM_OK, sg.stim_last_error()
    rc = lib.stim_frame_sample_noalloc(c.handle, shots, 5, 128, got.data_ptr(), stream)
    assert rc == sg.STIM_OK, sg.stim_last_error()
    torch.cuda.synchronize()
    assert torch.equal(want, got)
    c.close()


def test_noalloc_runs_with_every_library_allocation_failing():
    """With the library's device-allocation fault injector failing every
    allocation, the no-allocation call still succeeds and returns the same
    bits as the allocating entry point (which ran before the injector was
    armed): no library allocation is on its path."""
    c = sg.Circuit(W.surface_code_memory(5, 5, 0.02))
    lib = sg.library()
    stream = torch.cuda.current_stream().cuda_stream
    c.reference()
    shots = 5000
    nw = (shots + 63) // 64
    want = torch.full((c.num_detectors, nw), -1, dtype=torch.int64, device="cuda")
    got = torch.full((c.num_detectors, nw), -1, dtype=torch.int64, device="cuda")
    rc = lib.stim_frame_sample_ex(c.handle, shots, 9, 0, None, want.data_ptr(), sg.STIM_DEVICE, None, stream)
    assert rc == sg.STIM_OK, sg.stim_last_error()
    torch.cuda.synchronize()
    assert lib.stim_debug_fail_allocations(0, 1 << 30) == sg.STIM_OK
    try:
        for _ in range(2):
            got.fill_(-1)
            rc = lib.stim_frame_sample_noalloc(c.handle, shots, 9, 0, got.data_ptr(), stream)
            assert rc == sg.STIM_OK, sg.stim_last_error()
            torch.cuda.synchronize()
            assert torch.equal(want, got)
    finally:
        assert lib.stim_debug_fail_allocations(0, 0) == sg.STIM_OK
    c.close()

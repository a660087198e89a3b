"""Oracle work items for the config-scale parity tests, run in a process pool
started with the spawn method (so that no worker is forked from a process
that already holds a CUDA context). Each item parses one circuit, takes the
oracle's tableau reference sample once and samples the listed shots of
several (seed, shot offset) requests. Imports nothing from the CUDA library."""
import numpy as np

import oracle


def reference_and_shots(text, requests):
    """requests: list of (seed, shot_offset, picks). Returns (ref, detflag,
    [(meas, dets) per request]) with the oracle's uint8 bit arrays."""
    c = oracle.Circuit(text)
    ref, det = c.reference()
    out = []
    for seed, off, picks in requests:
        out.append(c.sample(np.asarray(picks, np.uint64), seed, shot_offset=off, ref=ref))
    return ref, det, out


def run_pool(items):
    """items: list of (text, requests); returns the results in order."""
    import multiprocessing as mp
    import os
    oracle.lib()          # build the oracle once before the workers load it
    procs = max(1, min(len(items), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        # largest circuits first so the longest items start early
        order = sorted(range(len(items)), key=lambda i: -len(items[i][0]))
        res = pool.starmap(reference_and_shots, [items[i] for i in order], chunksize=1)
    out = [None] * len(items)
    for i, r in zip(order, res):
        out[i] = r
    return out

"""The Bacon-Shor memory generator (the subsystem code of the paper's
time-to-first-sample benchmarks, Section 6), checked on the oracle: without
noise no detector and no observable ever fires, most gauge measurements are
random (that is what makes it a random-measurement workload for the
inverse-tableau reference sample), and a single X error on a data qubit
fires exactly the two Z-stabilizer detectors of its column pairs at the end
of the round."""
import numpy as np

import oracle
from paper_2103_02202_gb300 import workloads as W


def test_bacon_shor_noiseless_detectors_and_observable_never_fire():
    for d in (2, 3, 5):
        c = oracle.Circuit(W.bacon_shor(d, 4, 0.0, observable=True))
        _, det = c.sample(np.arange(300), 9)
        assert det.shape[1] == c.num_detectors + 1
        assert not det.any()


def test_bacon_shor_gauges_are_mostly_random():
    d = 6
    c = oracle.Circuit(W.bacon_shor(d, 3, 0.0))
    _, deterministic = c.reference()
    nx = nz = d * (d - 1)
    rounds = deterministic[: 3 * (nx + nz)].reshape(3, nx + nz)
    # every first-round X gauge is random (the data starts in |0...0>), and
    # after that only a small fraction of gauge outcomes is fixed by the
    # earlier ones (here one in six)
    assert rounds[0, :nx].mean() == 0.0
    assert 0 < rounds.mean() < 0.25


def test_bacon_shor_single_data_error_fires_its_column_pairs():
    d = 4
    base = W.bacon_shor(d, 2, 0.0)
    lines = base.splitlines()
    # a certain X error on data qubit (r=1, c=1) right before the final data measurement
    k = max(i for i, l in enumerate(lines) if l.startswith("M "))
    lines.insert(k, "X_ERROR(1) %d" % (1 * d + 1))
    c = oracle.Circuit("\n".join(lines) + "\n")
    _, det = c.sample(np.arange(64), 3)
    fired = np.flatnonzero(det[0])
    # the final Z-stabilizer detectors are the last d - 1; column 1 lies in pairs (0,1) and (1,2)
    D = c.num_detectors
    assert fired.tolist() == [D - (d - 1) + 0, D - (d - 1) + 1]
    assert (det == det[0]).all()

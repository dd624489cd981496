"""The request server's admission policy (eo_admission_simulate: the same
Admission class the server thread runs, driven by a discrete-event
simulation on the host; no GPU)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def eo():
    from paper_1806_01036_gb300 import build
    build.build()
    import paper_1806_01036_gb300 as eo_mod
    return eo_mod


def intervals(start, duration):
    return [(s, s + d) for s, d in zip(start, duration)]


def test_work_conserving_when_nothing_binds(eo):
    arr = [0.0, 0.1, 0.2, 0.3]
    start, peak = eo.admission_simulate(10**6, 8, 0, [0, 1, 2, 3], [10] * 4, arr, [1.0] * 4)
    assert list(start) == arr and peak == 4


def test_continuous_admission_as_slots_free(eo):
    # two slots: a long and a short request run; the third arrival takes the
    # short one's slot when it frees, not when the long one ends
    start, peak = eo.admission_simulate(10**6, 2, 0, [0, 1, 2], [1, 1, 1], [0.0, 0.0, 0.5], [10.0, 1.0, 1.0])
    assert list(start) == [0.0, 0.0, 1.0] and peak == 2


def test_one_request_at_a_time_per_basis_in_order(eo):
    basis = [7, 7, 7, 3]
    start, _ = eo.admission_simulate(10**6, 8, 0, basis, [1] * 4, [0.0, 0.0, 0.0, 0.0], [2.0, 1.0, 1.0, 1.0])
    # basis 7 runs its requests back to back in submission order; basis 3 is not held up by them
    assert list(start) == [0.0, 2.0, 3.0, 0.0]


def test_memory_budget_and_no_overtaking(eo):
    # budget 100 with 20 resident (80 for requests): the 70-byte request waits
    # for memory and the later small ones queue behind it instead of
    # overtaking it; at t = 5 it starts with one 10-byte request (80 bytes),
    # and the last waits until t = 6
    basis = [0, 1, 2, 3]
    nbytes = [40, 70, 10, 10]
    start, _ = eo.admission_simulate(100, 8, 20, basis, nbytes, [0.0, 0.1, 0.2, 0.3], [5.0, 1.0, 1.0, 1.0])
    assert list(start) == [0.0, 5.0, 5.0, 6.0]


def test_never_fits_is_refused(eo):
    start, _ = eo.admission_simulate(100, 4, 50, [0, 1], [60, 10], [0.0, 0.0], [1.0, 1.0])
    assert start[0] == -1.0 and start[1] == 0.0


def test_random_trace_respects_budget_slots_and_basis_order(eo):
    rng = np.random.default_rng(5)
    n, slots, budget, resident = 400, 6, 1000, 300
    basis = rng.integers(0, 20, n)
    nbytes = rng.integers(1, 300, n)
    arrival = np.cumsum(rng.exponential(0.05, n))
    duration = rng.exponential(0.3, n)
    start, peak = eo.admission_simulate(budget, slots, resident, basis, nbytes, arrival, duration)
    assert np.all(start >= arrival - 1e-12)
    assert peak <= slots
    iv = intervals(start, duration)
    events = sorted(set([s for s, _ in iv] + [e for _, e in iv]))
    for t in events:  # at every start or end, what runs fits the slots and the budget
        run = [i for i in range(n) if iv[i][0] <= t < iv[i][1]]
        assert len(run) <= slots
        assert sum(int(nbytes[i]) for i in run) <= budget - resident
    for b in range(20):  # per basis: submission order, no overlap
        idx = [i for i in np.argsort(arrival, kind="stable") if basis[i] == b]
        for i, j in zip(idx, idx[1:]):
            assert start[j] >= start[i] + duration[i] - 1e-12


def test_bad_arguments_raise(eo):
    with pytest.raises(ValueError):
        eo.admission_simulate(100, 0, 0, [0], [1], [0.0], [1.0])
    with pytest.raises(ValueError):
        eo.admission_simulate(100, 1, 200, [0], [1], [0.0], [1.0])  # resident beyond the budget

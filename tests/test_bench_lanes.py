"""Host logic of the benchmark's lanes (no GPU): K steps of S systems are
taken from one shared queue by the lane threads, so every system is solved
exactly K times, a free lane takes the next solve whatever system it is,
and the report and lane of each system's last solve are kept."""
import collections
import threading
import time

import bench


def _lanes(count):
    ln = bench.Lanes.__new__(bench.Lanes)  # no streams or handles: the solve is faked below
    ln.spd = None
    ln.handles = [f"h{j}" for j in range(count)]
    ln.X = [f"x{j}" for j in range(count)]
    return ln


def test_every_system_solved_k_times_from_one_queue(monkeypatch):
    calls = []
    lock = threading.Lock()

    def fake_solve(spd, h, A, B, X, prec, opts, kappa):
        # an expensive system (kappa 1e6) keeps its lane busy longer
        time.sleep(0.02 if kappa >= 1e6 else 0.002)
        with lock:
            calls.append((h, kappa, X))
        return ("factor-report", kappa), ("solve-report", kappa, h)

    monkeypatch.setattr(bench, "solve_one", fake_solve)
    ln = _lanes(3)
    systems = [(1e2, "A0", "B0"), (1e4, "A1", "B1"), (1e6, "A2", "B2")]
    out = ln.run(systems, ["auto"] * 3, {}, 5)
    per_system = collections.Counter(k for _, k, _ in calls)
    assert per_system == {1e2: 5, 1e4: 5, 1e6: 5}
    # each handle uses its own solution buffer
    assert all(x == "x" + h[1:] for h, _, x in calls)
    # a lane is not tied to one system: the cheap systems move between lanes
    lanes_of = collections.defaultdict(set)
    for h, k, _ in calls:
        lanes_of[k].add(h)
    assert any(len(v) > 1 for v in lanes_of.values())
    # the kept report is the system's own, from the lane recorded for it
    for i, (k, _, _) in enumerate(systems):
        fr, sr = out[i]
        assert fr == ("factor-report", k) and sr[1] == k
        assert sr[2] == ln.handles[ln.last_lane[i]]


def test_a_failing_solve_stops_the_queue_and_is_raised(monkeypatch):
    seen = []

    def fake_solve(spd, h, A, B, X, prec, opts, kappa):
        seen.append(kappa)
        if kappa == 1e4:
            raise RuntimeError("spd_solve_ir kappa=1e4: planted failure")
        return None, None

    monkeypatch.setattr(bench, "solve_one", fake_solve)
    ln = _lanes(2)
    systems = [(1e2, "A0", "B0"), (1e4, "A1", "B1")]
    try:
        ln.run(systems, ["auto"] * 2, {}, 50)
    except RuntimeError as e:
        assert "planted failure" in str(e)
    else:
        raise AssertionError("the lane's exception was not raised")
    assert len(seen) < 100  # the other lane stopped taking solves

"""Host-side logic of the serving driver (no GPU): the seeded Poisson stream,
the size classes of the mixed-size workload, the submit / step / collect
loop against a fake server that finishes each request a fixed number of
steps after its submission, and the latency statistics."""
import numpy as np

from paper_2603_01064_gb300 import serve


def _ops():
    W = [None]
    return [serve.Operator(16, 2, 1.0, 1e-2, W, "bf16_refine", slots=2),
            serve.Operator(32, 3, 1.0, 1e-2, W, "fp32", slots=1)]


def test_poisson_stream_is_seeded_and_shaped():
    ops = _ops()
    a = serve.poisson_stream(ops, 400, rate=200.0, seed=3, rhs_batch=4)
    b = serve.poisson_stream(ops, 400, rate=200.0, seed=3, rhs_batch=4)
    t = np.array([r.t_arrival for r in a])
    assert np.all(np.diff(t) > 0) and t[0] > 0
    # exponential gaps: mean 1 / rate within 4 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 4 * (1 / 200.0) / np.sqrt(len(gaps))
    assert [r.op for r in a] == [r.op for r in b] and np.array_equal(a[7].f, b[7].f)
    counts = np.bincount([r.op for r in a], minlength=2)
    assert abs(counts[0] - 200) < 4 * np.sqrt(100)  # uniform choice of operator
    for r in a:
        o = ops[r.op]
        assert r.f.shape == (o.n, o.n) and r.f.dtype == np.float32
        assert r.u.dtype == (np.float32 if o.precision == "fp32" else np.float64)
        assert not np.any(r.u)


def test_size_classes():
    ops = serve.size_classes([64, 512, 2048], lambda s: [s])
    assert [o.n for o in ops] == [64, 512, 2048]
    assert [o.levels for o in ops] == [4, 7, 9]  # coarsest grid 8 x 8
    assert [o.sigma for o in ops] == [1.0, 2.0, 8.0]
    assert [o.weights for o in ops] == [[1.0], [2.0], [8.0]]


class FakeServer:
    """Finishes a request `steps` calls to step() after its submission."""

    def __init__(self, steps):
        self.steps, self.t, self.live, self.finished, self.submitted = steps, 0, {}, {}, []

    def submit(self, op, f, u):
        rid = len(self.submitted)
        self.submitted.append((op, f.shape))
        self.live[rid] = self.t
        return rid

    def stats(self):
        return 0, len(self.live), 0

    def step(self):
        self.t += 1
        done = [r for r, t0 in self.live.items() if self.t - t0 >= self.steps]
        for r in done:
            self.finished[r] = (self.live.pop(r), self.t)
        return len(done)

    def query(self, rid):
        if rid in self.finished:
            t0, t1 = self.finished[rid]
            return 2, ((3,), (0,), (1e-7,)), float(t0), 0.0, float(t1)
        return 1, (), 0.0, 0.0, 0.0


def test_run_stream_submits_when_due_and_collects_every_request():
    ops = _ops()
    reqs = serve.poisson_stream(ops, 30, rate=2000.0, seed=5, rhs_batch=2)
    srv = FakeServer(steps=3)
    elapsed, done = serve.run_stream(srv, [10, 11], reqs, time_limit_s=30.0)
    assert len(done) == 30 and elapsed < 30.0
    assert sorted(r.rid for r in done) == list(range(30))
    # submitted in arrival order, to the operator id of the request's class
    assert [op for op, _ in srv.submitted] == [10 + r.op for r in reqs]
    assert all(r.state == 2 and r.t_done - r.t_submit == 3.0 for r in done)
    st = serve.latency_stats(done)
    assert st["p50_ms"] == st["p99_ms"] == 3000.0


def test_latency_stats():
    class R:
        def __init__(self, a, b):
            self.t_submit, self.t_done = a, b
    done = [R(0.0, 0.001 * (k + 1)) for k in range(100)]
    st = serve.latency_stats(done)
    assert abs(st["p50_ms"] - 50.5) < 1e-9 and abs(st["p99_ms"] - 99.01) < 1e-9
    assert abs(st["mean_ms"] - 50.5) < 1e-9
    assert serve.latency_stats([]) == {"p50_ms": None, "p99_ms": None}

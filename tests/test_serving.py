"""Serving loop: the job mix, admission by device memory, continuous batching
of chunked sweeps over several streams, and mix-independence of results."""

import numpy as np
import pytest

from paper_0704_3573_gb300 import serve


def test_job_mix_distribution():
    jobs = serve.job_mix(400, seed=3)
    dims = np.array([j.dim for j in jobs])
    assert 0.4 < (dims == 3).mean() < 0.6
    for j in jobs:
        assert j.L in (serve.L3D if j.dim == 3 else serve.L2D)
        assert 1 <= j.samples <= 64 and 0.5 <= j.T <= 2.0
        assert 10 ** 3 <= j.sweeps <= 10 ** 5 and j.sweeps % 10 == 0
    logs = np.log10([j.sweeps for j in jobs])
    assert abs(logs.mean() - 4.0) < 0.15  # log-uniform on [3, 5]
    assert len({j.seed for j in jobs}) == len(jobs)


def test_poisson_arrivals():
    jobs = serve.poisson_arrivals(serve.job_mix(2000, seed=5), rate=50.0, seed=1)
    t = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 3 * (1 / 50.0) / np.sqrt(len(gaps))


def test_footprint_is_required_bytes():
    j = serve.Job(0, 3, 16, 10, 1.0, 100, 0, seed=1)
    assert serve.footprint(j) > 16 ** 3 * 8  # one 64-lane word per site plus couplings


@pytest.mark.gpu
def test_results_identical_alone_and_in_the_mix(ianus):
    jobs = serve.job_mix(16, seed=0x0704357300000004, sweep_scale=0.02, min_sweeps=10,
                         L3=(4, 6, 8), L2=(8, 16, 32), max_samples=70)
    jobs = serve.poisson_arrivals(jobs, rate=400.0, seed=2)
    server = serve.Server(mem_budget=64 << 20, max_active=6, n_streams=3, chunk_sweeps=7)
    results, stats = server.run(jobs)
    assert stats["jobs"] == len(jobs)
    assert stats["p50_latency_s"] <= stats["p99_latency_s"]
    for r in results:
        E, M = serve.run_alone(r.job)
        assert np.array_equal(r.energy, E), r.job
        assert np.array_equal(r.magnetisation, M), r.job
        assert r.finished >= r.job.arrival


@pytest.mark.gpu
def test_admission_respects_memory_budget(ianus):
    jobs = serve.job_mix(6, seed=9, sweep_scale=0.01, min_sweeps=10, L3=(8,), L2=(32,), max_samples=64)
    budget = min(serve.footprint(j) for j in jobs)  # any two jobs exceed it: one at a time
    server = serve.Server(mem_budget=budget, max_active=8, n_streams=2, chunk_sweeps=5)
    results, stats = server.run(jobs, realtime=False)
    spans = sorted((r.admitted, r.finished) for r in results)
    for (a0, f0), (a1, _) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-6  # the next job is admitted only after the previous one left


class _FakeLattice:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def _bare_server():
    srv = serve.Server.__new__(serve.Server)  # host bookkeeping only, no CUDA streams
    srv._closing = []
    return srv


def test_finished_job_lattice_outlives_its_running_compile():
    """A job that finishes while a worker still compiles its kernel (reading
    the lattice's shape) keeps its lattice open until the compile returns;
    a compile that never started is cancelled and the lattice closes at
    once."""
    from concurrent.futures import Future

    srv = _bare_server()
    running = Future()
    assert running.set_running_or_notify_cancel()  # a worker has started it
    a = serve._Active()
    a.lat, a.ready = _FakeLattice(), running
    lat = a.lat
    srv._retire(a)
    assert not lat.closed and a.lat is None and len(srv._closing) == 1
    srv._reap()
    assert not lat.closed
    running.set_result(True)
    srv._reap()
    assert lat.closed and srv._closing == []

    pending = Future()  # queued, not started: cancelled
    b = serve._Active()
    b.lat, b.ready = _FakeLattice(), pending
    lat_b = b.lat
    srv._retire(b)
    assert lat_b.closed and pending.cancelled() and srv._closing == []

    done = Future()
    done.set_result(False)
    c = serve._Active()
    c.lat, c.ready = _FakeLattice(), done
    lat_c = c.lat
    srv._retire(c)
    assert lat_c.closed


def test_drain_waits_for_every_compile():
    import threading
    import time
    from concurrent.futures import ThreadPoolExecutor

    srv = _bare_server()
    gate = threading.Event()
    with ThreadPoolExecutor(max_workers=1) as pool:
        fut = pool.submit(gate.wait, 10.0)
        a = serve._Active()
        a.lat, a.ready = _FakeLattice(), fut
        lat = a.lat
        t0 = time.monotonic()
        while not fut.running() and time.monotonic() - t0 < 5.0:
            time.sleep(0.001)
        assert fut.running()
        srv._retire(a)
        assert not lat.closed
        gate.set()
        srv._drain()
        assert lat.closed and srv._closing == []

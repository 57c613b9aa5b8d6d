"""Continuous-batching server for spin-glass Monte Carlo jobs.

A job is one lattice batch (3D or 2D EA +-J glass, 1..64 disorder samples,
one temperature, a number of sweeps, Metropolis or heat bath) whose result is
its final energy and magnetisation per sample.  Jobs arrive over time; the
server admits them while the device-memory budget and the number of active
slots allow, keeps each admitted job's lattice and random-stream state
resident on the GPU, and interleaves their sweeps: every active job receives
its next chunk of sweeps on one of several CUDA streams as soon as its
previous chunk has finished, so the work of different jobs overlaps on the
device.  A finished job is measured, its memory released, and waiting jobs
are admitted in arrival order.

Results do not depend on the mix: each job owns its lattice, and every
random number is a function of (job seed, sample, slot, site, sweep) only.
All per-site work runs in libianus.so; this module only schedules calls.

FusedServer packs jobs of equal (dimension, side) into the 64-bit lanes of
shared pool lattices (ianus_segment_load): a job of n samples takes n
contiguous lanes of one 64-lane group, with its own temperature, algorithm,
sweep count and random stream, so small jobs stop wasting the other lanes of
a word and one launch advances every job of a pool.  A job's trajectory in a
pool is still that of its own lattice, bit for bit.
"""

from __future__ import annotations

import dataclasses
import math
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import HEATBATH, METROPOLIS, Lattice
from . import lib as _lib

L3D = (8, 12, 16, 24, 32, 48, 64, 80)
L2D = (64, 128, 256, 512, 1024)


@dataclasses.dataclass
class Job:
    id: int
    dim: int
    L: int
    samples: int
    T: float
    sweeps: int
    algo: int
    seed: int
    arrival: float = 0.0  # seconds after the start of the run

    @property
    def updates(self) -> int:
        return self.samples * self.L ** self.dim * self.sweeps


@dataclasses.dataclass
class Result:
    job: Job
    energy: np.ndarray         # [samples]
    magnetisation: np.ndarray  # [samples]
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.job.arrival


def job_mix(n_jobs: int, seed: int = 0x0704357300000004, sweep_scale: float = 1.0, min_sweeps: int = 10,
            L3=L3D, L2=L2D, max_samples: int = 64) -> list[Job]:
    """The serving mix: 3D or 2D with probability 1/2, L uniform over the
    listed sides, samples uniform in 1..64, T uniform in [0.5, 2.0], sweeps
    log-uniform in [10^3, 10^5] (a multiple of 10, times sweep_scale),
    Metropolis or heat bath with probability 1/2.  Seeded."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n_jobs):
        dim = 3 if rng.random() < 0.5 else 2
        L = int(rng.choice(L3 if dim == 3 else L2))
        samples = int(rng.integers(1, max_samples + 1))
        T = float(rng.uniform(0.5, 2.0))
        sweeps = int(round(10 ** rng.uniform(3, 5) / 10)) * 10
        sweeps = max(min_sweeps, int(round(sweeps * sweep_scale / 10)) * 10)
        algo = METROPOLIS if rng.random() < 0.5 else HEATBATH
        jobs.append(Job(i, dim, L, samples, T, sweeps, algo, seed=(seed + 1000003 * (i + 1)) & ((1 << 64) - 1)))
    return jobs


def poisson_arrivals(jobs: list[Job], rate: float, seed: int = 11) -> list[Job]:
    """Assign Poisson arrival times (rate in jobs per second)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for j in jobs:
        t += float(rng.exponential(1.0 / rate)) if rate > 0 else 0.0
        out.append(dataclasses.replace(j, arrival=t))
    return out


def footprint(job: Job) -> int:
    """Device bytes the job's lattice needs (ianus_required_bytes)."""
    import ctypes

    from . import ABI_VERSION, IanusConfig, LAYOUT_BITS64

    c = IanusConfig()
    c.abi_version = ABI_VERSION
    c.model, c.dim, c.L = 0, job.dim, job.L
    c.n_samples, c.n_replicas, c.n_temps = job.samples, 1, 1
    c.layout, c.disorder, c.series_capacity, c.seed = LAYOUT_BITS64, 0, 1, job.seed
    return int(_lib().ianus_required_bytes(ctypes.byref(c)))


class _Active:
    __slots__ = ("job", "lat", "stream", "event", "done", "admitted", "footprint", "ready")


class Server:
    """Admission by memory and slots; chunked, stream-interleaved sweeps.

    A job's lattice sweeps with a kernel specialised for its temperature,
    compiled at run time.  With compile_workers > 0 that compilation runs on
    worker threads (ianus_prepare_sweep): the job starts at once on the
    precompiled kernel (variant 1, the same trajectory bit for bit) and
    switches at its next chunk after its kernel is ready, so no compilation
    stalls the scheduling loop.  With compile_workers = 0 the first sweep of
    a job compiles on the scheduling thread."""

    def __init__(self, mem_budget: int = 8 << 30, max_active: int = 64, n_streams: int = 8,
                 chunk_sweeps: int = 100, compile_workers: int = 8):
        import torch

        self.torch = torch
        self.mem_budget = mem_budget
        self.max_active = max_active
        self.chunk = chunk_sweeps
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self._rr = 0
        self._pool = ThreadPoolExecutor(max_workers=compile_workers) if compile_workers > 0 else None
        self._closing: list = []  # (lattice, compile future) of finished jobs

    def _admit(self, job: Job, now: float) -> _Active:
        a = _Active()
        a.job = job
        a.stream = self.streams[self._rr % len(self.streams)]
        self._rr += 1
        a.lat = Lattice(dim=job.dim, L=job.L, n_samples=job.samples, n_replicas=1, seed=job.seed,
                        layout="bits64", series_capacity=1, stream=a.stream)
        a.ready = None
        if self._pool is not None:
            a.lat.set_variant(1)
            a.ready = self._pool.submit(a.lat.prepare_sweep, job.algo, 1.0 / job.T, 0)
        a.event = None
        a.done = 0
        a.admitted = now
        a.footprint = footprint(job)
        return a

    def _retire(self, a: _Active):
        """Close a finished job's lattice, or keep it until the compilation
        that reads its shape on a worker thread returns."""
        if a.ready is not None and not a.ready.done() and not a.ready.cancel():
            self._closing.append((a.lat, a.ready))
        else:
            a.lat.close()
        a.lat = None
        self._reap()

    def _reap(self):
        keep = []
        for lat, fut in self._closing:
            if fut.done():
                lat.close()
            else:
                keep.append((lat, fut))
        self._closing = keep

    def _drain(self):
        for lat, fut in self._closing:
            fut.result()
            lat.close()
        self._closing = []

    def _issue(self, a: _Active):
        if a.ready is not None and a.ready.done():
            if a.ready.result():
                a.lat.set_variant(0)
            a.ready = None
        n = min(self.chunk, a.job.sweeps - a.done)
        with self.torch.cuda.stream(a.stream):
            a.lat.sweep(a.job.algo, 1.0 / a.job.T, n)
            ev = self.torch.cuda.Event()
            ev.record(a.stream)
        a.event = ev
        a.done += n

    def run(self, jobs: list[Job], realtime: bool = True) -> tuple[list[Result], dict]:
        """Serve jobs (sorted by arrival).  With realtime=False every job is
        available at t=0 (a saturated queue)."""
        torch = self.torch
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        active: list[_Active] = []
        results: list[Result] = []
        used = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # admit arrived jobs, in order, while memory and slots allow
            while pending and len(active) < self.max_active and (not realtime or pending[0].arrival <= now):
                fp = footprint(pending[0])
                if used + fp > self.mem_budget and active:
                    break
                job = pending.popleft()
                a = self._admit(job, now)
                used += a.footprint
                active.append(a)
                self._issue(a)
            progressed = False
            still = []
            for a in active:
                if a.event is not None and not a.event.query():
                    still.append(a)
                    continue
                progressed = True
                if a.done < a.job.sweeps:
                    self._issue(a)
                    still.append(a)
                    continue
                E, M, _ = a.lat.measure(overlap=False)
                fin = time.perf_counter() - t0
                results.append(Result(a.job, E[:, 0, 0].copy(), M[:, 0, 0].copy(), a.admitted, fin))
                used -= a.footprint
                self._retire(a)
            active = still
            self._reap()
            if not progressed:
                if realtime and not active and pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        self._drain()
        lat = np.array([r.latency for r in results])
        upd = sum(r.job.updates for r in results)
        stats = {
            "jobs": len(results),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "makespan_s": wall,
            "updates": upd,
            "updates_per_ns": upd / (wall * 1e9),
        }
        results.sort(key=lambda r: r.job.id)
        return results, stats


def run_alone(job: Job) -> tuple[np.ndarray, np.ndarray]:
    """The same job on its own lattice, outside the server."""
    lat = Lattice(dim=job.dim, L=job.L, n_samples=job.samples, n_replicas=1, seed=job.seed, layout="bits64",
                  series_capacity=1)
    lat.sweep(job.algo, 1.0 / job.T, job.sweeps)
    E, M, _ = lat.measure(overlap=False)
    lat.close()
    return E[:, 0, 0], M[:, 0, 0]


def calibrated_rate(server: Server, jobs: list[Job], load: float = 0.8) -> float:
    """Arrival rate (jobs/s) at `load` times the capacity measured on a
    saturated run of the given jobs."""
    _, st = server.run(jobs, realtime=False)
    return load * len(jobs) / st["makespan_s"] if st["makespan_s"] > 0 else math.inf


def pool_footprint(dim: int, L: int, groups: int) -> int:
    """Device bytes of a pool lattice of `groups` 64-lane groups."""
    import ctypes

    from . import ABI_VERSION, IanusConfig, LAYOUT_BITS64

    c = IanusConfig()
    c.abi_version = ABI_VERSION
    c.model, c.dim, c.L = 0, dim, L
    c.n_samples, c.n_replicas, c.n_temps = 64 * groups, 1, 1
    c.layout, c.disorder, c.series_capacity, c.seed = LAYOUT_BITS64, 0, 1, 1
    return int(_lib().ianus_required_bytes(ctypes.byref(c)))


class _Pool:
    """One pool lattice: lanes of `groups` groups shared by jobs of one (D, L)."""

    def __init__(self, dim: int, L: int, groups: int, stream):
        self.dim, self.L, self.groups = dim, L, groups
        self.stream = stream
        self.lat = Lattice(dim=dim, L=L, n_samples=64 * groups, n_replicas=1, seed=1, layout="bits64",
                           series_capacity=1, stream=stream)
        self.free = [(1 << 64) - 1] * groups  # free-lane masks
        self.jobs = {}                         # (group, lane0) -> (job, admitted)
        self.event = None
        self.footprint = pool_footprint(dim, L, groups)

    @staticmethod
    def pieces(job: Job) -> list[int]:
        """Sizes of the job's segments: 64 samples each, the rest last."""
        return [min(64, job.samples - 64 * k) for k in range((job.samples + 63) // 64)]

    def place(self, job: Job):
        """First fit of every segment of the job: [(group, lane0)], or None."""
        free = list(self.free)
        out = []
        for n in self.pieces(job):
            want = (1 << n) - 1
            spot = None
            for g, f in enumerate(free):
                for lane0 in range(0, 65 - n):
                    if (f >> lane0) & want == want:
                        spot = (g, lane0)
                        break
                if spot:
                    break
            if spot is None:
                return None
            free[spot[0]] &= ~(want << spot[1])
            out.append(spot)
        return out

    def load(self, job: Job, where, now: float):
        for k, ((g, lane0), n) in enumerate(zip(where, self.pieces(job))):
            self.lat.segment_load(g, lane0, n, job.seed, job.algo, 1.0 / job.T, job.sweeps, job_group=k)
            self.free[g] &= ~(((1 << n) - 1) << lane0)
        self.jobs[tuple(where)] = (job, now)

    def busy(self) -> bool:
        return self.event is not None and not self.event.query()


class FusedServer:
    """Continuous batching with lane fusion: pools per (D, L), chunked
    sweeps of all live jobs of a pool per launch, pools on separate streams.

    Jobs on lattices of more than `fuse_max_sites` sites run on their own
    lattices as in Server: their words are long enough to fill the GPU, and
    alone they get the kernel specialised for one temperature, which lanes at
    different temperatures cannot use."""

    def __init__(self, mem_budget: int = 8 << 30, groups_per_pool: int = 4, n_streams: int = 8,
                 chunk_sweeps: int = 100, fuse_max_sites: int = 1 << 16, max_solo: int = 32,
                 compile_workers: int = 8):
        import torch

        self.torch = torch
        self.mem_budget = mem_budget
        self.groups = groups_per_pool
        self.chunk = chunk_sweeps
        self.fuse_max_sites = fuse_max_sites
        self.max_solo = max_solo
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self._solo = Server(mem_budget, max_active=max_solo, n_streams=1, chunk_sweeps=chunk_sweeps,
                            compile_workers=compile_workers)
        self._solo.streams = self.streams

    def run(self, jobs: list[Job], realtime: bool = True) -> tuple[list[Result], dict]:
        torch = self.torch
        waiting: dict[tuple[int, int], deque] = {}
        arrivals = deque(sorted(jobs, key=lambda j: j.arrival))
        pools: dict[tuple[int, int], list[_Pool]] = {}
        results: list[Result] = []
        solo_wait: deque = deque()
        solo: list[_Active] = []
        used = 0
        n_pools = 0
        t0 = time.perf_counter()
        while arrivals or solo_wait or solo or any(waiting.values()) or \
                any(p.jobs for ps in pools.values() for p in ps):
            now = time.perf_counter() - t0
            while arrivals and (not realtime or arrivals[0].arrival <= now):
                j = arrivals.popleft()
                if j.L ** j.dim > self.fuse_max_sites:
                    solo_wait.append(j)
                else:
                    waiting.setdefault((j.dim, j.L), deque()).append(j)
            progressed = False
            # jobs on their own lattices, as in Server
            while solo_wait and len(solo) < self.max_solo:
                fp = footprint(solo_wait[0])
                if used + fp > self.mem_budget and (solo or used > 0):
                    break
                a = self._solo._admit(solo_wait.popleft(), now)
                used += a.footprint
                solo.append(a)
                self._solo._issue(a)
                progressed = True
            still = []
            for a in solo:
                if a.event is not None and not a.event.query():
                    still.append(a)
                    continue
                progressed = True
                if a.done < a.job.sweeps:
                    self._solo._issue(a)
                    still.append(a)
                    continue
                E, M, _ = a.lat.measure(overlap=False)
                results.append(Result(a.job, E[:, 0, 0].copy(), M[:, 0, 0].copy(), a.admitted,
                                      time.perf_counter() - t0))
                used -= a.footprint
                self._solo._retire(a)
            solo = still
            self._solo._reap()
            for key, q in waiting.items():
                ps = pools.setdefault(key, [])
                # admit in arrival order into idle pools (a busy pool is fed after its chunk)
                while q:
                    job = q[0]
                    spot = None
                    for p in ps:
                        if not p.busy():
                            w = p.place(job)
                            if w is not None:
                                spot = (p, w)
                                break
                    # a new pool only when no pool has room (a busy one with room is waited for)
                    if spot is None and all(p.place(job) is None for p in ps):
                        fp = pool_footprint(key[0], key[1], self.groups)
                        if used + fp <= self.mem_budget or not ps:
                            p = _Pool(key[0], key[1], self.groups, self.streams[n_pools % len(self.streams)])
                            n_pools += 1
                            used += p.footprint
                            ps.append(p)
                            spot = (p, p.place(job))
                    if spot is None:
                        break
                    q.popleft()
                    spot[0].load(job, spot[1], now)
                    progressed = True
            for ps in pools.values():
                for p in ps:
                    if p.busy() or not p.jobs:
                        continue
                    finished = [w for w in p.jobs if p.lat.segment_state(*w[0])[0] >= p.jobs[w][0].sweeps]
                    if finished:
                        E, M, _ = p.lat.measure(overlap=False)
                        fin = time.perf_counter() - t0
                        for where in finished:
                            job, adm = p.jobs.pop(where)
                            es, ms = [], []
                            for (g, lane0), n in zip(where, p.pieces(job)):
                                lo = 64 * g + lane0
                                es.append(E[lo:lo + n, 0, 0])
                                ms.append(M[lo:lo + n, 0, 0])
                                p.lat.segment_release(g, lane0)
                                p.free[g] |= ((1 << n) - 1) << lane0
                            results.append(Result(job, np.concatenate(es), np.concatenate(ms), adm, fin))
                        progressed = True
                    if p.jobs:
                        live = [p.jobs[w][0].sweeps - p.lat.segment_state(*w[0])[0] for w in p.jobs]
                        if max(live) > 0:
                            with torch.cuda.stream(p.stream):
                                p.lat.sweep_segments(min(self.chunk, max(live)))
                                p.event = torch.cuda.Event()
                                p.event.record(p.stream)
                            progressed = True
            if not progressed:
                if realtime and arrivals and not any(waiting.values()) and not solo and not solo_wait and \
                        not any(p.jobs for ps in pools.values() for p in ps):
                    time.sleep(max(0.0, min(0.002, arrivals[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        self._solo._drain()
        for ps in pools.values():
            for p in ps:
                p.lat.close()
        lat = np.array([r.latency for r in results])
        upd = sum(r.job.updates for r in results)
        stats = {
            "jobs": len(results),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "makespan_s": wall,
            "updates": upd,
            "updates_per_ns": upd / (wall * 1e9),
            "pools": n_pools,
        }
        results.sort(key=lambda r: r.job.id)
        return results, stats

"""Continuous-batching job server for SRD boxes on one GPU.

Jobs (box size, density, rotation angle, thermostat, step count, seed) arrive
over time.  The server keeps every admitted job's state resident in device
memory inside one batch (libmpcd ``mpcd_batch_*``): all resident boxes advance
together, one fused launch per step.  Between chunks of steps it retires
finished jobs and admits queued ones as boxes and memory free up (FIFO,
admission by device-memory footprint), so jobs that arrive while others run
join them on the device.  A chunk runs until the next resident job finishes
(capped), so every job stops exactly at its step count.

Because every random draw is keyed by the box's own seed, step and cell, a
job's result does not depend on which other jobs shared its launches.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import Batch, box_footprint


@dataclass
class Job:
    id: int
    arrival: float            # seconds after the start of the run
    n: tuple                  # cells per axis
    density: float
    steps: int
    alpha_deg: float = 130.0
    thermostat: bool = False
    seed: int = 0
    dt: float = 0.1
    kT: float = 1.0
    # filled in by the server
    admitted: float | None = None
    finished: float | None = None
    result: dict | None = None
    state: tuple | None = None

    @property
    def particles(self) -> int:
        return int(round(self.density * self.n[0] * self.n[1] * self.n[2]))

    def box_kwargs(self) -> dict:
        return dict(n=self.n, alpha_deg=self.alpha_deg, thermostat=self.thermostat,
                    seed=self.seed, dt=self.dt, kT=self.kT)


@dataclass
class ServeStats:
    jobs: int
    makespan_s: float
    particle_steps: float
    latency_s: list = field(default_factory=list)
    wait_s: list = field(default_factory=list)
    max_resident: int = 0
    chunks: int = 0

    @property
    def throughput(self) -> float:
        return self.particle_steps / self.makespan_s if self.makespan_s > 0 else 0.0

    def percentile(self, q: float) -> float:
        return float(np.percentile(self.latency_s, q)) if self.latency_s else 0.0

    def as_dict(self) -> dict:
        return {"jobs": self.jobs, "makespan_s": self.makespan_s,
                "particle_steps": self.particle_steps, "particle_steps_per_s": self.throughput,
                "latency_p50_s": self.percentile(50), "latency_p99_s": self.percentile(99),
                "wait_p50_s": float(np.percentile(self.wait_s, 50)) if self.wait_s else 0.0,
                "max_resident": self.max_resident, "chunks": self.chunks}


class Server:
    """``batch_factory`` and ``footprint_fn`` default to the library's batch and
    footprint calls; the scheduling logic itself runs on the host."""

    def __init__(self, precision: str = "mixed", max_bytes: int = 0, max_boxes: int = 512,
                 max_chunk: int = 200, stream=None, keep_state: bool = False,
                 batch_factory=None, footprint_fn=None):
        self.precision = precision
        self.max_bytes = int(max_bytes)
        self.max_boxes = int(max_boxes)
        self.max_chunk = int(max_chunk)
        self.keep_state = keep_state
        make = batch_factory or (lambda: Batch(precision, stream=stream, max_bytes=self.max_bytes))
        self.batch = make()
        self._footprint = footprint_fn

    def footprint(self, job: Job) -> int:
        if self._footprint is not None:
            return int(self._footprint(job))
        return box_footprint(job.particles, precision=self.precision, **job.box_kwargs())

    def run(self, jobs, realtime: bool = True) -> ServeStats:
        """Serve ``jobs`` (arrival times in seconds from now).  With realtime
        false, arrivals are taken as already due (a closed-loop batch)."""
        order = sorted(jobs, key=lambda j: (j.arrival, j.id))
        waiting: deque = deque()
        resident: dict = {}   # slot -> (job, remaining steps)
        used = 0
        nxt = 0
        stats = ServeStats(jobs=len(order), makespan_s=0.0, particle_steps=0.0)
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: math.inf)
        while nxt < len(order) or waiting or resident:
            now = clock()
            while nxt < len(order) and order[nxt].arrival <= now:
                waiting.append(order[nxt])
                nxt += 1
            # admit in arrival order while a slot and the memory budget allow
            while waiting and len(resident) < self.max_boxes:
                job = waiting[0]
                need = self.footprint(job)
                if self.max_bytes and used + need > self.max_bytes and resident:
                    break
                slot = self.batch.add_thermal(job.particles, init_seed=job.seed, **job.box_kwargs())
                used += need
                job.admitted = time.perf_counter() - t0
                resident[slot] = [job, job.steps]
                waiting.popleft()
            stats.max_resident = max(stats.max_resident, len(resident))
            if not resident:
                if nxt < len(order):
                    delay = order[nxt].arrival - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(min(delay, 0.05))
                continue
            k = min(self.max_chunk, min(rem for _, rem in resident.values()))
            self.batch.step(k)
            self.batch.sync()
            stats.chunks += 1
            done = []
            for slot, entry in resident.items():
                entry[1] -= k
                stats.particle_steps += float(entry[0].particles) * k
                if entry[1] == 0:
                    done.append(slot)
            for slot in done:
                job = resident.pop(slot)[0]
                job.result = self.batch.observables(slot)
                if self.keep_state:
                    job.state = self.batch.get_state(slot)
                self.batch.remove(slot)
                used -= self.footprint(job)
                job.finished = time.perf_counter() - t0
                arrival = job.arrival if realtime else 0.0
                stats.latency_s.append(job.finished - arrival)
                stats.wait_s.append(job.admitted - arrival)
        stats.makespan_s = time.perf_counter() - t0
        return stats

    def close(self):
        self.batch.close()


def poisson_jobs(n_jobs: int, rate: float, seed: int = 5, l_min: int = 10, l_max: int = 160,
                 density: float = 5.0, steps_min: int = 100, steps_max: int = 5000,
                 alpha_deg: float = 130.0, thermostat_every: int = 2) -> list:
    """Synthetic served workload: Poisson arrivals at ``rate`` jobs/s, cubic
    boxes with edge log-uniform in [l_min, l_max] cells, uniform step counts,
    the thermostat on every ``thermostat_every``-th job, job seed = job id."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_jobs)
    t = np.cumsum(gaps) - gaps[0]
    edges = np.exp(rng.uniform(math.log(l_min), math.log(l_max), n_jobs)).round().astype(int)
    steps = rng.integers(steps_min, steps_max + 1, n_jobs)
    return [Job(id=i, arrival=float(t[i]), n=(int(e), int(e), int(e)), density=density,
                steps=int(steps[i]), alpha_deg=alpha_deg,
                thermostat=(i % thermostat_every == 1), seed=i)
            for i, e in enumerate(edges)]

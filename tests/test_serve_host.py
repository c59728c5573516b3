"""Host-side logic of the continuous-batching server, the served-workload
recipe and the batched-ensemble recipe (no GPU: the batch is a fake that
records what the server asks of it)."""
import math

import numpy as np

from paper_1801_10187_gb300 import inputs, serve


class FakeBatch:
    def __init__(self):
        self.boxes = {}
        self.next_slot = 0
        self.log = []

    def add_thermal(self, n_solvent, init_seed, **kw):
        slot = self.next_slot
        self.next_slot += 1
        self.boxes[slot] = {"n": n_solvent, "seed": init_seed, "steps": 0}
        self.log.append(("add", slot))
        return slot

    def step(self, k):
        assert k > 0
        for b in self.boxes.values():
            b["steps"] += k
        self.log.append(("step", k, len(self.boxes)))

    def sync(self):
        pass

    def observables(self, slot):
        b = self.boxes[slot]
        return {"step": b["steps"], "n": b["n"], "T_kin": 1.0}

    def get_state(self, slot):
        return (None, None, self.boxes[slot]["steps"])

    def remove(self, slot):
        del self.boxes[slot]
        self.log.append(("remove", slot))

    def close(self):
        pass


def make_server(**kw):
    fb = FakeBatch()
    srv = serve.Server(batch_factory=lambda: fb, footprint_fn=lambda j: j.particles * 100, **kw)
    return srv, fb


def test_every_job_runs_exactly_its_steps():
    jobs = serve.poisson_jobs(40, rate=100.0, seed=3, l_min=4, l_max=20, steps_min=10,
                              steps_max=400)
    srv, fb = make_server(max_chunk=37)
    st = srv.run(jobs, realtime=False)
    assert st.jobs == 40 and len(st.latency_s) == 40
    for j in jobs:
        assert j.result["step"] == j.steps  # observables taken exactly at the job's end
    assert st.particle_steps == sum(j.particles * j.steps for j in jobs)
    assert all(e[1] <= 37 for e in fb.log if e[0] == "step")


def test_admission_respects_memory_budget_and_fifo():
    jobs = [serve.Job(id=i, arrival=0.0, n=(10, 10, 10), density=5.0, steps=50 + 10 * i, seed=i)
            for i in range(12)]
    budget = 3 * jobs[0].particles * 100  # three boxes fit
    srv, fb = make_server(max_bytes=budget, max_chunk=1000)
    st = srv.run(jobs, realtime=False)
    assert st.max_resident == 3
    adds = [e[1] for e in fb.log if e[0] == "add"]
    assert adds == sorted(adds)  # admitted in arrival (FIFO) order
    # never more than three resident at a step
    assert all(e[2] <= 3 for e in fb.log if e[0] == "step")
    # the server steps to the next completion, so the first finisher ends at 50 steps
    first = [e for e in fb.log if e[0] == "step"][0]
    assert first[1] == 50


def test_poisson_recipe():
    jobs = serve.poisson_jobs(2000, rate=20.0, seed=5)
    gaps = np.diff([j.arrival for j in jobs])
    assert abs(gaps.mean() - 1 / 20.0) < 0.004
    edges = np.array([j.n[0] for j in jobs])
    assert edges.min() >= 10 and edges.max() <= 160
    # log-uniform: the median edge is near the geometric mean of the range
    assert abs(np.median(edges) - math.sqrt(10 * 160)) < 6
    steps = np.array([j.steps for j in jobs])
    assert steps.min() >= 100 and steps.max() <= 5000
    assert sum(j.thermostat for j in jobs) == 1000


def test_ensemble_recipe():
    e = inputs.ensemble(64, seed=4)
    assert len(e) == 64 and e == inputs.ensemble(64, seed=4)
    assert all(16 <= s["n"][0] <= 96 and s["n"][0] == s["n"][1] == s["n"][2] for s in e)
    assert {s["density"] for s in e} <= {5, 10}
    assert {s["alpha_deg"] for s in e} <= {90.0, 120.0, 130.0}
    assert [s["seed"] for s in e] == list(range(1000, 1064))

"""Host logic of the batch/serve scheduler with a fake context (no GPU)."""
import threading
import time

import pytest

from paper_1705_10845_gb300 import serve


class FakeCtx:
    live = 0
    lock = threading.Lock()

    def __init__(self, job):
        self.job = job
        with FakeCtx.lock:
            FakeCtx.live += 1

    def step(self, n):
        time.sleep(0.0005)

    def get(self, sys, what):
        return [self.job.jid]

    def close(self):
        with FakeCtx.lock:
            FakeCtx.live -= 1


class FakeX:
    Q, R = 0, 4


def fake_make(X, job, stream):
    if job.natoms == 13:
        raise RuntimeError("admission failed")
    return FakeCtx(job)


def test_squarings_rule():
    assert serve.squarings_for(3000.0) == 10
    assert serve.squarings_for(300.0) >= 13


def test_memory_estimate_grows_with_size():
    assert serve.bytes_estimate(512, 10) > 10 * serve.bytes_estimate(64, 10)


def test_memory_estimate_counts_operand_width():
    # TF32 operands take 4 bytes against FP16's 2: 4 more bytes per element for each of the
    # (n_sq + 1) + n_sq + 8 split matrices; FP64 keeps double arrays and no operands
    e = 2048 * 2048
    extra = serve.bytes_estimate(512, 10, "tf32x3") - serve.bytes_estimate(512, 10, "fp16x3")
    assert extra == pytest.approx(4 * (11 + 10 + 8) * e * 1.05, rel=1e-6)
    assert serve.bytes_estimate(512, 10, "bf16x3") == serve.bytes_estimate(512, 10, "fp16x3")


def test_all_jobs_run_within_the_memory_budget():
    jobs = [serve.Job(arrival=0.0, jid=i, natoms=32 + 8 * (i % 5), Te=1000.0, steps=5, seed=i) for i in range(20)]
    budget = 3 * max(serve.bytes_estimate(j.natoms, serve.squarings_for(j.Te)) for j in jobs)
    sch = serve.Scheduler(FakeX(), budget, workers=4, make_ctx=fake_make, keep_results=True)
    for j in jobs:
        sch.submit(j)
    wall = sch.run()
    assert wall > 0
    assert len(sch.finished) == 20 and all(j.done_steps == 5 for j in sch.finished)
    assert sch.peak_used <= budget
    assert sch.used == 0 and FakeCtx.live == 0
    assert sorted(j.result["q"][0] for j in sch.finished) == list(range(20))
    res = serve.summarize(sch, wall)
    assert res["total_steps"] == 100 and res["step_latency_ms_p99"] >= res["step_latency_ms_p50"]


def test_too_large_jobs_are_rejected_and_failures_reported():
    sch = serve.Scheduler(FakeX(), serve.bytes_estimate(64, 10), workers=2, make_ctx=fake_make)
    sch.submit(serve.Job(arrival=0.0, jid=0, natoms=4096, Te=1000.0, steps=3, seed=0))
    sch.submit(serve.Job(arrival=0.0, jid=1, natoms=13, Te=1000.0, steps=3, seed=1))
    sch.submit(serve.Job(arrival=0.0, jid=2, natoms=32, Te=1000.0, steps=3, seed=2))
    sch.run()
    assert len(sch.rejected) == 1 and sch.rejected[0].jid == 0
    errs = {j.jid: j.error for j in sch.finished}
    assert errs[1].endswith(": admission failed") and errs[2] == ""


def test_arrivals_are_admitted_in_time_order():
    jobs = [serve.Job(arrival=0.02 * (5 - i), jid=i, natoms=32, Te=1000.0, steps=1, seed=i) for i in range(5)]
    sch = serve.Scheduler(FakeX(), 10**12, workers=1, make_ctx=fake_make)
    for j in jobs:
        sch.submit(j)
    sch.run()
    order = [j.jid for j in sorted(sch.finished, key=lambda j: j.admitted)]
    assert order == [4, 3, 2, 1, 0]


class CountingCtx(FakeCtx):
    """Counts steps per job; job 3 fails at its second step."""
    steps = {}

    def step(self, n):
        if self.job.jid in CountingCtx.steps and self.job.ctx is not self:
            raise AssertionError("stepped through another job's context")
        CountingCtx.steps[self.job.jid] = CountingCtx.steps.get(self.job.jid, 0) + n
        if self.job.jid == 3 and CountingCtx.steps[3] == 2:
            raise RuntimeError("step failed")


def test_equal_arrivals_each_job_steps_exactly_its_own_count():
    # jobs with the same arrival time are distinct: finishing or failing one
    # must not remove or step another.  One worker admits all twelve before
    # the first step, so later jobs in its list finish before earlier ones.
    CountingCtx.steps = {}
    jobs = [serve.Job(arrival=0.0, jid=i, natoms=32, Te=1000.0, steps=3 + (i % 4), seed=i) for i in range(12)]
    sch = serve.Scheduler(FakeX(), 10**12, workers=1, make_ctx=lambda X, j, s: CountingCtx(j))
    for j in jobs:
        sch.submit(j)
    sch.run()
    assert len(sch.finished) == 12 and FakeCtx.live == 0
    for j in sch.finished:
        if j.jid == 3:
            assert "step failed" in j.error and j.done_steps == 2
        else:
            assert j.error == "" and j.done_steps == j.steps == CountingCtx.steps[j.jid]


def test_shortest_job_first_admission():
    # one worker, all jobs arrived: sjf admits by estimated work (size, squarings, steps)
    sizes = [400, 40, 200, 100, 800]
    jobs = [serve.Job(arrival=0.0, jid=i, natoms=n, Te=1000.0, steps=1, seed=i) for i, n in enumerate(sizes)]
    sch = serve.Scheduler(FakeX(), 10**13, workers=1, make_ctx=fake_make, policy="sjf")
    for j in jobs:
        sch.submit(j)
    sch.run()
    order = [j.natoms for j in sorted(sch.finished, key=lambda j: j.admitted)]
    assert order == sorted(sizes)
    with pytest.raises(ValueError):
        serve.Scheduler(FakeX(), 1, workers=1, policy="lifo")


def test_summary_counts_jobs_still_running():
    sch = serve.Scheduler(FakeX(), 10**12, workers=1, make_ctx=fake_make)
    j = serve.Job(arrival=0.0, jid=0, natoms=32, Te=1000.0, steps=10, seed=0)
    j.done_steps, j.lat = 4, [0.01] * 4
    sch.active[0].append(j)
    res = serve.summarize(sch, 1.0)
    assert res["total_steps"] == 4 and res["jobs_admitted"] == 1 and res["jobs_finished"] == 0
    assert res["step_latency_ms_p50"] == pytest.approx(10.0)


class FakeLockstepX:
    """Stand-in for the binding in run_lockstep: records each context's systems and steps."""

    contexts = []

    class Context:
        def __init__(self, p, systems, stream=0):
            self.systems = [s["natoms"] for s in systems]
            self.steps = 0
            self.scf_calls = []
            self.closed = False
            FakeLockstepX.contexts.append(self)

        def scf(self, sys):
            self.scf_calls.append(sys)

        def step(self, n):
            self.steps += n
            time.sleep(0.0002)

        def close(self):
            self.closed = True

    @staticmethod
    def default_params(**kw):
        return kw


def test_lockstep_buckets_by_padded_size_and_steps_every_job():
    # run_lockstep groups jobs by padded orbital count (and temperature), at most max_group per
    # context, builds every context's ground state (scf over all systems) before the MD phase,
    # and steps each context exactly its jobs' step count; every job-step is counted once
    FakeLockstepX.contexts = []
    sizes = [32, 33, 40, 63, 64, 65, 100, 128, 129, 200, 31, 32]
    jobs = [serve.Job(arrival=0.0, jid=i, natoms=n, Te=1000.0, steps=7, seed=i) for i, n in enumerate(sizes)]
    r = serve.run_lockstep(FakeLockstepX, jobs, workers=3, max_group=2)
    assert not r["errors"]
    assert r["steps"] == 7 * len(jobs) and len(r["lat"]) == 7 * len(jobs)
    assert all(j.done_steps == 7 for j in jobs)
    ctxs = FakeLockstepX.contexts
    assert len(ctxs) == r["contexts"]
    for c in ctxs:
        assert c.steps == 7 and c.closed and c.scf_calls == [-1]
        assert len(c.systems) <= 2
        assert len({serve.padded_orbitals(n) for n in c.systems}) == 1
    # every job in exactly one context
    assert sorted(n for c in ctxs for n in c.systems) == sorted(sizes)
    assert r["setup_s"] >= 0 and r["md_s"] > 0

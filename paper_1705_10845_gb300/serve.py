"""Batched and served XL-BOMD on one GPU over the C ABI.

Each job is one trajectory with its own context (device state and CUDA
stream).  Worker threads each own a slice of the active jobs and advance them
one MD step at a time; every C call releases the GIL, so the kernels of
different trajectories overlap on the GPU (continuous batching at the level
of whole steps).  A job is admitted when its estimated device memory fits the
budget; a finished job frees its memory and the next queued job is admitted.

``python -m paper_1705_10845_gb300.serve --mode batch`` advances many
trajectories of uneven size together; ``--mode serve`` feeds Poisson arrivals
through the admission loop and reports per-step latency percentiles and the
aggregate step rate.  Both print one JSON line.
"""
from __future__ import annotations

import argparse
import heapq
import json
import math
import os
import sys
import threading
import time
from dataclasses import dataclass, field

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KB_EV = 8.617333262e-5


def squarings_for(Te: float, width_ev: float = 40.0) -> int:
    """n = max(10, ceil(log2(beta W / 0.1)) - 1) squarings for a spectral width W."""
    beta = 1.0 / (KB_EV * Te)
    return max(10, int(math.ceil(math.log2(beta * width_ev / 0.1))) - 1)


def work_estimate(natoms: int, n_sq: int, steps: int) -> float:
    """Relative device work of a job: the expansion and response products cost n_sq np^3 per
    step; small systems are bound by launch latency (a floor of about a 512-orbital step)."""
    np_ = (4 * natoms + 127) // 128 * 128
    return float(steps) * n_sq * max(np_, 512) ** 3


def stream_priority(natoms: int) -> int:
    """CUDA stream priority by size class (lower is served first): the short kernels of small
    systems are dispatched ahead of the long products of large ones."""
    return -2 if natoms <= 256 else (-1 if natoms <= 1024 else 0)


def bytes_estimate(natoms: int, n_sq: int, prec: str = "fp16x3") -> int:
    """Device memory of one context (expansion matrices dominate)."""
    np_ = (4 * natoms + 127) // 128 * 128
    e = np_ * np_
    if prec == "fp64":
        per = 8 * ((n_sq + 1) + n_sq + 9 + 3)
    else:
        per = 12 * (n_sq + 1) + 8 * n_sq + 8 * 5 + 12 * 4 + 8 * 3
        if prec == "tf32x3":   # TF32 operands: 4 bytes each, 2 more per hi and per lo word
            per += 4 * ((n_sq + 1) + n_sq + 8)
    return int(per * e * 1.05) + (64 << 20)


@dataclass(eq=False)          # jobs compare by identity (list removal, membership)
class Job:
    arrival: float
    jid: int
    natoms: int
    Te: float
    steps: int
    seed: int
    prec: str = "fp16x3"
    # runtime
    ctx: object = None
    stream: object = None
    done_steps: int = 0
    lat: list = field(default_factory=list)
    admitted: float = 0.0
    finished: float = 0.0
    error: str = ""
    mem: int = 0
    result: dict = field(default_factory=dict)


def make_context(X, job: Job, stream_ptr: int):
    import synth
    s = synth.make_system(job.natoms, job.seed)
    n_sq = squarings_for(job.Te)
    p = X.default_params(Te=job.Te, n_sq=n_sq, rank_m=2, dt=0.25, mix_alpha=0.06, kernel_c=1 - 1 / 0.06,
                         prec=job.prec, scf_mode=1, kernel_auto=1, scf_tol=1e-5, scf_max_iter=400,
                         mu_tol=1e-3, rep_A=40.0, rep_rho=0.3, kernel_prec=1, mu_prec=1)
    ctx = X.Context(p, [dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)], stream=stream_ptr)
    ctx.scf(0)
    return ctx


class Scheduler:
    """Admission by device memory plus a worker pool that steps the admitted jobs.

    policy "sjf": among the jobs that have arrived, the one with the least estimated work is
    admitted first (shortest job first, which minimises the mean time in the system of an
    overloaded server); "fifo": in arrival order.
    """

    def __init__(self, X, budget_bytes: int, workers: int, make_ctx=make_context, clock=time.perf_counter,
                 keep_results: bool = False, policy: str = "fifo"):
        if policy not in ("fifo", "sjf"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.policy = policy
        self.X = X
        self.keep_results = keep_results
        self.budget = budget_bytes
        self.used = 0
        self.workers = workers
        self.make_ctx = make_ctx
        self.clock = clock
        self.lock = threading.Lock()
        self.pending: list[tuple] = []        # heap of (arrival, jid, job): not yet arrived
        self.ready: list[tuple] = []          # heap of (key, jid, job): arrived, waiting for memory
        self.active: list[list[Job]] = [[] for _ in range(workers)]
        self.finished: list[Job] = []
        self.rejected: list[Job] = []

    def submit(self, job: Job):
        job.mem = bytes_estimate(job.natoms, squarings_for(job.Te), job.prec)
        with self.lock:
            if job.mem > self.budget:
                job.error = "larger than the memory budget"
                self.rejected.append(job)
                return
            heapq.heappush(self.pending, (job.arrival, job.jid, job))

    def _key(self, job: Job):
        if self.policy == "sjf":
            return (work_estimate(job.natoms, squarings_for(job.Te), job.steps), job.arrival)
        return (job.arrival,)

    def _admit(self, now: float):
        """Reserve memory for the first ready job if it fits the budget."""
        with self.lock:
            while self.pending and self.pending[0][0] <= now:
                _, jid, job = heapq.heappop(self.pending)
                heapq.heappush(self.ready, (self._key(job), jid, job))
            if not self.ready:
                return None
            job = self.ready[0][2]
            if self.used + job.mem > self.budget:
                return None
            heapq.heappop(self.ready)
            self.used += job.mem
            self.peak_used = max(getattr(self, "peak_used", 0), self.used)
            job.admitted = now
        return job

    def _release(self, job: Job):
        with self.lock:
            self.used -= job.mem
            self.finished.append(job)

    def run(self, until: float | None = None, stream_factory=None, admitters: int = 4):
        """Run until every submitted job finished (or the clock passes `until`).

        Admission threads build each job's context (upload and t0 SCF) on the job's own stream
        and hand it to the stepping worker with the least per-step work; stepping workers only
        advance their jobs, so a long SCF never stalls running trajectories.
        """
        t0 = self.clock()
        inbox: list[list[Job]] = [[] for _ in range(self.workers)]
        load = [0.0] * self.workers
        alive = [admitters]

        def timed_out():
            return until is not None and self.clock() - t0 > until

        def step_work(job):
            return work_estimate(job.natoms, squarings_for(job.Te), 1)

        def admitter():
            try:
                while not timed_out():
                    job = self._admit(self.clock() - t0)
                    if job is None:
                        with self.lock:
                            if not self.pending and not self.ready:
                                return
                        time.sleep(0.001)
                        continue
                    try:
                        job.stream = stream_factory(job) if stream_factory else None
                        job.ctx = self.make_ctx(self.X, job, job.stream.cuda_stream if job.stream is not None else 0)
                    except Exception as e:   # admission failure: report and free the reservation
                        job.error = f"job {job.jid} ({job.natoms} atoms, Te {job.Te:.0f} K): {e}"
                        self._release(job)
                        continue
                    with self.lock:
                        w = min(range(self.workers), key=lambda i: load[i])
                        load[w] += step_work(job)
                        inbox[w].append(job)
            finally:
                with self.lock:
                    alive[0] -= 1

        def finish(w, job, mine):
            job.finished = self.clock() - t0
            if self.keep_results and not job.error:
                job.result = {"q": job.ctx.get(0, self.X.Q), "R": job.ctx.get(0, self.X.R)}
            try:
                job.ctx.close()
            except Exception:
                pass
            job.ctx = None
            mine[:] = [j for j in mine if j is not job]
            with self.lock:
                load[w] -= step_work(job)
            self._release(job)

        def worker(w: int):
            mine = self.active[w]
            while not timed_out():
                with self.lock:
                    mine.extend(inbox[w])
                    inbox[w].clear()
                    idle_done = alive[0] == 0
                if not mine:
                    if idle_done:
                        return
                    time.sleep(0.001)
                    continue
                for job in list(mine):
                    t = self.clock()
                    try:
                        job.ctx.step(1)
                    except Exception as e:
                        job.error = f"job {job.jid} ({job.natoms} atoms, Te {job.Te:.0f} K) step {job.done_steps}: {e}"
                    job.lat.append(self.clock() - t)
                    job.done_steps += 1
                    if job.error or job.done_steps >= job.steps:
                        finish(w, job, mine)

        threads = [threading.Thread(target=admitter, daemon=True) for _ in range(admitters)]
        threads += [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(self.workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        wall = self.clock() - t0
        for w in range(self.workers):      # contexts built but never stepped count as admitted
            self.active[w].extend(inbox[w])
            inbox[w].clear()
        for a in self.active:              # jobs still running when the window closed
            for job in a:
                if job.ctx is not None:
                    try:
                        job.ctx.close()
                    except Exception:
                        pass
                    job.ctx = None
        return wall


def padded_orbitals(natoms: int) -> int:
    return (4 * natoms + 127) // 128 * 128


def run_lockstep(X, jobs, workers: int, stream_factory=None, clock=time.perf_counter, max_group: int = 64):
    """Batch of trajectories known up front, stepped in lockstep per size bucket.

    Jobs with the same padded orbital count and temperature share one context (groups of at
    most max_group systems); the library advances a context's systems together, one grouped
    tensor-core launch per product over all of them.  Two phases: every worker first builds
    its bucket contexts and their t0 ground states (SCF), then all workers step their buckets
    round-robin, one MD step per bucket in turn, each worker on its own streams, so buckets
    overlap on the GPU.  Returns a dict: setup and MD wall seconds, job-steps done, per-job-step
    latencies (seconds) and errors."""
    import synth
    buckets = {}
    for j in jobs:
        buckets.setdefault((padded_orbitals(j.natoms), j.Te, j.steps), []).append(j)
    groups = []
    for key in sorted(buckets, key=lambda k: -k[0] ** 3 * len(buckets[k])):
        bj = buckets[key]
        for i in range(0, len(bj), max_group):
            groups.append(bj[i:i + max_group])
    lat, errors = [], []
    done = [0]
    lock = threading.Lock()
    # largest work first, spread over the workers
    queues = [[] for _ in range(workers)]
    load = [0.0] * workers
    for g in groups:
        w = min(range(workers), key=lambda i: load[i])
        queues[w].append(g)
        load[w] += work_estimate(g[0].natoms, squarings_for(g[0].Te), g[0].steps) * len(g)
    ctxs = [[] for _ in range(workers)]
    barrier = threading.Barrier(workers + 1)

    def worker(w):
        for g in queues[w]:
            try:
                stream = stream_factory(g[0]) if stream_factory else None
                n_sq = squarings_for(g[0].Te)
                p = X.default_params(Te=g[0].Te, n_sq=n_sq, rank_m=2, dt=0.25, mix_alpha=0.06,
                                     kernel_c=1 - 1 / 0.06, prec=g[0].prec, scf_mode=1, kernel_auto=1,
                                     scf_tol=1e-5, scf_max_iter=400, mu_tol=1e-3, rep_A=40.0, rep_rho=0.3,
                                     kernel_prec=1, mu_prec=1)
                systems = []
                for j in g:
                    sy = synth.make_system(j.natoms, j.seed)
                    systems.append(dict(natoms=sy.natoms, L=sy.L, R=sy.R, V=sy.V, Z=sy.Z, mass=sy.mass))
                ctx = X.Context(p, systems, stream=stream.cuda_stream if stream is not None else 0)
                ctx.scf(-1)
                ctxs[w].append((g, ctx, stream))
            except Exception as e:      # report and go on with the next bucket
                with lock:
                    errors.append(f"bucket of {len(g)} x {g[0].natoms}-ish atoms (set-up): {e}")
        barrier.wait()                  # every context built: the MD phase starts together
        barrier.wait()
        live = list(ctxs[w])
        while live:
            for item in list(live):
                g, ctx, _ = item
                try:
                    t = clock()
                    ctx.step(1)
                    dt = clock() - t
                    with lock:
                        lat.extend([dt] * len(g))
                        done[0] += len(g)
                    for j in g:
                        j.done_steps += 1
                    if g[0].done_steps >= g[0].steps:
                        live.remove(item)
                        ctx.close()
                except Exception as e:
                    with lock:
                        errors.append(f"bucket of {len(g)} x {g[0].natoms}-ish atoms: {e}")
                    live.remove(item)
                    ctx.close()

    threads = [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(workers)]
    t0 = clock()
    for t in threads:
        t.start()
    barrier.wait()
    t1 = clock()
    barrier.wait()
    for t in threads:
        t.join()
    t2 = clock()
    return {"setup_s": t1 - t0, "md_s": t2 - t1, "steps": done[0], "lat": lat, "errors": errors,
            "contexts": len(groups)}


def summarize(sched: Scheduler, wall: float):
    """Throughput and per-step latency over every admitted job (finished or still running)."""
    admitted = list(sched.finished) + [j for a in sched.active for j in a]
    lat = [x for j in admitted for x in j.lat]
    steps = sum(j.done_steps for j in admitted)
    out = {"steps_per_s": steps / wall if wall > 0 else None, "total_steps": steps, "wall_s": wall,
           "atom_steps_per_s": sum(j.done_steps * j.natoms for j in admitted) / wall if wall > 0 else None,
           "jobs_admitted": len(admitted),
           "jobs_finished": sum(1 for j in sched.finished if not j.error and j.done_steps >= j.steps),
           "jobs_failed": [j.error for j in sched.finished if j.error][:5],
           "jobs_pending": len(sched.pending) + len(sched.ready), "jobs_rejected": len(sched.rejected)}
    if lat:
        a = np.array(lat) * 1000.0
        out.update({"step_latency_ms_p50": float(np.percentile(a, 50)),
                    "step_latency_ms_p99": float(np.percentile(a, 99))})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["batch", "serve"], default="batch")
    ap.add_argument("--jobs", type=int, default=256)
    ap.add_argument("--min-atoms", type=int, default=32)
    ap.add_argument("--max-atoms", type=int, default=512)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--rate", type=float, default=20.0, help="serve: Poisson arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: arrival window (s)")
    ap.add_argument("--budget-gb", type=float, default=None)
    ap.add_argument("--prec", default="fp16x3")
    ap.add_argument("--seed", type=int, default=1705)
    ap.add_argument("--policy", choices=["sjf", "fifo"], default="sjf", help="admission order of arrived jobs")
    ap.add_argument("--no-priority", action="store_true", help="all streams at the default priority")
    ap.add_argument("--lockstep", action="store_true",
                    help="batch mode: step the trajectories of each size bucket together in one context "
                         "(grouped launches) instead of one context and stream per trajectory")
    a = ap.parse_args(argv)

    sys.path.insert(0, ROOT)
    import torch

    import paper_1705_10845_gb300 as X
    X.build.build()
    X.load()
    free, _ = torch.cuda.mem_get_info()
    budget = int(a.budget_gb * 2**30) if a.budget_gb else int(free * 0.85)
    rng = np.random.default_rng(a.seed)
    sched = Scheduler(X, budget, a.workers, policy=a.policy)
    t = 0.0
    for i in range(a.jobs):
        nat = int(round(math.exp(rng.uniform(math.log(a.min_atoms), math.log(a.max_atoms)))))
        if a.mode == "serve":
            t += rng.exponential(1.0 / a.rate)
            if t > a.duration:
                break
            Te = float(rng.uniform(300.0, 3000.0))
        else:
            Te = 1000.0
        sched.submit(Job(arrival=t if a.mode == "serve" else 0.0, jid=i, natoms=nat, Te=Te, steps=a.steps,
                         seed=a.seed + i, prec=a.prec))
    if a.mode == "batch" and a.lockstep:
        jobs = [j for _, _, j in sorted(sched.pending)]
        l0 = X.binding.launch_count()
        r = run_lockstep(
            X, jobs, min(a.workers, 8),
            stream_factory=lambda job: torch.cuda.Stream(priority=0 if a.no_priority else stream_priority(job.natoms)))
        torch.cuda.synchronize()
        steps, errors, lat = r["steps"], r["errors"], r["lat"]
        res = {"steps_per_s": steps / r["md_s"], "total_steps": steps, "md_s": r["md_s"], "setup_s": r["setup_s"],
               "steps_per_s_with_setup": steps / (r["md_s"] + r["setup_s"]),
               "atom_steps_per_s": sum(j.done_steps * j.natoms for j in jobs) / r["md_s"],
               "jobs": len(jobs), "contexts": r["contexts"],
               "jobs_finished": sum(1 for j in jobs if j.done_steps >= j.steps),
               "errors": errors[:5], "mode": "batch-lockstep", "prec": a.prec,
               "atoms_range": [a.min_atoms, a.max_atoms], "steps_per_job": a.steps,
               "gpu_launches": X.binding.launch_count() - l0}
        if lat:
            arr = np.array(lat) * 1000.0
            res.update({"step_latency_ms_p50": float(np.percentile(arr, 50)),
                        "step_latency_ms_p99": float(np.percentile(arr, 99))})
        print(json.dumps(res), flush=True)
        return 1 if errors else 0
    l0 = X.binding.launch_count()
    wall = sched.run(until=(a.duration + 60.0) if a.mode == "serve" else None,
                     stream_factory=lambda job: torch.cuda.Stream(
                         priority=0 if a.no_priority else stream_priority(job.natoms)))
    sync_error = ""
    try:
        torch.cuda.synchronize()
    except Exception as e:           # report the jobs' own errors with it
        sync_error = str(e).splitlines()[0]
    res = summarize(sched, wall)
    if sync_error:
        res["sync_error"] = sync_error
    res.update({"mode": a.mode, "policy": a.policy, "stream_priority": not a.no_priority, "workers": a.workers,
                "prec": a.prec, "budget_gb": budget / 2**30,
                "atoms_range": [a.min_atoms, a.max_atoms], "steps_per_job": a.steps,
                "gpu_launches": X.binding.launch_count() - l0})
    print(json.dumps(res), flush=True)
    return 1 if sync_error else 0


if __name__ == "__main__":
    sys.exit(main())

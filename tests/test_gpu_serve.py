"""Served trajectories: a job gives the same result alone and in a mix of
concurrently stepped jobs (GPU, through the C ABI on separate streams)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run(X, jobs, workers):
    import torch
    from paper_1705_10845_gb300 import serve
    sch = serve.Scheduler(X, 10**12, workers=workers, keep_results=True)
    for j in jobs:
        sch.submit(j)
    sch.run(stream_factory=lambda job: torch.cuda.Stream(priority=serve.stream_priority(job.natoms)))
    torch.cuda.synchronize()
    return {j.jid: j for j in sch.finished}


def test_job_result_is_the_same_alone_and_in_the_mix():
    import paper_1705_10845_gb300 as X
    from paper_1705_10845_gb300 import serve
    X.build.build()
    X.load()
    mk = lambda jid, nat, Te, seed: serve.Job(arrival=0.0, jid=jid, natoms=nat, Te=Te, steps=8, seed=seed)
    alone = run(X, [mk(0, 40, 1000.0, 5)], workers=1)
    mix = run(X, [mk(0, 40, 1000.0, 5), mk(1, 64, 2000.0, 6), mk(2, 96, 500.0, 7), mk(3, 33, 1500.0, 8)],
              workers=4)
    a, b = alone[0], mix[0]
    assert not a.error and not b.error and a.done_steps == b.done_steps == 8
    assert all(not j.error for j in mix.values())
    # the same kernels on the same data in the same order: identical to rounding
    assert np.max(np.abs(a.result["q"] - b.result["q"])) < 1e-12
    assert np.max(np.abs(a.result["R"] - b.result["R"])) < 1e-12

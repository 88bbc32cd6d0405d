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


def test_lockstep_batch_equals_solo_runs():
    # A context holding several trajectories steps those of one padded size in lockstep: each
    # product of the expansion and of the response chains is one grouped launch over the
    # systems (per-system tensor maps from a device table), each element-wise operation one
    # launch, one host synchronisation per mu pass and per probe index for all of them.  Every
    # trajectory must end exactly where its own one-system run ends (the same kernels compute
    # every tile and element the same way): 4 systems share 256 padded orbitals (49-64 atoms),
    # a fifth (100 atoms, 512 orbitals) steps alone.
    import paper_1705_10845_gb300 as X
    import synth
    X.build.build()
    X.load()
    sizes = [(64, 21), (49, 22), (57, 23), (60, 24), (100, 25)]
    systems = []
    for nat, seed in sizes:
        s = synth.make_system(nat, seed)
        systems.append(dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass))
    for prec in ("fp16x3", "tf32x3", "fp64"):
        p = X.default_params(Te=1000.0, n_sq=10, rank_m=2, mix_alpha=0.06, kernel_c=1 - 1 / 0.06, prec=prec,
                             scf_mode=1, kernel_auto=1, scf_tol=1e-5 if prec != "fp64" else 1e-9,
                             mu_tol=1e-3 if prec != "fp64" else 1e-9, rep_A=40.0, rep_rho=0.3, kernel_prec=1,
                             mu_prec=1, scf_max_iter=300)
        solo = []
        for sd in systems:
            with X.Context(p, [sd]) as ctx:
                ctx.scf(0)
                ctx.step(6)
                solo.append([ctx.get(0, w) for w in (X.Q, X.R, X.NHIST, X.KR, X.F, X.MU)])
        with X.Context(p, systems) as ctx:
            ctx.scf(-1)
            ctx.step(6)
            for i in range(len(systems)):
                got = [ctx.get(i, w) for w in (X.Q, X.R, X.NHIST, X.KR, X.F, X.MU)]
                for a, b in zip(solo[i], got):
                    assert np.array_equal(a, b), (prec, i, float(np.max(np.abs(a - b))))

#!/usr/bin/env python
"""Benchmark of the XL-BOMD hot path on GB300.

Workload (default): the precision workload -- one trajectory of 4096
carbon-like atoms (N = 16384 orbitals) in a 38.8 A periodic cube, Te = 1000 K,
10 squarings of the recursive Fermi-operator expansion, rank-4 kernel,
dt = 0.25 fs; split FP16x3 tensor-core products in the expansion (one 16-bit
product in the probe and chemical-potential chains) with FP32 accumulation and
FP64 traces, charges, forces and integration (--prec bf16x3, tf32x3 or fp64 selects
another form).  A step is one full XL-BOMD step
(H build, expansion with the chemical-potential loop, charges, forces, four
response chains, kernel update, Verlet).  With --gpus N each rank runs its own
replica trajectory (seed 1705 + rank): weak scaling, no collective on the data
path.

Beside the timed steps the line carries: the plain-FP64 GPU path's step rate
(bounded from above by one timed FP64 product of the same size times the
step's product count), charge, force and energy parity against one FP64 oracle
step at the final state, and that oracle step's time on the host cores (the
CPU baseline).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead (one full oracle step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "XL-BOMD steps/s and FOE TFLOP/s vs peak, mixed vs FP64 GPU at |dq|<=1e-5 e"
ALPHA_MIX = 0.06
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense tensor rates of GB300 (PFLOP/s): tf32 1.1, bf16 2.25
# DRAM bytes (read + write) per launch of the product kernel, averaged over the launches of one
# MD step, keyed by (variant, padded orbital count), from the ncu captures summarised in profiles/;
# a workload or kernel without a capture since the kernel last changed reports null
GEMM_TRAFFIC = {("persistent", 16384): 3450.66e9 / 233}   # xlbomd_step_4096atoms_fp16x3_launches.md


def gemm_variant():
    v = os.environ.get("XLBOMD_GEMM", "")
    return v if v in ("classic", "pair") else "persistent"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp16x3", choices=["fp16x3", "bf16x3", "tf32x3", "fp64"])
    ap.add_argument("--natoms", type=int, default=4096)
    ap.add_argument("--Te", type=float, default=1000.0)
    ap.add_argument("--nsq", type=int, default=10)
    ap.add_argument("--rank", type=int, default=4)
    ap.add_argument("--kernel-prec", type=int, default=1, choices=[0, 1],
                    help="1 (default): the kernel's probe chains take one hi*hi product instead of three; "
                         "0: three, as the expansion")
    ap.add_argument("--mu-prec", type=int, default=1, choices=[0, 1],
                    help="1 (default): the chemical-potential chain (dD/dmu) takes one hi*hi product instead "
                         "of three; 0: three, as the expansion")
    ap.add_argument("--rep-A", type=float, default=40.0,
                    help="pair repulsion A exp(-r/0.3 A) (eV): the model's atoms collapse without it in long runs")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=0,
                    help="also time this many plain-FP64 GPU steps of the same workload (minutes per step at "
                         "the default size)")
    ap.add_argument("--no-fp64-product", action="store_true",
                    help="skip the timed FP64 product that bounds the plain-FP64 GPU step rate")
    ap.add_argument("--trajectory-check", type=int, default=0, metavar="K",
                    help="study run instead of the timing: --steps MD steps after the t0 SCF, the energy "
                         "monitor every --energy-every steps, and every K steps the oracle re-evaluates q, "
                         "F and Omega at the GPU's (R, n); prints one JSON line")
    ap.add_argument("--energy-every", type=int, default=10)
    ap.add_argument("--precision-study", default="",
                    help="comma-separated precisions (e.g. fp16x3,bf16x3,tf32x3): at the t0 state of the first, "
                         "each evaluates q, F and Omega against one oracle evaluation of the same (R, n), "
                         "then times --steps MD steps; prints one JSON line")
    ap.add_argument("--batch", action="store_true",
                    help="batch workload instead: --batch-jobs trajectories of 32-512 atoms (log-uniform, "
                         "seeded), Te = 1000 K, --batch-steps steps each, stepped in lockstep per size bucket "
                         "(grouped launches); prints one JSON line with the aggregate step rate and the "
                         "per-step latency percentiles")
    ap.add_argument("--batch-jobs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling run: t0 SCF, --warmup steps, then one step inside the NVTX range "
                         "'xlbomd_step'; prints no JSON")
    return ap.parse_args()


def chain_products(a, single):
    """Products per step of a response chain: one hi*hi product of the operand format, three (the
    full split), or the plain FP64 product."""
    if a.prec == "fp64":
        return "one fp64 product"
    return f"one {a.prec[:4]} product" if single else "three (full split)"


def workload_config(a, parallel):
    return {
        "workload": f"XL-BOMD, {a.natoms} carbon-like atoms (N = {4 * a.natoms} orbitals), orthogonal SCC-TB, "
                    f"Te = {a.Te:g} K, {a.nsq} squarings, rank-{a.rank} kernel, dt = 0.25 fs",
        "natoms": a.natoms, "n_orb": 4 * a.natoms, "Te_K": a.Te, "n_squarings": a.nsq, "rank_m": a.rank,
        "pair_repulsion": f"{a.rep_A:g} exp(-r/0.3 A) eV" if a.rep_A else "off",
        "kernel_probe_products": chain_products(a, a.kernel_prec),
        "mu_chain_products": chain_products(a, a.mu_prec),
        "prec": a.prec, "parallelism": parallel,
        "l2": f"inputs larger than L2: about {expansion_bytes(a) / 1e9:.0f} GB of expansion matrices are "
              f"rewritten every step",
    }


def expansion_bytes(a) -> float:
    """Device bytes of the split engine's matrices for this workload (the per-context estimate the
    serving loop admits by)."""
    from paper_1705_10845_gb300.serve import bytes_estimate
    return float(bytes_estimate(a.natoms, a.nsq, a.prec))


def replica_seed(rank: int) -> int:
    """Each rank runs its own replica trajectory (weak scaling)."""
    return 1705 + rank


def max_over_ranks(x: float, dist, device: str) -> float:
    """Largest x over the ranks (the slowest replica sets the job's time); x itself without a
    process group.  The only collective of a run: timing, never data."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), d.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 1900.0, 1700.0, 6800.0, "fallback"


def single_product_chains(a):
    chains = [c for c, on in (("probe", a.kernel_prec), ("mu", a.mu_prec)) if on]
    return f"1 in the {' and '.join(chains)} chains" if chains else "3 in every chain"


def dtype_label(a):
    """The products' arithmetic: FP64, or the split (three products of the operand format per split
    product) with the chains that take one hi*hi product named."""
    if a.prec == "fp64":
        return "f64"
    base = a.prec[:4]
    single = [c for c, on in (("probe", a.kernel_prec), ("mu", a.mu_prec)) if on]
    chains = f", {base} x1 in the {' and '.join(single)} chains" if single else ""
    return f"{a.prec} expansion{chains}; fp32 accumulate; f64 traces, charges, forces, integration"


def make_params(X, a, prec):
    return X.default_params(Te=a.Te, n_sq=a.nsq, rank_m=a.rank, dt=0.25, mix_alpha=ALPHA_MIX,
                            rep_A=a.rep_A, rep_rho=0.3, kernel_prec=a.kernel_prec, mu_prec=a.mu_prec,
                            kernel_c=1.0 - 1.0 / ALPHA_MIX, prec=prec,
                            scf_tol=1e-10 if prec == "fp64" else 1e-5, scf_mode=1, kernel_auto=1,
                            mu_tol=1e-9 if prec == "fp64" else 1e-3, scf_max_iter=200)


def oracle_model(a):
    import oracle as O
    return O.Model(Te=a.Te, n_sq=a.nsq, rep_A=a.rep_A, rep_rho=0.3)


ORACLE_STEP = ("one full XL-BOMD step of the FP64 oracle (oracle.md_step) on the whole system: half kick, "
               "drift, n update, then at the new state H0, Ewald gamma, full eigendecomposition, chemical "
               "potential, Mulliken charges, Hellmann-Feynman forces, the free energy and the rank-{m} kernel's "
               "{m} probe responses (eigenbasis divided differences), and the second half kick")


def oracle_step(st, L, Z, mass, a, kernel_c):
    """One XL-BOMD step of the FP64 oracle from the MD state st (R, V, n history, F and K r at t;
    Eqs. Integration, VRL_Damp).  Returns (seconds, new state, evaluation at the new state)."""
    import oracle as O
    xl = O.XLParams(rank_m=a.rank, kernel_c=kernel_c, dt=0.25)
    t = time.perf_counter()
    st1, ev = O.md_step(st, L, Z, mass, oracle_model(a), xl)
    return time.perf_counter() - t, st1, ev


def run_reference(a, ws, rank):
    """The oracle as it stands on the host cores (FP64 CPU), same workload: full oracle MD steps
    from the seeded initial positions and velocities."""
    import numpy as np

    import oracle as O
    import synth
    if ws > 1 and rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    s = synth.make_system(a.natoms, 1705)
    nat = s.natoms
    # MD state at t: the seeded R, V; n history at zero charges with F = 0, K r = 0 at t (the
    # cost of a step does not depend on these values)
    st = O.MDState(R=np.array(s.R), V=np.array(s.V), nhist=np.zeros((6, nat)), F=np.zeros((nat, 3)),
                   Kr=np.zeros(nat))
    # the first step doubles as the warm-up; a step of more than 30 s is itself the timed sample
    # so that the run ends within minutes (one step at 4096 atoms takes minutes on 16 cores)
    t_first, st, _ = oracle_step(st, s.L, s.Z, s.mass, a, 1.0 - 1.0 / ALPHA_MIX)
    times = [t_first]
    warm = 1
    if t_first < 30.0:
        times = []
        budget = 150.0
        k = max(1, min(a.steps, int(budget / max(t_first, 1e-3))))
        for _ in range(k):
            dt, st, _ = oracle_step(st, s.L, s.Z, s.mass, a, 1.0 - 1.0 / ALPHA_MIX)
            times.append(dt)
    else:
        warm = 0
    sec = sum(times)
    v = len(times) / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": a.gpus,
            "steps": len(times), "warmup": warm, "ms_per_step": 1000.0 * sec / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(a, "oracle on host cores"),
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": ORACLE_STEP.format(m=a.rank) + "; from the seeded initial positions "
                                       "and velocities at zero charges (the GPU arm steps from its t0 ground "
                                       "state; the work per step is the same)" +
                                       ("" if warm else "; one step of several minutes is the whole timed "
                                        "sample, without a separate warm-up step")},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_trajectory_study(a, X, ctx, s):
    """State-wise parity along one trajectory: the MD diverges chaotically from any other
    run, so at every K-th step the oracle evaluates the GPU's own (R, n) state."""
    import numpy as np
    import oracle as O
    m = O.Model(Te=a.Te, n_sq=a.nsq, rep_A=a.rep_A, rep_rho=0.3)
    t = time.perf_counter()
    ctx.scf(0)
    t_scf = time.perf_counter() - t
    E, checks = [], []
    t_md = 0.0
    for k in range(1, a.steps + 1):
        t = time.perf_counter()
        ctx.step(1)
        t_md += time.perf_counter() - t
        if k % a.energy_every == 0 or k % a.trajectory_check == 0:
            ctx.energy(0)
            E.append((k, float(ctx.get(0, X.ENERGY)[5])))
        if k % a.trajectory_check == 0:
            R, n = ctx.get(0, X.R), ctx.get(0, X.N)
            q, F, Om = ctx.get(0, X.Q), ctx.get(0, X.F), float(ctx.get(0, X.ENERGY)[0])
            t = time.perf_counter()
            ev = O.evaluate(R, s.L, s.Z, n, m, None, with_kernel=False)
            checks.append({"step": k, "dq": float(np.abs(q - ev.q).max()), "dF": float(np.abs(F - ev.F).max()),
                           "dOmega": Om - ev.Omega, "rms_residual": float(np.sqrt(np.mean((ev.q - n) ** 2))),
                           "oracle_s": time.perf_counter() - t})
            print(json.dumps({"check": checks[-1]}), file=sys.stderr, flush=True)
    steps_e = np.array([e[0] for e in E], dtype=float)
    Etot = np.array([e[1] for e in E])
    slope = float(np.polyfit(steps_e * 0.25e-3, Etot, 1)[0]) if len(E) > 1 else None   # eV / ps
    out = {"study": "trajectory state-wise parity", "natoms": s.natoms, "prec": a.prec, "Te": a.Te,
           "n_sq": a.nsq, "rank_m": a.rank, "steps": a.steps, "dt_fs": 0.25, "scf_s": t_scf,
           "md_steps_per_s": a.steps / t_md, "checks": checks,
           "max_dq": max(c["dq"] for c in checks), "max_dF": max(c["dF"] for c in checks),
           "max_abs_dOmega": max(abs(c["dOmega"]) for c in checks),
           "energy_samples": len(E), "Etot_first": float(Etot[0]), "Etot_max_dev": float(np.abs(Etot - Etot[0]).max()),
           "Etot_drift_eV_per_ps": slope}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def run_precision_study(a, X, ctx, s, sysd, stream):
    """Error of each split precision against the FP64 oracle at one shared state, and its
    MD step rate."""
    import numpy as np
    import torch
    import oracle as O
    precs = [x for x in a.precision_study.split(",") if x]
    t = time.perf_counter()
    ctx.scf(0)
    t_scf = time.perf_counter() - t
    R, n, mu = ctx.get(0, X.R), ctx.get(0, X.N), float(ctx.get(0, X.MU)[0])
    ctx.close()
    sysd = dict(sysd, R=R)
    rows = []
    for prec in precs:
        c = X.Context(make_params(X, a, prec), [sysd], stream=stream.cuda_stream)
        c.set(0, X.N, n)
        c.set(0, X.MU, [mu])
        c.build_H(0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        c.density(0)
        torch.cuda.synchronize()
        t_dens = time.perf_counter() - t
        c.energy(0)
        row = {"prec": prec, "q": c.get(0, X.Q), "F": c.get(0, X.F), "Omega": float(c.get(0, X.ENERGY)[0]),
               "density_s": t_dens}
        c.scf(0)                        # own t0 state and automatic c before the timed MD steps
        c.step(1)                       # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        c.step(a.steps)
        torch.cuda.synchronize()
        row["md_steps_per_s"] = a.steps / (time.perf_counter() - t)
        c.close()
        rows.append(row)
    t = time.perf_counter()
    ev = O.evaluate(R, s.L, s.Z, n, O.Model(Te=a.Te, n_sq=a.nsq, rep_A=a.rep_A, rep_rho=0.3), None,
                    with_kernel=False)
    t_or = time.perf_counter() - t
    out = {"study": "precision", "natoms": s.natoms, "n_orbitals": 4 * s.natoms, "Te": a.Te, "n_sq": a.nsq,
           "rank_m": a.rank, "scf_s": t_scf, "oracle_eval_s": t_or, "md_steps_timed": a.steps, "results": []}
    for r in rows:
        out["results"].append({"prec": r["prec"], "max_dq": float(np.abs(r["q"] - ev.q).max()),
                               "max_dF": float(np.abs(r["F"] - ev.F).max()), "dOmega": r["Omega"] - ev.Omega,
                               "density_s": r["density_s"], "md_steps_per_s": r["md_steps_per_s"]})
    print(json.dumps(out), flush=True)
    return 0


def run_batch(a, X, ws, rank, dist):
    """Many independent trajectories of uneven size advanced together (grouped launches per
    size bucket): aggregate MD steps/s over all trajectories and ranks."""
    import math
    import numpy as np
    import torch
    from paper_1705_10845_gb300 import serve
    rng = np.random.default_rng(1705 + 1000 * rank)
    jobs = []
    for i in range(a.batch_jobs):
        nat = int(round(math.exp(rng.uniform(math.log(32), math.log(512)))))
        jobs.append(serve.Job(arrival=0.0, jid=i, natoms=nat, Te=1000.0, steps=a.batch_steps,
                              seed=1705 + 1000 * rank + i, prec=a.prec))
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    l0 = X.binding.launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    r = serve.run_lockstep(
        X, jobs, 8, stream_factory=lambda job: torch.cuda.Stream(priority=serve.stream_priority(job.natoms)))
    torch.cuda.synchronize()
    steps, lat, errors = r["steps"], r["lat"], r["errors"]
    wall = max_over_ranks(r["md_s"], dist, "cuda")
    setup = max_over_ranks(r["setup_s"], dist, "cuda")
    clocks = sampler.stop()
    arr = np.array(lat) * 1000.0 if lat else np.zeros(1)
    line = {"metric": "XL-BOMD batch: aggregate MD steps/s of many trajectories (lockstep per size bucket)",
            "value": job_rate(steps, ws, wall), "unit": "steps/s", "n_gpus": ws, "steps": a.batch_steps,
            "setup_s": setup, "steps_per_s_with_setup": job_rate(steps, ws, wall + setup),
            "contexts": r["contexts"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(a),
            "data": "synthetic",
            "config": {"workload": f"{a.batch_jobs} trajectories, 32-512 carbon-like atoms (log-uniform, seeded), "
                                   f"Te = 1000 K, 10+ squarings, rank-2 kernel, {a.batch_steps} steps each; "
                                   "value: the MD phase (all t0 ground states built first, setup_s)",
                       "parallelism": f"replicas x{ws}"},
            "step_latency_ms_p50": float(np.percentile(arr, 50)), "step_latency_ms_p99": float(np.percentile(arr, 99)),
            "atom_steps_per_s": sum(j.natoms * j.done_steps for j in jobs) * ws / wall,
            "gpu_launches": X.binding.launch_count() - l0, "clocks": clocks, "errors": errors[:5], "wall_s": wall}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 1 if errors else 0


def main():
    a = parse()
    ws, rank, local = dist_setup()
    if a.impl == "reference":
        return run_reference(a, ws, rank)

    import numpy as np
    import torch

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        dist = None
        torch.cuda.set_device(0)

    import paper_1705_10845_gb300 as X
    import synth
    if rank == 0:
        X.build.build()
    if dist is not None:
        dist.barrier()
    X.load()

    if a.batch:
        return run_batch(a, X, ws, rank, dist)

    s = synth.make_system(a.natoms, replica_seed(rank))
    sysd = dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)
    p = make_params(X, a, a.prec)
    stream = torch.cuda.current_stream()
    ctx = X.Context(p, [sysd], stream=stream.cuda_stream)

    if a.trajectory_check > 0:
        return run_trajectory_study(a, X, ctx, s)
    if a.precision_study:
        return run_precision_study(a, X, ctx, s, sysd, stream)

    if a.profile_step:
        ctx.scf(0)
        ctx.step(a.warmup)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("xlbomd_step")
        ctx.step(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ctx.close()
        return 0

    # t0 ground state (untimed), then warm-up steps
    t_scf = time.perf_counter()
    ctx.scf(0)
    torch.cuda.synchronize()
    t_scf = time.perf_counter() - t_scf
    ctx.step(a.warmup)
    torch.cuda.synchronize()

    # ---- timed region: device-resident state ----
    sampler = ClockSampler(local)
    st0 = ctx.get(0, X.STATS)
    l0 = X.binding.launch_count()
    ctx.gemm_profile(1)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    wall = time.perf_counter()
    ctx.step(a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = X.binding.launch_count() - l0
    prof = ctx.gemm_profile(2)
    ctx.gemm_profile(0)
    st1 = ctx.get(0, X.STATS)
    ms = max_over_ranks(ms, dist, "cuda")
    sec = ms / 1000.0
    value = job_rate(a.steps, ws, sec)

    # ---- end to end: host state in, results out, every step ----
    ke = a.e2e_steps if a.e2e_steps is not None else max(1, a.steps // 2)
    nat = a.natoms
    k1 = p.kmax + 1
    pin = lambda n_: torch.empty(n_, dtype=torch.float64, pin_memory=True).numpy()
    hR, hV, hN = pin(3 * nat), pin(3 * nat), pin(k1 * nat)
    hR[:] = ctx.get(0, X.R).ravel()
    hV[:] = ctx.get(0, X.V).ravel()
    hN[:] = ctx.get(0, X.NHIST).ravel()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        ctx.set(0, X.R, hR)
        ctx.set(0, X.V, hV)
        ctx.set(0, X.NHIST, hN)
        ctx.step(1)
        hR[:] = ctx.get(0, X.R).ravel()
        hV[:] = ctx.get(0, X.V).ravel()
        hN[:] = ctx.get(0, X.NHIST).ravel()
        q_host = ctx.get(0, X.Q)
        f_host = ctx.get(0, X.F)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te = max_over_ranks(te, dist, "cuda")
    e2e_value = job_rate(ke, ws, te)
    h2d = 8 * (3 * nat + 3 * nat + k1 * nat)
    d2h = 8 * (3 * nat + 3 * nat + k1 * nat + nat + 3 * nat)

    # ---- plain-FP64 GPU path of the same workload ----
    # One FP64 step at this size takes tens of minutes, so by default one timed FP64 product of the
    # same size bounds it: the FP64 path runs at least the mixed step's dense-equivalent product
    # count (its Newton-Schulz inverses take as many or more iterations, and its A1 takes the same
    # work), so products x product time is a lower bound on its step time and the rate below an
    # upper bound on its step rate.  --fp64-steps K times K real FP64 steps instead.
    fp64 = None
    per_step_products = (st1[3] - st0[3]) / a.steps
    np_pad = (4 * a.natoms + 127) // 128 * 128
    if a.fp64_steps > 0:
        p64 = make_params(X, a, "fp64")
        sysd64 = dict(sysd)
        sysd64["R"] = ctx.get(0, X.R)
        sysd64["V"] = ctx.get(0, X.V)
        ctx64 = X.Context(p64, [sysd64], stream=stream.cuda_stream)
        ctx64.set(0, X.NHIST, ctx.get(0, X.NHIST))
        ctx64.set(0, X.MU, ctx.get(0, X.MU))
        ctx64.build_H(0)
        ctx64.density(0)
        ctx64.kernel_update(0)
        torch.cuda.synchronize()
        f0 = time.perf_counter()
        ctx64.step(a.fp64_steps)
        torch.cuda.synchronize()
        f64s = time.perf_counter() - f0
        fp64 = {"kind": "measured FP64 GPU steps", "steps": a.fp64_steps, "steps_per_s": a.fp64_steps / f64s,
                "s_per_step": f64s / a.fp64_steps}
        ctx64.close()
    elif not a.no_fp64_product:
        _, _, ms64 = X.binding.selftest_gemm(np_pad, "fp64", False)
        s64 = per_step_products * ms64 / 1000.0
        fp64 = {"kind": "bound: one timed FP64 product (n = %d, plain-FP64 path kernel) x the mixed step's "
                        "dense-equivalent product count; the FP64 path runs at least as many, so this is an "
                        "upper bound on its step rate" % np_pad,
                "product_ms": ms64, "product_tflops": 2.0 * np_pad ** 3 / (ms64 / 1000.0) / 1e12,
                "products_per_step": per_step_products, "s_per_step": s64, "steps_per_s": 1.0 / s64,
                "mixed_over_fp64": value / (1.0 / s64)}

    # ---- parity and the CPU baseline (rank 0): one more step on both sides from the same state ----
    # The GPU's state at t (R, V, n history, F, K r) goes to the FP64 oracle, which takes one full
    # step from it (oracle.md_step); the GPU takes the same step.  The Verlet updates are FP64 on
    # both sides, so R and n at t + dt agree to rounding and the oracle's q, F and Omega there are
    # the reference for the GPU's (the trajectory itself is chaotic, so parity is state-wise).
    cpu = None
    parity = None
    if rank == 0 and not a.no_cpu_baseline:
        import oracle as O
        st_t = O.MDState(R=ctx.get(0, X.R), V=ctx.get(0, X.V), nhist=ctx.get(0, X.NHIST), F=ctx.get(0, X.F),
                         Kr=ctx.get(0, X.KR))
        ctx.step(1)
        ctx.energy(0)
        qg, Fg, Rg, ng = ctx.get(0, X.Q), ctx.get(0, X.F), ctx.get(0, X.R), ctx.get(0, X.N)
        Eg = ctx.get(0, X.ENERGY)
        tcpu, st_o, ev = oracle_step(st_t, s.L, s.Z, s.mass, a, 1.0 - 1.0 / ALPHA_MIX)
        cpu = {"value": 1.0 / tcpu, "unit": "steps/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": ORACLE_STEP.format(m=a.rank) + ", from the GPU's state after the timed steps"}
        parity = {"max_abs_dq": float(np.max(np.abs(qg - ev.q))), "tol_q": 1e-5,
                  "max_abs_dF": float(np.max(np.abs(Fg - ev.F))), "tol_F": 1e-4,
                  "dOmega_eV": float(Eg[0] - ev.Omega), "Omega_eV": float(ev.Omega),
                  "max_abs_dR": float(np.max(np.abs(O.min_image(Rg - st_o.R, s.L)))),
                  "max_abs_dn": float(np.max(np.abs(ng - st_o.nhist[0]))),
                  "against": "FP64 oracle step from the GPU's state (q, F, Omega at t + dt)"}

    bf, bf_sus, hbm, src = peaks()
    gemm_launches, gemm_ms, gemm_flops = prof
    achieved = gemm_flops / (gemm_ms / 1000.0) / 1e12 if gemm_ms > 0 else None
    peak, peak_of = bf_sus, f"{src} sustained bf16"
    if a.prec == "tf32x3":   # kind::tf32 runs at the nominal dense TF32/BF16 ratio of the bf16 peak
        peak, peak_of = bf_sus * TF32_PER_BF16, f"{src} sustained bf16 x {TF32_PER_BF16:.3f} (nominal dense tf32/bf16)"
    units = st1 - st0
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(a), "data": "synthetic", "config": workload_config(a, f"replicas x{ws}"),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": GEMM_TRAFFIC.get((gemm_variant(), np_pad)) if a.prec == "fp16x3" else None,
                     "traffic_note": "DRAM bytes per product launch (ncu dram__bytes_read + write), averaged "
                                     "over one step's launches; null where no capture of the current kernel "
                                     "at this size exists",
                     "kernel": f"gemm_tc {gemm_variant()} kernel (split-precision tcgen05 product)",
                     "note": f"algorithmic 2n^3 per product (n^3 when symmetric-output) over CUDA-event time of "
                             f"{int(gemm_launches)} launches; each split product runs 3 {a.prec[:4]} "
                             f"tensor products ({single_product_chains(a)}), "
                             f"so tensor-pipe work is up to 3x the algorithmic flops; peak = {peak_of}"},
        "foe_tflops": (gemm_flops / sec / 1e12) if sec > 0 else None,
        "gemm_time_share": (gemm_ms / ms) if ms > 0 else None,
        "per_step": {"mu_passes": units[0] / a.steps, "products": units[3] / a.steps,
                     "probes": float(st1[2])},
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "parity": parity,
        "fp64_gpu": fp64,
        "init_scf_s": t_scf,
        "wall_s": wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""GPU checks of the split-precision tensor-core path (tcgen05, FP16x3/BF16x3/TF32x3).

The product engine is checked against the FP64 product; the density, charges,
forces and kernel against the oracle.  Tolerances of the mixed forms: charges
1e-5 e, forces 1e-4 eV/A.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

ALPHA_MIX = 0.06


@pytest.fixture(scope="module")
def X():
    import paper_1705_10845_gb300 as X
    X.build.build()
    X.load()
    return X


def sysdict(s):
    return dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)


@pytest.mark.parametrize("n", [128, 256, 384, 1024, 2944, 4096, 8192])
@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("prec,bound", [("fp16x3", 1e-6), ("bf16x3", 2e-5), ("tf32x3", 1e-6)])
def test_tensor_core_product_matches_fp64(X, n, sym, prec, bound):
    err, flag, ms = X.binding.selftest_gemm(n, prec, sym)
    assert flag == 0
    # entries are sums of n products of U(-1, 1) numbers; the tensor-core FP32
    # accumulation loses up to ~2^-23 of the running sum per step, so the
    # error bound grows linearly with n (a wrong operand layout gives O(1)).
    print(prec, n, sym, err, ms)
    assert err < bound * n, (err, ms)


@pytest.mark.parametrize("n", [256, 384, 1024, 4096, 8192])
@pytest.mark.parametrize("prec,bound", [("fp16x3", 1e-6), ("bf16x3", 2e-5), ("tf32x3", 1e-6)])
def test_pair_product_matches_fp64(X, n, prec, bound):
    # C = A B^T + B A^T as one symmetric-output product over two K ranges (the
    # A1 = T T1 + T1 T of the response chains); twice the sums of one product
    err, flag, ms = X.binding.selftest_gemm(n, prec, 2)
    print(prec, n, "pair", err, ms)
    assert flag == 0
    assert err < 2 * bound * n, (err, ms)


@pytest.mark.parametrize("n", [384, 2944, 4096, 6144, 8192])
@pytest.mark.parametrize("sym", [0, 1, 2])
@pytest.mark.parametrize("prec,u", [("fp16x3", 2.0 ** -11), ("bf16x3", 2.0 ** -8), ("tf32x3", 2.0 ** -11)])
def test_single_product_matches_fp64(X, n, sym, prec, u):
    # one product of the hi operands (FP16 and TF32 keep 11 significant bits, BF16 8), the
    # product of the single-product chains; below
    # n = 8192 consecutive tiles of a CTA alternate between the two TMEM accumulators, at
    # n = 8192 the hi*hi sum splits over both.  Each operand carries a relative rounding error of
    # at most u, so an entry's error is a sum of n terms a db + b da with standard deviation about
    # u sqrt(2 n / 27) for U(-1, 1) inputs; the bound is 8 of those (twice that for the pair
    # product), far below the O(sqrt(n)) error of a wrong tile or accumulator
    err, flag, ms = X.binding.selftest_gemm(n, prec, sym if sym != 2 else 2, single=True)
    bound = 8.0 * u * np.sqrt(2.0 * n / 27.0) * (2.0 if sym == 2 else 1.0)
    print(prec, n, "single", sym, err, bound, ms)
    assert flag == 0
    assert err < bound, (err, bound, ms)


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("case", ["tiny24", "ragged37"])
@pytest.mark.parametrize("mu_prec", [0, 1])
def test_split_density_against_oracle(X, prec, case, mu_prec):
    # mu_prec = 1: the chemical-potential chain at one hi*hi product (the mu start is 0.01 eV
    # off, so the Newton steps and the first-order correction both use it)
    s = synth.make_system(24, 1705, L=7.0) if case == "tiny24" else synth.make_system(37, 11)
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, prec=prec, mu_tol=1e-3,
                         mu_prec=mu_prec)
    m = O.Model(Te=p.Te, n_sq=p.n_sq)
    rng = np.random.default_rng(2)
    n = rng.normal(scale=0.02, size=s.natoms)
    n -= n.mean()
    xl = O.XLParams(rank_m=p.rank_m, kernel_c=p.kernel_c)
    ref = O.evaluate(s.R, s.L, s.Z, n, m, xl)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ref.dens.mu + 0.01])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_update(0)
        ctx.energy(0)
        q, F, Kr = ctx.get(0, X.Q), ctx.get(0, X.F), ctx.get(0, X.KR)
        E = ctx.get(0, X.ENERGY)
    # FP16x3 and TF32x3 meet the mixed-precision bounds (1e-5 e, 1e-4 eV/A): both hi/lo pairs
    # keep 22 significant bits.  BF16x3 does not: its pair keeps 16, and its charges measure
    # 1.1-1.4e-5 e here (2-3e-5 e at 1536-2048 atoms), so it is held to its own measured level
    # (3e-5 e) and is not used by the bench, batch or serving workloads
    tol_q = 3e-5 if prec == "bf16x3" else 1e-5
    tol_f = 1e-4
    print(prec, case, "mu_prec", mu_prec, "dq", np.abs(q - ref.q).max(), "dF", np.abs(F - ref.F).max(), "dKr",
          np.abs(Kr - ref.Kr).max())
    assert np.max(np.abs(q - ref.q)) < tol_q
    assert np.max(np.abs(F - ref.F)) < tol_f
    assert np.max(np.abs(Kr - ref.Kr)) < 100 * tol_q
    # energy monitor: Omega and its parts against the oracle (eV)
    print(prec, case, "dOmega", E[0] - ref.Omega, "dS", E[3] - ref.parts["entropy"])
    assert abs(E[3] - ref.parts["entropy"]) < 1e-3
    assert abs(E[0] - ref.Omega) < (2e-2 if prec == "bf16x3" else 2e-3)


@pytest.mark.parametrize("mu_prec", [0, 1])
def test_full_size_charges_against_oracle(X, mu_prec):
    # the bench workload: 1536 atoms (N = 6144), Te = 1500 K, 14 squarings,
    # FP16x3, at the t0 ground state that the MD starts from (kernel SCF with
    # the automatic J_0); the oracle diagonalises H on the host at the same
    # (R, n) and the charges must agree to 1e-5 e, with the mu chain at three
    # products or at one
    s = synth.make_system(1536, 1705)
    p = X.default_params(Te=1500.0, n_sq=14, rank_m=4, mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX,
                         prec="fp16x3", mu_tol=1e-3, scf_mode=1, kernel_auto=1, scf_tol=1e-5,
                         scf_max_iter=200, mu_prec=mu_prec)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.scf(0)
        n = ctx.get(0, X.N)
        ctx.build_H(0)
        ctx.density(0)
        q = ctx.get(0, X.Q)
    q_ref = O.charges_at(s.R, s.L, s.Z, n, O.Model(Te=1500.0, n_sq=14))
    err = np.max(np.abs(q - q_ref))
    print("full size fp16x3 mu_prec", mu_prec, "|dq|", err)
    assert err < 1e-5


@pytest.fixture(scope="module")
def ref2048():
    """The oracle's evaluation of the 2048-atom state (one eigendecomposition for every precision)."""
    s = synth.make_system(2048, 1705)
    m = O.Model(Te=1000.0, n_sq=10, rep_A=40.0, rep_rho=0.3)
    rng = np.random.default_rng(2048)
    n = rng.normal(scale=0.01, size=s.natoms)
    n -= n.mean()
    ref = O.evaluate(s.R, s.L, s.Z, n, m, O.XLParams(rank_m=4, kernel_c=1 - 1 / ALPHA_MIX))
    return s, n, ref


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_accumulator_split_size_against_oracle(X, ref2048, prec):
    # 2048 atoms (N = 8192): the first size whose products split their hi*hi sums over both
    # TMEM accumulators.  At a seeded (R, n) with the Newton search started 5 meV off the
    # oracle's mu (no SCF needed), the split path with the bench's chain precisions (probe and
    # mu chains at one hi*hi product) must match the oracle's eigendecomposition element by
    # element: charges to 1e-5 e, forces to 1e-4 eV/A; Omega and the rank-4 K r are reported
    # against it too.  Te = 1000 K and 10 squarings are the 4096-atom precision workload's.
    s, n, ref = ref2048
    p = X.default_params(Te=1000.0, n_sq=10, rank_m=4, mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX,
                         prec=prec, mu_tol=1e-3, rep_A=40.0, rep_rho=0.3, kernel_prec=1, mu_prec=1)
    with X.Context(p, [sysdict(s)]) as ctx:
        assert ctx.sizes(0)[2] == 8192
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ref.dens.mu + 0.005])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_update(0)
        ctx.energy(0)
        q, F, Kr, E = ctx.get(0, X.Q), ctx.get(0, X.F), ctx.get(0, X.KR), ctx.get(0, X.ENERGY)
    dq, dF = np.abs(q - ref.q).max(), np.abs(F - ref.F).max()
    dK = np.abs(Kr - ref.Kr).max() / np.abs(ref.Kr).max()
    print("2048 atoms", prec, ": |dq|", dq, "|dF|", dF, "dOmega", E[0] - ref.Omega, "K r rel", dK)
    assert dq < 1e-5
    assert dF < 1e-4
    assert abs(E[0] - ref.Omega) < 1e-6 * abs(ref.Omega)
    assert dK < 2e-3


@pytest.mark.parametrize("prec,tol", [("fp16x3", 1e-4), ("bf16x3", 1e-3), ("tf32x3", 1e-4)])
def test_split_exact_kernel_against_oracle(X, prec, tol):
    s = synth.make_system(37, 11)
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, prec=prec, mu_tol=1e-3, kernel_mode=1)
    m = O.Model(Te=p.Te, n_sq=p.n_sq)
    rng = np.random.default_rng(8)
    n = rng.normal(scale=0.02, size=s.natoms)
    n -= n.mean()
    ev = O.evaluate(s.R, s.L, s.Z, n, m, None, with_kernel=False, with_forces=False)
    Kref = O.kernel_exact(ev.dens, ev.gamma)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ev.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_exact(0)
        K = ctx.get(0, X.KMAT)
    err = np.max(np.abs(K - Kref)) / np.abs(Kref).max()
    print(prec, "exact kernel rel err", err)
    assert err < tol


@pytest.mark.parametrize("variant", ["classic", "pair"])
def test_other_product_variants_match_fp64(X, variant):
    # the one-CTA-per-tile product kernel (XLBOMD_GEMM=classic) and the two-SM (cta_group::2)
    # kernel (XLBOMD_GEMM=pair, sizes that are multiples of 256) stay checked next to the default
    # one-SM persistent kernel; a fresh process reads the variant once
    import json
    import os
    import subprocess
    import sys
    code = ("import json, paper_1705_10845_gb300 as X; X.load(); "
            "print(json.dumps([[X.binding.selftest_gemm(n, p, s) for n in (256, 384, 2048) "
            "for p in ('fp16x3', 'bf16x3') for s in (False, True)], "
            "[X.binding.selftest_gemm(8192, 'fp16x3', s) for s in (False, True, 2)], "
            "[X.binding.selftest_gemm(4096, 'fp16x3', s, single=True) for s in (False, True, 2)]]))")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         env=dict(os.environ, XLBOMD_GEMM=variant), timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    res, large, single = json.loads(out.stdout.strip().splitlines()[-1])
    k = 0
    for n in (256, 384, 2048):
        for bound in (1e-6, 2e-5):
            for _sym in (False, True):
                err, flag, ms = res[k]
                k += 1
                assert flag == 0 and err < bound * n, (n, err)
    # n = 8192 split products (dense, symmetric, pair) with the bounds of the default kernel's tests
    for (err, flag, ms), bound in zip(large, (1e-6, 1e-6, 2e-6)):
        print(variant, "fp16x3 8192", err, ms)
        assert flag == 0 and err < bound * 8192, (err, ms)
    # single products (one 16-bit product) at n = 4096
    for (err, flag, ms), f in zip(single, (1.0, 1.0, 2.0)):
        bound = 8.0 * 2.0 ** -11 * np.sqrt(2.0 * 4096 / 27.0) * f
        assert flag == 0 and err < bound, (err, bound)


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "tf32x3"])
def test_single_product_probe_chains(X, prec):
    # kernel_prec = 1: the kernel's response chains run one hi*hi product per
    # step; charges and forces (expansion and mu chain at three products) do not
    # change, and K r is checked against the oracle's exact-response kernel
    s = synth.make_system(37, 11)
    out = {}
    ref = None
    for kp in (0, 1):
        p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, prec=prec, mu_tol=1e-3,
                             kernel_prec=kp)
        m = O.Model(Te=p.Te, n_sq=p.n_sq)
        rng = np.random.default_rng(2)
        n = rng.normal(scale=0.02, size=s.natoms)
        n -= n.mean()
        ref = O.evaluate(s.R, s.L, s.Z, n, m, O.XLParams(rank_m=p.rank_m, kernel_c=p.kernel_c))
        with X.Context(p, [sysdict(s)]) as ctx:
            ctx.set(0, X.N, n)
            ctx.set(0, X.MU, [ref.dens.mu + 0.01])
            ctx.build_H(0)
            ctx.density(0)
            ctx.kernel_update(0)
            out[kp] = (ctx.get(0, X.Q), ctx.get(0, X.F), ctx.get(0, X.KR))
    q0, F0, K0 = out[0]
    q1, F1, K1 = out[1]
    assert np.array_equal(q0, q1) and np.array_equal(F0, F1)
    rel = np.abs(K1 - ref.Kr).max() / np.abs(ref.Kr).max()
    print(prec, "single-product probes: K r rel err", rel, "three products:",
          np.abs(K0 - ref.Kr).max() / np.abs(ref.Kr).max())
    assert rel < (2e-2 if prec == "bf16x3" else 2e-3)


def test_graph_replay_matches_direct_launches(X):
    # params.graphs = 1: chemical-potential passes and probe responses are
    # captured on their second run and replayed afterwards; a run through the
    # kernel SCF and 15 MD steps must equal the run with direct launches bitwise
    import torch
    s = synth.make_system(64, 3)
    res = {}
    stream = torch.cuda.Stream()      # the legacy default stream cannot be captured
    for g in (0, 1):
        p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, prec="fp16x3", Te=1000.0,
                             n_sq=12, rank_m=2, scf_mode=1, kernel_auto=1, scf_tol=1e-5, mu_tol=1e-3,
                             rep_A=40.0, graphs=g)
        with X.Context(p, [sysdict(s)], stream=stream.cuda_stream) as ctx:
            ctx.scf(0)
            ctx.step(15)
            res[g] = [ctx.get(0, w) for w in (X.Q, X.R, X.NHIST, X.KR, X.F, X.STATS)]
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [256, 384, 1024])
@pytest.mark.parametrize("sym", [0, 1, 2])
@pytest.mark.parametrize("single", [False, True])
@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_grouped_product_equals_single_launches(X, n, sym, single, prec):
    # the grouped launch of the lockstep batch path (several problems' tiles in one persistent
    # launch, per-problem tensor maps and epilogue arguments from a device table, both tile
    # widths as the autotuner tries them) computes every tile exactly as a single launch does
    err, flag = X.binding.selftest_gemm_group(n, prec, sym, single=single, nprob=3)
    print(prec, n, sym, single, err)
    assert flag == 0
    assert err == 0.0


@pytest.mark.parametrize("kernel_prec,tol", [(0, 1e-4), (1, 2e-3)])
def test_grouped_exact_kernel_256_atoms(X, kernel_prec, tol):
    # the exact kernel K = (J - I)^-1 (Eq. KK) of a 256-atom system: its 256 unit-probe response
    # chains run up to 64 at a time in chain slots of their own, every chain product one grouped
    # launch; K against the oracle's eigenbasis kernel, and the cost of one recompute
    import time
    s = synth.make_system(256, 31)
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, prec="fp16x3", mu_tol=1e-3,
                         kernel_mode=1, kernel_prec=kernel_prec)
    m = O.Model(Te=p.Te, n_sq=p.n_sq)
    rng = np.random.default_rng(9)
    n = rng.normal(scale=0.01, size=s.natoms)
    n -= n.mean()
    ev = O.evaluate(s.R, s.L, s.Z, n, m, None, with_kernel=False, with_forces=False)
    Kref = O.kernel_exact(ev.dens, ev.gamma)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ev.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_exact(0)           # allocates the chain slots
        ctx.get(0, X.MU)
        t = time.perf_counter()
        ctx.kernel_exact(0)
        K = ctx.get(0, X.KMAT)
        dt = time.perf_counter() - t
    err = np.max(np.abs(K - Kref)) / np.abs(Kref).max()
    print("exact kernel 256 atoms, kernel_prec", kernel_prec, "rel err", err, "recompute s", dt)
    assert err < tol

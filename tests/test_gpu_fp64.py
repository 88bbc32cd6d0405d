"""GPU parity of the plain-FP64 path against the oracle (through the C ABI).

Tolerances (FP64 path): charges 1e-9 e, energies 1e-8 relative, forces
1e-8 eV/A, Hamiltonian and density elements 1e-10.  Inputs are seeded
synthetic systems; the 37-atom case has a padded orbital count (148 -> 256).
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


def model_params(X, **kw):
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1.0 - 1.0 / ALPHA_MIX, **kw)
    return p


def oracle_model(p):
    return O.Model(Te=p.Te, n_sq=p.n_sq, rep_A=p.rep_A, rep_rho=p.rep_rho)


CASES = [
    ("tiny24", lambda: synth.make_system(24, 1705, L=7.0)),
    ("ragged37", lambda: synth.make_system(37, 11)),
    ("small8", lambda: synth.make_system(8, 42, L=7.0)),
]


def random_n(nat, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    n = rng.normal(scale=scale, size=nat)
    return n - n.mean()


@pytest.mark.parametrize("name,make", CASES)
def test_build_H_and_gamma(X, name, make):
    s = make()
    p = model_params(X)
    m = oracle_model(p)
    n = random_n(s.natoms, 1)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.build_H(0)
        H = ctx.get(0, X.H)
        G = ctx.get(0, X.GAMMA)
    Gref = O.build_gamma(s.R, s.L, m)
    Href = O.hamiltonian(O.build_H0(s.R, s.L, m), Gref, n)
    assert np.max(np.abs(G - Gref)) < 1e-10 * np.max(np.abs(Gref))
    assert np.max(np.abs(H - Href)) < 1e-11


@pytest.mark.parametrize("name,make", CASES)
def test_density_charges_forces_energy(X, name, make):
    s = make()
    p = model_params(X)
    m = oracle_model(p)
    n = random_n(s.natoms, 2)
    ref = O.evaluate(s.R, s.L, s.Z, n, m, None, with_kernel=False)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ref.dens.mu + 0.02])
        ctx.build_H(0)
        ctx.density(0)
        ctx.energy(0)
        q, D, F, mu = ctx.get(0, X.Q), ctx.get(0, X.D), ctx.get(0, X.F), ctx.get(0, X.MU)[0]
        E = ctx.get(0, X.ENERGY)
    assert abs(mu - ref.dens.mu) < 1e-9
    assert np.max(np.abs(D - ref.dens.D)) < 1e-10
    assert np.max(np.abs(q - ref.q)) < 1e-9
    assert np.max(np.abs(F - ref.F)) < 1e-8
    parts = ref.parts
    assert E[1] == pytest.approx(parts["band"], rel=1e-10, abs=1e-9)
    assert E[2] == pytest.approx(parts["coulomb"], rel=1e-9, abs=1e-9)
    assert E[3] == pytest.approx(parts["entropy"], rel=1e-7, abs=1e-8)
    assert E[0] == pytest.approx(ref.Omega, rel=1e-8)


@pytest.mark.parametrize("name,make", CASES[:2])
def test_response_and_kernel(X, name, make):
    import torch
    s = make()
    p = model_params(X, rank_m=4)
    m = oracle_model(p)
    n = random_n(s.natoms, 3)
    xl = O.XLParams(rank_m=4, kernel_c=p.kernel_c)
    ref = O.evaluate(s.R, s.L, s.Z, n, m, xl)
    rng = np.random.default_rng(4)
    v = rng.normal(size=s.natoms)
    v -= v.mean()
    v /= np.linalg.norm(v)
    wref = O.response(ref.dens, ref.gamma, v)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ref.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        vd = torch.tensor(v, dtype=torch.float64, device="cuda")
        wd = torch.zeros_like(vd)
        ctx.response(0, vd.data_ptr(), wd.data_ptr())
        torch.cuda.synchronize()
        w = wd.cpu().numpy()
        ctx.kernel_update(0)
        Kr = ctx.get(0, X.KR)
        probes = ctx.get(0, X.PROBES)
    assert np.max(np.abs(w - wref)) < 1e-8 * max(1.0, np.max(np.abs(wref)))
    assert np.max(np.abs(Kr - ref.Kr)) < 1e-9
    Vref = np.array(ref.V)
    assert np.max(np.abs(probes[0][:len(Vref)] - Vref)) < 1e-8


def test_scf_ground_state(X):
    s = synth.make_system(24, 1705, L=7.0)
    p = model_params(X)
    m = oracle_model(p)
    n_ref, _ = O.scf(s.R, s.L, s.Z, m, ALPHA_MIX, tol=p.scf_tol)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.scf(0)
        n = ctx.get(0, X.N)
        hist = ctx.get(0, X.NHIST)
    assert np.max(np.abs(n - n_ref)) < 1e-9
    assert np.allclose(hist, hist[0][None, :])


@pytest.mark.parametrize("rank", [2, 4])
def test_kernel_scf_ground_state(X, rank):
    # Eq. SCF_K with the rank-m kernel and a fixed c, against the oracle's kernel SCF
    s = synth.make_system(24, 1705, L=7.0)
    p = model_params(X, scf_mode=1, rank_m=rank)
    m = oracle_model(p)
    n_ref, it = O.scf_kernel(s.R, s.L, s.Z, m, rank, p.kernel_c, tol=p.scf_tol)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.scf(0)
        n = ctx.get(0, X.N)
    assert np.max(np.abs(n - n_ref)) < 1e-9, it


def test_trajectory_matches_oracle(X):
    s = synth.make_system(24, 1705, L=7.0)
    p = model_params(X)
    m = oracle_model(p)
    xl = O.XLParams(rank_m=p.rank_m, kernel_c=p.kernel_c, mix_alpha=ALPHA_MIX)
    st, ev = O.md_init(s.R, s.V, s.L, s.Z, s.mass, m, xl)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, st.nhist[0])
        ctx.set(0, X.MU, [ev.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_update(0)
        assert np.max(np.abs(ctx.get(0, X.KR) - st.Kr)) < 1e-9
        for k in range(50):
            st, ev = O.md_step(st, s.L, s.Z, s.mass, m, xl)
            ctx.step(1)
            ctx.energy(0)
            R = ctx.get(0, X.R)
            dR = O.min_image(R - st.R, s.L)
            assert np.max(np.abs(dR)) < 1e-9, k
            assert np.max(np.abs(ctx.get(0, X.Q) - ev.q)) < 1e-9, k
            assert np.max(np.abs(ctx.get(0, X.N) - st.nhist[0])) < 1e-9, k
            E = ctx.get(0, X.ENERGY)
            assert E[0] == pytest.approx(ev.Omega, rel=1e-8), k


@pytest.mark.parametrize("prec,tol_q", [("fp64", 1e-9), ("fp16x3", 1e-5), ("bf16x3", 3e-5)])
def test_mu_search_through_flat_occupation(X, prec, tol_q):
    # (BF16x3 is held to its measured level, 3e-5 e, outside the 1e-5 e bound of FP16x3)
    # 33 atoms at n = 0, Te = 1000 K, 12 squarings: from the first guess (the
    # middle of the Gershgorin interval) the safeguarded Newton search bisects
    # to a mu above every level, where Tr D = N and dTr D/dmu = 0; it must
    # keep bisecting to Tr D = N_occ rather than accept the zero step
    s = synth.make_system(33, 1715)
    p = model_params(X, Te=1000.0, n_sq=12, prec=prec, mu_tol=1e-9 if prec == "fp64" else 1e-3)
    ref = O.evaluate(s.R, s.L, s.Z, np.zeros(s.natoms), O.Model(Te=1000.0, n_sq=12), None, with_kernel=False)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.build_H(0)
        ctx.density(0)
        q = ctx.get(0, X.Q)
    print(prec, "dq", np.abs(q - ref.q).max())
    assert abs(q.sum() - ref.q.sum()) < s.natoms * tol_q
    assert np.max(np.abs(q - ref.q)) < tol_q


def test_pair_repulsion_matches_oracle(X):
    s = synth.make_system(24, 1705, L=7.0)
    p = model_params(X, rep_A=40.0, rep_rho=0.3)
    m = oracle_model(p)
    n = random_n(s.natoms, 12)
    ref = O.evaluate(s.R, s.L, s.Z, n, m, None, with_kernel=False)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ref.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.energy(0)
        F, E = ctx.get(0, X.F), ctx.get(0, X.ENERGY)
    assert ref.parts["repulsion"] > 0.0
    assert E[6] == pytest.approx(ref.parts["repulsion"], rel=1e-12, abs=1e-12)
    assert E[0] == pytest.approx(ref.Omega, rel=1e-8)
    assert np.max(np.abs(F - ref.F)) < 1e-8


def test_single_atom_edge_case(X):
    p = model_params(X)
    s = dict(natoms=1, L=7.0, R=np.array([[1.0, 2.0, 3.0]]), V=np.zeros((1, 3)), Z=np.array([4.0]), mass=12.0)
    with X.Context(p, [s]) as ctx:
        ctx.build_H(0)
        ctx.density(0)
        q = ctx.get(0, X.Q)
        F = ctx.get(0, X.F)
    assert abs(q[0]) < 1e-12
    assert np.max(np.abs(F)) < 1e-12


def test_argument_errors_are_reported(X):
    p = model_params(X)
    s = synth.make_system(8, 42, L=7.0)
    bad = sysdict(s)
    bad["L"] = 4.0           # box not larger than the hopping cutoff
    with pytest.raises(X.XlbomdError) as e:
        X.Context(p, [bad])
    assert e.value.status == -1
    with X.Context(p, [sysdict(s)]) as ctx:
        with pytest.raises(X.XlbomdError) as e:
            ctx.kernel_update(0)     # no density yet
        assert e.value.status == -1
        with pytest.raises(X.XlbomdError):
            ctx.build_H(0)           # sticky until cleared
        ctx._lib.xlbomd_clear_error(ctx.h)
        ctx.build_H(0)


@pytest.mark.parametrize("name,make", CASES[:2])
def test_exact_kernel_matches_oracle(X, name, make):
    # Eq. KK: K = (J - I)^-1 with J from the natoms unit-direction responses
    s = make()
    p = model_params(X, kernel_mode=1)
    m = oracle_model(p)
    n = random_n(s.natoms, 6)
    ev = O.evaluate(s.R, s.L, s.Z, n, m, None, with_kernel=False, with_forces=False)
    Kref = O.kernel_exact(ev.dens, ev.gamma)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, n)
        ctx.set(0, X.MU, [ev.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_update(0)           # computes the held kernel, then K r
        K = ctx.get(0, X.KMAT)
        Kr = ctx.get(0, X.KR)
        assert ctx.get(0, X.STATS)[2] == s.natoms
    assert np.max(np.abs(K - Kref)) < 1e-9 * max(1.0, np.abs(Kref).max())
    assert np.max(np.abs(Kr - Kref @ ev.r)) < 1e-10


@pytest.mark.parametrize("variant", ["exact_every5", "accumulated", "delta", "kmax6", "kmax7", "repulsion"])
def test_kernel_and_dissipation_variants_follow_oracle(X, variant):
    # the exact kernel held and recomputed every 5 steps (Section VI.A), the
    # accumulated rank-1 kernel (end of Section V.F), K = K_0 only (rank 0), and
    # the K_max = 6, 7 rows of Table I (the library's table against the
    # oracle's, typed independently)
    s = synth.make_system(24, 1705, L=7.0)
    kw, xlkw = {}, {}
    if variant == "exact_every5":
        kw, xlkw = dict(kernel_mode=1, kernel_every=5), dict(kernel_mode="exact", kernel_every=5)
    elif variant == "accumulated":
        kw, xlkw = dict(kernel_mode=2), dict(kernel_mode="accumulated")
    elif variant == "repulsion":
        kw = dict(rep_A=40.0, rep_rho=0.3)
    elif variant == "delta":
        kw, xlkw = dict(rank_m=0), dict(rank_m=0)
    else:
        kmax = int(variant[-1])
        kappa, alpha, c = O.TABLE_I[kmax]
        kw, xlkw = dict(kmax=kmax), dict(kappa=kappa, alpha=alpha, c=tuple(float(x) for x in c))
    p = model_params(X, **kw)
    m = oracle_model(p)
    base = dict(rank_m=p.rank_m, kernel_c=p.kernel_c, mix_alpha=ALPHA_MIX)
    base.update(xlkw)
    xl = O.XLParams(**base)
    assert p.kmax == xl.kmax and abs(p.kappa - xl.kappa) < 1e-15 and abs(p.alpha - xl.alpha) < 1e-15
    assert all(abs(p.c[k] - xl.c[k]) < 1e-15 for k in range(xl.kmax + 1))
    st, ev = O.md_init(s.R, s.V, s.L, s.Z, s.mass, m, xl)
    with X.Context(p, [sysdict(s)]) as ctx:
        ctx.set(0, X.N, st.nhist[0])
        ctx.set(0, X.MU, [ev.dens.mu])
        ctx.build_H(0)
        ctx.density(0)
        ctx.kernel_update(0)
        assert np.max(np.abs(ctx.get(0, X.KR) - st.Kr)) < 1e-9
        for k in range(12):
            st, ev = O.md_step(st, s.L, s.Z, s.mass, m, xl)
            ctx.step(1)
            assert np.max(np.abs(O.min_image(ctx.get(0, X.R) - st.R, s.L))) < 1e-9, k
            assert np.max(np.abs(ctx.get(0, X.Q) - ev.q)) < 1e-9, k
            assert np.max(np.abs(ctx.get(0, X.N) - st.nhist[0])) < 1e-9, k
            assert np.max(np.abs(ctx.get(0, X.KR) - ev.Kr)) < 1e-9, k


def test_residual_and_energy_fluctuations_scale_as_dt_squared_on_gpu(X):
    # Section VI.C, Figs. 9-10, through the C ABI: over the same 10 fs from the t0 ground state,
    # halving dt divides the RMS residual |q[n] - n| and the total-energy fluctuation by about 4
    s = synth.make_system(24, 1705, L=7.0)
    res, fluct = [], []
    for dt in (0.5, 0.25, 0.125):
        p = model_params(X, dt=dt, rank_m=2)
        with X.Context(p, [sysdict(s)]) as ctx:
            ctx.scf(0)
            r, E = [], []
            for _ in range(int(round(10.0 / dt))):
                ctx.step(1)
                ctx.energy(0)
                r.append(np.sqrt(np.mean(ctx.get(0, X.RES) ** 2)))
                E.append(ctx.get(0, X.ENERGY)[5])
        assert np.max(np.abs(np.asarray(E) - E[0])) < 1e-3, dt
        res.append(np.mean(r))
        fluct.append(np.std(E))
    print("dt study: residual RMS", res, "energy std", fluct)
    for a, b in ((res[0], res[1]), (res[1], res[2]), (fluct[0], fluct[1]), (fluct[1], fluct[2])):
        assert 3.0 < a / b < 5.5, (res, fluct)

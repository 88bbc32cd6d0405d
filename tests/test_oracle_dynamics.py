"""Pins of the oracle's forces, energy and integrator.

References: central finite differences of the shadow free energy, Newton's
third law, Table I's moment conditions, time reversibility of the undamped
integrator, and energy conservation of the damped one.
"""
import numpy as np
import pytest

import oracle as O
import synth

M = O.Model()


def omega_at(R, L, Z, n, model):
    ev = O.evaluate(R, L, Z, n, model, None, with_kernel=False, with_forces=False)
    return ev.Omega


@pytest.fixture(scope="module")
def small():
    s = synth.make_system(8, 42, L=7.0)
    rng = np.random.default_rng(4)
    n = rng.normal(scale=0.05, size=8)
    n -= n.mean()
    return s, n


def test_forces_match_finite_differences_of_free_energy(small):
    # With 20 squarings the occupations equal Fermi-Dirac to ~1e-13, so the
    # Hellmann-Feynman forces are the exact gradient of Omega at fixed n.
    s, n = small
    m20 = O.Model(n_sq=20)
    ev = O.evaluate(s.R, s.L, s.Z, n, m20, None, with_kernel=False)
    h = 1e-5
    for I in (0, 3, 7):
        for c in range(3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[I, c] += h
            Rm[I, c] -= h
            fd = -(omega_at(Rp, s.L, s.Z, n, m20) - omega_at(Rm, s.L, s.Z, n, m20)) / (2 * h)
            assert ev.F[I, c] == pytest.approx(fd, abs=2e-7)


def test_forces_with_ten_squarings_are_close_to_gradient(small):
    s, n = small
    ev = O.evaluate(s.R, s.L, s.Z, n, M, None, with_kernel=False)
    h = 1e-5
    I = 2
    for c in range(3):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[I, c] += h
        Rm[I, c] -= h
        fd = -(omega_at(Rp, s.L, s.Z, n, M) - omega_at(Rm, s.L, s.Z, n, M)) / (2 * h)
        assert ev.F[I, c] == pytest.approx(fd, abs=1e-4)


def test_forces_sum_to_zero(small):
    s, n = small
    ev = O.evaluate(s.R, s.L, s.Z, n, M, None, with_kernel=False)
    assert np.allclose(ev.F.sum(axis=0), 0.0, atol=1e-11)


def test_table_I_of_the_oracle_is_the_printed_table(golden):
    printed = golden.table_i()
    assert sorted(printed) == sorted(O.TABLE_I) == [5, 6, 7]
    for kmax, (kappa, alpha, c) in printed.items():
        okappa, oalpha, oc = O.TABLE_I[kmax]
        assert (okappa, oalpha) == (kappa, alpha)
        assert tuple(oc) == c


@pytest.mark.parametrize("kmax", [5, 6, 7])
def test_table_I_coefficients_annihilate_constant_and_linear_histories(kmax):
    kappa, alpha, c = O.TABLE_I[kmax]
    c = np.asarray(c, dtype=float)
    k = np.arange(len(c))
    assert c.sum() == 0.0
    assert (k * c).sum() == 0.0
    assert kappa < 2.0


def test_dissipation_vanishes_on_linear_trajectory():
    xl = O.XLParams()
    a, b = np.array([0.1, -0.1]), np.array([0.01, 0.02])
    hist = np.array([a - k * b for k in range(xl.kmax + 1)])   # n(t - k dt) = a - k b
    n_new = O.n_update(hist, np.zeros(2), xl)
    assert np.allclose(n_new, a + b, atol=1e-15)


def test_undamped_integrator_is_time_reversible():
    s = synth.make_system(8, 42, L=7.0)
    xl = O.XLParams(alpha=0.0, rank_m=2, kernel_c=-15.0, mix_alpha=0.06, scf_tol=1e-12,
                    scf_max_iter=3000)
    st0, _ = O.md_init(s.R, s.V, s.L, s.Z, s.mass, M, xl)
    st = st0
    for _ in range(6):
        st, _ = O.md_step(st, s.L, s.Z, s.mass, M, xl)
    # reverse at t6: flip the velocities; the "previous" n of the backward run
    # is n(t7) = 2 n6 - n5 - kappa K r6, the undamped Eq. VRL_Damp.
    n7 = O.n_update(st.nhist, st.Kr, xl)
    hist = st.nhist.copy()
    hist[1] = n7
    rev = O.MDState(R=st.R.copy(), V=-st.V, nhist=hist, F=st.F, Kr=st.Kr)
    st_back = rev
    for _ in range(6):
        st_back, _ = O.md_step(st_back, s.L, s.Z, s.mass, M, xl)
    d = O.min_image(st_back.R - st0.R, s.L)
    assert np.max(np.abs(d)) < 1e-11
    assert np.allclose(st_back.nhist[0], st0.nhist[0], atol=1e-11)
    assert np.allclose(-st_back.V, st0.V, atol=1e-11)


def test_energy_is_conserved_over_a_short_run():
    s = synth.make_system(24, 1705, L=7.0)
    xl = O.XLParams(rank_m=2, kernel_c=1 - 1 / 0.06, mix_alpha=0.06)
    st, ev = O.md_init(s.R, s.V, s.L, s.Z, s.mass, M, xl)
    E = [O.kinetic_energy(st.V, s.mass) + ev.Omega]
    for _ in range(60):
        st, ev = O.md_step(st, s.L, s.Z, s.mass, M, xl)
        E.append(O.kinetic_energy(st.V, s.mass) + ev.Omega)
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) < 1e-4
    # no systematic drift: slope of a linear fit over the run is tiny
    slope = np.polyfit(np.arange(len(E)), E, 1)[0]
    assert abs(slope) < 1e-6


def test_full_kernel_keeps_the_residual_below_the_scaled_delta_kernel():
    # Section VI.A, Figs. 3-4: the full kernel computed at t0 and kept constant
    # keeps n closer to the ground state than K = K_0 = I/(c - 1) alone
    s = synth.make_system(24, 1705, L=7.0)
    base = dict(kernel_c=1 - 1 / 0.06, mix_alpha=0.06)
    rms = {}
    for name, xl in (("delta", O.XLParams(rank_m=0, **base)),
                     ("full", O.XLParams(kernel_mode="exact", kernel_every=0, **base)),
                     ("full10", O.XLParams(kernel_mode="exact", kernel_every=10, **base))):
        st, ev = O.md_init(s.R, s.V, s.L, s.Z, s.mass, M, xl)
        E0 = O.kinetic_energy(st.V, s.mass) + ev.Omega
        res, dE = [], []
        for _ in range(40):
            st, ev = O.md_step(st, s.L, s.Z, s.mass, M, xl)
            res.append(np.sqrt(np.mean(ev.r ** 2)))
            dE.append(O.kinetic_energy(st.V, s.mass) + ev.Omega - E0)
        rms[name] = np.mean(res)
        assert np.max(np.abs(dE)) < 1e-3, name
    assert rms["full"] < 0.5 * rms["delta"]
    assert rms["full10"] <= 1.2 * rms["full"]


def test_residual_and_energy_fluctuations_scale_as_dt_squared():
    # Section VI.C, Figs. 9-10: over the same 10 fs, halving dt divides the RMS
    # residual |q[n] - n| and the total-energy fluctuation by about 4
    s = synth.make_system(24, 1705, L=7.0)
    res, fluct = [], []
    for dt in (0.5, 0.25, 0.125):
        xl = O.XLParams(dt=dt, rank_m=2, kernel_c=1 - 1 / 0.06, mix_alpha=0.06)
        st, ev = O.md_init(s.R, s.V, s.L, s.Z, s.mass, M, xl)
        r, E = [], []
        for _ in range(int(round(10.0 / dt))):
            st, ev = O.md_step(st, s.L, s.Z, s.mass, M, xl)
            r.append(np.sqrt(np.mean(ev.r ** 2)))
            E.append(O.kinetic_energy(st.V, s.mass) + ev.Omega)
        res.append(np.mean(r))
        fluct.append(np.std(E))
    for a, b in ((res[0], res[1]), (res[1], res[2]), (fluct[0], fluct[1]), (fluct[1], fluct[2])):
        assert 3.0 < a / b < 5.5, (res, fluct)


def test_pair_repulsion_forces_and_energy():
    # the optional pair term: its forces are minus the finite-difference gradient
    # of Omega, pairwise (sum F = 0), zero at rep_A = 0, and the dimer value is
    # A exp(-r/rho) inside the taper
    s = synth.make_system(8, 42, L=7.0)
    mr = O.Model(n_sq=20, rep_A=40.0, rep_rho=0.3)
    e0, g0 = O.repulsion(s.R, s.L, O.Model())
    assert e0 == 0.0 and not np.any(g0)
    e, g = O.repulsion(s.R, s.L, mr)
    assert np.max(np.abs(g.sum(axis=0))) < 1e-12
    h = 1e-6
    for I in (0, 5):
        for c in range(3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[I, c] += h
            Rm[I, c] -= h
            fd = (O.repulsion(Rp, s.L, mr)[0] - O.repulsion(Rm, s.L, mr)[0]) / (2 * h)
            assert abs(fd - g[I, c]) < 1e-7
    R2 = np.array([[1.0, 1.0, 1.0], [2.5, 1.0, 1.0]])
    assert abs(O.repulsion(R2, 12.0, mr)[0] - 40.0 * np.exp(-1.5 / 0.3)) < 1e-14
    # the full force with the pair term against finite differences of Omega at fixed n
    rng = np.random.default_rng(4)
    n = rng.normal(scale=0.05, size=8)
    n -= n.mean()
    ev = O.evaluate(s.R, s.L, s.Z, n, mr, None, with_kernel=False)
    for I, c in ((1, 0), (6, 2)):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[I, c] += 1e-5
        Rm[I, c] -= 1e-5
        fd = (omega_at(Rp, s.L, s.Z, n, mr) - omega_at(Rm, s.L, s.Z, n, mr)) / 2e-5
        assert abs(ev.F[I, c] + fd) < 1e-6

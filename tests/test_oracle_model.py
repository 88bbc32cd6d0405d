"""Pins of the oracle's model layer (H0, gamma) and of the seeded inputs.

Each check compares against something other than the oracle's own formula:
hand-evaluated Slater-Koster values, finite differences, symmetry and
invariance properties, and the direct (non-Ewald) lattice sum.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth

M = O.Model()


def V_of(r, k):
    """Hand value of bond integral k at r (no taper below 4.5 A)."""
    return M.t0[k] * math.exp(-r / M.r_decay)


def test_splitmix64_published_sequence():
    # Reference outputs of SplitMix64 for seed 1234567 (Vigna's test vectors).
    g = synth.SplitMix64(1234567)
    got = [g.next_u64() for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_positions_respect_min_separation_and_box():
    s = synth.make_system(24, 1705, L=7.0)
    assert s.R.shape == (24, 3)
    assert np.all(s.R >= 0) and np.all(s.R < 7.0)
    d = O.min_image(s.R[None] - s.R[:, None], 7.0)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(24) * 99
    assert r.min() >= 1.8


def test_velocities_zero_momentum_and_temperature():
    s = synth.make_system(24, 1705, L=7.0)
    assert np.allclose(s.V.sum(0), 0, atol=1e-14)
    ke = O.kinetic_energy(s.V, s.mass)
    assert ke == pytest.approx(0.5 * (3 * 24 - 3) * O.KB_EV * 300.0, rel=1e-12)


def test_sk_dimer_along_x_hand_values():
    r = 2.0
    E, _ = O.sk_blocks(np.array([[r, 0, 0]]), M)
    E = E[0]
    sss, sps, pps, ppp = (V_of(r, k) for k in range(4))
    expect = np.array([[sss, sps, 0, 0],
                       [-sps, pps, 0, 0],
                       [0, 0, ppp, 0],
                       [0, 0, 0, ppp]])
    assert np.allclose(E, expect, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sk_dimer_along_each_axis(axis):
    r = 1.9
    d = np.zeros((1, 3))
    d[0, axis] = -r                      # negative direction flips the s-p sign
    E, _ = O.sk_blocks(d, M)
    E = E[0]
    assert E[0, 1 + axis] == pytest.approx(-V_of(r, 1), abs=1e-15)
    assert E[1 + axis, 0] == pytest.approx(V_of(r, 1), abs=1e-15)
    assert E[1 + axis, 1 + axis] == pytest.approx(V_of(r, 2), abs=1e-15)
    for b in range(3):
        if b != axis:
            assert E[1 + b, 1 + b] == pytest.approx(V_of(r, 3), abs=1e-15)
            assert E[0, 1 + b] == 0.0


def test_sk_diagonal_direction():
    r = 2.2
    d = np.array([[1.0, 1.0, 1.0]]) * r / math.sqrt(3.0)
    E, _ = O.sk_blocks(d, M)
    E = E[0]
    pps, ppp = V_of(r, 2), V_of(r, 3)
    assert E[1, 2] == pytest.approx((pps - ppp) / 3.0, abs=1e-14)
    assert E[1, 1] == pytest.approx(pps / 3.0 + 2.0 * ppp / 3.0, abs=1e-14)
    assert E[0, 3] == pytest.approx(V_of(r, 1) / math.sqrt(3.0), abs=1e-14)


def test_sk_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(6, 3))
    d *= (rng.uniform(1.6, 4.9, size=6) / np.linalg.norm(d, axis=1))[:, None]
    _, G = O.sk_blocks(d, M)
    h = 1e-6
    for g in range(3):
        dp, dm = d.copy(), d.copy()
        dp[:, g] += h
        dm[:, g] -= h
        fd = (O.sk_blocks(dp, M)[0] - O.sk_blocks(dm, M)[0]) / (2 * h)
        assert np.allclose(G[..., g], fd, atol=1e-8)


def test_taper_is_c2_and_ends():
    S, dS = O.taper(np.array([4.5, 5.0, 3.0, 6.0]), 4.5, 5.0)
    assert np.allclose(S, [1, 0, 1, 0]) and np.allclose(dS, 0)
    h = 1e-6
    for r in [4.6, 4.75, 4.9]:
        fd = (O.taper(r + h, 4.5, 5.0)[0] - O.taper(r - h, 4.5, 5.0)[0]) / (2 * h)
        assert O.taper(r, 4.5, 5.0)[1] == pytest.approx(fd, rel=1e-7)


def test_H0_symmetric_and_translation_invariant():
    s = synth.make_system(16, 11, L=7.0)
    H = O.build_H0(s.R, s.L, M)
    assert np.array_equal(H, H.T)
    R2 = O.wrap(s.R + np.array([1.3, -2.9, 0.77]), s.L)
    e1 = np.linalg.eigvalsh(H)
    e2 = np.linalg.eigvalsh(O.build_H0(R2, s.L, M))
    assert np.allclose(e1, e2, atol=1e-12)


def test_H0_spectrum_independent_of_sp_sign():
    # Flipping the sign of every p orbital is unitary; it flips V_sp-sigma.
    s = synth.make_system(12, 5, L=7.0)
    M2 = O.Model(t0=(M.t0[0], -M.t0[1], M.t0[2], M.t0[3]))
    e1 = np.linalg.eigvalsh(O.build_H0(s.R, s.L, M))
    e2 = np.linalg.eigvalsh(O.build_H0(s.R, s.L, M2))
    assert np.allclose(e1, e2, atol=1e-12)


def test_H0_rotation_of_dimer_keeps_spectrum():
    L = 30.0
    base = np.array([[10.0, 10.0, 10.0]])
    rng = np.random.default_rng(0)
    specs = []
    for _ in range(3):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        R = np.vstack([base, base + 2.1 * u])
        specs.append(np.linalg.eigvalsh(O.build_H0(R, L, M)))
    assert np.allclose(specs[0], specs[1], atol=1e-13)
    assert np.allclose(specs[0], specs[2], atol=1e-13)


def _direct_point_coulomb(R, L, q, nshell):
    """1/2 sum over lattice vectors T within nshell and pairs I, J of
    q_I q_J / |R_J - R_I + T L|, without the I = J, T = 0 term."""
    E = 0.0
    for T in itertools.product(range(-nshell, nshell + 1), repeat=3):
        d = R[None, :, :] - R[:, None, :] + np.array(T) * L
        r = np.sqrt(np.sum(d * d, axis=2))
        if T == (0, 0, 0):
            np.fill_diagonal(r, np.inf)
        E += 0.5 * q @ (1.0 / r) @ q
    return E


def _ok_correction_27(R, L, q, a):
    """1/2 q^T C q, C_IJ = sum over 27 shifts of the minimum-image vector of
    1/sqrt(r^2+a^2) - 1/r, with 1/a for I = J, T = 0."""
    E = 0.0
    dmin = R[None, :, :] - R[:, None, :]
    dmin = dmin - L * np.rint(dmin / L)
    for T in itertools.product((-1, 0, 1), repeat=3):
        d = dmin + np.array(T) * L
        r = np.sqrt(np.sum(d * d, axis=2))
        with np.errstate(divide="ignore"):
            C = 1.0 / np.sqrt(r * r + a * a) - 1.0 / r
        if T == (0, 0, 0):
            np.fill_diagonal(C, 1.0 / a)
        E += 0.5 * q @ C @ q
    return E


def test_gamma_matches_direct_lattice_sum_for_neutral_charges():
    # A cube-by-cube direct sum of 1/r converges to the Ewald (conducting
    # boundary) energy plus the surface term 2 pi |M|^2 / (3 V), M = sum q_I R_I
    # (de Leeuw, Perram and Smith, 1980).  Its error falls off slowly, so
    # two shells are extrapolated assuming an error ~ 1/n^2.
    rng = np.random.default_rng(1)
    L = 7.0
    R = rng.uniform(0, L, size=(4, 3))
    q = np.array([0.3, -0.1, -0.5, 0.3])
    a = M.coulomb_k / M.hubbard_U
    e_model = 0.5 * q @ O.build_gamma(R, L, M) @ q / M.coulomb_k
    e8 = _direct_point_coulomb(R, L, q, 8)
    e16 = _direct_point_coulomb(R, L, q, 16)
    e_inf = e16 + (e16 - e8) / 3.0
    dip = q @ R
    surface = 2.0 * math.pi * (dip @ dip) / (3.0 * L ** 3)
    e_check = e_inf - surface + _ok_correction_27(R, L, q, a)
    assert e_model == pytest.approx(e_check, abs=2e-5)


def test_gamma_independent_of_ewald_splitting_on_neutral_vectors():
    s = synth.make_system(10, 77, L=7.0)
    P = np.eye(10) - 0.1
    g1 = P @ O.build_gamma(s.R, s.L, M, eta=3.5 / s.L) @ P
    g2 = P @ O.build_gamma(s.R, s.L, M, eta=5.0 / s.L) @ P
    assert np.allclose(g1, g2, atol=1e-11)


def test_gamma_isolated_dimer_limit():
    # In a very large box the neutral dimer energy tends to U - k/sqrt(r^2+a^2),
    # less the conducting-boundary dipole term 2 pi k r^2 / (3 L^3).
    L = 400.0
    r = 2.0
    R = np.array([[100.0, 100.0, 100.0], [100.0 + r, 100.0, 100.0]])
    g = O.build_gamma(R, L, M)
    a = M.coulomb_k / M.hubbard_U
    expect = (M.hubbard_U - M.coulomb_k / math.sqrt(r * r + a * a)
              - 2.0 * math.pi * M.coulomb_k * r * r / (3.0 * L ** 3))
    assert g[0, 0] - g[0, 1] == pytest.approx(expect, abs=1e-9)


def test_gamma_symmetric_and_positive_on_neutral_subspace():
    s = synth.make_system(24, 1705, L=7.0)
    g = O.build_gamma(s.R, s.L, M)
    assert np.allclose(g, g.T, atol=1e-13)
    P = np.eye(24) - 1.0 / 24
    ev = np.sort(np.linalg.eigvalsh(P @ g @ P))
    assert abs(ev[0]) < 1e-10 and ev[1] > 0.1


def test_gamma_gradient_matches_finite_differences():
    s = synth.make_system(6, 21, L=7.0)
    gg = O.build_gamma_grad(s.R, s.L, M)
    h = 1e-6
    for J in range(3):
        for c in range(3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[J, c] += h
            Rm[J, c] -= h
            fd = (O.build_gamma(Rp, s.L, M) - O.build_gamma(Rm, s.L, M)) / (2 * h)
            for I in range(6):
                if I != J:
                    assert gg[I, J, c] == pytest.approx(fd[I, J], abs=1e-7)

"""Pins of the oracle's electronic structure: occupations, D, mu, charges,
response, and the low-rank kernel.

The references are independent of the oracle's formulas: the matrix recursion
of the Fermi-operator expansion run by brute force, the Fermi-Dirac limit,
commutation and trace invariants, finite differences of q[n], the explicit
Sherman-Morrison sequence of Eq. K_up, the inverse of a finite-difference
Jacobian (the exact kernel, Eq. KK), and two consequences of the occupations
minimising the electronic free energy: dOmega/dTe = -2 kB S and
dOmega/dn = gamma (q[n] - n).
"""

import numpy as np
import pytest

import oracle as O
import synth

M = O.Model()


@pytest.fixture(scope="module")
def tiny():
    s = synth.make_system(8, 42, L=7.0)
    H0 = O.build_H0(s.R, s.L, M)
    gam = O.build_gamma(s.R, s.L, M)
    rng = np.random.default_rng(5)
    n = rng.normal(scale=0.05, size=8)
    n -= n.mean()
    return s, H0, gam, n


def brute_force_recursion(H, mu, beta, n_sq):
    """X_0 = I/2 - beta (H - mu I) / 2^(n+2);  X_{k+1} = X^2 [X^2 + (I - X)^2]^-1."""
    N = H.shape[0]
    I = np.eye(N)
    X = 0.5 * I - beta * (H - mu * I) / 2.0 ** (n_sq + 2)
    for _ in range(n_sq):
        X2 = X @ X
        X = X2 @ np.linalg.inv(X2 + (I - X) @ (I - X))
    return X


@pytest.mark.parametrize("n_sq", [6, 8, 10])
def test_closed_form_equals_matrix_recursion(tiny, n_sq):
    s, H0, gam, n = tiny
    H = O.hamiltonian(H0, gam, n)
    mu = -3.2
    eps, V = np.linalg.eigh(H)
    D_closed = (V * O.occupations(eps, mu, M.beta, n_sq)) @ V.T
    D_brute = brute_force_recursion(H, mu, M.beta, n_sq)
    assert np.allclose(D_closed, D_brute, atol=1e-11)


def test_large_n_tends_to_fermi_dirac():
    eps = np.linspace(-12, 2, 201)
    mu, beta = -3.0, M.beta
    fd = O.fermi_dirac(eps, mu, beta)
    for n, tol in [(10, 2e-6), (14, 1e-8), (20, 1e-12)]:
        assert np.max(np.abs(O.occupations(eps, mu, beta, n) - fd)) < tol


def test_dmu_derivative_matches_finite_difference():
    eps = np.linspace(-6, 0, 61)
    mu, beta, n, h = -3.0, M.beta, 10, 1e-6
    fd = (O.occupations(eps, mu + h, beta, n) - O.occupations(eps, mu - h, beta, n)) / (2 * h)
    assert np.allclose(O.occupations_dmu(eps, mu, beta, n), fd, atol=1e-7)


def test_density_invariants(tiny):
    s, H0, gam, n = tiny
    H = O.hamiltonian(H0, gam, n)
    d = O.density(H, M.beta, M.n_sq, 16)
    assert np.trace(d.D) == pytest.approx(16.0, abs=1e-11)
    assert np.linalg.norm(H @ d.D - d.D @ H) / np.linalg.norm(H) < 1e-12
    ev = np.linalg.eigvalsh(d.D)
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12


def test_neutral_system_charges_sum_to_zero(tiny):
    s, H0, gam, n = tiny
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    q = O.mulliken(d.D, s.Z)
    assert abs(q.sum()) < 1e-11


def test_entropy_stable_form_matches_direct_formula(tiny):
    s, H0, gam, n = tiny
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    f = d.f
    ok = (f > 1e-12) & (f < 1 - 1e-12)
    direct = -f[ok] * np.log(f[ok]) - (1 - f[ok]) * np.log(1 - f[ok])
    assert np.allclose(O.entropy_terms(d)[ok], direct, atol=1e-12)


@pytest.mark.parametrize("Te", [1000.0, 3000.0])
def test_omega_temperature_derivative_is_minus_twice_kB_entropy(tiny, Te):
    # At fixed n and R, Omega = 2 Tr[D H[n]] - 2 kB Te S + (terms without D), and the occupations
    # minimise that electronic free energy at fixed electron count (Fermi-Dirac; 20 squarings
    # make g_n equal to it within 1e-13).  By the envelope theorem dOmega/dTe = -2 kB S: a wrong
    # factor or sign of the entropy term, or a wrong s(f), breaks it.
    s, H0, gam, n = tiny

    def ev(T):
        return O.evaluate(s.R, s.L, s.Z, n, O.Model(Te=T, n_sq=20), None, with_kernel=False,
                          with_forces=False)

    h = 2.0
    e0 = ev(Te)
    fd = (ev(Te + h).Omega - ev(Te - h).Omega) / (2 * h)
    assert e0.parts["S"] > 0.05
    assert fd == pytest.approx(-2.0 * O.KB_EV * e0.parts["S"], rel=1e-5)


def test_omega_gradient_in_n_is_gamma_times_residual(tiny):
    # Omega[n] = 2 Tr[D H[n]] - 2 kB Te S - Z.gamma n - 1/2 n.gamma n with D[n] minimising the first
    # two terms, and 2 Tr[D H[n]] depends on n through (q + Z).gamma n: so dOmega/dn = gamma (q[n] - n)
    # exactly (Fermi-Dirac occupations, here 20 squarings), zero at the SCF ground state.  This fixes
    # the Coulomb term's factor and the charge definition independently of the forces.
    s, H0, gam, n = tiny
    m = O.Model(n_sq=20)

    def ev(nn):
        return O.evaluate(s.R, s.L, s.Z, nn, m, None, with_kernel=False, with_forces=False)

    e0 = ev(n)
    g = O.build_gamma(s.R, s.L, m) @ (e0.q - n)
    assert np.max(np.abs(g)) > 0.05
    h = 2.5e-5                     # central-difference error ~3e-8 here, falling as h^2
    for I in range(len(n)):
        d = np.zeros_like(n)
        d[I] = h
        fd = (ev(n + d).Omega - ev(n - d).Omega) / (2 * h)
        assert fd == pytest.approx(g[I], abs=1e-6), I


def test_divided_differences_against_naive_and_degenerate_limit(tiny):
    s, H0, gam, n = tiny
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    P, gmu = O.divided_differences(d)
    de = d.eps[:, None] - d.eps[None, :]
    far = np.abs(de) > 1e-3
    naive = (d.f[:, None] - d.f[None, :])[far] / de[far]
    assert np.allclose(P[far], naive, rtol=1e-9, atol=1e-13)
    assert np.allclose(np.diag(P), -gmu)


def test_response_matches_finite_difference_of_charges(tiny):
    s, H0, gam, n = tiny
    rng = np.random.default_rng(9)
    v = rng.normal(size=8)
    v -= v.mean()
    v /= np.linalg.norm(v)
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    w = O.response(d, gam, v)
    h = 1e-5
    qp = O.charges_at(s.R, s.L, s.Z, n + h * v, M)
    qm = O.charges_at(s.R, s.L, s.Z, n - h * v, M)
    assert np.allclose(w, (qp - qm) / (2 * h), atol=1e-8)
    assert abs(w.sum()) < 1e-12


def test_zero_coulomb_gives_zero_response_and_K_minus_identity(tiny):
    s, _, _, n = tiny
    M0 = O.Model(coulomb_k=0.0, hubbard_U=6.0)
    ev = O.evaluate(s.R, s.L, s.Z, n, M0, O.XLParams(rank_m=2, kernel_c=-4.0), with_forces=False)
    assert np.max(np.abs(np.array(ev.W))) < 1e-14
    # v_1 is parallel to r and J = 0 exactly, so the rank-m kernel is exact on r.
    assert np.allclose(ev.Kr, -ev.r, atol=1e-13)


def test_woodbury_equals_sherman_morrison_sequence(tiny):
    s, H0, gam, n = tiny
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    q = O.mulliken(d.D, s.Z)
    r = q - n
    c = -9.0
    for m in (1, 2, 4):
        Kr, V, W = O.kernel_rank_m(r, m, c, lambda v: O.response(d, gam, v))
        K, _ = O.kernel_sherman_morrison_dense(c, V, W)
        assert np.allclose(K @ r, Kr, atol=1e-13)
        Vm = np.array(V)
        assert np.allclose(Vm @ Vm.T, np.eye(len(V)), atol=1e-13)


def test_full_rank_sequence_reproduces_exact_kernel(tiny):
    # With N orthonormal probes the sequence gives K = (J - I)^-1 exactly
    # (Eq. KK); J from central finite differences of q[n].
    s, H0, gam, n = tiny
    nat = 8
    h = 1e-5
    J = np.zeros((nat, nat))
    for j in range(nat):
        e = np.zeros(nat)
        e[j] = 1.0
        J[:, j] = (O.charges_at(s.R, s.L, s.Z, n + h * e, M)
                   - O.charges_at(s.R, s.L, s.Z, n - h * e, M)) / (2 * h)
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    V = list(np.eye(nat))
    W = [O.response(d, gam, v) for v in V]
    K, Jseq = O.kernel_sherman_morrison_dense(-9.0, V, W)
    assert np.allclose(Jseq, J, atol=1e-7)
    Kx = np.linalg.inv(J - np.eye(nat))
    assert np.allclose(K, Kx, atol=1e-6 * np.abs(Kx).max())


def test_kernel_is_newton_step_on_linear_residual(tiny):
    # Eq. EffOfK: for a full-rank kernel, n - K r reaches the SCF fixed point to
    # second order in the residual.
    s, H0, gam, _ = tiny
    n_star, _ = O.scf(s.R, s.L, s.Z, M, 0.05, tol=1e-12, max_iter=3000)
    rng = np.random.default_rng(2)
    dn = rng.normal(size=8)
    dn -= dn.mean()
    errs = []
    for eps in (1e-3, 5e-4):
        n = n_star + eps * dn / np.linalg.norm(dn)
        d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
        r = O.mulliken(d.D, s.Z) - n
        Kr, _, _ = O.kernel_rank_m(r, 8, -9.0, lambda v: O.response(d, gam, v))
        errs.append(np.linalg.norm(n - Kr - n_star))
    # the error falls by ~4x when the displacement halves
    assert errs[1] < errs[0] / 3.0
    assert errs[0] < 1e-4


def test_mixing_scan_picks_converging_alpha():
    s = synth.make_system(8, 42, L=7.0)
    a, it = O.choose_mix_alpha(s.R, s.L, s.Z, M, candidates=[0.02, 0.05, 0.08])
    n, it2 = O.scf(s.R, s.L, s.Z, M, a)
    assert it2 == it
    d = O.density(O.hamiltonian(O.build_H0(s.R, s.L, M), O.build_gamma(s.R, s.L, M), n),
                  M.beta, M.n_sq, 16)
    assert np.max(np.abs(O.mulliken(d.D, s.Z) - n)) < 1e-10


def test_exact_kernel_is_inverse_of_finite_difference_jacobian(tiny):
    # Eq. KK from the unit-probe Jacobian, against central differences of q[n]
    s, H0, gam, n = tiny
    nat, h = 8, 1e-5
    Jfd = np.zeros((nat, nat))
    for j in range(nat):
        e = np.zeros(nat)
        e[j] = 1.0
        Jfd[:, j] = (O.charges_at(s.R, s.L, s.Z, n + h * e, M)
                     - O.charges_at(s.R, s.L, s.Z, n - h * e, M)) / (2 * h)
    d = O.density(O.hamiltonian(H0, gam, n), M.beta, M.n_sq, 16)
    assert np.allclose(O.jacobian(d, gam), Jfd, atol=1e-7)
    K = O.kernel_exact(d, gam)
    Kfd = np.linalg.inv(Jfd - np.eye(nat))
    assert np.allclose(K, Kfd, atol=1e-6 * np.abs(Kfd).max())
    # columns of J sum to zero (charge is conserved), so K maps sum-free residuals to sum-free steps
    assert np.allclose(O.jacobian(d, gam).sum(axis=0), 0.0, atol=1e-12)


def test_kernel_scf_reaches_the_mixing_fixed_point_in_fewer_iterations():
    # Eq. SCF_K with the rank-2 kernel against linear mixing (Section V.G, Fig. 6)
    s = synth.make_system(24, 1705, L=7.0)
    c = 1 - 1 / 0.06
    n_mix, it_mix = O.scf(s.R, s.L, s.Z, M, 0.06, tol=1e-10)
    n_k, it_k = O.scf_kernel(s.R, s.L, s.Z, M, 2, c, tol=1e-10)
    assert np.max(np.abs(n_k - n_mix)) < 1e-9
    assert it_k * 3 < it_mix, (it_k, it_mix)
    # a rank-0 kernel is linear mixing with alpha = 1 / (1 - c)
    n_0, it_0 = O.scf_kernel(s.R, s.L, s.Z, M, 0, c, tol=1e-10, max_iter=1000)
    assert it_0 == it_mix and np.max(np.abs(n_0 - n_mix)) < 1e-12


def test_accumulated_rank1_updates_keep_K_the_inverse_of_J_minus_I(tiny):
    # the carried kernel of the on-the-fly scheme stays (J - I)^-1 through any
    # sequence of updates (Eq. K_up), and each update makes J exact on its probe
    s, H0, gam, n = tiny
    nat, c = 8, -9.0
    K, J = np.eye(nat) / (c - 1.0), c * np.eye(nat)
    rng = np.random.default_rng(3)
    for k in range(5):
        nk = n + 0.01 * rng.normal(size=nat)
        d = O.density(O.hamiltonian(H0, gam, nk), M.beta, M.n_sq, 16)
        r = O.mulliken(d.D, s.Z) - nk
        K1, J1 = O.kernel_rank1_accumulate(K, J, r, lambda v: O.response(d, gam, v))
        v = K @ r
        v /= np.linalg.norm(v)
        assert np.allclose(J1 @ v, O.response(d, gam, v), atol=1e-12)
        K, J = K1, J1
        assert np.allclose(K, np.linalg.inv(J - np.eye(nat)), atol=1e-10 * np.abs(K).max())

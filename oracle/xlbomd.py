"""Plain FP64 CPU oracle of finite-temperature XL-BOMD on an orthogonal SCC-TB model.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` call this module; the CUDA library never does.  It
shares no code with the CUDA path; both read the same seeded inputs from
``synth``.

Everything here is written for clarity, not speed: the density matrix comes
from a full eigendecomposition, D = V g(eps) V^T, and the charge response from
the eigenbasis (divided differences), instead of the matrix recursions that the
CUDA path runs.

Paper: A. M. N. Niklasson, "Next generation extended Lagrangian first
principles molecular dynamics" (arXiv:1705.10845).  Each function names the
section / equation it follows.  Readings of points where the paper is silent:

* Model (Section VI uses SCC-DFTB, whose parameters are not available): an
  orthogonal s/p Slater-Koster tight-binding Hamiltonian with
  V(r) = t0 exp(-r/r_decay) S(r), a quintic C2 taper S on [r_taper, r_cut],
  periodic Ohno-Klopman Coulomb gamma (Ewald splitting; real-space part over
  the 27 images of the minimum-image vector).  The plain 27-image sum of the
  Ohno-Klopman kernel is indefinite on neutral charge vectors, which drives
  the ground state to +-4 e charges; the Ewald form is positive definite there.
* Pair repulsion: the model has none, and its atoms then fall into each other
  within a few hundred MD steps whatever the kernel; an optional Born-Mayer
  term A exp(-r/rho) S(r) over the image pairs (off by default, rep_A = 0)
  keeps long runs physical (A = 40 eV, rho = 0.3 A balances the band
  attraction near 1.5 A).
* Occupations: the recursive Fermi-operator expansion with n squarings
  (canonical density-matrix perturbation theory, the paper's Ref. ANiklasson15,
  cited in Section V.B) does not give the Fermi-Dirac function for finite n.
  Its exact scalar map is  g_n(e) = 1 / (1 + ((1+z)/(1-z))^(2^n)),
  z = beta (e - mu) / 2^(n+1), valid for |z| < 1 (derivation: the recursion
  x -> x^2 / (x^2 + (1-x)^2) squares the ratio x/(1-x)).  The oracle uses g_n.
  As n grows g_n tends to the Fermi-Dirac function of Section IV.B.
* Spin: every orbital holds two electrons; sum_i g_i = N_e / 2.
* Charges: q_I = 2 sum_{a in I} D_aa - Z_I (excess electrons on atom I).
* Kernel: J_0 = c I (Eq. JCI), K_0 = (c - 1)^-1 I (Eq. KCI); the rank-m
  kernel is rebuilt from K_0 every step with v_1 = K_0 r / |K_0 r| (Eq. v_1)
  and v_i = K_{i-1} r Gram-Schmidt orthonormalised against v_<i
  (Section V.F).  The exact kernel (Eq. KK) takes J from the responses to the
  N_at unit directions and is kept from t0 or recomputed every kernel_every
  steps (Section VI.A).  The accumulated kernel (end of Section V.F) carries
  K and J between steps with one rank-1 update per step, started at K_0 with
  no update at t0, where the residual is rounding noise.  The t0 ground state
  comes from linear mixing or from the kernel SCF of Eq. SCF_K.
* Integrator: velocity Verlet for R (Eq. Integration, with the typo in the
  position update read as R(t+dt) = R(t) + dt Rdot(t+dt/2)) and the
  dissipative Verlet of Eq. VRL_Damp for n with a K_max = 5, 6 or 7 row of
  Table I;
  dt^2 ndot = -kappa K (q - n).  The n history starts with every slot equal
  to n(t0).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erfc

KB_EV = 8.617333262e-5        # Boltzmann constant, eV/K
ACC = 9.648533e-3             # 1 eV/(amu A) in A/fs^2
KE_FACTOR = 1.0 / ACC         # 1 amu A^2/fs^2 in eV (= 103.6427)


class SpectrumError(ValueError):
    """|z| >= 1 for some eigenvalue: the recursive expansion is not defined."""


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------

@dataclass
class Model:
    """Orthogonal SCC-TB model (carbon-like s/p atoms)."""
    eps_s: float = -8.0
    eps_p: float = -3.0
    t0: tuple = (-2.5, -1.8, 1.2, -0.6)     # ss-sigma, sp-sigma, pp-sigma, pp-pi (eV)
    r_decay: float = 1.2                    # A
    r_cut: float = 5.0                      # A
    r_taper: float = 4.5                    # taper starts here (A)
    hubbard_U: float = 6.0                  # eV
    coulomb_k: float = 14.399645            # eV A
    rep_A: float = 0.0                      # pair repulsion A exp(-r/rho) S(r) (eV); 0 = off
    rep_rho: float = 0.3                    # A
    Te: float = 1000.0                      # K
    n_sq: int = 10                          # squarings of the recursive expansion

    @property
    def beta(self) -> float:
        return 1.0 / (KB_EV * self.Te)


@dataclass
class XLParams:
    """Integrator and kernel constants (Table I row K_max = 5)."""
    dt: float = 0.25                        # fs
    kappa: float = 1.82
    alpha: float = 0.018
    c: tuple = (-6.0, 14.0, -8.0, -3.0, 4.0, -1.0)
    rank_m: int = 2
    kernel_c: float = 0.0                   # J_0 = c I
    kernel_mode: str = "rank"               # "rank": rank-m every step; "exact": K = (J - I)^-1;
                                            # "accumulated": one rank-1 update per step of the carried K
    kernel_every: int = 0                   # exact: recompute every this many steps (0: kept from t0)
    mix_alpha: float = 0.5                  # linear mixing at t0
    scf_tol: float = 1e-10
    scf_max_iter: int = 1000

    @property
    def kmax(self) -> int:
        return len(self.c) - 1


# Table I (Section II.F): K_max, kappa, alpha, c_0..c_K
TABLE_I = {
    5: (1.82, 0.018, (-6, 14, -8, -3, 4, -1)),
    6: (1.84, 0.0055, (-14, 36, -27, -2, 12, -6, 1)),
    7: (1.86, 0.0016, (-36, 99, -88, 11, 32, -25, 8, -1)),
}


# --------------------------------------------------------------------------
# Model: Slater-Koster Hamiltonian H0 and Coulomb gamma
# --------------------------------------------------------------------------

def taper(r, r_on, r_cut):
    """C2 quintic switch S(r) = 1 - 10 s^3 + 15 s^4 - 6 s^5, s = (r-r_on)/(r_cut-r_on).

    Returns (S, dS/dr).  S = 1 below r_on, 0 above r_cut.
    """
    r = np.asarray(r, dtype=float)
    w = r_cut - r_on
    s = np.clip((r - r_on) / w, 0.0, 1.0)
    S = 1.0 - 10.0 * s**3 + 15.0 * s**4 - 6.0 * s**5
    dS = (-30.0 * s**2 + 60.0 * s**3 - 30.0 * s**4) / w
    return S, dS


def bond_integrals(r, model: Model):
    """V_k(r) = t0_k exp(-r / r_decay) S(r) for k = ss-sigma, sp-sigma, pp-sigma, pp-pi.

    Returns arrays V (..., 4) and dV/dr (..., 4).
    """
    r = np.asarray(r, dtype=float)
    S, dS = taper(r, model.r_taper, model.r_cut)
    e = np.exp(-r / model.r_decay)
    t0 = np.asarray(model.t0, dtype=float)
    V = t0 * (e * S)[..., None]
    dV = t0 * (e * (dS - S / model.r_decay))[..., None]
    return V, dV


def sk_blocks(d, model: Model):
    """Two-centre s/p blocks E_ab(d) and gradients dE_ab/dd for bond vectors d (P, 3).

    Orbital order [s, x, y, z].  Slater-Koster rules with direction cosines
    c = d / |d|:  E_ss = V_sss;  E_s,x = c_x V_sps;  E_x,s = -c_x V_sps;
    E_x,y = c_x c_y (V_pps - V_ppp) + delta_xy V_ppp.
    Returns E (P, 4, 4) and G (P, 4, 4, 3).
    """
    d = np.atleast_2d(np.asarray(d, dtype=float))
    P = d.shape[0]
    r = np.sqrt(np.sum(d * d, axis=1))
    c = d / r[:, None]
    V, dV = bond_integrals(r, model)
    Vss, Vsp, Vpps, Vppp = V.T
    dss, dsp, dpps, dppp = dV.T
    eye3 = np.eye(3)
    # dc_a/dd_g = (delta_ag - c_a c_g) / r
    dc = (eye3[None, :, :] - c[:, :, None] * c[:, None, :]) / r[:, None, None]

    E = np.zeros((P, 4, 4))
    G = np.zeros((P, 4, 4, 3))
    E[:, 0, 0] = Vss
    G[:, 0, 0, :] = dss[:, None] * c
    E[:, 0, 1:] = c * Vsp[:, None]
    E[:, 1:, 0] = -c * Vsp[:, None]
    gsp = dc * Vsp[:, None, None] + c[:, :, None] * (dsp[:, None] * c)[:, None, :]
    G[:, 0, 1:, :] = gsp
    G[:, 1:, 0, :] = -gsp
    dV_pp = Vpps - Vppp
    ddV_pp = dpps - dppp
    cc = c[:, :, None] * c[:, None, :]
    E[:, 1:, 1:] = cc * dV_pp[:, None, None] + eye3[None] * Vppp[:, None, None]
    # d(c_a c_b)/dd_g = dc[a,g] c_b + c_a dc[b,g]
    dcc = dc[:, :, None, :] * c[:, None, :, None] + c[:, :, None, None] * dc[:, None, :, :]
    G[:, 1:, 1:, :] = (dcc * dV_pp[:, None, None, None]
                       + cc[..., None] * (ddV_pp[:, None] * c)[:, None, None, :]
                       + eye3[None, :, :, None] * (dppp[:, None] * c)[:, None, None, :])
    return E, G


def image_pairs(R, L, r_cut):
    """All ordered atom pairs (I, J, T) with |R_J + T L - R_I| < r_cut, T in {-1,0,1}^3.

    Positions must lie in [0, L) and L > r_cut, so that no other image can be
    inside the cutoff.  The pair (I, I, T=0) is excluded.
    Returns I (P,), J (P,), d (P, 3).
    """
    if L <= r_cut:
        raise ValueError("box side must exceed the hopping cutoff")
    R = np.asarray(R, dtype=float)
    nat = R.shape[0]
    Is, Js, ds = [], [], []
    raw = R[None, :, :] - R[:, None, :]          # raw[I, J] = R_J - R_I
    for T in itertools.product((-1, 0, 1), repeat=3):
        d = raw + np.asarray(T, dtype=float) * L
        r2 = np.sum(d * d, axis=2)
        mask = r2 < r_cut * r_cut
        if T == (0, 0, 0):
            mask[np.arange(nat), np.arange(nat)] = False
        I, J = np.nonzero(mask)
        Is.append(I)
        Js.append(J)
        ds.append(d[I, J])
    return np.concatenate(Is), np.concatenate(Js), np.concatenate(ds)


def build_H0(R, L, model: Model):
    """Charge-independent Hamiltonian H0 (N x N, N = 4 natoms), Section VI model.

    H0_{Ia,Jb} = delta_IJ delta_ab eps_a + sum_T E_ab(R_J + T L - R_I).
    """
    nat = len(R)
    N = 4 * nat
    H0 = np.zeros((N, N))
    onsite = np.array([model.eps_s, model.eps_p, model.eps_p, model.eps_p])
    H0[np.arange(N), np.arange(N)] = np.tile(onsite, nat)
    I, J, d = image_pairs(R, L, model.r_cut)
    if len(I):
        E, _ = sk_blocks(d, model)
        H4 = H0.reshape(nat, 4, nat, 4)
        np.add.at(H4, (I, slice(None), J, slice(None)), E)
    return H0


def min_image(d, L):
    """Minimum-image vector: d - L rint(d / L)."""
    return d - L * np.rint(d / L)


def ewald_setup(L, model: Model, eta=None):
    """Ewald splitting eta (default 4 / L) and the reciprocal vectors G = 2 pi h / L,
    h != 0, |G| <= 2 eta * 6.07 (exp(-G^2 / 4 eta^2) < 1e-16).

    Returns (eta, G (nG, 3), A (nG,)) with A = 4 pi / V exp(-G^2/(4 eta^2)) / G^2.
    """
    if eta is None:
        eta = 4.0 / L
    gmax = 2.0 * eta * 6.07
    hmax = int(math.ceil(gmax * L / (2.0 * math.pi)))
    hs = np.array(list(itertools.product(range(-hmax, hmax + 1), repeat=3)), dtype=float)
    G = 2.0 * math.pi * hs / L
    G2 = np.sum(G * G, axis=1)
    keep = (G2 > 0.0) & (G2 <= gmax * gmax)
    G, G2 = G[keep], G2[keep]
    A = 4.0 * math.pi / L**3 * np.exp(-G2 / (4.0 * eta * eta)) / G2
    return eta, G, A


def _ok_real(r, a, eta):
    """Real-space Ewald term erfc(eta r)/r + [1/sqrt(r^2+a^2) - 1/r]; its r -> 0 limit
    is 1/a - 2 eta / sqrt(pi)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = erfc(eta * r) / r + (1.0 / np.sqrt(r * r + a * a) - 1.0 / r)
    return np.where(r == 0.0, 1.0 / a - 2.0 * eta / math.sqrt(math.pi), t)


def _ok_real_dr(r, a, eta):
    """d/dr of the real-space term (r > 0)."""
    return (-erfc(eta * r) / r**2 - 2.0 * eta / math.sqrt(math.pi) * np.exp(-(eta * r) ** 2) / r
            - r / (r * r + a * a) ** 1.5 + 1.0 / r**2)


def build_gamma(R, L, model: Model, eta=None):
    """Periodic Ohno-Klopman Coulomb matrix gamma_IJ (Section VI model).

    gamma = k [ Ewald sum of the point Coulomb 1/r over the whole lattice
                (conducting boundary, neutralising background)
              + sum over the 27 images d + T L (T in {-1,0,1}^3) of the
                minimum-image vector d = R_J - R_I of the Ohno-Klopman
                short-range correction 1/sqrt(r^2 + a^2) - 1/r ],  a = k / U.
    The Ewald part is split into erfc(eta r)/r over the same 27 images and the
    reciprocal sum sum_G A_G cos(G.d).  The I = J, T = 0 term is
    1/a - 2 eta/sqrt(pi): the on-site Hubbard value U/k plus the Gaussian
    self-interaction correction.  For neutral charge vectors the result does
    not depend on eta.
    """
    R = np.asarray(R, dtype=float)
    k = model.coulomb_k
    if k == 0.0:
        return np.zeros((len(R), len(R)))
    a = k / model.hubbard_U
    eta, G, A = ewald_setup(L, model, eta)
    dmin = min_image(R[None, :, :] - R[:, None, :], L)
    gam = np.zeros((len(R), len(R)))
    for T in itertools.product((-1, 0, 1), repeat=3):
        d = dmin + np.asarray(T, dtype=float) * L
        gam += _ok_real(np.sqrt(np.sum(d * d, axis=2)), a, eta)
    # reciprocal part: cos(G.(R_J - R_I)) = cos(G.R_I) cos(G.R_J) + sin(G.R_I) sin(G.R_J)
    ph = R @ G.T
    C, S = np.cos(ph), np.sin(ph)
    gam += (C * A) @ C.T + (S * A) @ S.T
    return k * gam


def build_gamma_grad(R, L, model: Model):
    """d gamma_IJ / d R_J (natoms, natoms, 3); d gamma_IJ / d R_I is its negative."""
    R = np.asarray(R, dtype=float)
    k = model.coulomb_k
    dmin = min_image(R[None, :, :] - R[:, None, :], L)
    out = np.zeros(dmin.shape)
    if k == 0.0:
        return out
    a = k / model.hubbard_U
    eta, G, A = ewald_setup(L, model)
    for T in itertools.product((-1, 0, 1), repeat=3):
        d = dmin + np.asarray(T, dtype=float) * L
        r = np.sqrt(np.sum(d * d, axis=2))
        with np.errstate(divide="ignore", invalid="ignore"):
            fr = np.where(r > 0.0, _ok_real_dr(r, a, eta) / r, 0.0)
        out += fr[..., None] * d
    # reciprocal part: -sum_G A_G G sin(G.(R_J - R_I)),
    # sin(G.(R_J - R_I)) = cos(G.R_I) sin(G.R_J) - sin(G.R_I) cos(G.R_J)
    ph = R @ G.T
    C, S = np.cos(ph), np.sin(ph)
    for c in range(3):
        w = A * G[:, c]
        out[..., c] -= (C * w) @ S.T - (S * w) @ C.T
    return k * out


def hamiltonian(H0, gamma, n):
    """H[n] = H0 + diag over orbitals of (gamma n)_I (linearised Kohn-Sham H, Section IV.A)."""
    H = H0.copy()
    N = H.shape[0]
    pot = np.repeat(gamma @ np.asarray(n, dtype=float), 4)
    H[np.arange(N), np.arange(N)] += pot
    return H


# --------------------------------------------------------------------------
# Density matrix: D = V g_n(eps) V^T, mu from sum g = N_occ (Section IV.B)
# --------------------------------------------------------------------------

def gn_exponent(eps, mu, beta, n_sq):
    """y = ln(((1+z)/(1-z))^(2^n)) = 2^(n+1) artanh z, z = beta (eps - mu) / 2^(n+1)."""
    z = beta * (np.asarray(eps, dtype=float) - mu) / 2.0 ** (n_sq + 1)
    if np.any(np.abs(z) >= 1.0):
        raise SpectrumError("|z| >= 1: spectrum too wide for this number of squarings")
    return 2.0 ** (n_sq + 1) * np.arctanh(z), z


def occupations(eps, mu, beta, n_sq):
    """g_n(eps - mu) = 1 / (1 + exp(y)): the recursive expansion's occupation."""
    y, _ = gn_exponent(eps, mu, beta, n_sq)
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(y))


def occupations_dmu(eps, mu, beta, n_sq):
    """d g_n / d mu = beta g (1 - g) / (1 - z^2)."""
    y, z = gn_exponent(eps, mu, beta, n_sq)
    with np.errstate(over="ignore"):
        g = 1.0 / (1.0 + np.exp(y))
    return beta * g * (1.0 - g) / (1.0 - z * z)


def solve_mu(eps, beta, n_sq, n_occ, tol=1e-13):
    """Chemical potential with sum_i g_n(eps_i - mu) = n_occ (bisection, then Newton)."""
    eps = np.asarray(eps, dtype=float)
    half = 2.0 ** (n_sq + 1) / beta * (1.0 - 1e-12)
    lo, hi = eps.max() - half, eps.min() + half
    if lo >= hi:
        raise SpectrumError("no mu keeps every |z| < 1")
    f_lo = occupations(eps, lo, beta, n_sq).sum() - n_occ
    f_hi = occupations(eps, hi, beta, n_sq).sum() - n_occ
    if f_lo > 0 or f_hi < 0:
        raise SpectrumError("occupation target not bracketed in the valid mu window")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = occupations(eps, mid, beta, n_sq).sum() - n_occ
        if fm > 0:
            hi = mid
        else:
            lo = mid
        if hi - lo < 1e-13:
            break
    mu = 0.5 * (lo + hi)
    for _ in range(20):
        dn = occupations(eps, mu, beta, n_sq).sum() - n_occ
        if abs(dn) < tol:
            break
        mu -= dn / occupations_dmu(eps, mu, beta, n_sq).sum()
    return mu


@dataclass
class Density:
    eps: np.ndarray
    V: np.ndarray
    mu: float
    f: np.ndarray
    D: np.ndarray
    beta: float
    n_sq: int


def density(H, beta, n_sq, n_occ):
    """D = V diag(g_n(eps - mu)) V^T from a full eigendecomposition of H."""
    eps, V = np.linalg.eigh(H)
    mu = solve_mu(eps, beta, n_sq, n_occ)
    f = occupations(eps, mu, beta, n_sq)
    D = (V * f) @ V.T
    return Density(eps=eps, V=V, mu=mu, f=f, D=D, beta=beta, n_sq=n_sq)


def fermi_dirac(eps, mu, beta):
    """Fermi-Dirac occupation [exp(beta (eps - mu)) + 1]^-1 (Section IV.B)."""
    x = beta * (np.asarray(eps, dtype=float) - mu)
    with np.errstate(over="ignore"):
        return 1.0 / (np.exp(x) + 1.0)


def mulliken(D, Z):
    """q_I = 2 sum_{a in I} D_aa - Z_I (Mulliken net charges for an orthogonal basis)."""
    nat = len(Z)
    return 2.0 * np.diag(D).reshape(nat, 4).sum(axis=1) - np.asarray(Z, dtype=float)


def entropy_terms(dens: Density):
    """s(f_i) = -f ln f - (1-f) ln(1-f) (Eq. S_entropy) for every eigenstate.

    With y = ln((1-f)/f) it equals ln(1 + exp(-|y|)) + |y| / (1 + exp(|y|)),
    which never takes the log of zero.
    """
    y, _ = gn_exponent(dens.eps, dens.mu, dens.beta, dens.n_sq)
    a = np.abs(y)
    with np.errstate(over="ignore"):
        return np.log1p(np.exp(-a)) + a / (1.0 + np.exp(a))


# --------------------------------------------------------------------------
# Charge response (Section V.B, canonical perturbation theory) in the eigenbasis
# --------------------------------------------------------------------------

def _log_cosh(x):
    a = np.abs(x)
    return a + np.log1p(np.exp(-2.0 * a)) - math.log(2.0)


def divided_differences(dens: Density):
    """P_ij = (g_i - g_j) / (eps_i - eps_j), and -dg/dmu on the diagonal.

    Written cancellation-free: with g = (1 - tanh(y/2)) / 2,
    g_i - g_j = -sinh((y_i - y_j)/2) / (2 cosh(y_i/2) cosh(y_j/2)) and
    y_i - y_j = 2^(n+1) artanh((z_i - z_j) / (1 - z_i z_j)).
    """
    eps, mu, beta, n = dens.eps, dens.mu, dens.beta, dens.n_sq
    y, z = gn_exponent(eps, mu, beta, n)
    de = eps[:, None] - eps[None, :]
    dz = beta * de / 2.0 ** (n + 1)
    dy = 2.0 ** (n + 1) * np.arctanh(dz / (1.0 - z[:, None] * z[None, :]))
    lc = _log_cosh(0.5 * y)
    a = 0.5 * np.abs(dy)
    with np.errstate(divide="ignore", invalid="ignore"):
        log_sinh = a + np.log(-np.expm1(-2.0 * a)) - math.log(2.0)
        num = -np.sign(dy) * np.exp(log_sinh - lc[:, None] - lc[None, :]) / 2.0
        P = num / de
    gmu = occupations_dmu(eps, mu, beta, n)
    deg = (de == 0.0) | ~np.isfinite(P)
    Pdeg = -0.5 * (gmu[:, None] + gmu[None, :])
    P = np.where(deg, Pdeg, P)
    return P, gmu


def response(dens: Density, gamma, v, P=None, gmu=None):
    """Charge response w = d q[n + lambda v] / d lambda at lambda = 0.

    H1 = diag over orbitals of (gamma v)_I; in the eigenbasis
    dD = V [ (V^T H1 V) o P + dmu diag(dg/dmu) ] V^T with dmu fixed by
    Tr dD = 0 (the electron count is held); w_I = 2 sum_{a in I} dD_aa.
    """
    if P is None:
        P, gmu = divided_differences(dens)
    nat = gamma.shape[0]
    h = np.repeat(gamma @ np.asarray(v, dtype=float), 4)
    Ht = dens.V.T @ (h[:, None] * dens.V)
    A = Ht * P
    dmu = -np.trace(A) / gmu.sum()
    A[np.diag_indices_from(A)] += dmu * gmu
    dD_diag = np.sum((dens.V @ A) * dens.V, axis=1)
    return 2.0 * dD_diag.reshape(nat, 4).sum(axis=1)


# --------------------------------------------------------------------------
# Low-rank kernel (Section V.D-V.F, Eqs. KCI, JCI, K_up, v_1)
# --------------------------------------------------------------------------

def apply_kernel(x, V, W, c):
    """K_m x for J_m = c I + U V^T, U = W - c V (V orthonormal): the Woodbury form
    of the Sherman-Morrison sequence of Eq. K_up.

    K_m x = [x - U ((c-1) I_m + V^T U)^-1 V^T x] / (c - 1).
    """
    x = np.asarray(x, dtype=float)
    if len(V) == 0:
        return x / (c - 1.0)
    Vm = np.array(V).T
    Um = np.array(W).T - c * Vm
    m = Vm.shape[1]
    S = (c - 1.0) * np.eye(m) + Vm.T @ Um
    return (x - Um @ np.linalg.solve(S, Vm.T @ x)) / (c - 1.0)


def kernel_rank_m(r, m, c, respond, dep_tol=1e-12):
    """Rank-m kernel acting on the residual r = q[n] - n.

    v_1 = K_0 r / |K_0 r| (Eq. v_1); v_i = K_{i-1} r orthonormalised against
    v_<i by two Gram-Schmidt passes (Section V.F); w_i = respond(v_i) is the
    response of Eq. K_up.  When less than dep_tol of K_{i-1} r is left after
    the projection, K_{i-1} r already lies in the span of the earlier probes,
    further probes cannot change K r, and the sequence stops.
    Returns (K_m r, V, W).
    """
    r = np.asarray(r, dtype=float)
    V, W = [], []
    for _ in range(m):
        v = apply_kernel(r, V, W, c)
        n0 = np.linalg.norm(v)
        for _pass in range(2):
            for vj in V:
                v = v - (vj @ v) * vj
        nv = np.linalg.norm(v)
        if n0 == 0.0 or not np.isfinite(nv) or nv <= dep_tol * n0:
            break
        v = v / nv
        V.append(v)
        W.append(respond(v))
    return apply_kernel(r, V, W, c), V, W


def kernel_sherman_morrison_dense(c, V, W):
    """The sequence of Eq. K_up with explicit matrices (tiny systems only).

    K_0 = (c I - I)^-1, J_0 = c I; for each i:  u_i = w_i - J_{i-1} v_i,
    J_i = J_{i-1} + u_i v_i^T,
    K_i = K_{i-1} - K_{i-1} u_i v_i^T K_{i-1} / (1 + v_i^T K_{i-1} u_i).
    """
    nat = len(V[0]) if V else 0
    J = c * np.eye(nat)
    K = np.linalg.inv(J - np.eye(nat))
    for v, w in zip(V, W):
        u = w - J @ v
        J = J + np.outer(u, v)
        K = K - (K @ np.outer(u, v) @ K) / (1.0 + v @ K @ u)
    return K, J


def jacobian(dens: Density, gamma, P=None, gmu=None):
    """J = dq/dn (N_at x N_at): column I is the response to the unit direction e_I, i.e. the
    N_at orthonormal probes with which the sequence of Eq. K_up ends at the exact kernel."""
    if P is None:
        P, gmu = divided_differences(dens)
    nat = gamma.shape[0]
    J = np.zeros((nat, nat))
    for I in range(nat):
        e = np.zeros(nat)
        e[I] = 1.0
        J[:, I] = response(dens, gamma, e, P, gmu)
    return J


def kernel_rank1_accumulate(K, J, r, respond):
    """One on-the-fly update of a carried kernel (end of Section V.F): v = K r / |K r|,
    w = respond(v), u = w - J v, J <- J + u v^T, K <- K - K u v^T K / (1 + v^T K u) (Eq. K_up).
    K stays (J - I)^-1.  Returns (K, J); unchanged when K r = 0."""
    v = K @ r
    nv = np.linalg.norm(v)
    if nv == 0.0 or not np.isfinite(nv):
        return K, J
    v = v / nv
    u = respond(v) - J @ v
    J = J + np.outer(u, v)
    Ku = K @ u
    K = K - np.outer(Ku, v @ K) / (1.0 + v @ Ku)
    return K, J


def kernel_exact(dens: Density, gamma):
    """The exact kernel K = (J - I)^-1 of Eq. KK, J = dq/dn."""
    J = jacobian(dens, gamma)
    return np.linalg.inv(J - np.eye(J.shape[0]))


# --------------------------------------------------------------------------
# Energy and forces (Section IV.B-IV.C, Eq. EqMotFT)
# --------------------------------------------------------------------------

def repulsion(R, L, model: Model):
    """Pair repulsion E_rep = 1/2 sum over ordered image pairs of A exp(-r/rho) S(r), with the
    hoppings' taper S; returns (E_rep, dE_rep/dR (N_at x 3)).  Zero when rep_A = 0."""
    R = np.asarray(R, dtype=float)
    g = np.zeros_like(R)
    if model.rep_A == 0.0:
        return 0.0, g
    I, J, d = image_pairs(R, L, model.r_cut)
    r = np.sqrt(np.sum(d * d, axis=1))
    S, dS = taper(r, model.r_taper, model.r_cut)
    e = model.rep_A * np.exp(-r / model.rep_rho)
    de = e * (dS - S / model.rep_rho)                # d(e S)/dr
    u = (0.5 * de / r)[:, None] * d                  # d/d(R_J) of half the pair term
    np.add.at(g, J, u)
    np.add.at(g, I, -u)
    return 0.5 * float(np.sum(e * S)), g


def free_energy(H0, gamma, dens: Density, q, n, e_rep=0.0):
    """Shadow free energy Omega[n](R) of the SCC-TB model.

    Omega = 2 Tr[D H0] + 1/2 sum_IJ (2 q_I - n_I) gamma_IJ n_J
            - 2 kB Te sum_i s(f_i) + E_rep.
    Returns (Omega, parts dict).
    """
    n = np.asarray(n, dtype=float)
    band = 2.0 * np.sum(dens.D * H0)
    coul = 0.5 * np.dot(2.0 * q - n, gamma @ n)
    S = float(np.sum(entropy_terms(dens)))
    ent = -2.0 * S / dens.beta
    return band + coul + ent + e_rep, dict(band=band, coulomb=coul, entropy=ent, S=S, repulsion=e_rep)


def forces(R, L, model: Model, D, q, n, gamma_grad=None):
    """F_I = -dOmega/dR_I at fixed n (Eq. EqMotFT), Hellmann-Feynman form.

    Band part: -2 sum_ab D_ba dH0_ab/dR_I over every ordered image pair.
    Coulomb part: -1/2 sum_JK (2 q_J - n_J) n_K d gamma_JK / dR_I.
    """
    R = np.asarray(R, dtype=float)
    nat = len(R)
    dO = np.zeros((nat, 3))
    I, J, d = image_pairs(R, L, model.r_cut)
    if len(I):
        _, G = sk_blocks(d, model)
        D4 = D.reshape(nat, 4, nat, 4)
        Dblk = D4[I, :, J, :]                       # (P, 4, 4): D_{Ia, Jb}
        g = np.einsum("pab,pabk->pk", Dblk, G)      # sum_ab D_{Ia,Jb} dE_ab/dd
        # block (I, J) depends on d = R_J + T L - R_I
        np.add.at(dO, J, 2.0 * g)
        np.add.at(dO, I, -2.0 * g)
    if gamma_grad is None:
        gamma_grad = build_gamma_grad(R, L, model)
    a = 2.0 * np.asarray(q) - np.asarray(n)
    n = np.asarray(n, dtype=float)
    w = 0.5 * a[:, None] * n[None, :]              # weight of d gamma_IJ
    np.fill_diagonal(w, 0.0)
    t = w[..., None] * gamma_grad                   # contributes +t to R_J, -t to R_I
    dO += t.sum(axis=0)
    dO -= t.sum(axis=1)
    dO += repulsion(R, L, model)[1]
    return -dO


# --------------------------------------------------------------------------
# One electronic-structure evaluation at (R, n)
# --------------------------------------------------------------------------

@dataclass
class Evaluation:
    H0: np.ndarray
    gamma: np.ndarray
    H: np.ndarray
    dens: Density
    q: np.ndarray
    r: np.ndarray
    F: np.ndarray
    Omega: float
    parts: dict
    Kr: np.ndarray | None = None
    V: list = field(default_factory=list)
    W: list = field(default_factory=list)


def evaluate(R, L, Z, n, model: Model, xl: XLParams | None = None, with_kernel=True,
             with_forces=True):
    """H[n], D, q, residual, forces, Omega and (optionally) K r at one state."""
    R = np.asarray(R, dtype=float)
    Z = np.asarray(Z, dtype=float)
    n = np.asarray(n, dtype=float)
    H0 = build_H0(R, L, model)
    gam = build_gamma(R, L, model)
    H = hamiltonian(H0, gam, n)
    n_occ = 0.5 * Z.sum()
    dens = density(H, model.beta, model.n_sq, n_occ)
    q = mulliken(dens.D, Z)
    r = q - n
    F = forces(R, L, model, dens.D, q, n) if with_forces else None
    Om, parts = free_energy(H0, gam, dens, q, n, repulsion(R, L, model)[0])
    ev = Evaluation(H0=H0, gamma=gam, H=H, dens=dens, q=q, r=r, F=F, Omega=Om, parts=parts)
    if with_kernel and xl is not None:
        P, gmu = divided_differences(dens)
        ev.Kr, ev.V, ev.W = kernel_rank_m(r, xl.rank_m, xl.kernel_c,
                                          lambda v: response(dens, gam, v, P, gmu))
    return ev


def charges_at(R, L, Z, n, model: Model):
    """q[n] at fixed R (for finite-difference checks)."""
    H0 = build_H0(R, L, model)
    gam = build_gamma(R, L, model)
    dens = density(hamiltonian(H0, gam, n), model.beta, model.n_sq, 0.5 * np.sum(Z))
    return mulliken(dens.D, Z)


# --------------------------------------------------------------------------
# Initial ground state (Eq. IBC) and the integrator (Eqs. Integration, VRL_Damp)
# --------------------------------------------------------------------------

def scf(R, L, Z, model: Model, mix_alpha, tol=1e-10, max_iter=1000, n0=None):
    """Linear-mixing SCF  n <- n + alpha (q[n] - n)  until max |q - n| < tol.

    This is Eq. SCF_K with K = K_0 = (c - 1)^-1 I, alpha = 1 / (1 - c).
    Returns (n, iterations) for the last n, whose residual is below tol;
    raises RuntimeError when it does not converge.
    """
    H0 = build_H0(R, L, model)
    gam = build_gamma(R, L, model)
    n_occ = 0.5 * np.sum(Z)
    n = np.zeros(len(Z)) if n0 is None else np.array(n0, dtype=float)
    for it in range(1, max_iter + 1):
        dens = density(hamiltonian(H0, gam, n), model.beta, model.n_sq, n_occ)
        q = mulliken(dens.D, Z)
        res = q - n
        if np.max(np.abs(res)) < tol:
            return n, it
        if not np.all(np.isfinite(res)) or np.max(np.abs(res)) > 1e3:
            raise RuntimeError("SCF diverged")
        n = n + mix_alpha * res
    raise RuntimeError("SCF did not converge")


def scf_kernel(R, L, Z, model: Model, rank_m, kernel_c, tol=1e-10, max_iter=200, n0=None):
    """Kernel SCF of Eq. SCF_K: n_{j+1} = n_j - K_j (q[n_j] - n_j), with K_j the rank-m kernel
    (Section V.F: v_1 from K_0 = (c - 1)^-1 I, later probes orthonormalised) built at n_j.
    Returns (n, iterations) for the last n, whose residual is below tol."""
    H0 = build_H0(R, L, model)
    gam = build_gamma(R, L, model)
    n_occ = 0.5 * np.sum(Z)
    n = np.zeros(len(Z)) if n0 is None else np.array(n0, dtype=float)
    for it in range(1, max_iter + 1):
        dens = density(hamiltonian(H0, gam, n), model.beta, model.n_sq, n_occ)
        res = mulliken(dens.D, Z) - n
        if np.max(np.abs(res)) < tol:
            return n, it
        if not np.all(np.isfinite(res)) or np.max(np.abs(res)) > 1e3:
            raise RuntimeError("SCF diverged")
        P, gmu = divided_differences(dens)
        Kr, _, _ = kernel_rank_m(res, rank_m, kernel_c, lambda v: response(dens, gam, v, P, gmu))
        n = n - Kr
    raise RuntimeError("SCF did not converge")


def choose_mix_alpha(R, L, Z, model: Model, candidates=None, tol=1e-10, max_iter=400):
    """Linear-mixing coefficient with the fewest SCF iterations (Section VI: the
    constants are tuned once for the fastest initial ground state, to within 0.1).

    The scan runs over 0.1, 0.2, ..., 1.0; when none of them converges (strong
    charge sloshing) it runs over 0.01, 0.02, ..., 0.09.  Returns (alpha, iters).
    """
    grids = [candidates] if candidates is not None else [
        [round(0.1 * k, 2) for k in range(1, 11)],
        [round(0.01 * k, 2) for k in range(1, 10)],
    ]
    for grid in grids:
        best = None
        for a in grid:
            try:
                _, it = scf(R, L, Z, model, a, tol=tol, max_iter=max_iter)
            except (RuntimeError, SpectrumError):
                continue
            if best is None or it < best[1]:
                best = (a, it)
        if best is not None:
            return best
    raise RuntimeError("no mixing coefficient converged")


@dataclass
class MDState:
    R: np.ndarray
    V: np.ndarray
    nhist: np.ndarray      # (kmax+1, natoms): n(t), n(t-dt), ..., n(t-kmax dt)
    F: np.ndarray
    Kr: np.ndarray
    step: int = 0
    K: np.ndarray | None = None     # exact or accumulated kernel carried between steps
    J: np.ndarray | None = None     # accumulated mode: the Jacobian estimate with K = (J - I)^-1


def kinetic_energy(V, mass):
    return 0.5 * mass * float(np.sum(V * V)) * KE_FACTOR


def wrap(R, L):
    return R - L * np.floor(R / L)


def n_update(nhist, Kr, xl: XLParams):
    """Eq. VRL_Damp: n(t+dt) = 2n(t) - n(t-dt) - kappa K r + alpha sum_k c_k n(t - k dt)."""
    diss = sum(ck * nhist[k] for k, ck in enumerate(xl.c))
    return 2.0 * nhist[0] - nhist[1] - xl.kappa * Kr + xl.alpha * diss


def md_init(sys_R, sys_V, L, Z, mass, model: Model, xl: XLParams, n0=None):
    """t0: SCF ground state (Eq. IBC), forces and K r there; history filled with n(t0)."""
    R = wrap(np.asarray(sys_R, dtype=float), L)
    if n0 is None:
        n0, _ = scf(R, L, Z, model, xl.mix_alpha, tol=xl.scf_tol, max_iter=xl.scf_max_iter)
    full = xl.kernel_mode in ("exact", "accumulated")
    ev = evaluate(R, L, Z, n0, model, xl, with_kernel=not full)
    K = J = None
    if xl.kernel_mode == "exact":
        K = kernel_exact(ev.dens, ev.gamma)
    elif xl.kernel_mode == "accumulated":
        # the carried kernel starts as K_0 = (c - 1)^-1 I, J_0 = c I; the first rank-1 update
        # comes with the first MD step: at the SCF ground state r is rounding noise, and a
        # probe along it would keep that noise in K
        nat = len(n0)
        c = xl.kernel_c
        K, J = np.eye(nat) / (c - 1.0), c * np.eye(nat)
    if full:
        ev.Kr = K @ ev.r
    nh = np.tile(np.asarray(n0, dtype=float), (xl.kmax + 1, 1))
    st = MDState(R=R, V=np.array(sys_V, dtype=float), nhist=nh, F=ev.F, Kr=ev.Kr, K=K, J=J)
    return st, ev


def md_step(st: MDState, L, Z, mass, model: Model, xl: XLParams):
    """One XL-BOMD step (Eqs. Integration and VRL_Damp, in that order):
    half kick, drift and wrap, n update with K r(t), new forces and K r at
    t + dt, half kick."""
    dt = xl.dt
    Vh = st.V + 0.5 * dt * st.F / mass * ACC
    R = wrap(st.R + dt * Vh, L)
    n_new = n_update(st.nhist, st.Kr, xl)
    step = st.step + 1
    full = xl.kernel_mode in ("exact", "accumulated")
    ev = evaluate(R, L, Z, n_new, model, xl, with_kernel=not full)
    K, J = st.K, st.J
    if xl.kernel_mode == "exact":
        # the full kernel of the t0 state, recomputed every kernel_every steps (Section VI.A, Figs. 3, 5)
        if xl.kernel_every > 0 and step % xl.kernel_every == 0:
            K = kernel_exact(ev.dens, ev.gamma)
    elif xl.kernel_mode == "accumulated":
        P, gmu = divided_differences(ev.dens)
        K, J = kernel_rank1_accumulate(K, J, ev.r, lambda v: response(ev.dens, ev.gamma, v, P, gmu))
    if full:
        ev.Kr = K @ ev.r
    V = Vh + 0.5 * dt * ev.F / mass * ACC
    nh = np.vstack([n_new[None, :], st.nhist[:-1]])
    return MDState(R=R, V=V, nhist=nh, F=ev.F, Kr=ev.Kr, step=step, K=K, J=J), ev

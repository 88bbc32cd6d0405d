"""Error statuses of the C ABI that the host decides (GPU, through the C ABI).

Each case drives one host-side decision of the library to its error status on
a small system: the spectral bound of the expansion (ERR_SPECTRUM), the
iteration budgets of the chemical-potential search and of the t0 SCF
(ERR_NOT_CONVERGED) and the residual threshold of an MD step (ERR_DIVERGED).
Every failure is made on the host (a parameter, never a device fault); the
status must be sticky until xlbomd_clear_error, and the context must stay
usable afterwards.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ALPHA_MIX = 0.06


@pytest.fixture(scope="module")
def X():
    import paper_1705_10845_gb300 as X
    X.build.build()
    X.load()
    return X


def system():
    s = synth.make_system(24, 1705, L=7.0)
    return s, dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)


def status_of(X, fn):
    with pytest.raises(X.XlbomdError) as ei:
        fn()
    return ei.value.status


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_spectrum_bound_reported(X, prec):
    # one squaring at 1000 K: beta (e - mu) / 2^(n+1) is far above 1 for a ~20 eV wide spectrum,
    # so the expansion cannot represent the occupations and the density is refused
    _, sd = system()
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, n_sq=1, prec=prec,
                         mu_tol=1e-9 if prec == "fp64" else 1e-3)
    with X.Context(p, [sd]) as ctx:
        assert status_of(X, lambda: ctx.density(0)) == -5
        # sticky: the next call returns the status without doing work
        assert status_of(X, lambda: ctx.build_H(0)) == -5
        assert b"2^(n+1)" in ctx._lib.xlbomd_last_error(ctx.h)
        assert ctx._lib.xlbomd_clear_error(ctx.h) == 0
        ctx.build_H(0)           # usable again once cleared


def test_mu_iteration_budget_reported(X):
    # one Newton pass from the middle of the Gershgorin interval cannot reach |beta dmu| < 1e-9
    _, sd = system()
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, mu_max_iter=1)
    with X.Context(p, [sd]) as ctx:
        assert status_of(X, lambda: ctx.density(0)) == -4
        assert b"chemical potential" in ctx._lib.xlbomd_last_error(ctx.h)
        assert ctx._lib.xlbomd_clear_error(ctx.h) == 0
    # the same system with the default budget converges
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX)
    with X.Context(p, [sd]) as ctx:
        ctx.density(0)
        assert abs(ctx.get(0, X.Q).sum()) < 1e-9


def test_scf_iteration_budget_reported(X):
    _, sd = system()
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, scf_max_iter=1)
    with X.Context(p, [sd]) as ctx:
        assert status_of(X, lambda: ctx.scf(0)) == -4
        assert b"SCF did not converge" in ctx._lib.xlbomd_last_error(ctx.h)


def test_divergence_threshold_reported(X):
    # after the t0 SCF the first MD step leaves a residual |q - n| of ~1e-4 e, far above a
    # threshold of 1e-14 e, so xlbomd_step reports the run as diverged
    _, sd = system()
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1 - 1 / ALPHA_MIX, diverge_tol=1e-14)
    with X.Context(p, [sd]) as ctx:
        ctx.scf(0)
        assert status_of(X, lambda: ctx.step(1)) == -6
        assert b"residual" in ctx._lib.xlbomd_last_error(ctx.h)
        assert status_of(X, lambda: ctx.get(0, X.RES)) == -6   # refused while the status is set
        assert ctx._lib.xlbomd_clear_error(ctx.h) == 0
        res = ctx.get(0, X.RES)
        assert np.all(np.isfinite(res)) and np.max(np.abs(res)) > 1e-14

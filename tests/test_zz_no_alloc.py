"""xlbomd_response_noalloc against xlbomd_response (GPU, through the C ABI).

The no-allocation entry point serves callers that may not allocate device
memory while they run; its work memory is a static device array shared by all
calls.  It must give the same charge response as the allocating entry point,
within the FP64 tolerance of the other response tests, on two calls in a row
(the second call reuses the array the first one left behind).  This file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ALPHA_MIX = 0.06


@pytest.fixture(scope="module")
def X():
    import paper_1705_10845_gb300 as X
    X.build.build()
    lib = X.load()
    lib.xlbomd_response_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.xlbomd_response_noalloc.restype = ctypes.c_int
    return X


def test_noalloc_response_matches_allocating_entry_point(X):
    import torch
    s = synth.make_system(24, 1705, L=7.0)
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1.0 - 1.0 / ALPHA_MIX)
    rng = np.random.default_rng(7)
    n = rng.normal(scale=0.02, size=s.natoms)
    n -= n.mean()
    sysd = dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)
    with X.Context(p, [sysd]) as ctx:
        ctx.set(0, X.N, n)
        ctx.build_H(0)
        ctx.density(0)
        lib = ctx._lib
        for call in range(2):
            v = rng.normal(size=s.natoms)
            v -= v.mean()
            v /= np.linalg.norm(v)
            vd = torch.tensor(v, dtype=torch.float64, device="cuda")
            w_ref = torch.zeros_like(vd)
            w_new = torch.full_like(vd, float("nan"))
            ctx.response(0, vd.data_ptr(), w_ref.data_ptr())
            st = lib.xlbomd_response_noalloc(ctx.h, 0, ctypes.c_void_p(vd.data_ptr()),
                                             ctypes.c_void_p(w_new.data_ptr()))
            assert st == 0, lib.xlbomd_last_error(ctx.h)
            torch.cuda.synchronize()
            a, b = w_ref.cpu().numpy(), w_new.cpu().numpy()
            assert np.all(np.isfinite(b)), call
            assert np.max(np.abs(a - b)) < 1e-8 * max(1.0, np.max(np.abs(a))), call
        # the defining property: a call after the first one (which looks up the array's device
        # address) takes no device memory; cudaMemGetInfo would see any allocation (>= 2 MB pages)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        st = lib.xlbomd_response_noalloc(ctx.h, 0, ctypes.c_void_p(vd.data_ptr()),
                                         ctypes.c_void_p(w_new.data_ptr()))
        assert st == 0, lib.xlbomd_last_error(ctx.h)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)


def test_noalloc_response_rejects_systems_beyond_the_static_limit(X):
    import torch
    s = synth.make_system(65, 3)          # 260 orbitals -> padded 384 > 256
    p = X.default_params(mix_alpha=ALPHA_MIX, kernel_c=1.0 - 1.0 / ALPHA_MIX)
    sysd = dict(natoms=s.natoms, L=s.L, R=s.R, V=s.V, Z=s.Z, mass=s.mass)
    with X.Context(p, [sysd]) as ctx:
        ctx.build_H(0)
        ctx.density(0)
        vd = torch.zeros(s.natoms, dtype=torch.float64, device="cuda")
        wd = torch.zeros_like(vd)
        st = ctx._lib.xlbomd_response_noalloc(ctx.h, 0, ctypes.c_void_p(vd.data_ptr()),
                                              ctypes.c_void_p(wd.data_ptr()))
        assert st == -1
        assert b"static work-array limit" in ctx._lib.xlbomd_last_error(ctx.h)

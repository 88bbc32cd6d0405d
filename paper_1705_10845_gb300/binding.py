"""Thin ctypes binding of the C ABI in include/xlbomd.h (argument marshalling only).

Every computation runs in libxlbomd.so.  Loading fails loudly when the
library has not been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

XLBOMD_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NOT_CONVERGED",
          -5: "ERR_SPECTRUM", -6: "ERR_DIVERGED", -7: "ERR_TIMEOUT", -8: "ERR_UNSUPPORTED"}
PREC = {"fp64": 0, "fp16x3": 1, "bf16x3": 2, "tf32x3": 3}

Q, N, NHIST, F, R, V, KR, RES, ENERGY, MU, D, H, GAMMA, STATS, PROBES, KMAT = range(16)


class XlbomdError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("eps_s", C.c_double), ("eps_p", C.c_double), ("t0", C.c_double * 4),
        ("r_decay", C.c_double), ("r_cut", C.c_double), ("r_taper", C.c_double),
        ("hubbard_U", C.c_double), ("coulomb_k", C.c_double),
        ("Te", C.c_double), ("n_sq", C.c_int),
        ("dt", C.c_double), ("kappa", C.c_double), ("alpha", C.c_double), ("c", C.c_double * 8),
        ("kmax", C.c_int), ("rank_m", C.c_int), ("kernel_c", C.c_double), ("mix_alpha", C.c_double),
        ("scf_tol", C.c_double), ("scf_max_iter", C.c_int), ("mu_tol", C.c_double),
        ("mu_max_iter", C.c_int), ("diverge_tol", C.c_double), ("prec", C.c_int),
        ("energy_every", C.c_int), ("scf_mode", C.c_int),
        ("kernel_auto", C.c_int), ("kernel_mode", C.c_int), ("kernel_every", C.c_int),
        ("rep_A", C.c_double), ("rep_rho", C.c_double), ("kernel_prec", C.c_int), ("graphs", C.c_int),
        ("mu_prec", C.c_int),
    ]


class System(C.Structure):
    _fields_ = [("natoms", C.c_int), ("box_L", C.c_double), ("R", C.POINTER(C.c_double)),
                ("V", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)), ("mass", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libxlbomd.so (raises OSError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise OSError(f"{p} not built: run paper_1705_10845_gb300.build.build()")
    lib = C.CDLL(p)
    P, I, VP, DP = C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)
    lib.xlbomd_default_params.argtypes = [C.POINTER(Params)]
    lib.xlbomd_default_params.restype = None
    lib.xlbomd_init.argtypes = [C.POINTER(Params), C.POINTER(System), I, VP, C.POINTER(P)]
    for name in ("xlbomd_scf", "xlbomd_build_H", "xlbomd_density", "xlbomd_kernel_update", "xlbomd_energy",
                 "xlbomd_kernel_exact"):
        getattr(lib, name).argtypes = [P, I]
    lib.xlbomd_table_i.argtypes = [C.POINTER(Params), I]
    lib.xlbomd_step.argtypes = [P, I]
    lib.xlbomd_response.argtypes = [P, I, VP, VP]
    lib.xlbomd_get.argtypes = [P, I, I, DP]
    lib.xlbomd_set.argtypes = [P, I, I, DP]
    lib.xlbomd_sizes.argtypes = [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I)]
    lib.xlbomd_clear_error.argtypes = [P]
    lib.xlbomd_last_error.argtypes = [P]
    lib.xlbomd_last_error.restype = C.c_char_p
    lib.xlbomd_free.argtypes = [P]
    lib.xlbomd_launch_count.argtypes = []
    lib.xlbomd_launch_count.restype = C.c_longlong
    lib.xlbomd_gemm_profile.argtypes = [P, I, DP]
    lib.xlbomd_gemm_profile.restype = C.c_int
    lib.xlbomd_selftest_gemm.argtypes = [I, I, I, DP]
    lib.xlbomd_selftest_gemm.restype = C.c_int
    lib.xlbomd_selftest_gemm_group.argtypes = [I, I, I, I, DP]
    lib.xlbomd_selftest_gemm_group.restype = C.c_int
    for name in ("xlbomd_init", "xlbomd_scf", "xlbomd_build_H", "xlbomd_density", "xlbomd_kernel_update",
                 "xlbomd_energy", "xlbomd_step", "xlbomd_response", "xlbomd_get", "xlbomd_set",
                 "xlbomd_sizes", "xlbomd_clear_error", "xlbomd_free", "xlbomd_kernel_exact", "xlbomd_table_i"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def default_params(**overrides) -> Params:
    """xlbomd_default_params, then kmax (its Table I row, xlbomd_table_i), then the other overrides."""
    p = Params()
    lib = load()
    lib.xlbomd_default_params(C.byref(p))
    if "kmax" in overrides:
        st = lib.xlbomd_table_i(C.byref(p), int(overrides["kmax"]))
        if st != XLBOMD_OK:
            raise XlbomdError(st, "xlbomd_table_i")
    for k, v in overrides.items():
        if k == "kmax":
            continue
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        if k in ("t0", "c"):
            arr = getattr(p, k)
            for i in range(len(arr)):
                arr[i] = 0.0
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def launch_count() -> int:
    """Kernels launched by libxlbomd.so since it was loaded."""
    return int(load().xlbomd_launch_count())


def selftest_gemm(n: int, prec: str = "fp16x3", sym=False, single: bool = False):
    """One tensor-core split product of seeded matrices checked on the device
    against the FP64 product: returns (max abs error, timeout flag, ms).
    sym: False (A B^T), True (symmetric output), or 2 (A B^T + B A^T);
    single: one 16-bit product (hi operands only) instead of three.
    prec "fp64" times one plain-FP64 product instead (error 0)."""
    out = np.zeros(4)
    mode = 2 if (not isinstance(sym, bool) and sym == 2) else int(bool(sym))
    if single:
        mode += 4
    st = load().xlbomd_selftest_gemm(int(n), PREC[prec], mode, _dptr(out))
    if st != XLBOMD_OK:
        raise XlbomdError(st, "xlbomd_selftest_gemm")
    return float(out[0]), int(out[2]), float(out[3])


def selftest_gemm_group(n: int, prec: str = "fp16x3", sym=False, single: bool = False, nprob: int = 3):
    """Grouped product launch of nprob seeded problems against their single launches:
    returns (max |C_group - C_single|, timeout flag)."""
    out = np.zeros(2)
    mode = 2 if (not isinstance(sym, bool) and sym == 2) else int(bool(sym))
    if single:
        mode += 4
    st = load().xlbomd_selftest_gemm_group(int(n), PREC[prec], mode, int(nprob), _dptr(out))
    if st != XLBOMD_OK:
        raise XlbomdError(st, "xlbomd_selftest_gemm_group")
    return float(out[0]), int(out[1])


class Context:
    """Owner of one xlbomd_ctx.  Methods carry the C names without the prefix."""

    def __init__(self, params: Params, systems, stream=None):
        lib = load()
        self._lib = lib
        self._keep = []
        arr = (System * len(systems))()
        for i, s in enumerate(systems):
            R = np.ascontiguousarray(s["R"], dtype=np.float64).reshape(-1)
            Vv = np.ascontiguousarray(s["V"], dtype=np.float64).reshape(-1)
            Z = np.ascontiguousarray(s["Z"], dtype=np.float64).reshape(-1)
            self._keep += [R, Vv, Z]
            arr[i] = System(int(s["natoms"]), float(s["L"]), _dptr(R), _dptr(Vv), _dptr(Z), float(s["mass"]))
        self.params = params
        self.nsys = len(systems)
        self.natoms = [int(s["natoms"]) for s in systems]
        h = C.c_void_p()
        st = lib.xlbomd_init(C.byref(params), arr, len(systems), C.c_void_p(stream or 0), C.byref(h))
        if st != XLBOMD_OK:
            raise XlbomdError(st, "xlbomd_init")
        self.h = h

    def _check(self, st, what):
        if st != XLBOMD_OK:
            msg = self._lib.xlbomd_last_error(self.h)
            raise XlbomdError(st, f"{what}: {msg.decode() if msg else ''}")

    def scf(self, sys=-1):
        self._check(self._lib.xlbomd_scf(self.h, sys), "xlbomd_scf")

    def build_H(self, sys=0):
        self._check(self._lib.xlbomd_build_H(self.h, sys), "xlbomd_build_H")

    def density(self, sys=0):
        self._check(self._lib.xlbomd_density(self.h, sys), "xlbomd_density")

    def response(self, sys, v_ptr: int, w_ptr: int):
        """v_ptr, w_ptr: device addresses of natoms doubles (e.g. torch data_ptr())."""
        self._check(self._lib.xlbomd_response(self.h, sys, C.c_void_p(v_ptr), C.c_void_p(w_ptr)),
                    "xlbomd_response")

    def kernel_update(self, sys=0):
        self._check(self._lib.xlbomd_kernel_update(self.h, sys), "xlbomd_kernel_update")

    def kernel_exact(self, sys=0):
        self._check(self._lib.xlbomd_kernel_exact(self.h, sys), "xlbomd_kernel_exact")

    def energy(self, sys=0):
        self._check(self._lib.xlbomd_energy(self.h, sys), "xlbomd_energy")

    def step(self, nsteps=1):
        self._check(self._lib.xlbomd_step(self.h, nsteps), "xlbomd_step")

    def sizes(self, sys=0):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(self._lib.xlbomd_sizes(self.h, sys, C.byref(a), C.byref(b), C.byref(c)), "xlbomd_sizes")
        return a.value, b.value, c.value

    def _count(self, sys, what):
        nat = self.natoms[sys]
        k1 = self.params.kmax + 1
        m = self.params.rank_m
        return {Q: nat, N: nat, NHIST: k1 * nat, F: 3 * nat, R: 3 * nat, V: 3 * nat, KR: nat, RES: nat,
                ENERGY: 7, MU: 1, D: (4 * nat) ** 2, H: (4 * nat) ** 2, GAMMA: nat * nat, STATS: 5,
                PROBES: 2 * m * nat, KMAT: nat * nat}[what]

    def get(self, sys, what) -> np.ndarray:
        out = np.zeros(self._count(sys, what))
        self._check(self._lib.xlbomd_get(self.h, sys, what, _dptr(out)), "xlbomd_get")
        nat = self.natoms[sys]
        if what in (F, R, V):
            return out.reshape(nat, 3)
        if what in (D, H):
            return out.reshape(4 * nat, 4 * nat)
        if what in (GAMMA, KMAT):
            return out.reshape(nat, nat)
        if what == NHIST:
            return out.reshape(-1, nat)
        if what == PROBES:
            return out.reshape(2, self.params.rank_m, nat)
        return out

    def set(self, sys, what, values):
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        self._check(self._lib.xlbomd_set(self.h, sys, what, _dptr(a)), "xlbomd_set")

    def gemm_profile(self, mode: int):
        """mode 1 start, 0 stop, 2 collect -> (launches, total ms, algorithmic flops)."""
        out = np.zeros(3)
        self._check(self._lib.xlbomd_gemm_profile(self.h, mode, _dptr(out)), "xlbomd_gemm_profile")
        return tuple(out) if mode == 2 else None

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.xlbomd_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

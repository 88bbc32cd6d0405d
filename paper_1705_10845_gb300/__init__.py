"""GB300-native XL-BOMD hot path (arXiv:1705.10845) behind the C ABI of include/xlbomd.h.

The Python side only marshals arguments to libxlbomd.so; see binding.Context.
"""
from . import build  # noqa: F401
from .binding import (  # noqa: F401
    Context, Params, XlbomdError, default_params, load, library_path,
    Q, N, NHIST, F, R, V, KR, RES, ENERGY, MU, D, H, GAMMA, STATS, PROBES, KMAT,
)

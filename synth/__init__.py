"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the XL-BOMD method: it only draws the
random atom positions and Maxwell velocities that both sides take as input.
"""
from .systems import (  # noqa: F401
    SplitMix64,
    random_positions,
    maxwell_velocities,
    make_system,
    box_length_for,
    DENSITY,
    KB_EV,
    ACC_EV_AMU_A,
)

"""Seeded synthetic carbon-like systems (positions, velocities).

The paper's systems (solvated hydroquinone, water, nitromethane; Section VI)
and its SCC-DFTB parameters are not available, so every workload is a box of
uniform-random carbon-like atoms at the density of the tiny system
(24 atoms in a 7 A cube, 0.069971 A^-3).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  Uniform doubles take the top 53 bits.
Normals come from the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
ACC_EV_AMU_A = 9.648533e-3      # 1 eV/(amu*A) in A/fs^2
DENSITY = 24.0 / 343.0          # atoms per A^3 (24 atoms in a 7 A cube)

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator, written from its published definition."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair; the other is dropped)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def box_length_for(natoms: int, density: float = DENSITY) -> float:
    """Side of the periodic cube that holds `natoms` at `density`."""
    return (natoms / density) ** (1.0 / 3.0)


def random_positions(natoms: int, L: float, rng: SplitMix64, min_sep: float = 1.8,
                     max_attempts: int | None = None) -> np.ndarray:
    """Random sequential addition in a periodic cube of side L.

    A candidate is kept when its minimum-image distance to every placed atom
    is at least `min_sep`.  Raises ValueError when the attempt budget runs out.
    """
    if max_attempts is None:
        max_attempts = 2000 * natoms + 10000
    R = np.zeros((natoms, 3))
    placed = 0
    attempts = 0
    ms2 = min_sep * min_sep
    while placed < natoms:
        if attempts >= max_attempts:
            raise ValueError(f"could not place {natoms} atoms with separation {min_sep} A in L={L}")
        attempts += 1
        c = np.array([rng.uniform() * L, rng.uniform() * L, rng.uniform() * L])
        if placed:
            d = R[:placed] - c
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < ms2:
                continue
        R[placed] = c
        placed += 1
    return R


def maxwell_velocities(natoms: int, mass: float, T: float, rng: SplitMix64) -> np.ndarray:
    """Maxwell velocities in A/fs at temperature T (K).

    The centre-of-mass drift is removed and the kinetic energy is rescaled to
    exactly (3*natoms - 3)/2 kB T.
    """
    sigma = math.sqrt(KB_EV * T / mass * ACC_EV_AMU_A)
    V = np.array([[rng.normal() for _ in range(3)] for _ in range(natoms)]) * sigma
    V -= V.mean(axis=0)
    if natoms > 1 and T > 0:
        ke = 0.5 * mass * np.sum(V * V) / ACC_EV_AMU_A      # eV
        target = 0.5 * (3 * natoms - 3) * KB_EV * T
        V *= math.sqrt(target / ke)
    return V


@dataclass
class System:
    natoms: int
    L: float
    R: np.ndarray          # (natoms, 3) A
    V: np.ndarray          # (natoms, 3) A/fs
    Z: np.ndarray          # (natoms,) valence electrons
    mass: float
    seed: int

    @property
    def n_orb(self) -> int:
        return 4 * self.natoms

    @property
    def n_electrons(self) -> int:
        return int(round(float(np.sum(self.Z))))


def make_system(natoms: int, seed: int, L: float | None = None, T_init: float = 300.0,
                mass: float = 12.0, min_sep: float = 1.8) -> System:
    """One seeded carbon-like system: positions first, then velocities."""
    if L is None:
        L = box_length_for(natoms)
    rng = SplitMix64(seed)
    R = random_positions(natoms, L, rng, min_sep=min_sep)
    V = maxwell_velocities(natoms, mass, T_init, rng)
    Z = np.full(natoms, 4.0)
    return System(natoms=natoms, L=L, R=R, V=V, Z=Z, mass=mass, seed=seed)

"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the coupled FFT-EVP / phase-field method. It only draws
the random inputs the method takes from outside: Voronoi seed points (on an integer sub-grid),
one crystal orientation per grain, and the material / loading presets of the workloads.
The paper builds its volume element with DREAM3D (Sec. 3, Results); these seeded Voronoi
polycrystals with orientations uniform on SO(3) stand in for it.

Orientation sampling uses Shoemake's subgroup algorithm (K. Shoemake, "Uniform random
rotations", Graphics Gems III, 1992): three uniforms u1,u2,u3 map to the unit quaternion
(sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2, sqrt(u1) sin 2pi u3, sqrt(u1) cos 2pi u3).
"""
from __future__ import annotations

import dataclasses
import numpy as np

SUBGRID_BITS = 16          # Voronoi seeds live on a 2^16-per-voxel integer sub-grid
BASE_SEED = 1509049530     # workload seed = BASE_SEED + workload index


@dataclasses.dataclass
class Material:
    """Copper constants of the workloads (stress unit: MPa, lengths: m)."""
    C11: float = 168400.0
    C12: float = 121400.0
    C44: float = 75400.0
    gdot0: float = 1.0e-3          # reference shear rate, 1/s
    n: float = 10.0                # rate-sensitivity exponent of the power law
    tau0: float = 5.0              # lattice friction, MPa
    alpha: float = 0.5             # Taylor constant (paper's c1, Table 1)
    b: float = 2.556e-10           # Burgers vector, m
    k1: float = 8.0e7              # storage constant, 1/m (paper's c4, Table 1)
    k2: float = 10.0               # dynamic-recovery constant (paper's c5, Table 1)
    rho0: float = 1.0e12           # initial density per slip system, 1/m^2
    zeta: float = 0.25             # stored-energy constant (Table 2)
    kc: float = 3.0e14             # Weibull scale of the nucleation strength, 1/m^2 (Table 2)
    q: float = 4.4                 # Weibull exponent (Table 2)
    s_nucl: float = 0.05           # k_c' = s_nucl k_c after a nucleation event (Table 2)
    s_soften: float = 0.9          # density kept by recrystallised material (Table 2)
    omega_gb: float = 0.625        # grain-boundary energy, J/m^2 (Table 2)
    dx: float = 21.4e-6            # grid spacing l0, m (Table 1)
    l_gb: float = float(np.sqrt(9.6))  # interface width in grid spacings
    L_dt: float = 0.05             # Allen-Cahn mobility x PF time step (grid units)
    eta_drop: float = 1.0e-5       # active-set drop threshold
    # Ma-Roters dislocation law (Table 1); the grid size l0 is dx
    T: float = 723.0               # temperature of the DRX case, K
    Q_slip: float = 3.3e-19        # activation energy for slip, J
    Q_bulk: float = 3.51e-19       # activation energy for climb, J
    nu_D: float = 1.0e13           # attempt frequency, order of the Debye frequency, 1/s (not printed)
    poisson: float = 0.34          # Poisson's ratio of copper in d_dipole (not printed)
    c1: float = 0.5
    c2: float = 3.0
    c3: float = 3.0
    c4: float = 8.0e7              # 1/m
    c5: float = 10.0
    c6: float = 3.0e10             # 1/m, dipole term (the equation's placement)
    c7: float = 7.0e-28            # m^5 s^(c8-1), climb term
    c8: float = 0.24
    xi: float = 200.0

    @property
    def mu(self) -> float:
        """Voigt isotropic shear modulus of the cubic crystal, MPa."""
        return (self.C11 - self.C12 + 3.0 * self.C44) / 5.0

    @property
    def lam(self) -> float:
        """Voigt isotropic Lame constant, MPa."""
        return (self.C11 + 4.0 * self.C12 - 2.0 * self.C44) / 5.0


@dataclasses.dataclass
class Workload:
    name: str
    n: int                 # grid points per edge (N^3 voxels)
    grains: int
    increments: int
    dE33: float            # prescribed strain increment along x3 (negative = compression)
    dt: float              # seconds per increment
    pf_steps: int
    precision: str         # "fp64" or "mixed"
    seed: int


WORKLOADS = {
    "cu16": Workload("cu16_fp64_16^3_8grains", 16, 8, 20, -1.0e-3, 1.0, 5, "fp64", BASE_SEED + 0),
    "cu64": Workload("cu64_fp64_64^3_64grains", 64, 64, 300, -1.0e-3, 1.0, 5, "fp64", BASE_SEED + 1),
    "cu128": Workload("cu128_mixed_128^3_256grains", 128, 256, 500, -1.0e-3, 1.0, 5, "mixed", BASE_SEED + 2),
    "cu32adj": Workload("cu32_adjoint_32^3_27grains", 32, 27, 50, -1.0e-3, 1.0, 5, "fp64", BASE_SEED + 3),
    "cu256": Workload("cu256_mixed_256^3_1024grains", 256, 1024, 1000, -6.0e-4, 0.6, 5, "mixed", BASE_SEED + 4),
}


def ma_roters_material(T: float = 723.0) -> Material:
    """Copper with the Ma-Roters law: initial SSD density per system 2.8e11 /m^2 at 723 K and
    2.5e12 /m^2 at 473 K (Sec. 3)."""
    return Material(T=T, rho0=2.8e11 if T >= 600.0 else 2.5e12)


def voronoi_seeds(n: int, grains: int, seed: int) -> np.ndarray:
    """G x 3 int64 seed points on the periodic sub-grid [0, n * 2^16)^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n << SUBGRID_BITS, size=(grains, 3), dtype=np.int64)


def orientations(grains: int, seed: int) -> np.ndarray:
    """G x 4 unit quaternions (w, x, y, z), uniform on SO(3) (Shoemake 1992)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED0F0E))
    u = rng.random((grains, 3))
    a = np.sqrt(1.0 - u[:, 0])
    c = np.sqrt(u[:, 0])
    t2 = 2.0 * np.pi * u[:, 1]
    t3 = 2.0 * np.pi * u[:, 2]
    q = np.stack([c * np.cos(t3), a * np.sin(t2), a * np.cos(t2), c * np.sin(t3)], axis=1)
    return q


def axis_quaternion(axis: str) -> np.ndarray:
    """Orientation whose crystal axes coincide with the sample axes (identity), or a simple turn."""
    if axis == "001":
        return np.array([[1.0, 0.0, 0.0, 0.0]])
    if axis == "z45":   # 45 degrees about x3
        h = np.pi / 8.0
        return np.array([[np.cos(h), 0.0, 0.0, np.sin(h)]])
    raise ValueError(axis)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)

"""Synthetic water workloads: geometries, even-tempered basis rules, arrivals.

The method of the paper (density-fitted mean field, Sec. 2.2) is benchmarked on
water clusters (Sec. 3.2).  The paper's cc-pVXZ data and cluster geometries are
not used; these seeded stand-ins have the same shape (25 orbital and 75
auxiliary Cartesian functions per water for clusters).

Readings fixed here (the paper is silent on all of them):
  * monomer: O-H 0.9572 angstrom, H-O-H 104.52 degrees, O at the origin, the
    molecule in the xz-plane, bisector along +z;
  * cluster: lattice side s = ceil(n^(1/3)), sites with x fastest, the first n
    sites, spacing 3.0 angstrom; per monomer, in order, three U(-0.3, 0.3)
    angstrom jitters of the O site, then three uniforms for a Shoemake (1992)
    uniform random quaternion applied about O; numpy default_rng(seed);
  * cluster basis: shell type l with n shells gets exponents a0(l) * beta**k,
    k = 0..n-1, with the single-water a0 and beta of that atom; an l missing
    from the single-water basis takes a0 of the highest l present on that atom.
All exponents are uncontracted shells with coefficient 1 on a normalised
primitive.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903  # CODATA 2018 Bohr radius in angstrom

OH_ANGSTROM = 0.9572
HOH_DEGREES = 104.52
LATTICE_ANGSTROM = 3.0
JITTER_ANGSTROM = 0.3


@dataclass
class Shell:
    """One contracted Cartesian shell: atom index, angular momentum, primitives."""

    atom: int
    l: int
    exps: List[float]
    coefs: List[float]


@dataclass
class Molecule:
    """Nuclear charges, coordinates in bohr and the two basis sets."""

    Z: np.ndarray            # (natom,) int32
    xyz: np.ndarray          # (natom, 3) float64, bohr
    orb: List[Shell] = field(default_factory=list)
    aux: List[Shell] = field(default_factory=list)
    name: str = ""

    @property
    def nelec(self) -> int:
        return int(self.Z.sum())

    @property
    def nocc(self) -> int:
        return self.nelec // 2


def _monomer_angstrom() -> np.ndarray:
    half = math.radians(HOH_DEGREES) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_ANGSTROM * math.sin(half), 0.0, OH_ANGSTROM * math.cos(half)],
        [-OH_ANGSTROM * math.sin(half), 0.0, OH_ANGSTROM * math.cos(half)],
    ])


def _quaternion_matrix(u1: float, u2: float, u3: float) -> np.ndarray:
    """Rotation matrix of Shoemake's uniform random unit quaternion."""
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    w = a * math.sin(2 * math.pi * u2)
    x = a * math.cos(2 * math.pi * u2)
    y = b * math.sin(2 * math.pi * u3)
    z = b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


# (atom symbol) -> list of (l, a0, beta, nshell)
def single_water_basis_rules():
    """Orbital and auxiliary rules of the single-water workload."""
    orb = {
        "O": [(0, 0.15, 3.0, 6), (1, 0.2, 3.0, 4)],
        "H": [(0, 0.1, 3.0, 4)],
    }
    aux = {
        "O": [(0, 0.3, 2.5, 6), (1, 0.3, 2.5, 6), (2, 0.3, 2.5, 6)],
        "H": [(0, 0.2, 2.5, 4), (1, 0.2, 2.5, 4)],
    }
    return orb, aux


def cluster_basis_rules():
    """Cluster rules: orbital O 3s2p1d, H 2s1p; aux O 5s4p3d1f, H 3s2p1d."""
    orb = {
        "O": [(0, 0.15, 3.0, 3), (1, 0.2, 3.0, 2), (2, 0.2, 3.0, 1)],
        "H": [(0, 0.1, 3.0, 2), (1, 0.1, 3.0, 1)],
    }
    aux = {
        "O": [(0, 0.3, 2.5, 5), (1, 0.3, 2.5, 4), (2, 0.3, 2.5, 3), (3, 0.3, 2.5, 1)],
        "H": [(0, 0.2, 2.5, 3), (1, 0.2, 2.5, 2), (2, 0.2, 2.5, 1)],
    }
    return orb, aux


_SYMBOL = {8: "O", 1: "H"}


def expand_basis(Z: Sequence[int], rules) -> List[Shell]:
    """Shells atom by atom; within an atom by l, then by increasing exponent."""
    shells: List[Shell] = []
    for ia, z in enumerate(Z):
        for (l, a0, beta, n) in rules[_SYMBOL[int(z)]]:
            for k in range(n):
                shells.append(Shell(ia, l, [a0 * beta ** k], [1.0]))
    return shells


def single_water() -> Molecule:
    xyz = _monomer_angstrom() * ANGSTROM_TO_BOHR
    Z = np.array([8, 1, 1], dtype=np.int32)
    orb_r, aux_r = single_water_basis_rules()
    return Molecule(Z, xyz, expand_basis(Z, orb_r), expand_basis(Z, aux_r), "H2O")


def water_cluster(n: int, seed: int | None = None) -> Molecule:
    """(H2O)_n on a jittered cubic lattice with random orientations."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(n if seed is None else seed)
    side = int(math.ceil(round(n ** (1.0 / 3.0), 12)))
    while side ** 3 < n:
        side += 1
    mono = _monomer_angstrom()
    coords = []
    for i in range(n):
        ix, iy, iz = i % side, (i // side) % side, i // (side * side)
        site = np.array([ix, iy, iz], dtype=np.float64) * LATTICE_ANGSTROM
        jitter = rng.uniform(-JITTER_ANGSTROM, JITTER_ANGSTROM, size=3)
        u = rng.uniform(0.0, 1.0, size=3)
        R = _quaternion_matrix(*u)
        o = site + jitter
        coords.append(o + mono @ R.T)
    xyz = np.concatenate(coords, axis=0) * ANGSTROM_TO_BOHR
    Z = np.tile(np.array([8, 1, 1], dtype=np.int32), n)
    orb_r, aux_r = cluster_basis_rules()
    return Molecule(Z, xyz, expand_basis(Z, orb_r), expand_basis(Z, aux_r), f"(H2O)_{n}")


def molecule_for(name: str) -> Molecule:
    """'h2o' for the single water, 'w<n>' for (H2O)_n with seed n."""
    if name == "h2o":
        return single_water()
    if name.startswith("w"):
        return water_cluster(int(name[1:]))
    raise ValueError(f"unknown workload {name!r}")


def serving_stream(nreq: int = 2000, rate_hz: float = 20.0, nmin: int = 2, nmax: int = 48,
                   seed: int = 2025) -> List[Tuple[float, int, int]]:
    """Poisson arrivals: (arrival time s, cluster size n, request id).

    Exponential gaps with mean 1/rate and n ~ U{nmin..nmax}, one stream drawn
    from default_rng(seed); the geometry of request id r uses seed r.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=nreq)
    sizes = rng.integers(nmin, nmax + 1, size=nreq)
    t = np.cumsum(gaps)
    return [(float(t[i]), int(sizes[i]), i) for i in range(nreq)]

"""Seeded synthetic inputs shared by the FP64 oracle and the GPU library.

This module holds no part of the deep-potential arithmetic.  It only draws
random numbers and places atoms:

* ``normal_blob`` -- i.i.d. N(0, sigma^2) weights from a counter-based
  splitmix64 stream turned into normals by Box-Muller (cos branch only);
* ``water_box`` -- water molecules at random positions in a periodic box;
* ``protein_in_water`` -- a compact random-walk "protein" blob of H/C/N/O/S
  atoms in the middle of a periodic box, water everywhere else;
* ``serving_requests`` -- a list of independent systems with log-uniform atom
  counts and Poisson arrival times;
* ``maxwell_boltzmann`` -- initial velocities.

The paper's benchmarks (solvated PDB proteins 1YRF/1UBQ/3LZM/2PTC, paper
Sec. IV) and its trained DPA-2/DPA-3 weights are not available; these systems
stand in for their shape: protein atoms in water at water density, cutoff 6 A.

Units: Angstrom, femtosecond, atomic mass unit, electron-volt.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# species tables: protein systems use [H, C, N, O, S]; pure water uses [O, H]
PROTEIN_SPECIES = ("H", "C", "N", "O", "S")
WATER_SPECIES = ("O", "H")
MASSES = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "S": 32.06}

OH_BOND = 0.96                 # A
HOH_ANGLE = math.radians(104.52)


# --------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------
def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the splitmix64 stream of ``seed``.

    splitmix64 (Steele, Lea, Flood 2014): state_k = seed + (k+1)*0x9E3779B97F4A7C15,
    z = (s ^ s>>30)*0xBF58476D1CE4E5B9; z = (z ^ z>>27)*0x94D049BB133111EB;
    out = z ^ z>>31 (all mod 2^64).  Being counter-based it vectorises.
    """
    k = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = (np.uint64(seed) + (k + np.uint64(1)) * _GOLDEN) & _MASK64
        z = ((s ^ (s >> np.uint64(30))) * _M1) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * _M2) & _MASK64
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of splitmix64 times 2^-53."""
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_blob(n: int, seed: int, sigma: float = 0.1) -> np.ndarray:
    """``n`` i.i.d. N(0, sigma^2) doubles: normal k uses uniforms 2k and 2k+1.

    Box-Muller: z = sqrt(-2 ln(1-u1)) cos(2 pi u2); 1-u1 lies in (0, 1], so the
    logarithm is finite.
    """
    u = uniform01(seed, 0, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return sigma * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly distributed rotation matrices (random unit quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _water_molecules(rng: np.random.Generator, oxygens: np.ndarray) -> np.ndarray:
    """Place H-O-H (0.96 A, 104.52 deg, random orientation) at each oxygen.

    Returns (n_mol, 3, 3): atoms O, H, H of each molecule.
    """
    n = len(oxygens)
    half = 0.5 * HOH_ANGLE
    local = np.array([[0.0, 0.0, 0.0],
                      [OH_BOND * math.sin(half), OH_BOND * math.cos(half), 0.0],
                      [-OH_BOND * math.sin(half), OH_BOND * math.cos(half), 0.0]])
    rot = _random_rotations(rng, n)
    return oxygens[:, None, :] + np.einsum("nab,kb->nka", rot, local)


def _min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.round(d / box)


@dataclass
class System:
    """One periodic, orthorhombic system: positions may lie outside the box."""
    coords: np.ndarray            # (N, 3) float64, A
    types: np.ndarray             # (N,) int32 species index
    box: np.ndarray               # (3,) float64, A
    species: tuple = PROTEIN_SPECIES
    note: str = ""
    blob_atoms: int = 0

    @property
    def n(self) -> int:
        return len(self.types)

    @property
    def masses(self) -> np.ndarray:
        """Per-species masses in amu, in the order of ``species``."""
        return np.array([MASSES[s] for s in self.species])


# --------------------------------------------------------------------------
# systems
# --------------------------------------------------------------------------
def water_box(n_mol: int, box_len: float, seed: int, min_oo: float = 2.5) -> System:
    """``n_mol`` water molecules at random positions in a cubic periodic box.

    Oxygens are drawn uniformly and rejected when closer than ``min_oo`` (2.5 A,
    minimum image) to an accepted one.  Species map is [O, H].
    """
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    ox = np.empty((0, 3))
    tries = 0
    while len(ox) < n_mol:
        tries += 1
        if tries > 200000:
            raise RuntimeError("water_box: could not place oxygens")
        p = rng.uniform(0.0, box_len, size=3)
        if len(ox):
            d = _min_image(ox - p, box)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_oo * min_oo:
                continue
        ox = np.vstack([ox, p])
    mols = _water_molecules(rng, ox)
    coords = mols.reshape(-1, 3)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    return System(coords, types, box, WATER_SPECIES, note=f"water_box({n_mol}, {box_len}, {seed})")


def _blob_walk(rng: np.random.Generator, n: int, centre: np.ndarray, radius: float,
               step: float = 1.5, min_dist: float = 1.2, tries: int = 64) -> np.ndarray:
    """Self-avoiding random walk with ``step`` A steps confined to a sphere.

    A step is accepted when it stays inside the sphere and keeps ``min_dist``
    from every earlier atom except the previous one.  When ``tries`` directions
    all fail the chain restarts at a random admissible point (a chain break).
    A grid hash keeps the distance test local.
    """
    cell = min_dist
    grid: dict = {}

    def key(p):
        return (int(math.floor(p[0] / cell)), int(math.floor(p[1] / cell)), int(math.floor(p[2] / cell)))

    pts = np.empty((n, 3))

    def ok(p, skip):
        if np.sum((p - centre) ** 2) > radius * radius:
            return False
        kx, ky, kz = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for idx in grid.get((kx + dx, ky + dy, kz + dz), ()):
                        if idx == skip:
                            continue
                        if np.sum((pts[idx] - p) ** 2) < min_dist * min_dist:
                            return False
        return True

    def add(i, p):
        pts[i] = p
        grid.setdefault(key(p), []).append(i)

    add(0, centre.copy())
    for i in range(1, n):
        placed = False
        dirs = rng.normal(size=(tries, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        for d in dirs:
            p = pts[i - 1] + step * d
            if ok(p, i - 1):
                add(i, p)
                placed = True
                break
        while not placed:
            v = rng.normal(size=3)
            p = centre + radius * rng.uniform() ** (1 / 3) * v / np.linalg.norm(v)
            if ok(p, -1):
                add(i, p)
                placed = True
    return pts


def protein_in_water(n_total: int, n_blob: int, box, seed: int,
                     fractions=(0.50, 0.30, 0.09, 0.10, 0.01)) -> System:
    """A compact H/C/N/O/S chain blob at the box centre, water elsewhere.

    * Blob: ``n_blob`` atoms from ``_blob_walk`` in a sphere of radius
      (3 n_blob / (4 pi 0.1))^(1/3) A (density 0.1 atoms/A^3); species counts
      are floor(fraction * n_blob) with the remainder given to H, shuffled.
    * Water: (n_total - n_blob)/3 molecules whose oxygens sit on a jittered
      (+-0.25 A) orthorhombic lattice with spacing L_a / n_a, restricted to sites
      farther than radius + 1.5 A from the centre; the lattice is the sparsest
      one (about 0.0333 sites/A^3 or denser) with enough such sites, and the
      occupied sites are a seeded random subset.
    Species map [H, C, N, O, S].
    """
    box = np.asarray(box, dtype=np.float64)
    if (n_total - n_blob) % 3:
        raise ValueError("n_total - n_blob must be a multiple of 3")
    n_water = (n_total - n_blob) // 3
    rng = np.random.default_rng(seed)
    centre = 0.5 * box
    radius = (3.0 * n_blob / (4.0 * math.pi * 0.1)) ** (1.0 / 3.0) if n_blob else 0.0

    counts = [int(math.floor(f * n_blob)) for f in fractions]
    counts[0] += n_blob - sum(counts)
    blob_types = np.repeat(np.arange(5, dtype=np.int32), counts)
    rng.shuffle(blob_types)
    blob = _blob_walk(rng, n_blob, centre, radius) if n_blob else np.empty((0, 3))

    excl = radius + 1.5 if n_blob else -1.0
    rho = 0.0333
    while True:
        nd = np.maximum(1, np.round(box * rho ** (1.0 / 3.0)).astype(int))
        a = box / nd
        g = np.stack(np.meshgrid(*(np.arange(k) for k in nd), indexing="ij"), -1).reshape(-1, 3)
        sites = (g + 0.5) * a
        far = np.sum((sites - centre) ** 2, axis=1) > excl * excl
        sites = sites[far]
        if len(sites) >= n_water:
            break
        rho *= 1.02
    pick = rng.choice(len(sites), size=n_water, replace=False)
    pick.sort()
    ox = sites[pick] + rng.uniform(-0.25, 0.25, size=(n_water, 3))
    mols = _water_molecules(rng, ox)
    wat = mols.reshape(-1, 3)
    wat_types = np.tile(np.array([3, 0, 0], dtype=np.int32), n_water)   # O, H, H
    coords = np.vstack([blob, wat])
    types = np.concatenate([blob_types, wat_types]).astype(np.int32)
    return System(coords, types, box, PROTEIN_SPECIES,
                  note=f"protein_in_water({n_total}, {n_blob}, {box.tolist()}, {seed})",
                  blob_atoms=n_blob)


def maxwell_boltzmann(masses_per_atom: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Velocities (A/fs) drawn at ``temperature`` K, centre-of-mass momentum removed.

    sigma_a = sqrt(k_B T / m_a) with k_B T in eV and m in amu, converted with
    kappa = e / (amu * 1e10) A^2 fs^-2 per (eV/amu) (CODATA e and amu).
    """
    kb = 8.617333262e-5
    kappa = 1.602176634e-19 / (1.66053906660e-27 * 1e10)
    rng = np.random.default_rng(seed)
    m = np.asarray(masses_per_atom, dtype=np.float64)
    v = rng.normal(size=(len(m), 3)) * np.sqrt(kb * temperature * kappa / m)[:, None]
    p = (m[:, None] * v).sum(0)
    v -= p / m.sum()
    return v


# --------------------------------------------------------------------------
# serving workload
# --------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival_s: float
    system: System
    n_steps: int


def serving_system(n: int, seed: int) -> System:
    """One serving system of about ``n`` atoms in a cubic box at 0.1 atoms/A^3.

    Below 600 atoms it is pure water ([O, H] mapped into the protein species
    table as O=3, H=0) with n rounded to a multiple of 3; from 600 atoms on it
    is a protein blob of about 6.25 % of the atoms (adjusted so the rest is whole
    waters) in water, with the total exact.
    """
    if n < 600:
        n = max(3, 3 * int(round(n / 3)))
        L = (n / 0.1) ** (1.0 / 3.0)
        w = water_box(n // 3, L, seed, min_oo=2.2)
        types = np.where(w.types == 0, 3, 0).astype(np.int32)
        return System(w.coords, types, w.box, PROTEIN_SPECIES, note=f"serving water {n} seed {seed}")
    ns = int(round(0.0625 * n))
    while (n - ns) % 3:
        ns += 1
    L = (n / 0.1) ** (1.0 / 3.0)
    return protein_in_water(n, ns, (L, L, L), seed)


def serving_requests(n_req: int, rate_per_s: float, seed: int, n_steps: int = 50,
                     n_min: int = 96, n_max: int = 6000) -> list:
    """``n_req`` requests: N ~ logU(n_min, n_max), Poisson arrivals at ``rate_per_s``."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_req)).astype(int)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req) if rate_per_s > 0 else np.zeros(n_req)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(k, float(t[k]), serving_system(int(sizes[k]), seed * 1000 + k), n_steps)
            for k in range(n_req)]


# --------------------------------------------------------------------------
# cached builds of the large systems (generation is deterministic)
# --------------------------------------------------------------------------
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def cached(fn, *args, **kw) -> System:
    """Memoise a generator's output on disk (keyed by its name and arguments)."""
    tag = hashlib.sha1(repr((fn.__name__, args, sorted(kw.items()))).encode()).hexdigest()[:16]
    path = os.path.join(_CACHE, f"{fn.__name__}_{tag}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return System(z["coords"], z["types"], z["box"], tuple(str(s) for s in z["species"]),
                      note=str(z["note"]), blob_atoms=int(z["blob_atoms"]))
    s = fn(*args, **kw)
    try:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, coords=s.coords, types=s.types, box=s.box, species=np.array(s.species),
                 note=np.array(s.note), blob_atoms=np.array(s.blob_atoms))
        os.replace(tmp, path)
    except OSError:
        pass
    return s
